// Internal declarations of libmsrcg: device-visible level descriptors, solve
// state, error handling and small device helpers shared by the build and the
// solve translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "msrcg.h"

#define MSRCG_CUDA_TRY(expr)                      \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return msrcg_cuda_fail(e_, #expr, __FILE__, __LINE__); \
  } while (0)

int msrcg_cuda_fail(cudaError_t e, const char* what, const char* file, int line);

namespace msrcg {

constexpr int kMaxLev = MSRCG_MAXLEV;
constexpr int kThreads = 256;        // block size of the multi-CTA level kernels
#ifndef MSRCG_SMALL_THREADS
#define MSRCG_SMALL_THREADS 512
#endif
#ifndef MSRCG_SMALL_PER_SM
#define MSRCG_SMALL_PER_SM 1
#endif
constexpr int kSmallThreads = MSRCG_SMALL_THREADS;  // block size of the single-CTA solver
constexpr int kSmallPerSM = MSRCG_SMALL_PER_SM;     // single-CTA solvers resident per SM
constexpr int kMaxGrid = 4096;       // upper bound of blocks per multi-CTA launch
constexpr int kRestrictTI = 32;      // coarse columns per tile of the tiled restriction

// status bits written on the device (host maps them to MSRCG_E*)
constexpr int kStBreakdown = 1;
constexpr int kStNoConv = 2;
constexpr int kStTimeout = 4;
constexpr int kStNanInf = 8;

// One level of the hierarchy as the kernels see it.  Face arrays: Tx has
// (nx+1)*ny*nz entries (x fastest), Ty nx*(ny+1)*nz, Tz nx*ny*(nz+1).
// Vectors are stored with a ring of ghost cells that stay zero: cell
// (i, j, k) lives at off + i + px*j + plane*k with px = nx+2, plane =
// px*(ny+2); npad is the padded length.  A zero ghost makes every boundary
// face behave like the paper's boundary treatment without a branch: the
// Gauss-Seidel sum gains T_b * 0 and the operator T_b (x_c - 0).
struct DevLevel {
  int nx, ny, nz, dim;
  long long n;
  int px, py;
  long long plane, off, npad;
  const void* T[3];      // smoother-precision transmissibilities (float or double)
  const double* T64[3];  // FP64 transmissibilities
  // prolongation tables of the transfer to level k+1, indexed by fine cell
  // along each axis: coarse corners c0, c1 and the weight w of c1
  const int* c0[3];
  const int* c1[3];
  const void* w[3];      // smoother precision
  // restriction windows, indexed by coarse cell of level k+1 along each axis:
  // the fine cells [lo, hi] that interpolate from it, and their weights
  // rw[I*W + t] (fine cell lo[I] + t), W = the longest window of the axis
  const int* lo[3];
  const int* hi[3];
  const void* rw[3];     // smoother precision
  int W[3];
  // vectors: x, r, p, q in the level's vector type; z, t in smoother precision
  void* x;
  void* r;
  void* p;
  void* q;
  void* z;
  void* t;
  void* rp;              // r in smoother precision (aliases r when the types agree)
  double fk;             // f^k of the level test
  int maxit;
  int lap;               // constant coefficients (msrcg_build_laplace): compact face arrays, see face_row
};

// Constant-coefficient levels keep compact face arrays: Tx one row of nx+1
// faces (every row of x-faces is the same), Ty the face rows south boundary,
// interior, interior, north boundary (nx each; two rows when ny = 1), Tz
// the same four planes (nx*ny each).  Face row f of an axis with n cells
// (f = 0..n) is stored in compact row face_row(f, n); the cell rows of
// make_row address cell j's south face in row cell_row(j, n) and its north
// face in the next row.
__host__ __device__ __forceinline__ int face_row(int f, int n) {
  return n == 1 ? (f == 0 ? 0 : 1) : (f == 0 ? 0 : (f == n ? 3 : 1));
}
__host__ __device__ __forceinline__ int cell_row(int j, int n) {
  return n == 1 ? 0 : (j == 0 ? 0 : (j == n - 1 ? 2 : 1));
}
// entries of level L's face array along axis a (compact or full)
__host__ __device__ __forceinline__ long long face_count(const DevLevel& L, int a) {
  if (!L.lap)
    return (long long)(L.nx + (a == 0)) * (L.ny + (a == 1)) * (L.nz + (a == 2));
  if (a == 0) return L.nx + 1;
  if (a == 1) return (long long)L.nx * (L.ny == 1 ? 2 : 4);
  return (long long)L.nx * L.ny * (L.nz == 1 ? 2 : 4);
}
// index of face (i, j, k) along axis a (i = 0..nx for a = 0, and so on)
__host__ __device__ __forceinline__ long long face_index(int lap, int a, int nx, int ny, int nz, int i, int j, int k) {
  if (!lap) {
    if (a == 0) return i + (long long)(nx + 1) * (j + (long long)ny * k);
    if (a == 1) return i + (long long)nx * (j + (long long)(ny + 1) * k);
    return i + (long long)nx * (j + (long long)ny * k);
  }
  if (a == 0) return i;
  if (a == 1) return i + (long long)nx * face_row(j, ny);
  return i + (long long)nx * (j + (long long)ny * face_row(k, nz));
}

struct LevelState {
  double rho, rho_old, pq, rr, bb, thr;
  double alpha, beta;    // CG step scalars of the current iteration
  float alpha_f, beta_f; // the same in FP32 for FP32 levels
  long long iters, calls;
  int it, stop;
  // level 0 with the stall test: the last residual that halved the best so
  // far and its iteration; r_new . z_old of the last update (flexible beta)
  double rr_best, gamma;
  int it_best, gamma_ok;
};

struct SolveState {
  double eps2;           // eps^2 of the level test (Sec. 3)
  double bb0;            // ||b||^2 of the caller's right-hand side
  double tau2;
  double inner_floor2;
  int status;
  int pad;
  double rr_true;
  // flexible beta of the level-0 PCG (Polak-Ribiere): in use (flex), may be
  // switched on by the stall test or an inner level at its cap (allow_flex,
  // FP32 preconditioner), iterations without the residual halving before
  // the switch (stall_w, 0 = no stall test)
  int flex, allow_flex, stall_w, pad2;
  LevelState lv[kMaxLev];
  unsigned int ticket[kMaxLev];
};

// Everything one problem's single-CTA solve needs.
struct ProblemDesc {
  const DevLevel* L;     // device array, nlev entries
  int nlev, m;
  const double* Ainv;    // dense inverse of the coarsest operator, nc x nc
  int nc;
  int precision;
  SolveState* S;
  const double* b;       // caller right-hand side (level 0, unpadded)
  double* x;             // caller solution (level 0, unpadded)
  double* xs;            // padded FP64 accumulator of the level-0 solution
  double tol;
  long long work;        // scheduling weight (cells of level 0)
  int fuse;              // single-pass smoothing allowed on global-memory levels
  int fuse_width;        // its strip width cap (0: none)
  int fuse_min_cells;    // its smallest level (cells)
  int splitting;         // 0: red-black symmetric Gauss-Seidel, 1: modified Jacobi, 2: natural order
  int stall_w;           // stall test of the level-0 PCG (0: none)
  int allow_flex;        // the stall test / an inner cap may switch to the flexible beta
  int flex0;             // flexible beta from the first iteration
  int precond;           // 0: recursive multi-scale (eq. 2.10), 1: multigrid (eq. 2.9), 2: polynomial
  unsigned long long* trace;  // level-tree buffer (msrcg_set_trace) or null
  int trace_cap;              // its entries
};

}  // namespace msrcg

struct msrcg_hier {
  int device = 0;
  int dim = 2, nlev = 0, ks = 0;
  int dims[MSRCG_MAXLEV][3] = {};
  long long N[MSRCG_MAXLEV] = {};
  double hsz[3] = {1.0, 1.0, 1.0};      // cell sizes of level 0
  msrcg_opts o{};
  size_t bytes = 0;
  std::vector<void*> allocs;
  double* T64[MSRCG_MAXLEV][3] = {};
  void* TR[MSRCG_MAXLEV][3] = {};       // smoother precision copy (aliases T64 in FP64 mode)
  msrcg::DevLevel hL[MSRCG_MAXLEV] = {};
  msrcg::DevLevel* dL = nullptr;
  void* trace = nullptr;                // level-tree buffer (msrcg_set_trace), caller owned
  long long trace_cap = 0;
  double* Ainv = nullptr;
  int nc = 0;
  msrcg::SolveState* dS = nullptr;
  double* partials = nullptr;           // kMaxLev * kMaxGrid doubles
  double* b0 = nullptr;                 // internal right-hand side of the level-0 PCG
  double* xs = nullptr;                 // accumulated solution across restarts
  msrcg::ProblemDesc* dP = nullptr;     // device copy of this problem's descriptor
  // level loop graph
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  size_t sub_smem = 0;                  // dynamic shared memory of the graph's single-CTA launch
  bool dirty = false;                   // last solve failed: clear the vectors before the next
  cudaStream_t alloc_stream = nullptr;  // set: allocations are stream ordered on it
  int64_t last_iters[MSRCG_MAXLEV] = {};
  int64_t last_calls[MSRCG_MAXLEV] = {};
  int sms = 0;
  msrcg_hier* twin = nullptr;           // FP64-preconditioner twin of an FP32-mode hierarchy (escalation)
  // constant coefficients (msrcg_build_laplace): K per axis and the
  // boundary type of each side, kept for the twin
  int lap = 0;
  double lapK[3] = {};
  uint8_t lap_bc[6] = {};
  // tiled restriction of a wide 2D level k into k+1: the largest fine extent
  // (columns, rows) of a tile of msrcg::kRestrictTI x rtj coarse cells, 0 = no
  // tiled kernel (3D, or the tile does not fit the shared memory)
  int rfx[MSRCG_MAXLEV] = {}, rfy[MSRCG_MAXLEV] = {};
  int rtj = 0;
};

// allocation helper: records the buffer in h->allocs
int msrcg_alloc(msrcg_hier* h, void** p, size_t bytes);
// msrcg_build with an optional stream for stream-ordered allocation
int msrcg_build_ex(const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc, const msrcg_opts* opts,
                   cudaStream_t stream, cudaStream_t alloc_stream, msrcg_hier** out);
// batched solve split in two: enqueue everything on s (states copied into
// host_states), then, once s has passed the work, turn states into stats
int msrcg_batch_enqueue(int count, msrcg_hier* const* hs, const double* const* b, double tol, double* const* x,
                        cudaStream_t s, msrcg::SolveState* host_states);
int msrcg_batch_finish(int count, msrcg_hier* const* hs, const msrcg::SolveState* host_states, msrcg_stats* stats);
// the FP64-preconditioner twin of h (same level-0 transmissibilities), built
// on first use and kept in h->twin
int msrcg_twin(msrcg_hier* h, cudaStream_t stream, msrcg_hier** out);
// device bytes msrcg_build_ex allocates for a grid and options (0: rejected)
size_t msrcg_build_bytes(const msrcg_grid* grid, const msrcg_opts* opts);
// builds h inside the device buffer [base, base + cap) without allocating
int msrcg_build_into(msrcg_hier* h, const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                     const msrcg_opts* opts, cudaStream_t st, unsigned char* base, size_t cap);
int msrcg_status_from_bits(int bits);
