// Solve path of libmsrcg: the recursive multi-scale PCG of Lackner & Menikoff
// (eq. 2.10, Sec. 2.3, Sec. 3) on the GPU.
//
// Levels 0..ks-1 ("wide" levels) run as separate multi-CTA kernels that a CUDA
// graph sequences; each level's PCG loop is a graph WHILE node whose
// condition the last kernel of an iteration sets on the device, so no host
// round trip decides anything.  Levels ks..kmax ("narrow" levels, few cells)
// run inside one CTA that executes the whole remaining recursion from shared
// memory: the level stack is an explicit state machine, with __syncthreads
// between dependent steps.  The same single-CTA solver also runs complete
// problems, one per CTA, for the batched entry point.
//
// Vectors use the padded layout of DevLevel (a zero ghost ring), so stencils
// have no boundary branches, and threads map onto (column, row) directly.
//
// Smoothers (the splitting of Sec. 3): symmetric Gauss-Seidel in red-black
// order (default; in the single-CTA solver a level that stays in global
// memory runs all half-sweeps of a smoothing as one pipelined pass,
// fused_smooth), modified Jacobi (P = 2D) and symmetric Gauss-Seidel in the
// natural order of the cells (a plane wavefront, single CTA only).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "msrcg_internal.cuh"

using namespace msrcg;

namespace {

constexpr int kMaxCoarse = 1024;  // largest coarsest level (cells) of the dense inverse

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The CTA as one team.  sum(): deterministic total in the value's own
// precision with one barrier; warp sums go to one of two buffers
// (alternating, so a buffer is rewritten only after a later barrier), then
// every thread adds them in index order.  FP32 levels never touch the FP64
// pipe, which is narrow on this GPU.
struct BlockTeam {
  double* shd;  // 64 doubles of shared memory
  float* shf;   // 64 floats of shared memory
  int par;
  __device__ __forceinline__ void sync() { __syncthreads(); }
  template <typename T>
  __device__ __forceinline__ T sum(T v) {
    v = warp_sum_t<T>(v);
    T* b = (sizeof(T) == sizeof(double) ? (T*)shd : (T*)shf) + 32 * par;
    par ^= 1;
    if ((threadIdx.x & 31) == 0) b[threadIdx.x >> 5] = v;
    __syncthreads();
    // every warp folds the warp sums with the same butterfly, so all threads
    // hold the identical total (a + b == b + a exactly at each stage)
    const int lane = threadIdx.x & 31;
    return warp_sum_t<T>(lane < (int)(blockDim.x >> 5) ? b[lane] : (T)0);
  }
};

template <typename V>
__device__ __forceinline__ const V* Tvec(const DevLevel& L, int a);
template <>
__device__ __forceinline__ const double* Tvec<double>(const DevLevel& L, int a) {
  return L.T64[a];
}
template <>
__device__ __forceinline__ const float* Tvec<float>(const DevLevel& L, int a) {
  return (const float*)L.T[a];
}

// Position and strides of a thread in the (column, row) plane of a level.
struct Map {
  int x0, dx, y0, dy;
};

// The CTA (a power-of-two number of threads) laid over rows of `width`
// columns: a power-of-two row width, at most the CTA.
__device__ __forceinline__ Map team_map(int width) {
  const int bx = width <= 1 ? 1 : min(1 << (32 - __clz(width - 1)), (int)blockDim.x);
  const int sh = __ffs(bx) - 1;
  Map m;
  m.x0 = threadIdx.x & (bx - 1);
  m.dx = bx;
  m.y0 = threadIdx.x >> sh;
  m.dy = blockDim.x >> sh;
  return m;
}

// A 2D grid of 2D blocks laid over rows.
__device__ __forceinline__ Map grid_map() {
  Map m;
  m.x0 = blockIdx.x * blockDim.x + threadIdx.x;
  m.dx = gridDim.x * blockDim.x;
  m.y0 = blockIdx.y * blockDim.y + threadIdx.y;
  m.dy = gridDim.y * blockDim.y;
  return m;
}

// Offsets of column 0 of one row (j, k) of a level: padded vector index and
// the face-array indices.  Cell (i, j, k) of the row is at pc + i; its faces
// are Tx[fx + i], Tx[fx + i + 1], Ty[fy + i], Ty[fy + i + nx], Tz[fz + i],
// Tz[fz + i + nx*ny].  All level indices fit 32 bits (the build checks).
struct Row {
  int j, k, pc, fx, fy, fz;
};

// Level geometry and transfer tables held in registers.  The single-CTA
// solver keeps its level descriptors in shared memory; reading them through
// these copies keeps the compiler from re-loading descriptor fields after
// every store to the level's vectors (it cannot rule out aliasing).
struct Geo {
  int nx, ny, nz, px, py;
  int plane, off, npad, n;
  int lap;
};
struct Xf {
  int nx, ny, nz, px, py;
  int plane, off, npad, n;
  int lap;
  const int* c0[3];
  const int* c1[3];
  const void* w[3];
  const int* lo[3];
  const int* hi[3];
  const void* rw[3];
  int W[3];
};
__device__ __forceinline__ Geo geo_of(const DevLevel& L) {
  Geo g;
  g.nx = L.nx;
  g.ny = L.ny;
  g.nz = L.nz;
  g.px = L.px;
  g.py = L.py;
  g.plane = (int)L.plane;
  g.off = (int)L.off;
  g.npad = (int)L.npad;
  g.n = (int)L.n;
  g.lap = L.lap;
  return g;
}
__device__ __forceinline__ Xf xf_of(const DevLevel& L) {
  Xf x;
  x.nx = L.nx;
  x.ny = L.ny;
  x.nz = L.nz;
  x.px = L.px;
  x.py = L.py;
  x.plane = (int)L.plane;
  x.off = (int)L.off;
  x.npad = (int)L.npad;
  x.n = (int)L.n;
  x.lap = L.lap;
  for (int a = 0; a < 3; ++a) {
    x.c0[a] = L.c0[a];
    x.c1[a] = L.c1[a];
    x.w[a] = L.w[a];
    x.lo[a] = L.lo[a];
    x.hi[a] = L.hi[a];
    x.rw[a] = L.rw[a];
    x.W[a] = L.W[a];
  }
  return x;
}

// Face offsets of row (j, k) on a constant-coefficient level (compact face
// arrays, face_row).  Kept out of line: make_row is inlined into every
// stencil loop of the solver, and this rarely taken path would otherwise be
// copied into each of them.
__device__ __noinline__ int3 lap_row_faces(int nx, int ny, int nz, int j, int k) {
  return make_int3(0, nx * cell_row(j, ny), nx * (j + ny * cell_row(k, nz)));
}

template <int DIM, class LV>
__device__ __forceinline__ Row make_row(const LV& L, int row) {
  Row r;
  r.j = row;
  r.k = 0;
  if (DIM == 3) {
    r.k = row / L.ny;
    r.j = row - r.k * L.ny;
  }
  r.pc = (int)L.off + L.px * r.j + (int)L.plane * r.k;
  if (__builtin_expect(L.lap != 0, 0)) {
    const int3 f = lap_row_faces(L.nx, L.ny, L.nz, r.j, r.k);
    r.fx = f.x;
    r.fy = f.y;
    r.fz = f.z;
  } else {
    r.fx = (L.nx + 1) * row;
    r.fy = L.nx * (row + r.k);
    r.fz = L.nx * row;
  }
  return r;
}

// Visit every cell of the level: f(i, row).  A thread walks its column
// through all of its rows before taking its next column (measured faster for
// the single-CTA solver, where a thread holds two or more columns of the
// widest levels).
template <int DIM, class LV, class F>
__device__ __forceinline__ void for_cells(const Map& m, const LV& L, F&& f) {
  const int rows = L.ny * L.nz;
  for (int i = m.x0; i < L.nx; i += m.dx)
    for (int row = m.y0; row < rows; row += m.dy) f(i, make_row<DIM>(L, row));
}

// Visit the cells of one colour ((i + j + k) & 1 == colour): in a row they
// are i = 2*ii + ((j + k + colour) & 1).  f(i, i2, row) also gets the other
// colour's cell at the same pair position (i2); either may be >= nx.
template <int DIM, class LV, class F>
__device__ __forceinline__ void for_colour(const Map& m, const LV& L, int colour, F&& f) {
  const int rows = L.ny * L.nz;
  const int hx = (L.nx + 1) >> 1;
  for (int ii = m.x0; ii < hx; ii += m.dx)
    for (int row = m.y0; row < rows; row += m.dy) {
      const Row r = make_row<DIM>(L, row);
      const int s = (r.j + r.k + colour) & 1;
      f(2 * ii + s, 2 * ii + (s ^ 1), r);
    }
}

// Linear passes over a level's padded vectors: a thread visits c =
// threadIdx.x, + blockDim.x, ...  Each group of kLinUnroll consecutive
// visits first reads its operands (ld(c)) and then applies them in visit
// order (st(c, v)).  The arithmetic and its order are those of the plain
// loop, so results are bit-identical; but a thread keeps kLinUnroll loads in
// flight instead of one (the compiler cannot move a load above an earlier
// store through pointers that may alias).  The buffers a pass reads and the
// ones it writes must be distinct.
constexpr int kLinUnroll = 4;

template <class A, class B>
struct Two {
  A a;
  B b;
};
template <class V>
struct Four {
  V x, p, r, q;
};

template <class Ld, class St>
__device__ __forceinline__ void for_lin(int n, Ld&& ld, St&& st) {
  using T = decltype(ld(0));
  const int step = blockDim.x;
  int c = threadIdx.x;
  for (; c + (kLinUnroll - 1) * step < n; c += kLinUnroll * step) {
    T v[kLinUnroll];
#pragma unroll
    for (int u = 0; u < kLinUnroll; ++u) v[u] = ld(c + u * step);
#pragma unroll
    for (int u = 0; u < kLinUnroll; ++u) st(c + u * step, v[u]);
  }
  for (; c < n; c += step) st(c, ld(c));
}

// for_cells with the same split: calc(i, row) (loads and arithmetic, no
// stores) for kLinUnroll consecutive rows of a thread's column, then
// commit(i, row, value) in visit order.
template <int DIM, class LV, class Calc, class Commit>
__device__ __forceinline__ void for_cells_u(const Map& m, const LV& L, Calc&& calc, Commit&& commit) {
  using T = decltype(calc(0, Row{}));
  const int rows = L.ny * L.nz;
  for (int i = m.x0; i < L.nx; i += m.dx) {
    int row = m.y0;
    for (; row + (kLinUnroll - 1) * m.dy < rows; row += kLinUnroll * m.dy) {
      Row rw[kLinUnroll];
      T v[kLinUnroll];
#pragma unroll
      for (int u = 0; u < kLinUnroll; ++u) {
        rw[u] = make_row<DIM>(L, row + u * m.dy);
        v[u] = calc(i, rw[u]);
      }
#pragma unroll
      for (int u = 0; u < kLinUnroll; ++u) commit(i, rw[u], v[u]);
    }
    for (; row < rows; row += m.dy) {
      const Row rw = make_row<DIM>(L, row);
      commit(i, rw, calc(i, rw));
    }
  }
}

template <typename R>
__device__ __forceinline__ R quot(R a, R b);
template <>
__device__ __forceinline__ float quot<float>(float a, float b) {
  return __fdividef(a, b);
}
template <>
__device__ __forceinline__ double quot<double>(double a, double b) {
  return a / b;
}

// Sum of the face transmissibilities of a cell (the diagonal of A).
template <int DIM, typename R, class LV>
__device__ __forceinline__ R diag_of(const LV& L, const R* Tx, const R* Ty, const R* Tz, int i, const Row& r) {
  R d = Tx[r.fx + i];
  d += Tx[r.fx + i + 1];
  d += Ty[r.fy + i];
  d += Ty[r.fy + i + L.nx];
  if (DIM == 3) {
    d += Tz[r.fz + i];
    d += Tz[r.fz + i + L.nx * L.ny];
  }
  return d;
}

// Gauss-Seidel value of one cell: row c of A solved for x_c with the
// neighbours held, x_c = (rhs_c + sum_f T_f x_nb) / sum_f T_f  (Sec. 3); a
// boundary face meets a zero ghost.  The FP32 smoother divides with the
// fast hardware quotient; FP64 divides exactly.
// The x/y part of a Gauss-Seidel value: d = sum of the four face T, s += the
// four T x_nb terms, in this order.  Shared by every smoother so that all of
// them round identically.
template <typename R>
__device__ __forceinline__ void gs_terms2(R& d, R& s, R tw, R te, R ts, R tn, R xw, R xe, R xs, R xn) {
  d = tw;
  d += te;
  d += ts;
  d += tn;
  s += tw * xw;
  s += te * xe;
  s += ts * xs;
  s += tn * xn;
}

// The x/y part of (A x)_c, in this order (shared like gs_terms2).
template <typename R>
__device__ __forceinline__ R apply_terms2(R tw, R te, R ts, R tn, R xc, R xw, R xe, R xs, R xn) {
  R s = tw * (xc - xw);
  s += te * (xc - xe);
  s += ts * (xc - xs);
  s += tn * (xc - xn);
  return s;
}

template <int DIM, typename R, typename RX, class LV>
__device__ __forceinline__ R gs_value(const LV& L, const R* Tx, const R* Ty, const R* Tz, R rhs, const RX* x,
                                      int i, const Row& r) {
  const int pc = r.pc + i;
  const R tw = Tx[r.fx + i], te = Tx[r.fx + i + 1], ts = Ty[r.fy + i], tn = Ty[r.fy + i + L.nx];
  R d, s = rhs;
  gs_terms2<R>(d, s, tw, te, ts, tn, (R)x[pc - 1], (R)x[pc + 1], (R)x[pc - L.px], (R)x[pc + L.px]);
  if (DIM == 3) {
    const int pl = (int)L.plane;
    const R tb = Tz[r.fz + i], tt = Tz[r.fz + i + L.nx * L.ny];
    d += tb;
    d += tt;
    s += tb * (R)x[pc - pl];
    s += tt * (R)x[pc + pl];
  }
  return quot<R>(s, d);
}

// The numerator of gs_value alone, rhs_c + sum_f T_f x_nb (the same terms
// in the same order), for the FP64 smoother, which multiplies it by the
// cell's reciprocal diagonal instead of dividing.
template <int DIM, typename R, class LV>
__device__ __forceinline__ R gs_sum(const LV& L, const R* Tx, const R* Ty, const R* Tz, R rhs, const R* x, int i,
                                    const Row& r) {
  const int pc = r.pc + i;
  R s = rhs;
  s += Tx[r.fx + i] * x[pc - 1];
  s += Tx[r.fx + i + 1] * x[pc + 1];
  s += Ty[r.fy + i] * x[pc - L.px];
  s += Ty[r.fy + i + L.nx] * x[pc + L.px];
  if (DIM == 3) {
    const int pl = (int)L.plane;
    s += Tz[r.fz + i] * x[pc - pl];
    s += Tz[r.fz + i + L.nx * L.ny] * x[pc + pl];
  }
  return s;
}

// (A x)_c = sum_f T_f (x_c - x_nb); a boundary face gives T_f x_c.
template <int DIM, typename R, typename RX, class LV>
__device__ __forceinline__ R apply_value(const LV& L, const R* Tx, const R* Ty, const R* Tz, const RX* x, int i,
                                         const Row& r) {
  const int pc = r.pc + i;
  const R xc = (R)x[pc];
  R s = apply_terms2<R>(Tx[r.fx + i], Tx[r.fx + i + 1], Ty[r.fy + i], Ty[r.fy + i + L.nx], xc, (R)x[pc - 1],
                        (R)x[pc + 1], (R)x[pc - L.px], (R)x[pc + L.px]);
  if (DIM == 3) {
    const int pl = (int)L.plane;
    s += Tz[r.fz + i] * (xc - (R)x[pc - pl]);
    s += Tz[r.fz + i + L.nx * L.ny] * (xc - (R)x[pc + pl]);
  }
  return s;
}

// (R t)_C = (E^T t)_C for coarse cell (I, J, K) of level k+1: a gather over
// the window of fine cells that interpolate from it, with the tabled weights
// (Sec. 3, R = E^T).
template <int DIM, typename R, class FX>
__device__ __forceinline__ R restrict_value(const FX& F, const R* t, int I, int J, int K) {
  const R* rwx = (const R*)F.rw[0] + (long long)I * F.W[0];
  const R* rwy = (const R*)F.rw[1] + (long long)J * F.W[1];
  const int ilo = __ldg(F.lo[0] + I), ihi = __ldg(F.hi[0] + I), jlo = __ldg(F.lo[1] + J), jhi = __ldg(F.hi[1] + J);
  int klo = 0, khi = 0;
  const R* rwz = nullptr;
  if (DIM == 3) {
    klo = __ldg(F.lo[2] + K);
    khi = __ldg(F.hi[2] + K);
    rwz = (const R*)F.rw[2] + (long long)K * F.W[2];
  }
  R acc = 0;
  for (int kk = klo; kk <= khi; ++kk) {
    R accy = 0;
    for (int jj = jlo; jj <= jhi; ++jj) {
      const R* row = t + ((int)F.off + F.px * jj + (int)F.plane * kk);
      R accx = 0;
      for (int ii = ilo; ii <= ihi; ++ii) accx += __ldg(rwx + (ii - ilo)) * row[ii];
      accy += __ldg(rwy + (jj - jlo)) * accx;
    }
    acc += (DIM == 3 ? __ldg(rwz + (kk - klo)) : (R)1) * accy;
  }
  return acc;
}

// (E x_c) at fine cell (i, j, k): tensor product of the 1-D linear
// interpolation with zero slope at the boundary (Sec. 3).
template <int DIM, typename R, class FX, class CV>
__device__ __forceinline__ R prolong_value(const FX& F, const CV& C, const R* xc, int i, int j, int k) {
  const int coff = (int)C.off, cpl = (int)C.plane;
  const R wx = __ldg((const R*)F.w[0] + i), wy = __ldg((const R*)F.w[1] + j);
  const int i0 = __ldg(F.c0[0] + i), i1 = __ldg(F.c1[0] + i), j0 = __ldg(F.c0[1] + j), j1 = __ldg(F.c1[1] + j);
  if (DIM == 2) {
    const R* r0 = xc + (coff + C.px * j0);
    const R* r1 = xc + (coff + C.px * j1);
    const R a = ((R)1 - wx) * r0[i0] + wx * r0[i1];
    const R b = ((R)1 - wx) * r1[i0] + wx * r1[i1];
    return ((R)1 - wy) * a + wy * b;
  } else {
    const R wz = __ldg((const R*)F.w[2] + k);
    const int k0 = __ldg(F.c0[2] + k), k1 = __ldg(F.c1[2] + k);
    const R* r00 = xc + (coff + C.px * j0 + cpl * k0);
    const R* r10 = xc + (coff + C.px * j1 + cpl * k0);
    const R* r01 = xc + (coff + C.px * j0 + cpl * k1);
    const R* r11 = xc + (coff + C.px * j1 + cpl * k1);
    const R a0 = ((R)1 - wx) * r00[i0] + wx * r00[i1];
    const R b0 = ((R)1 - wx) * r10[i0] + wx * r10[i1];
    const R a1 = ((R)1 - wx) * r01[i0] + wx * r01[i1];
    const R b1 = ((R)1 - wx) * r11[i0] + wx * r11[i1];
    return ((R)1 - wz) * (((R)1 - wy) * a0 + wy * b0) + wz * (((R)1 - wy) * a1 + wy * b1);
  }
}

// ===========================================================================
// Single-CTA solver
// ===========================================================================

// One red-black half-sweep of colour `colour` by the CTA, with right-hand
// side rp (smoother precision).  Modes:
//  kZero: the iterate starts from x = 0: cells of `colour` get rhs/D, the
//         other colour is cleared; when the level's vectors are wider than
//         the smoother type, r is first rounded into rp at every cell.
//  kNormal: Gauss-Seidel update of the colour's cells.
//  kDot: as kNormal, and returns this thread's share of r . z over all cells
//        (r in the level's vector type; the other colour is final already).
enum : int { kNormal = 0, kZero = 1, kDot = 2 };

// A level's geometry, smoother-precision transmissibilities and the CTA's
// thread maps over all cells and over one colour, formed once for a run of
// phases on the level.
template <typename RP>
struct TLevel {
  Geo G;
  const RP *Tx, *Ty, *Tz;
  Map all, col;
};
template <typename RP>
__device__ __forceinline__ TLevel<RP> tlevel_of(const DevLevel& L) {
  TLevel<RP> t;
  t.G = geo_of(L);
  t.Tx = (const RP*)L.T[0];
  t.Ty = (const RP*)L.T[1];
  t.Tz = (const RP*)L.T[2];
  t.all = team_map(t.G.nx);
  t.col = team_map((t.G.nx + 1) >> 1);
  return t;
}

// One red/black half-sweep of a level by the team.  inv: the cells'
// reciprocal diagonals (padded layout), or null to divide.
template <int DIM, typename RP, typename V>
__device__ __forceinline__ V t_sweep(const TLevel<RP>& S, int colour, const V* r, RP* rp, RP* z, int mode,
                                     const RP* inv = nullptr) {
  const Geo& G = S.G;
  V acc = 0;
  if (mode == kZero) {
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      const int pc = rw.pc + i;
      RP rhs;
      if (sizeof(V) != sizeof(RP)) {
        rhs = (RP)r[pc];
        rp[pc] = rhs;
      } else {
        rhs = rp[pc];
      }
      z[pc] = ((i + rw.j + rw.k) & 1) == colour
                  ? (inv ? rhs * inv[pc] : quot<RP>(rhs, diag_of<DIM, RP>(G, S.Tx, S.Ty, S.Tz, i, rw)))
                  : (RP)0;
    });
  } else {
    const bool dot = mode == kDot;
    // every load of a cell comes before its store: the compiler cannot
    // move a load past a store it might alias
    for_colour<DIM>(S.col, G, colour, [&](int i, int i2, const Row& rw) {
      const int base = rw.pc;
      if (dot && i2 < G.nx) acc += r[base + i2] * (V)z[base + i2];
      if (i < G.nx) {
        const RP v = inv ? gs_sum<DIM, RP>(G, S.Tx, S.Ty, S.Tz, rp[base + i], z, i, rw) * inv[base + i]
                         : gs_value<DIM, RP, RP>(G, S.Tx, S.Ty, S.Tz, rp[base + i], z, i, rw);
        if (dot) acc += r[base + i] * (V)v;
        z[base + i] = v;
      }
    });
  }
  return acc;
}

// m modified Jacobi steps (P = 2D, Q = D - U - L, Sec. 3): every cell moves
// from the old values, z <- z + (rp - A z) / (2D), with A z formed first
// (into the t buffer, free during smoothing); from zero the first step is
// z = rp / (2D).  Returns r . z after the last step when `dot`.
template <int DIM, typename RP, typename V>
__device__ V t_jacobi(BlockTeam& tm, const DevLevel& L, const TLevel<RP>& S, int m, bool from_zero, bool dot) {
  const V* r = (const V*)L.r;
  RP* rp = (RP*)L.rp;
  RP* z = (RP*)L.z;
  RP* w = (RP*)L.t;
  const Geo& G = S.G;
  int s0 = 0;
  if (from_zero) {
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      const int pc = rw.pc + i;
      RP rhs;
      if (sizeof(V) != sizeof(RP)) {
        rhs = (RP)r[pc];
        rp[pc] = rhs;
      } else {
        rhs = rp[pc];
      }
      const RP d = diag_of<DIM, RP>(G, S.Tx, S.Ty, S.Tz, i, rw);
      z[pc] = quot<RP>(rhs, d + d);
    });
    tm.sync();
    s0 = 1;
  }
  V acc = 0;
  for (int st = s0; st < m; ++st) {
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      w[rw.pc + i] = apply_value<DIM, RP, RP>(G, S.Tx, S.Ty, S.Tz, z, i, rw);
    });
    tm.sync();
    const bool last = st == m - 1;
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      const int pc = rw.pc + i;
      const RP d = diag_of<DIM, RP>(G, S.Tx, S.Ty, S.Tz, i, rw);
      const RP v = z[pc] + quot<RP>(rp[pc] - w[pc], d + d);
      if (dot && last) acc += r[pc] * (V)v;
      z[pc] = v;
    });
    if (dot && last) return tm.sum<V>(acc);
    tm.sync();
  }
  return (V)0;
}

// m symmetric Gauss-Seidel steps in the natural order of the cells (i
// fastest, then j, then k): a forward sweep over increasing cell numbers,
// then a backward one.  A cell's update reads its lower neighbours (i-1, j-1,
// k-1) from the current sweep and its upper ones from before it, so the cells
// of one plane i + j + k = d are independent: each sweep runs plane by plane
// (forward: d ascending, backward: descending), a barrier apart.  Returns
// r . z at the end when `dot`.
template <int DIM, typename RP, typename V>
__device__ V t_lex(BlockTeam& tm, const DevLevel& L, const TLevel<RP>& S, int m, bool from_zero, bool dot) {
  const V* r = (const V*)L.r;
  RP* rp = (RP*)L.rp;
  RP* z = (RP*)L.z;
  const Geo& G = S.G;
  if (from_zero) {
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      const int pc = rw.pc + i;
      if (sizeof(V) != sizeof(RP)) rp[pc] = (RP)r[pc];
      z[pc] = (RP)0;
    });
    tm.sync();
  }
  const int rows = G.ny * G.nz, nd = G.nx + G.ny + G.nz - 3;  // planes d = 0 .. nd
  for (int st = 0; st < m; ++st)
    for (int dir = 0; dir < 2; ++dir)
      for (int e = 0; e <= nd; ++e) {
        const int d = dir == 0 ? e : nd - e;
        for (int row = threadIdx.x; row < rows; row += blockDim.x) {
          const Row rw = make_row<DIM>(G, row);
          const int i = d - rw.j - rw.k;
          if (i >= 0 && i < G.nx) z[rw.pc + i] = gs_value<DIM, RP, RP>(G, S.Tx, S.Ty, S.Tz, rp[rw.pc + i], z, i, rw);
        }
        tm.sync();
      }
  if (!dot) return (V)0;
  V acc = 0;
  for_cells<DIM>(S.all, G, [&](int i, const Row& rw) { acc += r[rw.pc + i] * (V)z[rw.pc + i]; });
  return tm.sum<V>(acc);
}

// m symmetric Gauss-Seidel steps (the smoothing factors of eq. 2.10):
// forward red, black, backward black, red; the repeated black half-sweep
// reproduces the same values, so m steps are the 2m+1 half-sweeps
// red (black red)^m.  Returns r . z after the last half-sweep when `dot`.
template <int DIM, typename RP, typename V>
__device__ V t_smooth(BlockTeam& tm, const DevLevel& L, const TLevel<RP>& S, int m, bool from_zero, bool dot,
                      int splitting) {
  if (splitting == 1) return t_jacobi<DIM, RP, V>(tm, L, S, m, from_zero, dot);
  if (splitting == 2) return t_lex<DIM, RP, V>(tm, L, S, m, from_zero, dot);
  const V* r = (const V*)L.r;
  RP* rp = (RP*)L.rp;
  RP* z = (RP*)L.z;
  const Geo& G = S.G;
  if (G.n <= (int)blockDim.x) {
    // one thread per cell: its face transmissibilities and diagonal stay in
    // registers for all half-sweeps (the terms and their order as in
    // diag_of / gs_value, so the values are the same)
    const int c = threadIdx.x;
    const bool own = c < G.n;
    int i = 0, j = 0, k = 0, pc = 0;
    RP tw = 0, te = 0, ts = 0, tn = 0, tb = 0, tt = 0, d = 1;
    if (own) {
      i = c % G.nx;
      const int row = c / G.nx;
      const Row rw = make_row<DIM>(G, row);
      j = rw.j;
      k = rw.k;
      pc = rw.pc + i;
      tw = S.Tx[rw.fx + i];
      te = S.Tx[rw.fx + i + 1];
      ts = S.Ty[rw.fy + i];
      tn = S.Ty[rw.fy + i + G.nx];
      d = tw;
      d += te;
      d += ts;
      d += tn;
      if (DIM == 3) {
        tb = S.Tz[rw.fz + i];
        tt = S.Tz[rw.fz + i + G.nx * G.ny];
        d += tb;
        d += tt;
      }
    }
    const int colour = (i + j + k) & 1;
    // FP64: multiply by the reciprocal diagonal, as the general path does
    const bool fp64 = sizeof(RP) == sizeof(double);
    const RP dinv = fp64 ? (RP)1 / d : (RP)0;
    auto gs = [&]() __attribute__((always_inline)) {
      RP dd, sm = rp[pc];
      gs_terms2<RP>(dd, sm, tw, te, ts, tn, z[pc - 1], z[pc + 1], z[pc - G.px], z[pc + G.px]);
      if (DIM == 3) {
        sm += tb * z[pc - G.plane];
        sm += tt * z[pc + G.plane];
      }
      z[pc] = fp64 ? sm * dinv : quot<RP>(sm, d);
    };
    if (own) {
      if (from_zero) {
        RP rhs;
        if (sizeof(V) != sizeof(RP)) {
          rhs = (RP)r[pc];
          rp[pc] = rhs;
        } else {
          rhs = rp[pc];
        }
        z[pc] = colour == 0 ? (fp64 ? rhs * dinv : quot<RP>(rhs, d)) : (RP)0;
      } else if (colour == 0) {
        gs();
      }
    }
    tm.sync();
    for (int h = 1; h <= 2 * m; ++h) {
      if (own && colour == (h & 1)) gs();
      if (h == 2 * m && dot) return tm.sum<V>(own ? r[pc] * (V)z[pc] : (V)0);
      tm.sync();
    }
    return (V)0;
  }
  // FP64: the reciprocal diagonals once per smoothing, in the t buffer (free
  // while smoothing): a half-sweep then multiplies instead of dividing (the
  // FP64 division is a long sequence on the narrow FP64 pipe)
  const RP* inv = nullptr;
  if (sizeof(RP) == sizeof(double)) {
    RP* w = (RP*)L.t;
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      w[rw.pc + i] = (RP)1 / diag_of<DIM, RP>(G, S.Tx, S.Ty, S.Tz, i, rw);
    });
    tm.sync();
    inv = w;
  }
  t_sweep<DIM, RP, V>(S, 0, r, rp, z, from_zero ? kZero : kNormal, inv);
  tm.sync();
  for (int s = 0; s < m; ++s) {
    t_sweep<DIM, RP, V>(S, 1, r, rp, z, kNormal, inv);
    tm.sync();
    const bool last = s == m - 1;
    const V d = t_sweep<DIM, RP, V>(S, 0, r, rp, z, dot && last ? kDot : kNormal, inv);
    if (dot && last) return tm.sum<V>(d);
    tm.sync();
  }
  return (V)0;
}

// Coarsest level: z = A^-1 r with the FP64 explicit inverse (the recursion
// ends with the exact inverse, Sec. 2.2).  rc: compact shared scratch.
template <int DIM, typename V, typename RP>
__device__ void t_coarsest(BlockTeam& tm, const DevLevel& L, const double* Ainv, bool transposed, int nc, const V* r,
                           RP* z, double* rc) {
  const Geo G = geo_of(L);
  for_cells<DIM>(team_map(G.nx), G, [&](int i, const Row& rw) {
    rc[i + G.nx * (rw.j + G.ny * rw.k)] = (double)r[rw.pc + i];
  });
  tm.sync();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    double s = 0.0;
    if (transposed) {
      for (int j = 0; j < nc; ++j) s += Ainv[j * nc + c] * rc[j];
    } else {
      const double* row = Ainv + (long long)c * nc;
      for (int j = 0; j < nc; ++j) s += __ldg(row + j) * rc[j];
    }
    const int i = c % G.nx, rw = c / G.nx, jj = rw % G.ny, kk = rw / G.ny;
    z[(int)G.off + i + G.px * jj + (int)G.plane * kk] = (RP)s;
  }
  tm.sync();
}

// r_{k+1} = R t by the CTA (the gather of restrict_value): G threads per
// coarse cell, G a power of two up to 8 chosen so the coarse cells cover
// the CTA, each taking every G-th fine row of the cell's window; the group
// then adds its partial sums with shuffles.  The loop over coarse cells has
// the same trip count in every thread, so every lane reaches the shuffles.
template <int DIM, typename R>
__device__ void t_restrict(const Xf& F, const Geo& Gc, const R* t, R* rc) {
  const int nc = Gc.nx * Gc.ny * Gc.nz;
  int lg = 0;
  while (lg < 3 && (nc << (lg + 1)) <= (int)blockDim.x) ++lg;
  const int G = 1 << lg, member = threadIdx.x & (G - 1), per = blockDim.x >> lg;
  for (int base = 0; base < nc; base += per) {
    const int cell = base + ((int)threadIdx.x >> lg);
    R part = 0;
    int pc = 0;
    if (cell < nc) {
      const int I = cell % Gc.nx, rest = cell / Gc.nx, J = rest % Gc.ny, K = rest / Gc.ny;
      pc = Gc.off + I + Gc.px * J + Gc.plane * K;
      const R* rwx = (const R*)F.rw[0] + I * F.W[0];
      const R* rwy = (const R*)F.rw[1] + J * F.W[1];
      const int ilo = __ldg(F.lo[0] + I), ihi = __ldg(F.hi[0] + I), jlo = __ldg(F.lo[1] + J), jhi = __ldg(F.hi[1] + J);
      int klo = 0, khi = 0;
      const R* rwz = nullptr;
      if (DIM == 3) {
        klo = __ldg(F.lo[2] + K);
        khi = __ldg(F.hi[2] + K);
        rwz = (const R*)F.rw[2] + K * F.W[2];
      }
      for (int kk = klo; kk <= khi; ++kk) {
        R accy = 0;
        for (int jj = jlo + member; jj <= jhi; jj += G) {
          const R* row = t + (F.off + F.px * jj + F.plane * kk);
          R accx = 0;
#pragma unroll 4
          for (int ii = ilo; ii <= ihi; ++ii) accx += __ldg(rwx + (ii - ilo)) * row[ii];
          accy += __ldg(rwy + (jj - jlo)) * accx;
        }
        part += (DIM == 3 ? __ldg(rwz + (kk - klo)) : (R)1) * accy;
      }
    }
    for (int o = G >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (cell < nc && member == 0) rc[pc] = part;
  }
}

__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Zero `bytes` (a multiple of 16) of shared memory at p, 16 bytes a store.
__device__ __forceinline__ void zero_block(unsigned char* p, size_t bytes) {
  float4* q = (float4*)p;
  for (size_t e = threadIdx.x; e < bytes / 16; e += blockDim.x) q[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// Single-pass red-black smoothing of a 2D level in global memory (one CTA)
// ---------------------------------------------------------------------------
// The 2m+1 half-sweeps of one smoothing run as the stages of a row pipeline
// that advances two rows a step: at step s, stage q updates its colour's cells
// in rows 2s - 3q and 2s - 3q + 1.  Those two rows hold one cell of each colour
// per column, so every column takes part in every stage at every step (column
// i: row 2s - 3q + (i & 1), the colour of half-sweep q there).  Stage q reads
// the other colour in rows 2s-3q-1 .. 2s-3q+2, which stage q-1 finished at
// earlier steps (it works on rows 2s-3q+3 and +4 now) and which stage q+1
// (rows 2s-3q-3 and -2 now) has not yet overwritten; no two stages of a step
// touch the same cells, so one barrier per step orders everything and every
// cell gets exactly the values of the plain half-sweep order.  The level is
// cut into column strips; a strip loads its columns and 2m+1 more on each side
// (the cells whose later stages go stale without the neighbouring strip; the
// neighbour recomputes them with the same arithmetic) into rings of rows in
// shared memory, prefetched kFuseAhead steps ahead with cp.async.  Each row of
// T, rp (and z) then crosses HBM once per smoothing instead of once per
// half-sweep.  kFuseShare threads own each column of the strip and share its
// stages; every load of a step precedes its stores.  The rings take the shared
// memory of the coarse levels resident there, whose vectors hold nothing live
// while a finer level smooths (they are zeroed again after).
//   pre  (from zero): stage 0 sets z = rp/D on red cells and 0 on black; rows
//        2s - 3S and 2s - 3S + 1, final by then, get t = rp - A z, and z and t
//        are written.
//   post (z holds the prolonged pre-smoothing result): the strip reads z and
//        writes the smoothed z to `zout` (strips read their halo from the
//        unsmoothed z, so the result cannot go back in place) two rows behind
//        the last stage; the last stage's two rows add r . z over the strip's
//        own cells (returned per thread).
constexpr int kFuseAhead = 3;    // steps (two rows each) prefetched ahead of stage 0
constexpr int kFuseMinWidth = 16;
constexpr int kFuseMinCells = 4096;  // default smallest level that takes the single pass
constexpr int kFuseMaxM = 4;     // stages per thread <= 5 (two threads per column)
#ifndef MSRCG_FUSE_SHARE
#define MSRCG_FUSE_SHARE 2
#endif
constexpr int kFuseShare = MSRCG_FUSE_SHARE;  // threads per ring column
// stage entries per thread and step: the column's 2m+1 stages dealt round
// kFuseShare threads
constexpr int kFuseE = (2 * kFuseMaxM + 1 + kFuseShare - 1) / kFuseShare;
constexpr int kFuseRoleZ = kFuseShare > 1 ? 1 : 0;  // share loading rp / z, adding the other colour's r.z
// share with the fewest stages: the result (pre) / write-back (post) rows and
// the r rows of the post-smoothing dot
constexpr int kFuseRoleR = kFuseShare - 1;

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Step s of the pipeline commits group s + kFuseAhead; group g holds rows 2g
// and 2g + 1 and the face rows above them.  Stage 0 at step s reads rows up to
// 2s + 2 (post-smoothing: the z row above, loaded from global memory), so all
// groups but the newest kFuseAhead - 1 must be complete.
__device__ __forceinline__ void cp_async_wait_ahead() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kFuseAhead - 1) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Ring depths (rows, even): T / rp / z rows live from the prefetch (rows
// 2(s + kFuseAhead) + 1 and the face row above) down to the result rows
// (2s - 3S, and the row below); r rows (post) only from their prefetch to
// the last stage.  A copy issued at step s may land while slower threads
// still compute step s - 1, hence one step more of each.
__host__ __device__ __forceinline__ int fuse_depth(int S) { return 3 * S + 2 * kFuseAhead + 5; }
__host__ __device__ __forceinline__ int fuse_rdepth() { return 2 * kFuseAhead + 4; }

// Output columns per strip that fit `bytes` of shared memory and a CTA of
// `threads` (kFuseShare threads per loaded column; a ring row also holds the
// two zero columns at its ends); 0: fusion off.
__host__ __device__ __forceinline__ int fuse_width(int m, size_t bytes, int vsz, int threads) {
  if (m < 1 || m > kFuseMaxM || bytes < 64) return 0;
  const int S = 2 * m + 1, D = fuse_depth(S);
  const size_t per_col = 16 * (size_t)D + (size_t)fuse_rdepth() * vsz;
  int ws = (int)((bytes - 16) / per_col);
  if (ws > threads / kFuseShare + 2) ws = threads / kFuseShare + 2;
  const int wo = ws - 2 * S - 2;
  return wo >= kFuseMinWidth ? wo : 0;
}

template <typename V>
__device__ V fused_smooth(const DevLevel& L, int m, bool pre, unsigned win_off, int Wo, float* zout) {
  // the rings, addressed from the kernel's dynamic shared memory itself so
  // that every ring access compiles to a shared-memory load or store
  extern __shared__ __align__(16) unsigned char fuse_smem[];
  float* const win = (float*)(fuse_smem + win_off);
  const int S = 2 * m + 1, D = fuse_depth(S), DR = fuse_rdepth();
  // result (pre) / write-back (post) rows of step s: 2s - lag and the next;
  // the last stage's rows: 2s - lastq and the next
  const int lag = pre ? 3 * S : 3 * S - 1, lastq = 3 * (S - 1);
  const int nx = L.nx, ny = L.ny, px = L.px, off = (int)L.off;
  const float* gTx = (const float*)L.T[0];
  const float* gTy = (const float*)L.T[1];
  const float* grp = (const float*)L.rp;
  const float* gz = (const float*)L.z;
  float* gzo = pre ? (float*)L.z : zout;
  float* gt = (float*)L.t;
  const V* gr = (const V*)L.r;
  const int bd = blockDim.x, share = bd / kFuseShare;
  // ring column (1 + the loaded column), and which share of the column's
  // stages (hs == kFuseShare: the few threads left over, idle)
  const int col = 1 + threadIdx.x % share, hs = threadIdx.x / share;
  const int s_end = (ny - 1 + lag) >> 1;  // the step whose result rows reach row ny - 1
  V acc = 0;
  for (int a0 = 0; a0 < nx; a0 += Wo) {
    const int a1 = min(nx, a0 + Wo), c0 = max(0, a0 - S), c1 = min(nx, a1 + S);
    const int Ws = c1 - c0 + 2;  // ring row: columns c0-1 .. c1; the two ends stay zero
    const int DW = D * Ws;       // one ring, in floats
    float* sTx = win;
    float* sTy = sTx + DW;
    float* srp = sTy + DW;
    float* sz = srp + DW;
    V* sr = (V*)(win + ((4 * DW + 3) & ~3));
    for (int e = threadIdx.x; e < 4 * DW; e += bd) win[e] = 0.f;
    __syncthreads();
    // this thread's ring column `col` is column i of the level
    const int i = c0 - 1 + col;
    const int ib = i & 1;  // the row of each stage's pair that has this column's cell
    const bool live = hs < kFuseShare;
    const bool mine = live && col <= Ws - 2;     // a loaded cell (and its west x-face)
    const bool east = mine && col == Ws - 2;     // ... and the strip's last x-face
    const bool own = live && i >= a0 && i < a1;  // a cell this strip writes
    // loads (share 0: T rows; share 1: rp and z rows; the last share: r rows)
    // walk down the level with running pointers
    // face rows: x-faces of cell row j at tx(j), y-faces of face row f at
    // ty(f) (compact rows on a constant-coefficient level)
    const bool lap = L.lap != 0;
    auto tx_row = [&](int j) __attribute__((always_inline)) { return gTx + (lap ? 0 : (nx + 1) * j) + i; };
    auto ty_row = [&](int f) __attribute__((always_inline)) { return gTy + nx * (lap ? face_row(f, ny) : f) + i; };
    const float* prp = grp + off + i;
    const float* pz = gz + off + i;
    if (mine && hs == 0) cp_async4(sTy + col, ty_row(0));  // face row 0
    int jl = 0, lo = 0;  // next row pair to load (rows jl, jl + 1) and the ring offset of row jl
    auto load_next = [&]() __attribute__((always_inline)) {
      if (jl <= ny && mine) {
        if (hs == 0) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int j = jl + r;
            if (j < ny) {
              const float* tx = tx_row(j);
              cp_async4(sTx + lo + r * Ws + col, tx);
              if (east) cp_async4(sTx + lo + r * Ws + col + 1, tx + 1);
              // face row j + 1 into the slot of row j + 1
              const int fo = lo + (r + 1) * Ws;
              cp_async4(sTy + (fo == DW ? 0 : fo) + col, ty_row(j + 1));
            }
          }
        }
        if (hs == kFuseRoleZ) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int j = jl + r;
            if (j < ny) {
              cp_async4(srp + lo + r * Ws + col, prp + r * px);
              if (!pre) cp_async4(sz + lo + r * Ws + col, pz + r * px);
            } else if (j == ny && !pre) {
              cp_async4(sz + lo + r * Ws + col, pz + r * px);  // the zero ghost row
            }
          }
        }
      }
      prp += 2 * px;
      pz += 2 * px;
      lo = lo + 2 * Ws == DW ? 0 : lo + 2 * Ws;
      jl += 2;
    };
    for (int k = 0; k < kFuseAhead; ++k) {
      load_next();
      cp_async_commit();
    }
    int sbo = 0;  // ring offset of row 2s
    for (int s = 0; s <= s_end; ++s) {
      load_next();
      int rs = 0;  // r ring offset of the last stage's first row at this column
      if (!pre) {
        if (hs == kFuseRoleR && own) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int jr = 2 * (s + kFuseAhead) - lastq + r;
            if (jr >= 0 && jr < ny) {
              V* dst = sr + (jr % DR) * Ws + col;
              if (sizeof(V) == 8) cp_async8(dst, gr + off + px * jr + i);
              else cp_async4(dst, gr + off + px * jr + i);
            }
          }
        }
        const int jd = 2 * s - lastq;  // even: rows jd, jd + 1 sit in neighbouring slots
        rs = (jd >= 0 ? jd % DR : 0) * Ws + col;
      }
      cp_async_commit();
      cp_async_wait_ahead();
      __syncthreads();
      if (pre && (2 * s == ny - 1 || 2 * s == ny)) {
        // the zero ghost row above the last row (its slot held an older row;
        // no stage reads that row at this step)
        const int sl = (ny % D) * Ws;
        for (int e = threadIdx.x; e < Ws; e += bd) sz[sl + e] = 0.f;
      }
      if (mine) {
        float v[kFuseE];
        int ro[kFuseE];
        bool act[kFuseE];
#pragma unroll
        for (int e = 0; e < kFuseE; ++e) {
          const int q = hs + kFuseShare * e;
          const int j = 2 * s - 3 * q + ib;
          act[e] = q < S && j >= 0 && j < ny;
          ro[e] = 0;
          v[e] = 0.f;
          if (act[e]) {
            int r0 = sbo - (3 * q - ib) * Ws;
            if (r0 < 0) r0 += DW;
            const int ru = r0 + Ws == DW ? 0 : r0 + Ws, rd = r0 == 0 ? DW - Ws : r0 - Ws;
            const int c = r0 + col;
            const float tw = sTx[c], te = sTx[c + 1], ts = sTy[c], tn = sTy[ru + col];
            float d, sm = srp[c];
            if (pre && q == 0) {
              // stage 0 of pre-smoothing (from zero): rp / D on red cells
              d = tw;
              d += te;
              d += ts;
              d += tn;
            } else {
              gs_terms2<float>(d, sm, tw, te, ts, tn, sz[c - 1], sz[c + 1], sz[rd + col], sz[ru + col]);
            }
            v[e] = quot<float>(sm, d);
            ro[e] = c;
            if (!pre && q == S - 1 && own) acc += sr[rs + ib * Ws] * (V)v[e];
          }
        }
        if (hs == 0 && pre && 2 * s + 1 - ib < ny) sz[sbo + (1 - ib) * Ws + col] = 0.f;  // stage 0's black cell
        if (hs == kFuseRoleR && own) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int jw = 2 * s - lag + r;
            if (jw >= 0 && jw < ny) {
              int r0 = sbo - (lag - r) * Ws;
              if (r0 < 0) r0 += DW;
              const int c = r0 + col;
              const float zc = sz[c];
              const int g = off + px * jw + i;
              if (pre) {
                const int ru = r0 + Ws == DW ? 0 : r0 + Ws, rd = r0 == 0 ? DW - Ws : r0 - Ws;
                const float a = apply_terms2<float>(sTx[c], sTx[c + 1], sTy[c], sTy[ru + col], zc, sz[c - 1],
                                                    sz[c + 1], sz[rd + col], sz[ru + col]);
                gt[g] = srp[c] - a;
              }
              gzo[g] = zc;
            }
          }
        }
        if (hs == kFuseRoleZ && !pre && own) {
          // the last stage's other row at this column: a cell of the other
          // colour, final already
          const int jo = 2 * s - lastq + 1 - ib;
          if (jo >= 0 && jo < ny) {
            int r0 = sbo - (lastq - 1 + ib) * Ws;
            if (r0 < 0) r0 += DW;
            acc += sr[rs + (1 - ib) * Ws] * (V)sz[r0 + col];
          }
        }
#pragma unroll
        for (int e = 0; e < kFuseE; ++e)
          if (act[e]) sz[ro[e]] = v[e];
      }
      sbo = sbo + 2 * Ws == DW ? 0 : sbo + 2 * Ws;
    }
    cp_async_wait_all();
    __syncthreads();
  }
  return acc;
}

// Control of one level of the single-CTA state machine.  Scalars are kept
// in both precisions so that an FP32 level never converts.
struct LvlCtl {
  double rho_d, rho_old_d, thrN_d;
  float rho_f, rho_old_f, thrN_f;
  int it, phase;
  // level 0: ||r||^2 of the last update, the stall test's best residual and
  // its iteration, r_new . z_old of the last update (flexible beta)
  double rr_d, rr_best, gamma_d;
  int it_best;
  bool gamma_ok;
};
enum : int { kStart = 0, kIterate = 1, kAfterCoarse = 2, kPrecondDone = 3, kReturn = 4 };

template <typename V>
struct Scal;
template <>
struct Scal<double> {
  static __device__ __forceinline__ double& rho(LvlCtl& c) { return c.rho_d; }
  static __device__ __forceinline__ double& rho_old(LvlCtl& c) { return c.rho_old_d; }
  // the level test ||r||^2 / N_k < thr, as ||r||^2 < thr N_k
  static __device__ __forceinline__ bool below(const LvlCtl& c, double rr) { return rr < c.thrN_d; }
};
template <>
struct Scal<float> {
  static __device__ __forceinline__ float& rho(LvlCtl& c) { return c.rho_f; }
  static __device__ __forceinline__ float& rho_old(LvlCtl& c) { return c.rho_old_f; }
  static __device__ __forceinline__ bool below(const LvlCtl& c, float rr) {
    // thr N_k below the normal FP32 range: decide in FP64
    return c.thrN_f > 1e-30f ? rr < c.thrN_f : (double)rr < c.thrN_d;
  }
};

struct RecArgs {
  int kmax, m, nc;
  const double* Ainv;
  bool ainv_t;      // Ainv held transposed (shared-memory copy)
  double eps2, floor2;
  float floor2_f;
  SolveState* S;
  bool top_double;  // level 0 keeps FP64 vectors
  double* rc;       // shared scratch of the coarsest solve
  // per level, in shared memory: f^k eps^2 N_k in both precisions, and the
  // iteration / call counters of this launch (added to S at the end)
  const double* thrN_d;
  const float* thrN_f;
  long long* iters;
  long long* calls;
  // rings of the single-pass smoother, when allowed: the shared memory from
  // the resident levels' vectors (free while a wider level smooths; zeroed
  // again after each pass) to the end
  unsigned win_off;    // byte offset in the dynamic shared memory
  unsigned vec_bytes;  // the resident vectors at its start
  size_t win_bytes;
  bool fuse;
  int fuse_width, fuse_min_cells;
  int splitting;  // 0: red-black symmetric Gauss-Seidel, 1: modified Jacobi, 2: natural-order SGS
  // flexible beta of the level-0 PCG: in use (*flex, the same value in every
  // thread), may be switched on (allow_flex), stall test length (0: none)
  bool* flex;
  bool allow_flex;
  int stall_w;
  int precond;  // 0: recursive multi-scale (eq. 2.10), 1: multigrid (eq. 2.9), 2: polynomial (eq. 2.6, W = P^-1)
  // level tree (msrcg_set_trace): count, pad, then entries (level, call,
  // iterations, pass); null when off
  unsigned long long* trace;
  int trace_cap;
  int pass;  // 0, or the restart from the true residual
};

// One level-tree entry (thread 0): level k's PCG call that just returned.
__device__ __forceinline__ void trace_call(const RecArgs& a, int k, int it) {
  const unsigned long long e = atomicAdd(a.trace, 1ULL);
  if (e < (unsigned long long)a.trace_cap)
    reinterpret_cast<int4*>(a.trace + 2)[e] = make_int4(k, (int)(a.calls[k] - 1), it, a.pass);
}

// Strip width of the single-pass smoother for level L, or 0 for the plain
// half-sweeps (levels in shared memory, small levels, no room).
template <typename V>
__device__ __forceinline__ int fuse_wo(const DevLevel& L, int m, const RecArgs& a) {
  if (!a.fuse || a.splitting != 0 || __isShared(L.z) || (long long)L.nx * L.ny < a.fuse_min_cells) return 0;
  int w = fuse_width(m, a.win_bytes, (int)sizeof(V), blockDim.x);
  if (w <= 0) return 0;
  // one strip over the whole level needs no halo columns
  if (L.nx <= w + 2 * (2 * m + 1)) w = L.nx;
  if (a.fuse_width > 0 && a.fuse_width < w) w = max(a.fuse_width, kFuseMinWidth);
  // strips of equal width: as many as width w needs
  const int ns = (L.nx + w - 1) / w;
  return (L.nx + ns - 1) / ns;
}

// After a single pass: the resident levels' vectors, which the rings
// overwrote, back to zero (their state at placement), then a barrier.
__device__ __forceinline__ void release_window(const RecArgs& a) {
  extern __shared__ __align__(16) unsigned char fuse_smem[];
  zero_block(fuse_smem + a.win_off, a.vec_bytes);
  __syncthreads();
}

// Per-level thresholds of the level test and zeroed counters (thread 0),
// then a barrier.
__device__ void level_consts(const DevLevel* sL, int nlev, double eps2, double* thrN_d, float* thrN_f,
                             long long* iters, long long* calls) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < nlev; ++k) {
      thrN_d[k] = sL[k].fk * eps2 * (double)sL[k].n;
      thrN_f[k] = (float)thrN_d[k];
      iters[k] = 0;
      calls[k] = 0;
    }
  }
  __syncthreads();
}

// Add this launch's counters to the problem's state (thread 0).
__device__ void flush_counts(SolveState* S, int nlev, const long long* iters, const long long* calls) {
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < nlev; ++k) {
      S->lv[k].iters += iters[k];
      S->lv[k].calls += calls[k];
    }
}

// Steps of one level with vector type V (double at level 0 of a full solve,
// the smoother type RP elsewhere).
template <int DIM, typename V, typename RP>
struct Ops {
  // PCG entry (x = 0; r holds b_k): ||b_k||^2.  An FP64 level with an
  // FP32 smoother also gets rp = (FP32) r here and at every update, the
  // smoother's copy of the right-hand side.
  static __device__ V enter(BlockTeam& tm, const DevLevel& L) {
    V* x = (V*)L.x;
    const V* r = (const V*)L.r;
    RP* rp = (RP*)L.rp;
    const int npad = (int)L.npad;
    V acc = 0;
    for_lin(npad, [&](int c) { return r[c]; }, [&](int c, V rv) {
      acc += rv * rv;
      x[c] = 0;
      if (sizeof(V) != sizeof(RP)) rp[c] = (RP)rv;
    });
    return tm.sum<V>(acc);
  }
  // pre-smoothing from zero, t = r - A z, r_{k+1} = R t
  static __device__ void presmooth_restrict(BlockTeam& tm, const DevLevel& L, const DevLevel& C, int m,
                                             const RecArgs& a) {
    if constexpr (DIM == 2 && sizeof(RP) == sizeof(float)) {
      const int wo = fuse_wo<V>(L, m, a);
      if (wo > 0) {
        // (rp, the smoother-precision copy of r, comes from the level entry
        // or the last update)
        fused_smooth<V>(L, m, true, a.win_off, wo, nullptr);
        release_window(a);
        t_restrict<DIM, RP>(xf_of(L), geo_of(C), (const RP*)L.t, (RP*)C.r);
        tm.sync();
        return;
      }
    }
    const TLevel<RP> S = tlevel_of<RP>(L);
    t_smooth<DIM, RP, V>(tm, L, S, m, true, false, a.splitting);
    const RP* rp = (const RP*)L.rp;
    const RP* z = (const RP*)L.z;
    RP* t = (RP*)L.t;
    const Geo& G = S.G;
    for_cells<DIM>(S.all, G, [&](int i, const Row& rw) {
      t[rw.pc + i] = rp[rw.pc + i] - apply_value<DIM, RP, RP>(G, S.Tx, S.Ty, S.Tz, z, i, rw);
    });
    tm.sync();
    t_restrict<DIM, RP>(xf_of(L), geo_of(C), t, (RP*)C.r);
    tm.sync();
  }
  // z += E x_c on the black cells only: the first post-smoothing half-sweep
  // recomputes every red cell from its black neighbours, so a red cell's
  // prolonged value would never be read (every cell for the other smoothers).
  // Then post-smoothing; returns r.z.
  static __device__ V prolong_postsmooth(BlockTeam& tm, const DevLevel& L, const DevLevel& C, int m,
                                         const RecArgs& a) {
    {
      RP* z = (RP*)L.z;
      const RP* xc = (const RP*)C.x;
      const Xf X = xf_of(L);
      const Geo Gc = geo_of(C);
      if (a.splitting != 0) {
        // the Jacobi and natural-order smoothers read every cell's prolonged
        // value
        for_cells<DIM>(team_map(X.nx), X, [&](int i, const Row& rw) {
          z[rw.pc + i] += prolong_value<DIM, RP>(X, Gc, xc, i, rw.j, rw.k);
        });
      } else {
        for_colour<DIM>(team_map((X.nx + 1) >> 1), X, 1, [&](int i, int, const Row& rw) {
          if (i < X.nx) z[rw.pc + i] += prolong_value<DIM, RP>(X, Gc, xc, i, rw.j, rw.k);
        });
      }
    }
    tm.sync();
    if constexpr (DIM == 2 && sizeof(RP) == sizeof(float)) {
      const int wo = fuse_wo<V>(L, m, a);
      if (wo > 0) {
        const V acc = fused_smooth<V>(L, m, false, a.win_off, wo, (float*)L.t);
        release_window(a);
        // the smoothed z went to the t buffer (free after the restriction):
        // swap the two in this CTA's copy of the level descriptor
        if (threadIdx.x == 0) {
          DevLevel& W = const_cast<DevLevel&>(L);
          void* z = W.z;
          W.z = W.t;
          W.t = z;
        }
        return tm.sum<V>(acc);
      }
    }
    return t_smooth<DIM, RP, V>(tm, L, tlevel_of<RP>(L), m, false, true, a.splitting);
  }
  static __device__ V coarsest(BlockTeam& tm, const DevLevel& L, const RecArgs& a) {
    t_coarsest<DIM, V, RP>(tm, L, a.Ainv, a.ainv_t, a.nc, (const V*)L.r, (RP*)L.z, a.rc);
    const V* r = (const V*)L.r;
    const RP* z = (const RP*)L.z;
    const int npad = (int)L.npad;
    V acc = 0;
    for (int c = threadIdx.x; c < npad; c += blockDim.x) acc += r[c] * (V)z[c];
    return tm.sum<V>(acc);
  }
  // p = z + beta p, q = A p, alpha = rho / p.q, x += alpha p, r -= alpha q.
  // Returns ||r||^2 (false on breakdown).  With `flex`, beta is the flexible
  // (Polak-Ribiere) factor (rho - r.z_old) / rho_old once the previous update
  // has formed r.z_old, and this update forms r_new . z for the next one.
  static __device__ bool cg_step(BlockTeam& tm, const DevLevel& L, LvlCtl& ct, V& rr_out, bool flex) {
    const V rho = Scal<V>::rho(ct);
    const bool first = ct.it == 0;
    const V beta = first ? (V)0
                         : (flex && ct.gamma_ok ? (rho - (V)ct.gamma_d) / Scal<V>::rho_old(ct)
                                                : rho / Scal<V>::rho_old(ct));
    V* p = (V*)L.p;
    V* q = (V*)L.q;
    const RP* z = (const RP*)L.z;
    const Geo G = geo_of(L);
    const int npad = G.npad;
    if (first)
      for_lin(npad, [&](int c) { return z[c]; }, [&](int c, RP zv) { p[c] = (V)zv; });
    else
      for_lin(npad, [&](int c) { return Two<RP, V>{z[c], p[c]}; },
              [&](int c, Two<RP, V> v) { p[c] = (V)v.a + beta * v.b; });
    tm.sync();
    const V *Tx = Tvec<V>(L, 0), *Ty = Tvec<V>(L, 1), *Tz = DIM == 3 ? Tvec<V>(L, 2) : nullptr;
    V acc = 0;
    // a = (A p)_c, b = p_c
    for_cells_u<DIM>(
        team_map(G.nx), G,
        [&](int i, const Row& rw) {
          return Two<V, V>{apply_value<DIM, V, V>(G, Tx, Ty, Tz, p, i, rw), p[rw.pc + i]};
        },
        [&](int i, const Row& rw, Two<V, V> v) {
          acc += v.b * v.a;
          q[rw.pc + i] = v.a;
        });
    const V pq = tm.sum<V>(acc);
    if (!(pq > (V)0) || !isfinite(pq) || !isfinite(rho)) return false;
    const V alpha = rho / pq;
    V* x = (V*)L.x;
    V* r = (V*)L.r;
    RP* rp = (RP*)L.rp;
    V acc2 = 0;
    if (flex) {
      V acc3 = 0;
      for_lin(npad, [&](int c) { return Two<Four<V>, RP>{Four<V>{x[c], p[c], r[c], q[c]}, z[c]}; },
              [&](int c, Two<Four<V>, RP> v) {
                const V xv = v.a.x + alpha * v.a.p;
                const V rv = v.a.r - alpha * v.a.q;
                acc2 += rv * rv;
                acc3 += rv * (V)v.b;
                x[c] = xv;
                r[c] = rv;
                if (sizeof(V) != sizeof(RP)) rp[c] = (RP)rv;
              });
      rr_out = tm.sum<V>(acc2);
      ct.gamma_d = (double)tm.sum<V>(acc3);
      ct.gamma_ok = true;
      return true;
    }
    for_lin(npad, [&](int c) { return Four<V>{x[c], p[c], r[c], q[c]}; }, [&](int c, Four<V> v) {
      const V xv = v.x + alpha * v.p;
      const V rv = v.r - alpha * v.q;
      acc2 += rv * rv;
      x[c] = xv;
      r[c] = rv;
      if (sizeof(V) != sizeof(RP)) rp[c] = (RP)rv;
    });
    rr_out = tm.sum<V>(acc2);
    ct.gamma_ok = false;
    return true;
  }
  // one CG step and the level test; returns 0 = continue, 1 = converged,
  // 2 = breakdown
  static __device__ int iterate(BlockTeam& tm, const DevLevel& L, LvlCtl& c, SolveState* S, const RecArgs& a, int k) {
    V rr;
    if (!cg_step(tm, L, c, rr, k == 0 && *a.flex)) return 2;
    c.rr_d = (double)rr;
    if (threadIdx.x == 0) {
      a.iters[k]++;
      if (k == 0) S->lv[0].rr = (double)rr;
    }
    return Scal<V>::below(c, rr) ? 1 : 0;
  }
};

// The recursion of eq. (2.10) from level ks down to kmax, run by the CTA.
// On entry r_ks holds the level's right-hand side; on exit x_ks holds the
// PCG result.
template <int DIM, typename RP>
__device__ void recursion(BlockTeam& tm, const DevLevel* sL, int ks, const RecArgs& a) {
  LvlCtl ct[kMaxLev];
  int k = ks;
  ct[k].phase = kStart;
  SolveState* S = a.S;
  for (;;) {
    const DevLevel& L = sL[k];
    LvlCtl& c = ct[k];
    const bool dbl = a.top_double && k == 0;
    if (c.phase == kStart) {
      if (threadIdx.x == 0) a.calls[k]++;
      c.it = 0;
      if (a.precond == 1 && k > 0) {
        // multigrid (eq. 2.9): this level applies its preconditioner once
        // to r_k; no PCG, no level test
        c.phase = kIterate;
        continue;
      }
      // level test of Sec. 3: ||r||^2 / N_k < f^k eps^2, kept as
      // ||r||^2 < f^k eps^2 N_k (thrN, precomputed per level); inner levels
      // may also stop at a floor relative to ||b_k||.  FP32 levels do this in
      // FP32 (FP64 only when the threshold leaves the normal FP32 range).
      bool live;
      if (dbl || sizeof(RP) == sizeof(double)) {
        const double bb = dbl ? (double)Ops<DIM, double, RP>::enter(tm, L) : (double)Ops<DIM, RP, RP>::enter(tm, L);
        live = bb > 0.0;
        c.rr_best = bb;
        c.thrN_d = a.thrN_d[k];
        if (k > 0 && a.floor2 > 0.0) c.thrN_d = fmax(c.thrN_d, a.floor2 * bb);
        c.thrN_f = (float)c.thrN_d;
      } else {
        const float bb = (float)Ops<DIM, RP, RP>::enter(tm, L);
        live = bb > 0.f;
        c.rr_best = (double)bb;
        c.thrN_f = fmaxf(a.thrN_f[k], a.floor2_f * bb);
        if (!(c.thrN_f > 1e-30f)) c.thrN_d = fmax(a.thrN_d[k], a.floor2 * (double)bb);
      }
      if (!live) {
        c.phase = kReturn;
        continue;
      }
      c.it = 0;
      c.rho_old_d = 0.0;
      c.rho_old_f = 0.f;
      c.gamma_ok = false;
      c.it_best = 0;
      c.phase = kIterate;
    } else if (c.phase == kIterate) {
      if (a.precond == 2 && k == 0 && a.kmax > 0) {
        // polynomial (eq. 2.6 with W = P^-1): 2m+1 splitting steps from zero
        const TLevel<RP> T = tlevel_of<RP>(L);
        if (dbl) c.rho_d = t_smooth<DIM, RP, double>(tm, L, T, 2 * a.m + 1, true, true, a.splitting);
        else Scal<RP>::rho(c) = t_smooth<DIM, RP, RP>(tm, L, T, 2 * a.m + 1, true, true, a.splitting);
        c.phase = kPrecondDone;
      } else if (k == a.kmax) {
        if (dbl) c.rho_d = Ops<DIM, double, RP>::coarsest(tm, L, a);
        else Scal<RP>::rho(c) = Ops<DIM, RP, RP>::coarsest(tm, L, a);
        c.phase = kPrecondDone;
      } else {
        if (dbl) Ops<DIM, double, RP>::presmooth_restrict(tm, L, sL[k + 1], a.m, a);
        else Ops<DIM, RP, RP>::presmooth_restrict(tm, L, sL[k + 1], a.m, a);
        c.phase = kAfterCoarse;
        ++k;
        ct[k].phase = kStart;
      }
    } else if (c.phase == kAfterCoarse) {
      if (dbl) c.rho_d = Ops<DIM, double, RP>::prolong_postsmooth(tm, L, sL[k + 1], a.m, a);
      else Scal<RP>::rho(c) = Ops<DIM, RP, RP>::prolong_postsmooth(tm, L, sL[k + 1], a.m, a);
      c.phase = kPrecondDone;
    } else if (c.phase == kPrecondDone) {
      if (a.precond == 1 && k > 0) {
        // multigrid: the level's result is M_k^-1 r_k itself
        RP* x = (RP*)L.x;
        const RP* z = (const RP*)L.z;
        for_lin((int)L.npad, [&](int e) { return z[e]; }, [&](int e, RP v) { x[e] = v; });
        tm.sync();
        c.phase = kReturn;
        continue;
      }
      const int st = dbl ? Ops<DIM, double, RP>::iterate(tm, L, c, S, a, k) : Ops<DIM, RP, RP>::iterate(tm, L, c, S, a, k);
      c.it++;
      // stall test of the level-0 PCG (every thread takes the same decision:
      // the residual norm is the same block-wide total in all of them)
      bool stalled = false;
      if (st == 0 && k == 0 && a.stall_w > 0) {
        if (c.rr_d < 0.25 * c.rr_best) {
          c.rr_best = c.rr_d;
          c.it_best = c.it;
        } else if (c.it - c.it_best >= a.stall_w) {
          if (!*a.flex && a.allow_flex) {
            *a.flex = true;
            c.it_best = c.it;
          } else {
            stalled = true;
          }
        }
      }
      if (st == 2) {
        if (threadIdx.x == 0) atomicOr(&S->status, kStBreakdown);
        c.phase = kReturn;
      } else if (st == 1) {
        c.phase = kReturn;
      } else if (stalled) {
        if (threadIdx.x == 0) atomicOr(&S->status, kStNoConv);
        c.phase = kReturn;
      } else if (c.it >= L.maxit) {
        // an inner level at its cap with the FP32 preconditioner: the outer
        // PCG goes on with the flexible beta; otherwise the solve fails
        if (k > 0 && a.allow_flex) *a.flex = true;
        else if (threadIdx.x == 0) atomicOr(&S->status, kStNoConv);
        c.phase = kReturn;
      } else {
        c.rho_old_d = c.rho_d;
        c.rho_old_f = c.rho_f;
        c.phase = kIterate;
      }
    } else {  // kReturn
      // (the multigrid preconditioner's inner levels run no PCG)
      if (a.trace && threadIdx.x == 0 && !(a.precond == 1 && k > 0)) trace_call(a, k, c.it);
      if (k == ks) break;
      --k;
    }
  }
  tm.sync();
}


// Shared-memory bytes of level L's arrays when it runs from shared memory:
// x, r, p, q in the level's vector type, z in RP, the residual t and the
// rounded right-hand side rp in RP (t shares q's and rp shares r's storage
// when the types agree), the face transmissibilities.
__host__ __device__ __forceinline__ size_t level_smem_bytes(const DevLevel& L, size_t vsz, size_t rsz, int dim) {
  const long long n = L.npad;
  size_t b = 4 * align16(n * vsz) + align16(n * rsz);
  if (vsz != rsz) b += 2 * align16(n * rsz);
  b += align16((size_t)face_count(L, 0) * rsz) + align16((size_t)face_count(L, 1) * rsz);
  if (dim == 3) b += align16((size_t)face_count(L, 2) * rsz);
  return b;
}

// Where place_levels put things in the dynamic shared memory.
struct Placement {
  int ksm;              // first level placed (kmax + 1: none)
  size_t ainv_off;      // the coarsest inverse (transposed), or SIZE_MAX
  size_t vec_off;       // the placed levels' vectors, one block ...
  size_t vec_bytes;     // ... of this many bytes, zero between solves
  size_t used;          // end of the block
};

// Place levels lo..kmax that fit (from the coarsest up) in the dynamic shared
// memory: rewrite their pointers in sL, zero their vectors (ghosts included)
// and copy their transmissibilities; then the coarsest inverse, transposed,
// when it fits as well.  Layout: transmissibilities, the inverse, the
// vectors.  The vectors come last, so that the single-pass smoother may take
// them with the free rest as its ring window while no placed level is live.
template <int DIM, typename RP>
__device__ Placement place_levels(DevLevel* sL, const DevLevel* gL, int lo, int kmax, bool top_double,
                                  unsigned char* dsm, size_t budget, const double* Ainv, int nc) {
  __shared__ Placement s_pl;
  if (threadIdx.x == 0) {
    size_t tot = 0;
    int ksm = kmax + 1;
    for (int k = kmax; k >= lo; --k) {
      const size_t vsz = (top_double && k == 0) ? sizeof(double) : sizeof(RP);
      const size_t need = level_smem_bytes(sL[k], vsz, sizeof(RP), DIM);
      if (tot + need > budget) break;
      tot += need;
      ksm = k;
    }
    size_t off = 0;
    for (int k = ksm; k <= kmax; ++k) {
      DevLevel& L = sL[k];
      for (int ax = 0; ax < DIM; ++ax) {
        const size_t nf = (size_t)face_count(L, ax);
        L.T[ax] = dsm + off;
        if (sizeof(RP) == sizeof(double)) L.T64[ax] = (const double*)(dsm + off);
        off += align16(nf * sizeof(RP));
      }
    }
    const size_t ainv = sizeof(double) * (size_t)nc * nc;
    Placement pl;
    pl.ksm = ksm;
    pl.ainv_off = SIZE_MAX;
    if (tot + align16(ainv) <= budget) {
      pl.ainv_off = off;
      off = align16(off + ainv);
    }
    pl.vec_off = off;
    for (int k = ksm; k <= kmax; ++k) {
      DevLevel& L = sL[k];
      const size_t vsz = (top_double && k == 0) ? sizeof(double) : sizeof(RP);
      void** vec[4] = {&L.x, &L.r, &L.p, &L.q};
      for (int v = 0; v < 4; ++v) {
        *vec[v] = dsm + off;
        off += align16(L.npad * vsz);
      }
      L.z = dsm + off;
      off += align16(L.npad * sizeof(RP));
      if (vsz != sizeof(RP)) {
        L.t = dsm + off;
        off += align16(L.npad * sizeof(RP));
        L.rp = dsm + off;
        off += align16(L.npad * sizeof(RP));
      } else {
        L.t = L.q;
        L.rp = L.r;
      }
    }
    pl.vec_bytes = off - pl.vec_off;
    pl.used = off;
    s_pl = pl;
  }
  __syncthreads();
  const Placement pl = s_pl;
  zero_block(dsm + pl.vec_off, pl.vec_bytes);
  for (int k = pl.ksm; k <= kmax; ++k) {
    for (int ax = 0; ax < DIM; ++ax) {
      const DevLevel& L = sL[k];
      const size_t nf = (size_t)face_count(L, ax);
      const RP* src = (const RP*)gL[k].T[ax];
      RP* dst = (RP*)L.T[ax];
      for (size_t e = threadIdx.x; e < nf; e += blockDim.x) dst[e] = __ldg(src + e);
    }
  }
  if (pl.ainv_off != SIZE_MAX) {
    double* dst = (double*)(dsm + pl.ainv_off);
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int c = e / nc, j = e - c * nc;
      dst[j * nc + c] = Ainv[e];
    }
  }
  __syncthreads();
  return pl;
}

// Single-CTA kernel.
//  mode 0: solve levels ks..kmax of problem P[0]; its r_ks (global) holds
//          b_ks and eps^2 comes from the problem state (set for the wide
//          levels); x_ks is written back to global memory.
//  mode 1: full solves of problems P[order[i]]; CTAs take the next problem
//          index from *next (problems sorted largest first).
//  mode 2: full solve of problem P[0] by CTA 0.
// A full solve copies b into r_0, sets eps^2 = tol^2 ||b||^2 / N_0 (Sec. 3),
// runs the recursion from level 0 with FP64 level-0 vectors, adds the result
// to xs, forms the true residual b - A xs in FP64 and, if that misses tol,
// runs the recursion again on it (at most 3 restarts); x = xs at the end.
template <int DIM, typename RP>
__global__ void __launch_bounds__(kSmallThreads, kSmallPerSM) k_small(const ProblemDesc* __restrict__ P,
                                                            const int* __restrict__ order, int nprob, int ks, int mode,
                                                            int* next, size_t smem_budget) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ DevLevel sL[kMaxLev];
  __shared__ double shd[64];
  __shared__ float shf[64];
  __shared__ double s_rc[kMaxCoarse];
  __shared__ double s_thrN_d[kMaxLev];
  __shared__ float s_thrN_f[kMaxLev];
  __shared__ long long s_iters[kMaxLev], s_calls[kMaxLev];
  __shared__ int s_pid;
  for (int round = 0;; ++round) {
    if (threadIdx.x == 0) s_pid = mode == 1 ? atomicAdd(next, 1) : (round == 0 && blockIdx.x == 0 ? 0 : nprob);
    __syncthreads();
    const int pid = s_pid;
    __syncthreads();
    if (pid >= nprob) break;
    const ProblemDesc& pd = P[mode == 1 ? order[pid] : 0];
    for (int e = threadIdx.x; e < pd.nlev * (int)(sizeof(DevLevel) / sizeof(int)); e += blockDim.x)
      ((int*)sL)[e] = ((const int*)pd.L)[e];
    __syncthreads();
    SolveState* S = pd.S;
    const int kmax = pd.nlev - 1;
    const bool full = mode != 0;
    const int lo = full ? 0 : ks;
    const Placement pl = place_levels<DIM, RP>(sL, pd.L, lo, kmax, full, dsm, smem_budget, pd.Ainv, pd.nc);
    RecArgs a;
    a.kmax = kmax;
    a.m = pd.m;
    a.nc = pd.nc;
    a.Ainv = pl.ainv_off != SIZE_MAX ? (const double*)(dsm + pl.ainv_off) : pd.Ainv;
    a.ainv_t = pl.ainv_off != SIZE_MAX;
    a.win_off = (unsigned)pl.vec_off;
    a.win_bytes = smem_budget > pl.vec_off ? smem_budget - pl.vec_off : 0;
    a.vec_bytes = (unsigned)pl.vec_bytes;
    a.fuse = pd.fuse != 0;
    a.fuse_width = pd.fuse_width;
    a.fuse_min_cells = pd.fuse_min_cells;
    a.splitting = pd.splitting;
    a.floor2 = S->inner_floor2;
    a.floor2_f = (float)a.floor2;
    bool flex = pd.flex0 != 0;
    a.flex = &flex;
    a.allow_flex = pd.allow_flex != 0;
    a.stall_w = pd.stall_w;
    a.precond = pd.precond;
    a.trace = pd.trace;
    a.trace_cap = pd.trace_cap;
    a.pass = 0;
    a.S = S;
    a.top_double = full;
    a.rc = s_rc;
    a.thrN_d = s_thrN_d;
    a.thrN_f = s_thrN_f;
    a.iters = s_iters;
    a.calls = s_calls;
    BlockTeam bt;
    bt.shd = shd;
    bt.shf = shf;
    bt.par = 0;
    if (!full) {
      // level ks's right-hand side into its (shared-memory) r
      const DevLevel& G = pd.L[ks];
      const RP* gr = (const RP*)G.r;
      RP* sr = (RP*)sL[ks].r;
      if (sr != gr)
        for (int c = threadIdx.x; c < (int)G.npad; c += blockDim.x) sr[c] = gr[c];
      __syncthreads();
      a.eps2 = S->eps2;
      level_consts(sL, pd.nlev, a.eps2, s_thrN_d, s_thrN_f, s_iters, s_calls);
      recursion<DIM, RP>(bt, sL, ks, a);
      flush_counts(S, pd.nlev, s_iters, s_calls);
      // an inner level at its cap switches the graph's level-0 PCG to the
      // flexible beta
      if (threadIdx.x == 0 && flex) S->flex = 1;
      RP* gx = (RP*)G.x;
      const RP* sx = (const RP*)sL[ks].x;
      if (sx != gx)
        for (int c = threadIdx.x; c < (int)G.npad; c += blockDim.x) gx[c] = sx[c];
      __syncthreads();
      continue;
    }
    const DevLevel& L0 = sL[0];
    const DevLevel& G0 = pd.L[0];
    double* r0 = (double*)L0.r;
    const double* x0 = (const double*)L0.x;
    double* xs = pd.xs;
    double bbl = 0.0;
    for_cells<DIM>(team_map(L0.nx), L0, [&](int i, const Row& rw) {
      const double v = pd.b[i + L0.nx * (rw.j + L0.ny * rw.k)];
      r0[rw.pc + i] = v;
      bbl += v * v;
    });
    for (int c = threadIdx.x; c < (int)L0.npad; c += blockDim.x) xs[c] = 0.0;
    const double bb = bt.sum<double>(bbl);
    const double eps2 = pd.tol * pd.tol * (bb / (double)L0.n);
    if (threadIdx.x == 0) {
      S->bb0 = bb;
      S->tau2 = pd.tol * pd.tol;
      S->eps2 = eps2;
      S->status = isfinite(bb) ? 0 : kStNanInf;
      for (int k = 0; k < pd.nlev; ++k) {
        S->lv[k].iters = 0;
        S->lv[k].calls = 0;
        S->lv[k].rr = 0.0;
      }
      S->lv[0].rr = bb;
      S->rr_true = bb;
      S->flex = pd.flex0;
    }
    __syncthreads();
    a.eps2 = eps2;
    level_consts(sL, pd.nlev, eps2, s_thrN_d, s_thrN_f, s_iters, s_calls);
    if (bb > 0.0 && isfinite(bb)) {
      for (int pass = 0; pass < 4; ++pass) {
        a.pass = pass;
        recursion<DIM, RP>(bt, sL, 0, a);
        for (int c = threadIdx.x; c < (int)L0.npad; c += blockDim.x) xs[c] += x0[c];
        __syncthreads();
        double rl = 0.0;
        for_cells<DIM>(team_map(L0.nx), L0, [&](int i, const Row& rw) {
          const double v = pd.b[i + L0.nx * (rw.j + L0.ny * rw.k)] -
                           apply_value<DIM, double, double>(G0, G0.T64[0], G0.T64[1], DIM == 3 ? G0.T64[2] : nullptr, xs,
                                                            i, rw);
          r0[rw.pc + i] = v;
          rl += v * v;
        });
        const double rt = bt.sum<double>(rl);
        if (threadIdx.x == 0) S->rr_true = rt;
        __syncthreads();
        if (S->status != 0 || rt < pd.tol * pd.tol * bb) break;
      }
    }
    flush_counts(S, pd.nlev, s_iters, s_calls);
    if (threadIdx.x == 0) S->flex = flex ? 1 : 0;
    for_cells<DIM>(team_map(L0.nx), L0, [&](int i, const Row& rw) {
      pd.x[i + L0.nx * (rw.j + L0.ny * rw.k)] = xs[rw.pc + i];
    });
    __syncthreads();
  }
}

// ===========================================================================
// Multi-CTA level kernels (wide levels, sequenced by the graph)
// ===========================================================================

// Reduction across the CTAs of one launch: each CTA writes its partial, the
// last CTA to arrive (ticket) sums the partials in index order and calls fin
// with the total.  Deterministic for a given launch shape.
template <typename T, class Fin>
__device__ void grid_total(T v, double* partials, unsigned int* ticket, Fin fin) {
  __shared__ T sh[32];
  __shared__ bool last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nt = blockDim.x * blockDim.y;
  const unsigned nb = gridDim.x * gridDim.y, bid = blockIdx.x + gridDim.x * blockIdx.y;
  v = warp_sum_t<T>(v);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    T s = 0;
    for (int w = 0; w < (nt >> 5); ++w) s += sh[w];
    partials[bid] = (double)s;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = t == nb - 1;
  }
  __syncthreads();
  if (last && tid < 32) {
    __threadfence();
    double s = 0.0;
    for (unsigned i = tid; i < nb; i += 32) s += __ldcg(partials + i);
    s = warp_sum(s);
    if (tid == 0) {
      *ticket = 0u;
      fin(s);
    }
  }
}

// grid_total for two values at once (partials holds 2 per CTA).
template <typename T, class Fin>
__device__ void grid_total2(T v0, T v1, double* partials, unsigned int* ticket, Fin fin) {
  __shared__ T sh[2][32];
  __shared__ bool last;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nt = blockDim.x * blockDim.y;
  const unsigned nb = gridDim.x * gridDim.y, bid = blockIdx.x + gridDim.x * blockIdx.y;
  v0 = warp_sum_t<T>(v0);
  v1 = warp_sum_t<T>(v1);
  if ((tid & 31) == 0) {
    sh[0][tid >> 5] = v0;
    sh[1][tid >> 5] = v1;
  }
  __syncthreads();
  if (tid == 0) {
    T s0 = 0, s1 = 0;
    for (int w = 0; w < (nt >> 5); ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
    }
    partials[2 * bid] = (double)s0;
    partials[2 * bid + 1] = (double)s1;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = t == nb - 1;
  }
  __syncthreads();
  if (last && tid < 32) {
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (unsigned i = tid; i < nb; i += 32) {
      s0 += __ldcg(partials + 2 * i);
      s1 += __ldcg(partials + 2 * i + 1);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (tid == 0) {
      *ticket = 0u;
      fin(s0, s1);
    }
  }
}

// rho of a post-smoothed level and the CG direction factor beta: rho /
// rho_old, or on level 0 with the flexible beta in use (rho - r.z_old) /
// rho_old once the previous update has formed r.z_old.
__device__ __forceinline__ void set_rho_beta(LevelState& ls, int k, const SolveState* S, double rho) {
  ls.rho = rho;
  if (ls.it == 0) ls.beta = 0.0;
  else if (k == 0 && S->flex && ls.gamma_ok) ls.beta = (rho - ls.gamma) / ls.rho_old;
  else ls.beta = rho / ls.rho_old;
  ls.beta_f = (float)ls.beta;
}

__device__ __forceinline__ long long lin_tid() {
  return (long long)(blockIdx.x + gridDim.x * blockIdx.y) * (blockDim.x * blockDim.y) + threadIdx.x +
         blockDim.x * threadIdx.y;
}
__device__ __forceinline__ long long lin_stride() {
  return (long long)gridDim.x * gridDim.y * blockDim.x * blockDim.y;
}

// PCG entry on a wide level: x = 0 (level 0: r = b0), ||b_k||^2, threshold,
// counters, and the WHILE condition of the level's loop.
template <typename V>
__global__ void k_init(DevLevel L, int k, SolveState* S, const double* b0, double* partials,
                       cudaGraphConditionalHandle hcond, int in_graph = 1) {
  V* x = (V*)L.x;
  V* r = (V*)L.r;
  V acc = 0;
  for (long long c = lin_tid(); c < L.npad; c += lin_stride()) {
    x[c] = 0;
    V v;
    if (b0) {
      v = (V)b0[c];
      r[c] = v;
    } else {
      v = r[c];
    }
    acc += v * v;
  }
  grid_total(acc, partials, &S->ticket[k], [&](double bb) {
    LevelState& ls = S->lv[k];
    ls.bb = bb;
    double thr = L.fk * S->eps2;
    if (k > 0 && S->inner_floor2 > 0.0) thr = fmax(thr, S->inner_floor2 * bb / (double)L.n);
    ls.thr = thr;
    ls.it = 0;
    ls.calls++;
    ls.rho_old = 0.0;
    ls.rr = bb;
    ls.rr_best = bb;
    ls.it_best = 0;
    ls.gamma_ok = 0;
    ls.stop = !(bb > 0.0) || !isfinite(bb);
    if (in_graph) cudaGraphSetConditional(hcond, ls.stop ? 0u : 1u);
  });
}

template <typename V>
__device__ __forceinline__ V beta_of(const LevelState& ls);
template <>
__device__ __forceinline__ double beta_of<double>(const LevelState& ls) {
  return ls.beta;
}
template <>
__device__ __forceinline__ float beta_of<float>(const LevelState& ls) {
  return ls.beta_f;
}
template <typename V>
__device__ __forceinline__ V alpha_of(const LevelState& ls);
template <>
__device__ __forceinline__ double alpha_of<double>(const LevelState& ls) {
  return ls.alpha;
}
template <>
__device__ __forceinline__ float alpha_of<float>(const LevelState& ls) {
  return ls.alpha_f;
}

// One red-black half-sweep over a wide level (see t_sweep).  With `zero`
// the iterate starts from x = 0 and, when the level's vectors are wider than
// the smoother type, r is rounded into rp on the way.
template <int DIM, typename RP, typename V>
__global__ void k_sweep(DevLevel L, int colour, int zero) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const V* r = (const V*)L.r;
  RP* rp = (RP*)L.rp;
  RP* z = (RP*)L.z;
  // FP64: the reciprocal diagonals k_inv_diag wrote into t for this smoothing
  const RP* inv = sizeof(RP) == sizeof(double) ? (const RP*)L.t : nullptr;
  if (zero) {
    for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
      const int pc = rw.pc + i;
      RP rhs;
      if (sizeof(V) != sizeof(RP)) {
        rhs = (RP)r[pc];
        rp[pc] = rhs;
      } else {
        rhs = rp[pc];
      }
      z[pc] = ((i + rw.j + rw.k) & 1) == colour
                  ? (inv ? rhs * inv[pc] : quot<RP>(rhs, diag_of<DIM, RP>(L, Tx, Ty, Tz, i, rw)))
                  : (RP)0;
    });
  } else {
    for_colour<DIM>(grid_map(), L, colour, [&](int i, int, const Row& rw) {
      if (i < L.nx)
        z[rw.pc + i] = inv ? gs_sum<DIM, RP>(L, Tx, Ty, Tz, rp[rw.pc + i], z, i, rw) * inv[rw.pc + i]
                           : gs_value<DIM, RP, RP>(L, Tx, Ty, Tz, rp[rw.pc + i], z, i, rw);
    });
  }
}

// The cells' reciprocal diagonals 1/D into the t buffer (free while the level
// smooths), for the FP64 half-sweeps of one smoothing.
template <int DIM, typename RP>
__global__ void k_inv_diag(DevLevel L) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  RP* w = (RP*)L.t;
  for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
    w[rw.pc + i] = (RP)1 / diag_of<DIM, RP>(L, Tx, Ty, Tz, i, rw);
  });
}

// The last red half-sweep of post-smoothing, with rho = r . z over all cells
// and the CG direction factor beta = rho / rho_old.
template <int DIM, typename RP, typename V>
__global__ void k_sweep_rho(DevLevel L, int k, SolveState* S, double* partials) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const V* r = (const V*)L.r;
  const RP* rp = (const RP*)L.rp;
  RP* z = (RP*)L.z;
  const RP* inv = sizeof(RP) == sizeof(double) ? (const RP*)L.t : nullptr;
  V acc = 0;
  for_colour<DIM>(grid_map(), L, 0, [&](int i, int i2, const Row& rw) {
    if (i2 < L.nx) acc += r[rw.pc + i2] * (V)z[rw.pc + i2];
    if (i < L.nx) {
      const RP v = inv ? gs_sum<DIM, RP>(L, Tx, Ty, Tz, rp[rw.pc + i], z, i, rw) * inv[rw.pc + i]
                       : gs_value<DIM, RP, RP>(L, Tx, Ty, Tz, rp[rw.pc + i], z, i, rw);
      acc += r[rw.pc + i] * (V)v;
      z[rw.pc + i] = v;
    }
  });
  grid_total(acc, partials, &S->ticket[k], [&](double rho) { set_rho_beta(S->lv[k], k, S, rho); });
}

template <int DIM, typename RP>
__global__ void k_residual(DevLevel L) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const RP* rp = (const RP*)L.rp;
  const RP* z = (const RP*)L.z;
  RP* t = (RP*)L.t;
  for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
    t[rw.pc + i] = rp[rw.pc + i] - apply_value<DIM, RP, RP>(L, Tx, Ty, Tz, z, i, rw);
  });
}

// r_{k+1} = R t on a 2D level, by tiles of kRestrictTI x TJ coarse cells: the
// CTA copies the tile's fine window of t into shared memory (coalesced rows),
// forms for every fine row the x-sums of each coarse column, then the
// y-sums: the products and their order are those of restrict_value, so the
// result is the gather's, bit for bit, with every fine value read once.
template <typename R>
__global__ void k_restrict2d(DevLevel L, DevLevel C, int TJ, int FXM, int FYM) {
  extern __shared__ __align__(16) unsigned char rsm[];
  R* tile = (R*)rsm;           // FYM rows of FXM
  R* hx = tile + FYM * FXM;    // FYM rows of kRestrictTI x-sums
  const int I0 = blockIdx.x * kRestrictTI, J0 = blockIdx.y * TJ;
  const int nI = min(kRestrictTI, C.nx - I0), nJ = min(TJ, C.ny - J0);
  const int fx0 = __ldg(L.lo[0] + I0), fx1 = __ldg(L.hi[0] + I0 + nI - 1);
  const int fy0 = __ldg(L.lo[1] + J0), fy1 = __ldg(L.hi[1] + J0 + nJ - 1);
  const int FX = fx1 - fx0 + 1, FY = fy1 - fy0 + 1;
  const R* t = (const R*)L.t + (int)L.off + L.px * fy0 + fx0;
  // warps walk rows, lanes columns (kRestrictTI = 32 coarse columns per tile)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < FY; r += nw)
    for (int c = lane; c < FX; c += 32) tile[r * FXM + c] = t[L.px * r + c];
  __syncthreads();
  const R* rwx = (const R*)L.rw[0];
  const R* rwy = (const R*)L.rw[1];
  if (lane < nI) {
    const int I = I0 + lane;
    const int lo = __ldg(L.lo[0] + I), hi = __ldg(L.hi[0] + I);
    const R* w = rwx + I * L.W[0] - lo;
    for (int r = warp; r < FY; r += nw) {
      const R* row = tile + r * FXM - fx0;
      R acc = 0;
      for (int ii = lo; ii <= hi; ++ii) acc += __ldg(w + ii) * row[ii];
      hx[r * kRestrictTI + lane] = acc;
    }
  }
  __syncthreads();
  R* rc = (R*)C.r + (int)C.off;
  if (lane < nI)
    for (int jl = warp; jl < nJ; jl += nw) {
      const int J = J0 + jl;
      const int lo = __ldg(L.lo[1] + J), hi = __ldg(L.hi[1] + J);
      const R* w = rwy + J * L.W[1] - lo;
      R acc = 0;
      for (int jj = lo; jj <= hi; ++jj) acc += __ldg(w + jj) * hx[(jj - fy0) * kRestrictTI + lane];
      rc[C.px * J + I0 + lane] = acc;
    }
}

template <int DIM, typename RP>
__global__ void k_restrict(DevLevel L, DevLevel C) {
  const RP* t = (const RP*)L.t;
  RP* rc = (RP*)C.r;
  for_cells<DIM>(grid_map(), C,
                 [&](int i, const Row& rw) { rc[rw.pc + i] = restrict_value<DIM, RP>(L, t, i, rw.j, rw.k); });
}

// z += E x_c on the black cells (see Ops::prolong_postsmooth)
template <int DIM, typename RP>
__global__ void k_prolong_black(DevLevel L, DevLevel C) {
  const RP* xc = (const RP*)C.x;
  RP* z = (RP*)L.z;
  for_colour<DIM>(grid_map(), L, 1, [&](int i, int, const Row& rw) {
    if (i < L.nx) z[rw.pc + i] += prolong_value<DIM, RP>(L, C, xc, i, rw.j, rw.k);
  });
}

// Modified Jacobi on a wide level (see t_jacobi): phase 0 (from zero)
// z = rp / 2D, rounding r into rp when the vector types differ; phase 1
// t = A z; phase 2 z += (rp - t) / 2D.
template <int DIM, typename RP, typename V>
__global__ void k_jacobi(DevLevel L, int phase) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const V* r = (const V*)L.r;
  RP* rp = (RP*)L.rp;
  RP* z = (RP*)L.z;
  RP* t = (RP*)L.t;
  for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
    const int pc = rw.pc + i;
    if (phase == 1) {
      t[pc] = apply_value<DIM, RP, RP>(L, Tx, Ty, Tz, z, i, rw);
      return;
    }
    const RP d = diag_of<DIM, RP>(L, Tx, Ty, Tz, i, rw);
    if (phase == 0) {
      RP rhs;
      if (sizeof(V) != sizeof(RP)) {
        rhs = (RP)r[pc];
        rp[pc] = rhs;
      } else {
        rhs = rp[pc];
      }
      z[pc] = quot<RP>(rhs, d + d);
    } else {
      z[pc] = z[pc] + quot<RP>(rp[pc] - t[pc], d + d);
    }
  });
}

// The last post-smoothing Jacobi update with rho = r . z and beta (as
// k_sweep_rho).
template <int DIM, typename RP, typename V>
__global__ void k_jacobi_rho(DevLevel L, int k, SolveState* S, double* partials) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const V* r = (const V*)L.r;
  const RP* rp = (const RP*)L.rp;
  const RP* t = (const RP*)L.t;
  RP* z = (RP*)L.z;
  V acc = 0;
  for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
    const int pc = rw.pc + i;
    const RP d = diag_of<DIM, RP>(L, Tx, Ty, Tz, i, rw);
    const RP v = z[pc] + quot<RP>(rp[pc] - t[pc], d + d);
    acc += r[pc] * (V)v;
    z[pc] = v;
  });
  grid_total(acc, partials, &S->ticket[k], [&](double rho) { set_rho_beta(S->lv[k], k, S, rho); });
}

// z += E x_c on every cell (the Jacobi smoother reads them all)
template <int DIM, typename RP>
__global__ void k_prolong_all(DevLevel L, DevLevel C) {
  const RP* xc = (const RP*)C.x;
  RP* z = (RP*)L.z;
  for_cells<DIM>(grid_map(), L,
                 [&](int i, const Row& rw) { z[rw.pc + i] += prolong_value<DIM, RP>(L, C, xc, i, rw.j, rw.k); });
}

// p = z (first iteration) or z + beta p
template <typename V, typename RP>
__global__ void k_direction(DevLevel L, int k, SolveState* S) {
  const LevelState& ls = S->lv[k];
  if (ls.stop) return;
  const bool first = ls.it == 0;
  const V beta = beta_of<V>(ls);
  V* p = (V*)L.p;
  const RP* z = (const RP*)L.z;
  const int n = (int)L.npad;
  for (int c = (int)lin_tid(); c < n; c += (int)lin_stride()) p[c] = first ? (V)z[c] : (V)z[c] + beta * p[c];
}

// q = A p, pq = p . q, alpha = rho / pq; breakdown check
template <int DIM, typename V>
__global__ void k_apply_dot(DevLevel L, int k, SolveState* S, double* partials) {
  if (S->lv[k].stop) return;
  const V *Tx = Tvec<V>(L, 0), *Ty = Tvec<V>(L, 1), *Tz = DIM == 3 ? Tvec<V>(L, 2) : nullptr;
  const V* p = (const V*)L.p;
  V* q = (V*)L.q;
  V acc = 0;
  for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
    const V v = apply_value<DIM, V, V>(L, Tx, Ty, Tz, p, i, rw);
    acc += p[rw.pc + i] * v;
    q[rw.pc + i] = v;
  });
  grid_total(acc, partials, &S->ticket[k], [&](double pq) {
    LevelState& ls = S->lv[k];
    ls.pq = pq;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(ls.rho)) {
      ls.stop = 1;
      atomicOr(&S->status, kStBreakdown);
    }
    ls.alpha = ls.rho / pq;
    ls.alpha_f = (float)ls.alpha;
  });
}

// x += alpha p, r -= alpha q, ||r||^2, the level test of Sec. 3 and the
// WHILE condition of the level's loop.  On level 0 with the flexible beta in
// use the pass also forms r_new . z (z still holds this iteration's
// preconditioned residual); the stall test may switch the flexible beta on
// or end the loop.
template <typename V, typename RP>
__global__ void k_update(DevLevel L, int k, SolveState* S, double* partials, cudaGraphConditionalHandle hcond,
                         int in_graph = 1) {
  const LevelState& ls = S->lv[k];
  if (ls.stop) {
    if (lin_tid() == 0 && in_graph) cudaGraphSetConditional(hcond, 0u);
    return;
  }
  const V alpha = alpha_of<V>(ls);
  V* x = (V*)L.x;
  V* r = (V*)L.r;
  const V* p = (const V*)L.p;
  const V* q = (const V*)L.q;
  const RP* z = (const RP*)L.z;
  const bool gam = k == 0 && S->flex;
  V acc = 0, acc2 = 0;
  const int n = (int)L.npad;
  for (int c = (int)lin_tid(); c < n; c += (int)lin_stride()) {
    const V xv = x[c] + alpha * p[c];
    const V rv = r[c] - alpha * q[c];
    acc += rv * rv;
    if (gam) acc2 += rv * (V)z[c];
    x[c] = xv;
    r[c] = rv;
  }
  auto fin = [&](double rr, double gamma) {
    LevelState& w = S->lv[k];
    w.rr = rr;
    w.iters++;
    w.it++;
    w.gamma = gamma;
    w.gamma_ok = gam;
    bool go = true;
    if (rr / (double)L.n < w.thr) {
      go = false;
    } else if (w.it >= L.maxit) {
      // an inner level at its cap with the FP32 preconditioner switches the
      // level-0 PCG to the flexible beta; otherwise the solve fails
      if (k > 0 && S->allow_flex) S->flex = 1;
      else atomicOr(&S->status, kStNoConv);
      go = false;
    } else if (k == 0 && S->stall_w > 0) {
      if (rr < 0.25 * w.rr_best) {
        w.rr_best = rr;
        w.it_best = w.it;
      } else if (w.it - w.it_best >= S->stall_w) {
        if (!S->flex && S->allow_flex) {
          S->flex = 1;
          w.it_best = w.it;
        } else {
          atomicOr(&S->status, kStNoConv);
          go = false;
        }
      }
    }
    w.rho_old = w.rho;
    if (!go) w.stop = 1;
    if (in_graph) cudaGraphSetConditional(hcond, go ? 1u : 0u);
  };
  if (gam) grid_total2(acc, acc2, partials, &S->ticket[k], fin);
  else grid_total(acc, partials, &S->ticket[k], [&](double rr) { fin(rr, 0.0); });
}

// Before a solve: b0 = b (padded), ||b||^2, eps^2 = tol^2 ||b||^2 / N_0
// (Sec. 3), counters cleared.  xs is zeroed by the caller.
template <int DIM>
__global__ void k_prepare(DevLevel L0, const double* b, double* b0, double tol, SolveState* S, int nlev,
                          double* partials, int flex0, int allow_flex, int stall_w) {
  double acc = 0.0;
  for_cells<DIM>(grid_map(), L0, [&](int i, const Row& rw) {
    const int pc = rw.pc + i;
    const int j = rw.j, k = rw.k;
    const double v = b[i + (long long)L0.nx * (j + (long long)L0.ny * k)];
    b0[pc] = v;
    acc += v * v;
  });
  grid_total(acc, partials, &S->ticket[kMaxLev - 1], [&](double bb) {
    S->bb0 = bb;
    S->tau2 = tol * tol;
    S->eps2 = tol * tol * (bb / (double)L0.n);
    S->status = isfinite(bb) ? 0 : kStNanInf;
    S->rr_true = bb;
    S->flex = flex0;
    S->allow_flex = allow_flex;
    S->stall_w = stall_w;
    for (int k = 0; k < nlev; ++k) {
      S->lv[k].iters = 0;
      S->lv[k].calls = 0;
      S->lv[k].stop = 0;
      S->lv[k].rr = 0.0;
    }
  });
}

// After the level-0 PCG: xs += x_0.
__global__ void k_accumulate(const double* __restrict__ x0, double* __restrict__ xs, long long n) {
  for (long long c = lin_tid(); c < n; c += lin_stride()) xs[c] += x0[c];
}

// True residual b - A xs in FP64 into b0 (the right-hand side of a restart).
template <int DIM>
__global__ void k_true_residual(DevLevel L0, const double* b, double* b0, const double* xs, SolveState* S,
                                double* partials) {
  const double *Tx = L0.T64[0], *Ty = L0.T64[1], *Tz = DIM == 3 ? L0.T64[2] : nullptr;
  double acc = 0.0;
  for_cells<DIM>(grid_map(), L0, [&](int i, const Row& rw) {
    const int pc = rw.pc + i;
    const int j = rw.j, k = rw.k;
    const double v = b[i + (long long)L0.nx * (j + (long long)L0.ny * k)] -
                     apply_value<DIM, double, double>(L0, Tx, Ty, Tz, xs, i, rw);
    b0[pc] = v;
    acc += v * v;
  });
  grid_total(acc, partials, &S->ticket[kMaxLev - 1], [&](double rt) { S->rr_true = rt; });
}

template <int DIM>
__global__ void k_copy_out(DevLevel L0, const double* xs, double* x) {
  for_cells<DIM>(grid_map(), L0, [&](int i, const Row& rw) {
    const int pc = rw.pc + i;
    const int j = rw.j, k = rw.k;
    x[i + (long long)L0.nx * (j + (long long)L0.ny * k)] = xs[pc];
  });
}

// ===========================================================================
// Host side
// ===========================================================================
struct Launch {
  dim3 grid, block;
};

// 2D launch over rows of `width` columns (width = pair positions or cells):
// a power-of-two block width, 256 threads per block, at most gmax blocks.
Launch rows_launch(int width, long long rows, int gmax) {
  int bx = 1;
  while (bx < width && bx < kThreads) bx <<= 1;
  const int by = kThreads / bx;
  Launch l;
  l.block = dim3(bx, by, 1);
  long long gx = (width + bx - 1) / bx;
  long long gy = (rows + by - 1) / by;
  if (gx > gmax) gx = gmax;
  long long cap = std::max(1LL, (long long)gmax / gx);
  if (gy > cap) gy = cap;
  if (gy > 65535) gy = 65535;
  l.grid = dim3((unsigned)gx, (unsigned)std::max(1LL, gy), 1);
  return l;
}

Launch lin_launch(long long n, int gmax) {
  Launch l;
  l.block = dim3(kThreads, 1, 1);
  long long g = (n + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  if (g > gmax) g = gmax;
  l.grid = dim3((unsigned)g, 1, 1);
  return l;
}

Launch cells_launch(const DevLevel& L, int gmax) { return rows_launch(L.nx, (long long)L.ny * L.nz, gmax); }
Launch pairs_launch(const DevLevel& L, int gmax) { return rows_launch((L.nx + 1) >> 1, (long long)L.ny * L.nz, gmax); }

size_t levels_smem(const msrcg_hier* h, int lo, bool top_double);

struct Emit {
  msrcg_hier* h;
  cudaStream_t cs[kMaxLev + 2];
  int err = 0;
};

template <int DIM, typename RP>
void emit_pcg(Emit& E, int k, cudaStream_t s);

// r_{k+1} = R t of a wide level: by tiles (2D, when the build sized one),
// else the per-cell gather
template <int DIM, typename RP>
void launch_restrict(const msrcg_hier* h, int k, int gmax, cudaStream_t s) {
  const DevLevel& L = h->hL[k];
  const DevLevel& C = h->hL[k + 1];
  if (DIM == 2 && h->rfx[k] > 0) {
    const int tj = h->rtj;
    const dim3 grid((C.nx + kRestrictTI - 1) / kRestrictTI, (C.ny + tj - 1) / tj);
    const size_t smem = sizeof(RP) * ((size_t)h->rfx[k] * h->rfy[k] + (size_t)h->rfy[k] * kRestrictTI);
    k_restrict2d<RP><<<grid, 256, smem, s>>>(L, C, tj, h->rfx[k], h->rfy[k]);
  } else {
    const Launch lcc = cells_launch(C, gmax);
    k_restrict<DIM, RP><<<lcc.grid, lcc.block, 0, s>>>(L, C);
  }
}

template <int DIM, typename RP, typename V>
void emit_smooth(const DevLevel& L, int m, bool from_zero, bool with_rho, int k, msrcg_hier* h, int gmax, cudaStream_t s) {
  const Launch lp = pairs_launch(L, gmax), lc = cells_launch(L, gmax);
  if (h->o.splitting == 1) {
    int s0 = 0;
    if (from_zero) {
      k_jacobi<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, 0);
      s0 = 1;
    }
    for (int i = s0; i < m; ++i) {
      k_jacobi<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, 1);
      if (with_rho && i == m - 1)
        k_jacobi_rho<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, k, h->dS, h->partials + (size_t)k * kMaxGrid);
      else
        k_jacobi<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, 2);
    }
    return;
  }
  if (sizeof(RP) == sizeof(double)) k_inv_diag<DIM, RP><<<lc.grid, lc.block, 0, s>>>(L);
  if (from_zero) k_sweep<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, 0, 1);
  else k_sweep<DIM, RP, V><<<lp.grid, lp.block, 0, s>>>(L, 0, 0);
  for (int i = 0; i < m; ++i) {
    k_sweep<DIM, RP, V><<<lp.grid, lp.block, 0, s>>>(L, 1, 0);
    if (with_rho && i == m - 1)
      k_sweep_rho<DIM, RP, V><<<lp.grid, lp.block, 0, s>>>(L, k, h->dS, h->partials + (size_t)k * kMaxGrid);
    else
      k_sweep<DIM, RP, V><<<lp.grid, lp.block, 0, s>>>(L, 0, 0);
  }
}

template <int DIM, typename RP>
void emit_precond(Emit& E, int k, cudaStream_t s) {
  msrcg_hier* h = E.h;
  const DevLevel& L = h->hL[k];
  const DevLevel& C = h->hL[k + 1];
  const int gmax = std::min(h->sms * 8, kMaxGrid);
  const Launch lc = cells_launch(L, gmax), lp = pairs_launch(L, gmax);
  const int m = h->o.m;
  // pre-smoothing from zero, residual, restriction
  if (k == 0) {
    emit_smooth<DIM, RP, double>(L, m, true, false, k, h, gmax, s);
    k_residual<DIM, RP><<<lc.grid, lc.block, 0, s>>>(L);
  } else {
    emit_smooth<DIM, RP, RP>(L, m, true, false, k, h, gmax, s);
    k_residual<DIM, RP><<<lc.grid, lc.block, 0, s>>>(L);
  }
  launch_restrict<DIM, RP>(h, k, gmax, s);
  // coarse solve: A_c^-1 applied by the PCG one level down (Sec. 2.3)
  if (k + 1 < h->ks) emit_pcg<DIM, RP>(E, k + 1, s);
  else k_small<DIM, RP><<<1, kSmallThreads, h->sub_smem, s>>>(h->dP, nullptr, 1, k + 1, 0, nullptr, h->sub_smem);
  // prolongation (black cells; every cell for the Jacobi smoother) and
  // post-smoothing with rho = r . z
  if (h->o.splitting == 1) k_prolong_all<DIM, RP><<<lc.grid, lc.block, 0, s>>>(L, C);
  else k_prolong_black<DIM, RP><<<lp.grid, lp.block, 0, s>>>(L, C);
  if (k == 0) emit_smooth<DIM, RP, double>(L, m, false, true, k, h, gmax, s);
  else emit_smooth<DIM, RP, RP>(L, m, false, true, k, h, gmax, s);
}

template <int DIM, typename RP>
void emit_pcg(Emit& E, int k, cudaStream_t s) {
  msrcg_hier* h = E.h;
  const DevLevel& L = h->hL[k];
  const int gmax = std::min(h->sms * 8, kMaxGrid);
  const Launch ll = lin_launch(L.npad, gmax), lc = cells_launch(L, gmax);
  // the update may reduce two values: two partials per CTA in the level's share
  const Launch lu = lin_launch(L.npad, std::min(gmax, kMaxGrid / 2));
  double* part = h->partials + (size_t)k * kMaxGrid;
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg;
  const cudaGraphNode_t* deps;
  const cudaGraphEdgeData* edata;
  size_t ndeps;
  if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, &edata, &ndeps) != cudaSuccess ||
      cst != cudaStreamCaptureStatusActive) {
    E.err = 1;
    return;
  }
  cudaGraphConditionalHandle hc;
  if (cudaGraphConditionalHandleCreate(&hc, cg, 0, 0) != cudaSuccess) {
    E.err = 2;
    return;
  }
  if (k == 0) k_init<double><<<ll.grid, ll.block, 0, s>>>(L, k, h->dS, h->b0, part, hc);
  else k_init<RP><<<ll.grid, ll.block, 0, s>>>(L, k, h->dS, nullptr, part, hc);
  if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, &edata, &ndeps) != cudaSuccess) {
    E.err = 3;
    return;
  }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hc;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, cg, deps, edata, ndeps, &np) != cudaSuccess) {
    E.err = 4;
    return;
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) {
    E.err = 5;
    return;
  }
  cudaStream_t b = E.cs[k + 1];
  if (cudaStreamBeginCaptureToGraph(b, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    E.err = 6;
    return;
  }
  emit_precond<DIM, RP>(E, k, b);
  if (k == 0) {
    k_direction<double, RP><<<ll.grid, ll.block, 0, b>>>(L, k, h->dS);
    k_apply_dot<DIM, double><<<lc.grid, lc.block, 0, b>>>(L, k, h->dS, part);
    k_update<double, RP><<<lu.grid, lu.block, 0, b>>>(L, k, h->dS, part, hc);
  } else {
    k_direction<RP, RP><<<ll.grid, ll.block, 0, b>>>(L, k, h->dS);
    k_apply_dot<DIM, RP><<<lc.grid, lc.block, 0, b>>>(L, k, h->dS, part);
    k_update<RP, RP><<<lu.grid, lu.block, 0, b>>>(L, k, h->dS, part, hc);
  }
  cudaGraph_t out;
  if (cudaStreamEndCapture(b, &out) != cudaSuccess) E.err = 7;
}

template <int DIM, typename RP>
int build_graph_t(msrcg_hier* h) {
  Emit E;
  E.h = h;
  for (int i = 0; i < kMaxLev + 2; ++i) {
    if (cudaStreamCreateWithFlags(&E.cs[i], cudaStreamNonBlocking) != cudaSuccess) return MSRCG_ECUDA;
  }
  cudaGraph_t g;
  int rc = MSRCG_OK;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) rc = MSRCG_ECUDA;
  if (!rc && cudaStreamBeginCaptureToGraph(E.cs[0], g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    rc = MSRCG_ECUDA;
  if (!rc) {
    emit_pcg<DIM, RP>(E, 0, E.cs[0]);
    cudaGraph_t out;
    if (cudaStreamEndCapture(E.cs[0], &out) != cudaSuccess || E.err) rc = MSRCG_ECUDA;
  }
  if (!rc && cudaGraphInstantiate(&h->gexec, g, 0) != cudaSuccess) rc = MSRCG_ECUDA;
  if (!rc) h->graph = g;
  else if (g) cudaGraphDestroy(g);
  for (int i = 0; i < kMaxLev + 2; ++i) cudaStreamDestroy(E.cs[i]);
  if (rc && getenv("MSRCG_DEBUG"))
    fprintf(stderr, "msrcg: graph build failed (step %d): %s\n", E.err, cudaGetErrorString(cudaGetLastError()));
  (void)cudaGetLastError();
  return rc;
}

int build_graph(msrcg_hier* h) {
  const bool f32 = h->o.precision == 1;
  h->sub_smem = levels_smem(h, h->ks, false);
  if (h->dim == 2) return f32 ? build_graph_t<2, float>(h) : build_graph_t<2, double>(h);
  return f32 ? build_graph_t<3, float>(h) : build_graph_t<3, double>(h);
}

// Largest dynamic shared memory a single-CTA launch may use, after the
// kernel's static shared memory; sets the attribute the launch needs.  The
// attribute belongs to the current device, so both are kept per device
// (under a lock: host threads may launch on several devices at once).
constexpr int kMaxDevs = 64;
template <int DIM, typename RP>
size_t small_smem_limit() {
  static std::mutex mu;
  static size_t lims[kMaxDevs] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevs) {
    (void)cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!lims[dev]) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, k_small<DIM, RP>);
    if (kSmallPerSM > 1) {
      int per_sm = 0;
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      optin = std::min(optin, per_sm / kSmallPerSM - 1024);
    }
    size_t l = (size_t)optin > fa.sharedSizeBytes + 1024 ? (size_t)optin - fa.sharedSizeBytes - 1024 : 0;
    cudaFuncSetAttribute(k_small<DIM, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l);
    (void)cudaGetLastError();
    lims[dev] = l;
  }
  return lims[dev];
}

size_t small_smem_limit_any(int dim, bool f32) {
  if (dim == 2) return f32 ? small_smem_limit<2, float>() : small_smem_limit<2, double>();
  return f32 ? small_smem_limit<3, float>() : small_smem_limit<3, double>();
}

template <int DIM, typename RP>
void launch_small(const ProblemDesc* P, const int* order, int nprob, int ks, int mode, int* next, int grid,
                  size_t smem, cudaStream_t s) {
  k_small<DIM, RP><<<grid, kSmallThreads, smem, s>>>(P, order, nprob, ks, mode, next, smem);
}

void launch_small_any(int dim, bool f32, const ProblemDesc* P, const int* order, int nprob, int ks, int mode, int* next,
                      int grid, size_t smem, cudaStream_t s) {
  if (dim == 2) {
    if (f32) launch_small<2, float>(P, order, nprob, ks, mode, next, grid, smem, s);
    else launch_small<2, double>(P, order, nprob, ks, mode, next, grid, smem, s);
  } else {
    if (f32) launch_small<3, float>(P, order, nprob, ks, mode, next, grid, smem, s);
    else launch_small<3, double>(P, order, nprob, ks, mode, next, grid, smem, s);
  }
}

// Whether the batched solver may smooth HBM-resident levels in one pass.
// Post-smoothing prefetches the r rows its last stage reads kFuseAhead steps
// ahead, starting at step 0 with rows 2 kFuseAhead - 3(S-1) and the next:
// the last stage's rows of the steps before must all lie below row 0
// (2 kFuseAhead - 1 < 6m), else they would never be loaded.
bool fuse_on(const msrcg_hier* h) { return h->o.plain_sweeps == 0 && 6 * h->o.m > 2 * kFuseAhead - 1; }

// Dynamic shared memory of a single-CTA launch for levels lo..kmax of h: the
// levels that fit (coarsest first) and the coarsest inverse; when a 2D FP32
// level of at least 4096 cells stays in global memory, the whole per-CTA
// limit, whose rest holds the rings of the single-pass smoother.  (512
// threads of 128 registers fill an SM's register file, so the CTA has the SM
// to itself either way; launches that need no rings keep the L1 share.)
size_t levels_smem(const msrcg_hier* h, int lo, bool top_double) {
  const bool f32 = h->o.precision == 1;
  const size_t rsz = f32 ? sizeof(float) : sizeof(double), lim = small_smem_limit_any(h->dim, f32);
  size_t tot = 0;
  int kfit = h->nlev;
  for (int k = h->nlev - 1; k >= lo; --k) {
    const size_t vsz = (top_double && k == 0) ? sizeof(double) : rsz;
    const size_t b = level_smem_bytes(h->hL[k], vsz, rsz, h->dim);
    if (tot + b > lim) break;
    tot += b;
    kfit = k;
  }
  const size_t ainv = align16(sizeof(double) * (size_t)h->nc * h->nc);
  if (tot + ainv <= lim) tot += ainv;
  const long long fmin = h->o.fuse_min_cells > 0 ? h->o.fuse_min_cells : kFuseMinCells;
  if (h->dim == 2 && f32 && fuse_on(h))
    for (int k = lo; k < kfit; ++k)
      if (h->N[k] >= fmin) return lim;
  return tot;
}

ProblemDesc make_desc(msrcg_hier* h, const double* b, double* x, double tol) {
  ProblemDesc pd;
  memset(&pd, 0, sizeof(pd));
  pd.L = h->dL;
  pd.nlev = h->nlev;
  pd.m = h->o.m;
  pd.Ainv = h->Ainv;
  pd.nc = h->nc;
  pd.precision = h->o.precision;
  pd.S = h->dS;
  pd.b = b;
  pd.x = x;
  pd.xs = h->xs;
  pd.tol = tol;
  pd.work = h->N[0];
  pd.fuse = fuse_on(h);
  pd.fuse_width = h->o.fuse_width;
  pd.fuse_min_cells = h->o.fuse_min_cells > 0 ? h->o.fuse_min_cells : kFuseMinCells;
  pd.splitting = h->o.splitting;
  pd.allow_flex = h->o.precision == 1;
  // the stall test watches the recursive multi-scale PCG (eq. 2.10); the
  // multigrid and polynomial preconditioners converge slowly by design
  pd.stall_w = pd.allow_flex && h->o.precond == 0 && h->o.stall_iters >= 0
                   ? (h->o.stall_iters > 0 ? h->o.stall_iters : 30)
                   : 0;
  pd.flex0 = h->o.flexible;
  pd.precond = h->o.precond;
  pd.trace = (unsigned long long*)h->trace;
  pd.trace_cap = (int)h->trace_cap;
  return pd;
}

void fill_stats(const msrcg_hier* h, const SolveState& S, msrcg_stats* st, int restarts) {
  memset(st, 0, sizeof(*st));
  st->levels = h->nlev;
  for (int k = 0; k < h->nlev; ++k) {
    for (int a = 0; a < 3; ++a) st->dims[k][a] = h->dims[k][a];
    st->iters[k] = S.lv[k].iters;
    st->calls[k] = S.lv[k].calls;
  }
  st->relres_recursive = S.bb0 > 0 ? sqrt(S.lv[0].rr / S.bb0) : 0.0;
  st->relres_true = S.bb0 > 0 ? sqrt(S.rr_true / S.bb0) : 0.0;
  st->restarts = restarts;
  st->status = msrcg_status_from_bits(S.status);
  st->flexible = S.flex != 0;
}

// After a failed solve, vectors may hold non-finite values (their ghosts
// included); clear every level's vectors so that the hierarchy is reusable.
int scrub(msrcg_hier* h, cudaStream_t s) {
  const size_t rsz = h->o.precision == 1 ? sizeof(float) : sizeof(double);
  for (int k = 0; k < h->nlev; ++k) {
    const DevLevel& L = h->hL[k];
    const size_t vsz = k == 0 ? sizeof(double) : rsz;
    void* v4[4] = {L.x, L.r, L.p, L.q};
    for (int v = 0; v < 4; ++v) MSRCG_CUDA_TRY(cudaMemsetAsync(v4[v], 0, vsz * L.npad, s));
    MSRCG_CUDA_TRY(cudaMemsetAsync(L.z, 0, rsz * L.npad, s));
    MSRCG_CUDA_TRY(cudaMemsetAsync(L.t, 0, rsz * L.npad, s));
  }
  MSRCG_CUDA_TRY(cudaMemsetAsync(h->b0, 0, sizeof(double) * h->hL[0].npad, s));
  return MSRCG_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" int msrcg_solve(msrcg_hier* h, const double* b, double tol, double* x, msrcg_stats* stats, void* stream) {
  if (!h || !b || !x || !(tol > 0.0) || !isfinite(tol)) return MSRCG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int dim = h->dim;
  const bool f32 = h->o.precision == 1;
  if (h->ks > 0 && !h->gexec) {
    int rc = build_graph(h);
    if (rc) return rc;
  }
  if (h->dirty) {
    int rc = scrub(h, s);
    if (rc) return rc;
    h->dirty = false;
  }
  {
    ProblemDesc pd = make_desc(h, b, x, tol);
    MSRCG_CUDA_TRY(cudaMemcpyAsync(h->dP, &pd, sizeof(pd), cudaMemcpyHostToDevice, s));
    const double floor2 = f32 ? h->o.inner_floor * h->o.inner_floor : 0.0;
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&h->dS->inner_floor2, &floor2, sizeof(double), cudaMemcpyHostToDevice, s));
  }
  SolveState hs;
  int restarts = 0;
  if (h->trace) MSRCG_CUDA_TRY(cudaMemsetAsync(h->trace, 0, sizeof(unsigned long long), s));
  if (h->ks == 0 || h->trace) {
    // every level fits one CTA, or the level tree is traced: one launch runs
    // the whole solve
    launch_small_any(dim, f32, h->dP, nullptr, 1, 0, 2, nullptr, 1, levels_smem(h, 0, true), s);
    MSRCG_CUDA_TRY(cudaGetLastError());
  } else {
    const int gmax = std::min(h->sms * 8, kMaxGrid);
    double* part = h->partials + (size_t)(kMaxLev - 1) * kMaxGrid;
    const DevLevel& L0 = h->hL[0];
    const Launch lc = cells_launch(L0, gmax), ll = lin_launch(L0.npad, gmax);
    MSRCG_CUDA_TRY(cudaMemsetAsync(h->xs, 0, sizeof(double) * L0.npad, s));
    const ProblemDesc pd = make_desc(h, b, x, tol);
    if (dim == 2)
      k_prepare<2><<<lc.grid, lc.block, 0, s>>>(L0, b, h->b0, tol, h->dS, h->nlev, part, pd.flex0, pd.allow_flex,
                                                pd.stall_w);
    else
      k_prepare<3><<<lc.grid, lc.block, 0, s>>>(L0, b, h->b0, tol, h->dS, h->nlev, part, pd.flex0, pd.allow_flex,
                                                pd.stall_w);
    MSRCG_CUDA_TRY(cudaGetLastError());
    for (;;) {
      MSRCG_CUDA_TRY(cudaGraphLaunch(h->gexec, s));
      k_accumulate<<<ll.grid, ll.block, 0, s>>>((const double*)L0.x, h->xs, L0.npad);
      if (dim == 2) k_true_residual<2><<<lc.grid, lc.block, 0, s>>>(L0, b, h->b0, h->xs, h->dS, part);
      else k_true_residual<3><<<lc.grid, lc.block, 0, s>>>(L0, b, h->b0, h->xs, h->dS, part);
      MSRCG_CUDA_TRY(cudaGetLastError());
      if (!stats) break;
      MSRCG_CUDA_TRY(cudaMemcpyAsync(&hs, h->dS, sizeof(hs), cudaMemcpyDeviceToHost, s));
      MSRCG_CUDA_TRY(cudaStreamSynchronize(s));
      if (hs.status != 0 || hs.rr_true < hs.tau2 * hs.bb0 || restarts >= 3 || !(hs.bb0 > 0)) break;
      ++restarts;
    }
    if (dim == 2) k_copy_out<2><<<lc.grid, lc.block, 0, s>>>(L0, h->xs, x);
    else k_copy_out<3><<<lc.grid, lc.block, 0, s>>>(L0, h->xs, x);
    MSRCG_CUDA_TRY(cudaGetLastError());
  }
  if (stats) {
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&hs, h->dS, sizeof(hs), cudaMemcpyDeviceToHost, s));
    MSRCG_CUDA_TRY(cudaStreamSynchronize(s));
    fill_stats(h, hs, stats, restarts);
    for (int k = 0; k < h->nlev; ++k) {
      h->last_iters[k] = stats->iters[k];
      h->last_calls[k] = stats->calls[k];
    }
    if (stats->status != MSRCG_OK) h->dirty = true;
    if (stats->status == MSRCG_ENOCONV && f32 && h->o.escalate) {
      // the FP32 preconditioner did not get there: solve again with the FP64
      // one (same operator, same tolerance)
      msrcg_hier* tw = nullptr;
      int rc = msrcg_twin(h, s, &tw);
      if (rc) return rc;
      const int flexible = stats->flexible;
      rc = msrcg_solve(tw, b, tol, x, stats, stream);
      stats->flexible = flexible;
      stats->escalated = 1;
      return rc;
    }
    return stats->status;
  }
  return MSRCG_OK;
}

int msrcg_batch_enqueue(int count, msrcg_hier* const* hs, const double* const* b, double tol, double* const* x,
                        cudaStream_t s, SolveState* host_states) {
  if (count < 0 || (count > 0 && (!hs || !b || !x || !host_states)) || !(tol > 0.0) || !isfinite(tol))
    return MSRCG_EINVAL;
  if (count == 0) return MSRCG_OK;
  const int dim = hs[0]->dim, prec = hs[0]->o.precision;
  std::vector<ProblemDesc> pds(count);
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b[i] || !x[i] || hs[i]->dim != dim || hs[i]->o.precision != prec) return MSRCG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return MSRCG_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    if (hs[i]->dirty) {
      int rc = scrub(hs[i], s);
      if (rc) return rc;
      hs[i]->dirty = false;
    }
    pds[i] = make_desc(hs[i], b[i], x[i], tol);
    if (hs[i]->trace) MSRCG_CUDA_TRY(cudaMemsetAsync(hs[i]->trace, 0, sizeof(unsigned long long), s));
    const double floor2 = prec == 1 ? hs[i]->o.inner_floor * hs[i]->o.inner_floor : 0.0;
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&hs[i]->dS->inner_floor2, &floor2, sizeof(double), cudaMemcpyHostToDevice, s));
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return pds[a].work > pds[c].work; });
  void *dp = nullptr, *dord = nullptr, *dnext = nullptr;
  MSRCG_CUDA_TRY(cudaMallocAsync(&dp, sizeof(ProblemDesc) * count, s));
  MSRCG_CUDA_TRY(cudaMallocAsync(&dord, sizeof(int) * count, s));
  MSRCG_CUDA_TRY(cudaMallocAsync(&dnext, sizeof(int), s));
  MSRCG_CUDA_TRY(cudaMemcpyAsync(dp, pds.data(), sizeof(ProblemDesc) * count, cudaMemcpyHostToDevice, s));
  MSRCG_CUDA_TRY(cudaMemcpyAsync(dord, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
  MSRCG_CUDA_TRY(cudaMemsetAsync(dnext, 0, sizeof(int), s));
  // shared memory per CTA: what the largest problem's coarse levels need
  size_t smem = 0;
  for (int i = 0; i < count; ++i) smem = std::max(smem, levels_smem(hs[i], 0, true));
  int sms = hs[0]->sms, per = 0;
  if (dim == 2) {
    if (prec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<2, float>, kSmallThreads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<2, double>, kSmallThreads, smem);
  } else {
    if (prec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<3, float>, kSmallThreads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<3, double>, kSmallThreads, smem);
  }
  int grid = std::max(1, std::min(count, sms * std::max(per, 1)));
  launch_small_any(dim, prec == 1, (const ProblemDesc*)dp, (const int*)dord, count, 0, 1, (int*)dnext, grid, smem, s);
  MSRCG_CUDA_TRY(cudaGetLastError());
  for (int i = 0; i < count; ++i)
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&host_states[i], hs[i]->dS, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  MSRCG_CUDA_TRY(cudaFreeAsync(dp, s));
  MSRCG_CUDA_TRY(cudaFreeAsync(dord, s));
  MSRCG_CUDA_TRY(cudaFreeAsync(dnext, s));
  return MSRCG_OK;
}

int msrcg_batch_finish(int count, msrcg_hier* const* hs, const SolveState* host_states, msrcg_stats* stats) {
  int rc = MSRCG_OK;
  for (int i = 0; i < count; ++i) {
    msrcg_stats one;
    fill_stats(hs[i], host_states[i], &one, 0);
    if (stats) stats[i] = one;
    for (int k = 0; k < hs[i]->nlev; ++k) {
      hs[i]->last_iters[k] = one.iters[k];
      hs[i]->last_calls[k] = one.calls[k];
    }
    if (one.status) {
      hs[i]->dirty = true;
      if (!rc) rc = one.status;
    }
  }
  return rc;
}

extern "C" int msrcg_set_trace(msrcg_hier* h, void* buf, int64_t capacity) {
  if (!h || capacity < 0 || capacity > INT32_MAX || ((uintptr_t)buf & 15)) return MSRCG_EINVAL;
  h->trace = buf;
  h->trace_cap = buf ? capacity : 0;
  return MSRCG_OK;
}

extern "C" int msrcg_batch_solve(int count, msrcg_hier* const* hs, const double* const* b, double tol, double* const* x,
                                 msrcg_stats* stats, void* stream) {
  if (count < 0) return MSRCG_EINVAL;
  if (count == 0) return MSRCG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<SolveState> st(count);
  int rc = msrcg_batch_enqueue(count, hs, b, tol, x, s, st.data());
  if (rc) return rc;
  MSRCG_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<msrcg_stats> one(count);
  rc = msrcg_batch_finish(count, hs, st.data(), one.data());
  // problems the FP32 preconditioner did not solve: again, one by one, with
  // the FP64 preconditioner
  bool again = false;
  for (int i = 0; i < count; ++i) {
    if (one[i].status != MSRCG_ENOCONV || hs[i]->o.precision != 1 || !hs[i]->o.escalate) continue;
    msrcg_hier* tw = nullptr;
    int e = msrcg_twin(hs[i], s, &tw);
    if (e) return e;
    const int flexible = one[i].flexible;
    msrcg_solve(tw, b[i], tol, x[i], &one[i], stream);
    one[i].flexible = flexible;
    one[i].escalated = 1;
    again = true;
  }
  if (again) {
    rc = MSRCG_OK;
    for (int i = 0; i < count && !rc; ++i) rc = one[i].status;
  }
  if (stats)
    for (int i = 0; i < count; ++i) stats[i] = one[i];
  return rc;
}

// ===========================================================================
// Standalone timing of the multi-CTA kernels of one wide level
// ===========================================================================
namespace {

// Interior cells of every vector of a level (and of the coarse level's x) set
// to 1 for the timing runs: finite values, p . A p > 0 (the Dirichlet faces),
// so that every kernel does its whole work.
template <int DIM, typename RP, typename V>
__global__ void k_fill_ones(DevLevel L, DevLevel C) {
  for_cells<DIM>(grid_map(), L, [&](int i, const Row& rw) {
    const int c = rw.pc + i;
    ((V*)L.x)[c] = (V)1;
    ((V*)L.r)[c] = (V)1;
    ((V*)L.p)[c] = (V)1;
    ((V*)L.q)[c] = (V)1;
    ((RP*)L.z)[c] = (RP)1;
    ((RP*)L.t)[c] = (RP)1;
    ((RP*)L.rp)[c] = (RP)1;
  });
  for_cells<DIM>(grid_map(), C, [&](int i, const Row& rw) { ((RP*)C.x)[rw.pc + i] = (RP)1; });
}

const char* const kProfNames[] = {
    "k_sweep (red-black half-sweep)", "k_sweep (first half-sweep, from zero)", "k_sweep_rho (last half-sweep + r.z)",
    "k_residual (t = rp - A z)", "k_restrict (r_c = R t)", "k_prolong_black (z += E x_c, black cells)",
    "k_direction (p = z + beta p)", "k_apply_dot (q = A p, p.q)", "k_update (x += alpha p, r -= alpha q, r.r)",
    "k_inv_diag (1/D for the FP64 half-sweeps)"};
constexpr int kProfCount = (int)(sizeof(kProfNames) / sizeof(kProfNames[0]));

template <int DIM, typename RP, typename V>
int profile_level_t(msrcg_hier* h, int k, int reps, cudaStream_t s, double* ms, double* bytes) {
  const DevLevel& L = h->hL[k];
  const DevLevel& C = h->hL[k + 1];
  const int gmax = std::min(h->sms * 8, kMaxGrid);
  const Launch lc = cells_launch(L, gmax), lp = pairs_launch(L, gmax);
  const Launch ll = lin_launch(L.npad, gmax), lu = lin_launch(L.npad, std::min(gmax, kMaxGrid / 2));
  double* part = h->partials + (size_t)k * kMaxGrid;
  SolveState* S = h->dS;
  // a state in which every kernel does its full work: level k live, not the
  // first iteration, finite scalars, a threshold that never stops it
  SolveState st;
  memset(&st, 0, sizeof(st));
  LevelState& ls = st.lv[k];
  ls.it = 1;
  ls.rho = ls.rho_old = ls.pq = 1.0;
  ls.alpha = ls.beta = 0.5;
  ls.alpha_f = ls.beta_f = 0.5f;
  ls.thr = -1.0;
  MSRCG_CUDA_TRY(cudaMemcpyAsync(S, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  const double n = (double)L.n, nc = (double)C.n, d = DIM, rsz = sizeof(RP), vsz = sizeof(V);
  const double iv = rsz == sizeof(double) ? 0.5 : 0.0;  // FP64: one colour's 1/D read
  const double bytes_of[kProfCount] = {
      (d + 1.5 + iv) * n * rsz,                               // T, rp and z of one colour, the other colour's z
      (iv > 0 ? iv * n * rsz : d * n * rsz) + n * vsz + (vsz != rsz ? n * rsz : 0.0) + n * rsz,  // T or 1/D, r (-> rp), z
      (d + 2.0 + iv) * n * rsz + n * vsz,                     // half-sweep + z and r of every cell
      (d + 3.0) * n * rsz,                                    // T, rp, z, t
      (n + nc) * rsz,                                         // t, r_c
      (n + nc) * rsz,                                         // x_c, black z read and written
      n * rsz + 2.0 * n * vsz,                                // z, p read, p written
      (d + 2.0) * n * vsz,                                    // T (vector precision), p, q
      6.0 * n * vsz,                                          // x, p, r, q read; x, r written
      (d + 1.0) * n * rsz};                                   // T read, 1/D written
  cudaEvent_t e0, e1;
  MSRCG_CUDA_TRY(cudaEventCreate(&e0));
  MSRCG_CUDA_TRY(cudaEventCreate(&e1));
  int rc = MSRCG_OK;
  for (int id = 0; id < kProfCount && !rc; ++id) {
    auto launch = [&]() {
      switch (id) {
        case 0: k_sweep<DIM, RP, V><<<lp.grid, lp.block, 0, s>>>(L, 0, 0); break;
        case 1: k_sweep<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, 0, 1); break;
        case 2: k_sweep_rho<DIM, RP, V><<<lp.grid, lp.block, 0, s>>>(L, k, S, part); break;
        case 3: k_residual<DIM, RP><<<lc.grid, lc.block, 0, s>>>(L); break;
        case 4: launch_restrict<DIM, RP>(h, k, gmax, s); break;
        case 5: k_prolong_black<DIM, RP><<<lp.grid, lp.block, 0, s>>>(L, C); break;
        case 6: k_direction<V, RP><<<ll.grid, ll.block, 0, s>>>(L, k, S); break;
        case 7: k_apply_dot<DIM, V><<<lc.grid, lc.block, 0, s>>>(L, k, S, part); break;
        case 8: k_update<V, RP><<<lu.grid, lu.block, 0, s>>>(L, k, S, part, 0, 0); break;
        default: k_inv_diag<DIM, RP><<<lc.grid, lc.block, 0, s>>>(L); break;
      }
    };
    k_fill_ones<DIM, RP, V><<<lc.grid, lc.block, 0, s>>>(L, C);
    if (cudaMemcpyAsync(S, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = MSRCG_ECUDA;
    for (int w = 0; w < 3; ++w) launch();  // warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) rc = MSRCG_ECUDA;
    for (int r = 0; r < reps && !rc; ++r) {
      launch();
      // keep the state live for the next launch (the update counts iterations)
      if (id == 8 && cudaMemcpyAsync(S, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = MSRCG_ECUDA;
    }
    if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = MSRCG_ECUDA;
    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = MSRCG_ECUDA;
    float t = 0.f;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = MSRCG_ECUDA;
    if (!rc && cudaGetLastError() != cudaSuccess) rc = MSRCG_ECUDA;
    ms[id] = (double)t / reps;
    bytes[id] = bytes_of[id];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)cudaGetLastError();
  h->dirty = true;  // the level's vectors hold timing garbage: cleared before the next solve
  return rc;
}

}  // namespace

extern "C" int msrcg_profile_kernel_count(void) { return kProfCount; }

extern "C" const char* msrcg_profile_kernel_name(int i) { return i >= 0 && i < kProfCount ? kProfNames[i] : ""; }

extern "C" int msrcg_profile_level(msrcg_hier* h, int level, int reps, double* ms, double* bytes, void* stream) {
  if (!h || !ms || !bytes || reps < 1 || level < 0 || level >= h->ks || level + 1 >= h->nlev) return MSRCG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const bool f32 = h->o.precision == 1;
  if (level == 0) {
    if (h->dim == 2) return f32 ? profile_level_t<2, float, double>(h, 0, reps, s, ms, bytes)
                                : profile_level_t<2, double, double>(h, 0, reps, s, ms, bytes);
    return f32 ? profile_level_t<3, float, double>(h, 0, reps, s, ms, bytes)
               : profile_level_t<3, double, double>(h, 0, reps, s, ms, bytes);
  }
  if (h->dim == 2) return f32 ? profile_level_t<2, float, float>(h, level, reps, s, ms, bytes)
                              : profile_level_t<2, double, double>(h, level, reps, s, ms, bytes);
  return f32 ? profile_level_t<3, float, float>(h, level, reps, s, ms, bytes)
             : profile_level_t<3, double, double>(h, level, reps, s, ms, bytes);
}

// ===========================================================================
// Solve without allocating (msrcg_solve_static)
//
// For callers that must not allocate device memory: code whose device memory
// is all owned by another allocator (a framework's caching pool, a fixed
// budget reserved at start-up), and code that runs where cudaMalloc is not
// allowed or not wanted (real-time loops).  The whole hierarchy of a small
// problem lives in one file-scope device array; the caller passes only the
// inputs and the output.
// ===========================================================================
namespace {

// The scratch of msrcg_solve_static.  Every device that loads the library
// holds it until the process exits.  Host code must not pass the symbol
// itself to a kernel: on the host it is only a stand-in, so its device
// address is looked up with cudaGetSymbolAddress (once per device).
static __device__ __align__(256) unsigned char g_static_scratch[MSRCG_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_static_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int msrcg_solve_static(const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                                  const msrcg_opts* opts, const double* b, double tol, double* x, msrcg_stats* stats,
                                  void* stream) {
  if (!grid || !K || !bc || !b || !x || !(tol > 0.0) || !isfinite(tol)) return MSRCG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  MSRCG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MSRCG_EINVAL;
  if (!g_static_ptr[dev]) {
    // first call on this device: find the device address of the scratch
    void* p = nullptr;
    MSRCG_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    if (!p) return MSRCG_ECUDA;
    g_static_ptr[dev] = p;
  }
  msrcg_hier h;  // host bookkeeping only; its device arrays are carved from the scratch
  // an MSRCG_EINVAL for a problem that does not fit comes before any work is
  // enqueued; every other error waits for the enqueued work first
  int rc = msrcg_build_into(&h, grid, K, ncomp, bc, opts, s, (unsigned char*)g_static_ptr[dev],
                            MSRCG_STATIC_SCRATCH_BYTES);
  if (rc) return rc;
  auto fail = [&](cudaError_t e, const char* what) {
    cudaStreamSynchronize(s);
    return msrcg_cuda_fail(e, what, __FILE__, __LINE__);
  };
  const bool f32 = h.o.precision == 1;
  ProblemDesc pd = make_desc(&h, b, x, tol);
  cudaError_t e = cudaMemcpyAsync(h.dP, &pd, sizeof(pd), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(e, "cudaMemcpyAsync(desc)");
  const double floor2 = f32 ? h.o.inner_floor * h.o.inner_floor : 0.0;
  e = cudaMemcpyAsync(&h.dS->inner_floor2, &floor2, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(e, "cudaMemcpyAsync(floor)");
  launch_small_any(h.dim, f32, h.dP, nullptr, 1, 0, 2, nullptr, 1, levels_smem(&h, 0, true), s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e, "k_small");
  SolveState hs;
  e = cudaMemcpyAsync(&hs, h.dS, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail(e, "cudaMemcpyAsync(state)");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e, "cudaStreamSynchronize");
  msrcg_stats one;
  fill_stats(&h, hs, &one, 0);
  if (stats) *stats = one;
  return one.status;
}
