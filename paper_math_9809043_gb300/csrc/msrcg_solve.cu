// Solve path of libmsrcg: the recursive multi-scale PCG of Lackner & Menikoff
// (eq. 2.10, Sec. 2.3, Sec. 3) on the GPU.
//
// Levels 0..ks-1 ("wide" levels) run as separate multi-CTA kernels that a CUDA
// graph sequences; each level's PCG loop is a graph WHILE node whose
// condition the last kernel of an iteration sets on the device, so no host
// round trip decides anything.  Levels ks..kmax ("narrow" levels, few cells)
// run inside one CTA that executes the whole remaining recursion: the level
// stack is an explicit state machine over levels, with __syncthreads between
// dependent steps.  The same single-CTA solver also runs complete problems,
// one per CTA, for the batched entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "msrcg_internal.cuh"

using namespace msrcg;

namespace {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum; every thread returns the total.  `sh` holds 33
// doubles of shared memory.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

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

struct Cell {
  int i, j, k;
  long long c;
};

__device__ __forceinline__ Cell cell_of(long long c, int nx, int ny) {
  Cell q;
  q.c = c;
  q.i = (int)(c % nx);
  long long rw = c / nx;
  q.j = (int)(rw % ny);
  q.k = (int)(rw / ny);
  return q;
}

// Cell (i, j, k) of colour `colour` for pair index p (the colour's cells of a
// row are i = 2*ii + ((j + k + colour) & 1)); returns false past the row end.
__device__ __forceinline__ bool colour_cell(long long p, int colour, int nx, int ny, Cell& q) {
  const int hx = (nx + 1) >> 1;
  int ii = (int)(p % hx);
  long long rw = p / hx;
  q.j = (int)(rw % ny);
  q.k = (int)(rw / ny);
  q.i = 2 * ii + ((q.j + q.k + colour) & 1);
  q.c = q.i + (long long)nx * rw;
  return q.i < nx;
}

// Sum of the face transmissibilities of a cell (the diagonal of A).
template <int DIM, typename R>
__device__ __forceinline__ R diag_of(const DevLevel& L, const R* Tx, const R* Ty, const R* Tz, const Cell& q) {
  const long long row = q.j + (long long)L.ny * q.k, ky = q.c + (long long)L.nx * q.k;
  R d = Tx[q.c + row];
  d += Tx[q.c + row + 1];
  d += Ty[ky];
  d += Ty[ky + L.nx];
  if (DIM == 3) {
    d += Tz[q.c];
    d += Tz[q.c + (long long)L.nx * L.ny];
  }
  return d;
}

// Gauss-Seidel value of one cell: row c of A solved for x_c with the
// neighbours held, x_c = (rhs_c + sum_f T_f x_nb) / sum_f T_f  (Sec. 3).
template <int DIM, typename R, typename RB>
__device__ __forceinline__ R gs_value(const DevLevel& L, const R* Tx, const R* Ty, const R* Tz, const RB* rhs,
                                      const R* x, const Cell& q) {
  const int nx = L.nx, ny = L.ny;
  const long long c = q.c, row = q.j + (long long)ny * q.k, ky = c + (long long)nx * q.k;
  R t = Tx[c + row], d = t, s = (R)rhs[c];
  if (q.i > 0) s += t * x[c - 1];
  t = Tx[c + row + 1];
  d += t;
  if (q.i < nx - 1) s += t * x[c + 1];
  t = Ty[ky];
  d += t;
  if (q.j > 0) s += t * x[c - nx];
  t = Ty[ky + nx];
  d += t;
  if (q.j < ny - 1) s += t * x[c + nx];
  if (DIM == 3) {
    const long long pl = (long long)nx * ny;
    t = Tz[c];
    d += t;
    if (q.k > 0) s += t * x[c - pl];
    t = Tz[c + pl];
    d += t;
    if (q.k < L.nz - 1) s += t * x[c + pl];
  }
  return s / d;
}

// (A x)_c = sum_f T_f (x_c - x_nb), T_f x_c on boundary faces.
template <int DIM, typename R, typename RX>
__device__ __forceinline__ R apply_value(const DevLevel& L, const R* Tx, const R* Ty, const R* Tz, const RX* x,
                                         const Cell& q) {
  const int nx = L.nx, ny = L.ny;
  const long long c = q.c, row = q.j + (long long)ny * q.k, ky = c + (long long)nx * q.k;
  const R xc = (R)x[c];
  R s = 0, t;
  t = Tx[c + row];
  s += q.i > 0 ? t * (xc - (R)x[c - 1]) : t * xc;
  t = Tx[c + row + 1];
  s += q.i < nx - 1 ? t * (xc - (R)x[c + 1]) : t * xc;
  t = Ty[ky];
  s += q.j > 0 ? t * (xc - (R)x[c - nx]) : t * xc;
  t = Ty[ky + nx];
  s += q.j < ny - 1 ? t * (xc - (R)x[c + nx]) : t * xc;
  if (DIM == 3) {
    const long long pl = (long long)nx * ny;
    t = Tz[c];
    s += q.k > 0 ? t * (xc - (R)x[c - pl]) : t * xc;
    t = Tz[c + pl];
    s += q.k < L.nz - 1 ? t * (xc - (R)x[c + pl]) : t * xc;
  }
  return s;
}

// Weight of fine index i on coarse index I in the 1-D interpolation table.
template <typename R>
__device__ __forceinline__ R tw(const int* c0, const int* c1, const R* w, int i, int I) {
  R v = 0;
  if (c0[i] == I) v += (R)1 - w[i];
  if (c1[i] == I) v += w[i];
  return v;
}

// (R t)_C = (E^T t)_C for coarse cell (I, J, K) of level k+1: a gather over
// the fine cells whose interpolation uses it (Sec. 3, R = E^T).
template <int DIM, typename R>
__device__ __forceinline__ R restrict_value(const DevLevel& F, const R* t, int I, int J, int K) {
  const R *wx = (const R*)F.w[0], *wy = (const R*)F.w[1];
  R acc = 0;
  const int klo = DIM == 3 ? F.lo[2][K] : 0, khi = DIM == 3 ? F.hi[2][K] : 0;
  for (int kk = klo; kk <= khi; ++kk) {
    const R wz = DIM == 3 ? tw<R>(F.c0[2], F.c1[2], (const R*)F.w[2], kk, K) : (R)1;
    R accy = 0;
    for (int jj = F.lo[1][J]; jj <= F.hi[1][J]; ++jj) {
      const R wyv = tw<R>(F.c0[1], F.c1[1], wy, jj, J);
      const R* row = t + (long long)F.nx * (jj + (long long)F.ny * kk);
      R accx = 0;
      for (int ii = F.lo[0][I]; ii <= F.hi[0][I]; ++ii) accx += tw<R>(F.c0[0], F.c1[0], wx, ii, I) * row[ii];
      accy += wyv * accx;
    }
    acc += wz * accy;
  }
  return acc;
}

// (E x_c)_c for fine cell q: tensor product of the 1-D linear interpolation
// with zero slope at the boundary (Sec. 3).
template <int DIM, typename R, typename RX>
__device__ __forceinline__ R prolong_value(const DevLevel& F, const DevLevel& Cc, const RX* xc, const Cell& q) {
  const R *wxp = (const R*)F.w[0], *wyp = (const R*)F.w[1];
  const R wx = wxp[q.i], wy = wyp[q.j];
  const int i0 = F.c0[0][q.i], i1 = F.c1[0][q.i], j0 = F.c0[1][q.j], j1 = F.c1[1][q.j];
  const int cnx = Cc.nx, cny = Cc.ny;
  if (DIM == 2) {
    const R a = ((R)1 - wx) * (R)xc[i0 + (long long)cnx * j0] + wx * (R)xc[i1 + (long long)cnx * j0];
    const R b = ((R)1 - wx) * (R)xc[i0 + (long long)cnx * j1] + wx * (R)xc[i1 + (long long)cnx * j1];
    return ((R)1 - wy) * a + wy * b;
  } else {
    const R wz = ((const R*)F.w[2])[q.k];
    const int k0 = F.c0[2][q.k], k1 = F.c1[2][q.k];
    const long long p0 = (long long)cnx * ((long long)cny * k0), p1 = (long long)cnx * ((long long)cny * k1);
    const R a0 = ((R)1 - wx) * (R)xc[p0 + i0 + (long long)cnx * j0] + wx * (R)xc[p0 + i1 + (long long)cnx * j0];
    const R b0 = ((R)1 - wx) * (R)xc[p0 + i0 + (long long)cnx * j1] + wx * (R)xc[p0 + i1 + (long long)cnx * j1];
    const R a1 = ((R)1 - wx) * (R)xc[p1 + i0 + (long long)cnx * j0] + wx * (R)xc[p1 + i1 + (long long)cnx * j0];
    const R b1 = ((R)1 - wx) * (R)xc[p1 + i0 + (long long)cnx * j1] + wx * (R)xc[p1 + i1 + (long long)cnx * j1];
    return ((R)1 - wz) * (((R)1 - wy) * a0 + wy * b0) + wz * (((R)1 - wy) * a1 + wy * b1);
  }
}

// ===========================================================================
// Single-CTA solver
// ===========================================================================
struct BlkShared {
  double red[33];
};

// One red-black half-sweep of the level (all threads of the CTA).  With
// `zero`, the iterate starts from x = 0: cells of `colour` get rhs/D and the
// other colour is cleared.
template <int DIM, typename RP, typename RB>
__device__ void b_sweep(const DevLevel& L, int colour, const RB* rhs, RP* z, bool zero) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  if (zero) {
    for (long long c = threadIdx.x; c < L.n; c += blockDim.x) {
      Cell q = cell_of(c, L.nx, L.ny);
      z[c] = ((q.i + q.j + q.k) & 1) == colour ? (RP)rhs[c] / diag_of<DIM, RP>(L, Tx, Ty, Tz, q) : (RP)0;
    }
  } else {
    const long long np = (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
    for (long long p = threadIdx.x; p < np; p += blockDim.x) {
      Cell q;
      if (colour_cell(p, colour, L.nx, L.ny, q)) z[q.c] = gs_value<DIM, RP, RB>(L, Tx, Ty, Tz, rhs, z, q);
    }
  }
  __syncthreads();
}

// m symmetric Gauss-Seidel steps in red-black order (eq. 2.10's (P^-1 Q)^m
// terms): forward red, black, backward black, red; the repeated black sweep
// reproduces the same values, so m steps are the 2m+1 half-sweeps
// red (black red)^m.
template <int DIM, typename RP, typename RB>
__device__ void b_smooth(const DevLevel& L, int m, const RB* rhs, RP* z, bool from_zero) {
  b_sweep<DIM, RP, RB>(L, 0, rhs, z, from_zero);
  for (int s = 0; s < m; ++s) {
    b_sweep<DIM, RP, RB>(L, 1, rhs, z, false);
    b_sweep<DIM, RP, RB>(L, 0, rhs, z, false);
  }
}

// t = r - A z, then r_{k+1} = R t.
template <int DIM, typename RP, typename V>
__device__ void b_residual_restrict(const DevLevel& L, const DevLevel& C, const V* r, const RP* z, RP* t, RP* rc) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  for (long long c = threadIdx.x; c < L.n; c += blockDim.x) {
    Cell q = cell_of(c, L.nx, L.ny);
    t[c] = (RP)r[c] - apply_value<DIM, RP, RP>(L, Tx, Ty, Tz, z, q);
  }
  __syncthreads();
  for (long long c = threadIdx.x; c < C.n; c += blockDim.x) {
    Cell q = cell_of(c, C.nx, C.ny);
    rc[c] = restrict_value<DIM, RP>(L, t, q.i, q.j, q.k);
  }
  __syncthreads();
}

template <int DIM, typename RP>
__device__ void b_prolong(const DevLevel& L, const DevLevel& C, const RP* xc, RP* z) {
  for (long long c = threadIdx.x; c < L.n; c += blockDim.x) {
    Cell q = cell_of(c, L.nx, L.ny);
    z[c] += prolong_value<DIM, RP, RP>(L, C, xc, q);
  }
  __syncthreads();
}

template <typename V>
__device__ double b_zero_dot(V* x, const V* r, long long n, double* sh) {
  V acc = 0;
  for (long long c = threadIdx.x; c < n; c += blockDim.x) {
    x[c] = 0;
    acc += r[c] * r[c];
  }
  return block_sum((double)acc, sh);
}

template <typename V, typename RP>
__device__ double b_dot(const V* a, const RP* b, long long n, double* sh) {
  V acc = 0;
  for (long long c = threadIdx.x; c < n; c += blockDim.x) acc += a[c] * (V)b[c];
  return block_sum((double)acc, sh);
}

template <typename V, typename RP>
__device__ void b_direction(V* p, const RP* z, long long n, bool first, V beta) {
  for (long long c = threadIdx.x; c < n; c += blockDim.x) p[c] = first ? (V)z[c] : (V)z[c] + beta * p[c];
  __syncthreads();
}

template <int DIM, typename V>
__device__ double b_apply_dot(const DevLevel& L, const V* p, V* q, double* sh) {
  const V *Tx = Tvec<V>(L, 0), *Ty = Tvec<V>(L, 1), *Tz = DIM == 3 ? Tvec<V>(L, 2) : nullptr;
  V acc = 0;
  for (long long c = threadIdx.x; c < L.n; c += blockDim.x) {
    Cell cq = cell_of(c, L.nx, L.ny);
    V v = apply_value<DIM, V, V>(L, Tx, Ty, Tz, p, cq);
    q[c] = v;
    acc += p[c] * v;
  }
  return block_sum((double)acc, sh);
}

template <typename V>
__device__ double b_update(V* x, V* r, const V* p, const V* q, long long n, V alpha, double* sh) {
  V acc = 0;
  for (long long c = threadIdx.x; c < n; c += blockDim.x) {
    x[c] += alpha * p[c];
    V rv = r[c] - alpha * q[c];
    r[c] = rv;
    acc += rv * rv;
  }
  return block_sum((double)acc, sh);
}

// Coarsest level: z = A^-1 r with the FP64 explicit inverse (Sec. 2.2, the
// recursion ends with the exact inverse).
template <typename V, typename RP>
__device__ void b_coarsest(const double* Ainv, int nc, const V* r, RP* z) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    double s = 0.0;
    const double* row = Ainv + (long long)i * nc;
    for (int j = 0; j < nc; ++j) s += row[j] * (double)r[j];
    z[i] = (RP)s;
  }
  __syncthreads();
}

// Per-level control of the single-CTA state machine.
struct LvlCtl {
  double rho_old, thr, rho;
  int it, phase;
};
enum : int { kStart = 0, kIterate = 1, kAfterCoarse = 2, kPrecondDone = 3, kReturn = 4 };

// Ops of one level with its vector type V (double at level 0 of a full
// solve, the smoother type RP elsewhere).
template <int DIM, typename V, typename RP>
struct LevelOps {
  // PCG entry: x = 0, r holds b_k; returns ||b_k||^2
  static __device__ double enter(const DevLevel& L, double* sh) { return b_zero_dot<V>((V*)L.x, (const V*)L.r, L.n, sh); }
  static __device__ void presmooth_restrict(const DevLevel& L, const DevLevel& C, int m) {
    b_smooth<DIM, RP, V>(L, m, (const V*)L.r, (RP*)L.z, true);
    b_residual_restrict<DIM, RP, V>(L, C, (const V*)L.r, (const RP*)L.z, (RP*)L.t, (RP*)C.r);
  }
  static __device__ void coarsest(const DevLevel& L, const double* Ainv, int nc) {
    b_coarsest<V, RP>(Ainv, nc, (const V*)L.r, (RP*)L.z);
  }
  static __device__ void postsmooth(const DevLevel& L, int m) { b_smooth<DIM, RP, V>(L, m, (const V*)L.r, (RP*)L.z, false); }
  // rho = r.z, p = z + beta p, q = A p, alpha, x += alpha p, r -= alpha q.
  // Returns ||r||^2, or -1 on breakdown.
  static __device__ double cg_step(const DevLevel& L, LvlCtl& ct, double* sh) {
    const double rho = b_dot<V, RP>((const V*)L.r, (const RP*)L.z, L.n, sh);
    const bool first = ct.it == 0;
    b_direction<V, RP>((V*)L.p, (const RP*)L.z, L.n, first, first ? (V)0 : (V)(rho / ct.rho_old));
    const double pq = b_apply_dot<DIM, V>(L, (const V*)L.p, (V*)L.q, sh);
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rho)) return -1.0;
    const V alpha = (V)(rho / pq);
    ct.rho = rho;
    return b_update<V>((V*)L.x, (V*)L.r, (const V*)L.p, (const V*)L.q, L.n, alpha, sh);
  }
};

// The recursion of eq. (2.10) from level ks down to kmax, run by one CTA.
// On entry level ks's r holds its right-hand side; on exit its x holds the
// PCG result.  sL: the levels in shared memory.  top_double: level 0 (if ks
// is 0) keeps FP64 vectors while the preconditioner runs in RP.
template <int DIM, typename RP>
__device__ void small_recursion(const DevLevel* sL, int ks, int kmax, int m, const double* Ainv, int nc, double eps2,
                                double floor2, SolveState* S, double* sh) {
  LvlCtl ct[kMaxLev];
  int k = ks;
  ct[k].phase = kStart;
  const bool top_double = ks == 0;
  for (;;) {
    const DevLevel& L = sL[k];
    LvlCtl& c = ct[k];
    const bool dbl = top_double && k == 0;
    if (c.phase == kStart) {
      if (threadIdx.x == 0) S->lv[k].calls++;
      const double bb = dbl ? LevelOps<DIM, double, RP>::enter(L, sh) : LevelOps<DIM, RP, RP>::enter(L, sh);
      if (bb == 0.0) {
        c.phase = kReturn;
        continue;
      }
      double thr = L.fk * eps2;
      if (k > 0 && floor2 > 0.0) thr = fmax(thr, floor2 * bb / (double)L.n);
      c.thr = thr;
      c.it = 0;
      c.rho_old = 0.0;
      c.phase = kIterate;
    } else if (c.phase == kIterate) {
      if (k == kmax) {
        if (dbl) LevelOps<DIM, double, RP>::coarsest(L, Ainv, nc);
        else LevelOps<DIM, RP, RP>::coarsest(L, Ainv, nc);
        c.phase = kPrecondDone;
      } else {
        if (dbl) LevelOps<DIM, double, RP>::presmooth_restrict(L, sL[k + 1], m);
        else LevelOps<DIM, RP, RP>::presmooth_restrict(L, sL[k + 1], m);
        c.phase = kAfterCoarse;
        ++k;
        ct[k].phase = kStart;
      }
    } else if (c.phase == kAfterCoarse) {
      b_prolong<DIM, RP>(L, sL[k + 1], (const RP*)sL[k + 1].x, (RP*)L.z);
      if (dbl) LevelOps<DIM, double, RP>::postsmooth(L, m);
      else LevelOps<DIM, RP, RP>::postsmooth(L, m);
      c.phase = kPrecondDone;
    } else if (c.phase == kPrecondDone) {
      const double rr = dbl ? LevelOps<DIM, double, RP>::cg_step(L, c, sh) : LevelOps<DIM, RP, RP>::cg_step(L, c, sh);
      if (rr < 0.0) {
        if (threadIdx.x == 0) atomicOr(&S->status, kStBreakdown);
        c.phase = kReturn;
        continue;
      }
      if (threadIdx.x == 0) S->lv[k].iters++;
      c.it++;
      if (k == 0 && threadIdx.x == 0) S->lv[0].rr = rr;
      if (rr / (double)L.n < c.thr) {
        c.phase = kReturn;
      } else if (c.it >= L.maxit) {
        if (threadIdx.x == 0) atomicOr(&S->status, kStNoConv);
        c.phase = kReturn;
      } else {
        c.rho_old = c.rho;
        c.phase = kIterate;
      }
    } else {  // kReturn
      if (k == ks) break;
      --k;
    }
  }
  __syncthreads();
}

// Single-CTA kernel.
//  mode 0: solve levels ks..kmax of problem P[0]; its r_ks already holds b_ks
//          and eps^2 comes from the problem's state (the wide levels set it).
//  mode 1: full solves of problems P[order[i]]; CTAs take the next problem
//          index from *next (problems are sorted largest first).
//  mode 2: full solve of problem P[0] by CTA 0.
// A full solve copies b into r_0, computes eps^2 = tol^2 ||b||^2 / N_0, runs
// the recursion from level 0 with FP64 level-0 vectors, adds the result to
// x, forms the true residual b - A x in FP64 and, if that misses tol, runs
// the recursion again on it (at most 3 restarts).
template <int DIM, typename RP>
__global__ void __launch_bounds__(kSmallThreads) k_small(const ProblemDesc* __restrict__ P, const int* __restrict__ order,
                                                         int nprob, int ks, int mode, int* next) {
  __shared__ DevLevel sL[kMaxLev];
  __shared__ double sh[33];
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
    if (mode == 0) {
      small_recursion<DIM, RP>(sL, ks, kmax, pd.m, pd.Ainv, pd.nc, S->eps2, S->inner_floor2, S, sh);
      continue;
    }
    const DevLevel& L0 = sL[0];
    double* r0 = (double*)L0.r;
    double* x0 = (double*)L0.x;
    double bbl = 0.0;
    for (long long c = threadIdx.x; c < L0.n; c += blockDim.x) {
      const double v = pd.b[c];
      r0[c] = v;
      pd.x[c] = 0.0;
      bbl += v * v;
    }
    const double bb = block_sum(bbl, sh);
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
    }
    __syncthreads();
    if (!(bb > 0.0) || !isfinite(bb)) continue;
    const double floor2 = S->inner_floor2;
    for (int pass = 0; pass < 4; ++pass) {
      small_recursion<DIM, RP>(sL, 0, kmax, pd.m, pd.Ainv, pd.nc, eps2, floor2, S, sh);
      for (long long c = threadIdx.x; c < L0.n; c += blockDim.x) pd.x[c] += x0[c];
      __syncthreads();
      double rl = 0.0;
      for (long long c = threadIdx.x; c < L0.n; c += blockDim.x) {
        Cell q = cell_of(c, L0.nx, L0.ny);
        const double v =
            pd.b[c] - apply_value<DIM, double, double>(L0, L0.T64[0], L0.T64[1], DIM == 3 ? L0.T64[2] : nullptr, pd.x, q);
        r0[c] = v;
        rl += v * v;
      }
      const double rt = block_sum(rl, sh);
      if (threadIdx.x == 0) S->rr_true = rt;
      __syncthreads();
      if (S->status != 0 || rt < pd.tol * pd.tol * bb) break;
    }
  }
}

// ===========================================================================
// Multi-CTA level kernels (wide levels, sequenced by the graph)
// ===========================================================================

// Reduction across the CTAs of one launch: each CTA writes its partial, the
// last CTA to arrive (ticket) sums the partials in index order and calls fin
// with the total.  Deterministic for a given grid size.
template <class Fin>
__device__ void grid_total(double v, double* partials, unsigned int* ticket, double* sh, Fin fin) {
  const double bs = block_sum(v, sh);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = t == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    if (threadIdx.x < 32) {
      for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) s += __ldcg(partials + i);
      s = warp_sum(s);
      if (threadIdx.x == 0) {
        *ticket = 0u;
        fin(s);
      }
    }
  }
}

__device__ __forceinline__ long long gtid() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// PCG entry on a wide level: x = 0 (level 0: r = b0), ||b_k||^2, threshold,
// counters, and the WHILE condition of the level's loop.
template <typename V>
__global__ void __launch_bounds__(kThreads) k_init(DevLevel L, int k, SolveState* S, const double* b0, double* partials,
                                                   cudaGraphConditionalHandle hcond) {
  __shared__ double sh[33];
  V* x = (V*)L.x;
  V* r = (V*)L.r;
  V acc = 0;
  for (long long c = gtid(); c < L.n; c += gstride()) {
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
  grid_total((double)acc, partials, &S->ticket[k], sh, [&](double bb) {
    LevelState& ls = S->lv[k];
    ls.bb = bb;
    double thr = L.fk * S->eps2;
    if (k > 0 && S->inner_floor2 > 0.0) thr = fmax(thr, S->inner_floor2 * bb / (double)L.n);
    ls.thr = thr;
    ls.it = 0;
    ls.calls++;
    ls.rho_old = 0.0;
    ls.rr = bb;
    ls.stop = !(bb > 0.0) || !isfinite(bb);
    cudaGraphSetConditional(hcond, ls.stop ? 0u : 1u);
  });
}

// One red-black half-sweep over a wide level (see b_sweep).
template <int DIM, typename RP, typename RB>
__global__ void __launch_bounds__(kThreads) k_sweep(DevLevel L, int colour, int zero) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const RB* rhs = (const RB*)L.r;
  RP* z = (RP*)L.z;
  if (zero) {
    for (long long c = gtid(); c < L.n; c += gstride()) {
      Cell q = cell_of(c, L.nx, L.ny);
      z[c] = ((q.i + q.j + q.k) & 1) == colour ? (RP)rhs[c] / diag_of<DIM, RP>(L, Tx, Ty, Tz, q) : (RP)0;
    }
  } else {
    const long long np = (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
    for (long long p = gtid(); p < np; p += gstride()) {
      Cell q;
      if (colour_cell(p, colour, L.nx, L.ny, q)) z[q.c] = gs_value<DIM, RP, RB>(L, Tx, Ty, Tz, rhs, z, q);
    }
  }
}

template <int DIM, typename RP, typename V>
__global__ void __launch_bounds__(kThreads) k_residual(DevLevel L) {
  const RP *Tx = (const RP*)L.T[0], *Ty = (const RP*)L.T[1], *Tz = (const RP*)L.T[2];
  const V* r = (const V*)L.r;
  const RP* z = (const RP*)L.z;
  RP* t = (RP*)L.t;
  for (long long c = gtid(); c < L.n; c += gstride()) {
    Cell q = cell_of(c, L.nx, L.ny);
    t[c] = (RP)r[c] - apply_value<DIM, RP, RP>(L, Tx, Ty, Tz, z, q);
  }
}

template <int DIM, typename RP>
__global__ void __launch_bounds__(kThreads) k_restrict(DevLevel L, DevLevel C) {
  const RP* t = (const RP*)L.t;
  RP* rc = (RP*)C.r;
  for (long long c = gtid(); c < C.n; c += gstride()) {
    Cell q = cell_of(c, C.nx, C.ny);
    rc[c] = restrict_value<DIM, RP>(L, t, q.i, q.j, q.k);
  }
}

template <int DIM, typename RP>
__global__ void __launch_bounds__(kThreads) k_prolong(DevLevel L, DevLevel C) {
  const RP* xc = (const RP*)C.x;
  RP* z = (RP*)L.z;
  for (long long c = gtid(); c < L.n; c += gstride()) {
    Cell q = cell_of(c, L.nx, L.ny);
    z[c] += prolong_value<DIM, RP, RP>(L, C, xc, q);
  }
}

// rho = r . z
template <typename V, typename RP>
__global__ void __launch_bounds__(kThreads) k_rho(DevLevel L, int k, SolveState* S, double* partials) {
  __shared__ double sh[33];
  if (S->lv[k].stop) return;
  const V* r = (const V*)L.r;
  const RP* z = (const RP*)L.z;
  V acc = 0;
  for (long long c = gtid(); c < L.n; c += gstride()) acc += r[c] * (V)z[c];
  grid_total((double)acc, partials, &S->ticket[k], sh, [&](double rho) { S->lv[k].rho = rho; });
}

// p = z (first iteration) or z + (rho/rho_old) p
template <typename V, typename RP>
__global__ void __launch_bounds__(kThreads) k_direction(DevLevel L, int k, SolveState* S) {
  const LevelState& ls = S->lv[k];
  if (ls.stop) return;
  const bool first = ls.it == 0;
  const V beta = first ? (V)0 : (V)(ls.rho / ls.rho_old);
  V* p = (V*)L.p;
  const RP* z = (const RP*)L.z;
  for (long long c = gtid(); c < L.n; c += gstride()) p[c] = first ? (V)z[c] : (V)z[c] + beta * p[c];
}

// q = A p, pq = p . q; breakdown check
template <int DIM, typename V>
__global__ void __launch_bounds__(kThreads) k_apply_dot(DevLevel L, int k, SolveState* S, double* partials) {
  __shared__ double sh[33];
  if (S->lv[k].stop) return;
  const V *Tx = Tvec<V>(L, 0), *Ty = Tvec<V>(L, 1), *Tz = DIM == 3 ? Tvec<V>(L, 2) : nullptr;
  const V* p = (const V*)L.p;
  V* q = (V*)L.q;
  V acc = 0;
  for (long long c = gtid(); c < L.n; c += gstride()) {
    Cell cq = cell_of(c, L.nx, L.ny);
    const V v = apply_value<DIM, V, V>(L, Tx, Ty, Tz, p, cq);
    q[c] = v;
    acc += p[c] * v;
  }
  grid_total((double)acc, partials, &S->ticket[k], sh, [&](double pq) {
    LevelState& ls = S->lv[k];
    ls.pq = pq;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(ls.rho)) {
      ls.stop = 1;
      atomicOr(&S->status, kStBreakdown);
    }
  });
}

// x += alpha p, r -= alpha q, ||r||^2, the level test of Sec. 3 and the
// WHILE condition of the level's loop.
template <typename V>
__global__ void __launch_bounds__(kThreads) k_update(DevLevel L, int k, SolveState* S, double* partials,
                                                     cudaGraphConditionalHandle hcond) {
  __shared__ double sh[33];
  const LevelState& ls = S->lv[k];
  if (ls.stop) {
    if (gtid() == 0) cudaGraphSetConditional(hcond, 0u);
    return;
  }
  const V alpha = (V)(ls.rho / ls.pq);
  V* x = (V*)L.x;
  V* r = (V*)L.r;
  const V* p = (const V*)L.p;
  const V* q = (const V*)L.q;
  V acc = 0;
  for (long long c = gtid(); c < L.n; c += gstride()) {
    x[c] += alpha * p[c];
    const V rv = r[c] - alpha * q[c];
    r[c] = rv;
    acc += rv * rv;
  }
  grid_total((double)acc, partials, &S->ticket[k], sh, [&](double rr) {
    LevelState& w = S->lv[k];
    w.rr = rr;
    w.iters++;
    w.it++;
    bool go = true;
    if (rr / (double)L.n < w.thr) {
      go = false;
    } else if (w.it >= L.maxit) {
      atomicOr(&S->status, kStNoConv);
      go = false;
    }
    w.rho_old = w.rho;
    if (!go) w.stop = 1;
    cudaGraphSetConditional(hcond, go ? 1u : 0u);
  });
}

// Before a solve: b0 = b, ||b||^2, eps^2 = tol^2 ||b||^2 / N_0 (Sec. 3), x = 0,
// counters cleared.
__global__ void __launch_bounds__(kThreads) k_prepare(const double* b, double* b0, double* xs, long long n, double tol,
                                                      SolveState* S, int nlev, double* partials) {
  __shared__ double sh[33];
  double acc = 0.0;
  for (long long c = gtid(); c < n; c += gstride()) {
    const double v = b[c];
    b0[c] = v;
    xs[c] = 0.0;
    acc += v * v;
  }
  grid_total(acc, partials, &S->ticket[kMaxLev - 1], sh, [&](double bb) {
    S->bb0 = bb;
    S->tau2 = tol * tol;
    S->eps2 = tol * tol * (bb / (double)n);
    S->status = isfinite(bb) ? 0 : kStNanInf;
    S->rr_true = bb;
    for (int k = 0; k < nlev; ++k) {
      S->lv[k].iters = 0;
      S->lv[k].calls = 0;
      S->lv[k].stop = 0;
      S->lv[k].rr = 0.0;
    }
  });
}

// After the level-0 PCG: xs += x_0.  The true residual b - A xs needs the
// neighbours of every cell, so it is taken by the next kernel.
__global__ void __launch_bounds__(kThreads) k_accumulate(const double* __restrict__ x0, double* __restrict__ xs, long long n) {
  for (long long c = gtid(); c < n; c += gstride()) xs[c] += x0[c];
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_true_residual(DevLevel L0, const double* b, double* b0, const double* xs,
                                                            SolveState* S, double* partials) {
  __shared__ double sh[33];
  const double *Tx = L0.T64[0], *Ty = L0.T64[1], *Tz = DIM == 3 ? L0.T64[2] : nullptr;
  double acc = 0.0;
  for (long long c = gtid(); c < L0.n; c += gstride()) {
    Cell q = cell_of(c, L0.nx, L0.ny);
    const double v = b[c] - apply_value<DIM, double, double>(L0, Tx, Ty, Tz, xs, q);
    b0[c] = v;
    acc += v * v;
  }
  grid_total(acc, partials, &S->ticket[kMaxLev - 1], sh, [&](double rt) { S->rr_true = rt; });
}

// ===========================================================================
// Host side
// ===========================================================================
int grid_for(long long n, int threads, int maxblocks) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > maxblocks) g = maxblocks;
  return (int)g;
}

struct Emit {
  msrcg_hier* h;
  cudaStream_t cs[kMaxLev + 2];
  int err = 0;
};

template <int DIM, typename RP>
void emit_pcg(Emit& E, int k, cudaStream_t s);

template <int DIM, typename RP>
void emit_precond(Emit& E, int k, cudaStream_t s) {
  msrcg_hier* h = E.h;
  const DevLevel& L = h->hL[k];
  const DevLevel& C = h->hL[k + 1];
  const int gmax = std::min(h->sms * 8, kMaxGrid);
  const long long npairs = (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
  const int gp = grid_for(npairs, kThreads, gmax), gc = grid_for(L.n, kThreads, gmax);
  const int m = h->o.m;
  // pre-smoothing from zero: red (black red)^m
  if (k == 0) {
    k_sweep<DIM, RP, double><<<gc, kThreads, 0, s>>>(L, 0, 1);
    for (int i = 0; i < m; ++i) {
      k_sweep<DIM, RP, double><<<gp, kThreads, 0, s>>>(L, 1, 0);
      k_sweep<DIM, RP, double><<<gp, kThreads, 0, s>>>(L, 0, 0);
    }
    k_residual<DIM, RP, double><<<gc, kThreads, 0, s>>>(L);
  } else {
    k_sweep<DIM, RP, RP><<<gc, kThreads, 0, s>>>(L, 0, 1);
    for (int i = 0; i < m; ++i) {
      k_sweep<DIM, RP, RP><<<gp, kThreads, 0, s>>>(L, 1, 0);
      k_sweep<DIM, RP, RP><<<gp, kThreads, 0, s>>>(L, 0, 0);
    }
    k_residual<DIM, RP, RP><<<gc, kThreads, 0, s>>>(L);
  }
  k_restrict<DIM, RP><<<grid_for(C.n, kThreads, gmax), kThreads, 0, s>>>(L, C);
  // coarse solve, A_c^-1 applied by the PCG one level down (Sec. 2.3)
  if (k + 1 < h->ks) {
    emit_pcg<DIM, RP>(E, k + 1, s);
  } else {
    k_small<DIM, RP><<<1, kSmallThreads, 0, s>>>(h->dP, nullptr, 1, k + 1, 0, nullptr);
  }
  k_prolong<DIM, RP><<<gc, kThreads, 0, s>>>(L, C);
  // post-smoothing: red (black red)^m
  if (k == 0) {
    k_sweep<DIM, RP, double><<<gp, kThreads, 0, s>>>(L, 0, 0);
    for (int i = 0; i < m; ++i) {
      k_sweep<DIM, RP, double><<<gp, kThreads, 0, s>>>(L, 1, 0);
      k_sweep<DIM, RP, double><<<gp, kThreads, 0, s>>>(L, 0, 0);
    }
  } else {
    k_sweep<DIM, RP, RP><<<gp, kThreads, 0, s>>>(L, 0, 0);
    for (int i = 0; i < m; ++i) {
      k_sweep<DIM, RP, RP><<<gp, kThreads, 0, s>>>(L, 1, 0);
      k_sweep<DIM, RP, RP><<<gp, kThreads, 0, s>>>(L, 0, 0);
    }
  }
}

template <int DIM, typename RP>
void emit_pcg(Emit& E, int k, cudaStream_t s) {
  msrcg_hier* h = E.h;
  const DevLevel& L = h->hL[k];
  const int gmax = std::min(h->sms * 8, kMaxGrid);
  const int gc = grid_for(L.n, kThreads, gmax);
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
  if (k == 0) k_init<double><<<gc, kThreads, 0, s>>>(L, k, h->dS, h->b0, part, hc);
  else k_init<RP><<<gc, kThreads, 0, s>>>(L, k, h->dS, nullptr, part, hc);
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
    k_rho<double, RP><<<gc, kThreads, 0, b>>>(L, k, h->dS, part);
    k_direction<double, RP><<<gc, kThreads, 0, b>>>(L, k, h->dS);
    k_apply_dot<DIM, double><<<gc, kThreads, 0, b>>>(L, k, h->dS, part);
    k_update<double><<<gc, kThreads, 0, b>>>(L, k, h->dS, part, hc);
  } else {
    k_rho<RP, RP><<<gc, kThreads, 0, b>>>(L, k, h->dS, part);
    k_direction<RP, RP><<<gc, kThreads, 0, b>>>(L, k, h->dS);
    k_apply_dot<DIM, RP><<<gc, kThreads, 0, b>>>(L, k, h->dS, part);
    k_update<RP><<<gc, kThreads, 0, b>>>(L, k, h->dS, part, hc);
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
  if (rc && getenv("MSRCG_DEBUG")) fprintf(stderr, "msrcg: graph build failed (step %d): %s\n", E.err,
                                           cudaGetErrorString(cudaGetLastError()));
  (void)cudaGetLastError();
  return rc;
}

int build_graph(msrcg_hier* h) {
  const bool f32 = h->o.precision == 1;
  if (h->dim == 2) return f32 ? build_graph_t<2, float>(h) : build_graph_t<2, double>(h);
  return f32 ? build_graph_t<3, float>(h) : build_graph_t<3, double>(h);
}

template <int DIM, typename RP>
void launch_small(const ProblemDesc* P, const int* order, int nprob, int ks, int mode, int* next, int grid, cudaStream_t s) {
  k_small<DIM, RP><<<grid, kSmallThreads, 0, s>>>(P, order, nprob, ks, mode, next);
}

void launch_small_any(int dim, bool f32, const ProblemDesc* P, const int* order, int nprob, int ks, int mode, int* next,
                      int grid, cudaStream_t s) {
  if (dim == 2) {
    if (f32) launch_small<2, float>(P, order, nprob, ks, mode, next, grid, s);
    else launch_small<2, double>(P, order, nprob, ks, mode, next, grid, s);
  } else {
    if (f32) launch_small<3, float>(P, order, nprob, ks, mode, next, grid, s);
    else launch_small<3, double>(P, order, nprob, ks, mode, next, grid, s);
  }
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
  pd.tol = tol;
  pd.work = h->N[0];
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
  {
    ProblemDesc pd = make_desc(h, b, x, tol);
    MSRCG_CUDA_TRY(cudaMemcpyAsync(h->dP, &pd, sizeof(pd), cudaMemcpyHostToDevice, s));
    const double floor2 = f32 ? h->o.inner_floor * h->o.inner_floor : 0.0;
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&h->dS->inner_floor2, &floor2, sizeof(double), cudaMemcpyHostToDevice, s));
  }
  SolveState hs;
  int restarts = 0;
  if (h->ks == 0) {
    // every level fits one CTA: one launch runs the whole solve
    launch_small_any(dim, f32, h->dP, nullptr, 1, 0, 2, nullptr, 1, s);
    MSRCG_CUDA_TRY(cudaGetLastError());
  } else {
    const int gmax = std::min(h->sms * 8, kMaxGrid);
    double* part = h->partials + (size_t)(kMaxLev - 1) * kMaxGrid;
    const int g0 = grid_for(h->N[0], kThreads, gmax);
    k_prepare<<<g0, kThreads, 0, s>>>(b, h->b0, h->xs, h->N[0], tol, h->dS, h->nlev, part);
    MSRCG_CUDA_TRY(cudaGetLastError());
    for (;;) {
      MSRCG_CUDA_TRY(cudaGraphLaunch(h->gexec, s));
      k_accumulate<<<g0, kThreads, 0, s>>>((const double*)h->hL[0].x, h->xs, h->N[0]);
      if (dim == 2) k_true_residual<2><<<g0, kThreads, 0, s>>>(h->hL[0], b, h->b0, h->xs, h->dS, part);
      else k_true_residual<3><<<g0, kThreads, 0, s>>>(h->hL[0], b, h->b0, h->xs, h->dS, part);
      MSRCG_CUDA_TRY(cudaGetLastError());
      if (!stats) break;
      MSRCG_CUDA_TRY(cudaMemcpyAsync(&hs, h->dS, sizeof(hs), cudaMemcpyDeviceToHost, s));
      MSRCG_CUDA_TRY(cudaStreamSynchronize(s));
      if (hs.status != 0 || hs.rr_true < hs.tau2 * hs.bb0 || restarts >= 3 || !(hs.bb0 > 0)) break;
      ++restarts;
    }
    MSRCG_CUDA_TRY(cudaMemcpyAsync(x, h->xs, sizeof(double) * h->N[0], cudaMemcpyDeviceToDevice, s));
  }
  if (stats) {
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&hs, h->dS, sizeof(hs), cudaMemcpyDeviceToHost, s));
    MSRCG_CUDA_TRY(cudaStreamSynchronize(s));
    fill_stats(h, hs, stats, restarts);
    for (int k = 0; k < h->nlev; ++k) {
      h->last_iters[k] = stats->iters[k];
      h->last_calls[k] = stats->calls[k];
    }
    return stats->status;
  }
  return MSRCG_OK;
}

extern "C" int msrcg_batch_solve(int count, msrcg_hier* const* hs, const double* const* b, double tol, double* const* x,
                                 msrcg_stats* stats, void* stream) {
  if (count < 0 || (count > 0 && (!hs || !b || !x)) || !(tol > 0.0)) return MSRCG_EINVAL;
  if (count == 0) return MSRCG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int dim = hs[0]->dim, prec = hs[0]->o.precision;
  std::vector<ProblemDesc> pds(count);
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b[i] || !x[i] || hs[i]->dim != dim || hs[i]->o.precision != prec) return MSRCG_EINVAL;
    pds[i] = make_desc(hs[i], b[i], x[i], tol);
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
  int sms = hs[0]->sms, per = 0;
  if (dim == 2) {
    if (prec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<2, float>, kSmallThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<2, double>, kSmallThreads, 0);
  } else {
    if (prec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<3, float>, kSmallThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_small<3, double>, kSmallThreads, 0);
  }
  int grid = std::max(1, std::min(count, sms * std::max(per, 1)));
  launch_small_any(dim, prec == 1, (const ProblemDesc*)dp, (const int*)dord, count, 0, 1, (int*)dnext, grid, s);
  MSRCG_CUDA_TRY(cudaGetLastError());
  int rc = MSRCG_OK;
  std::vector<SolveState> st(count);
  for (int i = 0; i < count; ++i)
    MSRCG_CUDA_TRY(cudaMemcpyAsync(&st[i], hs[i]->dS, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  MSRCG_CUDA_TRY(cudaFreeAsync(dp, s));
  MSRCG_CUDA_TRY(cudaFreeAsync(dord, s));
  MSRCG_CUDA_TRY(cudaFreeAsync(dnext, s));
  MSRCG_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) {
    msrcg_stats one;
    fill_stats(hs[i], st[i], &one, 0);
    if (stats) stats[i] = one;
    for (int k = 0; k < hs[i]->nlev; ++k) {
      hs[i]->last_iters[k] = one.iters[k];
      hs[i]->last_calls[k] = one.calls[k];
    }
    if (one.status && !rc) rc = one.status;
  }
  return rc;
}
