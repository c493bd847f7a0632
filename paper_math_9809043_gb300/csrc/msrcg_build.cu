// Hierarchy build of libmsrcg (Sec. 2.2 and Sec. 3 of Lackner & Menikoff):
// face transmissibilities, series-parallel coarse transmissibilities of every
// level, transfer tables, the exact inverse of the coarsest operator, plus
// the lifting right-hand side, the FP64 operator apply and bookkeeping.
//
// The build kernels use explicitly rounded FP64 operations (__dmul_rn and
// friends) so that no multiply-add is fused: the transmissibilities are then
// reproducible to the bit on any device and compiler setting.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "msrcg_internal.cuh"

using namespace msrcg;

int msrcg_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("MSRCG_DEBUG")) fprintf(stderr, "msrcg: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? MSRCG_ENOMEM : MSRCG_ECUDA;
}

int msrcg_alloc(msrcg_hier* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  // stream-ordered when the hierarchy has an allocation stream (the server),
  // plain cudaMalloc otherwise
  cudaError_t e = h->alloc_stream ? cudaMallocAsync(p, bytes, h->alloc_stream) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return MSRCG_ENOMEM;
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return MSRCG_OK;
}

int msrcg_status_from_bits(int bits) {
  if (bits & kStNanInf) return MSRCG_ENANINF;
  if (bits & kStTimeout) return MSRCG_ETIMEOUT;
  if (bits & kStBreakdown) return MSRCG_EBREAKDOWN;
  if (bits & kStNoConv) return MSRCG_ENOCONV;
  return MSRCG_OK;
}

namespace {

// ---------------------------------------------------------------------------
// Level sides: scale factor s (~4) adjusted to integer sizes, Sec. 3.  An axis
// longer than the coarsest side limit shrinks to max(2, floor(n/s + 1/2));
// the hierarchy ends when no axis is longer than the limit.
// ---------------------------------------------------------------------------
int level_sides(int dim, const int n[3], const double h[3], int s, int limit, int rule, int out[][3]) {
  int cur[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  double La[3] = {0.0, 0.0, 0.0};  // axis lengths, fixed over the levels
  for (int a = 0; a < dim; ++a) La[a] = (double)n[a] * h[a];
  int nl = 0;
  for (;;) {
    if (nl >= kMaxLev) return -1;
    for (int a = 0; a < 3; ++a) out[nl][a] = cur[a];
    ++nl;
    bool longer = false;
    for (int a = 0; a < dim; ++a) longer = longer || cur[a] > limit;
    if (!longer) return nl;
    // rule 1: coarse cells of size s * (smallest cell size of the level),
    // each axis rounded and never refined; when no axis changes, this level
    // is the coarsest
    double hmin = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double ha = La[a] / (double)cur[a];
      if (a == 0 || ha < hmin) hmin = ha;
    }
    int next[3] = {cur[0], cur[1], cur[2]};
    bool moved = false;
    for (int a = 0; a < dim; ++a)
      if (cur[a] > limit) {
        int c;
        if (rule == 0) {
          c = (2 * cur[a] + s) / (2 * s);
        } else {
          const double t = La[a] / ((double)s * hmin);
          c = (int)floor(t + 0.5);
          if (c > cur[a]) c = cur[a];
        }
        next[a] = std::max(2, c);
        moved = moved || next[a] != cur[a];
      }
    if (rule == 1 && !moved) return nl;
    for (int a = 0; a < 3; ++a) cur[a] = next[a];
  }
}

// Zero-slope linear interpolation between cell centres along one axis of
// the unit interval, Sec. 3: fine centre (i+1/2)/nf sits at coarse coordinate
// t = ((2i+1) nc - nf) / (2 nf) in units of the coarse spacing, measured from
// the first coarse centre.  Outside [0, nc-1] the end value is held.
struct Axis1D {
  std::vector<int> c0, c1, lo, hi;
  std::vector<double> w, rw;  // rw: restriction weights, W per coarse cell
  int W = 1;
};

// interp 1: piecewise constant (Sec. 3) -- the coarse cell holding the fine
// centre, floor((2i+1) nc / (2 nf)), weight 1.
Axis1D axis_tables(int nf, int nc, int interp) {
  Axis1D A;
  A.c0.resize(nf);
  A.c1.resize(nf);
  A.w.resize(nf);
  const long long den = 2LL * nf;
  for (int i = 0; i < nf; ++i) {
    long long num = (2LL * i + 1) * nc - nf;
    int a, b;
    double w;
    if (interp == 1) {
      a = b = (int)(((2LL * i + 1) * nc) / den);
      w = 0.0;
    } else if (num <= 0) {
      a = b = 0;
      w = 0.0;
    } else if (num / den >= nc - 1) {
      a = b = nc - 1;
      w = 0.0;
    } else if (num % den == 0) {
      a = b = (int)(num / den);
      w = 0.0;
    } else {
      a = (int)(num / den);
      b = a + 1;
      w = (double)(num % den) / (double)den;
    }
    A.c0[i] = a;
    A.c1[i] = b;
    A.w[i] = w;
  }
  // restriction windows: fine cells with a non-zero weight on coarse cell I
  A.lo.assign(nc, nf);
  A.hi.assign(nc, -1);
  for (int i = 0; i < nf; ++i) {
    int cs[2] = {A.c0[i], A.c1[i]};
    double ws[2] = {1.0 - A.w[i], A.w[i]};
    for (int e = 0; e < 2; ++e) {
      if (ws[e] == 0.0 && !(e == 0 && A.c0[i] == A.c1[i])) continue;
      A.lo[cs[e]] = std::min(A.lo[cs[e]], i);
      A.hi[cs[e]] = std::max(A.hi[cs[e]], i);
    }
  }
  A.W = 1;
  for (int I = 0; I < nc; ++I) A.W = std::max(A.W, A.hi[I] - A.lo[I] + 1);
  A.rw.assign((size_t)nc * A.W, 0.0);
  for (int I = 0; I < nc; ++I)
    for (int i = A.lo[I]; i <= A.hi[I]; ++i) {
      double v = 0.0;
      if (A.c0[i] == I) v += 1.0 - A.w[i];
      if (A.c1[i] == I) v += A.w[i];
      A.rw[(size_t)I * A.W + (i - A.lo[I])] = v;
    }
  return A;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Face transmissibilities, Sec. 3: T = (h_perp/h_par) K_face; K_face is the
// harmonic mean 2 K_L K_R / (K_L + K_R) of the adjacent cells; a Dirichlet
// boundary face (half a cell from the centre) has 2 (h_perp/h_par) K_cell, a
// Neumann face 0.
__global__ void k_face_trans(int ax, int nx, int ny, int nz, double ratio, const double* __restrict__ K,
                             const uint8_t* __restrict__ blo, const uint8_t* __restrict__ bhi,
                             double* __restrict__ T) {
  const int fx = nx + (ax == 0), fy = ny + (ax == 1), fz = nz + (ax == 2);
  const long long nf = (long long)fx * fy * fz;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    int i = (int)(f % fx);
    long long rest = f / fx;
    int j = (int)(rest % fy);
    int k = (int)(rest / fy);
    int g[3] = {i, j, k}, lim[3] = {nx, ny, nz};
    int e = g[ax];
    double t;
    if (e == 0 || e == lim[ax]) {
      // boundary face: index of the face inside its block
      long long bi;
      if (ax == 0) bi = j + (long long)ny * k;
      else if (ax == 1) bi = i + (long long)nx * k;
      else bi = i + (long long)nx * j;
      const uint8_t* msk = e == 0 ? blo : bhi;
      int gc[3] = {i, j, k};
      gc[ax] = e == 0 ? 0 : lim[ax] - 1;
      double kc = K[gc[0] + (long long)nx * (gc[1] + (long long)ny * gc[2])];
      t = msk[bi] ? __dmul_rn(ratio, __dmul_rn(2.0, kc)) : 0.0;
    } else {
      int gl[3] = {i, j, k};
      gl[ax] = e - 1;
      int gr[3] = {i, j, k};
      gr[ax] = e;
      double kl = K[gl[0] + (long long)nx * (gl[1] + (long long)ny * gl[2])];
      double kr = K[gr[0] + (long long)nx * (gr[1] + (long long)ny * gr[2])];
      double s = __dadd_rn(kl, kr);
      t = s > 0.0 ? __dmul_rn(ratio, __ddiv_rn(__dmul_rn(__dmul_rn(2.0, kl), kr), s)) : 0.0;
    }
    T[f] = t;
  }
}

// Face transmissibilities from face permeabilities (Sec. 3: K is face
// centred and its boundary faces carry the boundary condition): T =
// (h_perp/h_par) K_face on every face.
__global__ void k_face_scale(long long nf, double ratio, const double* __restrict__ Kf, double* __restrict__ T) {
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x)
    T[f] = __dmul_rn(ratio, Kf[f]);
}

__device__ __forceinline__ long long d_overlap(long long a0, long long a1, long long b0, long long b1) {
  long long lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
  return hi > lo ? hi - lo : 0;
}

// Coarse transmissibility of the faces normal to axis `ax`, Sec. 3:
//   1/T^c = sum_i 1/C_i,  C_i = (w_i / o_i) * sum_j (o_j / h_j) T(i, j)
// i runs over the fine faces along the normal whose conductor block (between
// adjacent cell centres, half a cell at the boundary) overlaps the coarse
// face's block by o_i (w_i = the fine block's width); j runs over the fine
// faces across the coarse face, weighted by the fraction of their extent
// inside it.  Lengths along an axis with nf fine / nc coarse cells are exact
// integers in units of 1/(2 nf nc) of the unit interval.  One thread per
// coarse face; sums run in ascending index order, one rounding per operation.
__global__ void k_upscale(int ax, int3 nf, int3 nc, const double* __restrict__ Tf, double* __restrict__ Tc) {
  const int p1 = (ax + 1) % 3, p2 = (ax + 2) % 3;
  const int F[3] = {nf.x, nf.y, nf.z}, Cn[3] = {nc.x, nc.y, nc.z};
  int fd[3] = {F[0], F[1], F[2]}, cd[3] = {Cn[0], Cn[1], Cn[2]};
  fd[ax] += 1;
  cd[ax] += 1;
  const long long ncf = (long long)cd[0] * cd[1] * cd[2];
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < ncf; f += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(f % cd[0]);
    long long rest = f / cd[0];
    c[1] = (int)(rest % cd[1]);
    c[2] = (int)(rest / cd[1]);
    const long long nfa = F[ax], nca = Cn[ax], L = 2 * nfa * nca;
    long long clo = (2LL * c[ax] - 1) * nfa, chi = (2LL * c[ax] + 1) * nfa;
    clo = clo < 0 ? 0 : clo;
    chi = chi > L ? L : chi;
    // fine faces i whose block [(2i-1) nc, (2i+1) nc] can meet [clo, chi]
    long long ia = (clo / nca - 1) / 2 - 1, ib = (chi / nca + 1) / 2 + 1;
    ia = ia < 0 ? 0 : ia;
    ib = ib > nfa ? nfa : ib;
    // fine cells j along p1 / p2 that can meet coarse cell c[p]
    auto win = [](int J, int nf_, int nc_, int* lo, int* hi) {
      long long a = ((long long)J * nf_) / nc_ - 1, b = (((long long)J + 1) * nf_) / nc_ + 1;
      *lo = a < 0 ? 0 : (int)a;
      *hi = b > nf_ - 1 ? nf_ - 1 : (int)b;
    };
    int alo, ahi, blo, bhi;
    win(c[p1], F[p1], Cn[p1], &alo, &ahi);
    win(c[p2], F[p2], Cn[p2], &blo, &bhi);
    double inv = 0.0;
    bool zero = false, any = false;
    for (long long i = ia; i <= ib && !zero; ++i) {
      long long flo = (2 * i - 1) * nca, fhi = (2 * i + 1) * nca;
      flo = flo < 0 ? 0 : flo;
      fhi = fhi > L ? L : fhi;
      long long o = d_overlap(flo, fhi, clo, chi);
      if (o == 0) continue;
      any = true;
      double S = 0.0;
      for (int b = blo; b <= bhi; ++b) {
        long long o2 = d_overlap(2LL * b * Cn[p2], 2LL * (b + 1) * Cn[p2], 2LL * c[p2] * F[p2], 2LL * (c[p2] + 1) * F[p2]);
        if (o2 == 0) continue;
        double f2 = __ddiv_rn((double)o2, (double)(2LL * Cn[p2]));
        double inner = 0.0;
        for (int a = alo; a <= ahi; ++a) {
          long long o1 = d_overlap(2LL * a * Cn[p1], 2LL * (a + 1) * Cn[p1], 2LL * c[p1] * F[p1], 2LL * (c[p1] + 1) * F[p1]);
          if (o1 == 0) continue;
          double f1 = __ddiv_rn((double)o1, (double)(2LL * Cn[p1]));
          int g[3];
          g[ax] = (int)i;
          g[p1] = a;
          g[p2] = b;
          double t = Tf[g[0] + (long long)fd[0] * (g[1] + (long long)fd[1] * g[2])];
          inner = __dadd_rn(inner, __dmul_rn(f1, t));
        }
        S = __dadd_rn(S, __dmul_rn(f2, inner));
      }
      double C = __ddiv_rn(__dmul_rn(S, (double)(fhi - flo)), (double)o);
      if (C == 0.0) {
        zero = true;
        break;
      }
      inv = __dadd_rn(inv, __ddiv_rn(1.0, C));
    }
    Tc[f] = (zero || !any) ? 0.0 : __ddiv_rn(1.0, inv);
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Dense operator of a (small) level: A[c][c] = sum of its face T,
// A[c][nb] = -T_face.  Row-major n x n.  lap: compact face arrays.
__global__ void k_dense_assemble(int nx, int ny, int nz, int lap, const double* __restrict__ Tx,
                                 const double* __restrict__ Ty, const double* __restrict__ Tz, double* __restrict__ A) {
  const long long n = (long long)nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n; e += (long long)gridDim.x * blockDim.x)
    A[e] = 0.0;
  __syncthreads();
  for (long long c = threadIdx.x; c < n; c += blockDim.x) {
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    double d = 0.0, t;
    t = Tx[face_index(lap, 0, nx, ny, nz, i, j, k)];
    d += t;
    if (i > 0) A[c * n + c - 1] = -t;
    t = Tx[face_index(lap, 0, nx, ny, nz, i + 1, j, k)];
    d += t;
    if (i < nx - 1) A[c * n + c + 1] = -t;
    t = Ty[face_index(lap, 1, nx, ny, nz, i, j, k)];
    d += t;
    if (j > 0) A[c * n + c - nx] = -t;
    t = Ty[face_index(lap, 1, nx, ny, nz, i, j + 1, k)];
    d += t;
    if (j < ny - 1) A[c * n + c + nx] = -t;
    if (Tz) {
      long long pl = (long long)nx * ny;
      t = Tz[face_index(lap, 2, nx, ny, nz, i, j, k)];
      d += t;
      if (k > 0) A[c * n + c - pl] = -t;
      t = Tz[face_index(lap, 2, nx, ny, nz, i, j, k + 1)];
      d += t;
      if (k < nz - 1) A[c * n + c + pl] = -t;
    }
    A[c * n + c] = d;
  }
}

// In-place Cholesky A = C C^T (lower), then the explicit inverse, by one
// CTA in FP64.  The coarsest level is solved exactly (Sec. 2.2 / 2.3); the
// inverse turns each coarsest solve into one matrix-vector product.
__global__ void k_chol_inverse(int n, double* __restrict__ A, double* __restrict__ Ainv, int* __restrict__ fail) {
  __shared__ double piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = A[(long long)j * n + j];
      if (!(d > 0.0)) *fail = 1;
      piv = sqrt(d > 0.0 ? d : 1.0);
      A[(long long)j * n + j] = piv;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(long long)i * n + j] /= piv;
    __syncthreads();
    const int m = n - j - 1;
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      int i = j + 1 + (int)(e / m), k = j + 1 + (int)(e % m);
      if (k <= i) A[(long long)i * n + k] -= A[(long long)i * n + j] * A[(long long)k * n + j];
    }
    __syncthreads();
  }
  // column c of the inverse: solve C y = e_c, C^T x = y (x stored in Ainv[:, c])
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= A[(long long)i * n + k] * Ainv[(long long)k * n + c];
      Ainv[(long long)i * n + c] = s / A[(long long)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = Ainv[(long long)i * n + c];
      for (int k = i + 1; k < n; ++k) s -= A[(long long)k * n + i] * Ainv[(long long)k * n + c];
      Ainv[(long long)i * n + c] = s / A[(long long)i * n + i];
    }
  }
}

// y = A x with FP64 transmissibilities: (A x)_c = sum_faces T (x_c - x_nb),
// T x_c on a boundary face.  lap: compact face arrays.
__global__ void k_apply64(int nx, int ny, int nz, int lap, const double* __restrict__ Tx, const double* __restrict__ Ty,
                          const double* __restrict__ Tz, const double* __restrict__ x, double* __restrict__ y) {
  const long long n = (long long)nx * ny * nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    double xc = x[c], s = 0.0, t;
    t = Tx[face_index(lap, 0, nx, ny, nz, i, j, k)];
    s += i > 0 ? t * (xc - x[c - 1]) : t * xc;
    t = Tx[face_index(lap, 0, nx, ny, nz, i + 1, j, k)];
    s += i < nx - 1 ? t * (xc - x[c + 1]) : t * xc;
    t = Ty[face_index(lap, 1, nx, ny, nz, i, j, k)];
    s += j > 0 ? t * (xc - x[c - nx]) : t * xc;
    t = Ty[face_index(lap, 1, nx, ny, nz, i, j + 1, k)];
    s += j < ny - 1 ? t * (xc - x[c + nx]) : t * xc;
    if (Tz) {
      long long pl = (long long)nx * ny;
      t = Tz[face_index(lap, 2, nx, ny, nz, i, j, k)];
      s += k > 0 ? t * (xc - x[c - pl]) : t * xc;
      t = Tz[face_index(lap, 2, nx, ny, nz, i, j, k + 1)];
      s += k < nz - 1 ? t * (xc - x[c + pl]) : t * xc;
    }
    y[c] = s;
  }
}

// Lifted right-hand side, Sec. 3: b = f vol + g_D - A P_bf.  lap: compact
// face arrays.
__global__ void k_lift(int nx, int ny, int nz, int lap, const double* __restrict__ Tx, const double* __restrict__ Ty,
                       const double* __restrict__ Tz, const uint8_t* __restrict__ bc, const double* __restrict__ gD,
                       const double* __restrict__ f, double vol, const double* __restrict__ pbf, double* __restrict__ b) {
  const long long n = (long long)nx * ny * nz;
  const long long nyz = (long long)ny * nz, nxz = (long long)nx * nz, nxy = (long long)nx * ny;
  const long long ox1 = nyz, oy0 = 2 * nyz, oy1 = 2 * nyz + nxz, oz0 = 2 * nyz + 2 * nxz, oz1 = oz0 + nxy;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / nxy);
    long long row = j + (long long)ny * k;
    const double tw = Tx[face_index(lap, 0, nx, ny, nz, i, j, k)], te = Tx[face_index(lap, 0, nx, ny, nz, i + 1, j, k)];
    const double ts = Ty[face_index(lap, 1, nx, ny, nz, i, j, k)], tn = Ty[face_index(lap, 1, nx, ny, nz, i, j + 1, k)];
    double v = f ? f[c] * vol : 0.0;
    if (i == 0 && bc[row]) v += tw * gD[row];
    if (i == nx - 1 && bc[ox1 + row]) v += te * gD[ox1 + row];
    long long xz = i + (long long)nx * k;
    if (j == 0 && bc[oy0 + xz]) v += ts * gD[oy0 + xz];
    if (j == ny - 1 && bc[oy1 + xz]) v += tn * gD[oy1 + xz];
    double tb = 0.0, tt = 0.0;
    if (Tz) {
      tb = Tz[face_index(lap, 2, nx, ny, nz, i, j, k)];
      tt = Tz[face_index(lap, 2, nx, ny, nz, i, j, k + 1)];
      long long xy = i + (long long)nx * j;
      if (k == 0 && bc[oz0 + xy]) v += tb * gD[oz0 + xy];
      if (k == nz - 1 && bc[oz1 + xy]) v += tt * gD[oz1 + xy];
    }
    // A P_bf
    double xc = pbf[c], s = 0.0;
    s += i > 0 ? tw * (xc - pbf[c - 1]) : tw * xc;
    s += i < nx - 1 ? te * (xc - pbf[c + 1]) : te * xc;
    s += j > 0 ? ts * (xc - pbf[c - nx]) : ts * xc;
    s += j < ny - 1 ? tn * (xc - pbf[c + nx]) : tn * xc;
    if (Tz) {
      s += k > 0 ? tb * (xc - pbf[c - nxy]) : tb * xc;
      s += k < nz - 1 ? tt * (xc - pbf[c + nxy]) : tt * xc;
    }
    b[c] = v - s;
  }
}

// Full face array of axis a of a constant-coefficient level from its compact
// one (msrcg_get_trans).
__global__ void k_expand_faces(int a, int nx, int ny, int nz, const double* __restrict__ Tc, double* __restrict__ T) {
  const int fx = nx + (a == 0), fy = ny + (a == 1), fz = nz + (a == 2);
  const long long nf = (long long)fx * fy * fz;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(f % fx), j = (int)((f / fx) % fy), k = (int)(f / ((long long)fx * fy));
    T[f] = Tc[face_index(1, a, nx, ny, nz, i, j, k)];
  }
}

int grid_for(long long n, int threads, int maxblocks) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > maxblocks) g = maxblocks;
  return (int)g;
}

// Upload a host table on the build stream (the pageable source is consumed
// before the call returns).
template <typename T>
int upload(msrcg_hier* h, const std::vector<T>& v, const void** out, cudaStream_t st) {
  void* p;
  int rc = msrcg_alloc(h, &p, sizeof(T) * v.size());
  if (rc) return rc;
  MSRCG_CUDA_TRY(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  *out = p;
  return MSRCG_OK;
}

void release(msrcg_hier* h) {
  if (!h) return;
  if (h->twin) {
    h->twin->alloc_stream = h->alloc_stream;
    release(h->twin);
    h->twin = nullptr;
  }
  if (h->alloc_stream) {
    // stream-ordered: freed after the work already queued on that stream
    for (void* p : h->allocs) cudaFreeAsync(p, h->alloc_stream);
  } else {
    cudaDeviceSynchronize();
    for (void* p : h->allocs) cudaFree(p);
  }
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  (void)cudaGetLastError();
  delete h;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" int msrcg_default_opts(msrcg_opts* o) {
  if (!o) return MSRCG_EINVAL;
  memset(o, 0, sizeof(*o));
  o->scale = 4;
  o->m = 4;
  o->f = 0.1;
  o->coarsest_max_side = 0;
  o->precision = 0;
  o->maxit_outer = 200;
  o->maxit_inner = 500;
  o->timeout_ns = 2000000000ull;
  o->inner_floor = 0.0;
  o->small_cells = 0;
  o->plain_sweeps = 0;
  o->fuse_width = 0;
  o->fuse_min_cells = 0;
  o->splitting = 0;
  o->coarsening = 0;
  o->interp = 0;
  o->stall_iters = 0;
  o->escalate = 1;
  o->flexible = 0;
  o->precond = 0;
  return MSRCG_OK;
}

extern "C" const char* msrcg_strerror(int code) {
  switch (code) {
    case MSRCG_OK: return "ok";
    case MSRCG_EINVAL: return "invalid argument";
    case MSRCG_ENOMEM: return "device allocation failed";
    case MSRCG_ENOCONV: return "iteration cap reached before the level tolerance";
    case MSRCG_EBREAKDOWN: return "conjugate gradient breakdown (p.Ap <= 0 or non-finite scalar)";
    case MSRCG_ETIMEOUT: return "bounded device wait timed out";
    case MSRCG_ENANINF: return "non-finite value in the right-hand side";
    case MSRCG_ECUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

extern "C" int msrcg_build(const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                           const msrcg_opts* opts, void* stream, msrcg_hier** out) {
  return msrcg_build_ex(grid, K, ncomp, bc, opts, (cudaStream_t)stream, nullptr, out);
}

namespace {
// Permeability of level 0: cell values with boundary types, or face values
// (Kf[0] set) whose boundary faces carry the boundary condition.
struct Level0K {
  const double* K = nullptr;
  int ncomp = 1;
  const uint8_t* bc = nullptr;
  const double* Kf[3] = {nullptr, nullptr, nullptr};
  const double* T0[3] = {nullptr, nullptr, nullptr};  // level-0 transmissibilities of another hierarchy
  // constant coefficients: K per axis and the boundary type of each side
  // (x-low, x-high, y-low, y-high, z-low, z-high; 1 = Dirichlet)
  bool lap = false;
  double lapK[3] = {0.0, 0.0, 0.0};
  uint8_t lap_bc[6] = {0, 0, 0, 0, 0, 0};
};
int build_hier(const msrcg_grid* grid, const Level0K& src, const msrcg_opts* opts, cudaStream_t stream,
               cudaStream_t alloc_stream, msrcg_hier** out);
}  // namespace

int msrcg_build_ex(const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc, const msrcg_opts* opts,
                   cudaStream_t stream, cudaStream_t alloc_stream, msrcg_hier** out) {
  if (!out) return MSRCG_EINVAL;
  *out = nullptr;
  if (!grid || !K || !bc) return MSRCG_EINVAL;
  if (ncomp != 1 && ncomp != grid->dim) return MSRCG_EINVAL;
  Level0K src;
  src.K = K;
  src.ncomp = ncomp;
  src.bc = bc;
  return build_hier(grid, src, opts, stream, alloc_stream, out);
}

extern "C" int msrcg_build_faces(const msrcg_grid* grid, const double* Kx, const double* Ky, const double* Kz,
                                 const msrcg_opts* opts, void* stream, msrcg_hier** out) {
  if (!out) return MSRCG_EINVAL;
  *out = nullptr;
  if (!grid || !Kx || !Ky || (grid->dim == 3 && !Kz)) return MSRCG_EINVAL;
  Level0K src;
  src.Kf[0] = Kx;
  src.Kf[1] = Ky;
  src.Kf[2] = grid->dim == 3 ? Kz : nullptr;
  return build_hier(grid, src, opts, (cudaStream_t)stream, nullptr, out);
}

int msrcg_twin(msrcg_hier* h, cudaStream_t stream, msrcg_hier** out) {
  if (!h->twin) {
    msrcg_grid g;
    g.dim = h->dim;
    for (int a = 0; a < 3; ++a) {
      g.n[a] = h->dims[0][a];
      g.h[a] = h->hsz[a];
    }
    msrcg_opts o = h->o;
    o.precision = 0;
    o.inner_floor = 0.0;
    o.escalate = 0;
    Level0K src;
    if (h->lap) {
      src.lap = true;
      for (int a = 0; a < 3; ++a) src.lapK[a] = h->lapK[a];
      for (int e = 0; e < 6; ++e) src.lap_bc[e] = h->lap_bc[e];
    } else {
      for (int a = 0; a < h->dim; ++a) src.T0[a] = h->T64[0][a];
    }
    // stream-ordered allocation (the server): build on the allocation stream,
    // so that every buffer exists before its first use; the build
    // synchronises that stream before it returns
    int rc = build_hier(&g, src, &o, h->alloc_stream ? h->alloc_stream : stream, h->alloc_stream, &h->twin);
    if (rc) return rc;
  }
  *out = h->twin;
  return MSRCG_OK;
}

extern "C" int msrcg_build_laplace(const msrcg_grid* grid, const double K[3], const uint8_t side_bc[6],
                                   const msrcg_opts* opts, void* stream, msrcg_hier** out) {
  if (!out) return MSRCG_EINVAL;
  *out = nullptr;
  if (!grid || !K || !side_bc || (grid->dim != 2 && grid->dim != 3)) return MSRCG_EINVAL;
  Level0K src;
  src.lap = true;
  for (int a = 0; a < 3; ++a) {
    src.lapK[a] = a < grid->dim ? K[a] : 0.0;
    if (a < grid->dim && !(K[a] > 0.0 && isfinite(K[a]))) return MSRCG_EINVAL;
  }
  for (int e = 0; e < 6; ++e) {
    if (side_bc[e] > 1) return MSRCG_EINVAL;
    src.lap_bc[e] = e < 2 * grid->dim ? side_bc[e] : 0;
  }
  return build_hier(grid, src, opts, (cudaStream_t)stream, nullptr, out);
}

namespace {
int build_hier(const msrcg_grid* grid, const Level0K& src, const msrcg_opts* opts, cudaStream_t stream,
               cudaStream_t alloc_stream, msrcg_hier** out) {
  const double* K = src.K;
  const int ncomp = src.ncomp;
  const uint8_t* bc = src.bc;
  const int dim = grid->dim;
  if (dim != 2 && dim != 3) return MSRCG_EINVAL;
  for (int a = 0; a < dim; ++a)
    if (grid->n[a] < 1 || !(grid->h[a] > 0.0) || !isfinite(grid->h[a])) return MSRCG_EINVAL;
  msrcg_opts o;
  if (opts) o = *opts;
  else msrcg_default_opts(&o);
  if (o.scale < 2 || o.m < 1 || !(o.f > 0.0) || o.maxit_outer < 1 || o.maxit_inner < 1 || o.fuse_width < 0 ||
      o.fuse_min_cells < 0 || o.splitting < 0 || o.splitting > 2 || o.coarsening < 0 || o.coarsening > 1 ||
      o.interp < 0 || o.interp > 1 || o.escalate < 0 || o.escalate > 1 || o.flexible < 0 || o.flexible > 1 ||
      o.precond < 0 || o.precond > 2)
    return MSRCG_EINVAL;
  if (o.precision != 0 && o.precision != 1) return MSRCG_EINVAL;
  if (o.coarsest_max_side <= 0) o.coarsest_max_side = dim == 2 ? 8 : 4;
  if (o.timeout_ns == 0) o.timeout_ns = 2000000000ull;
  if (o.small_cells <= 0) o.small_cells = o.precision == 1 ? 4096 : 4096;
  cudaStream_t st = (cudaStream_t)stream;

  msrcg_hier* h = new msrcg_hier();
  h->alloc_stream = alloc_stream;
  h->dim = dim;
  h->o = o;
  for (int a = 0; a < 3; ++a) h->hsz[a] = a < dim ? grid->h[a] : 1.0;
  int rc = MSRCG_OK;
  auto fail = [&](int code) {
    release(h);
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) return fail(MSRCG_ECUDA);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  int n3[3] = {grid->n[0], grid->n[1], dim == 3 ? grid->n[2] : 1};
  {
    const double h3[3] = {grid->h[0], grid->h[1], dim == 3 ? grid->h[2] : 1.0};
    h->nlev = level_sides(dim, n3, h3, o.scale, o.coarsest_max_side, o.coarsening, h->dims);
  }
  if (h->nlev < 1) return fail(MSRCG_EINVAL);
  for (int k = 0; k < h->nlev; ++k) h->N[k] = (long long)h->dims[k][0] * h->dims[k][1] * h->dims[k][2];
  if ((long long)(n3[0] + 2) * (n3[1] + 2) * (n3[2] + 2) >= (1LL << 31)) return fail(MSRCG_EINVAL);
  if (h->N[h->nlev - 1] > 1024) return fail(MSRCG_EINVAL);
  h->ks = h->nlev - 1;
  while (h->ks > 0 && h->N[h->ks - 1] <= o.small_cells) --h->ks;
  // the natural-order smoother runs plane by plane inside one CTA: every
  // level of a single solve goes to the single-CTA solver
  if (o.splitting == 2) h->ks = 0;
  // so do the multigrid and polynomial preconditioners
  if (o.precond != 0) h->ks = 0;

  const bool f32 = o.precision == 1;
  const size_t rsz = f32 ? sizeof(float) : sizeof(double);
  const int gmax = std::min(h->sms * 8, kMaxGrid);

  // ---- level 0 transmissibilities from cell K (A1) ----
  double hh[3] = {grid->h[0], grid->h[1], dim == 3 ? grid->h[2] : 1.0};
  double ratio[3] = {(hh[1] * hh[2]) / hh[0], (hh[0] * hh[2]) / hh[1], (hh[0] * hh[1]) / hh[2]};
  h->lap = src.lap ? 1 : 0;
  if (src.lap) {
    for (int a = 0; a < 3; ++a) h->lapK[a] = src.lapK[a];
    for (int e = 0; e < 6; ++e) h->lap_bc[e] = src.lap_bc[e];
  }
  // entries of level k's face array along axis a (compact when constant)
  auto nfaces = [&](int k, int a) -> long long {
    DevLevel t;
    memset(&t, 0, sizeof(t));
    t.nx = h->dims[k][0];
    t.ny = h->dims[k][1];
    t.nz = h->dims[k][2];
    t.lap = h->lap;
    return face_count(t, a);
  };
  for (int k = 0; k < h->nlev; ++k) {
    for (int a = 0; a < dim; ++a) {
      void* p;
      if ((rc = msrcg_alloc(h, &p, sizeof(double) * nfaces(k, a)))) return fail(rc);
      h->T64[k][a] = (double*)p;
    }
  }
  if (src.lap) {
    // constant coefficients (Sec. 4.1, the Laplace specialisation): every
    // level's interior faces carry (h_perp/h_par) K_face of that level's cells
    // (the domain fixed, the cells of level k of size L_a / n_a(k); K_face the
    // harmonic mean of two equal cells, formed as the cell-K build forms it),
    // a Dirichlet boundary face 2 (h_perp/h_par) K, a Neumann face 0 -- the
    // transmissibilities that the series-parallel coarsening of a constant
    // field reproduces
    std::vector<double> buf;
    for (int k = 0; k < h->nlev; ++k) {
      double hk[3];
      for (int a = 0; a < 3; ++a) hk[a] = a < dim ? hh[a] * n3[a] / (double)h->dims[k][a] : 1.0;
      const double rk[3] = {(hk[1] * hk[2]) / hk[0], (hk[0] * hk[2]) / hk[1], (hk[0] * hk[1]) / hk[2]};
      for (int a = 0; a < dim; ++a) {
        const double K = src.lapK[a];
        const double c = K + K > 0.0 ? rk[a] * (2.0 * K * K / (K + K)) : 0.0;
        const double lo = src.lap_bc[2 * a] ? rk[a] * (2.0 * K) : 0.0;
        const double hi = src.lap_bc[2 * a + 1] ? rk[a] * (2.0 * K) : 0.0;
        const int nx = h->dims[k][0], ny = h->dims[k][1], nz = h->dims[k][2];
        buf.assign((size_t)nfaces(k, a), c);
        if (a == 0) {
          buf[0] = lo;
          buf[nx] = hi;
        } else {
          const long long row = a == 1 ? nx : (long long)nx * ny;  // one compact row / plane
          const int n = a == 1 ? ny : nz;
          for (long long e = 0; e < row; ++e) {
            buf[e] = lo;
            buf[(size_t)row * (n == 1 ? 1 : 3) + e] = hi;
          }
        }
        if (cudaMemcpy(h->T64[k][a], buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice) != cudaSuccess)
          return fail(MSRCG_ECUDA);
      }
    }
  } else if (src.T0[0]) {
    for (int a = 0; a < dim; ++a) {
      long long nf = (long long)(n3[0] + (a == 0)) * (n3[1] + (a == 1)) * (n3[2] + (a == 2));
      if (cudaMemcpyAsync(h->T64[0][a], src.T0[a], sizeof(double) * nf, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(MSRCG_ECUDA);
    }
  } else if (src.Kf[0]) {
    for (int a = 0; a < dim; ++a) {
      long long nf = (long long)(n3[0] + (a == 0)) * (n3[1] + (a == 1)) * (n3[2] + (a == 2));
      k_face_scale<<<grid_for(nf, 256, gmax), 256, 0, st>>>(nf, ratio[a], src.Kf[a], h->T64[0][a]);
    }
  } else {
    const long long nyz = (long long)n3[1] * n3[2], nxz = (long long)n3[0] * n3[2], nxy = (long long)n3[0] * n3[1];
    const uint8_t* blo[3] = {bc, bc + 2 * nyz, bc + 2 * nyz + 2 * nxz};
    const uint8_t* bhi[3] = {bc + nyz, bc + 2 * nyz + nxz, bc + 2 * nyz + 2 * nxz + nxy};
    for (int a = 0; a < dim; ++a) {
      long long nf = (long long)(n3[0] + (a == 0)) * (n3[1] + (a == 1)) * (n3[2] + (a == 2));
      const double* Ka = K + (ncomp > 1 ? a * h->N[0] : 0);
      k_face_trans<<<grid_for(nf, 256, gmax), 256, 0, st>>>(a, n3[0], n3[1], n3[2], ratio[a], Ka, blo[a], bhi[a],
                                                             h->T64[0][a]);
    }
  }
  // ---- coarse transmissibilities (A2) ----
  for (int k = 0; k + 1 < h->nlev && !h->lap; ++k) {
    int3 nf = make_int3(h->dims[k][0], h->dims[k][1], h->dims[k][2]);
    int3 nc = make_int3(h->dims[k + 1][0], h->dims[k + 1][1], h->dims[k + 1][2]);
    for (int a = 0; a < dim; ++a) {
      long long ncf = (long long)(nc.x + (a == 0)) * (nc.y + (a == 1)) * (nc.z + (a == 2));
      k_upscale<<<grid_for(ncf, 128, gmax), 128, 0, st>>>(a, nf, nc, h->T64[k][a], h->T64[k + 1][a]);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return fail(MSRCG_ECUDA);
  // ---- smoother-precision copies ----
  for (int k = 0; k < h->nlev; ++k)
    for (int a = 0; a < dim; ++a) {
      const long long nf = nfaces(k, a);
      if (f32) {
        void* p;
        if ((rc = msrcg_alloc(h, &p, sizeof(float) * nf))) return fail(rc);
        k_to_float<<<grid_for(nf, 256, gmax), 256, 0, st>>>(h->T64[k][a], (float*)p, nf);
        h->TR[k][a] = p;
      } else {
        h->TR[k][a] = h->T64[k][a];
      }
    }
  // ---- transfer tables, vectors and level descriptors ----
  double fk = 1.0;
  for (int k = 0; k < h->nlev; ++k) {
    DevLevel& L = h->hL[k];
    memset(&L, 0, sizeof(L));
    L.nx = h->dims[k][0];
    L.ny = h->dims[k][1];
    L.nz = h->dims[k][2];
    L.dim = dim;
    L.n = h->N[k];
    L.px = L.nx + 2;
    L.py = L.ny + 2;
    L.plane = (long long)L.px * L.py;
    L.off = 1 + L.px + (dim == 3 ? L.plane : 0);
    L.npad = L.plane * (dim == 3 ? L.nz + 2 : 1);
    for (int a = 0; a < dim; ++a) {
      L.T[a] = h->TR[k][a];
      L.T64[a] = h->T64[k][a];
    }
    L.lap = h->lap;
    L.fk = fk;
    fk *= o.f;
    L.maxit = k == 0 ? o.maxit_outer : o.maxit_inner;
    if (k + 1 < h->nlev) {
      if (dim == 2) {
        // fine extent of the widest tile of the tiled restriction (kRestrictTI
        // x rtj coarse cells): the tables' windows are monotone, so a tile of
        // coarse cells I0..I1 reads fine cells lo[I0] .. hi[I1]
        const Axis1D tx = axis_tables(h->dims[k][0], h->dims[k + 1][0], o.interp);
        const Axis1D ty = axis_tables(h->dims[k][1], h->dims[k + 1][1], o.interp);
        h->rtj = f32 ? 8 : 4;
        int fx = 0, fy = 0;
        for (int I0 = 0; I0 < h->dims[k + 1][0]; I0 += kRestrictTI) {
          const int I1 = std::min(I0 + kRestrictTI, h->dims[k + 1][0]) - 1;
          fx = std::max(fx, tx.hi[I1] - tx.lo[I0] + 1);
        }
        for (int J0 = 0; J0 < h->dims[k + 1][1]; J0 += h->rtj) {
          const int J1 = std::min(J0 + h->rtj, h->dims[k + 1][1]) - 1;
          fy = std::max(fy, ty.hi[J1] - ty.lo[J0] + 1);
        }
        const size_t smem = rsz * ((size_t)fx * fy + (size_t)fy * kRestrictTI);
        if (smem <= 48 * 1024) {
          h->rfx[k] = fx;
          h->rfy[k] = fy;
        }
      }
      for (int a = 0; a < 3; ++a) {
        Axis1D ax = axis_tables(h->dims[k][a], h->dims[k + 1][a], o.interp);
        const void* p;
        if ((rc = upload(h, ax.c0, &p, st))) return fail(rc);
        L.c0[a] = (const int*)p;
        if ((rc = upload(h, ax.c1, &p, st))) return fail(rc);
        L.c1[a] = (const int*)p;
        if ((rc = upload(h, ax.lo, &p, st))) return fail(rc);
        L.lo[a] = (const int*)p;
        if ((rc = upload(h, ax.hi, &p, st))) return fail(rc);
        L.hi[a] = (const int*)p;
        if (f32) {
          std::vector<float> wf(ax.w.begin(), ax.w.end());
          if ((rc = upload(h, wf, &p, st))) return fail(rc);
          L.w[a] = p;
          std::vector<float> rf(ax.rw.begin(), ax.rw.end());
          if ((rc = upload(h, rf, &p, st))) return fail(rc);
          L.rw[a] = p;
        } else {
          if ((rc = upload(h, ax.w, &p, st))) return fail(rc);
          L.w[a] = p;
          if ((rc = upload(h, ax.rw, &p, st))) return fail(rc);
          L.rw[a] = p;
        }
        L.W[a] = ax.W;
      }
    }
    // padded vectors; the ghost ring is zeroed here and never written
    const size_t vsz = k == 0 ? sizeof(double) : rsz;
    void* p;
    void** vv[4] = {&L.x, &L.r, &L.p, &L.q};
    for (int v = 0; v < 4; ++v) {
      if ((rc = msrcg_alloc(h, &p, vsz * L.npad))) return fail(rc);
      MSRCG_CUDA_TRY(cudaMemsetAsync(p, 0, vsz * L.npad, st));
      *vv[v] = p;
    }
    if ((rc = msrcg_alloc(h, &p, rsz * L.npad))) return fail(rc);
    MSRCG_CUDA_TRY(cudaMemsetAsync(p, 0, rsz * L.npad, st));
    L.z = p;
    if ((rc = msrcg_alloc(h, &p, rsz * L.npad))) return fail(rc);
    MSRCG_CUDA_TRY(cudaMemsetAsync(p, 0, rsz * L.npad, st));
    L.t = p;
    if (vsz != rsz) {
      if ((rc = msrcg_alloc(h, &p, rsz * L.npad))) return fail(rc);
      MSRCG_CUDA_TRY(cudaMemsetAsync(p, 0, rsz * L.npad, st));
      L.rp = p;
    } else {
      L.rp = L.r;
    }

  }
  // ---- coarsest exact inverse (A3) ----
  {
    const int kc = h->nlev - 1;
    h->nc = (int)h->N[kc];
    void *A, *Ai, *fl;
    if ((rc = msrcg_alloc(h, &A, sizeof(double) * h->nc * h->nc))) return fail(rc);
    if ((rc = msrcg_alloc(h, &Ai, sizeof(double) * h->nc * h->nc))) return fail(rc);
    if ((rc = msrcg_alloc(h, &fl, sizeof(int)))) return fail(rc);
    MSRCG_CUDA_TRY(cudaMemsetAsync(fl, 0, sizeof(int), st));
    k_dense_assemble<<<1, 512, 0, st>>>(h->dims[kc][0], h->dims[kc][1], h->dims[kc][2], h->lap, h->T64[kc][0],
                                        h->T64[kc][1], dim == 3 ? h->T64[kc][2] : nullptr, (double*)A);
    k_chol_inverse<<<1, 512, 0, st>>>(h->nc, (double*)A, (double*)Ai, (int*)fl);
    int hf = 0;
    if (cudaMemcpyAsync(&hf, fl, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(MSRCG_ECUDA);
    if (hf) return fail(MSRCG_EBREAKDOWN);
    h->Ainv = (double*)Ai;
  }
  // ---- solve state ----
  {
    void* p;
    if ((rc = msrcg_alloc(h, &p, sizeof(DevLevel) * h->nlev))) return fail(rc);
    h->dL = (DevLevel*)p;
    MSRCG_CUDA_TRY(cudaMemcpyAsync(h->dL, h->hL, sizeof(DevLevel) * h->nlev, cudaMemcpyHostToDevice, st));
    if ((rc = msrcg_alloc(h, &p, sizeof(SolveState)))) return fail(rc);
    h->dS = (SolveState*)p;
    MSRCG_CUDA_TRY(cudaMemsetAsync(h->dS, 0, sizeof(SolveState), st));
    if ((rc = msrcg_alloc(h, &p, sizeof(double) * kMaxLev * (size_t)std::max(gmax, kMaxGrid)))) return fail(rc);
    h->partials = (double*)p;
    if ((rc = msrcg_alloc(h, &p, sizeof(double) * h->hL[0].npad))) return fail(rc);
    MSRCG_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(double) * h->hL[0].npad, st));
    h->b0 = (double*)p;
    if ((rc = msrcg_alloc(h, &p, sizeof(double) * h->hL[0].npad))) return fail(rc);
    MSRCG_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(double) * h->hL[0].npad, st));
    h->xs = (double*)p;
    if ((rc = msrcg_alloc(h, &p, sizeof(ProblemDesc)))) return fail(rc);
    h->dP = (ProblemDesc*)p;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(MSRCG_ECUDA);
  *out = h;
  return MSRCG_OK;
}

}  // namespace

// Device bytes msrcg_build_ex allocates for this grid and options (the same
// allocation list, in the same sizes; 0 for arguments it would reject).  The
// server charges this before a request is built.
size_t msrcg_build_bytes(const msrcg_grid* grid, const msrcg_opts* opts) {
  if (!grid || (grid->dim != 2 && grid->dim != 3)) return 0;
  const int dim = grid->dim;
  for (int a = 0; a < dim; ++a)
    if (grid->n[a] < 1 || !(grid->h[a] > 0.0)) return 0;
  msrcg_opts o;
  if (opts) o = *opts;
  else msrcg_default_opts(&o);
  if (o.scale < 2) return 0;
  if (o.coarsest_max_side <= 0) o.coarsest_max_side = dim == 2 ? 8 : 4;
  int n3[3] = {grid->n[0], grid->n[1], dim == 3 ? grid->n[2] : 1};
  const double h3[3] = {grid->h[0], grid->h[1], dim == 3 ? grid->h[2] : 1.0};
  int dims[kMaxLev][3];
  const int nlev = level_sides(dim, n3, h3, o.scale, o.coarsest_max_side, o.coarsening, dims);
  if (nlev < 1) return 0;
  const bool f32 = o.precision == 1;
  const size_t rsz = f32 ? sizeof(float) : sizeof(double);
  size_t tot = 0;
  auto add = [&](size_t b) { tot += b ? b : 16; };
  for (int k = 0; k < nlev; ++k)
    for (int a = 0; a < dim; ++a) {
      const size_t nf = (size_t)(dims[k][0] + (a == 0)) * (dims[k][1] + (a == 1)) * (dims[k][2] + (a == 2));
      add(sizeof(double) * nf);
      if (f32) add(sizeof(float) * nf);
    }
  long long npad0 = 0;
  for (int k = 0; k < nlev; ++k) {
    if (k + 1 < nlev)
      for (int a = 0; a < 3; ++a) {
        const Axis1D ax = axis_tables(dims[k][a], dims[k + 1][a], o.interp);
        add(sizeof(int) * ax.c0.size());
        add(sizeof(int) * ax.c1.size());
        add(sizeof(int) * ax.lo.size());
        add(sizeof(int) * ax.hi.size());
        add(rsz * ax.w.size());
        add(rsz * ax.rw.size());
      }
    const long long npad = (long long)(dims[k][0] + 2) * (dims[k][1] + 2) * (dim == 3 ? dims[k][2] + 2 : 1);
    if (k == 0) npad0 = npad;
    const size_t vsz = k == 0 ? sizeof(double) : rsz;
    for (int v = 0; v < 4; ++v) add(vsz * npad);
    add(rsz * npad);
    add(rsz * npad);
    if (vsz != rsz) add(rsz * npad);
  }
  const size_t nc = (size_t)dims[nlev - 1][0] * dims[nlev - 1][1] * dims[nlev - 1][2];
  add(sizeof(double) * nc * nc);
  add(sizeof(double) * nc * nc);
  add(sizeof(int));
  add(sizeof(DevLevel) * nlev);
  add(sizeof(SolveState));
  add(sizeof(double) * kMaxLev * (size_t)kMaxGrid);
  add(sizeof(double) * npad0);
  add(sizeof(double) * npad0);
  add(sizeof(ProblemDesc));
  return tot;
}

extern "C" int msrcg_lift_rhs(msrcg_hier* h, const uint8_t* bc, const double* gD, const double* f, const double* pbf,
                              double* b, void* stream) {
  if (!h || !bc || !gD || !pbf || !b) return MSRCG_EINVAL;
  const int* d = h->dims[0];
  const double vol = h->hsz[0] * h->hsz[1] * (h->dim == 3 ? h->hsz[2] : 1.0);
  k_lift<<<grid_for(h->N[0], 256, h->sms * 8), 256, 0, (cudaStream_t)stream>>>(
      d[0], d[1], d[2], h->lap, h->T64[0][0], h->T64[0][1], h->dim == 3 ? h->T64[0][2] : nullptr, bc, gD, f, vol, pbf,
      b);
  MSRCG_CUDA_TRY(cudaGetLastError());
  return MSRCG_OK;
}

extern "C" int msrcg_level_info(const msrcg_hier* h, int level, int dims[3], int64_t* iters, int64_t* calls) {
  if (!h || level < 0 || level >= h->nlev) return MSRCG_EINVAL;
  if (dims)
    for (int a = 0; a < 3; ++a) dims[a] = h->dims[level][a];
  if (iters) *iters = h->last_iters[level];
  if (calls) *calls = h->last_calls[level];
  return MSRCG_OK;
}

extern "C" int msrcg_get_trans(const msrcg_hier* h, int level, double* Tx, double* Ty, double* Tz, void* stream) {
  if (!h || level < 0 || level >= h->nlev || !Tx || !Ty || (h->dim == 3 && !Tz)) return MSRCG_EINVAL;
  const int* d = h->dims[level];
  double* outs[3] = {Tx, Ty, Tz};
  for (int a = 0; a < h->dim; ++a) {
    long long nf = (long long)(d[0] + (a == 0)) * (d[1] + (a == 1)) * (d[2] + (a == 2));
    if (h->lap) {
      k_expand_faces<<<grid_for(nf, 256, h->sms * 8), 256, 0, (cudaStream_t)stream>>>(a, d[0], d[1], d[2],
                                                                                       h->T64[level][a], outs[a]);
      MSRCG_CUDA_TRY(cudaGetLastError());
    } else {
      MSRCG_CUDA_TRY(cudaMemcpyAsync(outs[a], h->T64[level][a], sizeof(double) * nf, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream));
    }
  }
  return MSRCG_OK;
}

extern "C" int msrcg_apply(const msrcg_hier* h, int level, const double* x, double* y, void* stream) {
  if (!h || level < 0 || level >= h->nlev || !x || !y) return MSRCG_EINVAL;
  const int* d = h->dims[level];
  k_apply64<<<grid_for(h->N[level], 256, h->sms * 8), 256, 0, (cudaStream_t)stream>>>(
      d[0], d[1], d[2], h->lap, h->T64[level][0], h->T64[level][1], h->dim == 3 ? h->T64[level][2] : nullptr, x, y);
  MSRCG_CUDA_TRY(cudaGetLastError());
  return MSRCG_OK;
}

extern "C" int msrcg_num_levels(const msrcg_hier* h) { return h ? h->nlev : 0; }
extern "C" size_t msrcg_device_bytes(const msrcg_hier* h) { return h ? h->bytes : 0; }
extern "C" void msrcg_free(msrcg_hier* h) { release(h); }

// ===========================================================================
// Hierarchy in a caller-supplied device buffer (used by the entry point that
// allocates nothing).  Same kernels and layout as msrcg_build, but every array
// is carved out of [base, base + cap) and the transfer tables are computed on
// the device, so neither device nor host memory is allocated.  All levels run
// in one CTA (ks = 0).
// ===========================================================================
namespace {

// 1-D transfer tables of one axis (nf fine -> nc coarse cells) on the device:
// prolongation corners/weights per fine cell and, per coarse cell, the window
// of fine cells interpolating from it with their weights (row stride W).
__global__ void k_axis_tables(int nf, int nc, int W, int* c0, int* c1, void* w, int* lo, int* hi, void* rw, int f32,
                              int interp) {
  const long long den = 2LL * nf;
  auto corners = [&](int i, int* a, int* b, double* wt) {
    const long long num = (2LL * i + 1) * nc - nf;
    if (interp == 1) {
      *a = *b = (int)(((2LL * i + 1) * nc) / den);
      *wt = 0.0;
    } else if (num <= 0) {
      *a = *b = 0;
      *wt = 0.0;
    } else if (num / den >= nc - 1) {
      *a = *b = nc - 1;
      *wt = 0.0;
    } else if (num % den == 0) {
      *a = *b = (int)(num / den);
      *wt = 0.0;
    } else {
      *a = (int)(num / den);
      *b = *a + 1;
      *wt = (double)(num % den) / (double)den;
    }
  };
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nf; i += stride) {
    int a, b;
    double wt;
    corners(i, &a, &b, &wt);
    c0[i] = a;
    c1[i] = b;
    if (f32) ((float*)w)[i] = (float)wt;
    else ((double*)w)[i] = wt;
  }
  for (int I = tid; I < nc; I += stride) {
    const int wa = (int)(((long long)(I - 1) * nf) / nc) - 2, wb = (int)(((long long)(I + 2) * nf) / nc) + 2;
    const int a0 = wa < 0 ? 0 : wa, b0 = wb > nf - 1 ? nf - 1 : wb;
    int l = nf, h = -1;
    for (int i = a0; i <= b0; ++i) {
      int a, b;
      double wt;
      corners(i, &a, &b, &wt);
      const bool on = (a == I && (1.0 - wt != 0.0 || a == b)) || (b == I && wt != 0.0);
      if (on) {
        l = i < l ? i : l;
        h = i > h ? i : h;
      }
    }
    lo[I] = l;
    hi[I] = h;
    for (int t = 0; t < W; ++t) {
      const int i = l + t;
      double v = 0.0;
      if (i <= h) {
        int a, b;
        double wt;
        corners(i, &a, &b, &wt);
        if (a == I) v += 1.0 - wt;
        if (b == I) v += wt;
      }
      if (f32) ((float*)rw)[(long long)I * W + t] = (float)v;
      else ((double*)rw)[(long long)I * W + t] = v;
    }
  }
}

struct Carve {
  unsigned char* base;
  size_t cap, off;
  bool ok;
  void* take(size_t b) {
    off = (off + 255) & ~(size_t)255;
    if (off + b > cap) {
      ok = false;
      return nullptr;
    }
    void* p = base + off;
    off += b;
    return p;
  }
};

}  // namespace

int msrcg_build_into(msrcg_hier* h, const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                     const msrcg_opts* opts, cudaStream_t st, unsigned char* base, size_t cap) {
  if (!h || !grid || !K || !bc || !base) return MSRCG_EINVAL;
  const int dim = grid->dim;
  if (dim != 2 && dim != 3) return MSRCG_EINVAL;
  for (int a = 0; a < dim; ++a)
    if (grid->n[a] < 1 || !(grid->h[a] > 0.0) || !isfinite(grid->h[a])) return MSRCG_EINVAL;
  if (ncomp != 1 && ncomp != dim) return MSRCG_EINVAL;
  msrcg_opts o;
  if (opts) o = *opts;
  else msrcg_default_opts(&o);
  if (o.scale < 2 || o.m < 1 || !(o.f > 0.0) || o.maxit_outer < 1 || o.maxit_inner < 1 || o.fuse_width < 0 ||
      o.fuse_min_cells < 0 || o.splitting < 0 || o.splitting > 2 || o.coarsening < 0 || o.coarsening > 1 ||
      o.interp < 0 || o.interp > 1 || o.escalate < 0 || o.escalate > 1 || o.flexible < 0 || o.flexible > 1 ||
      o.precond < 0 || o.precond > 2)
    return MSRCG_EINVAL;
  if (o.precision != 0 && o.precision != 1) return MSRCG_EINVAL;
  if (o.coarsest_max_side <= 0) o.coarsest_max_side = dim == 2 ? 8 : 4;
  h->dim = dim;
  h->o = o;
  for (int a = 0; a < 3; ++a) h->hsz[a] = a < dim ? grid->h[a] : 1.0;
  if (cudaGetDevice(&h->device) != cudaSuccess) return MSRCG_ECUDA;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  int n3[3] = {grid->n[0], grid->n[1], dim == 3 ? grid->n[2] : 1};
  if ((long long)(n3[0] + 2) * (n3[1] + 2) * (n3[2] + 2) >= (1LL << 31)) return MSRCG_EINVAL;
  {
    const double h3[3] = {grid->h[0], grid->h[1], dim == 3 ? grid->h[2] : 1.0};
    h->nlev = level_sides(dim, n3, h3, o.scale, o.coarsest_max_side, o.coarsening, h->dims);
  }
  if (h->nlev < 1) return MSRCG_EINVAL;
  for (int k = 0; k < h->nlev; ++k) h->N[k] = (long long)h->dims[k][0] * h->dims[k][1] * h->dims[k][2];
  if (h->N[h->nlev - 1] > 1024) return MSRCG_EINVAL;
  h->ks = 0;
  const bool f32 = o.precision == 1;
  const size_t rsz = f32 ? sizeof(float) : sizeof(double);
  const int gmax = std::min(h->sms * 8, kMaxGrid);

  // ---- lay out every array first: a problem that does not fit is rejected
  // before anything is enqueued, so an MSRCG_EINVAL leaves no work behind on
  // the stream (the scratch is shared by every call) ----
  Carve cv{base, cap, 0, true};
  int tabW[kMaxLev][3] = {};
  for (int k = 0; k < h->nlev; ++k)
    for (int a = 0; a < dim; ++a) {
      const int* d = h->dims[k];
      long long nf = (long long)(d[0] + (a == 0)) * (d[1] + (a == 1)) * (d[2] + (a == 2));
      h->T64[k][a] = (double*)cv.take(sizeof(double) * nf);
      h->TR[k][a] = f32 ? cv.take(sizeof(float) * nf) : (void*)h->T64[k][a];
    }
  double fk = 1.0;
  for (int k = 0; k < h->nlev; ++k) {
    DevLevel& L = h->hL[k];
    memset(&L, 0, sizeof(L));
    L.nx = h->dims[k][0];
    L.ny = h->dims[k][1];
    L.nz = h->dims[k][2];
    L.dim = dim;
    L.n = h->N[k];
    L.px = L.nx + 2;
    L.py = L.ny + 2;
    L.plane = (long long)L.px * L.py;
    L.off = 1 + L.px + (dim == 3 ? L.plane : 0);
    L.npad = L.plane * (dim == 3 ? L.nz + 2 : 1);
    for (int a = 0; a < dim; ++a) {
      L.T[a] = h->TR[k][a];
      L.T64[a] = h->T64[k][a];
    }
    L.fk = fk;
    fk *= o.f;
    L.maxit = k == 0 ? o.maxit_outer : o.maxit_inner;
    if (k + 1 < h->nlev) {
      for (int a = 0; a < 3; ++a) {
        const int nf = h->dims[k][a], nc = h->dims[k + 1][a];
        const int W = 3 * ((nf + nc - 1) / nc) + 6;
        tabW[k][a] = W;
        L.c0[a] = (const int*)cv.take(sizeof(int) * nf);
        L.c1[a] = (const int*)cv.take(sizeof(int) * nf);
        L.w[a] = cv.take(rsz * nf);
        L.lo[a] = (const int*)cv.take(sizeof(int) * nc);
        L.hi[a] = (const int*)cv.take(sizeof(int) * nc);
        L.rw[a] = cv.take(rsz * (size_t)nc * W);
        L.W[a] = W;
      }
    }
    const size_t vsz = k == 0 ? sizeof(double) : rsz;
    L.x = cv.take(vsz * L.npad);
    L.r = cv.take(vsz * L.npad);
    L.p = cv.take(vsz * L.npad);
    L.q = cv.take(vsz * L.npad);
    L.z = cv.take(rsz * L.npad);
    L.t = cv.take(rsz * L.npad);
    L.rp = vsz != rsz ? cv.take(rsz * L.npad) : L.r;
  }
  const int kc = h->nlev - 1;
  h->nc = (int)h->N[kc];
  double* A = (double*)cv.take(sizeof(double) * h->nc * h->nc);
  double* Ai = (double*)cv.take(sizeof(double) * h->nc * h->nc);
  int* fl = (int*)cv.take(sizeof(int));
  h->dL = (DevLevel*)cv.take(sizeof(DevLevel) * h->nlev);
  h->dS = (SolveState*)cv.take(sizeof(SolveState));
  h->xs = (double*)cv.take(sizeof(double) * h->hL[0].npad);
  h->dP = (ProblemDesc*)cv.take(sizeof(ProblemDesc));
  h->partials = nullptr;
  h->b0 = nullptr;
  if (!cv.ok) return MSRCG_EINVAL;

  // ---- enqueue the build; from here on an error waits for the work
  // already enqueued before returning ----
  auto fail = [&](int code) {
    cudaStreamSynchronize(st);
    (void)cudaGetLastError();
    return code;
  };
  double hh[3] = {grid->h[0], grid->h[1], dim == 3 ? grid->h[2] : 1.0};
  double ratio[3] = {(hh[1] * hh[2]) / hh[0], (hh[0] * hh[2]) / hh[1], (hh[0] * hh[1]) / hh[2]};
  const long long nyz = (long long)n3[1] * n3[2], nxz = (long long)n3[0] * n3[2], nxy = (long long)n3[0] * n3[1];
  const uint8_t* blo[3] = {bc, bc + 2 * nyz, bc + 2 * nyz + 2 * nxz};
  const uint8_t* bhi[3] = {bc + nyz, bc + 2 * nyz + nxz, bc + 2 * nyz + 2 * nxz + nxy};
  for (int a = 0; a < dim; ++a) {
    long long nf = (long long)(n3[0] + (a == 0)) * (n3[1] + (a == 1)) * (n3[2] + (a == 2));
    const double* Ka = K + (ncomp > 1 ? a * h->N[0] : 0);
    k_face_trans<<<grid_for(nf, 256, gmax), 256, 0, st>>>(a, n3[0], n3[1], n3[2], ratio[a], Ka, blo[a], bhi[a],
                                                           h->T64[0][a]);
  }
  for (int k = 0; k + 1 < h->nlev; ++k) {
    int3 nf = make_int3(h->dims[k][0], h->dims[k][1], h->dims[k][2]);
    int3 nc = make_int3(h->dims[k + 1][0], h->dims[k + 1][1], h->dims[k + 1][2]);
    for (int a = 0; a < dim; ++a) {
      long long ncf = (long long)(nc.x + (a == 0)) * (nc.y + (a == 1)) * (nc.z + (a == 2));
      k_upscale<<<grid_for(ncf, 128, gmax), 128, 0, st>>>(a, nf, nc, h->T64[k][a], h->T64[k + 1][a]);
    }
  }
  for (int k = 0; k < h->nlev; ++k)
    for (int a = 0; a < dim && f32; ++a) {
      const int* d = h->dims[k];
      long long nf = (long long)(d[0] + (a == 0)) * (d[1] + (a == 1)) * (d[2] + (a == 2));
      k_to_float<<<grid_for(nf, 256, gmax), 256, 0, st>>>(h->T64[k][a], (float*)h->TR[k][a], nf);
    }
  for (int k = 0; k < h->nlev; ++k) {
    DevLevel& L = h->hL[k];
    if (k + 1 < h->nlev)
      for (int a = 0; a < 3; ++a) {
        const int nf = h->dims[k][a], nc = h->dims[k + 1][a];
        k_axis_tables<<<grid_for(std::max(nf, nc), 128, gmax), 128, 0, st>>>(
            nf, nc, tabW[k][a], (int*)L.c0[a], (int*)L.c1[a], (void*)L.w[a], (int*)L.lo[a], (int*)L.hi[a],
            (void*)L.rw[a], f32, o.interp);
      }
    // padded vectors; the ghost rings must be zero, and the buffer keeps the
    // previous call's contents, so every vector is cleared
    const size_t vsz = k == 0 ? sizeof(double) : rsz;
    void* vv[4] = {L.x, L.r, L.p, L.q};
    for (int v = 0; v < 4; ++v)
      if (cudaMemsetAsync(vv[v], 0, vsz * L.npad, st) != cudaSuccess) return fail(MSRCG_ECUDA);
    if (cudaMemsetAsync(L.z, 0, rsz * L.npad, st) != cudaSuccess ||
        cudaMemsetAsync(L.t, 0, rsz * L.npad, st) != cudaSuccess ||
        (vsz != rsz && cudaMemsetAsync(L.rp, 0, rsz * L.npad, st) != cudaSuccess))
      return fail(MSRCG_ECUDA);
  }
  if (cudaMemsetAsync(fl, 0, sizeof(int), st) != cudaSuccess) return fail(MSRCG_ECUDA);
  k_dense_assemble<<<1, 512, 0, st>>>(h->dims[kc][0], h->dims[kc][1], h->dims[kc][2], 0, h->T64[kc][0],
                                      h->T64[kc][1], dim == 3 ? h->T64[kc][2] : nullptr, A);
  k_chol_inverse<<<1, 512, 0, st>>>(h->nc, A, Ai, fl);
  int hf = 0;
  if (cudaMemcpyAsync(&hf, fl, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(MSRCG_ECUDA);
  if (hf) return MSRCG_EBREAKDOWN;
  h->Ainv = Ai;
  if (cudaMemcpyAsync(h->dL, h->hL, sizeof(DevLevel) * h->nlev, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(h->dS, 0, sizeof(SolveState), st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(MSRCG_ECUDA);
  h->bytes = cv.off;
  return MSRCG_OK;
}
