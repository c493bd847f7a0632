/*
 * Plain FP64 CPU oracle of the recursive multi-scale preconditioned conjugate
 * gradient (RMS-PCG) of Lackner & Menikoff, "Multi-scale linear solvers for
 * very large systems derived from PDEs" (arXiv math/9809043).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct checker
 * that the GPU library is compared with.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Every routine follows a passage of the paper; the passage is named above the
 * routine.  Readings where the paper is silent are stated where they are used:
 *   - sign: the paper writes div(K grad P) = S; we solve -div(K grad p) = f so
 *     that A is symmetric positive definite (Sec. 3).
 *   - a Dirichlet boundary face sits half a cell from the cell centre, so its
 *     transmissibility is 2 (h_perp/h_par) K_cell; a Neumann face has T = 0
 *     (Sec. 3, "the type of boundary condition affects the discretized K").
 *   - unknowns are visited in red-black order (colour = (i+j+k) mod 2, red
 *     first); the symmetric Gauss-Seidel splitting of Sec. 3 is applied in
 *     that ordering.  The alternatives (or_set_splitting) are the modified
 *     Jacobi splitting of Sec. 3 (P = 2D) and symmetric Gauss-Seidel in the
 *     natural order of the unknowns.
 *   - level sides: n_{k+1} = max(2, floor(n_k/s + 1/2)) per axis while the
 *     axis is longer than the coarsest side limit; stop when no axis is.
 *   - coarse transmissibility: the face-dual series/parallel reading of the
 *     formula of Sec. 3 (each fine face owns the conductor between the two
 *     cell centres it separates, half a cell at the boundary).
 *   - coarsest level: PCG whose preconditioner is the exact inverse, applied
 *     through a dense Cholesky factorisation.
 *
 * Floating point: compiled with -ffp-contract=off so that a*b+c is never
 * fused; the results are the same on x86-64 and aarch64 hosts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXLEV 16

/* status codes (same meaning as the library's, values restated here) */
#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ENOCONV (-3)
#define OR_EBREAKDOWN (-4)

typedef struct {
  int nx, ny, nz;
  int64_t n;
  double *Tx, *Ty, *Tz;                 /* face transmissibilities (Tz NULL in 2D) */
  /* transfer to the next coarser level, one table per axis over fine cells */
  int *i0[3], *i1[3];
  double *w[3];
  /* work vectors */
  double *b, *x, *r, *p, *z, *q, *t, *aw; /* aw: A x of a Jacobi step */
} or_level;

typedef struct {
  int dim, nlev;
  or_level L[OR_MAXLEV];
  int s, m;
  double f;
  int maxit_outer, maxit_inner;
  double eps2;                          /* epsilon^2 of the level test, Sec. 3 */
  double *chol;                         /* Cholesky factor of the coarsest A */
  int nc;
  int64_t iters[OR_MAXLEV], calls[OR_MAXLEV];
  int status;
  int splitting;                        /* 0: symmetric Gauss-Seidel (red-black), 1: modified
                                           Jacobi, 2: symmetric Gauss-Seidel (natural order) */
  int precond;                          /* preconditioner of the level-0 PCG (Sec. 2): 0 recursive
                                           multi-scale (eq. 2.10), 1 multigrid (eq. 2.9, Tatebe),
                                           2 polynomial (eq. 2.6 with W = P^-1) */
  /* level tree (Fig. 2): one entry (level, call, iterations, pass) per PCG
     call, written when the call returns; NULL when off */
  int32_t *trace;
  int64_t trace_cap, trace_n;
  int pass;                             /* restart of or_solve (0 .. 3) */
} or_hier;

static int64_t idx3(int i, int j, int k, int nx, int ny) {
  return (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
}

/* ---------------------------------------------------------------------------
 * Level sides.  Sec. 3 (scale factor about 4, adjusted to integer sizes).
 * rule 0: every axis longer than maxside shrinks by the factor s.
 * rule 1 (Sec. 4.4, anisotropic cells): coarsening aims at square cells --
 *   the coarse cell size is s times the smallest cell size h_min of the
 *   level, so an axis whose cells are already longer shrinks less or not at
 *   all (the "semi-coarsening" the paper describes); square cells coarsen as
 *   rule 0 up to rounding.  Axis a (if longer than maxside) gets
 *   max(2, min(n_a, round(L_a / (s h_min)))), L_a = n_a h_a; when no axis
 *   changes, the level is the coarsest (the paper's narrow channel also ends
 *   on a level of several hundred cells).
 * ------------------------------------------------------------------------- */
int or_hierarchy_dims2(int dim, const int n[3], const double h[3], int s, int maxside, int rule, int maxlev,
                       int *dims_out) {
  int cur[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  double La[3] = {0.0, 0.0, 0.0};
  int nlev = 0;
  if (s < 2 || maxside < 1 || rule < 0 || rule > 1) return OR_EINVAL;
  for (int a = 0; a < dim; ++a) La[a] = (double)n[a] * h[a];
  for (;;) {
    if (nlev >= maxlev) return OR_EINVAL;
    dims_out[3 * nlev + 0] = cur[0];
    dims_out[3 * nlev + 1] = cur[1];
    dims_out[3 * nlev + 2] = cur[2];
    nlev++;
    int any = 0;
    for (int a = 0; a < dim; ++a)
      if (cur[a] > maxside) any = 1;
    if (!any) break;
    double hmin = 0.0; /* smallest cell size over all axes */
    for (int a = 0; a < dim; ++a) {
      double ha = La[a] / (double)cur[a];
      if (a == 0 || ha < hmin) hmin = ha;
    }
    int next[3] = {cur[0], cur[1], cur[2]}, moved = 0;
    for (int a = 0; a < dim; ++a) {
      if (cur[a] > maxside) {
        int c;
        if (rule == 0) {
          c = (2 * cur[a] + s) / (2 * s); /* floor(n/s + 1/2) */
        } else {
          double t = La[a] / ((double)s * hmin);
          c = (int)floor(t + 0.5);
          if (c > cur[a]) c = cur[a];
        }
        next[a] = c < 2 ? 2 : c;
        if (next[a] != cur[a]) moved = 1;
      }
    }
    /* rule 1: no axis can coarsen without cells longer than s h_min -- this
     * level is the coarsest */
    if (rule == 1 && !moved) break;
    for (int a = 0; a < dim; ++a) cur[a] = next[a];
  }
  return nlev;
}

int or_hierarchy_dims(int dim, const int n[3], int s, int maxside, int maxlev, int *dims_out) {
  const double h[3] = {1.0, 1.0, 1.0};
  return or_hierarchy_dims2(dim, n, h, s, maxside, 0, maxlev, dims_out);
}

/* ---------------------------------------------------------------------------
 * Face transmissibilities from cell permeabilities.  Sec. 3: face K is the
 * harmonic mean of the two adjacent cell values; T_xx = (dy/dx) K_xx (times
 * dz in 3D); boundary faces carry the boundary condition.
 * K has ncomp components (1 = scalar, dim = diagonal tensor), each n cells.
 * bc: per boundary face, 1 = Dirichlet, 0 = Neumann, blocks in the order
 * x-low, x-high (ny*nz each), y-low, y-high (nx*nz each), z-low, z-high
 * (nx*ny each, 3D only).
 * ------------------------------------------------------------------------- */
void or_face_trans(int dim, const int n[3], const double h[3], const double *K, int ncomp,
                   const unsigned char *bc, double *Tx, double *Ty, double *Tz) {
  int nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
  double hx = h[0], hy = h[1], hz = dim == 3 ? h[2] : 1.0;
  int64_t N = (int64_t)nx * ny * nz;
  const double *Kx = K;
  const double *Ky = ncomp > 1 ? K + N : K;
  const double *Kz = ncomp > 2 ? K + 2 * N : K;
  double rx = (hy * hz) / hx, ry = (hx * hz) / hy, rz = (hx * hy) / hz;
  const unsigned char *bx0 = bc, *bx1 = bc + (int64_t)ny * nz;
  const unsigned char *by0 = bx1 + (int64_t)ny * nz, *by1 = by0 + (int64_t)nx * nz;
  const unsigned char *bz0 = by1 + (int64_t)nx * nz, *bz1 = bz0 + (int64_t)nx * ny;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        double t;
        if (i == 0) {
          t = bx0[j + (int64_t)ny * k] ? rx * (2.0 * Kx[idx3(0, j, k, nx, ny)]) : 0.0;
        } else if (i == nx) {
          t = bx1[j + (int64_t)ny * k] ? rx * (2.0 * Kx[idx3(nx - 1, j, k, nx, ny)]) : 0.0;
        } else {
          double kl = Kx[idx3(i - 1, j, k, nx, ny)], kr = Kx[idx3(i, j, k, nx, ny)];
          double s = kl + kr;
          t = s > 0.0 ? rx * (2.0 * kl * kr / s) : 0.0;
        }
        Tx[(int64_t)i + (int64_t)(nx + 1) * ((int64_t)j + (int64_t)ny * k)] = t;
      }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double t;
        if (j == 0) {
          t = by0[i + (int64_t)nx * k] ? ry * (2.0 * Ky[idx3(i, 0, k, nx, ny)]) : 0.0;
        } else if (j == ny) {
          t = by1[i + (int64_t)nx * k] ? ry * (2.0 * Ky[idx3(i, ny - 1, k, nx, ny)]) : 0.0;
        } else {
          double kl = Ky[idx3(i, j - 1, k, nx, ny)], kr = Ky[idx3(i, j, k, nx, ny)];
          double s = kl + kr;
          t = s > 0.0 ? ry * (2.0 * kl * kr / s) : 0.0;
        }
        Ty[(int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)(ny + 1) * k)] = t;
      }
  if (dim == 3) {
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double t;
          if (k == 0) {
            t = bz0[i + (int64_t)nx * j] ? rz * (2.0 * Kz[idx3(i, j, 0, nx, ny)]) : 0.0;
          } else if (k == nz) {
            t = bz1[i + (int64_t)nx * j] ? rz * (2.0 * Kz[idx3(i, j, nz - 1, nx, ny)]) : 0.0;
          } else {
            double kl = Kz[idx3(i, j, k - 1, nx, ny)], kr = Kz[idx3(i, j, k, nx, ny)];
            double s = kl + kr;
            t = s > 0.0 ? rz * (2.0 * kl * kr / s) : 0.0;
          }
          Tz[(int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k)] = t;
        }
  }
}

/* ---------------------------------------------------------------------------
 * Face transmissibilities from face permeabilities.  Sec. 3: the components
 * of K are face centred (K_xx half a cell off the centre in x), and the type
 * of boundary condition is carried by the discretised K of the boundary
 * faces; T_xx = (dy/dx) K_xx (times dz in 3D) on every face, boundary faces
 * included.  Kx has (nx+1)*ny*nz entries, Ky nx*(ny+1)*nz, Kz nx*ny*(nz+1).
 * ------------------------------------------------------------------------- */
void or_face_trans_faces(int dim, const int n[3], const double h[3], const double *Kx, const double *Ky,
                         const double *Kz, double *Tx, double *Ty, double *Tz) {
  int nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
  double hx = h[0], hy = h[1], hz = dim == 3 ? h[2] : 1.0;
  double rx = (hy * hz) / hx, ry = (hx * hz) / hy, rz = (hx * hy) / hz;
  int64_t nfx = (int64_t)(nx + 1) * ny * nz, nfy = (int64_t)nx * (ny + 1) * nz, nfz = (int64_t)nx * ny * (nz + 1);
  for (int64_t f = 0; f < nfx; ++f) Tx[f] = rx * Kx[f];
  for (int64_t f = 0; f < nfy; ++f) Ty[f] = ry * Ky[f];
  if (dim == 3)
    for (int64_t f = 0; f < nfz; ++f) Tz[f] = rz * Kz[f];
}

/* ---------------------------------------------------------------------------
 * Coarse transmissibility, Sec. 3: 1/T^c = sum_i 1/(sum_j T(i,j)) with the
 * partial-overlap scaling (fraction of height, inverse fraction of width).
 * Lengths along an axis with nf fine and nc coarse cells on a unit interval
 * are integers in units of 1/(2 nf nc).
 * ------------------------------------------------------------------------- */
static int64_t ov(int64_t a0, int64_t a1, int64_t b0, int64_t b1) {
  int64_t lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
  return hi > lo ? hi - lo : 0;
}
/* block of fine face i along its normal axis (between the adjacent centres) */
static void face_block(int i, int nf, int nc, int64_t *lo, int64_t *hi) {
  int64_t L = 2 * (int64_t)nf * nc;
  int64_t a = (2 * (int64_t)i - 1) * nc, b = (2 * (int64_t)i + 1) * nc;
  *lo = a < 0 ? 0 : a;
  *hi = b > L ? L : b;
}
static void cface_block(int I, int nf, int nc, int64_t *lo, int64_t *hi) {
  int64_t L = 2 * (int64_t)nf * nc;
  int64_t a = (2 * (int64_t)I - 1) * nf, b = (2 * (int64_t)I + 1) * nf;
  *lo = a < 0 ? 0 : a;
  *hi = b > L ? L : b;
}
/* fraction of fine cell j's extent inside coarse cell J */
static double cell_frac(int j, int J, int nf, int nc) {
  int64_t o = ov(2 * (int64_t)j * nc, 2 * ((int64_t)j + 1) * nc, 2 * (int64_t)J * nf, 2 * ((int64_t)J + 1) * nf);
  return (double)o / (double)(2 * (int64_t)nc);
}

/* Index windows that contain every fine face / cell overlapping a coarse one;
 * entries with zero overlap inside a window are skipped by the callers, so
 * the windows only bound the loops and never change a sum. */
static void normal_range(int I, int nf, int nc, int *lo, int *hi) {
  int64_t a = ((2 * (int64_t)I - 1) * nf) / (2 * (int64_t)nc) - 2, b = ((2 * (int64_t)I + 1) * nf) / (2 * (int64_t)nc) + 2;
  *lo = a < 0 ? 0 : (int)a;
  *hi = b > nf ? nf : (int)b;
}
static void par_range(int J, int nf, int nc, int *lo, int *hi) {
  int64_t a = ((int64_t)J * nf) / nc - 1, b = (((int64_t)J + 1) * nf + nc - 1) / nc + 1;
  *lo = a < 0 ? 0 : (int)a;
  *hi = b > nf - 1 ? nf - 1 : (int)b;
}

/* Upscale the faces normal to axis `ax` from fine dims nf[3] to coarse dims nc[3].
 * Tf / Tc are laid out with the normal axis having n+1 entries. */
static void upscale_axis(int ax, const int nf[3], const int nc[3], const double *Tf, double *Tc) {
  int p1 = (ax + 1) % 3, p2 = (ax + 2) % 3; /* the two parallel axes */
  int fdim[3] = {nf[0], nf[1], nf[2]}, cdim[3] = {nc[0], nc[1], nc[2]};
  fdim[ax] += 1;
  cdim[ax] += 1;
  int c[3];
  for (c[2] = 0; c[2] < cdim[2]; ++c[2])
    for (c[1] = 0; c[1] < cdim[1]; ++c[1])
      for (c[0] = 0; c[0] < cdim[0]; ++c[0]) {
        int64_t clo, chi;
        cface_block(c[ax], nf[ax], nc[ax], &clo, &chi);
        double inv = 0.0;
        int zero = 0, any = 0;
        int ilo, ihi, alo, ahi, blo, bhi;
        normal_range(c[ax], nf[ax], nc[ax], &ilo, &ihi);
        par_range(c[p1], nf[p1], nc[p1], &alo, &ahi);
        par_range(c[p2], nf[p2], nc[p2], &blo, &bhi);
        for (int i = ilo; i <= ihi; ++i) {
          int64_t flo, fhi;
          face_block(i, nf[ax], nc[ax], &flo, &fhi);
          int64_t o = ov(flo, fhi, clo, chi);
          if (o == 0) continue;
          any = 1;
          /* parallel sum over the fine faces of column i inside the coarse face */
          double S = 0.0;
          for (int b = blo; b <= bhi; ++b) {
            double f2 = cell_frac(b, c[p2], nf[p2], nc[p2]);
            if (f2 == 0.0) continue;
            double inner = 0.0;
            for (int a = alo; a <= ahi; ++a) {
              double f1 = cell_frac(a, c[p1], nf[p1], nc[p1]);
              if (f1 == 0.0) continue;
              int g[3];
              g[ax] = i;
              g[p1] = a;
              g[p2] = b;
              inner += f1 * Tf[(int64_t)g[0] + (int64_t)fdim[0] * ((int64_t)g[1] + (int64_t)fdim[1] * g[2])];
            }
            S += f2 * inner;
          }
          double C = (S * (double)(fhi - flo)) / (double)o;
          if (C == 0.0) {
            zero = 1;
            break;
          }
          inv += 1.0 / C;
        }
        double t = (zero || !any) ? 0.0 : 1.0 / inv;
        Tc[(int64_t)c[0] + (int64_t)cdim[0] * ((int64_t)c[1] + (int64_t)cdim[1] * c[2])] = t;
      }
}

void or_upscale(int dim, const int nf[3], const int nc[3], const double *Txf, const double *Tyf, const double *Tzf,
                double *Txc, double *Tyc, double *Tzc) {
  int f3[3] = {nf[0], nf[1], dim == 3 ? nf[2] : 1}, c3[3] = {nc[0], nc[1], dim == 3 ? nc[2] : 1};
  upscale_axis(0, f3, c3, Txf, Txc);
  upscale_axis(1, f3, c3, Tyf, Tyc);
  if (dim == 3) upscale_axis(2, f3, c3, Tzf, Tzc);
}

/* ---------------------------------------------------------------------------
 * Extension E: tensor product of 1-D linear interpolation between cell
 * centres with zero slope at the boundary; reduction R = E^T.  Sec. 3.
 * For fine cell i: t = x_i/H - 1/2 = ((2i+1) nc - nf) / (2 nf).
 * ------------------------------------------------------------------------- */
void or_transfer_table(int nf, int nc, int *i0, int *i1, double *w) {
  for (int i = 0; i < nf; ++i) {
    int64_t num = (2 * (int64_t)i + 1) * nc - nf;
    int64_t den = 2 * (int64_t)nf;
    if (num <= 0) {
      i0[i] = i1[i] = 0;
      w[i] = 0.0;
      continue;
    }
    int64_t fl = num / den, rem = num % den;
    if (fl >= nc - 1) {
      i0[i] = i1[i] = nc - 1;
      w[i] = 0.0;
    } else if (rem == 0) {
      i0[i] = i1[i] = (int)fl;
      w[i] = 0.0;
    } else {
      i0[i] = (int)fl;
      i1[i] = (int)fl + 1;
      w[i] = (double)rem / (double)den;
    }
  }
}

/* Piecewise constant interpolation (Sec. 3, "works nearly as well"): a fine
 * cell takes the value of the coarse cell that contains its centre,
 * floor((2i+1) nc / (2 nf)). */
void or_transfer_table_pc(int nf, int nc, int *i0, int *i1, double *w) {
  for (int i = 0; i < nf; ++i) {
    i0[i] = i1[i] = (int)(((2 * (int64_t)i + 1) * nc) / (2 * (int64_t)nf));
    w[i] = 0.0;
  }
}

/* x_f += E x_c (scatter-free: each fine cell reads its interpolation corners) */
static void prolong_add(const or_level *F, const or_level *Cc, const double *xc, double *xf) {
  for (int k = 0; k < F->nz; ++k)
    for (int j = 0; j < F->ny; ++j)
      for (int i = 0; i < F->nx; ++i) {
        int ia[2] = {F->i0[0][i], F->i1[0][i]}, ja[2] = {F->i0[1][j], F->i1[1][j]}, ka[2] = {F->i0[2][k], F->i1[2][k]};
        double wa[2] = {1.0 - F->w[0][i], F->w[0][i]};
        double wb[2] = {1.0 - F->w[1][j], F->w[1][j]};
        double wc[2] = {1.0 - F->w[2][k], F->w[2][k]};
        double v = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
              v += wc[c] * wb[b] * wa[a] * xc[idx3(ia[a], ja[b], ka[c], Cc->nx, Cc->ny)];
        xf[idx3(i, j, k, F->nx, F->ny)] += v;
      }
}

/* r_c = R r_f = E^T r_f: every fine value is sent to the coarse cells it was
 * interpolated from, with the same weights. */
static void restrict_(const or_level *F, const or_level *Cc, const double *rf, double *rc) {
  memset(rc, 0, sizeof(double) * Cc->n);
  for (int k = 0; k < F->nz; ++k)
    for (int j = 0; j < F->ny; ++j)
      for (int i = 0; i < F->nx; ++i) {
        int ia[2] = {F->i0[0][i], F->i1[0][i]}, ja[2] = {F->i0[1][j], F->i1[1][j]}, ka[2] = {F->i0[2][k], F->i1[2][k]};
        double wa[2] = {1.0 - F->w[0][i], F->w[0][i]};
        double wb[2] = {1.0 - F->w[1][j], F->w[1][j]};
        double wc[2] = {1.0 - F->w[2][k], F->w[2][k]};
        double v = rf[idx3(i, j, k, F->nx, F->ny)];
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
              rc[idx3(ia[a], ja[b], ka[c], Cc->nx, Cc->ny)] += wc[c] * wb[b] * wa[a] * v;
      }
}

/* ---------------------------------------------------------------------------
 * Operator, Sec. 3: (A x)_c = sum over the faces of c of T_f (x_c - x_nb);
 * a boundary face has no neighbour and contributes T_f x_c.
 * ------------------------------------------------------------------------- */
static double T_xl(const or_level *L, int i, int j, int k) { return L->Tx[(int64_t)i + (int64_t)(L->nx + 1) * ((int64_t)j + (int64_t)L->ny * k)]; }
static double T_yl(const or_level *L, int i, int j, int k) { return L->Ty[(int64_t)i + (int64_t)L->nx * ((int64_t)j + (int64_t)(L->ny + 1) * k)]; }
static double T_zl(const or_level *L, int i, int j, int k) { return L->Tz[(int64_t)i + (int64_t)L->nx * ((int64_t)j + (int64_t)L->ny * k)]; }

static void apply(const or_level *L, const double *x, double *y) {
  int nx = L->nx, ny = L->ny, nz = L->nz, d3 = L->Tz != NULL;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = idx3(i, j, k, nx, ny);
        double xc = x[c], s = 0.0, t;
        t = T_xl(L, i, j, k);
        s += i > 0 ? t * (xc - x[c - 1]) : t * xc;
        t = T_xl(L, i + 1, j, k);
        s += i < nx - 1 ? t * (xc - x[c + 1]) : t * xc;
        t = T_yl(L, i, j, k);
        s += j > 0 ? t * (xc - x[c - nx]) : t * xc;
        t = T_yl(L, i, j + 1, k);
        s += j < ny - 1 ? t * (xc - x[c + nx]) : t * xc;
        if (d3) {
          int64_t pl = (int64_t)nx * ny;
          t = T_zl(L, i, j, k);
          s += k > 0 ? t * (xc - x[c - pl]) : t * xc;
          t = T_zl(L, i, j, k + 1);
          s += k < nz - 1 ? t * (xc - x[c + pl]) : t * xc;
        }
        y[c] = s;
      }
}

/* ---------------------------------------------------------------------------
 * Splitting, Sec. 3: symmetric Gauss-Seidel P = (D+L) D^-1 (D+U), Q = L D^-1 U,
 * in red-black order.  One step x <- x + P^-1 (rhs - A x) is a forward sweep
 * (red cells, then black) followed by a backward sweep (black, then red).
 * Each cell update solves row c of A for x_c with the neighbours fixed.
 * ------------------------------------------------------------------------- */
/* Gauss-Seidel update of cell (i, j, k): row c of A solved for x_c with the
 * neighbours held at their current values. */
static void gs_cell(const or_level *L, int i, int j, int k, const double *rhs, double *x) {
  int nx = L->nx, ny = L->ny, nz = L->nz, d3 = L->Tz != NULL;
  int64_t c = idx3(i, j, k, nx, ny);
  double d = 0.0, s = rhs[c], t;
  t = T_xl(L, i, j, k);
  d += t;
  if (i > 0) s += t * x[c - 1];
  t = T_xl(L, i + 1, j, k);
  d += t;
  if (i < nx - 1) s += t * x[c + 1];
  t = T_yl(L, i, j, k);
  d += t;
  if (j > 0) s += t * x[c - nx];
  t = T_yl(L, i, j + 1, k);
  d += t;
  if (j < ny - 1) s += t * x[c + nx];
  if (d3) {
    int64_t pl = (int64_t)nx * ny;
    t = T_zl(L, i, j, k);
    d += t;
    if (k > 0) s += t * x[c - pl];
    t = T_zl(L, i, j, k + 1);
    d += t;
    if (k < nz - 1) s += t * x[c + pl];
  }
  x[c] = s / d;
}

static void colour_sweep(const or_level *L, int colour, const double *rhs, double *x) {
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i)
        if (((i + j + k) & 1) == colour) gs_cell(L, i, j, k, rhs, x);
}

/* Symmetric Gauss-Seidel in the natural order of the unknowns (i fastest,
 * then j, then k), the ordering in which A = D + U + L is read literally:
 * a forward sweep over c = 0 .. N-1, then a backward sweep over N-1 .. 0. */
static void lex_sgs_step(const or_level *L, const double *rhs, double *x) {
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i) gs_cell(L, i, j, k, rhs, x);
  for (int k = L->nz - 1; k >= 0; --k)
    for (int j = L->ny - 1; j >= 0; --j)
      for (int i = L->nx - 1; i >= 0; --i) gs_cell(L, i, j, k, rhs, x);
}

static void sgs_step(const or_level *L, const double *rhs, double *x) {
  colour_sweep(L, 0, rhs, x); /* forward: red */
  colour_sweep(L, 1, rhs, x); /* forward: black */
  colour_sweep(L, 1, rhs, x); /* backward: black */
  colour_sweep(L, 0, rhs, x); /* backward: red */
}

/* ---------------------------------------------------------------------------
 * Modified Jacobi splitting, Sec. 3: P = 2D, Q = D - U - L.  One step
 * x <- x + P^-1 (rhs - A x) updates every cell from the old values:
 * x_c += (rhs_c - (A x)_c) / (2 D_c), D_c = sum of the cell's face T.
 * ------------------------------------------------------------------------- */
static void jacobi_step(const or_level *L, const double *rhs, double *x) {
  int nx = L->nx, ny = L->ny, nz = L->nz, d3 = L->Tz != NULL;
  apply(L, x, L->aw);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = idx3(i, j, k, nx, ny);
        double d = T_xl(L, i, j, k) + T_xl(L, i + 1, j, k) + T_yl(L, i, j, k) + T_yl(L, i, j + 1, k);
        if (d3) d += T_zl(L, i, j, k) + T_zl(L, i, j, k + 1);
        x[c] += (rhs[c] - L->aw[c]) / (2.0 * d);
      }
}

static void smooth_step(const or_hier *H, const or_level *L, const double *rhs, double *x) {
  if (H->splitting == 1) jacobi_step(L, rhs, x);
  else if (H->splitting == 2) lex_sgs_step(L, rhs, x);
  else sgs_step(L, rhs, x);
}

static double dot(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* ---------------------------------------------------------------------------
 * Coarsest level, Sec. 2.2/2.3: solved exactly.  Dense assembly from T and a
 * plain Cholesky factorisation A = C C^T.
 * ------------------------------------------------------------------------- */
static void dense_assemble(const or_level *L, double *A) {
  int64_t n = L->n;
  double *e = calloc(n, sizeof(double)), *col = malloc(sizeof(double) * n);
  for (int64_t j = 0; j < n; ++j) {
    e[j] = 1.0;
    apply(L, e, col);
    for (int64_t i = 0; i < n; ++i) A[i * n + j] = col[i];
    e[j] = 0.0;
  }
  free(e);
  free(col);
}

static int cholesky(double *A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return OR_EBREAKDOWN;
    d = sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
    for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
  }
  return OR_OK;
}

static void chol_solve(const double *C, int n, const double *b, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= C[i * n + k] * x[k];
    x[i] = s / C[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= C[k * n + i] * x[k];
    x[i] = s / C[i * n + i];
  }
}

/* ---------------------------------------------------------------------------
 * Hierarchy.
 * ------------------------------------------------------------------------- */
void or_free(or_hier *H) {
  if (!H) return;
  for (int k = 0; k < H->nlev; ++k) {
    or_level *L = &H->L[k];
    free(L->Tx);
    free(L->Ty);
    free(L->Tz);
    for (int a = 0; a < 3; ++a) {
      free(L->i0[a]);
      free(L->i1[a]);
      free(L->w[a]);
    }
    free(L->b);
    free(L->x);
    free(L->r);
    free(L->p);
    free(L->z);
    free(L->q);
    free(L->t);
    free(L->aw);
  }
  free(H->chol);
  free(H);
}

/* opts: s, m, f, coarsest side limit, max outer / inner iterations, level-side
 * rule (0: factor s per long axis, 1: toward square cells), interpolation
 * (0: linear with zero slope at the boundary, 1: piecewise constant) */
/* Level-0 permeabilities: cell values with boundary types (K, ncomp, bc), or
 * face values with the boundary conditions in them (Kf[0..2], Kf[0] set). */
static or_hier *build_hier(int dim, const int n[3], const double h[3], const double *K, int ncomp,
                           const unsigned char *bc, const double *const *Kf, int s, int m, double f, int maxside,
                           int maxit_outer, int maxit_inner, int coarsening, int interp) {
  int dims[OR_MAXLEV * 3];
  int nlev = or_hierarchy_dims2(dim, n, h, s, maxside, coarsening, OR_MAXLEV, dims);
  if (interp < 0 || interp > 1) return NULL;
  if (nlev < 1) return NULL;
  or_hier *H = calloc(1, sizeof(or_hier));
  H->dim = dim;
  H->nlev = nlev;
  H->s = s;
  H->m = m;
  H->f = f;
  H->maxit_outer = maxit_outer;
  H->maxit_inner = maxit_inner;
  for (int k = 0; k < nlev; ++k) {
    or_level *L = &H->L[k];
    L->nx = dims[3 * k];
    L->ny = dims[3 * k + 1];
    L->nz = dims[3 * k + 2];
    L->n = (int64_t)L->nx * L->ny * L->nz;
    L->Tx = calloc((int64_t)(L->nx + 1) * L->ny * L->nz, sizeof(double));
    L->Ty = calloc((int64_t)L->nx * (L->ny + 1) * L->nz, sizeof(double));
    if (dim == 3) L->Tz = calloc((int64_t)L->nx * L->ny * (L->nz + 1), sizeof(double));
    L->b = calloc(L->n, sizeof(double));
    L->x = calloc(L->n, sizeof(double));
    L->r = calloc(L->n, sizeof(double));
    L->p = calloc(L->n, sizeof(double));
    L->z = calloc(L->n, sizeof(double));
    L->q = calloc(L->n, sizeof(double));
    L->t = calloc(L->n, sizeof(double));
    L->aw = calloc(L->n, sizeof(double));
  }
  if (Kf) or_face_trans_faces(dim, n, h, Kf[0], Kf[1], Kf[2], H->L[0].Tx, H->L[0].Ty, H->L[0].Tz);
  else or_face_trans(dim, n, h, K, ncomp, bc, H->L[0].Tx, H->L[0].Ty, H->L[0].Tz);
  for (int k = 0; k + 1 < nlev; ++k) {
    or_level *F = &H->L[k], *C = &H->L[k + 1];
    int nf[3] = {F->nx, F->ny, F->nz}, nc[3] = {C->nx, C->ny, C->nz};
    or_upscale(dim, nf, nc, F->Tx, F->Ty, F->Tz, C->Tx, C->Ty, C->Tz);
    for (int a = 0; a < 3; ++a) {
      F->i0[a] = malloc(sizeof(int) * nf[a]);
      F->i1[a] = malloc(sizeof(int) * nf[a]);
      F->w[a] = malloc(sizeof(double) * nf[a]);
      if (interp == 1) or_transfer_table_pc(nf[a], nc[a], F->i0[a], F->i1[a], F->w[a]);
      else or_transfer_table(nf[a], nc[a], F->i0[a], F->i1[a], F->w[a]);
    }
  }
  or_level *Lc = &H->L[nlev - 1];
  H->nc = (int)Lc->n;
  H->chol = malloc(sizeof(double) * Lc->n * Lc->n);
  dense_assemble(Lc, H->chol);
  if (cholesky(H->chol, H->nc) != OR_OK) {
    or_free(H);
    return NULL;
  }
  return H;
}

or_hier *or_build(int dim, const int n[3], const double h[3], const double *K, int ncomp, const unsigned char *bc,
                  int s, int m, double f, int maxside, int maxit_outer, int maxit_inner, int coarsening, int interp) {
  return build_hier(dim, n, h, K, ncomp, bc, NULL, s, m, f, maxside, maxit_outer, maxit_inner, coarsening, interp);
}

/* The same hierarchy from face permeabilities (or_face_trans_faces). */
or_hier *or_build_faces(int dim, const int n[3], const double h[3], const double *Kx, const double *Ky,
                        const double *Kz, int s, int m, double f, int maxside, int maxit_outer, int maxit_inner,
                        int coarsening, int interp) {
  const double *Kf[3] = {Kx, Ky, Kz};
  return build_hier(dim, n, h, NULL, 0, NULL, Kf, s, m, f, maxside, maxit_outer, maxit_inner, coarsening, interp);
}

int or_nlev(const or_hier *H) { return H->nlev; }
void or_level_dims(const or_hier *H, int k, int *d) {
  d[0] = H->L[k].nx;
  d[1] = H->L[k].ny;
  d[2] = H->L[k].nz;
}
void or_get_T(const or_hier *H, int k, double *Tx, double *Ty, double *Tz) {
  const or_level *L = &H->L[k];
  memcpy(Tx, L->Tx, sizeof(double) * (L->nx + 1) * L->ny * L->nz);
  memcpy(Ty, L->Ty, sizeof(double) * L->nx * (L->ny + 1) * L->nz);
  if (L->Tz && Tz) memcpy(Tz, L->Tz, sizeof(double) * L->nx * L->ny * (L->nz + 1));
}
void or_set_eps2(or_hier *H, double eps2) { H->eps2 = eps2; }
/* 0: symmetric Gauss-Seidel (red-black), 1: modified Jacobi, 2: symmetric
 * Gauss-Seidel in the natural order (Sec. 3) */
void or_set_splitting(or_hier *H, int splitting) { H->splitting = splitting; }
/* 0: recursive multi-scale (eq. 2.10), 1: multigrid V-step (eq. 2.9),
 * 2: polynomial (eq. 2.6 with W = P^-1) */
void or_set_precond(or_hier *H, int precond) { H->precond = precond; }
void or_get_stats(const or_hier *H, int64_t *iters, int64_t *calls) {
  for (int k = 0; k < H->nlev; ++k) {
    iters[k] = H->iters[k];
    calls[k] = H->calls[k];
  }
}
void or_reset_stats(or_hier *H) {
  memset(H->iters, 0, sizeof(H->iters));
  memset(H->calls, 0, sizeof(H->calls));
  H->status = OR_OK;
}

/* ---------------------------------------------------------------------------
 * Recursive multi-scale preconditioner, eq. (2.10) with m = s (Sec. 3):
 * m smoothing steps from zero, the coarse correction E A_c^-1 R on the
 * residual that remains, then m smoothing steps.  A_c^-1 is applied by the
 * PCG of the next level (Sec. 2.3); the coarsest level uses the exact inverse.
 *
 * The two other preconditioners of Sec. 2 share the smoothing and transfers:
 *  - multigrid (eq. 2.9, Tatebe): the same form with the coarse inverse
 *    replaced by one application of the next level's preconditioner
 *    M_{k+1}^-1, recursively, ending with the exact coarsest inverse;
 *  - polynomial (Sec. 2.1, eq. 2.6 with W = P^-1): the first 2m+1 terms of
 *    the series (2.4), sum_{j=0}^{2m} (P^-1 Q)^j P^-1, i.e. 2m+1 splitting
 *    steps from zero on the level itself, no coarse level.
 * ------------------------------------------------------------------------- */
static void pcg(or_hier *H, int k, const double *b, double *x);

static void precond(or_hier *H, int k, const double *r, double *z) {
  or_level *L = &H->L[k];
  if (k == H->nlev - 1) {
    chol_solve(H->chol, H->nc, r, z);
    return;
  }
  memset(z, 0, sizeof(double) * L->n);
  if (H->precond == 2) {
    for (int s = 0; s < 2 * H->m + 1; ++s) smooth_step(H, L, r, z);
    return;
  }
  or_level *C = &H->L[k + 1];
  for (int s = 0; s < H->m; ++s) smooth_step(H, L, r, z);
  apply(L, z, L->t);
  for (int64_t i = 0; i < L->n; ++i) L->t[i] = r[i] - L->t[i];
  restrict_(L, C, L->t, C->b);
  if (H->precond == 1) {
    H->calls[k + 1]++;
    precond(H, k + 1, C->b, C->x);
  } else {
    pcg(H, k + 1, C->b, C->x);
  }
  prolong_add(L, C, C->x, z);
  for (int s = 0; s < H->m; ++s) smooth_step(H, L, r, z);
}

/* ---------------------------------------------------------------------------
 * Conjugate gradient, Templates Fig. 2.5 as cited in Sec. 3, started from
 * x = 0.  Convergence on level k (Sec. 3): ||r||^2 / N_k < f^k eps^2, tested
 * after each update.  Level 0 uses eps^2 = tau^2 ||b||^2 / N_0.
 * ------------------------------------------------------------------------- */
static void pcg_run(or_hier *H, int k, const double *b, double *x) {
  or_level *L = &H->L[k];
  int64_t n = L->n;
  double fk = 1.0;
  for (int i = 0; i < k; ++i) fk *= H->f;
  double thr = fk * H->eps2;
  int maxit = k == 0 ? H->maxit_outer : H->maxit_inner;
  H->calls[k]++;
  memset(x, 0, sizeof(double) * n);
  memcpy(L->r, b, sizeof(double) * n);
  double bb = dot(b, b, n);
  if (bb == 0.0) return;
  double rho_old = 0.0;
  for (int it = 0;; ++it) {
    precond(H, k, L->r, L->z);
    double rho = dot(L->r, L->z, n);
    if (it == 0) {
      memcpy(L->p, L->z, sizeof(double) * n);
    } else {
      double beta = rho / rho_old;
      for (int64_t i = 0; i < n; ++i) L->p[i] = L->z[i] + beta * L->p[i];
    }
    apply(L, L->p, L->q);
    double pq = dot(L->p, L->q, n);
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rho)) {
      H->status = OR_EBREAKDOWN;
      return;
    }
    double alpha = rho / pq;
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * L->p[i];
    for (int64_t i = 0; i < n; ++i) L->r[i] -= alpha * L->q[i];
    H->iters[k]++;
    double rr = dot(L->r, L->r, n);
    if (rr / (double)n < thr) return;
    if (it + 1 >= maxit) {
      H->status = OR_ENOCONV;
      return;
    }
    rho_old = rho;
  }
}

/* One PCG call of level k and its entry in the level tree (Fig. 2: the
 * iterations each call of each level takes).  The call's index is the
 * level's call counter before it. */
static void pcg(or_hier *H, int k, const double *b, double *x) {
  const int64_t call = H->calls[k], it0 = H->iters[k];
  pcg_run(H, k, b, x);
  if (H->trace) {
    if (H->trace_n < H->trace_cap) {
      int32_t *e = H->trace + 4 * H->trace_n;
      e[0] = k;
      e[1] = (int32_t)call;
      e[2] = (int32_t)(H->iters[k] - it0);
      e[3] = H->pass;
    }
    H->trace_n++;
  }
}

void or_set_trace(or_hier *H, int32_t *buf, int64_t cap) {
  H->trace = buf;
  H->trace_cap = buf ? cap : 0;
  H->trace_n = 0;
}
int64_t or_trace_count(const or_hier *H) { return H->trace_n; }

/* Solve A x = b to relative residual tau.  The level-0 PCG runs on the
 * recursive residual; afterwards the true residual b - A x is formed and, if
 * it misses tau, the PCG is restarted from it (at most 3 restarts).
 * out[0] = recursive relative residual, out[1] = true relative residual. */
int or_solve(or_hier *H, const double *b, double tau, double *x, double *out) {
  or_level *L = &H->L[0];
  int64_t n = L->n;
  double bb = dot(b, b, n);
  or_reset_stats(H);
  H->trace_n = 0;
  H->pass = 0;
  memset(x, 0, sizeof(double) * n);
  out[0] = out[1] = 0.0;
  if (bb == 0.0) return OR_OK;
  H->eps2 = tau * tau * (bb / (double)n);
  double *rt = malloc(sizeof(double) * n), *dx = malloc(sizeof(double) * n);
  memcpy(rt, b, sizeof(double) * n);
  for (int restart = 0; restart < 4; ++restart) {
    H->pass = restart;
    pcg(H, 0, rt, dx);
    for (int64_t i = 0; i < n; ++i) x[i] += dx[i];
    out[0] = sqrt(dot(L->r, L->r, n) / bb);
    apply(L, x, rt);
    for (int64_t i = 0; i < n; ++i) rt[i] = b[i] - rt[i];
    out[1] = sqrt(dot(rt, rt, n) / bb);
    if (H->status != OR_OK || out[1] < tau) break;
  }
  free(rt);
  free(dx);
  return H->status;
}

/* ---------------------------------------------------------------------------
 * Level-wise entry points for the tests.
 * ------------------------------------------------------------------------- */
void or_apply_level(const or_hier *H, int k, const double *x, double *y) { apply(&H->L[k], x, y); }
void or_sgs_level(const or_hier *H, int k, const double *rhs, double *x) { sgs_step(&H->L[k], rhs, x); }
void or_jacobi_level(const or_hier *H, int k, const double *rhs, double *x) { jacobi_step(&H->L[k], rhs, x); }
void or_lex_level(const or_hier *H, int k, const double *rhs, double *x) { lex_sgs_step(&H->L[k], rhs, x); }
void or_sweep_level(const or_hier *H, int k, int colour, const double *rhs, double *x) {
  colour_sweep(&H->L[k], colour, rhs, x);
}
void or_restrict_level(const or_hier *H, int k, const double *rf, double *rc) {
  restrict_(&H->L[k], &H->L[k + 1], rf, rc);
}
void or_prolong_level(const or_hier *H, int k, const double *xc, double *xf) {
  prolong_add(&H->L[k], &H->L[k + 1], xc, xf);
}
void or_precond_level(or_hier *H, int k, const double *r, double *z) { precond(H, k, r, z); }
void or_pcg_level(or_hier *H, int k, const double *b, double *x) { pcg(H, k, b, x); }
int or_status(const or_hier *H) { return H->status; }

/* ---------------------------------------------------------------------------
 * Boundary lifting, Sec. 3: with a field P_bf that matches the boundary
 * values, solve for dP = P - P_bf with zero boundary data; the right-hand side
 * becomes  b = f vol + g_D - A P_bf,  where g_D collects T_f p_D over the
 * Dirichlet faces of each boundary cell (the boundary source term).
 * gD has the layout of bc; f is the source density per cell.
 * ------------------------------------------------------------------------- */
void or_lift_rhs(const or_hier *H, const double h[3], const unsigned char *bc, const double *gD, const double *f,
                 const double *pbf, double *b) {
  const or_level *L = &H->L[0];
  int nx = L->nx, ny = L->ny, nz = L->nz, d3 = H->dim == 3;
  double vol = h[0] * h[1] * (d3 ? h[2] : 1.0);
  const unsigned char *bx0 = bc, *bx1 = bc + (int64_t)ny * nz;
  const unsigned char *by0 = bx1 + (int64_t)ny * nz, *by1 = by0 + (int64_t)nx * nz;
  const unsigned char *bz0 = by1 + (int64_t)nx * nz, *bz1 = bz0 + (int64_t)nx * ny;
  const double *gx0 = gD, *gx1 = gD + (int64_t)ny * nz;
  const double *gy0 = gx1 + (int64_t)ny * nz, *gy1 = gy0 + (int64_t)nx * nz;
  const double *gz0 = gy1 + (int64_t)nx * nz, *gz1 = gz0 + (int64_t)nx * ny;
  double *Ap = malloc(sizeof(double) * L->n);
  apply(L, pbf, Ap);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t c = idx3(i, j, k, nx, ny);
        double v = f ? f[c] * vol : 0.0;
        if (i == 0 && bx0[j + (int64_t)ny * k]) v += T_xl(L, 0, j, k) * gx0[j + (int64_t)ny * k];
        if (i == nx - 1 && bx1[j + (int64_t)ny * k]) v += T_xl(L, nx, j, k) * gx1[j + (int64_t)ny * k];
        if (j == 0 && by0[i + (int64_t)nx * k]) v += T_yl(L, i, 0, k) * gy0[i + (int64_t)nx * k];
        if (j == ny - 1 && by1[i + (int64_t)nx * k]) v += T_yl(L, i, ny, k) * gy1[i + (int64_t)nx * k];
        if (d3) {
          if (k == 0 && bz0[i + (int64_t)nx * j]) v += T_zl(L, i, j, 0) * gz0[i + (int64_t)nx * j];
          if (k == nz - 1 && bz1[i + (int64_t)nx * j]) v += T_zl(L, i, j, nz) * gz1[i + (int64_t)nx * j];
        }
        b[c] = v - Ap[c];
      }
  free(Ap);
}
