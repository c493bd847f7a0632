/*
 * msrcg — recursive multi-scale preconditioned conjugate gradient on GB300.
 *
 * C ABI of libmsrcg.so.  Method: Lackner & Menikoff, "Multi-scale linear
 * solvers for very large systems derived from PDEs" (arXiv math/9809043):
 * a PCG (Sec. 3, Templates Fig. 2.5) whose preconditioner, eq. (2.10), is m
 * symmetric Gauss-Seidel steps, a coarse correction E A_c^-1 R in which A_c^-1
 * is applied by the same PCG one level down (Sec. 2.3), and m more smoothing
 * steps; the coarsest level is solved exactly.  The operator is the
 * cell-centred 5-point (2D) / 7-point (3D) discretisation of -div(K grad p)
 * with harmonic-mean face permeabilities (Sec. 3).
 *
 * Conventions shared by every entry point
 *  - Cells are numbered c = i + nx*(j + ny*k), x fastest.
 *  - "device" arrays live in the memory of the current CUDA device; the
 *    caller owns them and keeps them alive until the stream has passed the
 *    call.  "host" arrays are read before the call returns.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream ordered; a call returns once the work is enqueued unless it says
 *    that it synchronises.
 *  - Return value: MSRCG_OK (0) or a negative MSRCG_E* code;
 *    msrcg_strerror() names it.  No entry point falls back to the CPU.
 */
#ifndef MSRCG_H
#define MSRCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSRCG_OK 0
#define MSRCG_EINVAL (-1)      /* malformed argument */
#define MSRCG_ENOMEM (-2)      /* device allocation failed */
#define MSRCG_ENOCONV (-3)     /* a level hit its iteration cap */
#define MSRCG_EBREAKDOWN (-4)  /* p.Ap <= 0 or a non-finite CG scalar */
#define MSRCG_ETIMEOUT (-5)    /* a bounded device wait ran out */
#define MSRCG_ENANINF (-6)     /* non-finite value in b */
#define MSRCG_ECUDA (-7)       /* a CUDA runtime call failed */

#define MSRCG_MAXLEV 16

/* Grid: dim = 2 or 3; n = cells per axis (n[2] ignored in 2D); h = cell
 * sizes (h[2] ignored in 2D). */
typedef struct {
  int dim;
  int n[3];
  double h[3];
} msrcg_grid;

/* Method parameters (Sec. 3): scale factor s (about 4), smoothing degree m
 * (= s), level tolerance factor f (0.1), coarsest side limit (a level whose
 * every side is <= this is the coarsest; 0 = 8 in 2D, 4 in 3D), precision
 * (0 = FP64 everywhere, 1 = FP32 preconditioner inside the FP64 outer PCG),
 * iteration caps per level-0 PCG / inner PCG call, the bound of every
 * device-side wait in nanoseconds, and inner_floor (precision 1 only: an
 * inner level also stops once ||r_k|| < inner_floor ||b_k||; 0 disables). */
typedef struct {
  int scale;
  int m;
  double f;
  int coarsest_max_side;
  int precision;
  int maxit_outer;
  int maxit_inner;
  uint64_t timeout_ns;
  double inner_floor;
  int small_cells;   /* levels with at most this many cells run in one CTA; 0 = default */
  int plain_sweeps;  /* 1: one pass over a level per red/black half-sweep everywhere; 0 (default):
                        2D FP32-preconditioner levels in global memory that the single-CTA solver
                        handles run all half-sweeps of one smoothing in a single pass over the
                        level (same values, fewer memory passes) */
  int fuse_width;      /* single-pass smoothing: most output columns per strip (0 = as many as the
                          shared memory holds); a tile shape the autotuner may set */
  int fuse_min_cells;  /* single-pass smoothing only on levels of at least this many cells
                          (0 = 4096) */
  int splitting;       /* smoother of eq. 2.10 (Sec. 3): 0 = symmetric Gauss-Seidel in red-black
                          order (default), 1 = modified Jacobi P = 2D, Q = D - U - L,
                          2 = symmetric Gauss-Seidel in the natural order of the cells (a
                          wavefront over the planes i+j+k = d; single solves then run every
                          level in one CTA) */
  int coarsening;      /* level sides: 0 = every axis longer than the coarsest side shrinks by
                          `scale`; 1 = toward square cells (Sec. 4.4 semi-coarsening): the coarse
                          cell size is `scale` times the level's smallest cell size, an axis is
                          never refined, and the level where no axis changes is the coarsest */
  int interp;          /* extension E (R = E^T): 0 = tensor linear interpolation with zero slope at
                          the boundary, 1 = piecewise constant (Sec. 3) */
  int stall_iters;     /* precision 1, precond 0: stall test of the level-0 PCG: when its residual
                          norm has not
                          halved for
                          this many iterations it switches to the flexible (Polak-Ribiere) direction
                          factor beta = r_new.(z_new - z_old) / r_old.z_old, which keeps the CG
                          directions useful when the preconditioner is not exactly linear (the
                          inexact inner solves of Sec. 2.3, FP32 inner levels); stalling again
                          ends the solve with MSRCG_ENOCONV.  0 = 30 (the CG residual's 2-norm is
                          not monotone: a short window stops slow but steady solves); negative = no
                          stall test.
                          With precision 1 an inner level that hits its iteration cap also switches
                          the level-0 PCG to the flexible beta instead of failing the solve. */
  int escalate;        /* precision 1: a solve that ends in MSRCG_ENOCONV is run again with the FP64
                          preconditioner (a twin hierarchy built on the device from the level-0
                          transmissibilities, kept for later solves); 1 (default) = on, 0 = off.
                          Applies to calls that synchronise (msrcg_solve with stats, batch) and to
                          the server's requests; not to msrcg_solve_static (it cannot allocate). */
  int flexible;        /* 1: the flexible beta from the first iteration (testing); 0 (default) */
  int precond;         /* preconditioner of the level-0 PCG (Sec. 2): 0 = recursive multi-scale,
                          eq. 2.10 (default); 1 = multigrid, eq. 2.9 (Tatebe): each coarse level
                          applies the next one's preconditioner once instead of solving with a
                          PCG; 2 = polynomial, eq. 2.6 with W = P^-1 (Sec. 2.1): 2m+1 splitting
                          steps from zero, no coarse level.  1 and 2 run every level of a single
                          solve in one CTA. */
  int reserved[1];
} msrcg_opts;

/* Per-solve statistics.  iters[k] = PCG iterations summed over all calls at
 * level k, calls[k] = PCG invocations at level k (Table 1 of the paper). */
typedef struct {
  int levels;
  int dims[MSRCG_MAXLEV][3];
  int64_t iters[MSRCG_MAXLEV];
  int64_t calls[MSRCG_MAXLEV];
  double relres_recursive;  /* ||r||/||b|| of the level-0 recursion */
  double relres_true;       /* ||b - A x|| / ||b||, recomputed at the end */
  int status;
  int restarts;
  int flexible;             /* 1: the level-0 PCG used the flexible beta */
  int escalated;            /* 1: the result comes from the FP64-preconditioner rerun */
} msrcg_stats;

typedef struct msrcg_hier msrcg_hier;

/* Fill *o with the paper's defaults: s = m = 4, f = 0.1, FP64, caps 200/500,
 * 2 s wait bound, stall test after 30 iterations, escalation on.  Returns
 * MSRCG_OK, or MSRCG_EINVAL if o is NULL. */
int msrcg_default_opts(msrcg_opts* o);

/* Build the level hierarchy G_0..G_kmax (Sec. 2.2, 3) of one problem.
 *  grid     host; validated (dim 2/3, every n >= 1, h > 0).
 *  K        device, double, ncomp*N: cell permeability, scalar (ncomp 1) or
 *           the diagonal tensor (ncomp = dim), component-major.
 *  bc       device, uint8, one entry per boundary face (1 = Dirichlet,
 *           0 = Neumann) in blocks x-low, x-high (ny*nz each), y-low, y-high
 *           (nx*nz each), z-low, z-high (nx*ny each, 3D only).
 *  Computes on the device: face transmissibilities T = (h_perp/h_par) K_face
 *  with K_face the harmonic mean of the adjacent cells (Sec. 3; boundary
 *  Dirichlet face 2 (h_perp/h_par) K_cell, Neumann 0), the series-parallel
 *  coarse transmissibilities of every level (Sec. 3), FP32 copies, and the
 *  exact inverse of the coarsest operator (FP64 Cholesky).  The hierarchy owns
 *  all device memory it allocates.  Synchronises `stream`.
 *  Errors: MSRCG_EINVAL, MSRCG_ENOMEM, MSRCG_ECUDA, MSRCG_EBREAKDOWN (coarsest
 *  operator not positive definite). */
int msrcg_build(const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                const msrcg_opts* opts, void* stream, msrcg_hier** out);

/* Build the level hierarchy from face permeabilities (Sec. 3: the components
 * of K are face centred -- K_xx half a cell off the cell centre in x, K_yy in
 * y -- and the type of boundary condition is carried by the discretised K of
 * the boundary faces).
 *  grid  host; validated as msrcg_build.
 *  Kx    device, double, (nx+1)*ny*nz: K_xx on the x-faces, x fastest, the
 *        boundary faces i = 0 and i = nx included.  A Dirichlet boundary
 *        face holds the K of the half cell between the face and the centre
 *        (2 K_cell reproduces msrcg_build), a Neumann face holds 0.
 *  Ky    device, nx*(ny+1)*nz: K_yy on the y-faces, likewise.
 *  Kz    device, nx*ny*(nz+1) in 3D; ignored (may be NULL) in 2D.
 *  T = (h_perp/h_par) K_face on every face (one rounding); the rest of the
 *  hierarchy is built as by msrcg_build, which it equals bit for bit when
 *  the faces hold msrcg_build's harmonic means.  The arrays are read before
 *  the call returns.  Synchronises `stream`.
 *  Errors: as msrcg_build. */
int msrcg_build_faces(const msrcg_grid* grid, const double* Kx, const double* Ky, const double* Kz,
                      const msrcg_opts* opts, void* stream, msrcg_hier** out);

/* Build the hierarchy of a constant-coefficient problem (Sec. 4.1, the
 * solver specialised to the Laplace operator): K the same in every cell,
 * each side of the domain entirely Dirichlet or entirely Neumann.
 *  grid     host; validated as msrcg_build.
 *  K        host, 3 doubles: K_xx, K_yy (, K_zz) of every cell, > 0 (the
 *           third ignored in 2D).
 *  side_bc  host, 6 bytes: the boundary type of the sides x-low, x-high,
 *           y-low, y-high, z-low, z-high (1 = Dirichlet, 0 = Neumann; the
 *           z entries ignored in 2D).
 *  Level k's interior faces all carry (h_perp/h_par) K of its cells (the
 *  domain fixed, cells of size L/n_k), a Dirichlet face twice that, a Neumann
 *  face 0: what the series-parallel coarsening of a constant field gives.
 *  No face array is stored in full -- one x row, four y rows (and z planes)
 *  per level -- so the smoother and the operator read almost no coefficient
 *  data.  The result solves, applies and lifts as any hierarchy
 *  (msrcg_get_trans returns the full arrays); msrcg_lift_rhs takes the
 *  usual per-face boundary layout.  Synchronises `stream`.
 *  Errors: MSRCG_EINVAL (bad grid, K <= 0, a side_bc entry > 1),
 *  MSRCG_ENOMEM, MSRCG_ECUDA. */
int msrcg_build_laplace(const msrcg_grid* grid, const double K[3], const uint8_t side_bc[6], const msrcg_opts* opts,
                        void* stream, msrcg_hier** out);

/* Right-hand side of the lifted problem, Sec. 3: with a field P_bf that
 * matches the boundary values, writes b = f*vol + g_D - A P_bf, where g_D
 * sums T_face * gD over the Dirichlet faces of each boundary cell.
 *  bc, gD   device, the boundary layout of msrcg_build (gD = Dirichlet value).
 *  f        device, N source densities, or NULL for no source.
 *  pbf      device, N values of the lifting field.
 *  b        device, N, output.  Errors: MSRCG_EINVAL, MSRCG_ECUDA. */
int msrcg_lift_rhs(msrcg_hier* h, const uint8_t* bc, const double* gD, const double* f,
                   const double* pbf, double* b, void* stream);

/* Solve A x = b to relative residual tol with the recursive multi-scale PCG
 * (eq. 2.10, Sec. 3): level k stops once ||r||^2/N_k < f^k eps^2 with
 * eps^2 = tol^2 ||b||^2 / N_0.  x starts from zero.
 *  b  device, N doubles (read only).   x  device, N doubles (output).
 *  stats  host, or NULL.  With stats != NULL the call synchronises `stream`
 *  to read the counters; with NULL it only enqueues (no restart on a missed
 *  true residual in that case).
 *  Errors: MSRCG_EINVAL, MSRCG_ENANINF, MSRCG_ENOCONV, MSRCG_EBREAKDOWN,
 *  MSRCG_ETIMEOUT, MSRCG_ECUDA.  The hierarchy is reusable after an error. */
int msrcg_solve(msrcg_hier* h, const double* b, double tol, double* x, msrcg_stats* stats,
                void* stream);

/* Solve `count` independent problems, each with its own hierarchy, in one
 * persistent launch: one CTA runs the whole recursion of one problem, CTAs
 * take problems largest first.  The hierarchies must be distinct and built
 * on the current device.
 *  hs, b, x  host arrays of `count` entries; b[i], x[i] device, N_i doubles.
 *  stats     host, `count` entries, or NULL.  Synchronises `stream`.
 *  Errors: as msrcg_solve; the first failing problem's code is returned. */
int msrcg_batch_solve(int count, msrcg_hier* const* hs, const double* const* b, double tol,
                      double* const* x, msrcg_stats* stats, void* stream);

/* Level k's dimensions (dims[3], host) and the iteration / call counters of
 * the last solve.  Errors: MSRCG_EINVAL for a bad level. */
int msrcg_level_info(const msrcg_hier* h, int level, int dims[3], int64_t* iters, int64_t* calls);

/* The level tree of the solves of h (Fig. 2 of the paper: how many iterations
 * each call of each level's PCG takes, Sec. 3).  buf: device memory the
 * caller owns and keeps alive while attached, 16-byte aligned,
 * 16 + 16 * capacity bytes: a uint64 entry count (set to 0 at the start of
 * every msrcg_solve / msrcg_batch_solve of h; it counts past `capacity`, the
 * entries beyond are dropped), 8 unused bytes, then `capacity` entries of
 * four int32: level, call (0-based index of this call of the level's PCG
 * within the solve), iterations of that call, pass (0, or 1..3 for the
 * restarts from the true residual).  One entry per PCG call, written when
 * the call returns (so a coarse call precedes the finer call that made it);
 * the inner levels of the multigrid preconditioner (precond 1) run no PCG
 * and have none.  buf = NULL detaches.  While a buffer is attached,
 * msrcg_solve runs every level in the single-CTA solver (one launch, no
 * graph; slower on wide levels).
 *  Errors: MSRCG_EINVAL (h NULL, capacity < 0 or above 2^31 - 1, buf not
 *  16-byte aligned). */
int msrcg_set_trace(msrcg_hier* h, void* buf, int64_t capacity);

/* Copy level k's transmissibilities (FP64) into device arrays Tx
 * ((nx+1)*ny*nz), Ty (nx*(ny+1)*nz) and, in 3D, Tz (nx*ny*(nz+1)); Tz may be
 * NULL in 2D.  Stream ordered.  Errors: MSRCG_EINVAL, MSRCG_ECUDA. */
int msrcg_get_trans(const msrcg_hier* h, int level, double* Tx, double* Ty, double* Tz, void* stream);

/* Apply level k's operator: y = A_k x, device arrays of N_k doubles (FP64
 * transmissibilities).  Stream ordered.  Errors: MSRCG_EINVAL, MSRCG_ECUDA. */
int msrcg_apply(const msrcg_hier* h, int level, const double* x, double* y, void* stream);

/* Number of levels and device bytes held by the hierarchy. */
int msrcg_num_levels(const msrcg_hier* h);
size_t msrcg_device_bytes(const msrcg_hier* h);

/* Release everything the hierarchy owns (synchronises the device first). */
void msrcg_free(msrcg_hier* h);

/* ---- serving: continuous batching of independent solves ----------------
 * A server admits requests while their estimated device memory (hierarchy,
 * right-hand side, solution) fits `budget_bytes`, builds each admitted
 * request's hierarchy on a build stream with stream-ordered allocation, and
 * on every progress call launches the requests built since the last launch
 * as one batched wave (one thread block per request, msrcg_batch_solve's
 * kernel) on a stream of its own; waves overlap on the device, so requests
 * arriving while others run start as soon as they are built.  A finished
 * wave's requests get their solution copied to the caller's buffer and
 * their memory released, which admits waiting requests.  One host thread
 * drives a server; the calls are not thread safe. */
typedef struct msrcg_server msrcg_server;

/* max_waves: streams for concurrent waves (0 = 8).  opts as msrcg_build
 * (NULL = defaults).  Errors: MSRCG_EINVAL, MSRCG_ECUDA. */
int msrcg_server_create(size_t budget_bytes, int max_waves, const msrcg_opts* opts, msrcg_server** out);

/* Queue one request.  K (ncomp*N doubles), bc (boundary mask) and b (N
 * doubles) are host arrays read when the request is admitted; x (N doubles,
 * host) receives the solution when the request finishes.  All four stay
 * valid until msrcg_server_poll reports the request done.  *id identifies
 * it.  Runs one progress step.  Errors: MSRCG_EINVAL, MSRCG_ENOMEM (the
 * request alone exceeds the budget), MSRCG_ECUDA. */
int msrcg_server_submit(msrcg_server* sv, const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                        const double* b, double tol, double* x, int64_t* id);

/* Retire finished waves, admit waiting requests, launch built ones.
 * Returns the number of requests not yet done, or a negative error. */
int msrcg_server_progress(msrcg_server* sv);

/* 1 when request `id` is done (x written, *stats filled if non-NULL; the id
 * is then forgotten), 0 while pending, a negative code if it failed. */
int msrcg_server_poll(msrcg_server* sv, int64_t id, msrcg_stats* stats);

/* Progress until every submitted request is done. */
int msrcg_server_drain(msrcg_server* sv);

/* Device bytes currently charged to admitted requests. */
size_t msrcg_server_bytes_in_use(const msrcg_server* sv);

/* Wait for the device, release everything the server holds. */
void msrcg_server_destroy(msrcg_server* sv);

/* Bytes of the fixed device scratch that msrcg_solve_static works in. */
#define MSRCG_STATIC_SCRATCH_BYTES (4u << 20)

/* Build and solve one small problem without allocating any memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc — code whose device memory is all owned by another
 * allocator (a framework's caching pool, a budget reserved at start-up) and
 * code in which an allocation is not allowed or too slow (real-time loops).
 * It does what msrcg_build followed by msrcg_solve does (same operator,
 * hierarchy and recursion; every level runs in one thread block), but every
 * device array lives in one fixed array of MSRCG_STATIC_SCRATCH_BYTES inside
 * the library, which each device that loads the library holds until the
 * process exits.  No device or host memory is allocated.
 *  grid, K, ncomp, bc, opts  as msrcg_build (opts may be NULL: defaults).
 *  b  device, N doubles (read only).   x  device, N doubles (output).
 *  stats  host, or NULL.  The call synchronises `stream` before returning.
 * Errors: MSRCG_EINVAL also when the problem's hierarchy does not fit the
 * scratch (largest square grids with the default options: 230x230 in FP64,
 * 227x227 with the FP32 preconditioner; cubes: 35^3 and 34^3), returned
 * before anything is enqueued on `stream`; otherwise as msrcg_build and
 * msrcg_solve, after the work already enqueued has finished.
 * The first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one scratch and keep the previous call's contents
 * (the call clears what must start at zero): calls that overlap on the GPU,
 * from two streams or two host threads, race and corrupt each other. */
int msrcg_solve_static(const msrcg_grid* grid, const double* K, int ncomp, const uint8_t* bc,
                       const msrcg_opts* opts, const double* b, double tol, double* x, msrcg_stats* stats,
                       void* stream);

/* ---- measurement: the multi-CTA kernels of one level, timed standalone ----
 * Not a step of the method (the paper has no counterpart): a probe of how
 * close each kernel of the single-solve path comes to the memory roofline.
 * msrcg_profile_kernel_count() kernels, named by msrcg_profile_kernel_name(i)
 * (a static string; "" for a bad index), in this order: red-black half-sweep,
 * first half-sweep from zero, last half-sweep with r.z, residual,
 * restriction, prolongation onto the black cells, CG direction, operator
 * apply with p.q, CG update with r.r. */
int msrcg_profile_kernel_count(void);
const char* msrcg_profile_kernel_name(int i);

/* Launch each kernel of level `level` (a level the single-solve path runs as
 * multi-CTA kernels: level < the first single-CTA level, and not the
 * coarsest) reps times back to back on `stream` after 3 warm-up launches;
 * ms[i] = mean duration per launch (CUDA events), bytes[i] = the kernel's
 * algorithmic bytes per launch (every array element it must read or write
 * once, in the level's precisions).  ms and bytes are host arrays of
 * msrcg_profile_kernel_count() entries.  The level's vectors are
 * overwritten with garbage (the next solve clears them first).  Synchronises
 * `stream`.  Errors: MSRCG_EINVAL (bad level or arguments), MSRCG_ECUDA. */
int msrcg_profile_level(msrcg_hier* h, int level, int reps, double* ms, double* bytes, void* stream);

/* Static description of an error code. */
const char* msrcg_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* MSRCG_H */
