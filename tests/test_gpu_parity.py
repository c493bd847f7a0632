"""GPU path vs the CPU oracle, through the C ABI (marked gpu).

Bars: transmissibilities of every level bit-exact (integer overlap tables and
explicitly rounded FP64 on both sides); operator and lifting within FP64
rounding; solutions within 1e-6 relative error of the oracle at relative
residual 1e-8 (the accuracy target of the method's GB300 build), per-level
iteration counts equal in FP64 mode up to one iteration per call where a
residual sits at a level threshold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_math_9809043_gb300 import problems as P  # noqa: E402

SOL_RTOL = 1e-6


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_math_9809043_gb300 import build as B
    B.build()
    from paper_math_9809043_gb300 import msrcg
    return msrcg


def _prob_uniform(n, seed=5, span=2.0, lifted=True):
    rng = np.random.default_rng(seed)
    dim = len(n)
    N = int(np.prod(n))
    K = (10.0 ** rng.uniform(-span, span, N)).reshape(1, -1)
    bc, gD = P.standard_bc(dim, n)
    if lifted:
        return P.Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=K, bc=bc, gD=gD,
                         pbf=P.linear_lifting(dim, n), f=rng.standard_normal(N))
    return P.Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=K, bc=bc, gD=gD,
                     b=rng.standard_normal(N))


def _maxerr(xg, xr):
    """Largest deviation relative to the largest value (element-wise bar)."""
    xg = xg.cpu().numpy() if hasattr(xg, "cpu") else np.asarray(xg)
    return np.max(np.abs(xg - xr)) / max(np.max(np.abs(xr)), 1e-300)


def _counts_close(a, b, calls):
    """Per-level iteration totals agree up to threshold flips: the GPU and
    the oracle sum the residual norms in different orders, so a norm that
    lands within rounding of a level's threshold can take one more or one
    fewer iteration; allow 3% of the total (at least 1) per level."""
    for k, (x, y) in enumerate(zip(a, b)):
        assert abs(x - y) <= max(1, int(np.ceil(0.03 * y))), (k, a, b)


# ---------------------------------------------------------------------------
# build: transmissibilities, operator, lifting
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(32, 32), (37, 23), (1, 1), (3, 2), (64, 4), (12, 10, 9), (7, 5, 3)])
def test_transmissibility_bit_exact(M, n):
    prob = _prob_uniform(n, span=4.5)
    H = M.Hierarchy.from_problem(prob)
    R = O.Hierarchy(prob)
    assert H.nlev == R.nlev
    for k in range(R.nlev):
        got = [t.cpu().numpy() if t is not None else None for t in H.trans(k)]
        ref = R.T(k)
        for a in range(prob.dim):
            assert np.array_equal(got[a], ref[a]), (k, a, np.max(np.abs(got[a] - ref[a])))


def test_transmissibility_bit_exact_full_size(M):
    prob = P.config_problem(1)  # 1024^2, 1e9 contrast
    H = M.Hierarchy.from_problem(prob)
    R = O.Hierarchy(prob)
    for k in range(R.nlev):
        got = H.trans(k)
        ref = R.T(k)
        for a in range(2):
            assert np.array_equal(got[a].cpu().numpy(), ref[a]), (k, a)


@pytest.mark.parametrize("n", [(200, 50), (2000, 500)])
def test_transmissibility_bit_exact_square_cell_coarsening(M, n):
    """10:1 cells coarsened toward square cells (an axis kept at ratio 1 on
    the first level): same level sides as the oracle, every level's T
    bit-exact."""
    prob = P.strip_problem(n)
    H = M.Hierarchy.from_problem(prob, M.default_opts(coarsening=1))
    R = O.Hierarchy(prob, coarsening=1)
    assert [H.dims(k)[0] for k in range(H.nlev)] == R.dims
    for k in range(R.nlev):
        got = H.trans(k)
        ref = R.T(k)
        for a in range(2):
            assert np.array_equal(got[a].cpu().numpy(), ref[a]), (k, a)


@pytest.mark.parametrize("n", [(32, 32), (37, 23), (9, 8, 7)])
def test_apply_and_lift(M, n):
    prob = _prob_uniform(n, span=4.5)
    H = M.Hierarchy.from_problem(prob)
    R = O.Hierarchy(prob)
    rng = np.random.default_rng(1)
    for k in range(R.nlev):
        x = rng.standard_normal(R.ncells(k))
        y = H.apply(k, torch.as_tensor(x, device="cuda")).cpu().numpy()
        yr = R.apply(k, x)
        assert np.max(np.abs(y - yr)) <= 1e-12 * np.max(np.abs(yr))
    b = H.rhs_for(prob).cpu().numpy()
    br = R.lift_rhs()
    assert np.max(np.abs(b - br)) <= 1e-12 * np.max(np.abs(br))


# ---------------------------------------------------------------------------
# solve parity
# ---------------------------------------------------------------------------
CASES = [
    ("cfg0", lambda: P.config_problem(0), 0),
    ("ragged-37x23", lambda: _prob_uniform((37, 23)), 0),
    ("ragged-37x23-wide", lambda: _prob_uniform((37, 23)), 64),
    ("grf-128", lambda: P.config_problem(1, scale=128), 0),
    ("grf-200x72-wide", lambda: P.grf_problem((200, 72), seed=21, ell=6.0, half_span=4.5), 256),
    ("strip-64x4", lambda: _prob_uniform((64, 4)), 0),
    ("tiny-3x2", lambda: _prob_uniform((3, 2)), 0),
    ("direct-rhs-50x50", lambda: _prob_uniform((50, 50), lifted=False), 128),
    ("chan3d-16", lambda: P.config_problem(2, scale=16), 0),
    ("chan3d-24-wide", lambda: P.config_problem(2, scale=24), 256),
    ("ragged3d-13x9x7", lambda: _prob_uniform((13, 9, 7)), 64),
]


@pytest.mark.parametrize("name,mk,small", CASES, ids=[c[0] for c in CASES])
def test_solve_fp64_matches_oracle(M, name, mk, small):
    prob = mk()
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=0, small_cells=small))
    b = H.rhs_for(prob)
    x, st = H.solve(b, 1e-8)
    R = O.Hierarchy(prob)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0 and st["status"] == 0, (st, sr)
    assert st["relres_true"] < 1e-8
    xg = x.cpu().numpy()
    err = np.linalg.norm(xg - xr) / max(np.linalg.norm(xr), 1e-300)
    assert err <= SOL_RTOL, err
    assert _maxerr(xg, xr) <= SOL_RTOL, err
    _counts_close(st["iters"], sr["iters"], sr["calls"])
    # bookkeeping invariant of the recursion: calls(k+1) = iterations(k)
    for k in range(len(st["iters"]) - 1):
        assert st["calls"][k + 1] == st["iters"][k]


@pytest.mark.parametrize("name,mk,small", CASES, ids=[c[0] for c in CASES])
def test_solve_fp32_precond_matches_oracle(M, name, mk, small):
    prob = mk()
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=1, small_cells=small, inner_floor=1e-6))
    b = H.rhs_for(prob)
    x, st = H.solve(b, 1e-8)
    R = O.Hierarchy(prob)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert st["status"] == 0, st
    assert st["relres_true"] < 1e-8
    # the outer FP64 PCG needs about the oracle's level-0 iterations (band:
    # a quarter or 2); the inner levels stop at the FP32 floor instead.  On
    # the layered channel fields (1e9 contrast between 4-cell slabs) the
    # FP32-rounded preconditioner is a coarser approximation of the FP64 one
    # (Sec. 2.3: an inexact preconditioner costs outer iterations): band 2x + 2
    n0, r0 = st["iters"][0], sr["iters"][0]
    if name.startswith("chan"):
        assert r0 <= n0 <= 2 * r0 + 2, (st["iters"], sr["iters"])
    else:
        assert abs(n0 - r0) <= max(2, r0 // 4), (st["iters"], sr["iters"])
    err = np.linalg.norm(x.cpu().numpy() - xr) / max(np.linalg.norm(xr), 1e-300)
    assert err <= SOL_RTOL, err
    assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL, err


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_1024_matches_oracle(M, prec):
    prob = P.config_problem(1)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0))
    b = H.rhs_for(prob)
    x, st = H.solve(b, 1e-8)
    R = O.Hierarchy(prob)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert st["status"] == 0 and st["relres_true"] < 1e-8, st
    err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= SOL_RTOL, err
    assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL, err
    if prec == 0:
        _counts_close(st["iters"], sr["iters"], sr["calls"])


# ---------------------------------------------------------------------------
# modified Jacobi splitting (P = 2D, Sec. 3) as the smoother
# ---------------------------------------------------------------------------
JACOBI_CASES = [
    ("cfg0", lambda: P.config_problem(0), 0),
    ("ragged-37x23-wide", lambda: _prob_uniform((37, 23)), 64),
    ("grf-128", lambda: P.config_problem(1, scale=128), 0),
    ("grf-200x72-wide", lambda: P.grf_problem((200, 72), seed=21, ell=6.0, half_span=4.5), 256),
    ("tiny-3x2", lambda: _prob_uniform((3, 2)), 0),
    ("chan3d-16", lambda: P.config_problem(2, scale=16), 0),
    ("ragged3d-13x9x7", lambda: _prob_uniform((13, 9, 7)), 64),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,mk,small", JACOBI_CASES, ids=[c[0] for c in JACOBI_CASES])
def test_solve_jacobi_matches_oracle(M, name, mk, small, prec):
    """Single solves (wide levels as graph kernels, narrow levels in one CTA)
    with the modified Jacobi smoother against the oracle's Jacobi solve."""
    prob = mk()
    opts = M.default_opts(precision=prec, small_cells=small, splitting=1, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_problem(prob, opts)
    x, st = H.solve(H.rhs_for(prob), 1e-8)
    R = O.Hierarchy(prob, splitting=1)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0 and st["status"] == 0, (st, sr)
    assert st["relres_true"] < 1e-8
    err = np.linalg.norm(x.cpu().numpy() - xr) / max(np.linalg.norm(xr), 1e-300)
    assert err <= SOL_RTOL, err
    assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL, err
    if prec == 0:
        _counts_close(st["iters"], sr["iters"], sr["calls"])


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_jacobi_matches_oracle(M, prec):
    """The batched solver (whole recursion in one CTA per problem) with the
    modified Jacobi smoother: the 256^2 GRF problem and ragged 2D / 3D grids."""
    probs = [P.config_problem(1, scale=256), _prob_uniform((37, 23)), _prob_uniform((13, 9, 7))]
    opts = M.default_opts(precision=prec, splitting=1, inner_floor=1e-6 if prec else 0.0)
    for p in probs:
        H = M.Hierarchy.from_problem(p, opts)
        xs, sts = M.batch_solve([H], [H.rhs_for(p)], 1e-8)
        R = O.Hierarchy(p, splitting=1)
        xr, sr = R.solve(R.lift_rhs(), 1e-8)
        assert sts[0]["status"] == 0 and sts[0]["relres_true"] < 1e-8, sts[0]
        err = np.linalg.norm(xs[0].cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL, err
        assert _maxerr(xs[0].cpu().numpy(), xr) <= SOL_RTOL, err
        if prec == 0:
            _counts_close(sts[0]["iters"], sr["iters"], sr["calls"])


LEX_CASES = [
    ("cfg0", lambda: P.config_problem(0)),
    ("ragged-37x23", lambda: _prob_uniform((37, 23))),
    ("grf-128", lambda: P.config_problem(1, scale=128)),
    ("tiny-3x2", lambda: _prob_uniform((3, 2))),
    ("direct-rhs-50x50", lambda: _prob_uniform((50, 50), lifted=False)),
    ("chan3d-16", lambda: P.config_problem(2, scale=16)),
    ("ragged3d-13x9x7", lambda: _prob_uniform((13, 9, 7))),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,mk", LEX_CASES, ids=[c[0] for c in LEX_CASES])
def test_solve_natural_order_sgs_matches_oracle(M, name, mk, prec):
    """Symmetric Gauss-Seidel in the natural order (a plane-by-plane
    wavefront on the GPU) against the oracle's sequential sweeps, single and
    batched solves."""
    prob = mk()
    opts = M.default_opts(precision=prec, splitting=2, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_problem(prob, opts)
    b = H.rhs_for(prob)
    x, st = H.solve(b, 1e-8)
    xs, sts = M.batch_solve([H], [b], 1e-8)
    R = O.Hierarchy(prob, splitting=2)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0 and st["status"] == 0 and sts[0]["status"] == 0, (st, sr)
    for xg, sg in ((x, st), (xs[0], sts[0])):
        assert sg["relres_true"] < 1e-8
        err = np.linalg.norm(xg.cpu().numpy() - xr) / max(np.linalg.norm(xr), 1e-300)
        assert err <= SOL_RTOL, err
        assert _maxerr(xg.cpu().numpy(), xr) <= SOL_RTOL, err
        if prec == 0:
            _counts_close(sg["iters"], sr["iters"], sr["calls"])


def test_splitting_option_validated(M):
    prob = _prob_uniform((8, 8))
    with pytest.raises(M.MsrcgError):
        M.Hierarchy.from_problem(prob, M.default_opts(splitting=3))


# ---------------------------------------------------------------------------
# anisotropic cells: coarsening toward square cells, piecewise constant E
# ---------------------------------------------------------------------------
ANISO_CASES = [
    ("square-linear", 1, 0, 0),
    ("square-linear-wide", 1, 0, 256),
    ("square-piecewise-constant", 1, 1, 0),
    ("square-piecewise-constant-wide", 1, 1, 256),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,coarsening,interp,small", ANISO_CASES, ids=[c[0] for c in ANISO_CASES])
def test_anisotropic_strip_matches_oracle(M, name, coarsening, interp, small, prec):
    """The 200 x 50 strip with 10:1 cells: single (graph) and batched solves
    against the oracle with the same level rule and extension."""
    prob = P.strip_problem((200, 50))
    opts = M.default_opts(precision=prec, coarsening=coarsening, interp=interp, small_cells=small,
                          inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_problem(prob, opts)
    b = H.rhs_for(prob)
    x, st = H.solve(b, 1e-8)
    xs, sts = M.batch_solve([H], [b], 1e-8)
    R = O.Hierarchy(prob, coarsening=coarsening, interp=interp)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0, sr
    for xg, sg in ((x, st), (xs[0], sts[0])):
        assert sg["status"] == 0 and sg["relres_true"] < 1e-8, sg
        err = np.linalg.norm(xg.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL, err
        assert _maxerr(xg.cpu().numpy(), xr) <= SOL_RTOL, err
        if prec == 0:
            _counts_close(sg["iters"], sr["iters"], sr["calls"])


_ORACLE_CACHE = {}


def _oracle_solution(key, prob):
    if key not in _ORACLE_CACHE:
        R = O.Hierarchy(prob)
        _ORACLE_CACHE[key] = R.solve(R.lift_rhs(), 1e-8)
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_3d_grf_matches_oracle(M, prec):
    """128^3 Gaussian random field (1e9 contrast): the 3D workload's size on a
    field where the method converges (the layered channel field of that size
    stalls in the oracle as well)."""
    prob = P.grf3d_problem(128)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0))
    x, st = H.solve(H.rhs_for(prob), 1e-8)
    xr, sr = _oracle_solution("grf3d-128", prob)
    assert st["status"] == 0 and st["relres_true"] < 1e-8, st
    err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= SOL_RTOL, err
    assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL, err
    if prec == 0:
        _counts_close(st["iters"], sr["iters"], sr["calls"])


def test_channel_3d_32_fp64_matches_oracle(M):
    """The layered channel field at 32^3, where the FP64 method still
    converges (about 190 outer iterations in both implementations)."""
    prob = P.config_problem(2, scale=32)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=0))
    x, st = H.solve(H.rhs_for(prob), 1e-8)
    xr, sr = _oracle_solution("chan-32", prob)
    assert st["status"] == 0 and st["relres_true"] < 1e-8, st
    err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= SOL_RTOL, err
    assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL, err
    _counts_close(st["iters"], sr["iters"], sr["calls"])


@pytest.mark.parametrize("extra", [{}, {"plain_sweeps": 1}, {"fuse_width": 40}, {"fuse_min_cells": 262144}])
def test_batched_1024_single_pass_and_plain_sweeps(M, extra):
    """The batched solver on the full 1024^2 problem, whose two finest levels
    live in global memory: with the single-pass smoother (default, and with
    narrow 40-column strips, and on level 0 only) and with one pass per
    half-sweep.  All match the oracle."""
    prob = P.config_problem(1)
    opts = M.default_opts(precision=1, inner_floor=1e-6, **extra)
    H = M.Hierarchy.from_problem(prob, opts)
    xs, sts = M.batch_solve([H], [H.rhs_for(prob)], 1e-8)
    xr, sr = _oracle_solution("grf-1024", prob)
    assert sts[0]["status"] == 0 and sts[0]["relres_true"] < 1e-8, sts[0]
    err = np.linalg.norm(xs[0].cpu().numpy() - xr) / np.linalg.norm(xr)
    assert err <= SOL_RTOL, err
    assert _maxerr(xs[0].cpu().numpy(), xr) <= SOL_RTOL, err


@pytest.mark.parametrize("prec", [1, 0])
def test_bench_batch_full_launch(M, prec):
    """The launch the benchmark times: one problem per SM, each the 1024^2
    field with its own seeded N(0,1) source (the benchmark's seeds and, in the
    FP32 mode, its tuned tile shapes), in one batched launch.  Every solution's
    true residual, formed with the oracle's operator and right-hand side, meets
    1e-8 (to the rounding of that check); the first, middle and last problems
    match the oracle's solutions; a second solve of the whole batch and those
    problems solved alone give the same bits as the first batch (the solver is
    deterministic under any load, and the CTAs do not interact)."""
    from paper_math_9809043_gb300 import tune as TU
    nb = torch.cuda.get_device_properties(0).multi_processor_count
    base = P.config_problem(1)
    probs = [P.Problem(dim=2, n=base.n, h=base.h, K=base.K, bc=base.bc, gD=base.gD,
                       f=np.random.default_rng(1001 * 1000 + j).standard_normal(base.N), pbf=base.pbf)
             for j in range(nb)]
    tuned = (TU.best(torch.cuda.get_device_name(), f"grf1024x{nb}") or {}) if prec else {}
    opts = M.default_opts(precision=prec, **({"inner_floor": 1e-6, **tuned} if prec else {"inner_floor": 0.0}))
    hs = [M.Hierarchy.from_problem(p, opts) for p in probs]
    bs = [h.rhs_for(p) for h, p in zip(hs, probs)]
    xs, sts = M.batch_solve(hs, bs, 1e-8)
    R = O.Hierarchy(base)
    for j, (p, x, st) in enumerate(zip(probs, xs, sts)):
        assert st["status"] == 0 and st["relres_true"] < 1e-8, (j, st)
        b = R.lift_rhs(p)
        rel = np.linalg.norm(b - R.apply(0, x.cpu().numpy())) / np.linalg.norm(b)
        assert rel < 1.05e-8, (j, rel)
    xs2, _ = M.batch_solve(hs, bs, 1e-8)
    assert all(torch.equal(a, b) for a, b in zip(xs, xs2))
    for j in (0, nb // 2, nb - 1):
        Rj = O.Hierarchy(probs[j])
        xr, sr = Rj.solve(Rj.lift_rhs(), 1e-8)
        err = np.linalg.norm(xs[j].cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL, (j, err)
        assert _maxerr(xs[j].cpu().numpy(), xr) <= SOL_RTOL, (j, err)
        if prec == 0:
            _counts_close(sts[j]["iters"], sr["iters"], sr["calls"])
        x1, s1 = M.batch_solve([hs[j]], [bs[j]], 1e-8)
        assert torch.equal(x1[0], xs[j]) and s1[0]["iters"] == sts[j]["iters"], j


def test_repeat_solves_identical(M):
    """Deterministic reductions: two solves give the same bits."""
    prob = P.config_problem(1, scale=256)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=1, inner_floor=1e-6))
    b = H.rhs_for(prob)
    x1, s1 = H.solve(b, 1e-8)
    x2, s2 = H.solve(b, 1e-8)
    assert torch.equal(x1, x2) and s1["iters"] == s2["iters"]


# ---------------------------------------------------------------------------
# degenerate inputs and errors
# ---------------------------------------------------------------------------
def test_zero_rhs(M):
    prob = _prob_uniform((40, 40))
    for small in (0, 64):
        H = M.Hierarchy.from_problem(prob, M.default_opts(small_cells=small))
        x, st = H.solve(torch.zeros(1600, dtype=torch.float64, device="cuda"), 1e-8)
        assert st["status"] == 0 and torch.count_nonzero(x).item() == 0 and st["iters"][0] == 0


def test_nan_rhs_reports_enaninf(M):
    prob = _prob_uniform((40, 40))
    for small in (0, 64):
        H = M.Hierarchy.from_problem(prob, M.default_opts(small_cells=small))
        b = torch.ones(1600, dtype=torch.float64, device="cuda")
        b[7] = float("nan")
        x, st = H.solve(b, 1e-8, check=False)
        assert st["status"] == M.ENANINF


def test_invalid_arguments(M):
    prob = _prob_uniform((8, 8))
    with pytest.raises(M.MsrcgError):
        M.Hierarchy(2, (0, 8), (0.1, 0.1), prob.K, prob.bc)
    with pytest.raises(M.MsrcgError):
        M.Hierarchy(4, (8, 8), (0.1, 0.1), prob.K, prob.bc)
    H = M.Hierarchy.from_problem(prob)
    with pytest.raises(M.MsrcgError):
        H.solve(torch.ones(64, dtype=torch.float64, device="cuda"), tol=-1.0)
    # mis-sized arrays are refused on the host, before any launch
    f64 = dict(dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        H.solve(torch.ones(63, **f64))
    with pytest.raises(ValueError):
        H.solve(torch.ones(64, **f64), x=torch.empty(60, **f64))
    with pytest.raises(ValueError):
        H.solve(torch.ones(64, **f64), x=torch.empty(64, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        M.batch_solve([H], [torch.ones(65, **f64)])
    with pytest.raises(ValueError):
        M.batch_solve([H, H], [torch.ones(64, **f64)])
    with pytest.raises(ValueError):
        H.apply(0, torch.ones(5, **f64))
    with pytest.raises(ValueError):
        H.lift_rhs(prob.bc[:-1], prob.gD, prob.f, prob.pbf)
    with pytest.raises(ValueError):
        M.Hierarchy(2, (8, 8), (0.1, 0.1), prob.K.reshape(-1)[:60], prob.bc)
    with pytest.raises(ValueError):
        M.Hierarchy(2, (8, 8), (0.1, 0.1), prob.K, prob.bc[:10])


# ---------------------------------------------------------------------------
# batched solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle(M, prec):
    probs = [_prob_uniform((n, n), seed=100 + i, lifted=False) for i, n in enumerate([24, 40, 17, 64, 33, 9, 48, 30])]
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    hs = [M.Hierarchy.from_problem(p, opts) for p in probs]
    bs = [h.rhs_for(p) for h, p in zip(hs, probs)]
    xs, sts = M.batch_solve(hs, bs, 1e-8)
    for p, x, st in zip(probs, xs, sts):
        R = O.Hierarchy(p)
        xr, sr = R.solve(R.lift_rhs(), 1e-8)
        assert st["status"] == 0 and st["relres_true"] < 1e-8
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL
        assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL
        if prec == 0:
            _counts_close(st["iters"], sr["iters"], sr["calls"])



def test_uneven_batch_full_size(M):
    """The 256-problem uneven batch (sides 64..512) in one launch, FP32
    preconditioner: every result's true residual, formed with the oracle's
    operator, meets 1e-8 (to the rounding of that check); one problem per side
    class matches the oracle's solution."""
    probs = P.batch_problems(256)
    opts = M.default_opts(precision=1, inner_floor=1e-6)
    hs = [M.Hierarchy.from_problem(p, opts) for p in probs]
    bs = [h.rhs_for(p) for h, p in zip(hs, probs)]
    xs, sts = M.batch_solve(hs, bs, 1e-8)
    for p, x, st in zip(probs, xs, sts):
        assert st["status"] == 0, (p.name, st)
        R = O.Hierarchy(p)
        xv = x.cpu().numpy()
        rel = np.linalg.norm(p.b - R.apply(0, xv)) / np.linalg.norm(p.b)
        assert rel < 1.05e-8, (p.name, rel)
    first = {}
    for j, p in enumerate(probs):
        first.setdefault(p.n[0], j)
    for side, j in sorted(first.items()):
        R = O.Hierarchy(probs[j])
        xr, _ = R.solve(R.lift_rhs(), 1e-8)
        err = np.linalg.norm(xs[j].cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL, (side, err)
        assert _maxerr(xs[j].cpu().numpy(), xr) <= SOL_RTOL, (side, err)


@pytest.mark.parametrize("n", [(4100, 3), (8, 4096)], ids=["long-4100x3", "tall-8x4096"])
def test_single_pass_smoothing_on_thin_levels(M, n):
    """Single-pass smoothing on levels with fewer rows than the pipeline is
    deep (4100 x 3) and with a single strip narrower than its halo
    (8 x 4096), batched path, against the oracle and the plain sweeps."""
    prob = _prob_uniform(n, seed=41)
    R = O.Hierarchy(prob)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0
    for plain in (0, 1):
        opts = M.default_opts(precision=1, inner_floor=1e-6, plain_sweeps=plain)
        H = M.Hierarchy.from_problem(prob, opts)
        xs, sts = M.batch_solve([H], [H.rhs_for(prob)], 1e-8)
        assert sts[0]["status"] == 0 and sts[0]["relres_true"] < 1e-8, sts[0]
        err = np.linalg.norm(xs[0].cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL, (plain, err)
        assert _maxerr(xs[0].cpu().numpy(), xr) <= SOL_RTOL, (plain, err)


def test_tuner_picks_a_candidate(M):
    """The autotuner times every candidate tile shape on a small batch, all of
    them solve, and it keeps the fastest; its second stage times every other
    inner floor on that shape and keeps one only where it is faster (a floor
    that does not qualify is recorded as None)."""
    from paper_math_9809043_gb300 import tune as TU
    probs = [P.config_problem(1, scale=256) for _ in range(2)]
    cands = [{}, {"plain_sweeps": 1}, {"fuse_width": 64}]
    fastest, times = TU.tune(probs, steps=1, candidates=cands)
    shape = {k: v for k, v in fastest.items() if k != "inner_floor"}
    shape_keys = {TU.key_of(c) for c in cands}
    assert shape in cands and shape_keys <= set(times)
    assert times[TU.key_of(shape)] == min(times[k] for k in shape_keys)
    assert set(times) - shape_keys == {TU.key_of({**shape, "inner_floor": f}) for f in TU.FLOORS[1:]}
    if "inner_floor" in fastest:
        assert fastest["inner_floor"] in TU.FLOORS[1:]
        assert times[TU.key_of(fastest)] is not None and times[TU.key_of(fastest)] < times[TU.key_of(shape)]


@pytest.mark.parametrize("prec", [1, 0])
def test_smoothing_degree_one(M, prec):
    """m = 1 (three half-sweeps per smoothing) on a 256^2 field whose finest
    level the batched solver keeps in global memory: the single-pass
    smoother needs 4m >= its prefetch distance, so this runs the
    per-half-sweep passes; batched and single solves match the oracle run
    with the same m."""
    prob = P.config_problem(1, scale=256)
    opts = M.default_opts(m=1, precision=prec, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_problem(prob, opts)
    b = H.rhs_for(prob)
    R = O.Hierarchy(prob, m=1)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0
    xs, sts = M.batch_solve([H], [b], 1e-8)
    x1, s1 = H.solve(b, 1e-8)
    for x, st in ((xs[0], sts[0]), (x1, s1)):
        assert st["status"] == 0 and st["relres_true"] < 1e-8, st
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= SOL_RTOL, err
        assert _maxerr(x.cpu().numpy(), xr) <= SOL_RTOL, err
        if prec == 0:
            _counts_close(st["iters"], sr["iters"], sr["calls"])


# ---------------------------------------------------------------------------
# hierarchy from face permeabilities (msrcg_build_faces, Sec. 3)
# ---------------------------------------------------------------------------
def _random_faces(n, seed):
    """Face K that no cell field produces: the harmonic means of a Gaussian
    random field (correlation 6 cells, 1e6 contrast) each times its own
    factor in [0.5, 2]; Dirichlet x-faces with their own K (a few x-high
    faces Neumann), Neumann (0) on the other sides."""
    from faces import face_K_from_cells
    rng = np.random.default_rng(seed)
    dim = len(n)
    n3 = list(n) + [1] * (3 - dim)
    base = P.grf_problem(tuple(n), seed=seed, ell=6.0, half_span=3.0, source=False)
    Kf = [k * 2.0 ** rng.uniform(-1, 1, k.size) for k in face_K_from_cells(base)]
    Kx = Kf[0].reshape(n3[2], n3[1], n3[0] + 1)
    Kx[:, :, -1] *= rng.random((n3[2], n3[1])) < 0.7
    N = int(np.prod(n))
    bc, gD = P.standard_bc(dim, n)
    prob = P.Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=np.ones((1, N)), bc=bc, gD=gD,
                     b=rng.standard_normal(N))
    return prob, Kf


@pytest.mark.parametrize("n", [(37, 23), (300, 200), (12, 10, 9), (40, 24, 20)])
@pytest.mark.parametrize("prec", [0, 1])
def test_face_K_build_matches_oracle(M, n, prec):
    """Face values no cell field produces: transmissibilities of every level
    bit-exact against the oracle's face-K build, and the solve within the
    parity tolerance, norm-wise and element-wise."""
    prob, Kf = _random_faces(n, 81)
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_faces(prob.dim, prob.n, prob.h, Kf, opts)
    R = O.Hierarchy(prob, Kfaces=Kf)
    assert H.nlev == R.nlev
    for k in range(R.nlev):
        for tg, tr in zip(H.trans(k), R.T(k)):
            if tr is not None:
                assert np.array_equal(tg.cpu().numpy(), tr), k
    x, st = H.solve(torch.as_tensor(prob.b, device="cuda"), 1e-8)
    xr, sr = R.solve(prob.b, 1e-8)
    assert st["status"] == 0 and sr["status"] == 0 and st["relres_true"] < 1e-8, (st, sr)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= SOL_RTOL
    assert np.max(np.abs(xg - xr)) / np.max(np.abs(xr)) <= SOL_RTOL
    if prec == 0:
        _counts_close(st["iters"], sr["iters"], sr["calls"])


@pytest.mark.parametrize("n", [(64, 48), (13, 9, 7)])
def test_face_K_from_harmonic_means_equals_cell_K_build(M, n):
    """Faces holding the harmonic means of a cell field (2 K_cell on Dirichlet
    faces, 0 on Neumann ones) give the cell-K build's hierarchy to the bit."""
    from faces import face_K_from_cells
    prob = _prob_uniform(n, span=2.0)
    Kf = face_K_from_cells(prob)
    A = M.Hierarchy.from_problem(prob)
    B = M.Hierarchy.from_faces(prob.dim, prob.n, prob.h, Kf)
    for k in range(A.nlev):
        for ta, tb in zip(A.trans(k), B.trans(k)):
            if ta is not None:
                assert torch.equal(ta, tb), k
    b = A.rhs_for(prob)
    xa, _ = A.solve(b, 1e-8)
    xb, _ = B.solve(b, 1e-8)
    assert torch.equal(xa, xb)


# ---------------------------------------------------------------------------
# stall path of the FP32 preconditioner: flexible beta, then the FP64
# preconditioner (the inexact inner solves of Sec. 2.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", ["single", "batched"])
def test_fp32_channel_32_converges_through_the_stall_path(M, path):
    """The layered channel field at 32^3 stalls near 1e-6 with the FP32
    preconditioner and the plain beta; the stall test switches the outer PCG
    to the flexible beta and, if it stalls again, the solve is repeated with
    the FP64 preconditioner.  The result meets 1e-8 and the FP64 oracle's
    solution within the parity tolerance, and the stats say which path it
    took."""
    prob = P.config_problem(2, scale=32)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=1, inner_floor=1e-6))
    b = H.rhs_for(prob)
    if path == "single":
        x, st = H.solve(b, 1e-8)
    else:
        xs, sts = M.batch_solve([H], [b], 1e-8)
        x, st = xs[0], sts[0]
    xr, sr = _oracle_solution("chan-32", prob)
    assert st["status"] == 0 and st["relres_true"] < 1e-8, st
    assert st["flexible"] == 1 or st["escalated"] == 1, st
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= SOL_RTOL
    assert np.max(np.abs(xg - xr)) / np.max(np.abs(xr)) <= SOL_RTOL
    print(path, st["iters"], "flexible", st["flexible"], "escalated", st["escalated"])


@pytest.mark.parametrize("small", [0, 256])
@pytest.mark.parametrize("prec", [0, 1])
def test_flexible_beta_from_the_start_matches_oracle(M, small, prec):
    """With the flexible beta forced from the first iteration (single solve
    on graph + one-CTA levels, and batched), the result still meets 1e-8 and
    the oracle's solution: for a preconditioner that is linear up to the
    inner tolerances, r_new . z_old is near zero and the two betas agree."""
    prob = P.grf_problem((200, 72), seed=21, ell=6.0, half_span=4.5)
    opts = M.default_opts(precision=prec, small_cells=small, flexible=1, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_problem(prob, opts)
    b = H.rhs_for(prob)
    R = O.Hierarchy(prob)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    x, st = H.solve(b, 1e-8)
    xs, sts = M.batch_solve([H], [b], 1e-8)
    for xx, ss in ((x, st), (xs[0], sts[0])):
        assert ss["status"] == 0 and ss["relres_true"] < 1e-8 and ss["flexible"] == 1, ss
        xg = xx.cpu().numpy()
        assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= SOL_RTOL
        assert np.max(np.abs(xg - xr)) / np.max(np.abs(xr)) <= SOL_RTOL


def test_escalation_off_reports_enoconv(M):
    """With escalation off and the stall test on, a stalling FP32 solve ends
    with MSRCG_ENOCONV (and is reusable afterwards)."""
    prob = P.config_problem(2, scale=32)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=1, inner_floor=1e-6, escalate=0, maxit_outer=60))
    x, st = H.solve(H.rhs_for(prob), 1e-8, check=False)
    assert st["status"] in (M.OK, M.ENOCONV) and st["escalated"] == 0, st
    if st["status"] == M.ENOCONV:
        x2, st2 = H.solve(H.rhs_for(prob), 1e-8, check=False)
        assert st2["iters"] == st["iters"]


# ---------------------------------------------------------------------------
# the multigrid (eq. 2.9, Tatebe) and polynomial (eq. 2.6, W = P^-1)
# preconditioners on the same smoother and transfers
# ---------------------------------------------------------------------------
PRECOND_CASES = [
    ("cfg0", lambda: P.config_problem(0)),
    ("ragged-37x23", lambda: _prob_uniform((37, 23))),
    ("grf-128", lambda: P.config_problem(1, scale=128)),
    ("grf-200x72", lambda: P.grf_problem((200, 72), seed=21, ell=6.0, half_span=4.5)),
    ("ragged3d-13x9x7", lambda: _prob_uniform((13, 9, 7))),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("precond", [1, 2])
@pytest.mark.parametrize("name,mk", PRECOND_CASES, ids=[c[0] for c in PRECOND_CASES])
def test_other_preconditioners_match_oracle(M, name, mk, precond, prec):
    prob = mk()
    opts = M.default_opts(precision=prec, precond=precond, maxit_outer=2000, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.from_problem(prob, opts)
    b = H.rhs_for(prob)
    R = O.Hierarchy(prob, precond=precond, maxit_outer=2000)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert sr["status"] == 0
    x, st = H.solve(b, 1e-8)
    xs, sts = M.batch_solve([H], [b], 1e-8)
    for xx, ss in ((x, st), (xs[0], sts[0])):
        assert ss["status"] == 0 and ss["relres_true"] < 1e-8, ss
        xg = xx.cpu().numpy()
        assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= SOL_RTOL
        assert np.max(np.abs(xg - xr)) / np.max(np.abs(xr)) <= SOL_RTOL
        if prec == 0 and sr["iters"][0] <= 100:
            # (hundreds of CG iterations amplify the different summation
            # orders too much for a count comparison: the polynomial
            # preconditioner at 200 x 72 takes ~330)
            _counts_close(ss["iters"], sr["iters"], sr["calls"])


def test_profile_level_entry(M):
    """The standalone timing entry reports every multi-CTA kernel of a wide
    level with a positive duration and its algorithmic bytes, rejects a
    single-CTA level, and leaves the hierarchy solving correctly."""
    prob = P.config_problem(1, scale=256)
    H = M.Hierarchy.from_problem(prob, M.default_opts(precision=1, inner_floor=1e-6))
    rows = H.profile_level(0, reps=3)
    assert len(rows) == M.lib().msrcg_profile_kernel_count() == 10
    assert all(r["ms"] > 0 and r["bytes"] > 0 and r["kernel"] for r in rows)
    with pytest.raises(M.MsrcgError):
        H.profile_level(H.nlev - 1)
    x, st = H.solve(H.rhs_for(prob), 1e-8)
    R = O.Hierarchy(prob)
    xr, sr = R.solve(R.lift_rhs(), 1e-8)
    assert st["status"] == 0 and np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr) <= SOL_RTOL


# ---------------------------------------------------------------------------
# constant coefficients (msrcg_build_laplace, the Laplace specialisation of
# Sec. 4.1): compact face arrays, same operator as the cell-K build of a
# constant field
# ---------------------------------------------------------------------------
def _const_problem(n, K, seed=91):
    rng = np.random.default_rng(seed)
    dim = len(n)
    N = int(np.prod(n))
    Kc = np.repeat(np.asarray(K, np.float64).reshape(-1, 1), N, axis=1)
    bc, gD = P.standard_bc(dim, n)
    return P.Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=Kc, bc=bc, gD=gD,
                     f=rng.standard_normal(N), pbf=P.linear_lifting(dim, n))


LAP_CASES = [((64, 48), (1.0, 1.0)), ((37, 23), (3.0, 0.25)), ((1024, 1024), (1.0, 1.0)), ((12, 10, 9), (1.0, 2.0, 0.5)),
             ((64, 64, 64), (1.0, 1.0, 1.0))]


@pytest.mark.parametrize("n,K", LAP_CASES, ids=["x".join(map(str, c[0])) for c in LAP_CASES])
def test_laplace_transmissibilities_match_oracle(M, n, K):
    """The compact constant-coefficient levels expand to the oracle's
    transmissibilities of the same constant field: level 0 to the bit, the
    coarse levels (the oracle's series-parallel sums of equal conductors) to
    rounding."""
    prob = _const_problem(n, K)
    H = M.Hierarchy.laplace(prob.dim, prob.n, prob.h, K, [1, 1, 0, 0, 0, 0])
    R = O.Hierarchy(prob)
    assert H.nlev == R.nlev
    for k in range(R.nlev):
        for tg, tr in zip(H.trans(k), R.T(k)):
            if tr is None:
                continue
            tg = tg.cpu().numpy()
            if k == 0:
                assert np.array_equal(tg, tr)
            else:
                assert np.max(np.abs(tg - tr)) <= 1e-13 * np.max(np.abs(tr)), k


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,K", LAP_CASES, ids=["x".join(map(str, c[0])) for c in LAP_CASES])
def test_laplace_solve_matches_oracle(M, n, K, prec):
    """Single and batched solves of the constant-coefficient hierarchy (lifted
    right-hand side with a source) against the oracle's solve of the same
    constant field, norm-wise and element-wise."""
    prob = _const_problem(n, K)
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    H = M.Hierarchy.laplace(prob.dim, prob.n, prob.h, K, [1, 1, 0, 0, 0, 0], opts)
    b = H.rhs_for(prob)
    R = O.Hierarchy(prob)
    br = R.lift_rhs()
    assert np.max(np.abs(b.cpu().numpy() - br)) <= 1e-12 * np.max(np.abs(br))
    xr, sr = R.solve(br, 1e-8)
    assert sr["status"] == 0
    x, st = H.solve(b, 1e-8)
    xs, sts = M.batch_solve([H], [b], 1e-8)
    for xx, ss in ((x, st), (xs[0], sts[0])):
        assert ss["status"] == 0 and ss["relres_true"] < 1e-8, ss
        xg = xx.cpu().numpy()
        assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= SOL_RTOL
        assert np.max(np.abs(xg - xr)) / np.max(np.abs(xr)) <= SOL_RTOL
        if prec == 0:
            _counts_close(ss["iters"], sr["iters"], sr["calls"])


def test_laplace_uses_less_memory(M):
    """No full face array is kept: the constant-coefficient hierarchy of a
    1024^2 problem is smaller than the cell-K one by about the face arrays
    (two FP64 words per cell, and two FP32 ones with the FP32 preconditioner)."""
    prob = _const_problem((1024, 1024), (1.0, 1.0))
    for prec in (0, 1):
        opts = M.default_opts(precision=prec)
        A = M.Hierarchy.from_problem(prob, opts)
        B = M.Hierarchy.laplace(2, prob.n, prob.h, 1.0, [1, 1, 0, 0, 0, 0], opts)
        saved = A.device_bytes() - B.device_bytes()
        assert saved >= (16 + (8 if prec else 0)) * prob.N, (A.device_bytes(), B.device_bytes())


# ---------------------------------------------------------------------------
# level tree (Fig. 2; msrcg_set_trace)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_level_tree_trace(M, prec):
    """The level tree of a solve through the C ABI: its structure as eq. 2.10
    fixes it (tests/trees.py), against the solve's own counters; in FP64 the
    oracle's tree of the same problem (per-call iterations equal where the
    per-level totals are, else totals within the 3% band); the same tree from
    msrcg_solve (routed to the single-CTA solver while tracing) and from the
    batched path; a capacity below the number of calls keeps the first
    entries and counts them all; detaching stops the recording."""
    from trees import check_tree
    prob = P.grf_problem((200, 72), seed=21, ell=6.0, half_span=4.5)
    opts = M.default_opts(precision=prec, small_cells=256, **({"inner_floor": 1e-6} if prec else {}))
    H = M.Hierarchy.from_problem(prob, opts)
    assert H.nlev >= 3
    b = H.rhs_for(prob)
    H.set_trace(1 << 16)
    x, st = H.solve(b, 1e-8)
    assert st["status"] == 0 and st["relres_true"] < 1e-8
    count, tr = H.trace()
    assert count == len(tr) == sum(st["calls"])
    check_tree(tr, st["iters"], st["calls"], H.nlev)
    xs, sts = M.batch_solve([H], [b], 1e-8)
    count2, tr2 = H.trace()
    check_tree(tr2, sts[0]["iters"], sts[0]["calls"], H.nlev)
    if prec == 0:
        assert tr2 == tr  # same launch shape, same arithmetic
        R = O.Hierarchy(prob)
        xr, sr = R.solve(R.lift_rhs(), 1e-8, trace_cap=1 << 16)
        assert sr["trace_count"] == len(sr["trace"])
        if sr["iters"] == st["iters"]:
            assert [e[:3] for e in tr] == [e[:3] for e in sr["trace"]]
        else:
            _counts_close(st["iters"], sr["iters"], sr["calls"])
        assert [e[2] for e in tr if e[0] == 0] == [e[2] for e in sr["trace"] if e[0] == 0]
    H.set_trace(3)
    H.solve(b, 1e-8)
    count3, tr3 = H.trace()
    assert count3 == count and len(tr3) == 3 and tr3 == tr[:3]
    H.set_trace(0)
    x4, st4 = H.solve(b, 1e-8)
    assert st4["status"] == 0 and H.trace() == (0, [])


@pytest.mark.parametrize("precond", [1, 2])
def test_level_tree_without_inner_pcg(M, precond):
    """Multigrid and polynomial preconditioning record the level-0 calls
    alone (their inner levels run no PCG), as the oracle does."""
    prob = P.grf_problem((200, 72), seed=21, ell=6.0, half_span=4.5)
    opts = M.default_opts(precision=0, precond=precond, maxit_outer=2000)
    H = M.Hierarchy.from_problem(prob, opts)
    H.set_trace(64)
    x, st = H.solve(H.rhs_for(prob), 1e-8)
    assert st["status"] == 0
    count, tr = H.trace()
    assert count == len(tr) == st["calls"][0] and all(e[0] == 0 for e in tr)
    assert sum(e[2] for e in tr) == st["iters"][0]
    R = O.Hierarchy(prob, precond=precond, maxit_outer=2000)
    xr, sr = R.solve(R.lift_rhs(), 1e-8, trace_cap=64)
    assert len(sr["trace"]) == len(tr)
    _counts_close([e[2] for e in tr], [e[2] for e in sr["trace"]], None)
