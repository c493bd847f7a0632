"""The solve that allocates nothing (msrcg_solve_static) against the
allocating entry points, through the C ABI (marked gpu).

Some callers cannot call cudaMalloc (their device memory belongs to another
allocator, or allocation is not allowed where they run); for them the library
solves small problems inside a fixed scratch array.  This file is collected
last so that a run stopping at its first failure has already run every other
test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_math_9809043_gb300 import problems as P  # noqa: E402

SOL_RTOL = 1e-6  # the tolerance of the other parity tests


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_math_9809043_gb300 import build as B
    B.build()
    from paper_math_9809043_gb300 import msrcg
    return msrcg


def _problem(n, seed):
    rng = np.random.default_rng(seed)
    dim = len(n)
    N = int(np.prod(n))
    K = (10.0 ** rng.uniform(-2, 2, N)).reshape(1, -1)
    bc, gD = P.standard_bc(dim, n)
    return P.Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=K, bc=bc, gD=gD,
                     b=rng.standard_normal(N))


@pytest.mark.parametrize("n,prec", [((48, 40), 0), ((100, 90), 1), ((12, 10, 9), 0), ((20, 16, 18), 1)])
def test_static_matches_allocating_solve_twice(M, n, prec):
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    for call, seed in enumerate((11, 12)):  # two calls in a row share the scratch
        prob = _problem(n, seed)
        H = M.Hierarchy.from_problem(prob, opts)
        b = torch.as_tensor(prob.b, device="cuda")
        xa, sa = H.solve(b, 1e-8)
        xs, ss = M.solve_static(prob.dim, prob.n, prob.h, prob.K, prob.bc, b, 1e-8, opts=opts)
        torch.cuda.synchronize()
        assert ss["status"] == 0 and ss["relres_true"] < 1e-8, (call, ss)
        err = (torch.linalg.norm(xs - xa) / torch.linalg.norm(xa)).item()
        assert err <= SOL_RTOL, (call, err)
        assert ss["levels"] == sa["levels"]
        H.close()


@pytest.mark.parametrize("extra", [{"splitting": 1}, {"splitting": 2}, {"coarsening": 1, "interp": 1}],
                         ids=["jacobi", "natural-order", "square-cells-piecewise-constant"])
def test_static_matches_allocating_solve_with_options(M, extra):
    """The other smoothers, the square-cell level rule and the piecewise
    constant extension (built on the device in the static path) give the
    allocating solve's result; 10:1 cells for the level rule."""
    n = (90, 24)
    prob = _problem(n, 21)
    if "coarsening" in extra:
        prob = P.Problem(dim=2, n=n, h=(10.0 / n[0], 0.25 / n[1]), K=prob.K, bc=prob.bc, gD=prob.gD, b=prob.b)
    opts = M.default_opts(precision=1, inner_floor=1e-6, **extra)
    H = M.Hierarchy.from_problem(prob, opts)
    b = torch.as_tensor(prob.b, device="cuda")
    xa, sa = H.solve(b, 1e-8)
    xs, ss = M.solve_static(prob.dim, prob.n, prob.h, prob.K, prob.bc, b, 1e-8, opts=opts)
    torch.cuda.synchronize()
    assert ss["status"] == 0 and ss["relres_true"] < 1e-8, ss
    assert ss["levels"] == sa["levels"] and ss["dims"] == sa["dims"]
    err = (torch.linalg.norm(xs - xa) / torch.linalg.norm(xa)).item()
    assert err <= SOL_RTOL, err
    H.close()


@pytest.mark.parametrize("dim,prec,side", [(2, 0, 230), (2, 1, 227), (3, 0, 35), (3, 1, 34)])
def test_static_capacity(M, dim, prec, side):
    """The largest square / cubic grids the fixed scratch holds (the limits
    the header states): `side` solves and matches the allocating solve, one
    cell more per axis is rejected with MSRCG_EINVAL before anything is
    enqueued (the stream is idle right after the call)."""
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    prob = _problem((side,) * dim, 41)
    H = M.Hierarchy.from_problem(prob, opts)
    b = torch.as_tensor(prob.b, device="cuda")
    xa, sa = H.solve(b, 1e-8)
    xs, ss = M.solve_static(prob.dim, prob.n, prob.h, prob.K, prob.bc, b, 1e-8, opts=opts)
    torch.cuda.synchronize()
    assert ss["status"] == 0 and ss["relres_true"] < 1e-8, ss
    err = (torch.linalg.norm(xs - xa) / torch.linalg.norm(xa)).item()
    assert err <= SOL_RTOL, err
    H.close()
    big = _problem((side + 1,) * dim, 42)
    bb = torch.as_tensor(big.b, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with pytest.raises(M.MsrcgError) as ei:
        M.solve_static(big.dim, big.n, big.h, big.K, big.bc, bb, 1e-8, opts=opts, stream=s)
    assert ei.value.code == M.EINVAL
    assert s.query()  # nothing was left running on the stream


def test_static_calls_of_different_shapes_in_a_row(M):
    """Calls share the scratch and each lays it out for its own problem: a
    large 2D FP32 call, a small 3D FP64 call in the space the first one used,
    then the large one again; each matches the allocating solve."""
    seq = [((100, 90), 1, 51), ((12, 10, 9), 0, 52), ((100, 90), 1, 53)]
    for call, (n, prec, seed) in enumerate(seq):
        opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
        prob = _problem(n, seed)
        H = M.Hierarchy.from_problem(prob, opts)
        b = torch.as_tensor(prob.b, device="cuda")
        xa, sa = H.solve(b, 1e-8)
        xs, ss = M.solve_static(prob.dim, prob.n, prob.h, prob.K, prob.bc, b, 1e-8, opts=opts)
        torch.cuda.synchronize()
        assert ss["status"] == 0 and ss["relres_true"] < 1e-8, (call, ss)
        err = (torch.linalg.norm(xs - xa) / torch.linalg.norm(xa)).item()
        assert err <= SOL_RTOL, (call, err)
        H.close()


def test_static_rejects_oversize(M):
    prob = _problem((400, 400), 3)
    b = torch.as_tensor(prob.b, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with pytest.raises(M.MsrcgError) as ei:
        M.solve_static(prob.dim, prob.n, prob.h, prob.K, prob.bc, b, 1e-8, stream=s)
    assert ei.value.code == M.EINVAL
    assert s.query()
