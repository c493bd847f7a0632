"""Serving (continuous batching) through the C ABI (marked gpu): every result
is the same alone and in the mix, within the parity tolerance, and admission
keeps the device memory charged to requests under the budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_math_9809043_gb300 import problems as P  # noqa: E402

SOL_RTOL = 1e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_math_9809043_gb300 import build as B
    B.build()
    from paper_math_9809043_gb300 import msrcg, serve
    return msrcg, serve


def _mix(seed=0):
    rng = np.random.default_rng(seed)
    probs = []
    for j, side in enumerate([24, 200, 64, 33, 128, 96, 17, 150, 48, 80]):
        logk = P.rescale(P.gaussian_random_field((side, side), 6.0, rng), -3, 3)
        bc, gD = P.standard_bc(2, (side, side))
        probs.append(P.Problem(dim=2, n=(side, side), h=(1 / side,) * 2, K=(10 ** logk).reshape(1, -1), bc=bc, gD=gD,
                               b=rng.standard_normal(side * side)))
    return probs


@pytest.mark.parametrize("prec", [0, 1])
def test_results_same_alone_and_in_the_mix(S, prec):
    M, serve = S
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    probs = _mix()
    sv = serve.Server(8 << 30, max_waves=4, opts=opts)
    reqs = []
    # first group, progress, then the second group while the first may run
    for p in probs[:5]:
        reqs.append(sv.submit(p, p.b))
    sv.progress()
    for p in probs[5:]:
        reqs.append(sv.submit(p, p.b))
    sv.drain()
    for (rid, x), p in zip(reqs, probs):
        done, st = sv.poll(rid)
        assert done and st["status"] == 0 and st["relres_true"] < 1e-8
        H = M.Hierarchy.from_problem(p, opts)
        xa, sa = H.solve(torch.as_tensor(p.b, device="cuda"), 1e-8)
        xa = xa.cpu().numpy()
        assert np.linalg.norm(x - xa) / np.linalg.norm(xa) <= SOL_RTOL
        H.close()
    assert sv.bytes_in_use() == 0
    sv.close()


def test_admission_respects_budget(S):
    M, serve = S
    opts = M.default_opts(precision=1, inner_floor=1e-6)
    probs = _mix(1)
    budget = 8 << 20  # room for one or two requests at a time
    sv = serve.Server(budget, max_waves=4, opts=opts)
    reqs = [sv.submit(p, p.b) for p in probs]
    peak = 0
    while sv.progress() > 0:
        peak = max(peak, sv.bytes_in_use())
        assert sv.bytes_in_use() <= budget
    sv.drain()
    for rid, x in reqs:
        done, st = sv.poll(rid)
        assert done and st["status"] == 0
    assert 0 < peak <= budget
    sv.close()


def test_oversize_request_rejected(S):
    M, serve = S
    sv = serve.Server(1 << 20, max_waves=2)
    p = _mix()[1]
    with pytest.raises(M.MsrcgError) as ei:
        sv.submit(p, p.b)
    assert ei.value.code == M.ENOMEM
    sv.close()


def _thin(seed, n):
    rng = np.random.default_rng(seed)
    N = n[0] * n[1]
    K = (10.0 ** rng.uniform(-2, 2, N)).reshape(1, -1)
    bc, gD = P.standard_bc(2, n)
    return P.Problem(dim=2, n=n, h=(1.0 / n[0], 1.0 / n[1]), K=K, bc=bc, gD=gD, b=rng.standard_normal(N))


@pytest.mark.parametrize("prec", [0, 1])
def test_admission_charges_the_built_size(S, prec):
    """A request is charged exactly the device memory its hierarchy, right-
    hand side and solution take, also on thin grids whose levels shrink along
    one axis only (coarse levels add a third, not a fifteenth); with a budget
    for two such requests the charge never exceeds it and returns to zero."""
    M, serve = S
    opts = M.default_opts(precision=prec, inner_floor=1e-6 if prec else 0.0)
    probs = [_thin(60 + j, (3000 + 100 * j, 6)) for j in range(4)]
    sizes = []
    for p in probs:
        H = M.Hierarchy.from_problem(p, opts)
        sizes.append(H.device_bytes() + 16 * p.N)
        H.close()
    sv = serve.Server(1 << 30, max_waves=2, opts=opts)
    rid, _ = sv.submit(probs[0], probs[0].b)
    assert sv.bytes_in_use() == sizes[0]
    sv.drain()
    assert sv.poll(rid)[0] and sv.bytes_in_use() == 0
    sv.close()
    budget = sizes[-1] + sizes[-2]
    sv = serve.Server(budget, max_waves=2, opts=opts)
    reqs = [sv.submit(p, p.b) for p in probs]
    assert sv.bytes_in_use() <= budget
    while sv.progress() > 0:
        assert sv.bytes_in_use() <= budget
    sv.drain()
    for (rid, x), p in zip(reqs, probs):
        done, st = sv.poll(rid)
        assert done and st["status"] == 0 and st["relres_true"] < 1e-8
    assert sv.bytes_in_use() == 0
    sv.close()
