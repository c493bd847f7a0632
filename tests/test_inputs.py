"""The seeded synthetic inputs follow their stated recipes (CPU): the
Gaussian random field's covariance, the contrast spans, the uneven batch's
sides and size, the serving stream's arrival process, the channel and strip
geometries, and reproducibility from the seeds."""
import numpy as np
import pytest

from paper_math_9809043_gb300 import problems as P


def test_grf_covariance_is_gaussian_with_length_ell():
    # filter exp(-ell^2 |k|^2 / 8) on white noise: covariance exp(-r^2 / ell^2)
    ell = 8.0
    acc = np.zeros(4)
    for seed in range(6):
        g = P.gaussian_random_field((256, 256), ell, np.random.default_rng(seed))
        g = g - g.mean()
        c0 = np.mean(g * g)
        for i, r in enumerate((4, 8, 12, 16)):
            acc[i] += 0.5 * (np.mean(g * np.roll(g, r, axis=0)) + np.mean(g * np.roll(g, r, axis=1))) / c0
    acc /= 6
    expect = np.exp(-np.array([4, 8, 12, 16]) ** 2 / ell ** 2)
    assert np.allclose(acc, expect, atol=0.06), (acc, expect)


def test_contrast_spans():
    p0 = P.config_problem(0)
    l0 = np.log10(p0.K)
    assert p0.n == (32, 32) and l0.min() >= -1.5 and l0.max() <= 1.5 and p0.f is None
    p1 = P.config_problem(1)
    l1 = np.log10(p1.K)
    assert p1.n == (1024, 1024)
    assert l1.min() == pytest.approx(-4.5, abs=1e-12) and l1.max() == pytest.approx(4.5, abs=1e-12)
    assert p1.f.shape == (1024 * 1024,) and abs(p1.f.mean()) < 0.01 and abs(p1.f.std() - 1) < 0.01
    g3 = P.grf3d_problem(32)
    l3 = np.log10(g3.K)
    assert g3.n == (32, 32, 32) and l3.min() == pytest.approx(-4.5) and l3.max() == pytest.approx(4.5)
    st = P.strip_problem((200, 50))
    ls = np.log10(st.K)
    assert ls.min() == pytest.approx(-3.3) and ls.max() == pytest.approx(3.3)
    assert st.h[0] == pytest.approx(10 * st.h[1]) and st.n[1] * st.h[1] == pytest.approx(0.25)


def test_uneven_batch():
    probs = P.batch_problems(256)
    sides = [p.n[0] for p in probs]
    assert set(sides) <= set(P.BATCH_SIDES) and len(set(sides)) == len(P.BATCH_SIDES)
    assert sum(p.N for p in probs) == 21014528
    for p in probs[:8]:
        lk = np.log10(p.K)
        assert p.n[0] == p.n[1] and lk.min() == pytest.approx(-3) and lk.max() == pytest.approx(3)
        assert p.b is not None and p.b.shape == (p.N,)


def test_serving_stream():
    s = P.serving_stream(2000)
    t = np.array([a for a, _ in s])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # 2000 exponential gaps: the mean is 5 ms to within 5 % (its standard error is 2.2 %)
    assert abs(gaps.mean() * 200 - 1) < 0.05
    assert abs(np.std(gaps) / gaps.mean() - 1) < 0.1  # exponential: standard deviation = mean
    d2 = [sp for _, sp in s if sp["dim"] == 2]
    d3 = [sp for _, sp in s if sp["dim"] == 3]
    assert 0.45 < len(d2) / len(s) < 0.55
    assert min(sp["side"] for sp in d2) >= 32 and max(sp["side"] for sp in d2) <= 1024
    assert min(sp["side"] for sp in d3) >= 32 and max(sp["side"] for sp in d3) <= 96
    dec = np.array([sp["decades"] for _, sp in s])
    assert dec.min() >= 2 and dec.max() <= 9
    p = P.serving_problem(d3[0])
    assert p.dim == 3 and p.b.shape == (p.N,)


def test_channel_model_structure():
    p = P.channel_problem((16, 16, 16), seed=1002)
    K = p.K.reshape(16, 16, 16)
    assert set(np.unique(K)) <= {1e-9, 1.0}
    # every 4-cell z-slab holds at least one channel of K = 1 spanning the slab
    for s0 in range(0, 16, 4):
        slab = K[s0:s0 + 4]
        assert np.any(np.all(slab == 1.0, axis=0))


def test_inputs_reproduce_from_seeds():
    a, b = P.config_problem(1, scale=128), P.config_problem(1, scale=128)
    assert np.array_equal(a.K, b.K) and np.array_equal(a.f, b.f)
    p, q = P.batch_problem(7), P.batch_problem(7)
    assert np.array_equal(p.K, q.K) and np.array_equal(p.b, q.b)
    other = P.grf_problem((128, 128), seed=1002, ell=16.0, half_span=4.5)
    assert not np.array_equal(a.K, other.K)
