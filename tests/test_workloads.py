"""CPU checks of the seeded synthetic inputs: every generator is a pure
function of its seed, and each produces the shapes, ranges and structure its
recipe states (points in [0,1]^d, unit-norm vectors, probability marginals,
log-uniform sizes, the cost scaled to max 1 and rounded once to FP32)."""
import math

import numpy as np

from paper_2605_30267_gb300 import workloads as W


def test_generators_are_deterministic_in_the_seed():
    a = W.gmm_stored_cost_problem(seed=3, n=64, m=80)
    b = W.gmm_stored_cost_problem(seed=3, n=64, m=80)
    c = W.gmm_stored_cost_problem(seed=4, n=64, m=80)
    for k in ("C", "a", "b", "X", "Y"):
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["X"], c["X"])
    r1 = W.serving_requests(seed=5, count=3, hi=256)
    r2 = W.serving_requests(seed=5, count=3, hi=256)
    for p, q in zip(r1, r2):
        np.testing.assert_array_equal(p["X"], q["X"])
        assert p["eps"] == q["eps"]


def test_marginals_are_probability_vectors():
    g = W.rng(0)
    for n in (1, 7, 1000):
        a = W.dirichlet1(g, n)
        assert a.dtype == np.float64 and a.shape == (n,)
        assert np.all(a > 0) and abs(a.sum() - 1.0) < 1e-12
    u = W.uniform_marginal(5)
    assert np.allclose(u, 0.2) and abs(u.sum() - 1.0) < 1e-15


def test_stored_cost_is_the_fp64_cost_scaled_and_rounded_once():
    pr = W.gmm_stored_cost_problem(seed=1, n=50, m=70)
    X, Y, C = pr["X"], pr["Y"], pr["C"]
    assert C.dtype == np.float32 and C.shape == (50, 70)
    exact = ((X.astype(np.float64)[:, None, :] - Y.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(C, (exact / exact.max()).astype(np.float32))
    assert C.max() == np.float32(1.0) and C.min() >= 0.0


def test_colour_transfer_clouds_lie_in_the_unit_cube():
    pr = W.color_transfer_problem(seed=2, n=4096)
    for P in (pr["X"], pr["Y"]):
        assert P.dtype == np.float32 and P.shape == (4096, 3)
        assert P.min() >= 0.0 and P.max() <= 1.0
    # the target is clustered: far fewer distinct coarse cells than the uniform source
    cells = lambda P: len({tuple(v) for v in np.floor(P * 8).astype(int)})
    assert cells(pr["Y"]) < 0.6 * cells(pr["X"])


def test_word_alignment_batch_recipe():
    batch = W.word_alignment_batch(seed=0, count=40, d=300)
    assert len(batch) == 40
    for p in batch:
        n, m = p["X"].shape[0], p["Y"].shape[0]
        assert 16 <= n <= 2048 and 16 <= m <= 2048
        assert p["X"].shape[1] == p["Y"].shape[1] == 300
        np.testing.assert_allclose(np.linalg.norm(p["X"].astype(np.float64), axis=1), 1.0, atol=1e-6)
        assert 0.005 <= p["eps"] <= 0.05
        assert abs(p["a"].sum() - 1.0) < 1e-12 and abs(p["b"].sum() - 1.0) < 1e-12
    # log-uniform sizes: the median lies near the geometric mean of the range
    sizes = [p["X"].shape[0] for p in W.word_alignment_batch(seed=1, count=400, d=2)]
    assert 0.6 * math.sqrt(16 * 2048) < np.median(sizes) < 1.6 * math.sqrt(16 * 2048)


def test_serving_requests_recipe():
    reqs = W.serving_requests(seed=0, count=200, hi=1024)
    ds = {r["X"].shape[1] for r in reqs}
    assert min(ds) >= 2 and max(ds) <= 64 and len(ds) > 20
    for r in reqs:
        assert 64 <= r["X"].shape[0] <= 1024 and 64 <= r["Y"].shape[0] <= 1024
        assert 1e-3 <= r["eps"] <= 1e-1
        assert r["X"].min() >= 0.0 and r["X"].max() < 1.0
    t = W.poisson_arrivals(7, rate=100.0, count=5000)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 5000 - 0.01) < 0.001      # mean gap 1 / rate
