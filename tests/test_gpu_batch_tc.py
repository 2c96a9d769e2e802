"""GPU parity of the tensor-core formation of cosine costs in the batched
solver (tcgen05 MMAs on integer slices, batch_form_tc.cu).

Cosine problems with 32 <= d <= 480 form their costs on the tensor cores;
ACCSINK_BATCH_FORM=cuda selects the exact CUDA-core expansion instead. The
two must give the same solves to far below the solver's tolerances, and the
tensor-core path must meet the oracle's tolerances on its own, including
vectors whose slice sums are large (coherent signs, d = 480), ragged tile
edges (n, m not multiples of 128 and 64), the transposed cost of large
problems and a non-finite input.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from test_gpu_batch import DEV, Prob, check_against_oracle, run_batch
from paper_2605_30267_gb300 import binding as B
from paper_2605_30267_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def cuda_core_form(ctx, probs):
    os.environ["ACCSINK_BATCH_FORM"] = "cuda"
    try:
        return run_batch(ctx, probs)
    finally:
        del os.environ["ACCSINK_BATCH_FORM"]


def coherent_problem(seed, n, d, eps):
    """X and Y drawn from the same few directions (x ~ y up to small noise),
    so the slice products add with equal signs and the class sums reach
    about 2^23 for d = 480; costs scaled to max 1."""
    g = np.random.default_rng(seed)
    base = W.unit_gaussian_points(g, 4, d)
    X = (base[g.integers(0, 4, n)] + 1e-3 * g.standard_normal((n, d))).astype(np.float32)
    Y = (base[g.integers(0, 4, n + 7)] + 1e-3 * g.standard_normal((n + 7, d))).astype(np.float32)
    p = Prob.__new__(Prob)
    p.kind, p.eps, p.tol, p.method, p.scale, p.kw = "cosine", eps, 1e-6, B.ACC, True, {}
    p.X, p.Y = X, Y
    p.a, p.b = W.dirichlet1(g, n), W.dirichlet1(g, n + 7)
    p.n, p.m = n, n + 7
    p.cost = O.Cost(X=X, Y=Y, kind="cosine", scale_to_max=True)
    return p


def tc_problems():
    return [Prob("cosine", 129, 250, 41, 2e-2, d=40),
            Prob("cosine", 1, 65, 42, 1e-2, d=32),
            Prob("cosine", 200, 1, 43, 1e-2, d=33),
            Prob("cosine", 300, 191, 44, 5e-3, d=300),
            Prob("cosine", 64, 129, 45, 1e-2, d=480, scale=True),
            Prob("cosine", 257, 63, 46, 5e-3, d=100, method=B.PLAIN)]


def test_tensor_core_form_matches_oracle(ctx):
    probs = tc_problems()
    fs, gs, rs = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, fs, gs, rs):
        check_against_oracle(p, f, g, r)


def test_coherent_slices_match_oracle(ctx):
    probs = [coherent_problem(51, 150, 480, 5e-3), coherent_problem(52, 97, 64, 1e-2)]
    fs, gs, rs = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, fs, gs, rs):
        check_against_oracle(p, f, g, r)


def test_tensor_core_and_cuda_core_forms_agree(ctx):
    """Costs from the two formations differ by at most ~2^-31 |x||y|, so the
    steps match and the potentials agree to 1e-6 eps; the transport costs of
    the two converged iterates then agree to 1e-7 relative (measured:
    1.4e-8 on the coherent d = 480 problem), 100 times inside the oracle
    tolerance."""
    probs = tc_problems() + [coherent_problem(53, 130, 480, 5e-3)]
    f1, g1, r1 = run_batch(ctx, probs)
    f2, g2, r2 = cuda_core_form(ctx, probs)
    for k, p in enumerate(probs):
        assert abs(r1[k]["sinkhorn_steps"] - r2[k]["sinkhorn_steps"]) <= 1, k
        if r1[k]["sinkhorn_steps"] != r2[k]["sinkhorn_steps"]:
            continue
        sh = g1[k].mean() - g2[k].mean()
        d = max(np.abs(g1[k] - sh - g2[k]).max(), np.abs(f1[k] + sh - f2[k]).max())
        assert d <= 1e-6 * p.eps, (k, d)
        assert abs(r1[k]["transport_cost"] - r2[k]["transport_cost"]) <= \
            1e-7 * abs(r2[k]["transport_cost"]), k


def test_large_tensor_core_problem_uses_the_transposed_cost(ctx):
    """n m >= 2^20 also stores K^T (written by the tensor-core epilogue);
    parity with the oracle and identical potentials for two work splits."""
    probs = [Prob("cosine", 1100, 1000, 61, 2e-2, d=64),
             Prob("cosine", 1031, 1029, 62, 1e-2, d=96, scale=True)]
    ctx.accsink_batch_set_config()
    f1, g1, r1 = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, f1, g1, r1):
        check_against_oracle(p, f, g, r)
    ctx.accsink_batch_set_config(small_max_nm=64, row_tile_elems=50000)
    try:
        f2, g2, r2 = run_batch(ctx, probs)
    finally:
        ctx.accsink_batch_set_config()
    for k in range(len(probs)):
        assert r1[k]["sinkhorn_steps"] == r2[k]["sinkhorn_steps"]
        np.testing.assert_array_equal(f1[k], f2[k])
        np.testing.assert_array_equal(g1[k], g2[k])


def test_tensor_core_form_is_deterministic(ctx):
    probs = tc_problems()[:4]
    a = run_batch(ctx, probs)
    b = run_batch(ctx, probs)
    for k in range(len(probs)):
        np.testing.assert_array_equal(a[0][k], b[0][k])
        np.testing.assert_array_equal(a[1][k], b[1][k])


def test_nonfinite_tensor_core_problem_fails_alone(ctx):
    good = tc_problems()[:2]
    bad = Prob("cosine", 70, 90, 71, 1e-2, d=64)
    bad.Y = bad.Y.copy()
    bad.Y[5, 17] = np.nan
    probs = [good[0], bad, good[1]]
    structs = [p.struct() for p in probs]
    params = [p.params() for p in probs]
    fs = [torch.empty(p.n, dtype=torch.float64, device=DEV) for p in probs]
    gs = [torch.empty(p.m, dtype=torch.float64, device=DEV) for p in probs]
    k, pa, qa, fa, ga, ra = B.Context._batch_arrays(structs, params, fs, gs)
    rc = B.lib().accsink_solve_batch(ctx._h, k, pa, qa, None, fa, ga, ra)
    assert rc == B.ERR_NONFINITE
    assert ra[0].status == 0 and ra[1].status == B.ERR_NONFINITE and ra[2].status == 0
