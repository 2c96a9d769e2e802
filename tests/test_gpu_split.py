"""GPU parity of the warp-per-row passes when rows are split into column parts.

When whole rows would leave the last wave of warps part-empty (or leave warps
idle when there are fewer rows than resident warps), the row pass over C and
the column pass over C^T split the rows of that wave into column parts, and
the last part of a row to finish merges the parts in a fixed order. These
shapes force such splits, with a ragged last part (m % 4 != 0), in the single
row pass, the S map and whole solves (row split over C, column split over
C^T), and check that the merge does not depend on which part finished last:
repeated solves are bitwise identical.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_30267_gb300 import binding as B
from paper_2605_30267_gb300 import workloads as W
from test_gpu_parity import PASS_TOL, check_solve, gpu_solve, potential_like, rand_dense, to_dev

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def resident_warps(ctx):
    # three CTAs of eight warps per SM
    return ctx.accsink_launch_geometry(64, 64)["num_sms"] * 24


def split_shapes(ctx):
    w = resident_warps(ctx)
    return [(37, 16387),          # fewer rows than warps: 8 parts of 4 chunks
            (w // 3, 4099),       # two parts, ragged last part
            (w + 101, 8195)]      # one full wave of whole rows, then 101 split rows


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("eps", [1e-1, 1e-3])
def test_split_row_pass_matches_oracle(ctx, k, eps):
    n, m = split_shapes(ctx)[k]
    C, a, b = rand_dense(n * 5 + m + k, n, m)
    g = potential_like(n + 7 * m, m, eps)
    f = torch.empty(n, dtype=torch.float64, device=DEV)
    ctx.accsink_row_pass(B.problem_dense(to_dev(C), to_dev(a), to_dev(b)), eps, to_dev(g), f)
    torch.cuda.synchronize()
    ref = eps * O.row_pass(O.Cost(C=C), eps, np.log(a), g / eps)
    err = np.abs(f.cpu().numpy() - ref).max() / eps
    assert err <= PASS_TOL, err


def test_split_sinkhorn_map_matches_oracle(ctx):
    n, m = split_shapes(ctx)[2]
    eps = 1e-2
    C, a, b = rand_dense(4242, n, m)
    g = potential_like(99, m, eps)
    f = torch.empty(n, dtype=torch.float64, device=DEV)
    c = torch.empty(m, dtype=torch.float64, device=DEV)
    s = torch.empty(m, dtype=torch.float64, device=DEV)
    err = ctx.accsink_sinkhorn_map(B.problem_dense(to_dev(C), to_dev(a), to_dev(b)), eps,
                                   to_dev(g), f, c, s)
    rerr, ru, rc, rs = O.sinkhorn_map(O.Cost(C=C), eps, a, b, g / eps)
    assert np.abs(f.cpu().numpy() / eps - ru).max() <= PASS_TOL
    np.testing.assert_allclose(c.cpu().numpy(), rc, rtol=5 * PASS_TOL, atol=1e-300)
    assert np.abs(s.cpu().numpy() / eps - rs).max() <= 2 * PASS_TOL
    assert abs(err - rerr) <= 5 * PASS_TOL * max(1.0, rerr)


# (300, 8195): the row pass over C splits; (8195, 300): the column pass over C^T
@pytest.mark.parametrize("n,m", [(300, 8195), (8195, 300)])
def test_split_solves_match_oracle(ctx, n, m):
    pr = W.gmm_stored_cost_problem(seed=n + 2 * m, n=n, m=m, eps=3e-2)
    for method in (B.ACC, B.PLAIN):
        check_solve(ctx, pr["C"], pr["a"], pr["b"], 3e-2, 1e-6, method)


@pytest.mark.parametrize("n,m", [(300, 8195), (8195, 300)])
def test_split_solves_are_bitwise_reproducible(ctx, n, m):
    pr = W.gmm_stored_cost_problem(seed=n + 3 * m, n=n, m=m, eps=1e-2)
    runs = [gpu_solve(ctx, pr["C"], pr["a"], pr["b"], 1e-2, 1e-6, B.ACC, use_graph=ug)
            for ug in (1, 0, 1)]
    steps = {r[2]["sinkhorn_steps"] for r in runs}
    assert len(steps) == 1, steps
    for f, g, res in runs[1:]:
        np.testing.assert_array_equal(f, runs[0][0])
        np.testing.assert_array_equal(g, runs[0][1])
        assert res["dual_objective"] == runs[0][2]["dual_objective"]
        assert res["transport_cost"] == runs[0][2]["transport_cost"]
