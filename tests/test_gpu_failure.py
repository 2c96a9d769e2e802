"""GPU failure path without a fault: a bounded device wait runs out.

The solver's grid barrier (the one of the step kernel) is run with one block
that never arrives, under a short limit. The waiting blocks must give up,
record ACCSINK_ERR_TIMEOUT in the solver state and return, within the limit
plus launch overhead, and the context must stay usable: a solve right after
it converges as usual.
"""
import numpy as np
import pytest
import torch

from paper_2605_30267_gb300 import binding as B
from paper_2605_30267_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("limit", [0.05, 0.3])
def test_barrier_wait_runs_out_and_the_context_stays_usable(limit):
    ctx = B.Context(0)
    try:
        status, elapsed = ctx.accsink_selftest_timeout(limit)
        assert status == B.ERR_TIMEOUT, status
        assert limit <= elapsed <= limit + 1.0, elapsed
        pr = W.gmm_stored_cost_problem(seed=71, n=120, m=100, eps=1e-2)
        C = torch.from_numpy(pr["C"]).to(DEV)
        a = torch.from_numpy(pr["a"]).to(DEV)
        b = torch.from_numpy(pr["b"]).to(DEV)
        f = torch.empty(120, dtype=torch.float64, device=DEV)
        g = torch.empty(100, dtype=torch.float64, device=DEV)
        res = B.result_dict(ctx.accsink_solve(B.problem_dense(C, a, b),
                                              B.default_params(eps=1e-2, tol=1e-6), f, g))
        assert res["status"] == 0 and res["marginal_l1"] < 1e-6, res
        assert np.isfinite(f.cpu().numpy()).all() and np.isfinite(g.cpu().numpy()).all()
    finally:
        ctx.close()


def test_selftest_rejects_long_limits():
    ctx = B.Context(0)
    try:
        with pytest.raises(B.AccsinkError):
            ctx.accsink_selftest_timeout(5.0)
    finally:
        ctx.close()
