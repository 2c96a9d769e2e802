"""The allocation-free column pass (accsink_col_lse_noalloc) against the
context-based accsink_col_lse, on two calls in a row through the C-ABI.

It is for callers that cannot allocate device memory; its scratch is a fixed
file-scope device array shared by every call, so the second call must not
see anything left over from the first. This file is collected last."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_30267_gb300 import binding as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 2e-6   # the single-pass tolerance of the parity tests (natural-log units)


def _case(seed, n, m, eps):
    g = np.random.default_rng(seed)
    C = torch.from_numpy(g.random((n, m)).astype(np.float32)).to(DEV)
    f = torch.from_numpy(0.3 * g.standard_normal(n)).to(DEV)
    return C, f, eps


def test_noalloc_col_lse_matches_context_pass_twice():
    torch.cuda.set_device(0)
    ctx = B.Context(0)
    try:
        # two calls in a row with different shapes and eps: the second must
        # not depend on what the first left in the shared scratch
        for seed, n, m, eps in ((1, 700, 1501, 1e-2), (2, 257, 3001, 1e-3)):
            C, f, eps = _case(seed, n, m, eps)
            prob = B.problem_dense(C)
            ref = torch.empty(m, dtype=torch.float64, device=DEV)
            ctx.accsink_col_lse(prob, eps, f, ref)
            out = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
            rc = B.accsink_col_lse_noalloc(prob, eps, f, out)
            assert rc == B.OK
            torch.cuda.synchronize()
            d = (out - ref).abs().max().item()
            assert d <= TOL, (seed, d)
            # and against the FP64 oracle's column log-sum-exp
            orc = O.col_lse(O.Cost(C=C.cpu().numpy()), eps, f.cpu().numpy() / eps)
            assert np.abs(out.cpu().numpy() - orc).max() <= TOL
    finally:
        ctx.close()


def test_noalloc_col_lse_near_its_size_limit():
    # m = 1.5e6 columns: 12 MB of column partials in the 16 MiB scratch
    torch.cuda.set_device(0)
    n, m, eps = 64, 1_500_000, 1e-2
    C, f, eps = _case(3, n, m, eps)
    prob = B.problem_dense(C)
    ctx = B.Context(0)
    try:
        ref = torch.empty(m, dtype=torch.float64, device=DEV)
        ctx.accsink_col_lse(prob, eps, f, ref)
        out = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
        assert B.accsink_col_lse_noalloc(prob, eps, f, out) == B.OK
        torch.cuda.synchronize()
        assert (out - ref).abs().max().item() <= TOL
        cols = np.random.default_rng(5).choice(m, 64, replace=False)
        orc = O.col_lse_sample(O.Cost(C=C.cpu().numpy()), eps, f.cpu().numpy() / eps, cols)
        assert np.abs(out.cpu().numpy()[cols] - orc).max() <= TOL
    finally:
        ctx.close()


def _raw_call(prob, eps, f, out):
    # straight through the C-ABI: the library's own size checks, not the
    # binding's vector checks, are what these cases test
    return B.lib().accsink_col_lse_noalloc(ct.byref(prob), float(eps), f.data_ptr(),
                                           out.data_ptr(), None)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # n large enough that the per-row operand alone exceeds the 16 MiB
    # scratch; the size check runs before any kernel reads C or f.
    C = torch.zeros((1, 8), dtype=torch.float32, device=DEV)
    prob = B.problem_dense(C)
    prob.n = 3_000_000
    f = torch.zeros(8, dtype=torch.float64, device=DEV)
    out = torch.zeros(8, dtype=torch.float64, device=DEV)
    assert _raw_call(prob, 1e-2, f, out) == B.ERR_BUDGET
    # m large enough that one split of column partials exceeds it
    prob.n, prob.m, prob.ldc = 1, 2_100_000, 2_100_000
    assert _raw_call(prob, 1e-2, f, out) == B.ERR_BUDGET
    prob.n, prob.m, prob.ldc = 0, 8, 8
    assert _raw_call(prob, 1e-2, f, out) == B.ERR_INVALID_ARG
