"""GPU: warm starts and resumed solves (Algorithm 1-2 from a given point).

A solve's exported state (iterate x, momentum w, homotopy position, operand
shifts) resumed on the same problem at the same eps repeats one S evaluation
and then takes exactly the uninterrupted run's steps, so the potentials are
identical to the bit. At a new eps (continuation) and from a warm-start
potential the GPU is compared with the oracle's own warm_start / resume.
"""
import numpy as np
import pytest
import torch

import oracle as O
from solve_checks import check_truth, stop_tol
from paper_2605_30267_gb300 import binding as B
from paper_2605_30267_gb300 import workloads as W
from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def dense(pr):
    return B.problem_dense(to_dev(pr["C"]), to_dev(pr["a"]), to_dev(pr["b"]))


def outs(n, m):
    return (torch.empty(n, dtype=torch.float64, device=DEV),
            torch.empty(m, dtype=torch.float64, device=DEV))


def params(eps, tol, method=B.ACC, **kw):
    return B.default_params(eps=eps, tol=tol, method=method, **kw)


def solve(ctx, prob, n, m, p):
    f, g = outs(n, m)
    r = B.result_dict(ctx.accsink_solve(prob, p, f, g))
    return f.cpu().numpy(), g.cpu().numpy(), r


def export(ctx, m):
    x, w = outs(m, m)
    st = ctx.accsink_export_state(x, w)
    return st, x, w


MODES = [dict(method=B.ACC, stability=B.STAB_REPORT, carry=B.CARRY_Y),
         dict(method=B.ACC, stability=B.STAB_REPORT, carry=B.CARRY_W),
         dict(method=B.ACC, stability=B.STAB_GATE, carry=B.CARRY_Y),
         dict(method=B.ACC, stability=B.STAB_BACKTRACK, carry=B.CARRY_Y),
         dict(method=B.PLAIN)]


@pytest.mark.parametrize("mode", range(len(MODES)))
def test_resume_is_the_uninterrupted_run(ctx, mode):
    kw = MODES[mode]
    pr = W.gmm_stored_cost_problem(seed=31, n=300, m=257, eps=1e-2)
    n, m = 300, 257
    prob = dense(pr)
    f_full, g_full, full = solve(ctx, prob, n, m, params(1e-2, 1e-6, **kw))
    _, _, part = solve(ctx, prob, n, m, params(1e-2, 1e-3, **kw))
    st, x, w = export(ctx, m)
    assert st.m == m and st.method == kw["method"] and st.eps == 1e-2
    f, g = outs(n, m)
    res = B.result_dict(ctx.accsink_solve_from(prob, params(1e-2, 1e-6, **kw), st, f, g))
    k = part["sinkhorn_steps"]
    assert 1 < k < full["sinkhorn_steps"]
    assert res["sinkhorn_steps"] == full["sinkhorn_steps"] - k + 1
    assert res["status"] == full["status"] == 0
    np.testing.assert_array_equal(g.cpu().numpy(), g_full)
    np.testing.assert_array_equal(f.cpu().numpy(), f_full)
    if kw["method"] == B.ACC:
        assert res["outer_stages"] == full["outer_stages"]


def test_resume_point_clouds_is_the_uninterrupted_run(ctx):
    g0 = np.random.default_rng(5)
    n, m, d = 700, 600, 3
    X = g0.random((n, d)).astype(np.float32)
    Y = g0.random((m, d)).astype(np.float32)
    a, b = W.dirichlet1(g0, n), W.dirichlet1(g0, m)
    prob = B.problem_points(to_dev(X), to_dev(Y), kind="sqeuclid", a=to_dev(a), b=to_dev(b),
                            scale_to_max=True)
    f_full, g_full, full = solve(ctx, prob, n, m, params(5e-3, 1e-6))
    _, _, part = solve(ctx, prob, n, m, params(5e-3, 1e-3))
    st, _, _ = export(ctx, m)
    f, g = outs(n, m)
    res = B.result_dict(ctx.accsink_solve_from(prob, params(5e-3, 1e-6), st, f, g))
    assert res["sinkhorn_steps"] == full["sinkhorn_steps"] - part["sinkhorn_steps"] + 1
    np.testing.assert_array_equal(g.cpu().numpy(), g_full)
    np.testing.assert_array_equal(f.cpu().numpy(), f_full)


def gauge_close(f, g, rf, rg, tol):
    sh = g.mean() - rg.mean()
    return max(np.abs(g - sh - rg).max(), np.abs(f + sh - rf).max()) <= tol


def test_eps_continuation_matches_the_oracle(ctx):
    pr = W.gmm_stored_cost_problem(seed=32, n=200, m=180, eps=1e-2)
    n, m = 200, 180
    prob = dense(pr)
    e1, e2 = 5e-2, 5e-3
    cost = O.Cost(C=pr["C"])
    solve(ctx, prob, n, m, params(e1, 1e-4))
    st, _, _ = export(ctx, m)
    f, g = outs(n, m)
    res = B.result_dict(ctx.accsink_solve_from(prob, params(e2, 1e-6), st, f, g))
    o1 = O.solve(cost, pr["a"], pr["b"], e1, tol=stop_tol(1e-4))
    ores = O.resume(cost, pr["a"], pr["b"], e2, o1["state"], tol=stop_tol(1e-6))
    cold = O.solve(cost, pr["a"], pr["b"], e2, tol=1e-11)
    assert res["status"] == 0 and ores["status"] == O.CONVERGED
    rs, gs = ores["sinkhorn_steps"], res["sinkhorn_steps"]
    assert abs(gs - rs) <= max(1, int(0.05 * rs)), (gs, rs)
    assert gauge_close(f.cpu().numpy(), g.cpu().numpy(), cold["f"], cold["g"], 1e-3 * e2)
    ev = O.evaluate(cost, e2, cold["a"], cold["b"], f.cpu().numpy(), g.cpu().numpy())
    check_truth(ev, 1e-6)


@pytest.mark.parametrize("method", [B.ACC, B.PLAIN])
def test_warm_start_at_the_fixed_point_stops_at_once(ctx, method):
    pr = W.gmm_stored_cost_problem(seed=33, n=250, m=220, eps=1e-2)
    ref = O.solve(O.Cost(C=pr["C"]), pr["a"], pr["b"], 1e-2, tol=1e-11)
    f, g = outs(250, 220)
    res = B.result_dict(ctx.accsink_warm_start(dense(pr), params(1e-2, 1e-6, method),
                                               to_dev(ref["g"]), f, g))
    assert res["status"] == 0 and res["sinkhorn_steps"] == 1
    assert gauge_close(f.cpu().numpy(), g.cpu().numpy(), ref["f"], ref["g"], 1e-5 * 1e-2)


@pytest.mark.parametrize("method", [B.ACC, B.PLAIN])
def test_warm_start_matches_the_oracle(ctx, method):
    pr = W.gmm_stored_cost_problem(seed=34, n=220, m=260, eps=5e-3)
    cost = O.Cost(C=pr["C"])
    # start at the eps = 5e-2 solution
    g0 = O.solve(cost, pr["a"], pr["b"], 5e-2, tol=1e-9)["g"]
    f, g = outs(220, 260)
    res = B.result_dict(ctx.accsink_warm_start(dense(pr), params(5e-3, 1e-6, method),
                                               to_dev(g0), f, g))
    om = O.ACC if method == B.ACC else O.PLAIN
    ref = O.warm_start(cost, pr["a"], pr["b"], 5e-3, g0, tol=stop_tol(1e-6), method=om)
    cold = O.solve(cost, pr["a"], pr["b"], 5e-3, tol=1e-11)
    rs, gs = ref["sinkhorn_steps"], res["sinkhorn_steps"]
    assert res["status"] == 0 and abs(gs - rs) <= max(1, int(0.05 * rs)), (gs, rs)
    assert gauge_close(f.cpu().numpy(), g.cpu().numpy(), cold["f"], cold["g"], 1e-3 * 5e-3)


def test_warm_start_from_zero_is_the_cold_start_within_rounding(ctx):
    pr = W.gmm_stored_cost_problem(seed=35, n=150, m=170, eps=1e-2)
    prob = dense(pr)
    fc, gc, cold = solve(ctx, prob, 150, 170, params(1e-2, 1e-6))
    f, g = outs(150, 170)
    res = B.result_dict(ctx.accsink_warm_start(prob, params(1e-2, 1e-6),
                                               torch.zeros(170, dtype=torch.float64,
                                                           device=DEV), f, g))
    assert abs(res["sinkhorn_steps"] - cold["sinkhorn_steps"]) <= 1
    assert gauge_close(f.cpu().numpy(), g.cpu().numpy(), fc, gc, 1e-4 * 1e-2)


def test_state_errors(ctx):
    c2 = B.Context(0)
    try:
        x, w = outs(64, 64)
        with pytest.raises(B.AccsinkError):
            c2.accsink_export_state(x, w)            # no solve yet
        pr = W.gmm_stored_cost_problem(seed=36, n=64, m=64, eps=1e-2)
        prob = dense(pr)
        solve(c2, prob, 64, 64, params(1e-2, 1e-6))
        st = c2.accsink_export_state(x, w)
        with pytest.raises(B.AccsinkError):
            c2.accsink_export_state(*outs(63, 63))   # wrong m
        f, g = outs(64, 64)
        with pytest.raises(B.AccsinkError):          # method differs from the state's
            c2.accsink_solve_from(prob, params(1e-2, 1e-6, B.PLAIN), st, f, g)
        bad = B.accsink_state.from_buffer_copy(st)
        bad.j_in_stage = bad.m_stage
        with pytest.raises(B.AccsinkError):
            c2.accsink_solve_from(prob, params(1e-2, 1e-6), bad, f, g)
        c2.accsink_row_pass(prob, 1e-2, to_dev(np.zeros(64)), f)
        with pytest.raises(B.AccsinkError):
            c2.accsink_export_state(x, w)            # a single pass replaced the state
    finally:
        c2.close()


# Point-cloud solves with d <= 4 run on curve-sorted clouds: warm starts and
# exported states go through the permutation in both directions.

def points_prob(seed, n, m, d=3):
    g0 = np.random.default_rng(seed)
    X = g0.random((n, d)).astype(np.float32)
    Y = g0.random((m, d)).astype(np.float32)
    a, b = W.dirichlet1(g0, n), W.dirichlet1(g0, m)
    prob = B.problem_points(to_dev(X), to_dev(Y), kind="sqeuclid", a=to_dev(a), b=to_dev(b),
                            scale_to_max=True)
    return prob, O.Cost(X=X, Y=Y, kind="sqeuclid", scale_to_max=True), a, b


def test_points_warm_start_at_the_fixed_point_stops_at_once(ctx):
    prob, cost, a, b = points_prob(51, 900, 1100)
    ref = O.solve(cost, a, b, 1e-2, tol=1e-11)
    f, g = outs(900, 1100)
    res = B.result_dict(ctx.accsink_warm_start(prob, params(1e-2, 1e-6), to_dev(ref["g"]), f, g))
    assert res["status"] == 0 and res["sinkhorn_steps"] == 1
    assert gauge_close(f.cpu().numpy(), g.cpu().numpy(), ref["f"], ref["g"], 1e-5 * 1e-2)


def test_points_eps_continuation_matches_the_oracle(ctx):
    prob, cost, a, b = points_prob(52, 800, 700)
    e1, e2 = 5e-2, 5e-3
    solve(ctx, prob, 800, 700, params(e1, 1e-4))
    st, x, w = export(ctx, 700)
    o1 = O.solve(cost, a, b, e1, tol=stop_tol(1e-4))
    # the exported iterate is in the caller's column order: it is the same
    # potential as the oracle's to the solve's accuracy
    assert np.abs(e1 * (x.cpu().numpy() - x.cpu().numpy().mean())
                  - e1 * (o1["state"]["x"] - o1["state"]["x"].mean())).max() <= 1e-3 * e1
    f, g = outs(800, 700)
    res = B.result_dict(ctx.accsink_solve_from(prob, params(e2, 1e-6), st, f, g))
    ores = O.resume(cost, a, b, e2, o1["state"], tol=stop_tol(1e-6))
    cold = O.solve(cost, a, b, e2, tol=1e-11)
    rs, gs = ores["sinkhorn_steps"], res["sinkhorn_steps"]
    assert res["status"] == 0 and abs(gs - rs) <= max(1, int(0.05 * rs)), (gs, rs)
    assert gauge_close(f.cpu().numpy(), g.cpu().numpy(), cold["f"], cold["g"], 1e-3 * e2)
