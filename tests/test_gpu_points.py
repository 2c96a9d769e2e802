"""GPU parity of the point-cloud path (costs formed on the fly, Sec. 5's
colour-transfer and word-alignment costs) against the FP64 oracle, whose cost
is formed in FP64 from the same FP32 points.

Tolerances as for stored costs: potentials within 1e-3 eps max-abs after
centring, <C,P> within 1e-5 relative, step counts within 2% (or one step) of
the oracle run to the library's stopping threshold, and the FP64 truth of
eq. l1tol (row plus column L1) below tol with the row L1 at the FP32 floor.
"""
import numpy as np
import pytest
import torch

import oracle as O
from solve_checks import check_steps, check_truth, same_iterate, stop_tol
from paper_2605_30267_gb300 import binding as B
from paper_2605_30267_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def gpu_solve_points(ctx, X, Y, kind, a, b, eps, tol, method, scale, **kw):
    n, m = X.shape[0], Y.shape[0]
    f = torch.empty(n, dtype=torch.float64, device=DEV)
    g = torch.empty(m, dtype=torch.float64, device=DEV)
    p = B.default_params(eps=eps, tol=tol, method=method, **kw)
    prob = B.problem_points(to_dev(X), to_dev(Y), kind, to_dev(a), to_dev(b), scale)
    res = ctx.accsink_solve(prob, p, f, g)
    return f.cpu().numpy(), g.cpu().numpy(), B.result_dict(res)


def check_points(ctx, X, Y, kind, a, b, eps, tol=1e-6, method=B.ACC, scale=False, **kw):
    f, g, res = gpu_solve_points(ctx, X, Y, kind, a, b, eps, tol, method, scale, **kw)
    cost = O.Cost(X=X, Y=Y, kind=kind, scale_to_max=scale)
    okw = dict(method=O.ACC if method == B.ACC else O.PLAIN,
               carry_y=kw.get("carry", B.CARRY_Y) == B.CARRY_Y,
               stability=kw.get("stability", B.STAB_REPORT))
    ref = O.solve(cost, a, b, eps, stop_tol(tol), **okw)
    assert res["status"] == 0, res
    assert ref["status"] == O.CONVERGED
    rs, gs = ref["sinkhorn_steps"], res["sinkhorn_steps"]
    check_steps(cost, a, b, eps, tol, okw, rs, gs)
    ref = same_iterate(cost, a, b, eps, okw, ref, gs)
    sh = g.mean() - ref["g"].mean()
    dpot = max(np.abs(g - sh - ref["g"]).max(), np.abs(f + sh - ref["f"]).max())
    assert dpot <= 1e-3 * eps, dpot
    ev = O.evaluate(cost, eps, ref["a"], ref["b"], f, g)
    check_truth(ev, tol)
    evr = O.evaluate(cost, eps, ref["a"], ref["b"], ref["f"], ref["g"])
    assert abs(res["transport_cost"] - evr["transport_cost"]) <= \
        1e-5 * abs(evr["transport_cost"]), (res["transport_cost"], evr["transport_cost"])
    assert abs(res["dual_objective"] - ref["dual"]) <= 1e-5 * max(1e-3, abs(ref["dual"]))
    return f, g, res, ref


def sqeuclid_points(seed, n, m, d, spread=1.0):
    g = np.random.default_rng(seed)
    X = (spread * g.random((n, d))).astype(np.float32)
    Y = (spread * g.random((m, d))).astype(np.float32)
    return X, Y, W.dirichlet1(g, n), W.dirichlet1(g, m)


def cosine_points(seed, n, m, d):
    g = np.random.default_rng(seed)
    X = W.unit_gaussian_points(g, n, d)
    Y = W.unit_gaussian_points(g, m, d)
    return X, Y, W.dirichlet1(g, n), W.dirichlet1(g, m)


# ------------------------------------------------------ single passes --

PASS_TOL = 2e-6
PT_SHAPES = [(1, 1), (3, 5), (9, 1), (37, 129), (513, 2049), (1000, 1003)]


def points_for(kind, seed, n, m, d):
    return sqeuclid_points(seed, n, m, d) if kind == "sqeuclid" else cosine_points(seed, n, m, d)


def potential_like(seed, k):
    g = np.random.default_rng(seed)
    return 0.3 * g.standard_normal(k) + 0.05 * g.random(k)


@pytest.mark.parametrize("n,m", PT_SHAPES)
# d = 1..4 cover the exact-dimension kernels (d = 2, 3, 4) and the d < 4 bound
@pytest.mark.parametrize("kind,d", [("sqeuclid", 1), ("sqeuclid", 2), ("sqeuclid", 3),
                                    ("cosine", 4), ("sqeuclid", 9), ("cosine", 16),
                                    ("cosine", 64)])
@pytest.mark.parametrize("eps", [1e-1, 1e-3])
def test_point_row_pass_matches_oracle(ctx, n, m, kind, d, eps):
    X, Y, a, b = points_for(kind, n * 7 + m + d, n, m, d)
    g = potential_like(n + 3 * m, m)
    f = torch.empty(n, dtype=torch.float64, device=DEV)
    prob = B.problem_points(to_dev(X), to_dev(Y), kind, to_dev(a), to_dev(b))
    ctx.accsink_row_pass(prob, eps, to_dev(g), f)
    torch.cuda.synchronize()
    ref = eps * O.row_pass(O.Cost(X=X, Y=Y, kind=kind), eps, np.log(a), g / eps)
    err = np.abs(f.cpu().numpy() - ref).max() / eps
    assert err <= PASS_TOL, err


@pytest.mark.parametrize("n,m", PT_SHAPES)
@pytest.mark.parametrize("kind,d", [("sqeuclid", 3), ("cosine", 33)])
@pytest.mark.parametrize("eps", [1e-1, 1e-3])
def test_point_col_lse_matches_oracle(ctx, n, m, kind, d, eps):
    X, Y, a, b = points_for(kind, n * 11 + m + d, n, m, d)
    f = potential_like(2 * n + m, n)
    ell = torch.empty(m, dtype=torch.float64, device=DEV)
    prob = B.problem_points(to_dev(X), to_dev(Y), kind)
    ctx.accsink_col_lse(prob, eps, to_dev(f), ell)
    torch.cuda.synchronize()
    ref = O.col_lse(O.Cost(X=X, Y=Y, kind=kind), eps, f / eps)
    err = np.abs(ell.cpu().numpy() - ref).max()
    assert err <= PASS_TOL, err


@pytest.mark.parametrize("kind,d", [("sqeuclid", 3), ("cosine", 20)])
@pytest.mark.parametrize("scale", [False, True])
def test_point_sinkhorn_map_matches_oracle(ctx, kind, d, scale):
    n, m, eps = 257, 1000, 1e-2
    X, Y, a, b = points_for(kind, d + 3, n, m, d)
    g = potential_like(17, m)
    f = torch.empty(n, dtype=torch.float64, device=DEV)
    c = torch.empty(m, dtype=torch.float64, device=DEV)
    s = torch.empty(m, dtype=torch.float64, device=DEV)
    prob = B.problem_points(to_dev(X), to_dev(Y), kind, to_dev(a), to_dev(b), scale)
    err = ctx.accsink_sinkhorn_map(prob, eps, to_dev(g), f, c, s)
    cost = O.Cost(X=X, Y=Y, kind=kind, scale_to_max=scale)
    rerr, ru, rc, rs = O.sinkhorn_map(cost, eps, a, b, g / eps)
    assert np.abs(f.cpu().numpy() / eps - ru).max() <= PASS_TOL
    np.testing.assert_allclose(c.cpu().numpy(), rc, rtol=5 * PASS_TOL, atol=1e-300)
    assert np.abs(s.cpu().numpy() / eps - rs).max() <= 2 * PASS_TOL
    assert abs(err - rerr) <= 5 * PASS_TOL * max(1.0, rerr)


@pytest.mark.parametrize("kind,d", [("sqeuclid", 3), ("cosine", 12)])
@pytest.mark.parametrize("scale", [False, True])
def test_point_transport_cost_matches_oracle(ctx, kind, d, scale):
    n, m, eps = 300, 211, 2e-2
    X, Y, a, b = points_for(kind, 77 + d, n, m, d)
    cost = O.Cost(X=X, Y=Y, kind=kind, scale_to_max=scale)
    ref = O.solve(cost, a, b, eps, tol=1e-9, method=O.PLAIN)
    ev = O.evaluate(cost, eps, ref["a"], ref["b"], ref["f"], ref["g"])
    prob = B.problem_points(to_dev(X), to_dev(Y), kind, None, None, scale)
    out = ctx.accsink_transport_cost(prob, eps, to_dev(ref["f"]), to_dev(ref["g"]))
    assert abs(out - ev["transport_cost"]) <= 1e-6 * abs(ev["transport_cost"])


def test_dense_single_passes_honour_max_to_one(ctx):
    """The dense single-pass calls read C / max C under MAX_TO_ONE."""
    n, m, eps = 120, 340, 1e-2
    g0 = np.random.default_rng(4)
    C = (3.0 * g0.random((n, m))).astype(np.float32)
    a, b = W.dirichlet1(g0, n), W.dirichlet1(g0, m)
    cost = O.Cost(C=C, scale_to_max=True)
    g = potential_like(5, m)
    f = torch.empty(n, dtype=torch.float64, device=DEV)
    ctx.accsink_row_pass(B.problem_dense(to_dev(C), to_dev(a), to_dev(b), True), eps,
                         to_dev(g), f)
    torch.cuda.synchronize()
    ref = eps * O.row_pass(cost, eps, np.log(a), g / eps)
    assert np.abs(f.cpu().numpy() - ref).max() / eps <= PASS_TOL
    ell = torch.empty(m, dtype=torch.float64, device=DEV)
    ctx.accsink_col_lse(B.problem_dense(to_dev(C), None, None, True), eps, f, ell)
    torch.cuda.synchronize()
    ref2 = O.col_lse(cost, eps, f.cpu().numpy() / eps)
    assert np.abs(ell.cpu().numpy() - ref2).max() <= PASS_TOL
    ref3 = O.solve(cost, a, b, eps, tol=1e-9, method=O.PLAIN)
    ev = O.evaluate(cost, eps, ref3["a"], ref3["b"], ref3["f"], ref3["g"])
    out = ctx.accsink_transport_cost(B.problem_dense(to_dev(C), None, None, True), eps,
                                     to_dev(ref3["f"]), to_dev(ref3["g"]))
    assert abs(out - ev["transport_cost"]) <= 1e-6 * abs(ev["transport_cost"])


# -------------------------------------------------------------- solves --

def test_uniform_2d_256_matches_oracle(ctx):
    """The 256-point uniform [0,1]^2 problem, cost scaled to max 1, eps 1e-2."""
    pr = W.small_pointcloud_problem(0)
    for method in (B.ACC, B.PLAIN):
        check_points(ctx, pr["X"], pr["Y"], "sqeuclid", pr["a"], pr["b"], pr["eps"],
                     pr["tol"], method, scale=True)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
@pytest.mark.parametrize("n,m,d", [(333, 200, 3), (64, 1031, 2), (517, 515, 5)])
def test_sqeuclid_solves_match_oracle(ctx, eps, n, m, d):
    X, Y, a, b = sqeuclid_points(n * 3 + m + d, n, m, d)
    check_points(ctx, X, Y, "sqeuclid", a, b, eps, scale=True)


@pytest.mark.parametrize("n,m,d", [(300, 257, 16), (129, 250, 64), (200, 180, 7)])
@pytest.mark.parametrize("eps", [5e-3, 5e-2])
def test_cosine_solves_match_oracle(ctx, n, m, d, eps):
    X, Y, a, b = cosine_points(n + 5 * m + d, n, m, d)
    check_points(ctx, X, Y, "cosine", a, b, eps)


def test_unscaled_sqeuclid_with_large_coordinates(ctx):
    """Costs of size ~50 without scaling: the operand shifts stay exact."""
    X, Y, a, b = sqeuclid_points(41, 150, 170, 3, spread=4.0)
    f, g, res, ref = check_points(ctx, X, Y, "sqeuclid", a, b, 0.5)
    cost = O.Cost(X=X, Y=Y, kind="sqeuclid")
    assert abs(res["cost_max"] - cost.unscaled_max()) <= 1e-12 * cost.unscaled_max()


@pytest.mark.parametrize("n,m", [(1, 1), (1, 9), (9, 1), (5, 3)])
def test_tiny_point_solves(ctx, n, m):
    X, Y, a, b = sqeuclid_points(n * 10 + m, n, m, 2)
    for method in (B.ACC, B.PLAIN):
        check_points(ctx, X, Y, "sqeuclid", a, b, 5e-2, method=method, scale=True)


def test_point_solve_host_matches_device(ctx):
    X, Y, a, b = sqeuclid_points(8, 210, 190, 3)
    eps = 1e-2
    f1, g1, r1 = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, eps, 1e-6, B.ACC, True)
    f2 = np.empty(210)
    g2 = np.empty(190)
    p = B.default_params(eps=eps, tol=1e-6)
    res = ctx.accsink_solve_host(None, a, b, p, f2, g2, scale_to_max=True, X=X, Y=Y,
                                 kind="sqeuclid")
    assert res.status == 0
    assert res.sinkhorn_steps == r1["sinkhorn_steps"]
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(g1, g2)


def test_point_graph_and_host_loop_agree(ctx):
    X, Y, a, b = sqeuclid_points(12, 140, 260, 3)
    out = []
    for use_graph in (1, 0):
        f, g, res = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, 1e-6, B.ACC, True,
                                     use_graph=use_graph)
        assert res["loop_mode"] == use_graph
        out.append((f, g, res["sinkhorn_steps"]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_point_and_dense_problems_alternate_on_one_context(ctx):
    """A dense solve between two point solves leaves both paths' results
    unchanged (workspaces and cached graphs are told apart)."""
    X, Y, a, b = sqeuclid_points(14, 120, 100, 3)
    first = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, 1e-6, B.ACC, True)
    C = W.sqeuclid_cost_fp32(X, Y)
    f = torch.empty(120, dtype=torch.float64, device=DEV)
    g = torch.empty(100, dtype=torch.float64, device=DEV)
    ctx.accsink_solve(B.problem_dense(to_dev(C), to_dev(a), to_dev(b), True),
                      B.default_params(eps=1e-2, tol=1e-6), f, g)
    second = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, 1e-6, B.ACC, True)
    np.testing.assert_array_equal(first[0], second[0])
    np.testing.assert_array_equal(first[1], second[1])


def test_point_inputs_are_validated(ctx):
    X, Y, a, b = sqeuclid_points(3, 20, 30, 3)
    f = torch.empty(20, dtype=torch.float64, device=DEV)
    g = torch.empty(30, dtype=torch.float64, device=DEV)
    p = B.default_params(eps=1e-2)
    bad = X.copy()
    bad[4, 1] = np.nan
    with pytest.raises(B.AccsinkError) as e:
        ctx.accsink_solve(B.problem_points(to_dev(bad), to_dev(Y), "sqeuclid", to_dev(a),
                                           to_dev(b)), p, f, g)
    assert e.value.code == B.ERR_NONFINITE
    pr = B.problem_points(to_dev(X), to_dev(Y), "sqeuclid", to_dev(a), to_dev(b))
    pr.d = 65
    with pytest.raises(B.AccsinkError) as e:
        ctx.accsink_solve(pr, p, f, g)
    assert e.value.code == B.ERR_INVALID_ARG
    pr = B.problem_points(to_dev(X), to_dev(Y), "sqeuclid", to_dev(a), to_dev(b))
    pr.cost_kind = 7
    with pytest.raises(B.AccsinkError) as e:
        ctx.accsink_row_pass(pr, 1e-2, g, f)
    assert e.value.code == B.ERR_INVALID_ARG
    # the context still solves afterwards
    check_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, scale=True)


# ------------------------------------- colour-transfer shape, full size --

@pytest.fixture(scope="module")
def colour_problem():
    return W.color_transfer_problem(seed=0, n=65536, eps=1e-3)


def test_full_size_colour_transfer_solve(ctx, colour_problem):
    """n = m = 65536 RGB points, eps 1e-3, tol 1e-6 (cost scaled to max 1), the
    point-cloud workload's size: converged, and the FP64 truth of eq. l1tol at
    the returned potentials, every row and every column of the 4.3e9-entry
    plan summed by the oracle, is below tol."""
    pr = colour_problem
    eps, tol = pr["eps"], pr["tol"]
    f, g, res = gpu_solve_points(ctx, pr["X"], pr["Y"], "sqeuclid", pr["a"], pr["b"], eps,
                                 tol, B.ACC, True)
    assert res["status"] == 0 and res["marginal_l1"] < stop_tol(tol), res
    cost = O.Cost(X=pr["X"], Y=pr["Y"], kind="sqeuclid", scale_to_max=True)
    ev = O.marginal_l1(cost, eps, pr["a"], pr["b"], f, g)
    check_truth(ev, tol)


# ------------------------------------------------------------ export --

@pytest.mark.parametrize("kind,scale", [("dense", False), ("sqeuclid", True), ("cosine", False)])
def test_plan_and_barycentric_match_oracle(ctx, kind, scale):
    n, m, d, eps = 150, 97, 5, 2e-2
    g0 = np.random.default_rng(91)
    if kind == "dense":
        C = g0.random((n, m)).astype(np.float32)
        prob = B.problem_dense(to_dev(C), None, None, scale)
        cost = O.Cost(C=C, scale_to_max=scale)
        a, b = W.dirichlet1(g0, n), W.dirichlet1(g0, m)
    else:
        X, Y, a, b = points_for(kind, 92, n, m, d)
        prob = B.problem_points(to_dev(X), to_dev(Y), kind, None, None, scale)
        cost = O.Cost(X=X, Y=Y, kind=kind, scale_to_max=scale)
    ref = O.solve(cost, a, b, eps, 1e-8)
    f, g = to_dev(ref["f"]), to_dev(ref["g"])
    P64 = torch.empty((n, m), dtype=torch.float64, device=DEV)
    ctx.accsink_plan(prob, eps, f, g, P64)
    P32 = torch.zeros((n, m + 3), dtype=torch.float32, device=DEV)[:, :m]
    ctx.accsink_plan(prob, eps, f, g, P32)
    Z = g0.standard_normal((m, 20)).astype(np.float32)
    out = torch.empty((n, 20), dtype=torch.float64, device=DEV)
    ctx.accsink_barycentric(prob, eps, f, g, to_dev(Z), out)
    torch.cuda.synchronize()
    Pref = O.plan(cost, eps, ref["f"], ref["g"])
    np.testing.assert_allclose(P64.cpu().numpy(), Pref, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(P32.cpu().numpy(), Pref.astype(np.float32), rtol=2e-7, atol=1e-37)
    np.testing.assert_allclose(P64.cpu().numpy().sum(1), ref["a"], rtol=1e-7)
    np.testing.assert_allclose(out.cpu().numpy(), O.barycentric(cost, eps, ref["f"], ref["g"], Z),
                               rtol=1e-11, atol=1e-13)


# ------------------------------------------- sorted clouds, pruned passes --
# Solves with d <= 4 sort both clouds along a space-filling curve and skip the
# slots whose terms are all below 2^-80 of their rows' sums. These sizes give
# each row dozens of slots, so most of them are skipped.

def test_pruned_colour_solve_matches_oracle(ctx):
    pr = W.color_transfer_problem(seed=1, n=4096, eps=1e-3)
    for method in (B.ACC, B.PLAIN):
        check_points(ctx, pr["X"], pr["Y"], "sqeuclid", pr["a"], pr["b"], 1e-3, 1e-6, method,
                     scale=True)


def test_pruned_solve_on_offset_clouds(ctx):
    # coordinates near 100 and an unscaled cost: the exponent terms are ~1e7
    # log2 units, so the FP32 estimate's rounding (~1 unit) needs the
    # magnitude-relative margin of the skip test
    X, Y, a, b = sqeuclid_points(43, 2048, 1536, 3)
    X += np.float32(100.0)
    Y += np.float32(100.0)
    check_points(ctx, X, Y, "sqeuclid", a, b, 1e-2)


def test_pruned_cosine_solve_matches_oracle(ctx):
    X, Y, a, b = cosine_points(44, 2048, 2304, 3)
    check_points(ctx, X, Y, "cosine", a, b, 5e-3)


# ------------------------------------------------------------- precision --
# FP32 arguments (precision FP32, sorted clouds with d <= 4): the exponent
# arguments err by ~2^-22 of the terms' size k s (|x| + |y|)^2, about 1.4e-5
# log2 units here (eps = 0.1, points in the unit cube, cost scaled to max 1),
# i.e. ~1e-5 relative in every P_ij: potentials within ~1e-5 eps and a
# marginal floor of a few 1e-5.

def test_fp32_point_solves_match_oracle_at_loose_tolerance(ctx):
    pr = W.color_transfer_problem(seed=2, n=2048, eps=0.1)
    X, Y, a, b = pr["X"], pr["Y"], pr["a"], pr["b"]
    cost = O.Cost(X=X, Y=Y, kind="sqeuclid", scale_to_max=True)
    ref = O.solve(cost, a, b, 0.1, tol=1e-11)
    for method in (B.ACC, B.PLAIN):
        f, g, res = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 0.1, 1e-5, method, True,
                                     precision=B.PREC_FP32)
        assert res["status"] == 0, res
        sh = g.mean() - ref["g"].mean()
        dpot = max(np.abs(g - sh - ref["g"]).max(), np.abs(f + sh - ref["f"]).max())
        assert dpot <= 1e-4 * 0.1, dpot
        ev = O.evaluate(cost, 0.1, ref["a"], ref["b"], f, g)
        assert ev["col_l1"] <= 5e-5 and ev["row_l1"] <= 5e-5, ev


def test_df32_is_the_default_precision(ctx):
    X, Y, a, b = sqeuclid_points(45, 700, 650, 3)
    f0, g0, r0 = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, 1e-6, B.ACC, True)
    f1, g1, r1 = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, 1e-6, B.ACC, True,
                                  precision=B.PREC_DF32)
    assert r0["sinkhorn_steps"] == r1["sinkhorn_steps"]
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(g0, g1)
    with pytest.raises(B.AccsinkError):
        gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, 1e-2, 1e-6, B.ACC, True, precision=3)


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
def test_pruned_solves_repeat_bit_for_bit(ctx, eps):
    """The 333 x 200 squared-Euclidean solves (d = 3: sorted clouds, pruned
    slots) run 20 times give bit-identical potentials and step counts: the
    skip decision reads only the lane's own registers and a warp-wide vote
    that every lane reaches, so nothing in it depends on scheduling."""
    n, m, d = 333, 200, 3
    X, Y, a, b = sqeuclid_points(n * 3 + m + d, n, m, d)
    f0, g0, r0 = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, eps, 1e-6, B.ACC, True)
    assert r0["status"] == 0, r0
    for _ in range(19):
        f1, g1, r1 = gpu_solve_points(ctx, X, Y, "sqeuclid", a, b, eps, 1e-6, B.ACC, True)
        assert r1["sinkhorn_steps"] == r0["sinkhorn_steps"]
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(g1, g0)
