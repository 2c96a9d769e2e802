"""GPU parity of the batched solver (many problems, one persistent launch)
against the FP64 oracle, problem by problem.

Each problem of a batch must meet the single-solve tolerances: potentials
within 1e-3 eps max-abs after centring (at the same iterate), <C,P> within
1e-5 relative, steps within 2% (or one step), and the FP64 truth of Sec. 5
eq. l1tol (row plus column L1) below tol. The work split (whole-problem items
or row / column tiles) must not change any potential. Large dense problems
(and a batch's only problem when it is dense) are solved one at a time by the
single-solve path: their potentials are those of accsink_solve bit for bit.
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


class Prob:
    """One host problem plus its device tensors and oracle cost."""

    def __init__(self, kind, n, m, seed, eps, d=3, scale=False, method=B.ACC, tol=1e-6,
                 spread=1.0, **kw):
        g = np.random.default_rng(seed)
        self.kind, self.eps, self.tol, self.method, self.scale, self.kw = kind, eps, tol, method, scale, kw
        if kind == "dense":
            self.C = (spread * g.random((n, m))).astype(np.float32)
            self.cost = O.Cost(C=self.C, scale_to_max=scale)
        elif kind == "sqeuclid":
            self.X = (spread * g.random((n, d))).astype(np.float32)
            self.Y = (spread * g.random((m, d))).astype(np.float32)
            self.cost = O.Cost(X=self.X, Y=self.Y, kind="sqeuclid", scale_to_max=scale)
        else:
            self.X = W.unit_gaussian_points(g, n, d)
            self.Y = W.unit_gaussian_points(g, m, d)
            self.cost = O.Cost(X=self.X, Y=self.Y, kind="cosine", scale_to_max=scale)
        self.a = W.dirichlet1(g, n)
        self.b = W.dirichlet1(g, m)
        self.n, self.m = n, m

    def struct(self):
        if self.kind == "dense":
            return B.problem_dense(to_dev(self.C), to_dev(self.a), to_dev(self.b), self.scale)
        return B.problem_points(to_dev(self.X), to_dev(self.Y), self.kind, to_dev(self.a),
                                to_dev(self.b), self.scale)

    def params(self):
        return B.default_params(eps=self.eps, tol=self.tol, method=self.method, **self.kw)


def run_batch(ctx, probs):
    structs = [p.struct() for p in probs]
    params = [p.params() for p in probs]
    fs = [torch.empty(p.n, dtype=torch.float64, device=DEV) for p in probs]
    gs = [torch.empty(p.m, dtype=torch.float64, device=DEV) for p in probs]
    res = ctx.accsink_solve_batch(structs, params, fs, gs)
    torch.cuda.synchronize()
    return [f.cpu().numpy() for f in fs], [g.cpu().numpy() for g in gs], \
        [B.result_dict(r) for r in res]


def check_against_oracle(p, f, g, res, cost=None):
    cost = cost or p.cost
    okw = dict(method=O.ACC if p.method == B.ACC else O.PLAIN,
               carry_y=p.kw.get("carry", B.CARRY_Y) == B.CARRY_Y,
               stability=p.kw.get("stability", B.STAB_REPORT))
    ref = O.solve(cost, p.a, p.b, p.eps, stop_tol(p.tol), **okw)
    assert res["status"] == 0, res
    assert ref["status"] == O.CONVERGED
    rs, gs_ = ref["sinkhorn_steps"], res["sinkhorn_steps"]
    check_steps(cost, p.a, p.b, p.eps, p.tol, okw, rs, gs_)
    ref = same_iterate(cost, p.a, p.b, p.eps, okw, ref, gs_)
    sh = g.mean() - ref["g"].mean()
    dpot = max(np.abs(g - sh - ref["g"]).max(), np.abs(f + sh - ref["f"]).max())
    assert dpot <= 1e-3 * p.eps, dpot
    ev = O.evaluate(cost, p.eps, ref["a"], ref["b"], f, g)
    check_truth(ev, p.tol)
    evr = O.evaluate(cost, p.eps, ref["a"], ref["b"], ref["f"], ref["g"])
    assert abs(res["transport_cost"] - evr["transport_cost"]) <= \
        1e-5 * abs(evr["transport_cost"]), (res["transport_cost"], evr["transport_cost"])
    assert abs(res["dual_objective"] - ref["dual"]) <= 1e-5 * max(1e-3, abs(ref["dual"]))


def mixed_problems():
    return [
        Prob("dense", 1, 1, 1, 5e-2),
        Prob("dense", 1, 9, 2, 5e-2),
        Prob("dense", 9, 1, 3, 5e-2, method=B.PLAIN),
        Prob("dense", 37, 129, 4, 1e-2),
        Prob("sqeuclid", 200, 333, 5, 1e-3, d=3, scale=True),
        Prob("sqeuclid", 513, 257, 6, 1e-2, d=2, scale=True, method=B.PLAIN),
        Prob("cosine", 129, 250, 7, 2e-2, d=40),
        Prob("cosine", 300, 161, 8, 5e-3, d=17),
        Prob("dense", 150, 120, 9, 1e-2, scale=True, spread=3.5),
        Prob("sqeuclid", 64, 1031, 10, 1e-1, d=5, scale=True, stability=B.STAB_GATE),
        Prob("dense", 257, 300, 11, 1e-2, carry=B.CARRY_W),
        Prob("sqeuclid", 150, 170, 12, 0.5, d=3, spread=4.0),
        Prob("dense", 120, 100, 13, 1e-2, stability=B.STAB_BACKTRACK),
    ]


def test_mixed_batch_matches_oracle(ctx):
    """Dense, squared-Euclidean and cosine problems of ragged sizes, each with
    its own eps, method and modes, solved whole by one CTA each."""
    ctx.accsink_batch_set_config()          # defaults: all of these are small
    probs = mixed_problems()
    fs, gs, rs = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, fs, gs, rs):
        assert r["loop_mode"] == 2
        check_against_oracle(p, f, g, r)


def test_tiled_work_split_gives_identical_potentials(ctx):
    """Row and column tiles (many CTAs per problem, phase hand-offs through
    the queue) give the same potentials and steps as whole-problem items."""
    probs = mixed_problems()
    ctx.accsink_batch_set_config()
    f1, g1, r1 = run_batch(ctx, probs)
    ctx.accsink_batch_set_config(small_max_nm=64, row_tile_elems=700)
    try:
        f2, g2, r2 = run_batch(ctx, probs)
    finally:
        ctx.accsink_batch_set_config()
    for k in range(len(probs)):
        assert r1[k]["sinkhorn_steps"] == r2[k]["sinkhorn_steps"], k
        np.testing.assert_array_equal(f1[k], f2[k])
        np.testing.assert_array_equal(g1[k], g2[k])
        assert abs(r1[k]["dual_objective"] - r2[k]["dual_objective"]) <= \
            1e-12 * max(1.0, abs(r1[k]["dual_objective"]))
        assert abs(r1[k]["transport_cost"] - r2[k]["transport_cost"]) <= \
            1e-9 * abs(r1[k]["transport_cost"])


def test_tiled_batch_matches_oracle(ctx):
    ctx.accsink_batch_set_config(small_max_nm=1000, row_tile_elems=4096)
    try:
        probs = mixed_problems()[3:8]
        fs, gs, rs = run_batch(ctx, probs)
    finally:
        ctx.accsink_batch_set_config()
    for p, f, g, r in zip(probs, fs, gs, rs):
        check_against_oracle(p, f, g, r)


def test_batch_of_one_equals_batch_member(ctx):
    """A problem's result does not depend on the rest of its batch."""
    probs = mixed_problems()
    fs, gs, rs = run_batch(ctx, probs)
    for k in (4, 7):
        f1, g1, r1 = run_batch(ctx, [probs[k]])
        np.testing.assert_array_equal(f1[0], fs[k])
        np.testing.assert_array_equal(g1[0], gs[k])
        assert r1[0]["sinkhorn_steps"] == rs[k]["sinkhorn_steps"]


def large_problems():
    # m = 777 and 1029 leave the last 128-column group partly empty
    return [Prob("sqeuclid", 1100, 1000, 31, 1e-2, d=3, scale=True),
            Prob("cosine", 1500, 777, 32, 2e-2, d=24),
            Prob("dense", 1031, 1029, 33, 5e-3, scale=True)]


def test_large_problems_use_the_transposed_column_pass(ctx):
    """Problems from 2^20 entries keep K^T too and run the column phase as
    row tiles over it; parity with the oracle, and identical potentials for
    two work splits."""
    probs = large_problems()
    ctx.accsink_batch_set_config()
    # leave non-zero values in the workspace first (a larger batch of others)
    run_batch(ctx, mixed_problems() + large_problems()[::-1])
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


def test_word_alignment_shaped_batch(ctx):
    """24 cosine problems with unit-norm Gaussian points in R^300, n, m
    log-uniform in [16, 512], eps in [0.005, 0.05] (the oracle reads the cost
    formed once in FP64)."""
    batch = W.word_alignment_batch(seed=3, count=24, lo=16, hi=512, d=300)
    probs = []
    for k, pr in enumerate(batch):
        p = Prob.__new__(Prob)
        p.kind, p.eps, p.tol, p.method, p.scale, p.kw = "cosine", pr["eps"], 1e-6, B.ACC, False, {}
        p.X, p.Y, p.a, p.b = pr["X"], pr["Y"], pr["a"], pr["b"]
        p.n, p.m = p.X.shape[0], p.Y.shape[0]
        p.cost = O.Cost(X=p.X, Y=p.Y, kind="cosine").materialised()
        probs.append(p)
    fs, gs, rs = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, fs, gs, rs):
        check_against_oracle(p, f, g, r)


def test_bad_problem_fails_alone(ctx):
    probs = mixed_problems()[:6]
    bad = Prob("sqeuclid", 40, 50, 99, 1e-2, d=3)
    bad.X = bad.X.copy()
    bad.X[3, 1] = np.nan
    zero = Prob("dense", 20, 30, 98, 1e-2)
    zero.b = zero.b.copy()
    zero.b[4] = 0.0
    probs = probs[:3] + [bad] + probs[3:] + [zero]
    structs = [p.struct() for p in probs]
    params = [p.params() for p in probs]
    fs = [torch.empty(p.n, dtype=torch.float64, device=DEV) for p in probs]
    gs = [torch.empty(p.m, dtype=torch.float64, device=DEV) for p in probs]
    with pytest.raises(B.AccsinkError) as e:
        ctx.accsink_solve_batch(structs, params, fs, gs)
    assert e.value.code in (B.ERR_NONFINITE, B.ERR_NONPOSITIVE_MARGINAL)
    # the other problems were still solved: rerun just them and compare
    good = [p for p in probs if p is not bad and p is not zero]
    f1, g1, r1 = run_batch(ctx, good)
    for p, f, g, r in zip(good, f1, g1, r1):
        assert r["status"] == 0


def test_bad_problem_statuses_are_reported(ctx):
    import ctypes as ct
    bad = Prob("sqeuclid", 40, 50, 99, 1e-2, d=3)
    bad.X = bad.X.copy()
    bad.X[3, 1] = np.inf
    ok = Prob("dense", 30, 20, 97, 1e-2)
    probs = [ok, bad]
    k, pa, qa, fa, ga, ra = B.Context._batch_arrays(
        [p.struct() for p in probs], [p.params() for p in probs],
        [torch.empty(p.n, dtype=torch.float64, device=DEV) for p in probs],
        [torch.empty(p.m, dtype=torch.float64, device=DEV) for p in probs])
    rc = B.lib().accsink_solve_batch(ctx._h, k, pa, qa, None, fa, ga, ra)
    assert rc == B.ERR_NONFINITE
    assert ra[0].status == 0 and ra[1].status == B.ERR_NONFINITE


def test_empty_batch_and_invalid_arguments(ctx):
    assert ctx.accsink_solve_batch([], [], [], []) == []
    p = Prob("dense", 5, 6, 1, 1e-2)
    s = p.struct()
    s.n = 0
    with pytest.raises(B.AccsinkError) as e:
        ctx.accsink_solve_batch([s], [p.params()], [torch.empty(5, dtype=torch.float64,
                                                                 device=DEV)],
                                [torch.empty(6, dtype=torch.float64, device=DEV)])
    assert e.value.code == B.ERR_INVALID_ARG
    q = Prob("cosine", 5, 6, 1, 1e-2, d=8)
    s = q.struct()
    s.d = 5000
    with pytest.raises(B.AccsinkError) as e:
        ctx.accsink_solve_batch([s], [q.params()], [torch.empty(5, dtype=torch.float64,
                                                                 device=DEV)],
                                [torch.empty(6, dtype=torch.float64, device=DEV)])
    assert e.value.code == B.ERR_INVALID_ARG


def test_autotune_picks_a_candidate(ctx):
    probs = mixed_problems()
    structs = [p.struct() for p in probs]
    params = [p.params() for p in probs]
    fs = [torch.empty(p.n, dtype=torch.float64, device=DEV) for p in probs]
    gs = [torch.empty(p.m, dtype=torch.float64, device=DEV) for p in probs]
    best, times = ctx.accsink_batch_autotune(structs, params, fs, gs)
    assert len(times) == 18 and all(t > 0 for t in times)
    assert ctx.accsink_batch_get_config() == best
    ctx.accsink_batch_set_config()


def split_step_problems():
    # m >= 4096 and tiled: the step's P2 and update loops run as work items;
    # the first keeps K^T (n m >= 2^20), the second sweeps column tiles of K
    return [Prob("sqeuclid", 300, 4200, 41, 1e-2, d=3, scale=True),
            Prob("cosine", 200, 4100, 42, 2e-2, d=24),
            Prob("dense", 150, 4099, 43, 1e-2, method=B.PLAIN)]


def test_split_step_matches_oracle(ctx):
    probs = split_step_problems()
    fs, gs, rs = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, fs, gs, rs):
        check_against_oracle(p, f, g, r)


def test_large_dimension_points_match_oracle(ctx):
    """Point clouds above the tensor-core range and at the dimension limit
    (d = 481 and 4096) form their costs with the CUDA-core expansion; each
    problem meets the oracle."""
    probs = [Prob("cosine", 40, 37, 71, 1e-2, d=481),
             Prob("sqeuclid", 20, 30, 72, 1e-2, d=4096, scale=True),
             Prob("cosine", 25, 50, 73, 2e-2, d=4096)]
    fs, gs, rs = run_batch(ctx, probs)
    for p, f, g, r in zip(probs, fs, gs, rs):
        assert r["loop_mode"] == 2
        check_against_oracle(p, f, g, r)


def test_graph_replay_equals_direct_launches(ctx):
    """The batch's launch sequence replayed as a CUDA graph (the default; the
    second run updates the executable graph in place, a batch of another
    shape re-instantiates it) gives the potentials of the same sequence
    issued directly, bit for bit."""
    import os
    probs = mixed_problems() + large_problems()[:2]
    f1, g1, r1 = run_batch(ctx, probs)
    run_batch(ctx, probs[:5])
    f2, g2, r2 = run_batch(ctx, probs)
    os.environ["ACCSINK_BATCH_GRAPH"] = "0"
    try:
        f3, g3, r3 = run_batch(ctx, probs)
    finally:
        del os.environ["ACCSINK_BATCH_GRAPH"]
    for k in range(len(probs)):
        for f, g, r in ((f2, g2, r2), (f3, g3, r3)):
            assert r[k]["sinkhorn_steps"] == r1[k]["sinkhorn_steps"], k
            np.testing.assert_array_equal(f[k], f1[k])
            np.testing.assert_array_equal(g[k], g1[k])
    t = ctx.accsink_batch_last_timing()
    assert t["total_ms"] >= t["form_ms"] > 0.0


def test_wide_batch_keeps_each_problems_potentials(ctx):
    """A batch whose tiled problems have row items enough for the resident
    CTAs gives every row item four rows per warp (40 problems of 1000 rows:
    1280 items of 32 rows against 608 CTAs); a problem's potentials are
    those it gets in a small batch (8-row items), bit for bit, and match the
    oracle."""
    probs = [Prob("sqeuclid", 1000, 100 + 3 * k, 60 + k, 1e-2, d=3, scale=True)
             for k in range(40)]
    f1, g1, r1 = run_batch(ctx, probs)
    for k in (0, 17, 39):
        f2, g2, r2 = run_batch(ctx, [probs[k], probs[(k + 1) % 40]])
        assert r2[0]["sinkhorn_steps"] == r1[k]["sinkhorn_steps"]
        np.testing.assert_array_equal(f2[0], f1[k])
        np.testing.assert_array_equal(g2[0], g1[k])
    for k in (0, 39):
        check_against_oracle(probs[k], f1[k], g1[k], r1[k])


def test_split_step_equals_one_cta_step(ctx):
    """The step's column loops as work items give the potentials of the
    one-CTA step bit for bit (only the order of Theorem 4's P2 sum differs,
    which feeds the stability report alone)."""
    import os
    probs = split_step_problems()
    f1, g1, r1 = run_batch(ctx, probs)
    os.environ["ACCSINK_BATCH_STEP_ITEMS"] = "0"
    try:
        f2, g2, r2 = run_batch(ctx, probs)
    finally:
        del os.environ["ACCSINK_BATCH_STEP_ITEMS"]
    for k in range(len(probs)):
        assert r1[k]["sinkhorn_steps"] == r2[k]["sinkhorn_steps"], k
        np.testing.assert_array_equal(f1[k], f2[k])
        np.testing.assert_array_equal(g1[k], g2[k])
        assert abs(r1[k]["stability_failures"] - r2[k]["stability_failures"]) <= 1


def test_full_word_alignment_batch_meets_tol_in_fp64_truth(ctx):
    """The batch the benchmark times (512 cosine problems, unit-norm Gaussian
    points in R^300, n, m log-uniform in [16, 2048], eps in [0.005, 0.05]) in
    one launch with the autotuner's usual split: every problem converges and
    the FP64 truth of Sec. 5 eq. l1tol at its potentials (every row and column
    of its plan, the cost formed in FP64 from the points) is below tol."""
    batch = W.word_alignment_batch(seed=0, count=512)
    probs = []
    for pr in batch:
        p = Prob.__new__(Prob)
        p.kind, p.eps, p.tol, p.method, p.scale, p.kw = "cosine", pr["eps"], 1e-6, B.ACC, False, {}
        p.X, p.Y, p.a, p.b = pr["X"], pr["Y"], pr["a"], pr["b"]
        p.n, p.m = p.X.shape[0], p.Y.shape[0]
        probs.append(p)
    ctx.accsink_batch_set_config(row_tile_elems=16384)
    try:
        fs, gs, rs = run_batch(ctx, probs)
    finally:
        ctx.accsink_batch_set_config()
    worst = 0.0
    for p, f, g, r in zip(probs, fs, gs, rs):
        assert r["status"] == 0, r
        cost = O.Cost(X=p.X, Y=p.Y, kind="cosine")
        ev = O.marginal_l1(cost, p.eps, O.normalise(p.a), O.normalise(p.b), f, g)
        check_truth(ev, p.tol)
        worst = max(worst, ev["row_l1"] + ev["col_l1"])
    assert worst < 1e-6


def single_solve(ctx, p):
    f = torch.empty(p.n, dtype=torch.float64, device=DEV)
    g = torch.empty(p.m, dtype=torch.float64, device=DEV)
    q = p.params()
    q.use_graph = 1
    r = ctx.accsink_solve(p.struct(), q, f, g)
    torch.cuda.synchronize()
    return f.cpu().numpy(), g.cpu().numpy(), B.result_dict(r)


def test_large_dense_problems_take_the_single_solve_path(ctx):
    """Dense problems from dense_solo_min_nm entries on run one at a time by
    the single-solve path (loop_mode 1, potentials of accsink_solve bit for
    bit, parity with the oracle); the rest of the batch stays in the batched
    launch (loop_mode 2) with its usual results."""
    big = [Prob("dense", 300, 400, 51, 1e-2, scale=True),
           Prob("dense", 257, 513, 52, 5e-3, method=B.PLAIN)]
    rest = mixed_problems()[3:8]
    probs = rest[:2] + [big[0]] + rest[2:] + [big[1]]
    ctx.accsink_batch_set_config(dense_solo_min_nm=100000)
    try:
        assert ctx.accsink_batch_get_config()["dense_solo_min_nm"] == 100000
        fs, gs, rs = run_batch(ctx, probs)
        t = ctx.accsink_batch_last_timing()
    finally:
        ctx.accsink_batch_set_config()
    assert ctx.accsink_batch_get_config()["dense_solo_min_nm"] == 1 << 24
    solo_ms = 0.0
    for p, f, g, r in zip(probs, fs, gs, rs):
        check_against_oracle(p, f, g, r)
        if p in big:
            assert r["loop_mode"] == 1, r
            f1, g1, r1 = single_solve(ctx, p)
            np.testing.assert_array_equal(f, f1)
            np.testing.assert_array_equal(g, g1)
            assert r["sinkhorn_steps"] == r1["sinkhorn_steps"]
            solo_ms += r["gpu_ms"]
        else:
            assert r["loop_mode"] == 2, r
    assert t["total_ms"] >= solo_ms > 0.0
    # the batched members' results do not depend on the routed ones
    f2, g2, r2 = run_batch(ctx, rest)
    for k, p in enumerate(rest):
        j = probs.index(p)
        np.testing.assert_array_equal(fs[j], f2[k])
        np.testing.assert_array_equal(gs[j], g2[k])


def test_lone_dense_problem_takes_the_single_solve_path(ctx):
    """A batch of one dense problem is solved by the single-solve path at any
    size; with dense_solo_min_nm < 0 it stays in the batched launch, and both
    meet the oracle."""
    p = Prob("dense", 150, 120, 9, 1e-2, scale=True, spread=3.5)
    f, g, r = run_batch(ctx, [p])
    assert r[0]["loop_mode"] == 1
    f1, g1, _ = single_solve(ctx, p)
    np.testing.assert_array_equal(f[0], f1)
    np.testing.assert_array_equal(g[0], g1)
    check_against_oracle(p, f[0], g[0], r[0])
    ctx.accsink_batch_set_config(dense_solo_min_nm=-1)
    try:
        f2, g2, r2 = run_batch(ctx, [p])
    finally:
        ctx.accsink_batch_set_config()
    assert r2[0]["loop_mode"] == 2
    check_against_oracle(p, f2[0], g2[0], r2[0])
    # a lone point-cloud problem stays in the batched launch
    q = mixed_problems()[4]
    _, _, r3 = run_batch(ctx, [q])
    assert r3[0]["loop_mode"] == 2
    # the autotuner on a batch whose only problem leaves the batched launch:
    # solved once, nothing left to time, the outputs still the single solve's
    fa = torch.empty(p.n, dtype=torch.float64, device=DEV)
    ga = torch.empty(p.m, dtype=torch.float64, device=DEV)
    best, times = ctx.accsink_batch_autotune([p.struct()], [p.params()], [fa], [ga])
    torch.cuda.synchronize()
    assert len(times) == 18 and all(t == 0.0 for t in times)
    np.testing.assert_array_equal(fa.cpu().numpy(), f1)
    np.testing.assert_array_equal(ga.cpu().numpy(), g1)
    ctx.accsink_batch_set_config()
