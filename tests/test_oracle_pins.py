"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks one part of the oracle against a library routine, a closed
form, brute force or an invariant stated in the paper, chosen so that a
dropped term, a wrong sign, a wrong index or a transposed operand in the
oracle fails at least one of them. CPU only.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.special import logsumexp

import oracle as O
from paper_2605_30267_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(seed, n, m, scale=1.0):
    g = np.random.default_rng(seed)
    C = (scale * g.random((n, m))).astype(np.float32)
    a = g.random(n) + 0.1
    b = g.random(m) + 0.1
    return C, a / a.sum(), b / b.sum()


def _plan(C64, f, g, eps):
    return np.exp((f[:, None] + g[None, :] - C64) / eps)


# --------------------------------------------------------------------------
# Row and column passes (Sec. 2 u/v-updates) against scipy's logsumexp.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,eps", [(7, 13, 0.3), (33, 5, 0.05), (64, 64, 1e-3)])
def test_row_pass_is_log_a_minus_logsumexp(n, m, eps):
    C, a, b = _rand_problem(1, n, m)
    x = np.random.default_rng(2).standard_normal(m) * 3
    cost = O.Cost(C=C)
    u = O.row_pass(cost, eps, np.log(a), x)
    ref = np.log(a) - logsumexp(x[None, :] - C.astype(np.float64) / eps, axis=1)
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * max(1, np.abs(ref).max()))


@pytest.mark.parametrize("n,m,eps", [(7, 13, 0.3), (33, 5, 0.05), (64, 64, 1e-3)])
def test_col_lse_is_logsumexp_over_rows(n, m, eps):
    C, a, b = _rand_problem(3, n, m)
    u = np.random.default_rng(4).standard_normal(n) * 3
    cost = O.Cost(C=C)
    ell = O.col_lse(cost, eps, u)
    ref = logsumexp(u[:, None] - C.astype(np.float64) / eps, axis=0)
    np.testing.assert_allclose(ell, ref, rtol=0, atol=1e-12 * max(1, np.abs(ref).max()))


def test_row_pass_brute_force_without_shift():
    # At eps = 1 and small values the plain sum needs no max-shift.
    C, a, b = _rand_problem(5, 6, 9)
    x = np.linspace(-1, 1, 9)
    u = O.row_pass(O.Cost(C=C), 1.0, np.log(a), x)
    for i in range(6):
        s = sum(math.exp(x[j] - float(C[i, j])) for j in range(9))
        assert abs(u[i] - (math.log(a[i]) - math.log(s))) < 1e-13


def test_sinkhorn_map_is_centred_v_update():
    C, a, b = _rand_problem(6, 11, 17)
    eps = 0.2
    x = np.random.default_rng(7).standard_normal(17)
    x -= x.mean()
    err, u, c, s = O.sinkhorn_map(O.Cost(C=C), eps, a, b, x)
    C64 = C.astype(np.float64)
    P = np.exp(u[:, None] + x[None, :] - C64 / eps)
    np.testing.assert_allclose(P.sum(1), a, rtol=1e-12)       # row pass exact
    np.testing.assert_allclose(c, P.sum(0), rtol=1e-12)        # column sums
    assert abs(err - np.abs(P.sum(0) - b).sum()) < 1e-13       # eq. l1tol
    raw = x + np.log(b / P.sum(0))                             # eq. v-update
    np.testing.assert_allclose(s, raw - raw.mean(), atol=1e-12)
    assert abs(s.mean()) < 1e-13                               # in N-perp


def test_sinkhorn_map_gauge_invariant():
    # f(v + c1) = f(v) (Sec. 3): shifting x by a constant changes nothing.
    C, a, b = _rand_problem(8, 9, 12)
    x = np.random.default_rng(9).standard_normal(12)
    r1 = O.sinkhorn_map(O.Cost(C=C), 0.1, a, b, x)
    r2 = O.sinkhorn_map(O.Cost(C=C), 0.1, a, b, x + 3.7)
    assert abs(r1[0] - r2[0]) < 1e-12
    np.testing.assert_allclose(r1[3], r2[3], atol=1e-11)
    np.testing.assert_allclose(r1[1], r2[1] + 3.7, atol=1e-11)


# --------------------------------------------------------------------------
# Whole solves against closed forms.
# --------------------------------------------------------------------------

def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


def _two_by_two_p11(C, a1, b1, eps):
    # P11 P22 / (P12 P21) = K with K = exp(-(C11+C22-C12-C21)/eps); with
    # P12 = a1-p, P21 = b1-p, P22 = 1-a1-b1+p this is a quadratic in p.
    K = math.exp(-(C[0][0] + C[1][1] - C[0][1] - C[1][0]) / eps)
    A = 1.0 - K
    B = (1.0 - a1 - b1) + K * (a1 + b1)
    Cq = -K * a1 * b1
    if abs(A) < 1e-15:
        return -Cq / B
    disc = math.sqrt(B * B - 4 * A * Cq)
    for p in ((-B + disc) / (2 * A), (-B - disc) / (2 * A)):
        if 0 < p < min(a1, b1) and 1 - a1 - b1 + p > 0:
            return p
    raise AssertionError("no feasible root")


@pytest.mark.parametrize("method", [O.PLAIN, O.ACC])
def test_two_by_two_golden(method):
    eps, c11, c12, c21, c22, a1, b1, p11 = _golden_rows("two_by_two.txt")[0]
    C = np.array([[c11, c12], [c21, c22]], np.float32)
    a = np.array([a1, 1 - a1]); b = np.array([b1, 1 - b1])
    r = O.solve(O.Cost(C=C), a, b, eps, tol=1e-13, method=method)
    P = _plan(C.astype(np.float64), r["f"], r["g"], eps)
    assert abs(P[0, 0] - p11) < 1e-12
    assert abs(_two_by_two_p11(C.astype(np.float64).tolist(), a1, b1, eps) - p11) < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("method", [O.PLAIN, O.ACC])
def test_two_by_two_random_closed_form(seed, method):
    g = np.random.default_rng(seed)
    C = g.random((2, 2)).astype(np.float32)
    a1, b1 = g.uniform(0.2, 0.8, 2)
    eps = [0.5, 0.1, 0.03][seed]
    r = O.solve(O.Cost(C=C), [a1, 1 - a1], [b1, 1 - b1], eps, tol=1e-12, method=method)
    P = _plan(C.astype(np.float64), r["f"], r["g"], eps)
    p = _two_by_two_p11(C.astype(np.float64).tolist(), a1, b1, eps)
    assert abs(P[0, 0] - p) < 1e-10
    assert abs(P[0, 1] - (a1 - p)) < 1e-10
    assert abs(P[1, 0] - (b1 - p)) < 1e-10


@pytest.mark.parametrize("method", [O.PLAIN, O.ACC])
def test_separable_cost_gives_product_plan(method):
    # C_ij = r_i + s_j  =>  P = a b' exactly (the cost only shifts the gauge).
    g = np.random.default_rng(11)
    n, m = 13, 7
    # dyadic r_i, s_j (multiples of 2^-10) so that r_i + s_j is exact in FP32
    r_ = g.integers(0, 1024, n) / 1024.0
    s_ = g.integers(0, 1024, m) / 1024.0
    C = (r_[:, None] + s_[None, :]).astype(np.float32)
    assert np.array_equal(C.astype(np.float64), r_[:, None] + s_[None, :])
    a, b = W.dirichlet1(g, n), W.dirichlet1(g, m)
    eps = 0.05
    res = O.solve(O.Cost(C=C), a, b, eps, tol=1e-12, method=method)
    P = _plan(C.astype(np.float64), res["f"], res["g"], eps)
    np.testing.assert_allclose(P, np.outer(a, b), rtol=1e-9, atol=1e-14)
    if method == O.PLAIN:
        # x_0 = 0 then one v-update reaches the fixed point.
        assert res["sinkhorn_steps"] <= 2


@pytest.mark.parametrize("method", [O.PLAIN, O.ACC])
def test_symmetric_cost_equal_marginals_symmetric_plan(method):
    g = np.random.default_rng(12)
    n = 15
    M = g.random((n, n))
    C = ((M + M.T) / 2).astype(np.float32)
    a = W.dirichlet1(g, n)
    eps = 0.05
    res = O.solve(O.Cost(C=C), a, a, eps, tol=1e-12, method=method)
    P = _plan(C.astype(np.float64), res["f"], res["g"], eps)
    np.testing.assert_allclose(P, P.T, atol=1e-12)
    # P_ij = P_ji forces f_i - g_i to be the same constant for every i
    d = res["f"] - res["g"]
    assert np.ptp(d) < 1e-9


def test_one_row_and_one_column_problems():
    g = np.random.default_rng(13)
    C = g.random((1, 9)).astype(np.float32)
    b = W.dirichlet1(g, 9)
    r = O.solve(O.Cost(C=C), [1.0], b, 0.1, tol=1e-14, method=O.PLAIN)
    P = _plan(C.astype(np.float64), r["f"], r["g"], 0.1)
    np.testing.assert_allclose(P[0], b, rtol=1e-12)
    assert r["sinkhorn_steps"] == 2          # one v-update makes P = b exactly
    C = g.random((9, 1)).astype(np.float32)
    a = W.dirichlet1(g, 9)
    r = O.solve(O.Cost(C=C), a, [1.0], 0.1, tol=1e-14, method=O.ACC)
    assert r["sinkhorn_steps"] == 1          # the row pass alone solves it
    P = _plan(C.astype(np.float64), r["f"], r["g"], 0.1)
    np.testing.assert_allclose(P[:, 0], a, rtol=1e-12)


@pytest.mark.parametrize("eps", [0.05, 0.02, 0.01])
def test_small_eps_brute_force_assignment(eps):
    # 0 <= <C,P^eps> - OT <= eps log(nm) (Sec. 4 complexity discussion); OT
    # for uniform n = m marginals is attained at a permutation (Birkhoff).
    g = np.random.default_rng(21)
    n = 6
    C = g.random((n, n)).astype(np.float32)
    C64 = C.astype(np.float64)
    ot = min(sum(C64[i, s[i]] for i in range(n)) / n
             for s in itertools.permutations(range(n)))
    a = np.full(n, 1.0 / n)
    r = O.solve(O.Cost(C=C), a, a, eps, tol=1e-10, method=O.ACC)
    ev = O.evaluate(O.Cost(C=C), eps, a, a, r["f"], r["g"])
    slack = C64.max() * (ev["row_l1"] + ev["col_l1"])
    assert ev["transport_cost"] - ot >= -slack - 1e-12
    assert ev["transport_cost"] - ot <= eps * math.log(n * n) + slack


# --------------------------------------------------------------------------
# Dynamics.
# --------------------------------------------------------------------------

def test_plain_sinkhorn_dual_ascent():
    # f(v+) <= f(v) (Lemma sinkhorn-descent, App. A): the dual D = -eps f never
    # decreases along plain Sinkhorn.
    pr = W.gmm_stored_cost_problem(0, n=120, m=90, eps=1e-2, tol=1e-9)
    r = O.solve(O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"], tol=1e-9,
                method=O.PLAIN, history=100000)
    d = r["history"]["dual"]
    assert len(d) > 10
    assert np.all(np.diff(d) >= -1e-14 * np.abs(d[1:]).max())


def test_dual_after_row_pass_matches_explicit_dual():
    C, a, b = _rand_problem(14, 10, 8)
    eps = 0.1
    x = np.random.default_rng(15).standard_normal(8)
    err, u, c, s = O.sinkhorn_map(O.Cost(C=C), eps, a, b, x)
    d1 = O.dual_after_row_pass(O.Cost(C=C), eps, a, b, u, x)
    f, g = eps * u, eps * x
    P = _plan(C.astype(np.float64), f, g, eps)
    d2 = f @ a + g @ b - eps * P.sum()
    assert abs(d1 - d2) < 1e-14
    # F(u + c1, v - c1) = F(u, v) (eq. Fc)
    P2 = _plan(C.astype(np.float64), f + 0.3, g - 0.3, eps)
    assert abs((f + 0.3) @ a + (g - 0.3) @ b - eps * P2.sum() - d2) < 1e-13


@pytest.mark.parametrize("eps", [1e-1, 1e-2])
def test_plain_and_acc_reach_the_same_potentials(eps):
    pr = W.gmm_stored_cost_problem(3, n=80, m=60, eps=eps)
    cost = O.Cost(C=pr["C"])
    rp = O.solve(cost, pr["a"], pr["b"], eps, tol=1e-11, method=O.PLAIN)
    ra = O.solve(cost, pr["a"], pr["b"], eps, tol=1e-11, method=O.ACC)
    assert rp["status"] == O.CONVERGED and ra["status"] == O.CONVERGED
    for key in ("g", "f"):
        sp = rp["g"].mean()
        sa = ra["g"].mean()
        sign = -1 if key == "g" else 1
        np.testing.assert_allclose(rp[key] + sign * sp, ra[key] + sign * sa, atol=1e-6 * eps)


def _indep_S(C64, eps, a, b, x):
    """Normalised Sinkhorn map from scipy's logsumexp (independent of the oracle)."""
    u = np.log(a) - logsumexp(x[None, :] - C64 / eps, axis=1)
    ell = logsumexp(u[:, None] - C64 / eps, axis=0)
    raw = np.log(b) - ell
    return raw - raw.mean()


@pytest.mark.parametrize("carry_y", [True, False])
def test_acc_iterates_match_the_xy_scheme(carry_y):
    # Algorithm 1 (x, w) with w = alpha y must reproduce the two-sequence
    # scheme of Sec. 4, with grad phi*(grad f(x)) = x - S(x) on N-perp and
    # alpha = sqrt(2 mu), under the homotopy of Algorithm 2. carry_y=True keeps
    # y across a stage change; carry_y=False keeps w (so y jumps by
    # alpha_old / alpha_new).
    pr = W.gmm_stored_cost_problem(4, n=40, m=30, eps=5e-2)
    C64 = pr["C"].astype(np.float64)
    a, b, eps = pr["a"], pr["b"], pr["eps"]
    K = 40
    r = O.solve(O.Cost(C=pr["C"]), a, b, eps, tol=1e-300, method=O.ACC, mu0=0.25, m0=4,
                max_steps=K, history=K, keep_x=True, stability=O.STAB_OFF,
                carry_y=carry_y)
    xs = r["history"]["x"]
    x = np.zeros(30)
    y = np.zeros(30)
    mu, m_stage, j = 0.25, 4, 0
    for k in range(1, K):
        al = math.sqrt(2 * mu)
        grad_x = x - _indep_S(C64, eps, a, b, x)
        # (x_{k+1} - x_k)/al = y_k - x_{k+1} - grad/al
        x_new = (x + al * y - grad_x) / (1 + al)
        grad_new = x_new - _indep_S(C64, eps, a, b, x_new)
        # (y_{k+1} - y_k)/al = x_{k+1} - y_{k+1} - grad_new/mu
        y_new = (y + al * x_new - al / mu * grad_new) / (1 + al)
        x, y = x_new, y_new
        np.testing.assert_allclose(xs[k], x, atol=1e-9 * max(1, np.abs(x).max()))
        j += 1
        if j == m_stage:
            mu /= 2
            m_stage = int(math.floor(math.sqrt(2) * m_stage)) + 1
            j = 0
            if not carry_y:
                y *= al / math.sqrt(2 * mu)


def test_acc_fixed_point():
    # x* = S(x*), w* = alpha x* is a fixed point of Algorithm 1: starting
    # there, one step changes nothing.
    pr = W.gmm_stored_cost_problem(8, n=30, m=20, eps=5e-2)
    cost = O.Cost(C=pr["C"])
    ref = O.solve(cost, pr["a"], pr["b"], pr["eps"], tol=1e-13, method=O.PLAIN)
    xstar = ref["g"] / pr["eps"]
    err, u, c, s = O.sinkhorn_map(cost, pr["eps"], ref["a"], ref["b"], xstar)
    np.testing.assert_allclose(s, xstar - xstar.mean(), atol=1e-10)
    al = math.sqrt(2 * 0.25)
    x1 = (al * s + s) / (1 + al)
    np.testing.assert_allclose(x1, s, atol=1e-14)
    e1, u1, c1, s1 = O.sinkhorn_map(cost, pr["eps"], ref["a"], ref["b"], x1)
    w1 = (al * s + (al * al - 2) * x1 + 2 * s1) / (1 + al)
    np.testing.assert_allclose(w1, al * s, atol=1e-10)


def test_homotopy_schedule_golden():
    pr = W.gmm_stored_cost_problem(5, n=20, m=20, eps=1e-2)
    rows = _golden_rows("homotopy_schedule.txt")
    total = int(sum(r[2] for r in rows))
    r = O.solve(O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"], tol=1e-300, method=O.ACC,
                mu0=0.25, m0=4, max_steps=total + 1, history=total + 1)
    mu = r["history"]["mu"]
    e = 1                                   # evaluation 0 is x_0
    for stage, mu_s, length in rows:
        for _ in range(int(length)):
            assert mu[e] == mu_s
            e += 1
    assert r["outer_stages"] == len(rows)


# --------------------------------------------------------------------------
# Stability quantities (eq. D, Theorem 4).
# --------------------------------------------------------------------------

def _phi_star_numeric(xi, b):
    """phi*(xi) = sup_v <xi, v> - sum b (e^v - v), by 1-D maximisation."""
    tot = 0.0
    for xj, bj in zip(xi, b):
        res = minimize_scalar(lambda v: -(xj * v - bj * (math.exp(v) - v)),
                              bounds=(-30, 30), method="bounded",
                              options={"xatol": 1e-12})
        tot += -res.fun
    return tot


def test_metric_D_identities():
    g = np.random.default_rng(31)
    b = W.dirichlet1(g, 6)
    c = b * np.exp(g.uniform(-0.8, 0.8, 6))
    p = np.log(c / b)
    D = np.array([O.metric_D(bj, pj) for bj, pj in zip(b, p)])
    xi = c - b
    np.testing.assert_allclose(D * p, xi, rtol=1e-13)          # D(z) z = grad phi(z)
    np.testing.assert_allclose(D, (c - b) / np.log(c / b), rtol=1e-12)  # log mean
    assert O.metric_D(0.3, 0.0) == 0.3                          # D(0) = diag(b)
    # ||p||_D^2 = D_phi*(xi, 0) + D_phi*(0, xi) (App. C). The constant
    # phi*(0) = -sum b cancels in both divergences; take it numerically too.
    ps = _phi_star_numeric(xi, b)
    p0 = _phi_star_numeric(np.zeros_like(xi), b)
    grad_ps = p                                                 # grad phi*(xi)
    d_xi_0 = ps - p0                                            # grad phi*(0) = 0
    d_0_xi = p0 - ps - grad_ps @ (0 - xi)
    assert abs((p * p * D).sum() - (d_xi_0 + d_0_xi)) < 1e-7
    # and D_phi*(0, xi) is what the oracle uses for Cond 1's right side
    t = O.stability_terms(b, c, c, np.zeros(6), np.zeros(6), np.zeros(6), np.zeros(6), 0.5)
    kappa1 = (4 - 0.25 - 2 * math.sqrt(0.5)) / (2 * 0.5 * 1.5 ** 2)
    assert abs(t["cond1_rhs"] - kappa1 * d_0_xi) < 1e-7


def test_stability_terms_match_theorem_norms():
    g = np.random.default_rng(32)
    m = 9
    b = W.dirichlet1(g, m)
    c0 = b * np.exp(g.uniform(-0.5, 0.5, m))
    c1 = b * np.exp(g.uniform(-0.3, 0.3, m))
    x0, w0, x1, w1 = (g.standard_normal(m) for _ in range(4))
    alpha = 0.4
    t = O.stability_terms(b, c0, c1, x0, w0, x1, w1, alpha)
    D0 = (c0 - b) / np.log(c0 / b)
    D1 = (c1 - b) / np.log(c1 / b)
    xi0 = c0 - b
    # ||grad f(x_k)||^2_{D_k^-1 D_{k+1} D_k^-1}
    lhs1 = (xi0 * xi0 * D1 / (D0 * D0)).sum()
    assert abs(t["cond1_lhs"] - lhs1) < 1e-12 * max(1, lhs1)
    # kappa from the appendix derivation with c = 1 and its chosen xi
    xi_c = (4 - alpha ** 2 - 2 * alpha ** 0.5) / (4 * alpha * (alpha + 1))
    k1 = xi_c * 4 * (1 - 0.5) / (1 + alpha)
    kl = (b * np.log(b / c0)).sum() + (c0 - b).sum()
    assert abs(t["cond1_rhs"] - k1 * kl) < 1e-12
    v0 = w0 / alpha - x0
    v1 = w1 / alpha - x1
    kappa2 = -(alpha / 2) * ((1 + 4 * xi_c) * alpha ** 2 + 4 * xi_c * alpha - 4)
    assert abs(kappa2 - alpha ** 1.5) < 1e-14
    assert abs(t["cond2_lhs"] - (v0 * v0 * (D1 - D0)).sum()) < 1e-12
    assert abs(t["cond2_rhs"] - kappa2 * (v1 * v1 * D1).sum()) < 1e-11
    assert t["cond1_ok"] == (t["cond1_lhs"] <= t["cond1_rhs"])


def test_gate_restarts_momentum():
    # With the gate on, a failed check sets w_{k+1} = alpha x_{k+1} (y = x).
    pr = W.gmm_stored_cost_problem(6, n=50, m=50, eps=1e-2)
    cost = O.Cost(C=pr["C"])
    rg = O.solve(cost, pr["a"], pr["b"], pr["eps"], tol=1e-8, method=O.ACC,
                 stability=O.STAB_GATE, history=5000)
    rr = O.solve(cost, pr["a"], pr["b"], pr["eps"], tol=1e-8, method=O.ACC,
                 stability=O.STAB_REPORT, history=5000)
    assert rr["stability_failures"] > 0
    assert rg["status"] == O.CONVERGED
    first = int(np.nonzero(rr["history"]["stab"])[0][0])
    # the failed check at evaluation `first` changes w there, so the runs
    # agree up to that evaluation and part at the next one
    np.testing.assert_array_equal(rr["history"]["err"][:first + 1], rg["history"]["err"][:first + 1])
    assert rr["history"]["err"][first + 1] != rg["history"]["err"][first + 1]


def test_backtracking_halves_mu_at_each_failure():
    """BACKTRACK follows Algorithm 2's schedule except that a failed check ends
    the stage at once: replaying the schedule from the recorded stability bits
    reproduces the recorded mu of every step; runs agree with REPORT until the
    first failure and both converge."""
    pr = W.gmm_stored_cost_problem(6, n=50, m=50, eps=1e-2)
    cost = O.Cost(C=pr["C"])
    kw = dict(tol=1e-8, method=O.ACC, history=5000)
    rb = O.solve(cost, pr["a"], pr["b"], pr["eps"], stability=O.STAB_BACKTRACK, **kw)
    rr = O.solve(cost, pr["a"], pr["b"], pr["eps"], stability=O.STAB_REPORT, **kw)
    assert rb["status"] == O.CONVERGED and rr["status"] == O.CONVERGED
    assert rb["stability_failures"] > 0
    hb = rb["history"]
    mu, m_stage, j, stages = 0.25, 4, 0, 0
    for e in range(1, rb["sinkhorn_steps"]):
        assert hb["mu"][e] == mu, (e, hb["mu"][e], mu)
        j += 1
        if j == m_stage or hb["stab"][e] != 0:
            mu /= 2.0
            m_stage = int(math.floor(math.sqrt(2.0) * m_stage)) + 1
            j = 0
            stages += 1
    assert rb["outer_stages"] == stages
    first = int(np.nonzero(rr["history"]["stab"])[0][0])
    np.testing.assert_array_equal(rr["history"]["err"][:first + 1], hb["err"][:first + 1])
    assert rr["history"]["err"][first + 1] != hb["err"][first + 1]


# --------------------------------------------------------------------------
# Evaluation of given potentials and fixed-point identity.
# --------------------------------------------------------------------------

def test_evaluate_matches_numpy_plan():
    C, a, b = _rand_problem(41, 12, 9)
    eps = 0.07
    g = np.random.default_rng(42)
    f, gg = g.standard_normal(12) * 0.1, g.standard_normal(9) * 0.1
    ev = O.evaluate(O.Cost(C=C), eps, a, b, f, gg)
    C64 = C.astype(np.float64)
    P = _plan(C64, f, gg, eps)
    assert abs(ev["row_l1"] - np.abs(P.sum(1) - a).sum()) < 1e-12
    assert abs(ev["col_l1"] - np.abs(P.sum(0) - b).sum()) < 1e-12
    assert abs(ev["transport_cost"] - (C64 * P).sum()) < 1e-12
    assert abs(ev["primal"] - ((C64 * P).sum() + eps * (P * (np.log(P) - 1)).sum())) < 1e-12
    r, cs = O.rows_sample(O.Cost(C=C), eps, f, gg, [3, 0, 11])
    np.testing.assert_allclose(r, P.sum(1)[[3, 0, 11]], rtol=1e-13)
    np.testing.assert_allclose(cs, (C64 * P).sum(1)[[3, 0, 11]], rtol=1e-13)
    cc = O.cols_sample(O.Cost(C=C), eps, f, gg, [8, 1])
    np.testing.assert_allclose(cc, P.sum(0)[[8, 1]], rtol=1e-13)


def test_fixed_point_and_strong_duality():
    # At the solution P = diag(e^{f/eps}) K diag(e^{g/eps}) lies in Pi(a, b)
    # and primal = dual (eq. EOT vs eq. dual-obj).
    pr = W.gmm_stored_cost_problem(7, n=64, m=48, eps=2e-2)
    r = O.solve(O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"], tol=1e-12, method=O.ACC)
    C64 = pr["C"].astype(np.float64)
    K = np.exp(-C64 / pr["eps"])
    P = np.exp(r["f"] / pr["eps"])[:, None] * K * np.exp(r["g"] / pr["eps"])[None, :]
    np.testing.assert_allclose(P.sum(1), r["a"], rtol=1e-11)
    assert np.abs(P.sum(0) - r["b"]).sum() < 1e-12
    ev = O.evaluate(O.Cost(C=pr["C"]), pr["eps"], r["a"], r["b"], r["f"], r["g"])
    assert abs(ev["primal"] - ev["dual"]) < 1e-10


def test_point_cloud_costs_match_direct_formulas():
    g = np.random.default_rng(51)
    X = g.random((5, 3)).astype(np.float32)
    Y = g.random((4, 3)).astype(np.float32)
    c = O.Cost(X=X, Y=Y, kind="sqeuclid")
    M = ((X.astype(np.float64)[:, None, :] - Y.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    np.testing.assert_allclose(c.matrix(), M, rtol=1e-15)
    cs = O.Cost(X=X, Y=Y, kind="sqeuclid", scale_to_max=True)
    np.testing.assert_allclose(cs.matrix(), M / M.max(), rtol=1e-15)
    cc = O.Cost(X=X, Y=Y, kind="cosine")
    np.testing.assert_allclose(cc.matrix(), 1 - X.astype(np.float64) @ Y.astype(np.float64).T,
                               rtol=1e-15)
    # dense cost: entries are the FP32 values, transposition-sensitive
    C = g.random((3, 5)).astype(np.float32)
    d = O.Cost(C=C)
    assert d.entry(2, 4) == float(C[2, 4]) and d.entry(0, 1) == float(C[0, 1])


def test_sampled_passes_match_full_passes():
    C, a, b = _rand_problem(61, 20, 30)
    cost = O.Cost(C=C)
    x = np.random.default_rng(62).standard_normal(30)
    u = O.row_pass(cost, 0.05, np.log(a), x)
    us = O.row_pass_sample(cost, 0.05, np.log(a), x, [19, 2, 7])
    np.testing.assert_array_equal(us, u[[19, 2, 7]])
    ell = O.col_lse(cost, 0.05, u)
    es = O.col_lse_sample(cost, 0.05, u, [29, 0])
    np.testing.assert_array_equal(es, ell[[29, 0]])


def test_materialised_cost_reproduces_the_point_cloud_cost():
    """A cost formed once as an FP64 matrix is the same problem: entries equal
    to the definition (checked against numpy), transposition-sensitive, and a
    whole solve on it is bitwise identical to the solve on the points."""
    g = np.random.default_rng(71)
    X = W.unit_gaussian_points(g, 9, 40)
    Y = W.unit_gaussian_points(g, 6, 40)
    cost = O.Cost(X=X, Y=Y, kind="cosine")
    mc = cost.materialised()
    direct = 1.0 - X.astype(np.float64) @ Y.astype(np.float64).T
    np.testing.assert_allclose(mc.matrix(), direct, rtol=0, atol=1e-15)
    assert mc.entry(8, 5) == cost.entry(8, 5) and mc.entry(5, 2) == cost.entry(5, 2)
    assert mc.entry(1, 4) != mc.entry(4, 1) or direct[1, 4] == direct[4, 1]
    a, b = W.dirichlet1(g, 9), W.dirichlet1(g, 6)
    r1 = O.solve(cost, a, b, 0.02, 1e-9, method=O.ACC)
    r2 = O.solve(mc, a, b, 0.02, 1e-9, method=O.ACC)
    assert r1["sinkhorn_steps"] == r2["sinkhorn_steps"]
    np.testing.assert_array_equal(r1["f"], r2["f"])
    np.testing.assert_array_equal(r1["g"], r2["g"])
    # the scale is carried by the matrix
    cs = O.Cost(X=X, Y=Y, kind="sqeuclid", scale_to_max=True)
    np.testing.assert_array_equal(cs.materialised().matrix(), cs.matrix())


def test_plan_and_barycentric_projection():
    """Separable cost C_ij = r_i + s_j: the solution's plan is a b^T, so the
    barycentric projection of any features is their b-weighted mean in every
    row; the plan's rows sum to a (the row pass is exact) and it matches the
    plan evaluate() sums."""
    g = np.random.default_rng(81)
    n, m = 7, 11
    r = np.round(g.random(n) * 64) / 64
    sv = np.round(g.random(m) * 64) / 64
    C = (r[:, None] + sv[None, :]).astype(np.float32)
    a, b = W.dirichlet1(g, n), W.dirichlet1(g, m)
    cost = O.Cost(C=C)
    res = O.solve(cost, a, b, 0.1, tol=1e-13, method=O.PLAIN)
    P = O.plan(cost, 0.1, res["f"], res["g"])
    np.testing.assert_allclose(P, np.outer(res["a"], res["b"]), rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(P.sum(1), res["a"], rtol=1e-12)
    Z = g.standard_normal((m, 3)).astype(np.float32)
    bary = O.barycentric(cost, 0.1, res["f"], res["g"], Z)
    want = (res["b"][:, None] * Z.astype(np.float64)).sum(0)
    np.testing.assert_allclose(bary, np.tile(want, (n, 1)), rtol=1e-9, atol=1e-12)
    # the plan of arbitrary potentials: transposition-sensitive, and its total
    # equals evaluate()'s mass
    f = g.standard_normal(n) * 0.1
    gg = g.standard_normal(m) * 0.1
    P2 = O.plan(cost, 0.3, f, gg)
    assert P2.shape == (n, m)
    assert abs(P2[2, 5] - np.exp((f[2] + gg[5] - float(C[2, 5])) / 0.3)) <= 1e-15
    ev = O.evaluate(cost, 0.3, a, b, f, gg)
    assert abs(P2.sum() - ev["mass"]) <= 1e-12 * ev["mass"]


# --------------------------------------------------------------------------
# Warm starts and resumed solves (Algorithm 1-2 from a given point).
# --------------------------------------------------------------------------

@pytest.mark.parametrize("method,carry_y,stability", [
    (O.ACC, True, O.STAB_REPORT), (O.ACC, False, O.STAB_REPORT), (O.ACC, True, O.STAB_GATE),
    (O.ACC, True, O.STAB_BACKTRACK), (O.PLAIN, True, O.STAB_REPORT)])
def test_resume_matches_the_uninterrupted_run(method, carry_y, stability):
    # A solve stopped at a loose tolerance and resumed from its state repeats
    # S(x) once and then takes exactly the uninterrupted run's steps: the
    # stage position, the momentum (gate and carry included) and the iterate
    # all carry over, so the final potentials are identical to the bit.
    pr = W.gmm_stored_cost_problem(21, n=50, m=40, eps=2e-2)
    cost, a, b, eps = O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"]
    kw = dict(method=method, carry_y=carry_y, stability=stability)
    # (w handed over unchanged between stages stalls near 1e-9 on this problem)
    tol = 1e-10 if carry_y else 1e-8
    full = O.solve(cost, a, b, eps, tol=tol, history=4000, **kw)
    part = O.solve(cost, a, b, eps, tol=1e-3, **kw)
    res = O.resume(cost, a, b, eps, part["state"], tol=tol, history=4000, **kw)
    assert full["status"] == O.CONVERGED
    k = part["sinkhorn_steps"]
    assert 1 < k < full["sinkhorn_steps"]
    assert res["sinkhorn_steps"] == full["sinkhorn_steps"] - k + 1
    np.testing.assert_array_equal(res["g"], full["g"])
    np.testing.assert_array_equal(res["f"], full["f"])
    np.testing.assert_array_equal(res["history"]["err"][1:], full["history"]["err"][k:])
    if method == O.ACC:
        assert res["outer_stages"] == full["outer_stages"]
        assert part["state"]["mu"] == 0.25 * 2.0 ** -part["state"]["stages"]


def test_warm_start_at_the_fixed_point_stops_at_once():
    pr = W.gmm_stored_cost_problem(22, n=40, m=30, eps=1e-2)
    cost, a, b, eps = O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"]
    ref = O.solve(cost, a, b, eps, tol=1e-12)
    for method in (O.ACC, O.PLAIN):
        r = O.warm_start(cost, a, b, eps, ref["g"], tol=1e-9, method=method)
        assert r["status"] == O.CONVERGED and r["sinkhorn_steps"] == 1


def test_warm_start_from_zero_is_the_cold_start():
    pr = W.gmm_stored_cost_problem(23, n=30, m=40, eps=2e-2)
    cost, a, b, eps = O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"]
    cold = O.solve(cost, a, b, eps, tol=1e-9)
    warm = O.warm_start(cost, a, b, eps, np.zeros(40), tol=1e-9)
    assert warm["sinkhorn_steps"] == cold["sinkhorn_steps"]
    np.testing.assert_array_equal(warm["g"], cold["g"])


def test_eps_continuation_reaches_the_unique_fixed_point():
    # A state taken at eps1 resumed at eps2 keeps its potential g = eps x and
    # converges to the eps2 solution (unique up to the gauge, Sec. 2).
    pr = W.gmm_stored_cost_problem(24, n=40, m=35, eps=1e-2)
    cost, a, b = O.Cost(C=pr["C"]), pr["a"], pr["b"]
    e1, e2 = 5e-2, 1e-2
    s1 = O.solve(cost, a, b, e1, tol=1e-4)
    r = O.resume(cost, a, b, e2, s1["state"], tol=1e-11, history=2, keep_x=True)
    np.testing.assert_allclose(e2 * r["history"]["x"][0], s1["state"]["x"] * e1, rtol=1e-15,
                               atol=1e-300)
    cold = O.solve(cost, a, b, e2, tol=1e-11)
    assert r["status"] == O.CONVERGED
    sh = r["g"].mean() - cold["g"].mean()
    np.testing.assert_allclose(r["g"] - sh, cold["g"], atol=1e-6 * e2)
    np.testing.assert_allclose(r["f"] + sh, cold["f"], atol=1e-6 * e2)


# --------------------------------------------------------------------------
# Full-size FP64 marginal errors (eq. l1tol) and the recorded Theorem 4 terms.
# --------------------------------------------------------------------------

def test_marginal_l1_closed_form_on_a_separable_cost():
    # C_ij = r_i + s_j with f_i = r_i + eps log a_i and g_j = s_j + eps log b_j
    # + eps d_j gives P_ij = a_i b_j e^{d_j}: column sums b_j e^{d_j}, row sums
    # a_i sum_j b_j e^{d_j}, both errors in closed form.
    g = np.random.default_rng(71)
    n, m, eps = 37, 23, 0.05
    r_ = g.integers(0, 1024, n) / 1024.0
    s_ = g.integers(0, 1024, m) / 1024.0
    C = (r_[:, None] + s_[None, :]).astype(np.float32)
    a, b = W.dirichlet1(g, n), W.dirichlet1(g, m)
    d = g.uniform(-1e-3, 1e-3, m)
    f = r_ + eps * np.log(a)
    gg = s_ + eps * np.log(b) + eps * d
    out = O.marginal_l1(O.Cost(C=C), eps, a, b, f, gg)
    col = np.abs(b * np.expm1(d)).sum()
    row = np.abs(a * ((b * np.exp(d)).sum() - 1.0)).sum()
    assert abs(out["col_l1"] - col) <= 1e-12 * col
    assert abs(out["row_l1"] - row) <= 1e-11 * max(row, 1e-300) + 1e-16
    # a transposed cost or swapped marginals would break it
    ev = O.evaluate(O.Cost(C=C), eps, a, b, f, gg)
    assert abs(ev["col_l1"] - out["col_l1"]) <= 1e-13
    assert abs(ev["row_l1"] - out["row_l1"]) <= 1e-13


def test_marginal_l1_thread_count_does_not_matter():
    C, a, b = _rand_problem(72, 61, 45)
    eps = 0.1
    res = O.solve(O.Cost(C=C), a, b, eps, tol=1e-3, method=O.PLAIN)
    t0 = O.set_threads(0)
    try:
        O.set_threads(1)
        one = O.marginal_l1(O.Cost(C=C), eps, res["a"], res["b"], res["f"], res["g"])
        O.set_threads(3)
        three = O.marginal_l1(O.Cost(C=C), eps, res["a"], res["b"], res["f"], res["g"])
    finally:
        O.set_threads(t0)
    assert abs(one["col_l1"] - three["col_l1"]) <= 1e-15
    assert abs(one["row_l1"] - three["row_l1"]) <= 1e-15
    assert abs(one["col_l1"] - res["marginal_l1"]) <= 1e-12


def test_history_records_theorem4_terms_behind_the_bits():
    pr = W.gmm_stored_cost_problem(73, n=60, m=50, eps=1e-2)
    r = O.solve(O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"], tol=1e-8, method=O.ACC,
                history=5000)
    h = r["history"]
    cond, stab = h["cond"], h["stab"]
    assert np.all(cond[0] == 0.0)                       # x_0: no step, no test
    k = len(stab)
    assert k > 5 and stab.any()
    np.testing.assert_array_equal(stab & 1, (cond[:k, 0] > cond[:k, 1]).astype(np.int32))
    np.testing.assert_array_equal((stab >> 1) & 1, (cond[:k, 2] > cond[:k, 3]).astype(np.int32))
    # the Cond 1 right side is kappa1(alpha) times KL(b || c_k) of the previous
    # iterate, KL >= 0 and kappa1 > 0 for mu0 <= 0.5
    assert np.all(cond[1:k, 1] >= 0.0) and np.all(cond[1:k, 0] >= 0.0)
    assert np.all(cond[1:k, 3] >= 0.0)
    off = O.solve(O.Cost(C=pr["C"]), pr["a"], pr["b"], pr["eps"], tol=1e-8, method=O.ACC,
                  history=5000, stability=O.STAB_OFF)
    assert np.all(off["history"]["cond"] == 0.0)
