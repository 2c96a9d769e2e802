"""Plain FP64 CPU oracle for Sinkhorn / Acc-Sinkhorn -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package. The GPU product path
never imports it, and it imports nothing from the GPU package.

The arithmetic lives in ``acc_sinkhorn_oracle.c`` (IEEE double, libm); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes. The only logic here is problem preparation that the paper states
outside the algorithms: marginals normalised to unit mass (Sec. 2 assumes
1'a = 1'b = 1) and the optional division of the cost by its maximum entry
(Sec. 5, colour transfer).

Parity notes: every routine is pinned by ``tests/test_oracle_pins.py`` except
the iteration counts of the paper's Tables 2-3 (their data are not public
here) -- those are "parity unpinned".
"""
from __future__ import annotations

import ctypes as ct
import math
import os
import subprocess
import tempfile


import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acc_sinkhorn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DENSE, SQEUCLID, COSINE, DENSE64 = 0, 1, 2, 3
PLAIN, ACC = 0, 1
STAB_OFF, STAB_REPORT, STAB_GATE, STAB_BACKTRACK = 0, 1, 2, 3
CONVERGED, MAXITER = 0, 7


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP).

    ``ACCSINK_ORACLE_LIB`` names a prebuilt copy to load instead (used by the
    test that plants mistakes in the oracle to check that the pins catch them)."""
    alt = os.environ.get("ACCSINK_ORACLE_LIB")
    if alt:
        return alt
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Cost(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("n", ct.c_long), ("m", ct.c_long),
                ("d", ct.c_long), ("ldc", ct.c_long),
                ("C", ct.c_void_p), ("X", ct.c_void_p), ("Y", ct.c_void_p),
                ("scale", ct.c_double), ("C64", ct.c_void_p)]


class _Problem(ct.Structure):
    _fields_ = [("cost", ct.POINTER(_Cost)), ("eps", ct.c_double),
                ("a", ct.c_void_p), ("b", ct.c_void_p),
                ("loga", ct.c_void_p), ("logb", ct.c_void_p)]


class _Result(ct.Structure):
    _fields_ = [("status", ct.c_int), ("sinkhorn_steps", ct.c_int),
                ("outer_stages", ct.c_int), ("stability_failures", ct.c_int),
                ("marginal_l1", ct.c_double), ("dual", ct.c_double)]


class _History(ct.Structure):
    _fields_ = [("cap", ct.c_long), ("err", ct.c_void_p), ("dual", ct.c_void_p),
                ("mu", ct.c_void_p), ("stab", ct.c_void_p), ("x", ct.c_void_p),
                ("cond", ct.c_void_p)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        d, vp, lg = ct.c_double, ct.c_void_p, ct.c_long
        _lib.orc_cost_entry.restype = d
        _lib.orc_cost_entry.argtypes = [vp, lg, lg]
        _lib.orc_cost_max.restype = d
        _lib.orc_cost_max.argtypes = [vp]
        _lib.orc_cost_matrix.argtypes = [vp, vp]
        _lib.orc_row_pass.argtypes = [vp, d, vp, vp, vp]
        _lib.orc_col_lse.argtypes = [vp, d, vp, vp]
        _lib.orc_sinkhorn_map.restype = d
        _lib.orc_sinkhorn_map.argtypes = [vp, vp, vp, vp, vp]
        _lib.orc_dual_after_row_pass.restype = d
        _lib.orc_dual_after_row_pass.argtypes = [vp, vp, vp]
        _lib.orc_metric_D.restype = d
        _lib.orc_metric_D.argtypes = [d, d]
        _lib.orc_stability_terms.argtypes = [lg, vp, vp, vp, vp, vp, vp, vp, d, vp]
        _lib.orc_solve.restype = ct.c_int
        _lib.orc_solve.argtypes = [vp, d, ct.c_int, d, ct.c_int, ct.c_int,
                                   ct.c_int, ct.c_int, vp, vp, vp, vp]
        _lib.orc_solve_from.restype = ct.c_int
        _lib.orc_solve_from.argtypes = [vp, d, ct.c_int, d, ct.c_int, ct.c_int, ct.c_int,
                                        ct.c_int, vp, vp, d, lg, lg, ct.c_int, vp, vp, vp,
                                        vp, vp, vp, vp]
        _lib.orc_evaluate.argtypes = [vp, d, vp, vp, vp, vp, vp]
        _lib.orc_marginal_l1.argtypes = [vp, d, vp, vp, vp, vp, vp]
        _lib.orc_plan.argtypes = [vp, d, vp, vp, vp]
        _lib.orc_barycentric.argtypes = [vp, d, vp, vp, vp, lg, vp]
        _lib.orc_rows_sample.argtypes = [vp, d, vp, vp, vp, lg, vp, vp]
        _lib.orc_cols_sample.argtypes = [vp, d, vp, vp, vp, lg, vp]
        _lib.orc_row_pass_sample.argtypes = [vp, d, vp, vp, vp, lg, vp]
        _lib.orc_col_lse_sample.argtypes = [vp, d, vp, vp, lg, vp]
        _lib.orc_set_threads.restype = ct.c_int
        _lib.orc_set_threads.argtypes = [ct.c_int]
    return _lib


def _p(arr):
    return ct.c_void_p(arr.ctypes.data) if arr is not None else None


def _f64(v):
    return np.ascontiguousarray(v, dtype=np.float64)


class Cost:
    """An EOT cost: a dense FP32 matrix or FP32 point clouds (formed in FP64).

    ``scale_to_max`` divides every entry by the largest one (Sec. 5)."""

    def __init__(self, C=None, X=None, Y=None, kind=None, scale_to_max=False):
        if C is not None:
            C = np.asarray(C)
            if C.dtype != np.float32:
                raise TypeError("dense cost must be float32 (the problem is the FP32 values)")
            if not C.flags.c_contiguous:
                C = np.ascontiguousarray(C)
            self.C, self.X, self.Y = C, None, None
            self.kind, self.n, self.m, self.d = DENSE, C.shape[0], C.shape[1], 0
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
            Y = np.ascontiguousarray(Y, dtype=np.float32)
            self.C, self.X, self.Y = None, X, Y
            self.kind = SQEUCLID if kind in (None, "sqeuclid", SQEUCLID) else COSINE
            self.n, self.m, self.d = X.shape[0], Y.shape[0], X.shape[1]
        self._s = _Cost(self.kind, self.n, self.m, self.d, self.m,
                        _p(self.C), _p(self.X), _p(self.Y), 1.0)
        self.scale = 1.0
        if scale_to_max:
            self.scale = 1.0 / _L().orc_cost_max(ct.byref(self._s))
            self._s.scale = self.scale

    @property
    def ref(self):
        return ct.byref(self._s)

    def entry(self, i, j):
        return _L().orc_cost_entry(self.ref, int(i), int(j))

    def matrix(self):
        out = np.empty((self.n, self.m), np.float64)
        _L().orc_cost_matrix(self.ref, _p(out))
        return out

    def unscaled_max(self):
        return _L().orc_cost_max(self.ref)

    def materialised(self):
        """The same cost formed once as an FP64 matrix (entries identical to
        ``entry``, scale applied), so that each pass reads instead of forming
        them: much faster for high-dimensional point clouds."""
        return MaterialisedCost(self.matrix())


class MaterialisedCost(Cost):
    """A cost given as an FP64 n x m matrix (already scaled)."""

    def __init__(self, C64):
        C64 = np.ascontiguousarray(C64, dtype=np.float64)
        self.C64, self.C, self.X, self.Y = C64, None, None, None
        self.kind, self.n, self.m, self.d = DENSE64, C64.shape[0], C64.shape[1], 0
        self._s = _Cost(DENSE64, self.n, self.m, 0, self.m, None, None, None, 1.0, _p(C64))
        self.scale = 1.0


def normalise(v):
    v = _f64(v)
    return v / v.sum()


def set_threads(t: int = 0) -> int:
    """Set (t > 0) and return the OpenMP thread count the oracle uses."""
    return _L().orc_set_threads(int(t))


def row_pass(cost: Cost, eps, loga, x):
    loga, x = _f64(loga), _f64(x)
    u = np.empty(cost.n)
    _L().orc_row_pass(cost.ref, float(eps), _p(loga), _p(x), _p(u))
    return u


def col_lse(cost: Cost, eps, u):
    u = _f64(u)
    ell = np.empty(cost.m)
    _L().orc_col_lse(cost.ref, float(eps), _p(u), _p(ell))
    return ell


def _problem(cost, eps, a, b):
    a, b = _f64(a), _f64(b)
    loga, logb = np.log(a), np.log(b)
    keep = (a, b, loga, logb)
    pr = _Problem(ct.pointer(cost._s), float(eps), _p(a), _p(b), _p(loga), _p(logb))
    return pr, keep


def sinkhorn_map(cost: Cost, eps, a, b, x):
    """S(x): returns (err, u, c, s) -- see orc_sinkhorn_map."""
    pr, keep = _problem(cost, eps, a, b)
    x = _f64(x)
    u, c, s = np.empty(cost.n), np.empty(cost.m), np.empty(cost.m)
    err = _L().orc_sinkhorn_map(ct.byref(pr), _p(x), _p(u), _p(c), _p(s))
    return err, u, c, s


def dual_after_row_pass(cost: Cost, eps, a, b, u, x):
    pr, keep = _problem(cost, eps, a, b)
    u, x = _f64(u), _f64(x)
    return _L().orc_dual_after_row_pass(ct.byref(pr), _p(u), _p(x))


def metric_D(bj, z):
    return _L().orc_metric_D(float(bj), float(z))


def stability_terms(b, c_k, c_k1, x_k, w_k, x_k1, w_k1, alpha):
    arrs = [_f64(v) for v in (b, c_k, c_k1, x_k, w_k, x_k1, w_k1)]
    out = np.empty(6)
    _L().orc_stability_terms(len(arrs[0]), *[_p(v) for v in arrs], float(alpha), _p(out))
    return {"cond1_lhs": out[0], "cond1_rhs": out[1], "cond2_lhs": out[2],
            "cond2_rhs": out[3], "cond1_ok": bool(out[4]), "cond2_ok": bool(out[5])}


def solve(cost: Cost, a, b, eps, tol=1e-6, method=ACC, mu0=0.25, m0=4,
          max_steps=100000, stability=STAB_REPORT, history=0, keep_x=False,
          carry_y=True, x0=None, w0=None, stage=None):
    """Plain Sinkhorn (method=PLAIN) or Acc-Sinkhorn with homotopy (ACC).

    The history's ``cond`` rows hold Theorem 4's four terms (Cond 1 lhs, rhs,
    Cond 2 lhs, rhs) of the step that produced each iterate.
    ``carry_y`` selects how Algorithm 2 hands w to the next homotopy stage:
    True keeps y = w / alpha (the (x_k, y_k) state of Theorem 1), False hands
    w over unchanged as Algorithm 2 is printed.
    Marginals are normalised to unit mass first. Returns a dict with f, g
    (cost units), status, step counts and, if ``history`` > 0, per-evaluation
    histories (err, dual, mu, stability bits and optionally the iterates).

    ``x0``, ``w0`` (m each) and ``stage`` ({mu, m_stage, j, stages}) start the
    iteration there instead of at zero with (mu0, m0). The result's ``state``
    holds the point the iteration would continue from: (x, w) and the stage,
    so solve(..., x0=s["x"], w0=s["w"], stage=s) resumes it."""
    a, b = normalise(a), normalise(b)
    pr, keep = _problem(cost, eps, a, b)
    f, g = np.empty(cost.n), np.empty(cost.m)
    res = _Result()
    hist = None
    h = {}
    if history > 0:
        h["err"] = np.full(history, np.nan)
        h["dual"] = np.full(history, np.nan)
        h["mu"] = np.full(history, np.nan)
        h["stab"] = np.zeros(history, np.int32)
        h["x"] = np.full((history, cost.m), np.nan) if keep_x else None
        h["cond"] = np.zeros((history, 4))
        hist = _History(history, _p(h["err"]), _p(h["dual"]), _p(h["mu"]),
                        _p(h["stab"]), _p(h["x"]), _p(h["cond"]))
    x0 = None if x0 is None else _f64(x0)
    w0 = None if w0 is None else _f64(w0)
    stage = stage or {"mu": mu0, "m_stage": m0, "j": 0, "stages": 0}
    xo, wo, so = np.empty(cost.m), np.empty(cost.m), np.zeros(4)
    st = _L().orc_solve_from(ct.byref(pr), float(tol), int(method), float(mu0), int(m0),
                             int(max_steps), int(stability), int(bool(carry_y)),
                             _p(x0) if x0 is not None else None,
                             _p(w0) if w0 is not None else None,
                             float(stage["mu"]), int(stage["m_stage"]), int(stage["j"]),
                             int(stage["stages"]), _p(f), _p(g), ct.byref(res),
                             ct.byref(hist) if hist is not None else None,
                             _p(xo), _p(wo), _p(so))
    if st not in (CONVERGED, MAXITER):
        raise ValueError(f"oracle rejected the arguments (status {st})")
    out = {"f": f, "g": g, "status": res.status, "sinkhorn_steps": res.sinkhorn_steps,
           "outer_stages": res.outer_stages, "stability_failures": res.stability_failures,
           "marginal_l1": res.marginal_l1, "dual": res.dual, "a": a, "b": b,
           "state": {"x": xo, "w": wo, "mu": so[0], "m_stage": int(so[1]), "j": int(so[2]),
                     "stages": int(so[3]), "eps": float(eps)}}
    if history > 0:
        k = min(res.sinkhorn_steps, history)
        out["history"] = {key: (v[:k] if v is not None else None) for key, v in h.items()}
    return out


def warm_start(cost: Cost, a, b, eps, g0, mu0=0.25, m0=4, **kw):
    """Acc or plain Sinkhorn started at the potential g0 (cost units) instead
    of zero: x0 = g0 / eps and, for Algorithm 1, w0 = alpha0 x0 (y0 = x0)
    with alpha0 = sqrt(2 mu0)."""
    x0 = _f64(g0) / eps
    return solve(cost, a, b, eps, mu0=mu0, m0=m0, x0=x0, w0=math.sqrt(2.0 * mu0) * x0, **kw)


def resume(cost: Cost, a, b, eps, state, mu0=0.25, m0=4, **kw):
    """Continues a solve from its returned ``state`` (x, w, stage, eps). At a
    new eps the iterate keeps its potential g = eps x: x and w are scaled by
    state eps / eps."""
    mul = state["eps"] / eps
    return solve(cost, a, b, eps, mu0=mu0, m0=m0, x0=state["x"] * mul,
                 w0=state["w"] * mul, stage=state, **kw)


def evaluate(cost: Cost, eps, a, b, f, g):
    """FP64 evaluation of P(f, g): marginal L1s, <C,P>, dual, primal, mass."""
    a, b, f, g = _f64(a), _f64(b), _f64(f), _f64(g)
    out = np.empty(6)
    _L().orc_evaluate(cost.ref, float(eps), _p(a), _p(b), _p(f), _p(g), _p(out))
    return {"row_l1": out[0], "col_l1": out[1], "transport_cost": out[2],
            "dual": out[3], "primal": out[4], "mass": out[5]}


def marginal_l1(cost: Cost, eps, a, b, f, g):
    """FP64 row and column L1 errors of P(f, g) (eq. l1tol), rows split over
    the OpenMP threads: for full-size problems."""
    a, b, f, g = _f64(a), _f64(b), _f64(f), _f64(g)
    out = np.empty(2)
    _L().orc_marginal_l1(cost.ref, float(eps), _p(a), _p(b), _p(f), _p(g), _p(out))
    return {"row_l1": out[0], "col_l1": out[1]}


def plan(cost: Cost, eps, f, g):
    """The plan P(f, g) as an FP64 n x m matrix."""
    f, g = _f64(f), _f64(g)
    P = np.empty((cost.n, cost.m))
    _L().orc_plan(cost.ref, float(eps), _p(f), _p(g), _p(P))
    return P


def barycentric(cost: Cost, eps, f, g, Z):
    """out_i = sum_j P_ij Z_j / sum_j P_ij for FP32 features Z (m x dz)."""
    f, g = _f64(f), _f64(g)
    Z = np.ascontiguousarray(Z, dtype=np.float32)
    out = np.empty((cost.n, Z.shape[1]))
    _L().orc_barycentric(cost.ref, float(eps), _p(f), _p(g), _p(Z), int(Z.shape[1]), _p(out))
    return out


def rows_sample(cost: Cost, eps, f, g, rows):
    f, g = _f64(f), _f64(g)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    r, cs = np.empty(len(rows)), np.empty(len(rows))
    _L().orc_rows_sample(cost.ref, float(eps), _p(f), _p(g), _p(rows), len(rows), _p(r), _p(cs))
    return r, cs


def cols_sample(cost: Cost, eps, f, g, cols):
    f, g = _f64(f), _f64(g)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    c = np.empty(len(cols))
    _L().orc_cols_sample(cost.ref, float(eps), _p(f), _p(g), _p(cols), len(cols), _p(c))
    return c


def row_pass_sample(cost: Cost, eps, loga, x, rows):
    loga, x = _f64(loga), _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    u = np.empty(len(rows))
    _L().orc_row_pass_sample(cost.ref, float(eps), _p(loga), _p(x), _p(rows), len(rows), _p(u))
    return u


def col_lse_sample(cost: Cost, eps, u, cols):
    u = _f64(u)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    ell = np.empty(len(cols))
    _L().orc_col_lse_sample(cost.ref, float(eps), _p(u), _p(cols), len(cols), _p(ell))
    return ell
