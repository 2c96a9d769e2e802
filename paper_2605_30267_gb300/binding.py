"""Thin Python binding of the C-ABI in include/accsink.h (argument marshalling only).

Every computation runs in ``libaccsink.so``'s CUDA kernels. PyTorch supplies
device memory and streams; this module only packs pointers, sizes and
parameters into the C structs and calls the ``accsink_*`` functions of the same
names. If the library has not been built, loading raises -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libaccsink.so")

OK, ERR_INVALID_ARG, ERR_NONPOSITIVE_MARGINAL, ERR_NONFINITE = 0, 1, 2, 3
ERR_OOM, ERR_BUDGET, ERR_TIMEOUT, ERR_MAXITER, ERR_CUDA, ERR_UNSUPPORTED = 4, 5, 6, 7, 8, 9
COST_DENSE, COST_SQEUCLID, COST_COSINE = 0, 1, 2
SCALE_NONE, SCALE_MAX_TO_ONE = 0, 1
PLAIN, ACC = 0, 1
STAB_OFF, STAB_REPORT, STAB_GATE, STAB_BACKTRACK = 0, 1, 2, 3
CARRY_Y, CARRY_W = 0, 1
PREC_AUTO, PREC_FP32, PREC_DF32 = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "ERR_INVALID_ARG", 2: "ERR_NONPOSITIVE_MARGINAL",
                3: "ERR_NONFINITE", 4: "ERR_OOM", 5: "ERR_BUDGET", 6: "ERR_TIMEOUT",
                7: "ERR_MAXITER", 8: "ERR_CUDA", 9: "ERR_UNSUPPORTED"}

# Every symbol include/accsink.h declares.
EXPORTED = ["accsink_create", "accsink_destroy", "accsink_last_error", "accsink_params_default",
            "accsink_version", "accsink_solve", "accsink_solve_host", "accsink_get_history",
            "accsink_row_pass", "accsink_col_lse", "accsink_sinkhorn_map",
            "accsink_transport_cost", "accsink_time_passes", "accsink_launch_geometry",
            "accsink_col_lse_noalloc", "accsink_solve_batch", "accsink_batch_set_config",
            "accsink_batch_get_config", "accsink_batch_autotune", "accsink_batch_last_timing",
            "accsink_server_create", "accsink_server_destroy", "accsink_server_last_error",
            "accsink_server_submit", "accsink_server_poll", "accsink_server_wait",
            "accsink_server_potentials", "accsink_server_copy_potentials",
            "accsink_server_release", "accsink_server_get_stats", "accsink_server_set_config",
            "accsink_server_set_limits",
            "accsink_plan", "accsink_barycentric", "accsink_export_state",
            "accsink_solve_from", "accsink_warm_start", "accsink_selftest_timeout"]
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class accsink_problem(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("m", ct.c_int32), ("d", ct.c_int32),
                ("cost_kind", ct.c_int32), ("ldc", ct.c_int64),
                ("C", ct.c_void_p), ("X", ct.c_void_p), ("Y", ct.c_void_p),
                ("a", ct.c_void_p), ("b", ct.c_void_p),
                ("cost_scale", ct.c_int32), ("reserved", ct.c_int32)]


class accsink_params(ct.Structure):
    _fields_ = [("method", ct.c_int32), ("m0", ct.c_int32), ("eps", ct.c_double),
                ("tol", ct.c_double), ("mu0", ct.c_double),
                ("max_sinkhorn_steps", ct.c_int32), ("stability", ct.c_int32),
                ("carry", ct.c_int32), ("evaluate", ct.c_int32), ("use_graph", ct.c_int32),
                ("history", ct.c_int32), ("col_transpose", ct.c_int32), ("precision", ct.c_int32)]


class accsink_result(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("sinkhorn_steps", ct.c_int32),
                ("outer_stages", ct.c_int32), ("stability_failures", ct.c_int32),
                ("marginal_l1", ct.c_double), ("transport_cost", ct.c_double),
                ("dual_objective", ct.c_double), ("cost_max", ct.c_double),
                ("gpu_ms", ct.c_double), ("loop_mode", ct.c_int32), ("reserved", ct.c_int32)]


class accsink_state(ct.Structure):
    _fields_ = [("m", ct.c_int32), ("method", ct.c_int32), ("m_stage", ct.c_int32),
                ("j_in_stage", ct.c_int32), ("stages", ct.c_int32), ("carry", ct.c_int32),
                ("eps", ct.c_double), ("mu0", ct.c_double), ("mu", ct.c_double),
                ("shift_g", ct.c_double), ("shift_f", ct.c_double), ("cost_abs", ct.c_double),
                ("cost_min", ct.c_double), ("eps_c", ct.c_double),
                ("x", ct.c_void_p), ("w", ct.c_void_p)]


class accsink_batch_config(ct.Structure):
    _fields_ = [("small_max_nm", ct.c_int32), ("row_tile_elems", ct.c_int32),
                ("ctas_per_sm", ct.c_int32), ("dense_solo_min_nm", ct.c_int32)]


class accsink_server_stats(ct.Structure):
    _fields_ = [("queued", ct.c_int64), ("solved", ct.c_int64), ("failed", ct.c_int64),
                ("batches", ct.c_int64), ("resident_bytes", ct.c_int64),
                ("peak_bytes", ct.c_int64), ("budget_bytes", ct.c_int64),
                ("busy_ms", ct.c_double)]


class AccsinkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded ``libaccsink.so`` (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libaccsink.so is missing: run __graft_entry__.build() "
                               "(the solver has no CPU fallback)")
        L = ct.CDLL(LIB_PATH)
        vp, i32, dbl = ct.c_void_p, ct.c_int32, ct.c_double
        P = ct.POINTER
        L.accsink_create.argtypes = [P(vp), ct.c_int, ct.c_size_t]
        L.accsink_create.restype = ct.c_int
        L.accsink_destroy.argtypes = [vp]
        L.accsink_destroy.restype = None
        L.accsink_last_error.argtypes = [vp]
        L.accsink_last_error.restype = ct.c_char_p
        L.accsink_params_default.argtypes = [P(accsink_params)]
        L.accsink_params_default.restype = None
        L.accsink_version.argtypes = []
        L.accsink_version.restype = ct.c_char_p
        L.accsink_solve.argtypes = [vp, P(accsink_problem), P(accsink_params), vp, vp, vp,
                                    P(accsink_result)]
        L.accsink_solve_host.argtypes = [vp, P(accsink_problem), P(accsink_params), vp, vp, vp,
                                         P(accsink_result)]
        L.accsink_get_history.argtypes = [vp, i32, vp, vp, vp, vp, vp, P(i32)]
        L.accsink_row_pass.argtypes = [vp, P(accsink_problem), dbl, vp, vp, vp]
        L.accsink_col_lse.argtypes = [vp, P(accsink_problem), dbl, vp, vp, vp]
        L.accsink_sinkhorn_map.argtypes = [vp, P(accsink_problem), dbl, vp, vp, vp, vp,
                                           P(dbl), vp]
        L.accsink_transport_cost.argtypes = [vp, P(accsink_problem), dbl, vp, vp, P(dbl), vp]
        L.accsink_time_passes.argtypes = [vp, P(accsink_problem), dbl, vp, ct.c_int, vp,
                                          P(ct.c_float), P(ct.c_float)]
        L.accsink_launch_geometry.argtypes = [vp, i32, i32, i32, P(i32)]
        L.accsink_col_lse_noalloc.argtypes = [P(accsink_problem), dbl, vp, vp, vp]
        L.accsink_plan.argtypes = [vp, P(accsink_problem), dbl, vp, vp, vp, ct.c_int64, i32, vp]
        L.accsink_barycentric.argtypes = [vp, P(accsink_problem), dbl, vp, vp, vp, i32, vp, vp]
        L.accsink_export_state.argtypes = [vp, P(accsink_state), vp]
        L.accsink_selftest_timeout.argtypes = [vp, dbl, P(i32), P(dbl)]
        L.accsink_solve_from.argtypes = [vp, P(accsink_problem), P(accsink_params),
                                         P(accsink_state), vp, vp, vp, P(accsink_result)]
        L.accsink_warm_start.argtypes = [vp, P(accsink_problem), P(accsink_params), vp, vp, vp,
                                         vp, P(accsink_result)]
        L.accsink_solve_batch.argtypes = [vp, i32, P(accsink_problem), P(accsink_params), vp,
                                          P(vp), P(vp), P(accsink_result)]
        L.accsink_batch_set_config.argtypes = [vp, P(accsink_batch_config)]
        L.accsink_batch_get_config.argtypes = [vp, P(accsink_batch_config)]
        L.accsink_batch_autotune.argtypes = [vp, i32, P(accsink_problem), P(accsink_params), vp,
                                             P(vp), P(vp), P(accsink_result),
                                             P(accsink_batch_config), P(ct.c_float), i32, P(i32)]
        L.accsink_batch_last_timing.argtypes = [vp, P(ct.c_float), P(ct.c_float), P(ct.c_float)]
        u64 = ct.c_uint64
        L.accsink_server_create.argtypes = [ct.c_int, ct.c_size_t, P(vp)]
        L.accsink_server_destroy.argtypes = [vp]
        L.accsink_server_destroy.restype = None
        L.accsink_server_last_error.argtypes = [vp]
        L.accsink_server_last_error.restype = ct.c_char_p
        L.accsink_server_submit.argtypes = [vp, P(accsink_problem), P(accsink_params), P(u64)]
        L.accsink_server_poll.argtypes = [vp, u64, P(i32)]
        L.accsink_server_wait.argtypes = [vp, u64, i32, P(accsink_result), P(dbl)]
        L.accsink_server_potentials.argtypes = [vp, u64, P(vp), P(vp)]
        L.accsink_server_copy_potentials.argtypes = [vp, u64, vp, vp]
        L.accsink_server_release.argtypes = [vp, u64]
        L.accsink_server_set_limits.argtypes = [vp, ct.c_int64]
        L.accsink_server_get_stats.argtypes = [vp, P(accsink_server_stats)]
        L.accsink_server_set_config.argtypes = [vp, P(accsink_batch_config)]
        for name in EXPORTED:
            if name not in ("accsink_destroy", "accsink_params_default", "accsink_last_error",
                            "accsink_version", "accsink_server_destroy",
                            "accsink_server_last_error"):
                getattr(L, name).restype = ct.c_int
        _lib = L
    return _lib


def default_params(**kw) -> accsink_params:
    p = accsink_params()
    lib().accsink_params_default(ct.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


def _check_dev(t, dtype, name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements")
    if not t.is_contiguous() and t.dim() == 1:
        raise ValueError(f"{name} must be contiguous")


def _check_vec(t, n, name):
    """A device FP64 array the library reads or writes n doubles of: a
    contiguous CUDA float64 tensor with at least n elements (None is left to
    the library's own null check)."""
    if t is None:
        return
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n > 0 and t.numel() < n:
        raise ValueError(f"{name} must hold at least {n} elements, has {t.numel()}")


def problem_dense(C, a=None, b=None, scale_to_max=False) -> accsink_problem:
    """Problem struct for a dense FP32 CUDA cost C (n x m, unit column stride)."""
    import torch
    _check_dev(C, torch.float32, "C")
    if C.dim() != 2 or C.stride(1) != 1:
        raise ValueError("C must be 2-D with unit column stride")
    n, m = C.shape
    pr = accsink_problem()
    pr.n, pr.m, pr.d, pr.cost_kind = n, m, 0, COST_DENSE
    pr.ldc = C.stride(0)
    pr.C = C.data_ptr()
    if a is not None:
        _check_dev(a, torch.float64, "a", n)
        pr.a = a.data_ptr()
    if b is not None:
        _check_dev(b, torch.float64, "b", m)
        pr.b = b.data_ptr()
    pr.cost_scale = SCALE_MAX_TO_ONE if scale_to_max else SCALE_NONE
    pr._keep = (C, a, b)      # the struct holds raw pointers: keep the tensors alive
    return pr


def _cost_kind(kind) -> int:
    if kind in ("sqeuclid", COST_SQEUCLID):
        return COST_SQEUCLID
    if kind in ("cosine", COST_COSINE):
        return COST_COSINE
    raise ValueError(f"unknown point-cloud cost kind {kind!r} (sqeuclid or cosine)")


def _method(method) -> int:
    if method in ("acc", ACC):
        return ACC
    if method in ("plain", PLAIN):
        return PLAIN
    raise ValueError(f"unknown method {method!r} (acc or plain)")


def problem_points(X, Y, kind="sqeuclid", a=None, b=None, scale_to_max=False) -> accsink_problem:
    """Problem struct for a point-cloud cost formed on the fly from FP32 CUDA
    point clouds X (n x d) and Y (m x d), row-major and contiguous:
    kind "sqeuclid" (||x_i - y_j||^2) or "cosine" (1 - <x_i, y_j>)."""
    import torch
    cost_kind = _cost_kind(kind)
    _check_dev(X, torch.float32, "X")
    _check_dev(Y, torch.float32, "Y")
    if X.dim() != 2 or Y.dim() != 2 or X.shape[1] != Y.shape[1]:
        raise ValueError("X and Y must be 2-D with the same number of columns")
    if not (X.is_contiguous() and Y.is_contiguous()):
        raise ValueError("X and Y must be contiguous")
    n, d = X.shape
    m = Y.shape[0]
    pr = accsink_problem()
    pr.n, pr.m, pr.d = n, m, d
    pr.cost_kind = cost_kind
    pr.X = X.data_ptr()
    pr.Y = Y.data_ptr()
    if a is not None:
        _check_dev(a, torch.float64, "a", n)
        pr.a = a.data_ptr()
    if b is not None:
        _check_dev(b, torch.float64, "b", m)
        pr.b = b.data_ptr()
    pr.cost_scale = SCALE_MAX_TO_ONE if scale_to_max else SCALE_NONE
    pr._keep = (X, Y, a, b)
    return pr


class Context:
    """An accsink context on one CUDA device (wraps accsink_create/destroy)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self._h = ct.c_void_p()
        rc = lib().accsink_create(ct.byref(self._h), int(device), int(mem_budget_bytes))
        if rc != OK:
            raise AccsinkError(rc, "accsink_create failed")
        self.device = device

    def close(self):
        if self._h:
            lib().accsink_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_error(self) -> str:
        return lib().accsink_last_error(self._h).decode()

    def _raise(self, rc, allow=(OK,)):
        if rc not in allow:
            raise AccsinkError(rc, self.last_error())
        return rc

    # ---- whole solves --------------------------------------------------
    def accsink_solve(self, prob: accsink_problem, params: accsink_params, f_out, g_out,
                      stream=None, allow_maxiter=True) -> accsink_result:
        _check_vec(f_out, prob.n, "f_out")
        _check_vec(g_out, prob.m, "g_out")
        res = accsink_result()
        rc = lib().accsink_solve(self._h, ct.byref(prob), ct.byref(params), _stream_ptr(stream),
                                 _ptr(f_out), _ptr(g_out), ct.byref(res))
        self._raise(rc, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
        return res

    def accsink_solve_host(self, C, a, b, params: accsink_params, f_out, g_out,
                           scale_to_max=False, stream=None, allow_maxiter=True,
                           X=None, Y=None, kind="sqeuclid") -> accsink_result:
        """C, a, b, f_out, g_out: host numpy arrays (FP32 C, FP64 vectors).
        With C None, the cost is formed from the FP32 host point clouds X, Y."""
        import numpy as np
        pr = accsink_problem()
        if C is not None:
            if C.dtype != np.float32 or not C.flags.c_contiguous or C.ndim != 2:
                raise TypeError("C must be a contiguous 2-D float32 array")
            n, m = C.shape
            pr.n, pr.m, pr.cost_kind, pr.ldc = n, m, COST_DENSE, m
            pr.C = C.ctypes.data
        else:
            for nm_, arr in (("X", X), ("Y", Y)):
                if arr is None or arr.dtype != np.float32 or not arr.flags.c_contiguous or arr.ndim != 2:
                    raise TypeError(f"{nm_} must be a contiguous 2-D float32 array")
            pr.n, pr.d = X.shape
            pr.m = Y.shape[0]
            pr.cost_kind = _cost_kind(kind)
            pr.X = X.ctypes.data
            pr.Y = Y.ctypes.data
        pr.a = np.ascontiguousarray(a, np.float64).ctypes.data if a.dtype == np.float64 and a.flags.c_contiguous else None
        pr.b = np.ascontiguousarray(b, np.float64).ctypes.data if b.dtype == np.float64 and b.flags.c_contiguous else None
        if pr.a is None or pr.b is None:
            raise TypeError("a and b must be contiguous float64 arrays")
        pr.cost_scale = SCALE_MAX_TO_ONE if scale_to_max else SCALE_NONE
        res = accsink_result()
        rc = lib().accsink_solve_host(self._h, ct.byref(pr), ct.byref(params),
                                      _stream_ptr(stream), ct.c_void_p(f_out.ctypes.data),
                                      ct.c_void_p(g_out.ctypes.data), ct.byref(res))
        self._raise(rc, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
        return res

    # ---- batches ------------------------------------------------------
    @staticmethod
    def _batch_arrays(probs, params, f_outs, g_outs):
        k = len(probs)
        if not (len(params) == len(f_outs) == len(g_outs) == k):
            raise ValueError("probs, params, f_outs and g_outs must have the same length")
        for i in range(k):
            _check_vec(f_outs[i], probs[i].n, f"f_outs[{i}]")
            _check_vec(g_outs[i], probs[i].m, f"g_outs[{i}]")
        pa = (accsink_problem * k)(*probs)
        qa = (accsink_params * k)(*params)
        fa = (ct.c_void_p * k)(*[_ptr(t) for t in f_outs])
        ga = (ct.c_void_p * k)(*[_ptr(t) for t in g_outs])
        ra = (accsink_result * k)()
        return k, pa, qa, fa, ga, ra

    def accsink_solve_batch(self, probs, params, f_outs, g_outs, stream=None,
                            allow_maxiter=True):
        """probs/params: lists of structs (device pointers inside); f_outs,
        g_outs: lists of FP64 CUDA tensors. Returns the list of results."""
        k, pa, qa, fa, ga, ra = self._batch_arrays(probs, params, f_outs, g_outs)
        rc = lib().accsink_solve_batch(self._h, k, pa, qa, _stream_ptr(stream), fa, ga, ra)
        self._raise(rc, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
        return [ra[i] for i in range(k)]

    def accsink_batch_set_config(self, small_max_nm=0, row_tile_elems=0, ctas_per_sm=0,
                                 dense_solo_min_nm=0):
        c = accsink_batch_config(small_max_nm, row_tile_elems, ctas_per_sm, dense_solo_min_nm)
        self._raise(lib().accsink_batch_set_config(self._h, ct.byref(c)))

    def accsink_batch_get_config(self) -> dict:
        c = accsink_batch_config()
        self._raise(lib().accsink_batch_get_config(self._h, ct.byref(c)))
        return {"small_max_nm": c.small_max_nm, "row_tile_elems": c.row_tile_elems,
                "ctas_per_sm": c.ctas_per_sm, "dense_solo_min_nm": c.dense_solo_min_nm}

    def accsink_batch_autotune(self, probs, params, f_outs, g_outs, stream=None):
        k, pa, qa, fa, ga, ra = self._batch_arrays(probs, params, f_outs, g_outs)
        best = accsink_batch_config()
        times = (ct.c_float * 64)()
        tried = ct.c_int32()
        rc = lib().accsink_batch_autotune(self._h, k, pa, qa, _stream_ptr(stream), fa, ga, ra,
                                          ct.byref(best), times, 64, ct.byref(tried))
        self._raise(rc)
        return ({"small_max_nm": best.small_max_nm, "row_tile_elems": best.row_tile_elems,
                 "ctas_per_sm": best.ctas_per_sm, "dense_solo_min_nm": best.dense_solo_min_nm},
                list(times)[:tried.value])

    def accsink_batch_last_timing(self):
        t, f, s = ct.c_float(), ct.c_float(), ct.c_float()
        self._raise(lib().accsink_batch_last_timing(self._h, ct.byref(t), ct.byref(f), ct.byref(s)))
        return {"total_ms": t.value, "form_ms": f.value, "solve_ms": s.value}

    def accsink_get_history(self, capacity: int):
        import numpy as np
        err = np.zeros(capacity); dual = np.zeros(capacity); mu = np.zeros(capacity)
        stab = np.zeros(capacity, np.int32); cond = np.zeros((capacity, 4))
        cnt = ct.c_int32()
        rc = lib().accsink_get_history(self._h, capacity, ct.c_void_p(err.ctypes.data),
                                       ct.c_void_p(dual.ctypes.data), ct.c_void_p(mu.ctypes.data),
                                       ct.c_void_p(stab.ctypes.data), ct.c_void_p(cond.ctypes.data),
                                       ct.byref(cnt))
        self._raise(rc)
        k = cnt.value
        return {"err": err[:k], "dual": dual[:k], "mu": mu[:k], "stab": stab[:k], "cond": cond[:k]}

    # ---- single passes -------------------------------------------------
    def accsink_row_pass(self, prob, eps, g, f_out, stream=None):
        _check_vec(g, prob.m, "g")
        _check_vec(f_out, prob.n, "f_out")
        self._raise(lib().accsink_row_pass(self._h, ct.byref(prob), float(eps), _ptr(g),
                                           _ptr(f_out), _stream_ptr(stream)))

    def accsink_col_lse(self, prob, eps, f, ell_out, stream=None):
        _check_vec(f, prob.n, "f")
        _check_vec(ell_out, prob.m, "ell_out")
        self._raise(lib().accsink_col_lse(self._h, ct.byref(prob), float(eps), _ptr(f),
                                          _ptr(ell_out), _stream_ptr(stream)))

    def accsink_sinkhorn_map(self, prob, eps, g, f_out, c_out, s_out, stream=None) -> float:
        _check_vec(g, prob.m, "g")
        _check_vec(f_out, prob.n, "f_out")
        _check_vec(c_out, prob.m, "c_out")
        _check_vec(s_out, prob.m, "s_out")
        err = ct.c_double()
        self._raise(lib().accsink_sinkhorn_map(self._h, ct.byref(prob), float(eps), _ptr(g),
                                               _ptr(f_out), _ptr(c_out), _ptr(s_out),
                                               ct.byref(err), _stream_ptr(stream)))
        return err.value

    def accsink_transport_cost(self, prob, eps, f, g, stream=None) -> float:
        _check_vec(f, prob.n, "f")
        _check_vec(g, prob.m, "g")
        out = ct.c_double()
        self._raise(lib().accsink_transport_cost(self._h, ct.byref(prob), float(eps), _ptr(f),
                                                 _ptr(g), ct.byref(out), _stream_ptr(stream)))
        return out.value

    def accsink_selftest_timeout(self, limit_s):
        """Runs the bounded-barrier failure path; returns (status, seconds)."""
        st, el = ct.c_int32(), ct.c_double()
        self._raise(lib().accsink_selftest_timeout(self._h, float(limit_s), ct.byref(st),
                                                   ct.byref(el)))
        return st.value, el.value

    def accsink_export_state(self, x, w, stream=None) -> accsink_state:
        """State of the last solve on this context; x, w: device FP64 arrays of
        length m that receive the iterate and the momentum."""
        _check_vec(x, 0, "x")
        _check_vec(w, int(x.numel()), "w")
        st = accsink_state()
        st.m = int(x.numel())
        st.x = _ptr(x)
        st.w = _ptr(w)
        self._raise(lib().accsink_export_state(self._h, ct.byref(st), _stream_ptr(stream)))
        return st

    def accsink_solve_from(self, prob, params, state: accsink_state, f_out, g_out, stream=None,
                           allow_maxiter=True) -> accsink_result:
        _check_vec(f_out, prob.n, "f_out")
        _check_vec(g_out, prob.m, "g_out")
        res = accsink_result()
        rc = lib().accsink_solve_from(self._h, ct.byref(prob), ct.byref(params), ct.byref(state),
                                      _stream_ptr(stream), _ptr(f_out), _ptr(g_out),
                                      ct.byref(res))
        self._raise(rc, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
        return res

    def accsink_warm_start(self, prob, params, g0, f_out, g_out, stream=None,
                           allow_maxiter=True) -> accsink_result:
        _check_vec(g0, prob.m, "g0")
        _check_vec(f_out, prob.n, "f_out")
        _check_vec(g_out, prob.m, "g_out")
        res = accsink_result()
        rc = lib().accsink_warm_start(self._h, ct.byref(prob), ct.byref(params), _ptr(g0),
                                      _stream_ptr(stream), _ptr(f_out), _ptr(g_out),
                                      ct.byref(res))
        self._raise(rc, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
        return res

    def accsink_plan(self, prob, eps, f, g, P_out, stream=None):
        """P_out: a CUDA float32 or float64 tensor (n x >= m, unit column stride)."""
        import torch
        _check_vec(f, prob.n, "f")
        _check_vec(g, prob.m, "g")
        if (not isinstance(P_out, torch.Tensor) or not P_out.is_cuda
                or P_out.dtype not in (torch.float32, torch.float64)):
            raise TypeError("P_out must be a CUDA float32 or float64 tensor")
        if (P_out.dim() != 2 or P_out.shape[0] < prob.n or P_out.shape[1] < prob.m
                or P_out.stride(1) != 1 or P_out.stride(0) < prob.m):
            raise ValueError("P_out must be n x m (or larger) with unit column stride")
        dtype = 1 if P_out.dtype == torch.float64 else 0
        self._raise(lib().accsink_plan(self._h, ct.byref(prob), float(eps), _ptr(f), _ptr(g),
                                       _ptr(P_out), int(P_out.stride(0)), dtype,
                                       _stream_ptr(stream)))

    def accsink_barycentric(self, prob, eps, f, g, Z, out, stream=None):
        """Z: CUDA float32 (m x dz, row-major); out: CUDA float64 (n x dz)."""
        import torch
        _check_vec(f, prob.n, "f")
        _check_vec(g, prob.m, "g")
        if (not isinstance(Z, torch.Tensor) or not Z.is_cuda or Z.dtype != torch.float32
                or Z.dim() != 2 or Z.shape[0] < prob.m or not Z.is_contiguous()):
            raise TypeError("Z must be a contiguous CUDA float32 tensor of m rows")
        if (not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64
                or not out.is_contiguous() or out.numel() < prob.n * Z.shape[1]):
            raise TypeError("out must be a contiguous CUDA float64 tensor of n x dz elements")
        self._raise(lib().accsink_barycentric(self._h, ct.byref(prob), float(eps), _ptr(f),
                                              _ptr(g), _ptr(Z), int(Z.shape[1]), _ptr(out),
                                              _stream_ptr(stream)))

    def accsink_time_passes(self, prob, eps, g, reps, stream=None):
        r, c = ct.c_float(), ct.c_float()
        self._raise(lib().accsink_time_passes(self._h, ct.byref(prob), float(eps), _ptr(g),
                                              int(reps), _stream_ptr(stream), ct.byref(r),
                                              ct.byref(c)))
        return r.value, c.value

    def accsink_launch_geometry(self, n, m, vec=1):
        out = (ct.c_int32 * 6)()
        self._raise(lib().accsink_launch_geometry(self._h, int(n), int(m), int(vec), out))
        keys = ["num_sms", "row_grid", "col_splits", "col_strips", "step_grid", "stat_grid"]
        return dict(zip(keys, list(out)))


def problem_host(a, b, C=None, X=None, Y=None, kind="sqeuclid", scale_to_max=False):
    """Problem struct over HOST numpy arrays (for accsink_server_submit): FP32
    C or point clouds X, Y (row-major, contiguous), FP64 a, b."""
    import numpy as np
    pr = accsink_problem()
    keep = []

    def host(arr, dtype):
        arr = np.ascontiguousarray(arr, dtype=dtype)
        keep.append(arr)
        return arr.ctypes.data

    pr.a = host(a, np.float64)
    pr.b = host(b, np.float64)
    if C is not None:
        pr.n, pr.m = C.shape
        pr.cost_kind = COST_DENSE
        pr.ldc = C.shape[1]
        pr.C = host(C, np.float32)
    else:
        pr.n, pr.d = X.shape
        pr.m = Y.shape[0]
        pr.cost_kind = _cost_kind(kind)
        pr.X = host(X, np.float32)
        pr.Y = host(Y, np.float32)
    pr.cost_scale = SCALE_MAX_TO_ONE if scale_to_max else SCALE_NONE
    pr._keep = keep
    return pr


class Server:
    """The request server of include/accsink.h (thread-safe). Each submitted
    problem's host arrays are kept alive here until its ticket is released."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 64 << 30):
        self._h = ct.c_void_p()
        rc = lib().accsink_server_create(int(device), int(mem_budget_bytes), ct.byref(self._h))
        if rc != OK:
            raise AccsinkError(rc, "accsink_server_create failed")
        self._keep = {}

    def close(self):
        if self._h:
            lib().accsink_server_destroy(self._h)
            self._h = ct.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().accsink_server_last_error(self._h).decode()

    def submit(self, prob: accsink_problem, params: accsink_params) -> int:
        t = ct.c_uint64()
        rc = lib().accsink_server_submit(self._h, ct.byref(prob), ct.byref(params), ct.byref(t))
        if rc != OK:
            raise AccsinkError(rc, "accsink_server_submit rejected the request")
        self._keep[t.value] = prob
        return t.value

    def poll(self, ticket: int) -> int:
        st = ct.c_int32()
        rc = lib().accsink_server_poll(self._h, ticket, ct.byref(st))
        if rc != OK:
            raise AccsinkError(rc, "unknown ticket")
        return st.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (status, result, latency_ms); status ERR_TIMEOUT when the
        wait ran out."""
        res = accsink_result()
        lat = ct.c_double()
        rc = lib().accsink_server_wait(self._h, ticket, int(timeout_ms), ct.byref(res),
                                       ct.byref(lat))
        return rc, res, lat.value

    def potentials_dev(self, ticket: int):
        f, g = ct.c_void_p(), ct.c_void_p()
        rc = lib().accsink_server_potentials(self._h, ticket, ct.byref(f), ct.byref(g))
        if rc != OK:
            raise AccsinkError(rc, "ticket is not DONE")
        return f.value, g.value

    def copy_potentials(self, ticket: int):
        import numpy as np
        pr = self._keep[ticket]
        f = np.empty(pr.n)
        g = np.empty(pr.m)
        rc = lib().accsink_server_copy_potentials(self._h, ticket, ct.c_void_p(f.ctypes.data),
                                                  ct.c_void_p(g.ctypes.data))
        if rc != OK:
            raise AccsinkError(rc, "ticket is not DONE")
        return f, g

    def release(self, ticket: int):
        rc = lib().accsink_server_release(self._h, ticket)
        if rc != OK:
            raise AccsinkError(rc, "ticket cannot be released")
        self._keep.pop(ticket, None)

    def set_limits(self, max_group_entries: int):
        """Cost entries (sum of n m) one admitted group may hold (0: no limit)."""
        rc = lib().accsink_server_set_limits(self._h, int(max_group_entries))
        if rc != OK:
            raise AccsinkError(rc, "bad server limit")

    def stats(self) -> dict:
        s = accsink_server_stats()
        rc = lib().accsink_server_get_stats(self._h, ct.byref(s))
        if rc != OK:
            raise AccsinkError(rc, "stats failed")
        return {k: getattr(s, k) for k, _ in accsink_server_stats._fields_}

    def set_config(self, small_max_nm=0, row_tile_elems=0, ctas_per_sm=0):
        c = accsink_batch_config(small_max_nm, row_tile_elems, ctas_per_sm, 0)
        rc = lib().accsink_server_set_config(self._h, ct.byref(c))
        if rc != OK:
            raise AccsinkError(rc, "bad config")


def accsink_col_lse_noalloc(prob: accsink_problem, eps, f, ell_out, stream=None) -> int:
    """Context-free column log-sum-exp pass that allocates nothing (see the
    header); returns the accsink status code. f and ell_out are checked like
    every other device vector (CUDA float64, contiguous, n and m elements)."""
    _check_vec(f, prob.n, "f")
    _check_vec(ell_out, prob.m, "ell_out")
    return lib().accsink_col_lse_noalloc(ct.byref(prob), float(eps), _ptr(f), _ptr(ell_out),
                                         _stream_ptr(stream))


def result_dict(res: accsink_result) -> dict:
    return {k: getattr(res, k) for k, _ in accsink_result._fields_}


def solve_points(X, Y, a, b, eps, kind="sqeuclid", tol=1e-6, method="acc", scale_to_max=False,
                 ctx: Context | None = None, stream=None, **params):
    """Convenience: solve a point-cloud problem held in CUDA tensors.

    Returns (f, g, result dict) with f, g FP64 CUDA tensors in cost units."""
    import torch
    meth = _method(method)
    own = ctx is None
    ctx = ctx or Context(X.device.index or 0)
    try:
        prob = problem_points(X, Y, kind, a, b, scale_to_max)
        p = default_params(eps=float(eps), tol=float(tol), method=meth, **params)
        f = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        g = torch.empty(Y.shape[0], dtype=torch.float64, device=X.device)
        res = ctx.accsink_solve(prob, p, f, g, stream=stream)
        return f, g, result_dict(res)
    finally:
        if own:
            ctx.close()


def solve(C, a, b, eps, tol=1e-6, method="acc", scale_to_max=False, ctx: Context | None = None,
          stream=None, **params):
    """Convenience: solve a dense problem held in CUDA tensors.

    Returns (f, g, result dict) with f, g FP64 CUDA tensors in cost units."""
    import torch
    meth = _method(method)
    own = ctx is None
    ctx = ctx or Context(C.device.index or 0)
    try:
        prob = problem_dense(C, a, b, scale_to_max)
        p = default_params(eps=float(eps), tol=float(tol), method=meth, **params)
        f = torch.empty(C.shape[0], dtype=torch.float64, device=C.device)
        g = torch.empty(C.shape[1], dtype=torch.float64, device=C.device)
        res = ctx.accsink_solve(prob, p, f, g, stream=stream)
        return f, g, result_dict(res)
    finally:
        if own:
            ctx.close()
