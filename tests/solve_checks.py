"""Shared checks of a GPU solve against the FP64 oracle (imported by the GPU
parity tests).

Stopping (Sec. 5 eq. l1tol). The library tests the FP64 sum of the column
errors that its FP32 passes give and stops once it is below tol - 2^-22 (the
guard band its header documents for the FP32 path's error in that estimate
and in the row marginal). The oracle's own errors are exact to FP64
rounding, so the step-count comparison runs the oracle with the same
threshold, and the FP64 truth of the GPU's returned potentials, row plus
column error, must be below tol itself."""
import warnings

import numpy as np

import oracle as O

STOP_GUARD = 2.0 ** -22
KNIFE_EDGE = 0.08


def stop_tol(tol):
    """The threshold the library's stopping test applies to its estimate."""
    return tol - STOP_GUARD


class KnifeEdgeWarning(UserWarning):
    """Step counts differ beyond 2% at a knife edge of the stopping test."""


def check_steps(cost, a, b, eps, tol, okw, rs, gs):
    """Step counts agree within 2% (at least one step). A larger difference
    is accepted only at a knife edge of the stopping test (Sec. 5 eq. l1tol):
    at the earlier of the two stopping steps the oracle's own marginal error
    lies within KNIFE_EDGE (relative) of the threshold. The GPU tests its
    estimate of that error from the FP32 passes, which differs from the FP64
    value at the same potentials by up to 5.3% of it (measured on GB300 over
    the stored-cost parity cases at tol = 1e-6), so within that band the
    arithmetic decides on which side of the threshold the step falls, after
    which Acc-Sinkhorn's error can oscillate for several steps before
    crossing again. Every use of the exemption is reported as a
    KnifeEdgeWarning."""
    if abs(gs - rs) <= max(1, int(0.02 * rs)):
        return
    t = stop_tol(tol)
    k = min(gs, rs)
    o = O.solve(cost, a, b, eps, 1e-300, max_steps=k, history=k, **okw)
    e = o["history"]["err"][k - 1]
    assert abs(e - t) <= KNIFE_EDGE * t, ("step counts differ beyond 2% away from a knife edge",
                                          gs, rs, e)
    warnings.warn(KnifeEdgeWarning(
        f"knife-edge exemption used: gpu steps {gs}, oracle steps {rs}, oracle error "
        f"{e:.6e} at step {k} against the threshold {t:.6e}"))


def check_truth(ev, tol):
    """FP64 truth of eq. l1tol at the GPU's potentials: row plus column error
    below tol, and the row error at the FP32 floor."""
    assert ev["row_l1"] + ev["col_l1"] < tol, ev
    assert ev["row_l1"] <= 2e-7, ev


def same_iterate(cost, a, b, eps, okw, ref, gs):
    """The oracle's iterate after gs steps (the GPU's stopping step)."""
    if ref["sinkhorn_steps"] == gs:
        return ref
    return dict(O.solve(cost, a, b, eps, 1e-300, max_steps=gs, **okw), status=ref["status"])


def centred_gap(f, g, ref):
    """max |potential difference| after shifting g to the oracle's mean."""
    sh = g.mean() - ref["g"].mean()
    return max(np.abs(g - sh - ref["g"]).max(), np.abs(f + sh - ref["f"]).max())
