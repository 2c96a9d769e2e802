"""Shared checks of a GPU solve against the FP64 oracle (imported by the GPU
parity tests)."""
import numpy as np

import oracle as O


def check_steps(cost, a, b, eps, tol, okw, rs, gs):
    """Step counts agree within 2% (at least one step). A larger difference
    is accepted only at a knife edge of the stopping test (Sec. 5 eq. l1tol):
    at the earlier of the two stopping steps the oracle's own marginal error
    lies within 1% of tol, so the GPU's ~1e-3 relative arithmetic difference
    decides on which side of tol that step falls (after which Acc-Sinkhorn's
    error can oscillate for several steps before crossing again)."""
    if abs(gs - rs) <= max(1, int(0.02 * rs)):
        return
    k = min(gs, rs)
    o = O.solve(cost, a, b, eps, 1e-300, max_steps=k, history=k, **okw)
    e = o["history"]["err"][k - 1]
    assert abs(e - tol) <= 0.01 * tol, ("step counts differ beyond 2% away from a knife edge",
                                        gs, rs, e)


def same_iterate(cost, a, b, eps, okw, ref, gs):
    """The oracle's iterate after gs steps (the GPU's stopping step)."""
    if ref["sinkhorn_steps"] == gs:
        return ref
    return dict(O.solve(cost, a, b, eps, 1e-300, max_steps=gs, **okw), status=ref["status"])


def centred_gap(f, g, ref):
    """max |potential difference| after shifting g to the oracle's mean."""
    sh = g.mean() - ref["g"].mean()
    return max(np.abs(g - sh - ref["g"]).max(), np.abs(f + sh - ref["f"]).max())
