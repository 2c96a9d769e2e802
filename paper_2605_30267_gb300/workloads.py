"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random problems; it contains none of the solver's
arithmetic. Both the GPU path and the FP64 oracle consume exactly what it
returns, so it imports neither.

The paper's own data (two photographs for colour transfer, fastText/MUSE
word vectors for alignment) are not available here; the generators below
stand in for them with the same shapes, cost kinds and marginal types:

* ``sqeuclid_points`` problems: RGB-like clouds in [0,1]^3 or Gaussian
  mixtures, cost ||x - y||^2 divided by its maximum (Sec. 5, colour transfer).
* ``cosine`` problems: unit-norm Gaussian vectors in R^300, cost 1 - <x, y>
  (Sec. 5, word alignment).
* marginals uniform (Sec. 5) or Dirichlet(1) (normalised i.i.d. Exp(1)).

All draws use numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_points(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n i.i.d. points uniform in [0,1]^d, FP32."""
    return g.random((n, d)).astype(np.float32)


def gmm_points(g: np.random.Generator, n: int, d: int, k: int, sigma: float,
               clip01: bool = False) -> np.ndarray:
    """n points from a k-component isotropic Gaussian mixture in R^d with
    equal weights, means uniform in [0,1]^d and std ``sigma``; FP32."""
    means = g.random((k, d))
    comp = g.integers(0, k, size=n)
    pts = means[comp] + sigma * g.standard_normal((n, d))
    if clip01:
        pts = np.clip(pts, 0.0, 1.0)
    return pts.astype(np.float32)


def unit_gaussian_points(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n standard Gaussian vectors in R^d scaled to unit norm (in FP64), FP32."""
    v = g.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


def dirichlet1(g: np.random.Generator, n: int) -> np.ndarray:
    """A Dirichlet(1,...,1) probability vector (normalised Exp(1) draws), FP64."""
    e = g.exponential(1.0, size=n)
    return e / e.sum()


def uniform_marginal(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n)


def sqeuclid_cost_fp32(X: np.ndarray, Y: np.ndarray, scale_to_max: bool = True,
                       block: int = 2048) -> np.ndarray:
    """Dense cost C_ij = ||x_i - y_j||^2 formed in FP64 from the FP32 points,
    optionally divided by its maximum entry, then rounded once to FP32.

    This is input construction: the FP32 matrix it returns *is* the problem
    both solvers are given."""
    X64 = X.astype(np.float64)
    Y64 = Y.astype(np.float64)
    x2 = (X64 * X64).sum(1)
    y2 = (Y64 * Y64).sum(1)
    n, m = X.shape[0], Y.shape[0]

    def blockc(i0, i1):
        c = x2[i0:i1, None] + y2[None, :] - 2.0 * (X64[i0:i1] @ Y64.T)
        np.maximum(c, 0.0, out=c)
        return c

    mx = 1.0
    if scale_to_max:
        mx = 0.0
        for i0 in range(0, n, block):
            mx = max(mx, float(blockc(i0, min(n, i0 + block)).max()))
    out = np.empty((n, m), np.float32)
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        c = blockc(i0, i1)
        if scale_to_max:
            c /= mx
        out[i0:i1] = c
    return out


def uniform_dense_cost(g: np.random.Generator, n: int, m: int) -> np.ndarray:
    """Synthetic-experiment cost of Sec. 5: i.i.d. U[0,1] entries rescaled to
    unit total mass, FP32."""
    c = g.random((n, m))
    c /= c.sum()
    return c.astype(np.float32)


# --------------------------------------------------------------------------
# The benchmark problems.
# --------------------------------------------------------------------------

def small_pointcloud_problem(seed: int = 0, n: int = 256, m: int | None = None,
                             d: int = 2, eps: float = 1e-2, tol: float = 1e-6) -> dict:
    """Uniform points in [0,1]^d, squared-Euclidean cost scaled to max 1,
    uniform marginals (n = m = 256, d = 2, eps = 1e-2 by default)."""
    m = n if m is None else m
    g = rng(seed)
    X = uniform_points(g, n, d)
    Y = uniform_points(g, m, d)
    return {"C": sqeuclid_cost_fp32(X, Y), "a": uniform_marginal(n),
            "b": uniform_marginal(m), "eps": eps, "tol": tol, "X": X, "Y": Y,
            "name": f"uniform-{d}d-sqeuclid n={n} m={m}"}


def gmm_stored_cost_problem(seed: int = 0, n: int = 16384, m: int | None = None,
                            eps: float = 1e-2, tol: float = 1e-6,
                            with_cost: bool = True) -> dict:
    """Stored-cost problem: X and Y each from an 8-component Gaussian mixture
    in R^3 (sigma 0.05, means uniform in [0,1]^3), dense FP32 squared-Euclidean
    cost scaled to max 1, Dirichlet(1) marginals."""
    m = n if m is None else m
    g = rng(seed)
    X = gmm_points(g, n, 3, 8, 0.05)
    Y = gmm_points(g, m, 3, 8, 0.05)
    a = dirichlet1(g, n)
    b = dirichlet1(g, m)
    C = sqeuclid_cost_fp32(X, Y) if with_cost else None
    return {"C": C, "a": a, "b": b, "eps": eps, "tol": tol, "X": X, "Y": Y,
            "name": f"gmm8-r3-sqeuclid-dense n={n} m={m}"}


def color_transfer_problem(seed: int = 0, n: int = 65536, eps: float = 1e-3,
                           tol: float = 1e-6) -> dict:
    """Colour-transfer-shaped point clouds: source uniform in [0,1]^3, target
    a 16-cluster mixture (sigma 0.03) clipped to [0,1]^3; uniform marginals."""
    g = rng(seed)
    X = uniform_points(g, n, 3)
    Y = gmm_points(g, n, 3, 16, 0.03, clip01=True)
    return {"X": X, "Y": Y, "a": uniform_marginal(n), "b": uniform_marginal(n),
            "eps": eps, "tol": tol, "name": f"rgb-colour-transfer n=m={n}"}


def word_alignment_batch(seed: int = 0, count: int = 512, lo: int = 16, hi: int = 2048,
                         d: int = 300, eps_lo: float = 0.005, eps_hi: float = 0.05,
                         tol: float = 1e-6) -> list[dict]:
    """Batch of word-alignment-shaped problems: n, m log-uniform in [lo, hi],
    unit-norm Gaussian points in R^d, cosine cost, Dirichlet(1) marginals,
    eps uniform in [eps_lo, eps_hi]."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        m = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        X = unit_gaussian_points(g, n, d)
        Y = unit_gaussian_points(g, m, d)
        out.append({"X": X, "Y": Y, "a": dirichlet1(g, n), "b": dirichlet1(g, m),
                    "eps": float(g.uniform(eps_lo, eps_hi)), "tol": tol})
    return out


def paper_synthetic_problem(seed: int = 0, n: int = 100, m: int = 50, eps: float = 1e-2,
                            tol: float = 1e-6) -> dict:
    """The synthetic experiment of Sec. 5: a, b with i.i.d. U[0,1] entries
    normalised; C i.i.d. U[0,1] rescaled to unit total."""
    g = rng(seed)
    a = g.random(n)
    b = g.random(m)
    C = uniform_dense_cost(g, n, m)
    return {"C": C, "a": a / a.sum(), "b": b / b.sum(), "eps": eps, "tol": tol,
            "name": f"paper-synthetic n={n} m={m}"}


def serving_requests(seed: int = 0, count: int = 64, lo: int = 64, hi: int = 16384,
                     d_lo: int = 2, d_hi: int = 64, eps_lo: float = 1e-3, eps_hi: float = 1e-1,
                     tol: float = 1e-6) -> list[dict]:
    """Requests of the serving workload: squared-Euclidean problems with
    points uniform in [0,1]^d, d uniform in {d_lo..d_hi}, n and m
    independently log-uniform in [lo, hi], Dirichlet(1) marginals, eps
    log-uniform in [eps_lo, eps_hi], cost scaled to max 1."""
    g = rng(seed)
    out = []
    for _ in range(count):
        d = int(g.integers(d_lo, d_hi + 1))
        n = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        m = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        out.append({"X": uniform_points(g, n, d), "Y": uniform_points(g, m, d),
                    "a": dirichlet1(g, n), "b": dirichlet1(g, m),
                    "eps": float(math.exp(g.uniform(math.log(eps_lo), math.log(eps_hi)))),
                    "tol": tol})
    return out


def poisson_arrivals(seed: int, rate: float, count: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate, size=count))
