"""CPU checks of the arithmetic the tensor-core formation of batched cosine
costs relies on (the error-free splitting of Ozaki, Ogita, Oishi and Rump):

  x_k = 2^e sum_{l<6} q_{l,k} 2^{-7(l+1)} + r_k,  2^{e-1} <= max|x_k| < 2^e,

rounding to nearest at each level in FP32, as the slicing kernel does. For
the products of slice pairs grouped by class c = i + j:
  * every slice is an integer in [-128, 128] (exact in FP16);
  * every class sum, and every partial sum of its terms, is an integer of
    magnitude below 2^24 for d <= 480 (so an FP32 accumulator holds it
    exactly, whatever the order of the additions);
  * the six classes reproduce <x, y> to within d 2^-39 |x| |y|.
The exact dot product is math.fsum of the FP32 products (exact in FP64).
"""
import math

import numpy as np

BETA, LEVELS = 7, 6


def slices(x):
    x = np.asarray(x, dtype=np.float32)
    amax = float(np.max(np.abs(x)))
    if not amax >= 2.0 ** -60:
        return 0, [np.zeros(x.shape, dtype=np.int64) for _ in range(LEVELS)]
    e = math.frexp(amax)[1]
    t = np.ldexp(x, -e).astype(np.float32)              # exact power-of-two scaling
    qs = []
    for _ in range(LEVELS):
        w = (t * np.float32(1 << BETA)).astype(np.float32)
        q = np.rint(w).astype(np.float32)                 # round half to even, as rintf
        t = (w - q).astype(np.float32)
        qs.append(q.astype(np.int64))
    return e, qs


def class_sums(qx, qy):
    return [sum(int(np.dot(qx[i], qy[c - i])) for i in range(c + 1)) for c in range(LEVELS)]


def model_dot(x, y):
    ex, qx = slices(x)
    ey, qy = slices(y)
    cs = class_sums(qx, qy)
    val = math.fsum(math.ldexp(float(s), ex + ey - 2 * BETA - BETA * c) for c, s in enumerate(cs))
    return val, qx, qy, cs


def exact_dot(x, y):
    return math.fsum(float(a) * float(b) for a, b in
                     zip(np.asarray(x, np.float32), np.asarray(y, np.float32)))


def check(x, y):
    d = len(x)
    val, qx, qy, cs = model_dot(x, y)
    for q in qx + qy:
        assert np.all(np.abs(q) <= 128)
    for c, s in enumerate(cs):
        # the bound on every partial sum: the sum of the terms' magnitudes
        mag = sum(int(np.dot(np.abs(qx[i]), np.abs(qy[c - i]))) for i in range(c + 1))
        assert abs(s) <= mag < 2 ** 24, (c, mag)
    nx = math.sqrt(math.fsum(float(v) ** 2 for v in np.asarray(x, np.float32)))
    ny = math.sqrt(math.fsum(float(v) ** 2 for v in np.asarray(y, np.float32)))
    err = abs(val - exact_dot(x, y))
    assert err <= d * 2.0 ** -39 * nx * ny + 1e-300, (err, d * 2.0 ** -39 * nx * ny)
    return err / max(nx * ny, 1e-300)


def test_random_unit_vectors_d300():
    g = np.random.default_rng(1)
    worst = 0.0
    for _ in range(40):
        x = g.standard_normal(300)
        y = g.standard_normal(300)
        worst = max(worst, check(x / np.linalg.norm(x), y / np.linalg.norm(y)))
    assert worst < 2.0 ** -38      # typical errors sit far inside the d 2^-39 bound


def test_class_sums_stay_below_2_24_at_d480():
    """Components all just below the exponent's power of two (slice 0 at
    +-128) with equal signs in x and y: the largest class sums the slicing
    can produce at the maximum d."""
    d = 480
    g = np.random.default_rng(2)
    for trial in range(20):
        mags = np.float32(1.0) - g.integers(1, 64, d).astype(np.float32) * np.float32(2.0 ** -9)
        sign = np.where(g.random(d) < 0.5, -1.0, 1.0).astype(np.float32)
        x = (sign * mags).astype(np.float32)
        y = (sign * mags[::-1]).astype(np.float32) if trial % 2 else x.copy()
        check(x, y)


def test_wide_dynamic_range_and_sparse_vectors():
    g = np.random.default_rng(3)
    for d in (32, 97, 480):
        for _ in range(10):
            x = (g.standard_normal(d) * np.exp2(g.integers(-30, 30, d))).astype(np.float32)
            y = (g.standard_normal(d) * np.exp2(g.integers(-30, 30, d))).astype(np.float32)
            x[g.random(d) < 0.5] = 0.0
            check(x, y)
            check(x, x)


def test_zero_and_tiny_vectors():
    d = 64
    z = np.zeros(d, dtype=np.float32)
    y = np.random.default_rng(4).standard_normal(d).astype(np.float32)
    assert model_dot(z, y)[0] == 0.0
    tiny = np.full(d, 2.0 ** -70, dtype=np.float32)      # below 2^-60: treated as zero
    assert model_dot(tiny, y)[0] == 0.0
    assert abs(exact_dot(tiny, y)) < 2.0 ** -60 * np.linalg.norm(y) * 8
