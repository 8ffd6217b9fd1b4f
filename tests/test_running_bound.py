"""The running error bound that lets the recheck kernels decide a sign in binary32 (the
tensor-core engine's recheck: one FMA chain per column; the binary32 engine's warp recheck:
32 lane chains joined by a butterfly of additions), checked on the CPU against exact rational
arithmetic.  Every binary32 operation is emulated with correct rounding to nearest, and the
bound with the host's constants must cover the exact error of the computed sum:

    |s^ - x.w| <= runc * R^ + runabs,  R^ = binary32 sum of |every rounded partial result|,

with runc = u / ((1 - u)(1 - gamma_m)) * 1.01 (m bounds the additions any term of R^ passes
through) and runabs = (number of rounding steps) * 2^-149.  Inputs are chosen to cancel
(|x.w| tiny against |x||w|) and to reach the subnormal range, where the bound is tight."""
from fractions import Fraction

import numpy as np
import pytest

U = Fraction(1, 2 ** 24)
F32_MIN_SUB = Fraction(1, 2 ** 149)


def rn32(q: Fraction) -> np.float32:
    """q rounded to the nearest binary32 (ties to even), exactly."""
    c = np.float32(float(q))  # within one binary32 step of the answer
    cands = {c, np.nextafter(c, np.float32(np.inf)), np.nextafter(c, np.float32(-np.inf))}
    best = None
    for v in cands:
        if not np.isfinite(v):
            continue
        err = abs(Fraction(float(v)) - q)
        key = (err, int(np.float32(v).view(np.uint32)) & 1)  # ties: even significand
        if best is None or key < best[0]:
            best = (key, v)
    return np.float32(best[1])


def fma32(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def add32(a, b):
    return rn32(Fraction(float(a)) + Fraction(float(b)))


def gamma(m):
    return m * U / (1 - m * U)


def chain(x, w):
    """One FMA chain in index order with the running sum of |partial results|."""
    s = r = np.float32(0)
    for xi, wi in zip(x, w):
        s = fma32(xi, wi, s)
        r = add32(r, abs(s))
    return s, r, len(x)


def warp(x, w):
    """Lane l sums coordinates l, l + 32, ...; a butterfly joins the 32 lanes' sums."""
    s = [np.float32(0)] * 32
    r = [np.float32(0)] * 32
    steps = 0
    for t, (xi, wi) in enumerate(zip(x, w)):
        lane = t % 32
        s[lane] = fma32(xi, wi, s[lane])
        r[lane] = add32(r[lane], abs(s[lane]))
        steps += 1
    off = 16
    while off:
        ns, nr = s[:], r[:]
        for lane in range(32):
            ns[lane] = add32(s[lane], s[lane ^ off])
            nr[lane] = add32(add32(r[lane], r[lane ^ off]), abs(ns[lane]))
        s, r = ns, nr
        off //= 2
    assert all(v == s[0] for v in s) and all(v == r[0] for v in r)  # every lane agrees
    return s[0], r[0], steps + 31


def cases(rng, d, n):
    out = []
    for k in range(n):
        w = rng.standard_normal(d)
        x = rng.standard_normal(d) * np.exp(rng.uniform(-6, 6, size=d))  # wide exponent spread
        x = x - (x @ w) / (w @ w) * w  # nearly orthogonal: heavy cancellation
        x = x + [0.0, 1e-9, 1e-6, 1e-3][k % 4] * np.linalg.norm(x) / np.linalg.norm(w) * w
        if k % 5 == 4:
            x = x * 2.0 ** -130  # products and partial sums in the subnormal range
        out.append((x.astype(np.float32), w.astype(np.float32)))
    return out


@pytest.mark.parametrize("mode", ["chain", "warp"])
def test_running_bound_covers_the_exact_error(mode):
    rng = np.random.default_rng(5)
    d = 41 if mode == "chain" else 70  # a warp of 32 lanes with a ragged last pass
    worst = 0.0
    for x, w in cases(rng, d, 60):
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, w))
        s, r, steps = (chain if mode == "chain" else warp)(x, w)
        m = steps + (0 if mode == "chain" else 64)  # additions a term of R^ may pass through
        runc = U / ((1 - U) * (1 - gamma(m))) * Fraction(101, 100)
        bound = runc * Fraction(float(r)) + steps * F32_MIN_SUB
        err = abs(Fraction(float(s)) - exact)
        assert err <= bound, (mode, float(err), float(bound))
        if bound > 0:
            worst = max(worst, float(err / bound))
    assert worst > 1e-3  # the bound is exercised, not vacuous


def test_rn32_is_correct_rounding():
    """Pin the emulation itself: exact midpoints round to even, others to nearest."""
    one = Fraction(1)
    step = Fraction(1, 2 ** 23)
    assert rn32(one + step / 2) == np.float32(1.0)  # tie: even
    assert rn32(one + 3 * step / 2) == np.float32(1.0 + 2 * 2.0 ** -23)  # tie: even (up)
    assert rn32(one + step / 2 + Fraction(1, 2 ** 60)) == np.float32(1.0 + 2.0 ** -23)
    assert rn32(F32_MIN_SUB / 2) == np.float32(0.0)  # tie below the smallest subnormal
    assert rn32(F32_MIN_SUB * 3 / 4) == np.float32(2.0 ** -149)
