"""The single-precision filter of the narrow kernel decides an interval only
when its FP32 hull proves the FP64 decision; that rests on one claim: every
FP32 corner value is within e32 = 40 * 2^-24 * max(m, 2^-100) of the exact
corner (m = the largest |coordinate| on the axis).  Checked here against exact
rational arithmetic, with float32 operations emulated exactly (round to
nearest even of the exact result), over random queries and intervals with
levels <= 24, across coordinate scales."""
from fractions import Fraction as Q
import math

import numpy as np
import pytest


def round_f32(x: Q) -> Q:
    """Exact round-to-nearest-even of a rational to float32 (normal range)."""
    if x == 0:
        return Q(0)
    s = -1 if x < 0 else 1
    a = -x if x < 0 else x
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Q(2) ** e > a:
        e -= 1
    while Q(2) ** (e + 1) <= a:
        e += 1
    assert e >= -126, "test inputs stay in the normal range"
    scaled = a * Q(2) ** (23 - e)            # in [2^23, 2^24)
    n = scaled.numerator // scaled.denominator
    r = scaled - n
    if r > Q(1, 2) or (r == Q(1, 2) and n % 2 == 1):
        n += 1
    return s * Q(n) * Q(2) ** (e - 23)


def fma32(a, b, c):
    return round_f32(Q(a) * Q(b) + Q(c))


def e32_bound(m: float) -> float:
    v = np.float32(40.0 * 2.0 ** -24 * max(m, 2.0 ** -100))
    if float(v) < 40.0 * 2.0 ** -24 * max(m, 2.0 ** -100):
        v = np.nextafter(v, np.float32(np.inf))
    return float(v)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp32_corners_within_e32(seed):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(60):
        vf = bool(rng.integers(2))
        scale = 2.0 ** rng.integers(-30, 30)
        x0 = rng.uniform(-1, 1, (4, 3)) * scale
        x1 = x0 + rng.uniform(-1, 1, (4, 3)) * scale * rng.choice([1e-6, 1e-2, 1.0])
        # vectors as the set-up forms them (FP64, then rounded to float32)
        if vf:
            pairs = [(0, 1), (2, 1), (3, 1)]
        else:
            pairs = [(0, 2), (1, 0), (3, 2)]
        c0 = np.array([[x0[a, x] - x0[b, x] for x in range(3)] for a, b in pairs])
        c1 = np.array([[x1[a, x] - x1[b, x] for x in range(3)] for a, b in pairs])
        dc = c1 - c0
        c0f = c0.astype(np.float32).astype(np.float64)
        dcf = dc.astype(np.float32).astype(np.float64)
        lv = rng.integers(0, 25, 3)
        nv = [int(rng.integers(0, 2 ** int(l))) for l in lv]
        ends = [(Q(nv[k], 2 ** int(lv[k])), Q(nv[k] + 1, 2 ** int(lv[k]))) for k in range(3)]
        for x in range(3):
            m = max(abs(x0[:, x]).max(), abs(x1[:, x]).max())
            bound = e32_bound(m)
            for t in ends[0]:
                w = fma32(t, dcf[0, x], c0f[0, x])
                a = fma32(t, dcf[1, x], c0f[1, x])
                b = fma32(t, dcf[2, x], c0f[2, x])
                for u in ends[1]:
                    for v in ends[2]:
                        if vf:
                            f = fma32(-u, a, fma32(-v, b, w))
                        else:
                            f = fma32(-v, b, fma32(u, a, w))
                        P = [[Q(x0[k, x]) + t * (Q(x1[k, x]) - Q(x0[k, x]))] for k in range(4)]
                        P = [p[0] for p in P]
                        if vf:
                            exact = P[0] - P[1] - u * (P[2] - P[1]) - v * (P[3] - P[1])
                        else:
                            exact = P[0] + u * (P[1] - P[0]) - P[2] - v * (P[3] - P[2])
                        err = abs(f - exact)
                        assert err <= Q(bound), (float(err), bound)
                        worst = max(worst, float(err) / (2.0 ** -24 * max(m, 2.0 ** -100)))
    assert worst < 40.0
