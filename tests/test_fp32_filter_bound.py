"""The single-precision filter of the narrow kernel decides an interval only
when its FP32 hull proves the FP64 decision; that rests on one claim: on every
axis the FP32 hull and the FP64 hull are less than e32 = 8 * 2^-24 * S apart,
S = sum over the three vectors of |c0| + |dc| (the FP64 set-up values).  The
derivation passes through R, the hull evaluated exactly from c0 and dc: the
FP32 hull is within 6 * 2^-24 S of R, the FP64 hull within 4 * 2^-53 S.

Checked here against exact rational arithmetic, with float32 and float64
fused multiply-adds emulated exactly (round to nearest even of the exact
result), with the kernel's corner choice by the sign of each computed vector,
over random queries and intervals with levels <= 24, across coordinate scales
and with coordinates far larger than their differences (the case where a bound
built from the coordinates would be loose)."""
from fractions import Fraction as Q

import numpy as np
import pytest

U32 = Q(1, 2 ** 24)
U64 = Q(1, 2 ** 53)


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


def fma64(a, b, c):
    # float(Fraction) rounds to nearest even: one correctly rounded FP64 fma
    return Q(float(Q(a) * Q(b) + Q(c)))


def hull_axis(c0, dc, t_ends, u_ends, v_ends, vf, fma):
    """Hull of F on one axis with the kernel's expression tree and corner
    choice (by the sign of each computed vector), every operation an fma
    rounded by `fma`; fma=None evaluates exactly (R)."""
    ul, ur = u_ends
    vl, vr = v_ends
    lo = hi = None
    for t in t_ends:
        if fma is None:
            w, a, b = (Q(c0[j]) + t * Q(dc[j]) for j in range(3))
            op = lambda p, q, r: p * q + r
        else:
            w, a, b = (fma(t, dc[j], c0[j]) for j in range(3))
            op = fma
        ap, bp = a > 0, b > 0
        if vf:
            gmin = op(-(vr if bp else vl), b, w)
            gmax = op(-(vl if bp else vr), b, w)
            fmin = op(-(ur if ap else ul), a, gmin)
            fmax = op(-(ul if ap else ur), a, gmax)
        else:
            gmin = op(ul if ap else ur, a, w)
            gmax = op(ur if ap else ul, a, w)
            fmin = op(-(vr if bp else vl), b, gmin)
            fmax = op(-(vl if bp else vr), b, gmax)
        lo = fmin if lo is None else min(lo, fmin)
        hi = fmax if hi is None else max(hi, fmax)
    return lo, hi


def exact_hull_axis(c0, dc, t_ends, u_ends, v_ends, vf):
    """R by brute force: min and max of F over the eight corners, exactly."""
    vals = []
    for t in t_ends:
        w, a, b = (Q(c0[j]) + t * Q(dc[j]) for j in range(3))
        for u in u_ends:
            for v in v_ends:
                vals.append(w - u * a - v * b if vf else w + u * a - v * b)
    return min(vals), max(vals)


def random_query(rng):
    vf = bool(rng.integers(2))
    scale = 2.0 ** rng.integers(-30, 30)
    kind = rng.integers(3)
    if kind == 0:        # differences of the size of the coordinates
        x0 = rng.uniform(-1, 1, (4, 3)) * scale
    else:                # coordinates far from the origin, small differences
        off = rng.uniform(-1, 1, 3) * scale * (2.0 ** rng.integers(4, 20))
        x0 = off + rng.uniform(-1, 1, (4, 3)) * scale
    x1 = x0 + rng.uniform(-1, 1, (4, 3)) * scale * rng.choice([1e-6, 1e-2, 1.0])
    if kind == 2:        # a vector that changes sign inside [0, 1]
        x1[2] = x0[2] + 2.0 * (x0[1] - x0[2]) if vf else x1[2]
    pairs = [(0, 1), (2, 1), (3, 1)] if vf else [(0, 2), (1, 0), (3, 2)]
    c0 = np.array([[x0[a, x] - x0[b, x] for x in range(3)] for a, b in pairs])
    c1 = np.array([[x1[a, x] - x1[b, x] for x in range(3)] for a, b in pairs])
    return vf, c0, c1 - c0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp32_hull_within_e32_of_fp64_hull(seed):
    rng = np.random.default_rng(seed)
    worst32 = worst64 = worst = 0.0
    for _ in range(60):
        vf, c0, dc = random_query(rng)
        c0f = c0.astype(np.float32).astype(np.float64)
        dcf = dc.astype(np.float32).astype(np.float64)
        lv = rng.integers(0, 25, 3)
        nv = [int(rng.integers(0, 2 ** int(l))) for l in lv]
        ends = [(Q(nv[k], 2 ** int(lv[k])), Q(nv[k] + 1, 2 ** int(lv[k]))) for k in range(3)]
        for x in range(3):
            S = sum(abs(Q(c0[j, x])) + abs(Q(dc[j, x])) for j in range(3))
            if S == 0:
                continue
            R = exact_hull_axis(c0[:, x], dc[:, x], *ends, vf)
            R2 = hull_axis(c0[:, x], dc[:, x], *ends, vf, None)
            assert R2 == R, "sign-chosen corners give the exact extremes"
            h32 = hull_axis(c0f[:, x], dcf[:, x], *ends, vf, fma32)
            h64 = hull_axis(c0[:, x], dc[:, x], *ends, vf, fma64)
            for k in range(2):
                d32 = abs(h32[k] - R[k])
                d64 = abs(h64[k] - R[k])
                d = abs(h32[k] - h64[k])
                assert d32 <= 6 * U32 * S, float(d32 / (U32 * S))
                assert d64 <= 4 * U64 * S, float(d64 / (U64 * S))
                assert d < 8 * U32 * S
                worst32 = max(worst32, float(d32 / (U32 * S)))
                worst64 = max(worst64, float(d64 / (U64 * S)))
                worst = max(worst, float(d / (U32 * S)))
    assert worst < 8.0 and worst32 <= 6.0 and worst64 <= 4.0


def test_bound_is_local_not_global():
    """A query 2^20 units from the origin with differences of order 1: the
    bound follows the differences (S), so it is about 2^20 times smaller than
    one built from the largest coordinate."""
    rng = np.random.default_rng(7)
    x0 = 2.0 ** 20 + rng.uniform(-1, 1, (4, 3))
    x1 = x0 + rng.uniform(-1e-2, 1e-2, (4, 3))
    c0 = np.array([[x0[a, x] - x0[b, x] for x in range(3)] for a, b in [(0, 1), (2, 1), (3, 1)]])
    dc = np.array([[x1[a, x] - x1[b, x] for x in range(3)] for a, b in [(0, 1), (2, 1), (3, 1)]]) - c0
    S = max(sum(abs(c0[j, x]) + abs(dc[j, x]) for j in range(3)) for x in range(3))
    m = np.abs(np.concatenate([x0, x1])).max()
    assert 8 * S < 40 * m / 2.0 ** 17


# ---------------------------------------------------------------------------
# Certified ends: per-corner running error bounds (settle hull ends at 0).
# ---------------------------------------------------------------------------

def to_float_error(d: float) -> Q:
    """The bound the set-up uses for |float(d) - d|: 0 for a float, one
    float ulp at d's exponent otherwise, 2^-126 below the normal range (where
    the set-up's conversion gives 0)."""
    if d == 0:
        return Q(0)
    m, E = np.frexp(abs(d))          # abs(d) = m 2^E, m in [0.5, 1)
    E = int(E) - 1                   # unbiased exponent
    if E < -126:
        return Q(1, 2 ** 126)
    assert E <= 126
    if float(np.float32(d)) == d:
        return Q(0)
    return Q(2) ** (E - 23)


def test_to_float_error_bounds_the_conversion():
    rng = np.random.default_rng(3)
    for _ in range(4000):
        d = float(rng.uniform(-1, 1) * 2.0 ** rng.integers(-140, 120))
        if rng.integers(4) == 0:
            d = float(np.float32(d))          # some exact floats
        err = abs(Q(float(np.float32(d))) - Q(d))
        b = to_float_error(d)
        assert err <= b
        assert (b == 0) == (err == 0) or abs(d) < 2.0 ** -126


def round_f32_dir(x: Q, up: bool) -> Q:
    """Exact rounding of a rational to float32 toward +inf (up) or -inf,
    subnormals included."""
    if x == 0:
        return Q(0)
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Q(2) ** e > a:
        e -= 1
    while Q(2) ** (e + 1) <= a:
        e += 1
    q = Q(2) ** (max(e, -126) - 23)          # spacing of floats at |x|
    n = a / q
    k = n.numerator // n.denominator          # floor of |x| / q
    exact = k * q == a
    # toward +inf: up for x > 0 means away from zero; for x < 0 toward zero
    away = (not exact) and (up == (x > 0))
    r = (k + 1) * q if away else k * q
    return r if x > 0 else -r


def fma32u(a, b, c):
    return round_f32_dir(Q(a) * Q(b) + Q(c), True)


def fma32d(a, b, c):
    return round_f32_dir(Q(a) * Q(b) + Q(c), False)


def test_directed_rounding_emulation():
    rng = np.random.default_rng(5)
    for _ in range(500):
        x = Q(float(rng.uniform(-1, 1) * 2.0 ** rng.integers(-130, 60)))
        x += Q(int(rng.integers(-3, 4)), 2 ** 170)
        u, d = round_f32_dir(x, True), round_f32_dir(x, False)
        assert d <= x <= u
        assert float(np.float32(float(u))) == float(u) and float(np.float32(float(d))) == float(d)
        assert (u == d) == (u == x)
        if u != d:                       # adjacent floats
            assert float(np.nextafter(np.float32(float(d)), np.float32(np.inf))) == float(u)


def certified_ends(c0f, dcf, cc0, cdc, t_ends, u_ends, v_ends, vf):
    """The kernel's certified ends: the selected low and high corners in
    interval arithmetic (outward-rounded fmas), widened by conv(t)."""
    ul, ur = u_ends
    vl, vr = v_ends
    L = H = None
    for t in t_ends:
        w, a, b = (fma32(t, dcf[j], c0f[j]) for j in range(3))
        wu, au, bu = (fma32u(t, dcf[j], c0f[j]) for j in range(3))
        wd, ad, bd = (fma32d(t, dcf[j], c0f[j]) for j in range(3))
        ap, bp = a > 0, b > 0
        if vf:
            vlo, vhi = (vr, vl) if bp else (vl, vr)
            ulo, uhi = (ur, ul) if ap else (ul, ur)
            Lt = fma32u(-ulo, ad, fma32u(-vlo, bd, wu))
            Ht = fma32d(-uhi, au, fma32d(-vhi, bu, wd))
        else:
            ulo, uhi = (ul, ur) if ap else (ur, ul)
            vlo, vhi = (vr, vl) if bp else (vl, vr)
            Lt = fma32u(-vlo, bd, fma32u(ulo, au, wu))
            Ht = fma32d(-vhi, bu, fma32d(uhi, ad, wd))
        conv = round_f32_dir(t * cdc + cc0, True)
        Lt = round_f32_dir(Lt + conv, True)
        Ht = round_f32_dir(Ht - conv, False)
        L = Lt if L is None else min(L, Lt)
        H = Ht if H is None else max(H, Ht)
    return L, H


def conv_terms(c0, dc, x):
    """cc0, cdc as the set-up forms them (float sums rounded upward)."""
    cc0 = cdc = Q(0)
    for j in range(3):
        cc0 = round_f32_dir(cc0 + to_float_error(c0[j, x]), True)
        cdc = round_f32_dir(cdc + to_float_error(dc[j, x]), True)
    return cc0, cdc


@pytest.mark.parametrize("seed", [0, 1])
def test_certified_ends_bound_exact_hull(seed):
    """L is an upper bound of R's low end, H a lower bound of its high end."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(60):
        vf, c0, dc = random_query(rng)
        c0f = c0.astype(np.float32).astype(np.float64)
        dcf = dc.astype(np.float32).astype(np.float64)
        lv = rng.integers(0, 25, 3)
        nv = [int(rng.integers(0, 2 ** int(l))) for l in lv]
        ends = [(Q(nv[k], 2 ** int(lv[k])), Q(nv[k] + 1, 2 ** int(lv[k]))) for k in range(3)]
        for x in range(3):
            cc0, cdc = conv_terms(c0, dc, x)
            R = exact_hull_axis(c0[:, x], dc[:, x], *ends, vf)
            L, H = certified_ends(c0f[:, x], dcf[:, x], cc0, cdc, *ends, vf)
            assert R[0] <= L and H <= R[1]


def grid_query(rng, vf, n=512, layer_z=0.0):
    """A query between elements of one flat layer of an n x n grid that moves
    only along z: grid-aligned x, y (exact zeros at corners), z equal at t = 0."""
    i, j = rng.integers(1, n - 2, 2)
    pts = np.array([[i, j], [i + 1, j], [i, j + 1], [i + 1, j + 1], [i - 1, j], [i, j - 1]]) / n
    idx = rng.choice(len(pts), 4, replace=False)
    x0 = np.zeros((4, 3))
    x0[:, :2] = pts[idx]
    x0[:, 2] = layer_z
    x1 = x0.copy()
    x1[:, 2] += rng.uniform(-0.01, 0.01, 4)
    pairs = [(0, 1), (2, 1), (3, 1)] if vf else [(0, 2), (1, 0), (3, 2)]
    c0 = np.array([[x0[a, k] - x0[b, k] for k in range(3)] for a, b in pairs])
    c1 = np.array([[x1[a, k] - x1[b, k] for k in range(3)] for a, b in pairs])
    m = np.abs(np.concatenate([x0, x1])).max(axis=0)
    return c0, c1 - c0, m


def test_certified_ends_settle_exact_zero_ends():
    """On a flat grid layer moving along z, hull ends exactly at 0 (a vertex on
    a grid line of the other element, where terms cancel exactly; every z
    corner at t = 0) are settled as 'no miss' by the certified ends, and
    whenever an end is settled the FP64 hull agrees."""
    rng = np.random.default_rng(11)
    settled = at_zero = 0
    for _ in range(80):
        vf = bool(rng.integers(2))
        c0, dc, m = grid_query(rng, vf, layer_z=float(rng.choice([0.0, 1e-3])))
        c0f = c0.astype(np.float32).astype(np.float64)
        dcf = dc.astype(np.float32).astype(np.float64)
        lt, lu, lv = (int(v) for v in rng.integers(1, 12, 3))
        ends = [(Q(0), Q(1, 2 ** lt)),
                (Q(int(rng.integers(0, 2 ** lu)), 2 ** lu), None),
                (Q(int(rng.integers(0, 2 ** lv)), 2 ** lv), None)]
        ends = [(a, b if b is not None else a + Q(1, 2 ** l)) for (a, b), l in zip(ends, (lt, lu, lv))]
        for x in range(3):
            S = sum(abs(Q(c0[j, x])) + abs(Q(dc[j, x])) for j in range(3))
            eps = Q(float(m[x])) * 48 * U64            # the FP64 error box (min_sep = 0)
            e64 = 4 * U64 * S + Q(1, 2 ** 1060)
            tn = eps - e64
            cc0, cdc = conv_terms(c0, dc, x)
            R = exact_hull_axis(c0[:, x], dc[:, x], *ends, vf)
            L, H = certified_ends(c0f[:, x], dcf[:, x], cc0, cdc, *ends, vf)
            h64 = hull_axis(c0[:, x], dc[:, x], *ends, vf, fma64)
            for end, cert, val in ((0, L <= tn, h64[0]), (1, H >= -tn, h64[1])):
                if R[end] == 0:
                    at_zero += 1
                    assert cert, (x, vf)
                if cert:
                    settled += 1
                    assert (val <= eps) if end == 0 else (val >= -eps)
    assert at_zero > 50 and settled >= at_zero
