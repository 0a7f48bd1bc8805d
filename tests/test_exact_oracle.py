"""Pins for the exact time-of-impact oracle (oracle/exact.py): the paper's
printed cubic against mpmath, closed-form trajectories, a brute-force solver
on a rational time grid written here independently, and symmetry invariants."""
import os
from fractions import Fraction as Q

import numpy as np
import pytest

from oracle import exact as X
from paper_2112_06300_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "printed_cubic.txt")


def _read_golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = line.split("=")
            vals[k.strip()] = int(v)
    return vals


def test_printed_cubic_root_matches_mpmath():
    mpmath = pytest.importorskip("mpmath")
    g = _read_golden()
    p = [Q(g["c0"]), Q(g["c1"]), Q(g["c2"]), Q(g["c3"])]
    roots = X.real_roots(p)
    assert len(roots) == 3
    r = roots[g["index"] - 1]
    lo, hi = r.bracket(200) if isinstance(r, X.Alg) else (r, r)
    mpmath.mp.dps = 100
    ref = sorted(x.real for x in mpmath.polyroots([g["c3"], g["c2"], g["c1"], g["c0"]],
                                                  maxsteps=500, extraprec=600))
    target = ref[g["index"] - 1]
    assert mpmath.mpf(lo.numerator) / lo.denominator <= target + mpmath.mpf(10) ** -90
    assert mpmath.mpf(hi.numerator) / hi.denominator >= target - mpmath.mpf(10) ** -90
    assert abs(float(r) - 0.8579233907431208) < 1e-15


# --- an independent feasibility test at rational t ---------------------------

def _solve_feasible(a, b, c, omega):
    """Is there (u, v) in omega with a u + b v = c (3 rows, exact)?  omega is
    'simplex' or 'square'.  Rank-by-rank linear algebra, written from scratch."""
    verts = [(Q(0), Q(0)), (Q(1), Q(0)), (Q(0), Q(1))] if omega == "simplex" else \
        [(Q(0), Q(0)), (Q(1), Q(0)), (Q(1), Q(1)), (Q(0), Q(1))]

    def inside(u, v):
        if omega == "simplex":
            return u >= 0 and v >= 0 and u + v <= 1
        return 0 <= u <= 1 and 0 <= v <= 1

    rows = list(zip(a, b, c))
    for i in range(3):
        for j in range(i + 1, 3):
            det = rows[i][0] * rows[j][1] - rows[i][1] * rows[j][0]
            if det != 0:
                u = (rows[i][2] * rows[j][1] - rows[i][1] * rows[j][2]) / det
                v = (rows[i][0] * rows[j][2] - rows[i][2] * rows[j][0]) / det
                ok = all(r[0] * u + r[1] * v == r[2] for r in rows)
                return ok and inside(u, v)
    nz = [r for r in rows if r[0] != 0 or r[1] != 0]
    if not nz:
        return all(r[2] == 0 for r in rows)
    al, be, ga = nz[0]
    for r in rows:   # rank 1: every row must be a multiple of (al, be, ga)
        k = r[0] / al if al != 0 else r[1] / be
        if r[0] != k * al or r[1] != k * be or r[2] != k * ga:
            return False
    vals = [al * u + be * v - ga for u, v in verts]
    return min(vals) <= 0 <= max(vals)


def brute_feasible(vf, x0, x1, t):
    P = [[Q(x0[k][i]) + t * (Q(x1[k][i]) - Q(x0[k][i])) for i in range(3)] for k in range(4)]
    if vf:
        w = [P[0][i] - P[1][i] for i in range(3)]
        e1 = [P[2][i] - P[1][i] for i in range(3)]
        e2 = [P[3][i] - P[1][i] for i in range(3)]
        return _solve_feasible(e1, e2, w, "simplex")
    w = [P[0][i] - P[2][i] for i in range(3)]
    ea = [P[1][i] - P[0][i] for i in range(3)]
    eb = [P[3][i] - P[2][i] for i in range(3)]
    return _solve_feasible(ea, [-x for x in eb], [-x for x in w], "square")


def _small_queries(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        vf = bool(i % 2)
        kind = i % 5
        if kind == 0:
            a = rng.integers(-8, 9, (4, 3)) / 8
            b = rng.integers(-8, 9, (4, 3)) / 8
        elif kind in (1, 2):     # constructed contact at t* on a coarse grid
            C = rng.integers(-4, 5, (1, 3)) / 8
            R = rng.integers(-2, 3, (3, 3)) / 8
            if vf:
                R[2] = -(R[0] + R[1]) / 2 if kind == 1 else R[2]
                star = np.concatenate([C, C + R[0:1], C + R[1:2], C + R[2:3]])
            else:
                star = np.concatenate([C - R[0:1], C + R[0:1], C - R[1:2], C + R[1:2]])
            D = rng.integers(-4, 5, (4, 3)) / 8
            ts = rng.integers(0, 5) / 4
            a = star - ts * D
            b = a + D
        elif kind == 3:          # coplanar / parallel
            a = rng.integers(-8, 9, (4, 3)) / 8
            D = rng.integers(-4, 5, (4, 3)) / 8
            if vf:
                a[:, 2] = a[0, 2]
                D[:, 2] = 0
            else:
                d = rng.integers(-4, 5, 3) / 8
                a[1] = a[0] + d
                a[3] = a[2] + 2 * d
                D[1] = D[0]
                D[3] = D[2]
            b = a + D
        else:                    # integer-ish motion through each other
            a = rng.integers(-2, 3, (4, 3)) / 2
            b = rng.integers(-2, 3, (4, 3)) / 2
        out.append((vf, a.tolist(), b.tolist()))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_toi_against_rational_time_grid(seed):
    grid = [Q(k, 32) for k in range(33)]
    n_hits = 0
    for vf, a, b in _small_queries(seed, 60):
        r = X.toi(vf, a, b)
        feas = [brute_feasible(vf, a, b, t) for t in grid]
        if r is None:
            assert not any(feas)
            continue
        n_hits += 1
        for t, f in zip(grid, feas):
            if f:
                assert X.compare(r, t) <= 0
            if X.compare(t, r) < 0:
                assert not f
        rr = r if isinstance(r, Q) else r.exact
        if rr is not None:
            assert brute_feasible(vf, a, b, rr)
        else:   # irrational: feasible at no rational point just below
            lo, hi = r.bracket(40)
            assert not brute_feasible(vf, a, b, lo)
    assert n_hits >= 10


def test_closed_form_point_falls_on_triangle():
    rng = np.random.default_rng(5)
    for _ in range(40):
        T = rng.integers(-16, 17, (3, 2)) / 16
        if abs((T[1, 0] - T[0, 0]) * (T[2, 1] - T[0, 1]) - (T[1, 1] - T[0, 1]) * (T[2, 0] - T[0, 0])) < 0.1:
            continue
        lam = np.array([1, 1, 2]) / 4
        P = lam @ T
        z = rng.integers(-8, 9) / 8
        h = rng.integers(1, 64) / 64
        s = rng.integers(1, 5) * 0.5 + h        # speed > height, t* = h / s
        x0 = [(P[0], P[1], z + h)] + [(t[0], t[1], z) for t in T]
        x1 = [(P[0], P[1], z + h - s)] + [(t[0], t[1], z) for t in T]
        r = X.toi(True, x0, x1)
        assert r is not None and X.compare(r, Q(h) / Q(s)) == 0


def test_closed_form_edges_cross():
    rng = np.random.default_rng(6)
    for _ in range(40):
        c = rng.integers(-8, 9, 2) / 8
        da = rng.integers(-8, 9, 2) / 8
        db = np.array([-da[1], da[0]]) + rng.integers(-2, 3, 2) / 8
        if np.linalg.norm(da) == 0 or abs(da[0] * db[1] - da[1] * db[0]) < 1e-3:
            continue
        h = rng.integers(1, 32) / 32
        s = h * rng.integers(2, 9) / 2
        A0, A1 = c - da / 2, c + da / 2
        B0, B1 = c - db, c + db
        x0 = [(A0[0], A0[1], h), (A1[0], A1[1], h), (B0[0], B0[1], 0.0), (B1[0], B1[1], 0.0)]
        x1 = [(A0[0], A0[1], h - s), (A1[0], A1[1], h - s), (B0[0], B0[1], 0.0), (B1[0], B1[1], 0.0)]
        r = X.toi(False, x0, x1)
        assert r is not None and X.compare(r, Q(h) / Q(s)) == 0


def test_static_and_miss_special_cases():
    tri = [(0, 0, 0), (1, 0, 0), (0, 1, 0)]
    inside = [(0.25, 0.25, 0.0)] + tri
    assert X.toi(True, inside, inside) == 0
    outside = [(0.75, 0.75, 0.0)] + tri
    assert X.toi(True, outside, outside) is None
    edge = [(0.5, 0.5, 0.0)] + tri        # on the hypotenuse
    assert X.toi(True, edge, edge) == 0
    above = [(0.25, 0.25, 1.0)] + tri
    moving = [(0.25, 0.25, 0.5)] + tri     # stops before the triangle
    assert X.toi(True, above, moving) is None


def _transforms(rng):
    perm = rng.permutation(3)
    flip = rng.choice([-1.0, 1.0], 3)
    shift = rng.integers(-8, 9, 3) / 8
    scale = 2.0 ** rng.integers(-3, 4)
    return lambda p: tuple(float(scale * flip[i] * p[perm[i]] + shift[i]) for i in range(3))


@pytest.mark.parametrize("seed", [3, 4])
def test_symmetry_invariants(seed):
    rng = np.random.default_rng(seed)
    for vf, a, b in _small_queries(seed + 10, 30):
        r = X.toi(vf, a, b)
        variants = []
        f = _transforms(rng)
        variants.append(([f(p) for p in a], [f(p) for p in b]))
        if vf:
            for perm in ([0, 2, 3, 1], [0, 3, 1, 2], [0, 2, 1, 3]):
                variants.append(([a[i] for i in perm], [b[i] for i in perm]))
        else:
            for perm in ([2, 3, 0, 1], [1, 0, 2, 3], [0, 1, 3, 2]):
                variants.append(([a[i] for i in perm], [b[i] for i in perm]))
        for a2, b2 in variants:
            r2 = X.toi(vf, a2, b2)
            if r is None:
                assert r2 is None
            else:
                assert r2 is not None and X.compare(r, r2) == 0


def test_generator_constructed_queries_collide_by_tstar():
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(200, seed=7)
    col = np.nonzero(kind == scenes.KINDS.index("collide"))[0][:20]
    for q in col:
        r = X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist())
        assert r is not None
    miss = np.nonzero(kind == scenes.KINDS.index("near_miss"))[0][:20]
    for q in miss:
        assert X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist()) is None
