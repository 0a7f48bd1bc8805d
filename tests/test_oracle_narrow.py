"""Pins for the FP64 narrow-phase oracle (Algorithm 3).

  * conservative: never later than the exact time of impact, never a miss
    (Sections "Guarantees" and "Time of Impact Validation and Accuracy");
  * close to closed-form times: the stop rule bounds the gap by
    (delta + 2 eps) / speed for a point falling straight onto a triangle;
  * order independence: the earliest-TOI mode (one shared t*) returns exactly
    the minimum of the per-query results, for any thread count.
"""
from fractions import Fraction as Q

import numpy as np
import pytest

from oracle import exact as X
from oracle import oracle as O
from paper_2112_06300_gb300 import scenes


def run(vf, x0, x1, delta=1e-6, ms=0.0, max_iter=10 ** 6):
    V0 = np.asarray(x0, float).reshape(4, 3)
    V1 = np.asarray(x1, float).reshape(4, 3)
    toi, flags, iters, _ = O.narrow_queries(np.array([int(vf)], np.uint8),
                                            np.array([[0, 1, 2, 3]]), V0, V1,
                                            delta, ms, max_iter)
    return float(toi[0]), int(flags[0]), int(iters[0])


@pytest.mark.parametrize("seed", [0, 1])
def test_no_false_negative_and_never_late_stress_mix(seed):
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(400, seed=seed)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    toi_vf, toi_ee, _, _, _ = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F)
    toi = np.empty(len(is_vf))
    toi[order] = np.concatenate([toi_vf, toi_ee])
    hits = 0
    for q in range(len(is_vf)):
        r = X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist())
        if r is None:
            continue
        hits += 1
        assert np.isfinite(toi[q]), f"false negative on query {q} ({scenes.KINDS[kind[q]]})"
        assert X.le_float(toi[q], r), f"late TOI on query {q}"
    assert hits >= 100


def test_closed_form_gap_bound():
    rng = np.random.default_rng(3)
    delta = 1e-6
    for _ in range(60):
        T = rng.integers(-16, 17, (3, 2)) / 16
        area = (T[1, 0] - T[0, 0]) * (T[2, 1] - T[0, 1]) - (T[1, 1] - T[0, 1]) * (T[2, 0] - T[0, 0])
        if abs(area) < 0.1:
            continue
        P = np.array([1, 1, 2]) / 4 @ T
        h = rng.integers(1, 64) / 64
        s = rng.integers(1, 5) * 0.5 + h
        x0 = [(P[0], P[1], h)] + [(t[0], t[1], 0.0) for t in T]
        x1 = [(P[0], P[1], h - s)] + [(t[0], t[1], 0.0) for t in T]
        toi, flags, _ = run(True, x0, x1, delta)
        exact = h / s
        m = max(1.0, np.abs(np.array(x0 + x1)).max())
        eps = 48 * 2.0 ** -53 * m
        assert flags == 0
        assert toi <= exact
        assert exact - toi <= (delta + 2 * eps) / s * 1.0001 + 1e-15


def test_min_separation_is_conservative():
    # point falling toward the triangle: with min_sep the reported time is at
    # or before the time the gap closes to min_sep (exact: (h - ms) / s)
    x0 = [(0.25, 0.25, 0.5), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    x1 = [(0.25, 0.25, -0.5), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    for ms in (0.0, 1e-4):
        toi, flags, _ = run(True, x0, x1, 1e-6, ms)
        assert flags == 0
        assert 0.5 - ms - 2e-6 <= toi <= 0.5 - ms + 1e-12
    # min_sep enlarges C_eps on every axis, so the first contact is a whole
    # patch of (u, v); resolving it to delta needs ~(2 ms / delta)^2 intervals
    # and hits the iteration cap: the answer must stay conservative and flagged
    for ms in (1e-2, 0.25):
        toi, flags, iters = run(True, x0, x1, 1e-6, ms, max_iter=20000)
        assert flags & 1 and iters == 20001
        assert toi <= 0.5 - ms
    # a miss by 0.1 becomes a hit when min_sep exceeds the gap
    y0 = [(2.0, 2.0, 0.1), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    assert run(True, y0, y0, 1e-6, 0.0)[0] == np.inf
    assert run(True, [(0.25, 0.25, 0.1)] + y0[1:], [(0.25, 0.25, 0.1)] + y0[1:], 1e-6, 0.2)[0] == 0.0


def test_earliest_mode_equals_min_of_per_query_any_threads():
    s = scenes.icosphere_on_plane(0, level=3, plane_n=17)
    vf, ee = O.broad(s.V0, s.V1, s.E, s.F)
    per = O.narrow(vf, ee, s.V0, s.V1, s.E, s.F, mode=0)
    ref = min(per[0].min(initial=np.inf), per[1].min(initial=np.inf))
    assert np.isfinite(ref)
    for nt in (1, 3, 8):
        e = O.narrow(vf, ee, s.V0, s.V1, s.E, s.F, mode=1, nthreads=nt)[4]
        assert e == ref
        p = O.narrow(vf, ee, s.V0, s.V1, s.E, s.F, mode=0, nthreads=nt)
        np.testing.assert_array_equal(p[0], per[0])
        np.testing.assert_array_equal(p[1], per[1])


def test_icosphere_without_jitter_first_contact_closed_form():
    # a translating convex polytope first meets a plane with a vertex: the
    # exact time is (min z) / 0.1 for the lowest sphere vertex over the plane
    s = scenes.icosphere_on_plane(0, level=2, plane_n=9, jitter=0.0)
    t = O.step(s.V0, s.V1, s.E, s.F)
    nsph = 10 * 16 + 2
    zmin = s.V0[:nsph, 2].min()
    exact = zmin / 0.1
    assert t <= exact
    assert exact - t < 1e-4


def test_iteration_cap_is_conservative_and_flagged():
    x0 = [(0.3, 0.3, 0.5), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    x1 = [(0.3, 0.3, -0.5), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    full, f0, it = run(True, x0, x1)
    assert f0 == 0 and it > 20
    capped, f1, it1 = run(True, x0, x1, max_iter=10)
    assert f1 & 1 and it1 == 11
    assert capped <= full


def test_touching_at_endpoints_and_degenerate():
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(300, seed=9)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    toi_vf, toi_ee, *_ = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F)
    toi = np.empty(len(is_vf))
    toi[order] = np.concatenate([toi_vf, toi_ee])
    touch = np.nonzero(kind == scenes.KINDS.index("touch"))[0]
    for q in touch:
        r = X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist())
        assert r is not None and X.le_float(toi[q], r)
    # a query touching at t = 0 must report 0 exactly
    zero = [q for q in touch if X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist()) == 0]
    assert zero and all(toi[q] == 0.0 for q in zero)


def test_no_zero_toi_rule():
    # a point 2^-12 above a triangle moving down at speed 1: first contact at
    # t = 2^-12; with min_sep = 0.01 the first pass reports 0, the rerun with
    # min_sep = 0 and the zero-TOI rule must give 0 < t <= 2^-12 (scaled 0.8)
    h = 2.0 ** -12
    tri = [(0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)]
    V0 = np.array([(0.25, 0.25, h)] + tri)
    V1 = np.array([(0.25, 0.25, h - 1.0)] + tri)
    E = np.array([[1, 2], [2, 3], [3, 1]], np.int32)
    F = np.array([[1, 2, 3]], np.int32)
    assert O.step(V0, V1, E, F, min_sep=0.01) == 0.0
    t = O.step(V0, V1, E, F, min_sep=0.01, no_zero_toi=True)
    assert 0.0 < t <= 0.8 * h
    assert t >= 0.8 * (h - 2e-6)
    # without a zero first pass the rule changes nothing
    assert O.step(V0, V1, E, F, no_zero_toi=True) == O.step(V0, V1, E, F)
    # touching at t = 0 stays 0 (the split reaches the level cap and accepts)
    W0 = np.array([(0.25, 0.25, 0.0)] + tri)
    W1 = np.array([(0.25, 0.25, -1.0)] + tri)
    assert O.step(W0, W1, E, F, no_zero_toi=True) == 0.0
    # conservative on the stress mix: never later than exact, positive when
    # the exact time is positive
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(200, seed=13)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    toi_vf, toi_ee, *_ = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F, no_zero=True)
    toi = np.empty(len(is_vf))
    toi[order] = np.concatenate([toi_vf, toi_ee])
    for q in range(len(is_vf)):
        r = X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist())
        if r is None:
            continue
        assert X.le_float(toi[q], r)
        if X.compare(r, Q(0)) > 0:
            assert toi[q] > 0.0
