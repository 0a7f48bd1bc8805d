"""Pins for the oracle's box construction (Section "Construction of the
Boxes"): FP64 extents over t = 0 and t = 1, and the single-precision box that
rounds them outward.  Checked against numpy reductions and nextafter, not
against the oracle's own formulas."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_06300_gb300 import scenes


def _random_mesh(rng, nv=40, nf=30, scale=1.0):
    V0 = rng.normal(0, scale, (nv, 3))
    V1 = V0 + rng.normal(0, 0.1 * scale, (nv, 3))
    F = np.array([rng.choice(nv, 3, replace=False) for _ in range(nf)], np.int32)
    return V0, V1, scenes.edges_of(F), F


@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e20, 3.0])
def test_extents_are_min_max_over_both_times(scale):
    rng = np.random.default_rng(11)
    V0, V1, E, F = _random_mesh(rng, scale=scale)
    lo64, hi64, _, _ = O.boxes(V0, V1, E, F)
    both = np.stack([V0, V1], 0)                     # (2, nV, 3)
    prims = [np.array([[v] for v in range(len(V0))])[:, 0:1], E, F]
    ref_lo, ref_hi = [], []
    for P in prims:
        pts = both[:, P, :]                          # (2, n, k, 3)
        ref_lo.append(pts.min(axis=(0, 2)))
        ref_hi.append(pts.max(axis=(0, 2)))
    np.testing.assert_array_equal(lo64, np.concatenate(ref_lo))
    np.testing.assert_array_equal(hi64, np.concatenate(ref_hi))


def test_fp32_box_is_tightest_outward_rounding():
    rng = np.random.default_rng(12)
    # values that are exact floats, halfway cases, negatives, tiny and large
    vals = np.concatenate([
        rng.normal(0, 1, 500), rng.normal(0, 1e-38, 50), rng.normal(0, 1e30, 50),
        np.array([0.0, -0.0, 1.0, -1.0, 0.1, -0.1, 1 + 2 ** -24, 1 + 2 ** -23,
                  np.float32(0.3).item(), -np.float32(0.3).item(), 2 ** -149, -2 ** -149]),
    ])
    n = len(vals)
    V0 = np.stack([vals, -vals, vals * 3], 1)
    V1 = V0.copy()
    lo64, hi64, lo32, hi32 = O.boxes(V0, V1, np.zeros((0, 2), np.int32), np.zeros((0, 3), np.int32))
    assert lo64.shape == (n, 3)
    lo32d = lo32.astype(np.float64)
    hi32d = hi32.astype(np.float64)
    assert np.all(lo32d <= lo64) and np.all(hi32d >= hi64)
    # tightest: the next float toward the value overshoots it
    up = np.nextafter(lo32, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(hi32, np.float32(-np.inf)).astype(np.float64)
    assert np.all(up > lo64)
    assert np.all(dn < hi64)
    # exactly representable extents are kept as they are (reading: "<=")
    exact = lo64 == lo64.astype(np.float32).astype(np.float64)
    assert np.all(lo32d[exact] == lo64[exact])


def test_box_counts_icosphere_scene():
    s = scenes.icosphere_on_plane(0)
    assert (len(s.V0), len(s.E), len(s.F)) == (3651, 10816, 7168)
    assert s.n_boxes == 21635
    lo64, hi64, lo32, hi32 = O.boxes(s.V0, s.V1, s.E, s.F)
    assert lo64.shape == (21635, 3)
    assert np.all(lo32 <= lo64) and np.all(hi32 >= hi64)
