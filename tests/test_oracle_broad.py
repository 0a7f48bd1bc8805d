"""Pins for the oracle's broad phase.  The candidate set is defined by the
"Guarantees" section: all vertex-face and edge-edge pairs (no shared vertex)
whose boxes overlap.  Three independent computations must agree: the C brute
force, the C serial sweep (Algorithm 2 without its queue) and a numpy
broadcast written here from the definition."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_06300_gb300 import scenes


def numpy_pairs(V0, V1, E, F, fp32=False):
    lo64, hi64, lo32, hi32 = O.boxes(V0, V1, E, F)
    lo, hi = (lo32, hi32) if fp32 else (lo64, hi64)
    nV, nE = len(V0), len(E)
    vlo, vhi = lo[:nV], hi[:nV]
    elo, ehi = lo[nV:nV + nE], hi[nV:nV + nE]
    flo, fhi = lo[nV + nE:], hi[nV + nE:]
    ov = np.all((vlo[:, None, :] <= fhi[None]) & (flo[None] <= vhi[:, None, :]), axis=2)
    inface = (np.arange(nV)[:, None, None] == F[None, :, :]).any(axis=2)
    v, f = np.nonzero(ov & ~inface)
    vf = np.stack([v, f], 1)
    ov = np.all((elo[:, None, :] <= ehi[None]) & (elo[None] <= ehi[:, None, :]), axis=2)
    share = (E[:, None, :, None] == E[None, :, None, :]).any(axis=(2, 3))
    a, b = np.nonzero(np.triu(ov & ~share, 1))
    ee = np.stack([a, b], 1)
    return vf.astype(np.int64), ee.astype(np.int64)


def random_scene(rng, nv, nf, spread=1.0, motion=0.3):
    V0 = rng.uniform(-spread, spread, (nv, 3))
    V1 = V0 + rng.normal(0, motion, (nv, 3))
    F = np.array([rng.choice(nv, 3, replace=False) for _ in range(nf)], np.int32)
    return V0, V1, scenes.edges_of(F), F


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("fp32", [False, True])
def test_three_implementations_agree_random(seed, fp32):
    rng = np.random.default_rng(seed)
    V0, V1, E, F = random_scene(rng, 60, 50)
    ref = numpy_pairs(V0, V1, E, F, fp32)
    for method in ("brute", "sweep"):
        vf, ee = O.broad(V0, V1, E, F, method, fp32)
        np.testing.assert_array_equal(vf, ref[0])
        np.testing.assert_array_equal(ee, ref[1])


def test_hand_built_scene():
    # triangle 0 at z=0; vertex 3 drops through it; vertex 4 stays far away;
    # triangle 1 shares vertex 2 with triangle 0 and is above it.
    V0 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0],      # tri 0
                   [0.2, 0.2, 1.0],                      # falls through tri 0
                   [5, 5, 5],                            # far
                   [0.5, 1, 0.5], [0, 2, 0.5]], float)   # tri 1 = (2, 5, 6)
    V1 = V0.copy()
    V1[3, 2] = -1.0
    F = np.array([[0, 1, 2], [2, 5, 6]], np.int32)
    E = scenes.edges_of(F)
    vf, ee = O.broad(V0, V1, E, F, "brute")
    vf = {tuple(p) for p in vf}
    assert (3, 0) in vf
    assert all(p[0] != 4 for p in vf)
    assert (2, 0) not in vf and (2, 1) not in vf          # shared vertex
    for a, b in ee:                                       # no shared endpoint
        assert not set(E[a]) & set(E[b])
        assert a < b


def test_brute_equals_sweep_icosphere_scene():
    s = scenes.icosphere_on_plane(0)
    b = O.broad(s.V0, s.V1, s.E, s.F, "brute")
    w = O.broad(s.V0, s.V1, s.E, s.F, "sweep")
    np.testing.assert_array_equal(b[0], w[0])
    np.testing.assert_array_equal(b[1], w[1])
    assert len(b[0]) > 1000 and len(b[1]) > 1000


def test_fp32_set_contains_fp64_set_cloth():
    s = scenes.folded_cloth(48, seed=1)
    v64, e64 = O.broad(s.V0, s.V1, s.E, s.F, "sweep", fp32=False)
    v32, e32 = O.broad(s.V0, s.V1, s.E, s.F, "sweep", fp32=True)
    b64 = O.broad(s.V0, s.V1, s.E, s.F, "brute", fp32=False)
    np.testing.assert_array_equal(v64, b64[0])
    np.testing.assert_array_equal(e64, b64[1])
    s64 = {tuple(p) for p in v64}
    s32 = {tuple(p) for p in v32}
    assert s64 <= s32
    assert {tuple(p) for p in e64} <= {tuple(p) for p in e32}
