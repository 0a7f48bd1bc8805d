"""Parity at the benchmark's full size (folded cloth, 512 x 512 vertices,
1,568,771 boxes, ~4.9M candidate pairs), in the configuration bench.py times
(ccd_step, earliest-TOI mode, default context): the whole pair set against
the oracle's sweep, the step's earliest time against the oracle's, and the
per-pair times of a seeded sample of 20,000 queries (GPU per-pair run over
all pairs; the oracle evaluates only the sample)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_06300_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    from paper_2112_06300_gb300 import build
    build.build()
    from paper_2112_06300_gb300 import ccd
    s = scenes.folded_cloth(512, seed=1)
    c = ccd.CCD(0)
    yield ccd, c, s
    c.close()


def test_full_size_pairs_and_step(setup):
    ccd, c, s = setup
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    vf, ee = c.broad(V0, V1, E, F)
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    a = vf.cpu().numpy().astype(np.int64)
    b = ee.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(a[np.lexsort((a[:, 1], a[:, 0]))], ovf)
    np.testing.assert_array_equal(b[np.lexsort((b[:, 1], b[:, 0]))], oee)
    t = c.step(V0, V1, E, F)
    to = O.narrow(ovf, oee, s.V0, s.V1, s.E, s.F, mode=1)[4]
    assert t == to

    # per-pair mode on every pair, checked on a seeded sample
    r = c.narrow(vf, ee, V0, V1, E, F, mode=0)
    g = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    gf = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    pairs_vf, pairs_ee = a, b
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(len(g), 20000, replace=False))
    sv = idx[idx < len(pairs_vf)]
    se = idx[idx >= len(pairs_vf)] - len(pairs_vf)
    o = O.narrow(pairs_vf[sv], pairs_ee[se], s.V0, s.V1, s.E, s.F, mode=0)
    ot = np.concatenate([o[0], o[1]])
    of = np.concatenate([o[2], o[3]])
    ok = (gf[idx] == 0) & (of == 0)
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(g[idx][ok].view(np.uint64), ot[ok].view(np.uint64))
    assert r.toi_min == t
