"""The multi-GPU decomposition of a step, run shard by shard on one GPU
(the paper's multi-GPU broad phase, Section "Conclusion and Future Work").

Each shard sweeps its own contiguous part of the sorted cell copies
(ccd_broad_shard): the shards' pair sets must be disjoint and together equal
the whole broad phase's set, and the minimum over the shards of the narrow
phase run on each shard's pairs alone (mode 1, a separate call per shard, the
minimum taken on the host: the one exchange a multi-GPU step needs) must equal
the single-call step and the oracle bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_06300_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccd():
    from paper_2112_06300_gb300 import build
    build.build()
    from paper_2112_06300_gb300 import ccd as m
    return m


def keyset(vf, ee):
    a = vf.cpu().numpy().astype(np.int64).reshape(-1, 2)
    b = ee.cpu().numpy().astype(np.int64).reshape(-1, 2)
    return np.sort(a[:, 0] * (1 << 32) + a[:, 1]), np.sort(b[:, 0] * (1 << 32) + b[:, 1])


@pytest.mark.parametrize("scene", ["cloth96", "icosphere", "rigid"])
def test_shards_partition_the_pairs_and_their_minimum_is_the_step(ccd, scene):
    s = {"cloth96": lambda: scenes.folded_cloth(96, seed=2),
         "icosphere": lambda: scenes.icosphere_on_plane(0),
         "rigid": lambda: scenes.rigid_environment(5, 2000, 6000, vmax=0.2)}[scene]()
    d = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    c = ccd.CCD(0)
    try:
        full_vf, full_ee = keyset(*c.broad(*d))
        t_step = c.step(*d)
        for n_shards in (1, 3, 7):
            vfs, ees, mins = [], [], []
            for k in range(n_shards):
                vf, ee = c.broad_shard(*d, k, n_shards)
                a, b = keyset(vf, ee)
                vfs.append(a)
                ees.append(b)
                mins.append(c.narrow(vf, ee, *d, 1e-6, 0.0, 10 ** 6, 1).toi_min)
            allv, alle = np.concatenate(vfs), np.concatenate(ees)
            assert len(np.unique(allv)) == len(allv) and len(np.unique(alle)) == len(alle), "shards overlap"
            np.testing.assert_array_equal(np.sort(allv), full_vf)
            np.testing.assert_array_equal(np.sort(alle), full_ee)
            t = min(mins)
            assert np.float64(t).view(np.uint64) == np.float64(t_step).view(np.uint64), (n_shards, t, t_step)
    finally:
        c.close()
    assert t_step == O.step(s.V0, s.V1, s.E, s.F)
