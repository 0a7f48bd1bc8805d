"""Batched step (many scenes of uneven size in one launch sequence) against
the oracle run on each scene alone: every scene's earliest time must be
bit-identical.  The environments share one region of space, so a pair across
scenes would show up as a spurious collision; an empty scene must report +inf."""
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


def empty_scene():
    return scenes.Scene(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 2), np.int32),
                        np.zeros((0, 3), np.int32), {"name": "empty"})


@pytest.mark.parametrize("sweep,width", [(0, 0.0), (0, 0.5), (0, 1e-3), (2, 0.0)],
                         ids=["strips", "narrow-strips", "strips-overflow", "tiled"])
def test_batch_matches_each_scene_alone(ccd, sweep, width):
    envs = [scenes.rigid_environment(s, 500, 4000) for s in range(12)]
    batch = envs[:5] + [empty_scene()] + [scenes.folded_cloth(24, seed=3)] + envs[5:] + \
        [scenes.icosphere_on_plane(2, level=2, plane_n=9)]
    c = ccd.CCD(0, sweep_kernel=sweep, strip_width=width)
    try:
        got = c.step_batch(batch)
        again = c.step_batch(batch)
    finally:
        c.close()
    ref = np.array([O.step(s.V0, s.V1, s.E, s.F) if len(s.V0) else np.inf for s in batch])
    np.testing.assert_array_equal(got.view(np.uint64), ref.view(np.uint64))
    np.testing.assert_array_equal(again.view(np.uint64), ref.view(np.uint64))
    assert np.isfinite(ref).sum() >= 3 and np.isinf(ref).sum() >= 2


def test_batch_single_scene_equals_step(ccd):
    s = scenes.folded_cloth(48, seed=1)
    c = ccd.CCD(0)
    try:
        got = c.step_batch([s])
        d = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        assert got[0] == c.step(*d) == O.step(s.V0, s.V1, s.E, s.F)
    finally:
        c.close()


def test_graph_replay_step_and_batch(ccd):
    c = ccd.CCD(0, use_graph=1)
    try:
        s = scenes.folded_cloth(40, seed=1)
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        ref = O.step(s.V0, s.V1, s.E, s.F)
        for _ in range(3):                       # capture, then replays
            ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
            torch.cuda.synchronize()
            assert float(out.item()) == ref
        # new positions in the same buffers: a replay must read them
        s2 = scenes.folded_cloth(40, seed=7)
        V1.copy_(torch.from_numpy(np.ascontiguousarray(s2.V1.T)).cuda())
        ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
        torch.cuda.synchronize()
        assert float(out.item()) == O.step(s.V0, s2.V1, s.E, s.F)
        # batched step under a graph
        envs = [scenes.rigid_environment(k, 500, 3000) for k in range(6)]
        Vb0, Vb1, Eb, Fb, vo, eo, fo = scenes.concat_scenes(envs)
        d = ccd.mesh_to_device(Vb0, Vb1, Eb, Fb)
        offs = [torch.from_numpy(a).cuda() for a in (vo, eo, fo)]
        tb = torch.empty(len(envs), dtype=torch.float64, device="cuda")
        refb = np.array([O.step(e.V0, e.V1, e.E, e.F) for e in envs])
        for _ in range(2):
            ccd.ccd_step_batch(c.ctx, *offs, *d, 1e-6, 0.0, 10 ** 6, tb)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(tb.cpu().numpy().view(np.uint64), refb.view(np.uint64))
        assert c.status()[0] == 0
    finally:
        c.close()
