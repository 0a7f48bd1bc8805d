"""Serving runtime and memory model on the GPU.

Every scene served in a mix of others (continuous batching over two slots,
batches bounded by scene count) gets the earliest time it gets alone and the
oracle's, bit for bit; scenes submitted from two threads at once, an empty
scene and a batch limit of one scene are covered.  The memory model predicts
what a context allocates for a step."""
import threading

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


def mix():
    envs = [scenes.rigid_environment(s, 500, 3000, vmax=0.2) for s in range(24)]
    return envs[:7] + [empty_scene(), scenes.folded_cloth(24, seed=3)] + envs[7:] + \
        [scenes.icosphere_on_plane(2, level=2, plane_n=9)]


@pytest.mark.parametrize("max_scenes,n_slots,tune", [(6, 2, 0), (1, 1, 0), (256, 3, 0), (8, 2, 1)])
def test_served_scene_equals_alone_and_oracle(ccd, max_scenes, n_slots, tune):
    batch = mix()
    ref = np.array([O.step(s.V0, s.V1, s.E, s.F) if len(s.V0) else np.inf for s in batch])
    c = ccd.CCD(0)
    try:
        alone = np.array([c.step_batch([s])[0] for s in batch])
    finally:
        c.close()
    np.testing.assert_array_equal(alone.view(np.uint64), ref.view(np.uint64))
    srv = ccd.Server(0, n_slots=n_slots, max_scenes=max_scenes, arena_bytes=64 << 20, memory_cap=8 << 30,
                     autotune=tune)
    try:
        tickets = [srv.submit_scene(s.V0, s.V1, s.E, s.F) for s in batch]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    toi = np.array([g[0] for g in got])
    np.testing.assert_array_equal(toi.view(np.uint64), ref.view(np.uint64))
    assert all(g[1] >= 0 for g in got)
    assert st["n_done"] == len(batch) and st["max_batch_scenes"] <= max_scenes
    assert np.isfinite(ref).sum() >= 3


def test_two_submitting_threads(ccd):
    envs = [scenes.rigid_environment(s, 500, 2000, vmax=0.2) for s in range(30, 50)]
    ref = {k: O.step(e.V0, e.V1, e.E, e.F) for k, e in enumerate(envs)}
    srv = ccd.Server(0, n_slots=2, max_scenes=4, arena_bytes=32 << 20, memory_cap=8 << 30)
    out = {}

    def client(ks):
        tick = [(k, srv.submit_scene(envs[k].V0, envs[k].V1, envs[k].E, envs[k].F)) for k in ks]
        for k, t in tick:
            out[k] = srv.wait(t)[0]

    try:
        th = [threading.Thread(target=client, args=(range(i, len(envs), 2),)) for i in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    finally:
        srv.close()
    assert out == ref


def test_memory_model_matches_allocation(ccd):
    s = scenes.folded_cloth(96, seed=1)
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    c = ccd.CCD(0)
    try:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        assert c.status()[0] == 0
    finally:
        c.close()
    m = ccd.ccd_get_memory_model()
    nB = s.n_boxes
    pairs = max(1 << 20, 4 * nB)
    model = m["bytes_fixed"] + max(nB, 1024) * m["bytes_per_box"] + pairs * m["bytes_per_pair"]
    assert 0.9 * model <= used <= 1.15 * model + (64 << 20), (used, model)
    # the capacity the model grants for that budget is the one used above
    assert abs(ccd.ccd_pair_capacity_for(model, nB) - pairs) <= 1


def test_memory_cap_binds(ccd):
    """A memory cap that fits two scenes per slot: scenes submitted at once
    are held until a slot and its memory share free up, every batch stays
    within the share, the batches in flight together stay within the cap,
    the device memory the server's contexts hold stays near it, and every
    result equals the oracle's bit for bit."""
    batch = [scenes.folded_cloth(64, seed=10 + k) for k in range(7)]
    ref = np.array([O.step(s.V0, s.V1, s.E, s.F) for s in batch])
    m = ccd.ccd_get_memory_model()
    ppb = 64.0
    nb = batch[0].n_boxes

    def need(k):   # the server's memory-model estimate of a batch of k scenes
        boxes = k * nb
        return (m["bytes_fixed"] + max(boxes, 1024) * m["bytes_per_box"] + k * m["bytes_per_scene"]
                + max(1 << 20, int(ppb * boxes)) * m["bytes_per_pair"])

    assert need(2) < need(3)
    n_slots = 2
    share = (need(2) + need(3)) // 2
    cap = n_slots * share
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    srv = ccd.Server(0, n_slots=n_slots, max_scenes=256, arena_bytes=64 << 20, memory_cap=cap,
                     pairs_per_box=ppb)
    try:
        # write every scene first and queue them last-first: the scheduler
        # takes scenes in request order, so nothing starts before the first
        # one is queued and all seven are waiting at once
        tickets = []
        for s in batch:
            t, a, b, e, f = srv.request(len(s.V0), len(s.E), len(s.F))
            a[...] = s.V0.T
            b[...] = s.V1.T
            e[...] = s.E
            f[...] = s.F
            tickets.append(t)
        for t in reversed(tickets):
            srv.submit(t)
        got = [srv.wait(t) for t in tickets]
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        st = srv.stats()
    finally:
        srv.close()
    toi = np.array([g[0] for g in got])
    np.testing.assert_array_equal(toi.view(np.uint64), ref.view(np.uint64))
    assert st["max_batch_scenes"] == 2, st
    assert st["n_batches"] >= 4, st
    assert st["max_batch_bytes"] <= share and st["max_inflight_bytes"] <= cap, st
    assert used <= 1.15 * cap + (64 << 20), (used, cap)


def test_submit_scene_copies_from_caller_arrays(ccd):
    """ccd_server_submit_scene (copy into the arena and queue in one call),
    from two client threads: every result equals the oracle's."""
    envs = [scenes.rigid_environment(s, 500, 3000, vmax=0.2) for s in range(60, 72)]
    ref = {k: O.step(e.V0, e.V1, e.E, e.F) for k, e in enumerate(envs)}
    soa = [(np.ascontiguousarray(e.V0.T), np.ascontiguousarray(e.V1.T), np.ascontiguousarray(e.E, np.int32),
            np.ascontiguousarray(e.F, np.int32)) for e in envs]
    srv = ccd.Server(0, n_slots=2, max_scenes=3, arena_bytes=32 << 20, memory_cap=8 << 30)
    out = {}

    def client(ks):
        tick = [(k, srv.submit_soa(*soa[k])) for k in ks]
        for k, t in tick:
            out[k] = srv.wait(t)[0]

    try:
        th = [threading.Thread(target=client, args=(range(i, len(envs), 2),)) for i in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    finally:
        srv.close()
    assert out == ref
