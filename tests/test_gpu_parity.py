"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Broad phase: the pair set is compared exactly (sorted; the GPU returns it in
unspecified order), and the single-precision superset count equals the
oracle's single-precision pair set.  Narrow phase: per-pair times of impact
are bit-identical on every pair neither side flagged (the result of an
uncapped query does not depend on the traversal order), flags agree, and the
earliest time is bit-identical.  Sizes span several tiles and ragged tails;
edge cases: empty inputs, vertices only, forced queue hand-offs, a tiny
queue, max_iter = 0, min_sep > 0."""
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


@pytest.fixture(scope="module")
def ctx(ccd):
    c = ccd.CCD(0)
    yield c
    c.close()


def sorted_pairs(t):
    a = t.cpu().numpy().astype(np.int64).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a


def random_scene(seed, nv=300, nf=250, motion=0.05):
    rng = np.random.default_rng(seed)
    V0 = rng.uniform(-1, 1, (nv, 3))
    V1 = V0 + rng.normal(0, motion, (nv, 3))
    F = np.array([rng.choice(nv, 3, replace=False) for _ in range(nf)], np.int32)
    return scenes.Scene(V0, V1, scenes.edges_of(F), F, {"name": f"random-{seed}"})


def scene_list():
    out = [scenes.icosphere_on_plane(0),                       # 21,635 boxes
           scenes.icosphere_on_plane(3, level=2, plane_n=9),
           scenes.folded_cloth(40, seed=1),
           scenes.folded_cloth(97, seed=4),                    # ragged sort tiles
           random_scene(0), random_scene(1, nv=31, nf=7)]
    return out


SCENES = scene_list()


@pytest.mark.parametrize("s", SCENES, ids=[s.info["name"] + str(i) for i, s in enumerate(SCENES)])
def test_broad_pairs_match_oracle(ctx, ccd, s):
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    vf, ee = ctx.broad(V0, V1, E, F)
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    np.testing.assert_array_equal(sorted_pairs(vf), ovf)
    np.testing.assert_array_equal(sorted_pairs(ee), oee)
    rc, st = ctx.status()
    assert rc == 0
    v32, e32 = O.broad(s.V0, s.V1, s.E, s.F, fp32=True)
    assert st["n_superset"] == len(v32) + len(e32)
    assert st["n_boxes"] == s.n_boxes


def test_broad_empty_and_vertices_only(ctx, ccd):
    z = np.zeros((0, 3))
    V0, V1, E, F = ccd.mesh_to_device(z, z, np.zeros((0, 2), np.int32), np.zeros((0, 3), np.int32))
    vf, ee = ctx.broad(V0, V1, E, F)
    assert vf.shape[0] == 0 and ee.shape[0] == 0
    pts = np.random.default_rng(0).uniform(0, 1, (500, 3))
    V0, V1, E, F = ccd.mesh_to_device(pts, pts, np.zeros((0, 2), np.int32), np.zeros((0, 3), np.int32))
    vf, ee = ctx.broad(V0, V1, E, F)
    assert vf.shape[0] == 0 and ee.shape[0] == 0


@pytest.mark.parametrize("offset", [2.0 ** 20, -(2.0 ** 24)])
def test_broad_far_from_origin_matches_oracle(ctx, ccd, offset):
    """A scene moved far from the origin: the outward-rounded float boxes grow
    to the float spacing there (1/8 at 2^20, 2 at 2^24, where every box
    overlaps every other and the cell grid collapses to one cell), so the
    single-precision superset grows (1.5x and 3.6x the exact set here) and
    the exact FP64 filter alone brings it back to the oracle's set."""
    s = random_scene(7, nv=200, nf=160)
    s = scenes.Scene(s.V0 + offset, s.V1 + offset, s.E, s.F, {"name": "far"})
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    vf, ee = ctx.broad(V0, V1, E, F)
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    np.testing.assert_array_equal(sorted_pairs(vf), ovf)
    np.testing.assert_array_equal(sorted_pairs(ee), oee)
    rc, st = ctx.status()
    assert rc == 0
    v32, e32 = O.broad(s.V0, s.V1, s.E, s.F, fp32=True)
    assert st["n_superset"] == len(v32) + len(e32)
    assert len(v32) + len(e32) > len(ovf) + len(oee)


def test_broad_truncation_reports_totals(ctx, ccd):
    s = scenes.icosphere_on_plane(0)
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    vf = torch.empty((10, 2), dtype=torch.int32, device="cuda")
    ee = torch.empty((10, 2), dtype=torch.int32, device="cuda")
    rc, nvf, nee = ccd.ccd_broad(ctx.ctx, V0, V1, E, F, vf, ee)
    assert rc == ccd.CCD_ETRUNC
    assert (nvf, nee) == (len(ovf), len(oee))
    got = {tuple(p) for p in vf.cpu().numpy().tolist()}
    assert got <= {tuple(p) for p in ovf.tolist()}


def _narrow_both(ctx, ccd, s, vf, ee, delta=1e-6, ms=0.0, max_iter=10 ** 6, mode=0):
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    vfd = torch.from_numpy(np.ascontiguousarray(vf, np.int32)).cuda().reshape(-1, 2)
    eed = torch.from_numpy(np.ascontiguousarray(ee, np.int32)).cuda().reshape(-1, 2)
    r = ctx.narrow(vfd, eed, V0, V1, E, F, delta, ms, max_iter, mode)
    o = O.narrow(vf, ee, s.V0, s.V1, s.E, s.F, delta, ms, max_iter, mode)
    return r, o


def _assert_per_pair(r, o):
    g = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    gf = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    t = np.concatenate([o[0], o[1]])
    f = np.concatenate([o[2], o[3]])
    both = (gf == 0) & (f == 0)
    assert both.mean() > 0.99
    np.testing.assert_array_equal(g[both].view(np.uint64), t[both].view(np.uint64))
    # a flagged result is still conservative: never later than the uncapped one
    np.testing.assert_array_equal(gf, f)
    assert r.toi_min == o[4]


@pytest.mark.parametrize("s", SCENES[:5], ids=[s.info["name"] + str(i) for i, s in enumerate(SCENES[:5])])
def test_narrow_per_pair_matches_oracle(ctx, ccd, s):
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    r, o = _narrow_both(ctx, ccd, s, ovf, oee)
    _assert_per_pair(r, o)


def _stress(n, seed):
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(n, seed)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    return sc, vf, ee


@pytest.mark.parametrize("n,seed", [(5000, 2), (777, 5)])
def test_narrow_stress_mix_matches_oracle(ctx, ccd, n, seed):
    sc, vf, ee = _stress(n, seed)
    r, o = _narrow_both(ctx, ccd, sc, vf, ee)
    _assert_per_pair(r, o)


@pytest.mark.parametrize("scale,offset", [(1.0, 2.0 ** 16), (1.0, 2.0 ** 30), (2.0 ** -13, 0.0),
                                          (2.0 ** -100, 0.0), (2.0 ** 20, -3.0), (2.0 ** -40, 1.0)])
def test_narrow_stress_scaled_matches_oracle(ctx, ccd, scale, offset):
    """The stress mix shrunk, grown and moved away from the origin, with delta
    scaled alike.  The single-precision filter's thresholds follow the
    coordinates (bounds relative to the per-axis sums of |c0| + |dc|, floors
    near the bottom of the float range at 2^-100); far from the origin the
    error box outgrows delta (2^30) or the 2^-60 grid rounds away (2^-40 at
    1.0), leaving degenerate, noisy queries.  Every decision the filter takes
    must still be the FP64 one.  A few of these queries take over 10^6
    intervals, so the cap is 10^7, which no query reaches on either side (a
    query split across lanes reaches a cap elsewhere than the oracle does)."""
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(1500, 11)
    sc, vf, ee, order = scenes.pack_queries(X0 * scale + offset, X1 * scale + offset, is_vf)
    r, o = _narrow_both(ctx, ccd, sc, vf, ee, delta=1e-6 * scale, max_iter=10 ** 7)
    assert not np.concatenate([o[2], o[3]]).any()
    _assert_per_pair(r, o)


def test_narrow_deep_trees_match_oracle(ctx, ccd):
    """delta = 1e-10 takes the bisection past 31 and 63 levels in total (most
    of the evaluations here), beyond the 31 levels below a unit's start that
    the kernel's path masks cover: deeper units backtrack by walking the path,
    and the pieces other lanes take from them start masks of their own at
    their depth.  The reference is the oracle without an
    iteration cap: the GPU result equals it wherever the GPU did not cap the
    query, and is never later where it did (a query split across lanes can
    reach the cap in a different place; capped results are conservative)."""
    sc, vf, ee = _stress(2000, 9)
    delta = 1e-10
    r, _ = _narrow_both(ctx, ccd, sc, vf, ee, delta=delta)
    ox = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F, delta, 0.0, 10 ** 8, 0)
    t = np.concatenate([ox[0], ox[1]])
    assert not np.concatenate([ox[2], ox[3]]).any()
    g = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    gf = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    assert (gf == 0).mean() > 0.99
    np.testing.assert_array_equal(g[gf == 0].view(np.uint64), t[gf == 0].view(np.uint64))
    assert (g[gf != 0] <= t[gf != 0]).all()
    r1, _ = _narrow_both(ctx, ccd, sc, vf, ee, delta=delta, mode=1)
    assert r1.toi_min <= ox[4]
    if not gf.any():
        assert r1.toi_min == ox[4]


def test_narrow_min_sep_matches_oracle(ctx, ccd):
    sc, vf, ee = _stress(600, 8)
    r, o = _narrow_both(ctx, ccd, sc, vf, ee, ms=1e-4, max_iter=20000)
    g = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    gf = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    t = np.concatenate([o[0], o[1]])
    f = np.concatenate([o[2], o[3]])
    both = (gf == 0) & (f == 0)
    np.testing.assert_array_equal(g[both].view(np.uint64), t[both].view(np.uint64))


def test_narrow_max_iter_zero(ctx, ccd):
    sc, vf, ee = _stress(300, 3)
    r, o = _narrow_both(ctx, ccd, sc, vf, ee, max_iter=0)
    g = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    t = np.concatenate([o[0], o[1]])
    np.testing.assert_array_equal(g.view(np.uint64), t.view(np.uint64))


def test_narrow_earliest_mode_capped(ctx, ccd):
    """max_iter = 0 caps every query at its root, whose left end is 0: the
    capped value must reach the earliest time in mode 1 as in mode 0."""
    sc, vf, ee = _stress(300, 3)
    for mode in (0, 1):
        r, o = _narrow_both(ctx, ccd, sc, vf, ee, max_iter=0, mode=mode)
        assert r.toi_min == o[4] == 0.0


def test_narrow_earliest_mode(ctx, ccd):
    for s in SCENES[:4]:
        ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
        r, o = _narrow_both(ctx, ccd, s, ovf, oee, mode=1)
        per = O.narrow(ovf, oee, s.V0, s.V1, s.E, s.F, mode=0)
        assert r.toi_min == o[4] == per[4]


@pytest.mark.parametrize("budget,qcap", [(1, 0), (4, 0), (2, 64)])
def test_narrow_handoff_paths_keep_results(ccd, budget, qcap):
    # hand-offs every 32 evaluations of a warp (most work goes through the
    # ring), and a ring too small to take most hand-offs: results must not change
    c = ccd.CCD(0, export_budget=budget, queue_capacity=qcap)
    try:
        s = scenes.folded_cloth(40, seed=1)
        ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
        r, o = _narrow_both(c, ccd, s, ovf, oee)
        _assert_per_pair(r, o)
        rc, st = c.status()
        assert rc == 0
        if qcap == 0:
            assert st["n_exported"] > 0
        r1, o1 = _narrow_both(c, ccd, s, ovf, oee, mode=1)
        assert r1.toi_min == o1[4]
    finally:
        c.close()


@pytest.mark.parametrize("s", [SCENES[0], SCENES[2], SCENES[3]], ids=["icosphere", "cloth40", "cloth97"])
def test_step_matches_oracle(ctx, ccd, s):
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
    t = ctx.step(V0, V1, E, F)
    assert t == O.step(s.V0, s.V1, s.E, s.F)
    # device-pointer output, asynchronous path
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    ccd.ccd_step(ctx.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
    torch.cuda.synchronize()
    assert float(out.item()) == t


def test_step_grows_pair_buffers(ccd):
    c = ccd.CCD(0, pair_capacity=64)
    try:
        s = scenes.folded_cloth(40, seed=1)
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        assert c.step(V0, V1, E, F) == O.step(s.V0, s.V1, s.E, s.F)
    finally:
        c.close()


def test_fp64_peak_probe(ccd):
    g = ccd.ccd_measure_fp64_peak(0)
    assert 10.0 < g < 1e6


@pytest.mark.parametrize("sweep,width", [(0, 0.0), (0, 0.5), (0, 1e-3), (1, 0.0)],
                         ids=["strips", "narrow-strips", "strips-overflow", "warp-per-box"])
@pytest.mark.parametrize("s", [SCENES[0], SCENES[3], SCENES[4]], ids=["icosphere", "cloth97", "random"])
def test_plain_fp64_form_matches_oracle(ccd, s, sweep, width):
    # all-FP64 broad phase: 64-bit keys, exact comparisons, no single-precision
    # stage (strips binned on FP64 extents, or one warp per box)
    c = ccd.CCD(0, broad_fp64=1, sweep_kernel=sweep, strip_width=width)
    try:
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        vf, ee = c.broad(V0, V1, E, F)
        ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
        np.testing.assert_array_equal(sorted_pairs(vf), ovf)
        np.testing.assert_array_equal(sorted_pairs(ee), oee)
        rc, st = c.status()
        assert rc == 0 and st["n_superset"] == len(ovf) + len(oee)
        assert c.step(V0, V1, E, F) == O.step(s.V0, s.V1, s.E, s.F)
    finally:
        c.close()


def big_box_scene(seed=5):
    """Small random triangles plus one triangle spanning the whole scene: its
    box overlaps every strip."""
    s = random_scene(seed, nv=400, nf=300, motion=0.02)
    V0 = np.vstack([s.V0, [[-1.5, -1.5, 0.0], [1.5, -1.5, 0.1], [0.0, 1.5, -0.1]]])
    V1 = np.vstack([s.V1, [[-1.5, -1.5, 0.0], [1.5, -1.5, 0.1], [0.0, 1.5, -0.1]]])
    F = np.vstack([s.F, [[400, 401, 402]]]).astype(np.int32)
    return scenes.Scene(V0, V1, scenes.edges_of(F), F, {"name": "big-box"})


@pytest.mark.parametrize("sweep,width", [(1, 0.0), (2, 0.0), (0, 0.5), (0, 1.0), (0, 4.0), (0, 1e6), (0, 1e-3)],
                         ids=["warp-per-box", "tiled", "strips0.5", "strips1", "strips4", "one-strip",
                              "strips-overflow"])
@pytest.mark.parametrize("s", [SCENES[0], SCENES[3], SCENES[5], big_box_scene()],
                         ids=["icosphere", "cloth97", "tiny", "big-box"])
def test_sweep_variants_match_oracle(ccd, s, sweep, width):
    """Every sweep kernel and strip width gives the oracle's pair set and the
    single-precision superset count (each pair reported once); a strip width
    of 1e-3 mean widths overflows the copy buffers and takes the one-strip
    fallback."""
    c = ccd.CCD(0, sweep_kernel=sweep, strip_width=width)
    try:
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        vf, ee = c.broad(V0, V1, E, F)
        ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
        np.testing.assert_array_equal(sorted_pairs(vf), ovf)
        np.testing.assert_array_equal(sorted_pairs(ee), oee)
        rc, st = c.status()
        assert rc == 0
        v32, e32 = O.broad(s.V0, s.V1, s.E, s.F, fp32=True)
        assert st["n_superset"] == len(v32) + len(e32)
        if sweep != 0 or width == 1e-3:
            assert st["n_box_copies"] == s.n_boxes
        else:
            assert st["n_box_copies"] >= s.n_boxes
    finally:
        c.close()


def test_no_zero_toi_rule_matches_oracle(ccd):
    c = ccd.CCD(0, no_zero_toi=1)
    try:
        h = 2.0 ** -12
        tri = [(0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)]
        V0 = np.array([(0.25, 0.25, h)] + tri)
        V1 = np.array([(0.25, 0.25, h - 1.0)] + tri)
        E = np.array([[1, 2], [2, 3], [3, 1]], np.int32)
        F = np.array([[1, 2, 3]], np.int32)
        d = ccd.mesh_to_device(V0, V1, E, F)
        t = c.step(*d, min_sep=0.01)
        assert t == O.step(V0, V1, E, F, min_sep=0.01, no_zero_toi=True) and t > 0
        # scenes whose first pass is 0 with a large min_sep (that pass ends as
        # soon as one pair is within min_sep at t = 0), and one whose is not
        for s, ms in ((SCENES[2], 0.05), (SCENES[0], 0.3), (SCENES[0], 0.0)):
            d = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
            t = c.step(*d, min_sep=ms)
            assert t == O.step(s.V0, s.V1, s.E, s.F, min_sep=ms, no_zero_toi=True)
    finally:
        c.close()


@pytest.mark.parametrize("pairs", [20000, 3000])
def test_memory_limited_step_runs_in_ranges(ccd, pairs):
    """A memory limit that fits fewer candidate pairs than the step has: the
    step sweeps ranges of the sorted boxes (the paper's batching) and still
    returns the oracle's earliest time."""
    s = scenes.folded_cloth(64, seed=1)
    m = ccd.ccd_get_memory_model()
    limit = m["bytes_fixed"] + max(s.n_boxes, 1024) * m["bytes_per_box"] + pairs * m["bytes_per_pair"]
    c = ccd.CCD(0, memory_limit=limit)
    try:
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        t = c.step(V0, V1, E, F)
        rc, st = c.status()
        assert rc == 0 and st["n_ranges"] >= 2
        assert t == O.step(s.V0, s.V1, s.E, s.F)
    finally:
        c.close()
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    assert len(ovf) + len(oee) > pairs


def test_cloth_min_sep_step(ccd):
    """The cloth with min_sep = 1e-4: the first contact within min_sep is a
    patch, so some queries may reach the iteration cap.  Per pair (own t*
    per query): bit-identical to the oracle on every query neither side
    flagged; where the two earliest times differ, the earlier one comes from
    a flagged (capped) query.  The earliest-time step equals the oracle's
    unless a query was capped, and stays conservative (no later than with
    min_sep = 0)."""
    s = scenes.folded_cloth(64, seed=1)
    c = ccd.CCD(0)
    try:
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        vf, ee = c.broad(V0, V1, E, F)
        gvf, gee = sorted_pairs(vf), sorted_pairs(ee)
        r = c.narrow(torch.from_numpy(gvf.astype(np.int32)).cuda(), torch.from_numpy(gee.astype(np.int32)).cuda(),
                     V0, V1, E, F, 1e-6, 1e-4, 10 ** 6, 0)
        assert c.status()[0] == 0
        t = c.step(V0, V1, E, F, min_sep=1e-4)
        rc, st = c.status()
        assert rc == 0
        gpu_capped = st["n_capped"]
        t0 = c.step(V0, V1, E, F, min_sep=0.0)
    finally:
        c.close()
    ovf, oee = O.broad(s.V0, s.V1, s.E, s.F)
    assert np.array_equal(gvf, ovf) and np.array_equal(gee, oee)
    otv, ote, ofv, ofe, _ = O.narrow(ovf, oee, s.V0, s.V1, s.E, s.F, 1e-6, 1e-4, 10 ** 6, 0)
    g = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    gf = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    o = np.concatenate([otv, ote])
    of = np.concatenate([ofv, ofe])
    ok = (gf == 0) & (of == 0)
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(g[ok].view(np.uint64), o[ok].view(np.uint64))
    if g.min() != o.min():
        first = int(np.argmin(g)) if g.min() < o.min() else int(np.argmin(o))
        assert gf[first] != 0 or of[first] != 0, "earliest times differ on an unflagged query"
    # earliest-time step (one shared t*)
    to_vf, to_ee, fo_vf, fo_ee, to = O.narrow(ovf, oee, s.V0, s.V1, s.E, s.F, 1e-6, 1e-4, 10 ** 6, 1)
    oracle_capped = int(np.count_nonzero(np.concatenate([fo_vf, fo_ee]) & 1))
    assert 0.0 < t <= t0
    if gpu_capped == 0 and oracle_capped == 0:
        assert t == to
    else:
        # a capped query's result is the earliest left end of its live
        # intervals: conservative, and no later than the uncapped minimum
        assert t <= np.min(g[ok]) and to <= np.min(o[ok])
