"""The narrow-phase stress workload at full size: 2^24 standalone queries
(50/50 vertex-face / edge-edge on the 2^-20 grid; 40/20/10/10/20 % generic /
collide at a seeded dyadic time / coplanar-or-parallel / touching at t = 0 or
1 / near miss at 2^-30..2^-40), per-pair times on the GPU.

Checked: bit-identical to the FP64 oracle on a seeded sample of 50,000
queries neither side flagged; against the exact rational oracle on the
100,000-query subset stored in tests/golden/stress_exact_1e5.txt.gz (exact
times computed by make_stress_exact.py with oracle/exact.py only): no false
negative and never later than the exact time.  The false-positive count (a
collision reported where the exact oracle finds none) and the distribution
of t_exact - t_gpu are printed."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_06300_gb300 import scenes
from tests.golden import make_stress_exact as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 1 << 24


def test_stress_full_size_sampled():
    rng = np.random.default_rng(0)
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(N, 2)
    head, exact_idx, exact_rd = G.read()
    assert head["sha256"] == G.fingerprint(X0, X1, is_vf, exact_idx), "stress generator changed"

    from paper_2112_06300_gb300 import build
    build.build()
    from paper_2112_06300_gb300 import ccd
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    V0, V1, E, F = ccd.mesh_to_device(sc.V0, sc.V1, sc.E, sc.F)
    c = ccd.CCD(0)
    try:
        vfd = torch.from_numpy(vf).cuda()
        eed = torch.from_numpy(ee).cuda()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = c.narrow(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 0)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        assert c.status()[0] == 0
        stacked = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
        sflags = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    finally:
        c.close()
    del V0, V1, E, F
    toi = np.empty(N)
    flags = np.empty(N, np.uint8)
    toi[order] = stacked
    flags[order] = sflags
    print(f"\n2^24 stress queries: narrow phase {ms:.1f} ms ({N / ms * 1e3:.3g} queries/s), "
          f"{int(np.isfinite(toi).sum())} collisions, {int((flags != 0).sum())} flagged")

    # FP64 oracle on a sample: bit-identical where neither side flagged
    s = rng.choice(N, size=50000, replace=False)
    s_sc, s_vf, s_ee, s_order = scenes.pack_queries(X0[s], X1[s], is_vf[s])
    o = O.narrow(s_vf, s_ee, s_sc.V0, s_sc.V1, s_sc.E, s_sc.F, 1e-6, 0.0, 10 ** 6, 0)
    otoi = np.empty(len(s))
    oflag = np.empty(len(s), np.uint8)
    otoi[s_order] = np.concatenate([o[0], o[1]])
    oflag[s_order] = np.concatenate([o[2], o[3]])
    both = (oflag == 0) & (flags[s] == 0)
    assert both.mean() > 0.99
    np.testing.assert_array_equal(toi[s][both].view(np.uint64), otoi[both].view(np.uint64))

    # exact oracle on the stored 1e5 subset: conservative, no false negative
    r = G.summarize(toi[exact_idx], flags[exact_idx], exact_rd)
    print(f"exact-oracle subset: {r['n']} queries, {r['n_collide']} collide; false negatives {r['fn']}, "
          f"late {r['late']}, false positives {r['fp']} ({r['fp_rate']:.3%} of non-colliding); "
          f"t_exact - t_gpu: median {r['err_median']:.3g}, mean {r['err_mean']:.3g}, max {r['err_max']:.3g}")
    assert r["fn"] == 0 and r["late"] == 0

