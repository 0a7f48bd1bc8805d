"""The allocation-free narrow phase (ccd_narrow_noalloc) through the C ABI,
against the FP64 oracle and against the context-based ccd_narrow, on several
calls in a row.

It serves callers that cannot allocate device memory at the point of the
query.  Its scratch is a fixed array inside the library that every call
reuses, so the calls after the first also check that a call starts clean
after the previous one (another mode, another number of queries).  Kept in
a file that pytest collects last."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2112_06300_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(ccd, vfd, eed, V0, V1, E, F, mode):
    nv, ne = len(vfd), len(eed)
    tv = torch.full((nv,), -1.0, dtype=torch.float64, device="cuda")
    te = torch.full((ne,), -1.0, dtype=torch.float64, device="cuda")
    fv = torch.full((nv,), 255, dtype=torch.uint8, device="cuda")
    fe = torch.full((ne,), 255, dtype=torch.uint8, device="cuda")
    tm = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    if mode == 0:
        ccd.ccd_narrow_noalloc(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 0, tv, te, fv, fe, tm, st)
    else:
        ccd.ccd_narrow_noalloc(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 1, None, None, None, None, tm, st)
    torch.cuda.synchronize()
    assert int(st.item()) == ccd.CCD_OK, f"device status {int(st.item())}"
    return (np.concatenate([tv.cpu().numpy(), te.cpu().numpy()]),
            np.concatenate([fv.cpu().numpy(), fe.cpu().numpy()]), float(tm.item()))


def test_noalloc_matches_oracle_and_narrow_over_calls():
    from paper_2112_06300_gb300 import build
    build.build()
    from paper_2112_06300_gb300 import ccd
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(3000, seed=11)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    # the FP64 oracle on the same pairs
    otv, ote, ofv, ofe, omin = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F, 1e-6, 0.0, 10 ** 6, 0)
    og = np.concatenate([otv, ote])
    of = np.concatenate([ofv, ofe])
    V0, V1, E, F = ccd.mesh_to_device(sc.V0, sc.V1, sc.E, sc.F)
    vfd = torch.from_numpy(vf).cuda()
    eed = torch.from_numpy(ee).cuda()
    c = ccd.CCD(0)
    try:
        ref = c.narrow(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 0)
    finally:
        c.close()
    rg = np.concatenate([ref.toi_vf.cpu().numpy(), ref.toi_ee.cpu().numpy()])
    assert ref.toi_min == omin
    half_vf, half_ee = len(vf) // 2, len(ee) // 2
    for call, mode, part in ((0, 0, "all"), (1, 1, "all"), (2, 0, "half"), (3, 0, "all")):
        if part == "all":
            g, gf, tm = _noalloc(ccd, vfd, eed, V0, V1, E, F, mode)
            sel = np.arange(len(og))
        else:
            g, gf, tm = _noalloc(ccd, vfd[:half_vf], eed[:half_ee], V0, V1, E, F, mode)
            sel = np.concatenate([np.arange(half_vf), len(vf) + np.arange(half_ee)])
        if mode == 1:
            assert tm == omin, f"call {call}: earliest time {tm} != oracle {omin}"
            continue
        ok = (gf == 0) & (of[sel] == 0)
        assert ok.mean() > 0.99, f"call {call}"
        # bit-identical to the oracle and to ccd_narrow on unflagged queries
        np.testing.assert_array_equal(g[ok].view(np.uint64), og[sel][ok].view(np.uint64))
        np.testing.assert_array_equal(g[ok].view(np.uint64), rg[sel][ok].view(np.uint64))
        if not of[sel].any() and not gf.any():
            assert tm == np.min(og[sel]), f"call {call}: earliest time"


def test_noalloc_rejects_more_pairs_than_its_scratch():
    from paper_2112_06300_gb300 import ccd
    n = (1 << 16) + 1
    vf = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    ee = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    V = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    E = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    F = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    tm = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ccd.CCDError) as e:
        ccd.ccd_narrow_noalloc(vf, ee, V, V, E, F, 1e-6, 0.0, 10, 1, None, None, None, None, tm, st)
    assert e.value.status == ccd.CCD_EINVAL
