"""The allocation-free narrow phase (ccd_narrow_noalloc) against the
context-based one (ccd_narrow), through the C ABI, twice in a row.

It serves callers that cannot allocate device memory at the point of the
query.  Its scratch is a fixed array inside the library that every call
reuses, so the second call also checks that a call starts clean after the
previous one.  Kept in a file that pytest collects last."""
import numpy as np
import pytest

from paper_2112_06300_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_narrow_two_calls():
    from paper_2112_06300_gb300 import build
    build.build()
    from paper_2112_06300_gb300 import ccd
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(3000, seed=11)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    V0, V1, E, F = ccd.mesh_to_device(sc.V0, sc.V1, sc.E, sc.F)
    vfd = torch.from_numpy(vf).cuda()
    eed = torch.from_numpy(ee).cuda()
    c = ccd.CCD(0)
    try:
        ref = c.narrow(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 0)
    finally:
        c.close()
    rg = np.concatenate([ref.toi_vf.cpu().numpy(), ref.toi_ee.cpu().numpy()])
    rf = np.concatenate([ref.flags_vf.cpu().numpy(), ref.flags_ee.cpu().numpy()])
    for call in range(2):
        tv = torch.full((len(vf),), -1.0, dtype=torch.float64, device="cuda")
        te = torch.full((len(ee),), -1.0, dtype=torch.float64, device="cuda")
        fv = torch.full((len(vf),), 255, dtype=torch.uint8, device="cuda")
        fe = torch.full((len(ee),), 255, dtype=torch.uint8, device="cuda")
        tm = torch.empty(1, dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        ccd.ccd_narrow_noalloc(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 0, tv, te, fv, fe, tm, st)
        torch.cuda.synchronize()
        assert int(st.item()) == ccd.CCD_OK, f"call {call}: device status {int(st.item())}"
        g = np.concatenate([tv.cpu().numpy(), te.cpu().numpy()])
        gf = np.concatenate([fv.cpu().numpy(), fe.cpu().numpy()])
        ok = (gf == 0) & (rf == 0)
        assert ok.mean() > 0.99
        np.testing.assert_array_equal(g[ok].view(np.uint64), rg[ok].view(np.uint64))
        assert float(tm.item()) == ref.toi_min
        # earliest-only mode on the same scratch
        ccd.ccd_narrow_noalloc(vfd, eed, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, 1, None, None, None, None, tm, st)
        torch.cuda.synchronize()
        assert int(st.item()) == ccd.CCD_OK and float(tm.item()) == ref.toi_min


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
