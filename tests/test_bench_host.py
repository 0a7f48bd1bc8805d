"""Host logic of bench.py that needs no GPU: the default launch (one GPU, at
least 3 warm-up steps) and the algorithmic work per stage that the roofline
fractions divide by (bytes per box, copy and candidate; FP64-equivalent flops
per interval and per unit of narrow-phase work)."""
import sys

import bench


def test_default_launch_is_one_gpu_with_warmup(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.workload == "cloth" and a.n == 512
    assert a.warmup >= 3 and 1 <= a.steps <= 100


def test_stage_work_per_unit():
    nV, nE, nF = 262144, 784385, 522242          # the 512 x 512 cloth
    st = {"n_vf": 1000, "n_ee": 3000, "n_box_copies": 2_000_000, "n_superset": 6000,
          "n_intervals": 50_000, "n_exported": 200}
    w = bench.stage_algorithmic(st, nV, nE, nF)
    nB = nV + nE + nF
    assert nB == 1_568_771
    assert w["boxes"] == ("hbm", 48 * nV + 8 * nE + 12 * nF + 88 * nB)
    # a counting read of the keys (8 B) and 7 radix passes over the copies (24 B each:
    # 8 B key and 4 B value, read and written)
    assert w["sort"] == ("hbm", 8 * nB + (12 + 8 + 7 * 24 + 84) * 2_000_000)
    assert w["sweep"] == ("hbm", 44 * 2_000_000 + 112 * 6000 + 8 * 4000)
    # per interval 42 DFMA (2 flops) + 3 DADD; per unit 45 FP64 operations
    assert bench.FLOPS_PER_INTERVAL == 87 and bench.FLOPS_PER_UNIT == 45
    assert w["narrow"] == ("alu", 87 * 50_000 + 45 * (4000 + 200))
    # copies default to one per box when the sweep did not report them
    st.pop("n_box_copies")
    assert bench.stage_algorithmic(st, nV, nE, nF)["sort"][1] == 8 * nB + (12 + 8 + 168 + 84) * nB


def test_source_hash_is_short_hex():
    h = bench.src_hash("ccd_narrow.cu")
    assert len(h) == 16 and int(h, 16) >= 0
