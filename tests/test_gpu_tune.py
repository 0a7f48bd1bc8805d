"""Autotuner: the settings it keeps are valid, the interval queue shrinks to
the 16x-headroom power of two (or stays), and every call after tuning still
gives the oracle's earliest time, with and without a captured graph."""
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


@pytest.mark.parametrize("use_graph", [0, 1])
def test_autotune_then_step_matches_oracle(ccd, use_graph):
    s = scenes.folded_cloth(64, seed=2)
    ref = O.step(s.V0, s.V1, s.E, s.F)
    c = ccd.CCD(0, use_graph=use_graph)
    try:
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)      # captured before tuning
        t = c.autotune(V0, V1, E, F, reps=2)
        assert t["sweep_kernel"] in (0, 2)
        assert t["export_budget"] in (8, 16, 32, 64)
        assert t["sweep_kernel"] == 2 or t["strip_width"] in (1.5, 2.0, 3.0, 4.0, 6.0)
        q = t["queue_capacity"]
        assert q >= 1024 and q & (q - 1) == 0 and q <= 1 << 21
        assert t["n_trials"] >= 14 and t["broad_ms"] > 0 and t["narrow_ms"] > 0
        for _ in range(2):
            ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
            torch.cuda.synchronize()
            assert float(out.item()) == ref
        assert c.step(V0, V1, E, F) == ref
        assert c.status()[0] == 0
    finally:
        c.close()
