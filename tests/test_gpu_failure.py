"""Failure detection of the narrow phase, exercised without a GPU fault.

Every wait in the narrow kernel is bounded and its warps leave after a fixed
number of idle rounds, so work that can never finish must end the launch with
CCD_ETIMEOUT rather than hold the GPU.  The self-test entry point plants the
failure on the device side in the plainest way: one unit counted as pending
that no lane will ever take (a count that nothing brings back to zero).  The
test checks the status, that the launch ended within its idle limit, and that
the same context then runs a normal step with the oracle's result."""
import time

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


def test_unfinished_work_is_reported_and_the_context_recovers(ccd):
    c = ccd.CCD(0)
    try:
        t0 = time.time()
        st = ccd.ccd_selftest_unfinished_work(c.ctx)
        took = time.time() - t0
        assert st == ccd.CCD_ETIMEOUT
        assert took < 20.0
        rc, _ = c.status()
        assert rc == ccd.CCD_ETIMEOUT
        # a normal call on the same context: status reset, result unchanged
        s = scenes.icosphere_on_plane(0)
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        assert c.step(V0, V1, E, F) == O.step(s.V0, s.V1, s.E, s.F)
        rc, _ = c.status()
        assert rc == ccd.CCD_OK
    finally:
        c.close()


def test_finished_launches_raise_no_timeout(ccd):
    """The check at the end of the launch must not fire on a launch that
    finished its work, including one whose queries were all handed around
    (export budget 1, a small ring)."""
    c = ccd.CCD(0, export_budget=1, queue_capacity=64)
    try:
        s = scenes.folded_cloth(40, seed=1)
        V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F)
        for _ in range(3):
            c.step(V0, V1, E, F)
            rc, _ = c.status()
            assert rc == ccd.CCD_OK
    finally:
        c.close()
