"""Failure detection without a GPU fault: the grid-wide stage barrier waits
with a time limit and, when it runs out, raises a status bit that the host
turns into HEOM_ETIMEOUT.  Here that bounded wait is made to run out on
purpose (it waits for a counter that nothing raises, with a 20 ms limit);
the kernel returns, and the device keeps working."""
import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    timed_out, ms = heom.selftest_bounded_wait(20.0)
    assert timed_out
    assert 19.0 <= ms < 500.0, ms
    # the same process and device propagate correctly afterwards
    w = workloads.fmo_trap(K=2, nsteps=100)
    o = oracle.propagate(w["params"], w["rho0"], 1.0, 100, 10)
    with heom.Context(w["params"], "fp64") as c:
        c.set_launch(mode=1)  # the grid launch, whose stage barrier is this wait
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 100, 10)
    assert np.abs(r["pops"] - o["pops"]).max() < 1e-10


def test_bounded_wait_rejects_bad_limits():
    for bad in (0.0, -1.0, 2000.0):
        with pytest.raises(heom.HeomError) as e:
            heom.selftest_bounded_wait(bad)
        assert e.value.code == heom.EINVAL
