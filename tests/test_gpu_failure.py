"""Failure detection without a GPU fault.

* The grid-wide stage barrier waits with a time limit and, when it runs out,
  raises a status bit that the host turns into HEOM_ETIMEOUT.  Here that
  bounded wait is made to run out on purpose (it waits for a counter that
  nothing raises, with a 20 ms limit); the kernel returns, and the device
  keeps working.
* Results that come out NaN or infinite (a diverging run, or a non-finite
  initial state handed over through the unvalidated device path) raise
  another status bit: the call returns HEOM_ENONFINITE instead of HEOM_OK.
  The failures are made on the host: a NaN planted in rho(0), or a time step
  beyond the stability limit of RK4 (ordinary floating-point overflow).
"""
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


NONFINITE_SHAPES = [("fp64", None), ("fp32", None), ("fp32", dict(mode=0, team_ctas=2, block_threads=256,
                                                                   node_threads=8)),
                    ("fp32", dict(mode=2, team_ctas=4, block_threads=256, node_threads=4)),
                    ("fp64", dict(mode=1, team_ctas=1, block_threads=256, node_threads=8))]


@pytest.mark.parametrize("precision,shape", NONFINITE_SHAPES,
                         ids=lambda v: v if isinstance(v, str) else ("default" if v is None else "m%d" % v["mode"]))
def test_non_finite_initial_state_is_reported(precision, shape):
    """A NaN planted in rho(0) on the host and handed over through the device
    path (which does not validate) makes every later row non-finite; the call
    returns HEOM_ENONFINITE instead of HEOM_OK, with and without output rows,
    and the context works again after a valid rho(0)."""
    import torch
    w = workloads.fmo_trap(K=3, nsteps=40)
    bad = np.array(w["rho0"], dtype=np.complex128)
    bad[0, 0] = np.nan
    d_bad = torch.from_numpy(bad).cuda()
    o = oracle.propagate(w["params"], w["rho0"], 1.0, 40, 10)
    with heom.Context(w["params"], precision) as c:
        if shape:
            c.set_launch(**shape)
        for rows in (True, False):
            c.set_rho0_device(d_bad)
            with pytest.raises(heom.HeomError) as e:
                if rows:
                    c.propagate(1.0, 40, 10)
                else:
                    c.propagate_device(1.0, 40, 40)
                    c.synchronize()
            assert e.value.code == heom.ENONFINITE, str(e.value)
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 40, 10)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert np.abs(r["pops"] - o["pops"]).max() < tol


def test_diverging_instance_in_a_batch_is_reported():
    """A time step far beyond the stability limit of RK4 for these baths
    (200 fs) makes one instance of a batch grow until it overflows: the
    batch call returns HEOM_ENONFINITE; the same batch at 1 fs is fine."""
    ws = [workloads.random_instance(N, 2, seed=70 + N, trap=True) for N in (3, 5)]
    with heom.Batch([w["params"] for w in ws], "fp32") as b:
        b.set_rho0([w["rho0"] for w in ws])
        with pytest.raises(heom.HeomError) as e:
            b.propagate([1.0, 200.0], 400, 50)
        assert e.value.code == heom.ENONFINITE
        b.set_rho0([w["rho0"] for w in ws])
        res = b.propagate(1.0, 100, 50)
    for w, r in zip(ws, res):
        o = oracle.propagate(w["params"], w["rho0"], 1.0, 100, 50)
        assert np.abs(r["pops"] - o["pops"]).max() < 1e-5


def test_diverging_request_fails_in_the_server():
    """The server marks a request whose rows came out non-finite as failed
    (HEOM_ENONFINITE from its result) and serves the others normally."""
    import time
    from paper_1012_4382_gb300 import serving
    w = workloads.random_instance(4, 2, seed=9, trap=True)
    with serving.Server(1 << 30, 16 << 20, 4) as srv:
        bad = srv.submit(w["params"], w["rho0"], 200.0, 400, 50)
        good = srv.submit(w["params"], w["rho0"], 1.0, 100, 50)
        t0 = time.time()
        while {srv.status(bad), srv.status(good)} & {serving.QUEUED, serving.RUNNING}:
            srv.progress()
            assert time.time() - t0 < 60.0
            time.sleep(1e-3)
        assert srv.status(bad) == serving.FAILED
        with pytest.raises(heom.HeomError) as e:
            srv.result(bad)
        assert e.value.code == heom.ENONFINITE
        assert srv.status(good) == serving.DONE
        r = srv.result(good)
    o = oracle.propagate(w["params"], w["rho0"], 1.0, 100, 50)
    assert np.abs(r["pops"] - o["pops"]).max() < 1e-5
