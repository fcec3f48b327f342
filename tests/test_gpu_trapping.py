"""Trapping time <t> (Eq. trappingtime) and the t_max stop rule of the
section on trapping times, CUDA path against the oracle.

<t> = t eta(t) - int_0^t eta dt', so its error is bounded by t_end times the
eta tolerance, twice: 2 tol_eta t_end.  The stop step is an integer and must
match exactly; the cases decay by about 2 % per step near the threshold, far
from any rounding tie.
"""
import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-10), "fp32": (1e-5, 1e-4)}  # (populations, eta)


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def fast_decay(w, rate=20.0):
    """The same hierarchy with a strong trap on every site (ps^-1)."""
    p = dict(w["params"])
    N = p["N"]
    p["trap"] = np.full(N, rate)
    p["recomb"] = np.full(N, 1.0)
    return dict(w, params=p)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_trapping_time_matches_oracle_across_calls(precision):
    w = workloads.fmo_trap(K=3)
    n1, n2 = 600, 900
    o = oracle.propagate(w["params"], w["rho0"], 1.0, n1 + n2, n1 + n2)
    with heom.Context(w["params"], precision) as c:
        c.set_rho0(w["rho0"])
        c.propagate(1.0, n1, 10)
        c.propagate(1.0, n2, 10)
        t, n = c.trapping_time()
    assert n == n2
    tol = 2 * TOL[precision][1] * (n1 + n2)
    assert abs(t - o["tmean"][-1]) < tol, (t, o["tmean"][-1])
    assert o["tmean"][-1] > 1.0  # a non-trivial value


STOP_CASES = [
    ("fp64", None), ("fp32", None),
    ("fp64", dict(mode=0, team_ctas=2, block_threads=256, node_threads=2)),
    ("fp64", dict(mode=1, team_ctas=1, block_threads=256, node_threads=8)),
    ("fp32", dict(mode=0, team_ctas=1, block_threads=512, node_threads=1)),
    ("fp32", dict(mode=1, team_ctas=1, block_threads=256, node_threads=32)),
    ("fp32", dict(mode=2, team_ctas=2, block_threads=256, node_threads=4)),
]


@pytest.mark.parametrize("precision,shape", STOP_CASES,
                         ids=lambda v: v if isinstance(v, str) else ("default" if v is None else
                                                                     "m%d_c%d_b%d_g%d" % tuple(v.values())))
def test_stop_rule_matches_oracle(precision, shape):
    w = fast_decay(workloads.fmo_trap(K=3))
    nsteps, every = 3000, 10
    o = oracle.propagate(w["params"], w["rho0"], 1.0, nsteps, 1, stop_trace=1e-5)
    n_stop = o["steps_done"]
    assert 0 < n_stop < nsteps
    with heom.Context(w["params"], precision) as c:
        if shape:
            c.set_launch(**shape)
        c.set_stop(1e-5)
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, nsteps, every)
        t, n = c.trapping_time()
    assert n == n_stop
    rows = n_stop // every + 1
    tp, te = TOL[precision]
    assert np.abs(r["pops"][:rows] - o["pops"][: n_stop + 1: every]).max() < tp
    assert np.abs(r["eta"][:rows] - o["eta"][: n_stop + 1: every]).max() < te
    assert np.isnan(r["pops"][rows:]).all() and np.isnan(r["eta"][rows:]).all()
    assert abs(t - o["tmean"][n_stop]) < 2 * te * n_stop


def test_stop_rule_large_hierarchy():
    """N = 10 sites runs on the large-N engine."""
    w = fast_decay(workloads.random_instance(10, 2, seed=77))
    nsteps = 2000
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], nsteps, 1, stop_trace=1e-5)
    for precision in ("fp64", "fp32"):
        with heom.Context(w["params"], precision) as c:
            c.set_stop(1e-5)
            c.set_rho0(w["rho0"])
            r = c.propagate(w["dt"], nsteps, 5)
            t, n = c.trapping_time()
        assert n == o["steps_done"] < nsteps
        rows = n // 5 + 1
        assert np.abs(r["pops"][:rows] - o["pops"][: n + 1: 5]).max() < TOL[precision][0]
        assert abs(t - o["tmean"][n]) < 2 * TOL[precision][1] * n * w["dt"]


def test_batch_trapping_times_and_stop():
    ws = [fast_decay(workloads.fmo_trap(K=K, seed=1234 + K)) for K in (1, 2, 3)]
    ws.append(workloads.fmo_trap(K=2, seed=99))  # slow: runs to the end
    nsteps = 2500
    with heom.Batch([w["params"] for w in ws], "fp32") as b:
        b.set_stop(1e-5)
        b.set_rho0([w["rho0"] for w in ws])
        b.propagate([1.0] * len(ws), [nsteps] * len(ws), 10)
        t, n = b.trapping_time()
    for i, w in enumerate(ws):
        o = oracle.propagate(w["params"], w["rho0"], 1.0, nsteps, 1, stop_trace=1e-5)
        assert n[i] == o["steps_done"]
        assert abs(t[i] - o["tmean"][n[i]]) < 2 * TOL["fp32"][1] * n[i]
    assert n[-1] == nsteps and n[0] < nsteps


def test_stop_value_checked():
    w = workloads.fmo_trap(K=1)
    with heom.Context(w["params"], "fp64") as c:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(heom.HeomError) as e:
                c.set_stop(bad)
            assert e.value.code == heom.EINVAL
