"""Parity with the FP64 oracle over the whole horizon of every workload the
benchmark times, in the launch shapes it times (default shapes).

* FMO-like trap model, N = 7, depth 6 (1716 nodes), 10 000 steps of 1 fs:
  FP64 within 1e-10 and mixed precision within 1e-5 (populations) / 1e-4
  (eta), every 10 fs row; the trapping time <t> at 10 ps within the bound the
  eta tolerance implies (|d<t>| <= 2 t max|d eta|); the final rho.
* Batched scan: the full 256-instance launch over its 5000 steps, one
  instance of every depth 4..8 against the oracle on every 10 fs row.
* 24-site trimer (20 475 nodes): 50 steps of the full hierarchy in both
  precisions, FP64 node by node.
* The depth sweep of the paper's timing table: its largest hierarchy (N = 7,
  depth 12, 50 388 nodes), 20 steps, every node, in the default and the
  autotuned launch shape.

Paper: App. B (RK4 over the whole run; only rho and eta copied out), Eq. eta
and Eq. trappingtime.  The oracle runs once per workload on the host cores.
"""
import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32_POP = 1e-5
TOL32_ETA = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


@pytest.fixture(scope="module")
def fmo_full():
    w = workloads.fmo_trap()
    assert w["nsteps"] == 10000 and w["out_every"] == 10
    return w, oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fmo_trap_full_10ps_matches_oracle(fmo_full, precision):
    w, o = fmo_full
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    with heom.Context(w["params"], precision) as c:
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], w["nsteps"], w["out_every"])
        eta_end, loss_end = c.efficiency()
        tmean, done = c.trapping_time()
        rho = c.rho()
    assert done == w["nsteps"]
    assert r["pops"].shape == o["pops"].shape == (1001, 7)
    assert np.abs(r["pops"] - o["pops"]).max() < tp
    assert np.abs(r["trace"] - o["trace"]).max() < tp * 7
    assert np.abs(r["eta"] - o["eta"]).max() < te
    assert abs(eta_end - o["eta"][-1]) < te
    assert abs(loss_end - o["loss"][-1]) < te
    assert np.abs(rho - o["rho"][:7, :7]).max() < tp
    t_end = w["dt"] * w["nsteps"]
    assert abs(tmean - o["tmean"][-1]) < 2.0 * t_end * te
    assert o["eta"][-1] > 0.1  # the trap has taken a visible share by 10 ps


def test_batched_scan_full_5000_steps_matches_oracle():
    ws = workloads.batched_scan()
    nsteps = ws[0]["nsteps"]
    assert nsteps == 5000 and len(ws) == 256
    with heom.Batch([w["params"] for w in ws], "fp32") as b:
        b.set_rho0([w["rho0"] for w in ws])
        res = b.propagate(1.0, nsteps, 10)
        eta_end, _ = b.efficiency()
    seen = {}
    for i, w in enumerate(ws):
        seen.setdefault(w["params"]["K"], i)
    assert sorted(seen) == [4, 5, 6, 7, 8]
    for K, i in sorted(seen.items()):
        o = oracle.propagate(ws[i]["params"], ws[i]["rho0"], 1.0, nsteps, 10)
        assert res[i]["pops"].shape == o["pops"].shape == (501, 7)
        assert np.abs(res[i]["pops"] - o["pops"]).max() < TOL32_POP, K
        assert np.abs(res[i]["eta"] - o["eta"]).max() < TOL32_ETA, K
        assert abs(eta_end[i] - o["eta"][-1]) < TOL32_ETA, K


@pytest.fixture(scope="module")
def trimer_50():
    w = workloads.large_trimer(nsteps=50)
    w["out_every"] = 5
    return w, oracle.propagate(w["params"], w["rho0"], w["dt"], 50, 5, want_state=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_large_trimer_50_steps_full_hierarchy(trimer_50, precision):
    w, o = trimer_50
    N, K = 24, 4
    with heom.Context(w["params"], precision) as c:
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], 50, 5)
        state, _ = c.state()
    tp = TOL64 if precision == "fp64" else TOL32_POP
    assert np.abs(r["pops"] - o["pops"]).max() < tp
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(o["multi"].tolist())}
    perm = np.array([pos[tuple(m)] for m in multi.tolist()])
    ref = o["state"][perm][:, :N, :N]
    err = np.abs(state - ref).max()
    if precision == "fp64":
        assert err < TOL64, err
    else:
        # float auxiliaries: relative to the largest auxiliary element
        assert err < 1e-5 * max(1.0, np.abs(ref).max()), (err, np.abs(ref).max())


@pytest.fixture(scope="module")
def depth12_20():
    w = workloads.fmo_trap(K=12, nsteps=20)
    return w, oracle.propagate(w["params"], w["rho0"], 1.0, 20, 5, want_state=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["default", "tuned"])
def test_table2_depth12_every_node(depth12_20, precision, shape):
    """The largest hierarchy of the paper's timing table (N = 7, N_max = 12,
    50 388 matrices), in the launch shape the benchmark's depth sweep times:
    the default one and the one the autotuner picks.  20 steps, every node of
    the state against the oracle (FP64 1e-10; mixed 1e-5 of the largest
    element), populations and eta on every row."""
    w, o = depth12_20
    N, K = 7, 12
    with heom.Context(w["params"], precision) as c:
        if shape == "tuned":
            c.autotune(trial_steps=5)
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 20, 5)
        state, _ = c.state()
    assert state.shape[0] == 50388
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(r["pops"] - o["pops"]).max() < tp
    assert np.abs(r["eta"] - o["eta"]).max() < te
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(o["multi"].tolist())}
    perm = np.array([pos[tuple(m)] for m in multi.tolist()])
    ref = o["state"][perm][:, :N, :N]
    err = np.abs(state - ref).max()
    if precision == "fp64":
        assert err < TOL64, err
    else:
        assert err < 1e-5 * max(1.0, np.abs(ref).max()), (err, np.abs(ref).max())
