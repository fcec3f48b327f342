"""The dataflow engine (launch mode 3: one hierarchy on the whole GPU, no
grid barrier, neighbour values exchanged as stage-tagged words) against the
FP64 oracle.

Tolerances as everywhere: FP64 1e-10 max-abs on populations, eta and every
node of the state; mixed precision 1e-5 on populations, 1e-4 on eta.
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


def units(N):
    return N * (N + 1) // 2


def run(w, precision, nodes_per_cta, nsteps=None, out_every=None, stop=0.0):
    nsteps = w["nsteps"] if nsteps is None else nsteps
    out_every = w["out_every"] if out_every is None else out_every
    N = w["params"]["N"]
    with heom.Context(w["params"], precision) as c:
        c.set_launch(mode=3, block_threads=nodes_per_cta * units(N))
        if stop:
            c.set_stop(stop)
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], nsteps, out_every)
        r["eta_end"], r["loss_end"] = c.efficiency()
        r["tmean"], r["done"] = c.trapping_time()
        r["state"], r["extra"] = c.state()
        r["rho"] = c.rho()
        assert c.get_launch()["mode"] == 3
    return r


def compare_states(gpu_state, ref, N, K, tol):
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(ref["multi"].tolist())}
    perm = np.array([pos[tuple(m)] for m in multi.tolist()])
    err = np.abs(gpu_state - ref["state"][perm][:, :N, :N]).max()
    assert err < tol, err


CASES = [(N, K, cplx, term) for N, K in [(1, 0), (1, 4), (2, 5), (3, 3), (4, 3), (5, 3), (6, 2), (7, 3), (8, 2)]
         for cplx, term in [(False, 0), (True, 1)]]


@pytest.mark.parametrize("N,K,cplx,term", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_random_instances(N, K, cplx, term, precision):
    w = workloads.random_instance(N, K, seed=900 + 10 * N + K, complex_h=cplx, terminator=term)
    g = run(w, precision, 4)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], want_state=True)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    assert abs(g["eta_end"] - o["eta"][-1]) < te
    compare_states(g["state"], o, N, K, TOL64 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("S", [1, 3, 12, 13])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_fmo_depth6_cta_sizes(S, precision):
    """The headline hierarchy (N = 7, depth 6, 1716 nodes) with several nodes
    per CTA that let every CTA be resident at once, a ragged last CTA included
    (1716 is no multiple of 12 or 13)."""
    w = workloads.fmo_trap(nsteps=200)
    g = run(w, precision, S)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], 200, w["out_every"], want_state=True)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    assert abs(g["loss_end"] - o["loss"][-1]) < te
    compare_states(g["state"], o, 7, 6, TOL64 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_scaled_and_low_temperature(precision):
    w = workloads.random_instance(6, 3, seed=41, complex_h=True, terminator=1)
    w["params"]["scaled"] = 1
    w["params"]["low_temp"] = 1
    w["params"]["T"] = 120.0
    g = run(w, precision, 6)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], want_state=True)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    compare_states(g["state"], o, 6, 3, TOL64 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_stop_rule_and_trapping_time(precision):
    """A site that decays within the run: the stop rule ends the call after
    the same step as the oracle, later rows are NaN, <t> matches."""
    w = workloads.fmo_trap(K=3, nsteps=3000)
    p = dict(w["params"])
    p["trap"] = np.full(7, 5.0)
    w = dict(w, params=p)
    g = run(w, precision, 8, nsteps=3000, out_every=10, stop=1e-3)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], 3000, 1, stop_trace=1e-3)  # every step
    n = o["steps_done"]
    assert g["done"] == n < 3000
    rows = n // 10 + 1
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"][:rows] - o["pops"][:n + 1:10]).max() < tp
    assert np.all(np.isnan(g["pops"][rows:]))
    # <t> at the stop step n (the oracle's row n), within 2 t max|d eta|
    assert abs(g["tmean"] - o["tmean"][n]) < 2.0 * w["dt"] * n * te


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_resume_and_mode_switch(precision):
    """Calls continue one another bit for bit (tags advance per call), and a
    context may switch between the grid engine and the dataflow engine."""
    w = workloads.fmo_trap(K=4, nsteps=120)
    with heom.Context(w["params"], precision) as c:
        c.set_launch(mode=3, block_threads=8 * 28)
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 120, 120)
        one = c.state()[0]
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 50, 50)
        c.propagate(1.0, 70, 70)
        two = c.state()[0]
        assert np.array_equal(one, two)
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 40, 40)
        c.set_launch(mode=1, block_threads=256, node_threads=32)
        c.propagate(1.0, 40, 40)
        c.set_launch(mode=3, block_threads=8 * 28)
        r = c.propagate(1.0, 40, 10)
    o = oracle.propagate(w["params"], w["rho0"], 1.0, 120, 10)
    tol = TOL64 if precision == "fp64" else TOL32_POP
    assert np.abs(r["pops"] - o["pops"][8:]).max() < tol


def test_flow_rejects_oversized_ctas_and_hierarchies_that_cannot_be_resident():
    w = workloads.fmo_trap(nsteps=10)
    with heom.Context(w["params"], "fp32") as c:
        with pytest.raises(heom.HeomError) as e:
            c.set_launch(mode=3, block_threads=16 * 28)  # beyond the 384 threads the kernels are built for
        assert e.value.code == heom.EINVAL
    w = workloads.fmo_trap(K=8, nsteps=10)  # 6435 nodes: more CTAs than can be resident at once
    with heom.Context(w["params"], "fp32") as c:
        c.set_launch(mode=3, team_ctas=1, block_threads=13 * 28)  # one node per thread
        with pytest.raises(heom.HeomError) as e:
            c.propagate(1.0, 10, 10)
        assert e.value.code == heom.EINVAL and "resident" in str(e.value)
        c.set_launch(mode=1, block_threads=512, node_threads=32)  # the context stays usable
        c.propagate(1.0, 10, 10)


def test_flow_rejects_batches_and_large_hierarchies():
    ws = [workloads.random_instance(3, 2, seed=1), workloads.random_instance(3, 2, seed=2)]
    with heom.Batch([w["params"] for w in ws], "fp32") as b:
        with pytest.raises(heom.HeomError) as e:
            b.set_launch(mode=3)
        assert e.value.code == heom.EINVAL
    w = workloads.random_instance(10, 1, seed=3)
    with heom.Context(w["params"], "fp32") as c:
        with pytest.raises(heom.HeomError) as e:
            c.set_launch(mode=3, block_threads=55)
        assert e.value.code == heom.EINVAL


# ---------------------------------------------------------------- several nodes per thread

def run_npt(w, precision, npt, rows_per_cta, nsteps=None, out_every=None, stop=0.0):
    """Mode 3 with `npt` nodes per thread and `rows_per_cta` unit rows per CTA
    (a CTA's slice holds rows_per_cta * npt nodes)."""
    nsteps = w["nsteps"] if nsteps is None else nsteps
    out_every = w["out_every"] if out_every is None else out_every
    N = w["params"]["N"]
    with heom.Context(w["params"], precision) as c:
        c.set_launch(mode=3, team_ctas=npt, block_threads=rows_per_cta * units(N))
        if stop:
            c.set_stop(stop)
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], nsteps, out_every)
        r["eta_end"], r["loss_end"] = c.efficiency()
        r["tmean"], r["done"] = c.trapping_time()
        r["state"], r["extra"] = c.state()
        L = c.get_launch()
        assert L["mode"] == 3 and L["team_ctas"] == npt
    return r


NPT_CASES = [(4, 5, 0, 2, 4), (5, 4, 1, 3, 5), (6, 3, 0, 4, 5), (7, 3, 1, 5, 7), (8, 2, 0, 6, 3), (7, 4, 0, 6, 9),
             (8, 3, 1, 4, 7)]


@pytest.mark.parametrize("N,K,term,npt,rows", NPT_CASES)
def test_flow_nodes_per_thread_mixed(N, K, term, npt, rows):
    """2..6 nodes per thread, small and large unit rows, ragged last slices
    (the node counts are no multiple of rows * npt), every node of the state."""
    w = workloads.random_instance(N, K, seed=1300 + 10 * N + K, terminator=term)
    g = run_npt(w, "fp32", npt, rows)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], want_state=True)
    assert np.abs(g["pops"] - o["pops"]).max() < TOL32_POP
    assert np.abs(g["eta"] - o["eta"]).max() < TOL32_ETA
    assert abs(g["eta_end"] - o["eta"][-1]) < TOL32_ETA
    compare_states(g["state"], o, N, K, 1e-5)


@pytest.mark.parametrize("N,K,rows", [(4, 5, 5), (7, 4, 7), (8, 3, 5)])
def test_flow_two_nodes_per_thread_fp64(N, K, rows):
    w = workloads.random_instance(N, K, seed=1400 + 10 * N + K, terminator=1)
    g = run_npt(w, "fp64", 2, rows)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], want_state=True)
    assert np.abs(g["pops"] - o["pops"]).max() < TOL64
    assert np.abs(g["eta"] - o["eta"]).max() < TOL64
    compare_states(g["state"], o, N, K, TOL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flow_nodes_per_thread_scaled_stop_and_resume(precision):
    """The scaled hierarchy with the low-temperature correction, the stop rule
    and a call split in two, with several nodes per thread."""
    npt = 2 if precision == "fp64" else 3
    w = workloads.fmo_trap(K=4, nsteps=3000)
    p = dict(w["params"], scaled=1, low_temp=1)
    p["trap"] = np.full(7, 5.0)
    w = dict(w, params=p)
    g = run_npt(w, precision, npt, 4, nsteps=3000, out_every=10, stop=1e-3)
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], 3000, 1, stop_trace=1e-3)
    n = o["steps_done"]
    assert g["done"] == n < 3000
    rows = n // 10 + 1
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"][:rows] - o["pops"][:n + 1:10]).max() < tp
    assert abs(g["eta_end"] - o["eta"][n]) < te
    q = workloads.fmo_trap(K=5, nsteps=120)
    with heom.Context(q["params"], precision) as c:
        c.set_launch(mode=3, team_ctas=npt, block_threads=6 * 28)
        c.set_rho0(q["rho0"])
        c.propagate(1.0, 120, 120)
        one = c.state()[0]
        c.set_rho0(q["rho0"])
        c.propagate(1.0, 50, 50)
        c.propagate(1.0, 70, 70)
        assert np.array_equal(one, c.state()[0])


@pytest.mark.parametrize("K,npt", [(7, 3), (8, 5)])
def test_flow_default_takes_several_nodes_per_thread(K, npt):
    """Depth 7 (3432 nodes) and depth 8 (6435 nodes) of the FMO-like model do
    not fit with one node per thread; the default then carries several, and
    the result matches the oracle node by node."""
    w = workloads.fmo_trap(K=K, nsteps=30)
    with heom.Context(w["params"], "fp32") as c:
        L = c.get_launch()
        assert L["mode"] == 3 and L["team_ctas"] == npt, L
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 30, 10)
        state, _ = c.state()
    o = oracle.propagate(w["params"], w["rho0"], 1.0, 30, 10, want_state=True)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL32_POP
    assert np.abs(r["eta"] - o["eta"]).max() < TOL32_ETA
    compare_states(state, o, 7, K, 1e-5)


def test_flow_several_nodes_per_thread_refused_where_not_built():
    w = workloads.random_instance(5, 3, seed=77, complex_h=True)
    with heom.Context(w["params"], "fp32") as c:
        c.set_launch(mode=3, team_ctas=2, block_threads=4 * units(5))
        c.set_rho0(w["rho0"])
        with pytest.raises(heom.HeomError) as e:
            c.propagate(1.0, 5, 5)
        assert e.value.code == heom.EUNSUPPORTED
        c.set_launch(mode=3, team_ctas=1)  # one node per thread runs complex H
        c.propagate(1.0, 5, 5)
    w = workloads.random_instance(7, 3, seed=78)
    with heom.Context(w["params"], "fp32") as c:
        with pytest.raises(heom.HeomError) as e:
            c.set_launch(mode=3, team_ctas=7, block_threads=4 * 28)  # beyond 6 nodes per thread
        assert e.value.code == heom.EINVAL
        with pytest.raises(heom.HeomError) as e:
            c.set_launch(mode=3, team_ctas=2, block_threads=10 * 28)  # beyond 256 threads
        assert e.value.code == heom.EINVAL
