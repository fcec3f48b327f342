"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances: FP64 path 1e-10 max-abs on populations and eta; FP32-mixed path
1e-5 on populations and 1e-4 on eta.  Inputs are the seeded synthetic
workloads; the oracle runs on the host cores.
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


def run_gpu(w, precision="fp64", launch=None, nsteps=None, out_every=None):
    nsteps = w["nsteps"] if nsteps is None else nsteps
    out_every = w["out_every"] if out_every is None else out_every
    with heom.Context(w["params"], precision) as c:
        if launch:
            c.set_launch(**launch)
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], nsteps, out_every)
        r["eta_end"], r["loss_end"] = c.efficiency()
        r["rho"] = c.rho()
        r["state"], r["extra"] = c.state()
    return r


def run_oracle(w, nsteps=None, out_every=None, want_state=False):
    nsteps = w["nsteps"] if nsteps is None else nsteps
    out_every = w["out_every"] if out_every is None else out_every
    return oracle.propagate(w["params"], w["rho0"], w["dt"], nsteps, out_every, want_state=want_state)


def compare_states(gpu_state, ref, N, K, tol):
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(ref["multi"].tolist())}
    perm = np.array([pos[tuple(m)] for m in multi.tolist()])
    ref_sites = ref["state"][perm][:, :N, :N]
    err = np.abs(gpu_state - ref_sites).max()
    assert err < tol, err


def test_dimer_fp64_matches_oracle():
    w = workloads.dimer()
    g = run_gpu(w)
    o = run_oracle(w, want_state=True)
    assert np.abs(g["pops"] - o["pops"]).max() < TOL64
    assert np.abs(g["trace"] - o["trace"]).max() < TOL64
    assert np.all(g["eta"] == 0.0)
    compare_states(g["state"], o, 2, 4, TOL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fmo_trap_matches_oracle(precision):
    w = workloads.fmo_trap(nsteps=400)
    g = run_gpu(w, precision)
    o = run_oracle(w, want_state=True)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    assert abs(g["eta_end"] - o["eta"][-1]) < te
    assert abs(g["loss_end"] - o["loss"][-1]) < te
    assert np.abs(g["rho"] - o["rho"][:7, :7]).max() < tp
    compare_states(g["state"], o, 7, 6, TOL64 if precision == "fp64" else 1e-5)


CASES = [(N, K, cplx, term) for N, K in [(1, 0), (1, 3), (2, 0), (2, 5), (3, 3), (4, 3), (5, 2), (6, 2), (7, 3),
                                         (8, 2)]
         for cplx, term in [(False, 0), (True, 1)]]


@pytest.mark.parametrize("N,K,cplx,term", CASES)
def test_random_instances_fp64(N, K, cplx, term):
    w = workloads.random_instance(N, K, seed=100 * N + K, complex_h=cplx, terminator=term)
    g = run_gpu(w)
    o = run_oracle(w, want_state=True)
    assert np.abs(g["pops"] - o["pops"]).max() < TOL64
    assert np.abs(g["eta"] - o["eta"]).max() < TOL64
    compare_states(g["state"], o, N, K, TOL64)


@pytest.mark.parametrize("N,K,cplx,term", CASES)
def test_random_instances_fp32(N, K, cplx, term):
    w = workloads.random_instance(N, K, seed=7 + N + K, complex_h=cplx, terminator=term)
    g = run_gpu(w, "fp32")
    o = run_oracle(w)
    assert np.abs(g["pops"] - o["pops"]).max() < TOL32_POP
    assert np.abs(g["eta"] - o["eta"]).max() < TOL32_ETA


LARGE = [(9, 2, False, 0), (10, 2, True, 1), (12, 2, False, 1), (16, 1, True, 0), (24, 2, False, 0),
         (24, 1, True, 1)]


@pytest.mark.parametrize("N,K,cplx,term", LARGE)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_large_site_counts(N, K, cplx, term, precision):
    w = workloads.random_instance(N, K, seed=300 + N + K, complex_h=cplx, terminator=term)
    w["nsteps"], w["out_every"] = 30, 10
    g = run_gpu(w, precision)
    o = run_oracle(w, want_state=precision == "fp64")
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    if precision == "fp64":
        compare_states(g["state"], o, N, K, TOL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_large_trimer_full_size_first_steps(precision):
    """The 24-site trimer at depth 4 (20 475 nodes), full hierarchy, first steps
    element by element against the oracle (which takes seconds per step here)."""
    w = workloads.large_trimer(nsteps=3)
    w["out_every"] = 1
    g = run_gpu(w, precision)
    o = run_oracle(w, want_state=precision == "fp64")
    tp = TOL64 if precision == "fp64" else TOL32_POP
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["trace"] - 1.0).max() < (1e-12 if precision == "fp64" else 1e-6)
    if precision == "fp64":
        compare_states(g["state"], o, 24, 4, TOL64)


SHAPES = ([dict(mode=0, team_ctas=c, block_threads=b, node_threads=G) for c in (1, 2, 4, 8, 16)
           for b in (128, 512) for G in (1, 2, 3, 8, 32)]
          + [dict(mode=1, team_ctas=1, block_threads=b, node_threads=G) for b in (128, 256) for G in (1, 8, 28)])


@pytest.fixture(scope="module")
def k4_reference():
    w = workloads.fmo_trap(K=4, nsteps=60)
    w["out_every"] = 6
    return w, run_oracle(w)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "m%d_c%d_b%d_g%d" % (s["mode"], s["team_ctas"],
                                                                          s["block_threads"], s["node_threads"]))
def test_launch_shapes_fp64(shape, k4_reference):
    w, o = k4_reference
    if shape["block_threads"] > 256:
        # the FP64 kernels are compiled for at most 256 threads per block: refused on the host
        with pytest.raises(heom.HeomError) as e:
            run_gpu(w, "fp64", launch=shape)
        assert e.value.code == heom.EINVAL and "block_threads" in str(e.value)
        return
    g = run_gpu(w, "fp64", launch=shape)
    assert np.abs(g["pops"] - o["pops"]).max() < TOL64
    assert np.abs(g["eta"] - o["eta"]).max() < TOL64


SHAPES32 = SHAPES[::3] + [dict(mode=2, team_ctas=c, block_threads=b, node_threads=G) for c in (1, 2, 4, 8, 16)
                          for b in (256, 512) for G in (1, 2, 5, 8, 32)]


@pytest.mark.parametrize("shape", SHAPES32, ids=lambda s: "m%d_c%d_b%d_g%d" % (
    s["mode"], s["team_ctas"], s["block_threads"], s["node_threads"]))
def test_launch_shapes_fp32(shape, k4_reference):
    w, o = k4_reference
    try:
        g = run_gpu(w, "fp32", launch=shape)
    except heom.HeomError as e:
        # the shared-memory mode refuses hierarchies that do not fit its CTAs
        assert shape["mode"] == 2 and e.code == heom.EINVAL and "shared memory" in str(e)
        return
    assert np.abs(g["pops"] - o["pops"]).max() < TOL32_POP
    assert np.abs(g["eta"] - o["eta"]).max() < TOL32_ETA


def test_resume_is_bitwise_identical():
    w = workloads.fmo_trap(K=4, nsteps=100)
    with heom.Context(w["params"], "fp64") as c:
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 100, 100)
        one = c.state()[0]
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 37, 37)
        c.propagate(1.0, 63, 63)
        two = c.state()[0]
    assert np.array_equal(one, two)


def test_state_roundtrip_and_hermiticity():
    w = workloads.random_instance(5, 3, seed=3, complex_h=True)
    with heom.Context(w["params"], "fp64") as c:
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 40, 40)
        st, extra = c.state()
        assert np.abs(st - np.conj(np.transpose(st, (0, 2, 1)))).max() == 0.0
        a = c.propagate(1.0, 30, 10)
        c.set_state(st, extra)
        b = c.propagate(1.0, 30, 10)
    assert np.array_equal(a["pops"], b["pops"])
    assert np.array_equal(a["eta"], b["eta"])


def test_probability_is_conserved_on_gpu():
    w = workloads.fmo_trap(K=4, nsteps=2000)
    with heom.Context(w["params"], "fp64") as c:
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 2000, 2000)
        eta, loss = c.efficiency()
        tr = np.trace(c.rho()).real
    assert eta > 0.05
    assert abs(tr + eta + loss - 1.0) < 1e-12


def test_batch_matches_oracle_and_single_contexts():
    ws = [workloads.random_instance(N, K, seed=50 + i, terminator=i % 2)
          for i, (N, K) in enumerate([(3, 3), (3, 2), (5, 2), (7, 3), (7, 2), (2, 4)])]
    steps = [50, 20, 33, 50, 0, 41]
    with heom.Batch([w["params"] for w in ws], "fp64") as b:
        b.set_rho0([w["rho0"] for w in ws])
        res = b.propagate(1.0, steps, 5)
        eta, loss = b.efficiency()
    for i, w in enumerate(ws):
        o = run_oracle(w, nsteps=steps[i], out_every=5)
        assert np.abs(res[i]["pops"] - o["pops"]).max() < TOL64
        assert np.abs(res[i]["eta"] - o["eta"]).max() < TOL64
        if steps[i] > 0:
            o_end = run_oracle(w, nsteps=steps[i], out_every=steps[i])
            assert abs(eta[i] - o_end["eta"][-1]) < TOL64
            assert abs(loss[i] - o_end["loss"][-1]) < TOL64
        else:
            assert eta[i] == 0.0 and loss[i] == 0.0


def test_batch_fp32_matches_oracle():
    ws = workloads.batched_scan(count=6, nsteps=200)
    for w in ws:
        w["params"]["K"] = min(w["params"]["K"], 5)
    with heom.Batch([w["params"] for w in ws], "fp32") as b:
        b.set_rho0([w["rho0"] for w in ws])
        res = b.propagate(1.0, 200, 10)
    for i, w in enumerate(ws):
        o = run_oracle(w, nsteps=200, out_every=10)
        assert np.abs(res[i]["pops"] - o["pops"]).max() < TOL32_POP
        assert np.abs(res[i]["eta"] - o["eta"]).max() < TOL32_ETA


def test_full_batched_scan_sampled_against_oracle():
    """The full 256-instance scan in the launch shape the benchmark times (the
    default), 20 steps; one sampled instance of every depth against the oracle."""
    ws = workloads.batched_scan(nsteps=20)
    with heom.Batch([w["params"] for w in ws], "fp32") as b:
        b.set_rho0([w["rho0"] for w in ws])
        res = b.propagate(1.0, 20, 10)
    seen = {}
    for i, w in enumerate(ws):
        seen.setdefault(w["params"]["K"], i)
    assert sorted(seen) == [4, 5, 6, 7, 8]
    for K, i in seen.items():
        o = run_oracle(ws[i], nsteps=20, out_every=10)
        assert np.abs(res[i]["pops"] - o["pops"]).max() < TOL32_POP, K
        assert np.abs(res[i]["eta"] - o["eta"]).max() < TOL32_ETA, K


def test_zero_steps_and_sparse_outputs():
    w = workloads.fmo_trap(K=3, nsteps=25)
    with heom.Context(w["params"], "fp64") as c:
        c.set_rho0(w["rho0"])
        r0 = c.propagate(1.0, 0, 1)
        assert r0["pops"].shape == (1, 7)
        assert r0["pops"][0, 0] == 1.0 and r0["eta"][0] == 0.0
        r = c.propagate(1.0, 25, 10)  # rows at steps 0, 10, 20
    o = run_oracle(w, nsteps=25, out_every=1)
    assert r["pops"].shape == (3, 7)
    assert np.abs(r["pops"] - o["pops"][[0, 10, 20]]).max() < TOL64


def test_set_rho0_from_device_buffer():
    import torch
    w = workloads.fmo_trap(K=3, nsteps=30)
    rho = np.zeros((7, 7), complex)
    rho[0, 0] = 0.5
    rho[1, 1] = 0.5
    rho[0, 1] = 0.3 - 0.2j
    rho[1, 0] = 0.3 + 0.2j
    w["rho0"] = rho
    d = torch.from_numpy(rho.copy()).cuda()
    with heom.Context(w["params"], "fp64") as c:
        c.set_rho0_device(d)
        torch.cuda.synchronize()
        r = c.propagate(1.0, 30, 10)
    o = run_oracle(w, nsteps=30, out_every=10)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL64


def test_torch_caching_allocator_hook():
    import torch
    heom.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        w = workloads.fmo_trap(K=4, nsteps=50)
        with heom.Context(w["params"], "fp32") as c:
            assert torch.cuda.memory_allocated() > before
            c.set_rho0(w["rho0"])
            r = c.propagate(1.0, 50, 10)
        o = run_oracle(w, nsteps=50, out_every=10)
        assert np.abs(r["pops"] - o["pops"]).max() < TOL32_POP
        assert torch.cuda.memory_allocated() == before
    finally:
        heom.use_torch_allocator(False)


def test_invalid_launch_shapes_rejected():
    w = workloads.dimer()
    with heom.Context(w["params"]) as c:
        for bad in [dict(mode=2), dict(team_ctas=17), dict(block_threads=48), dict(node_threads=33)]:
            with pytest.raises(heom.HeomError) as e:
                c.set_launch(**bad)
            assert e.value.code == heom.EINVAL


def test_shared_memory_mode_rejects_hierarchies_that_do_not_fit():
    w = workloads.fmo_trap(K=6, nsteps=10)
    with heom.Context(w["params"], "fp32") as c:
        c.set_launch(mode=2, team_ctas=1)
        with pytest.raises(heom.HeomError) as e:
            c.propagate(1.0, 10, 10)
        assert e.value.code == heom.EINVAL
        c.set_launch(mode=2, team_ctas=16)
        c.propagate(1.0, 10, 10)
    with heom.Context(w["params"], "fp64") as c:
        with pytest.raises(heom.HeomError) as e:
            c.set_launch(mode=2)
        assert e.value.code == heom.EINVAL


def test_autotune_keeps_state_and_result():
    w = workloads.fmo_trap(K=4, nsteps=40)
    w["out_every"] = 10
    o = run_oracle(w)
    with heom.Context(w["params"], "fp64") as c:
        c.set_rho0(w["rho0"])
        us = c.autotune(trial_steps=5)
        assert us > 0
        r = c.propagate(1.0, 40, 10)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL64


def test_autotune_over_nodes_per_thread_keeps_state_and_result():
    """Depth 7 (3432 nodes) in mixed precision: the autotuner's candidates
    include the dataflow engine with several nodes per thread; whichever it
    keeps, the state is restored and the run matches the oracle."""
    w = workloads.fmo_trap(K=7, nsteps=30)
    w["out_every"] = 10
    o = run_oracle(w)
    with heom.Context(w["params"], "fp32") as c:
        c.set_rho0(w["rho0"])
        assert c.autotune(trial_steps=5) > 0
        r = c.propagate(1.0, 30, 10)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL32_POP
    assert np.abs(r["eta"] - o["eta"]).max() < TOL32_ETA


@pytest.mark.parametrize("N,K", [(3, 3), (7, 2), (10, 2)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_low_temperature_correction_matches_oracle(N, K, precision):
    """HEOM_FLAG_LOW_TEMP at 77 K (small-N engine, complex H at N = 7, large-N engine)."""
    w = workloads.random_instance(N, K, seed=500 + N, complex_h=(N == 7))
    w["params"]["low_temp"] = 1
    w["params"]["T"] = 77.0
    g = run_gpu(w, precision)
    o = run_oracle(w)
    off = run_oracle(dict(w, params=dict(w["params"], low_temp=0)))
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    assert np.abs(o["pops"] - off["pops"]).max() > 20 * tp  # the correction is visible


def test_unknown_flags_rejected():
    w = workloads.random_instance(3, 2, seed=5)
    p = dict(w["params"])
    keep = heom._Keep(p, heom.FP64)
    keep.c.flags = 6
    h = heom.ctypes.c_void_p()
    assert heom.lib().heom_create(heom.ctypes.byref(keep.c), None, heom.ctypes.byref(h)) == heom.EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_autotune_keeps_state_and_result(precision):
    ws = [workloads.random_instance(N, K, seed=60 + N) for N, K in ((3, 3), (5, 2), (7, 3), (9, 1))]
    with heom.Batch([w["params"] for w in ws], precision) as b:
        b.set_rho0([w["rho0"] for w in ws])
        b.propagate(1.0, 20, 20)
        ms = b.autotune(trial_steps=5)
        assert ms > 0
        for N in (3, 5, 7, 9):
            shape = b.get_launch(N)
            assert shape["mode"] in (0, 2) and 1 <= shape["team_ctas"] <= 16
        rs = b.propagate(1.0, 20, 10)
    tol = TOL64 if precision == "fp64" else TOL32_POP
    for w, r in zip(ws, rs):
        o = oracle.propagate(w["params"], w["rho0"], 1.0, 40, 10)
        assert np.abs(r["pops"] - o["pops"][2:]).max() < tol
