"""Scaled hierarchy (HEOM_FLAG_SCALED): the auxiliaries are stored as
sigma~_n = sigma_n / prod_j sqrt(n_j! s_j^{n_j}).  The CUDA path is compared
with the oracle's scaled mode element by element (populations, eta and, in
FP64, every stored auxiliary), and against its own unscaled path, which must
give the same rho."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, serving, workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32_POP = 1e-5
TOL32_ETA = 1e-4
W = 2.0 * math.pi * 2.99792458e-5  # cm^-1 -> rad/fs
KB = 0.6950348004  # cm^-1 / K


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def _scaled(w):
    return dict(w, params=dict(w["params"], scaled=1))


def _run(w, precision, launch=None):
    with heom.Context(w["params"], precision) as c:
        if launch:
            c.set_launch(**launch)
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], w["nsteps"], w["out_every"])
        r["state"], r["extra"] = c.state()
    return r


def _oracle_sites(w, N, K):
    o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], want_state=True)
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(o["multi"].tolist())}
    perm = np.array([pos[tuple(m)] for m in multi.tolist()])
    o["sites"] = o["state"][perm][:, :N, :N]
    return o


CASES = [(1, 3, False, 0), (2, 5, True, 1), (3, 3, False, 1), (5, 2, True, 0), (7, 3, True, 1), (8, 2, False, 0),
         (10, 2, True, 1), (24, 1, False, 0)]


@pytest.mark.parametrize("N,K,cplx,term", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scaled_hierarchy_matches_oracle(N, K, cplx, term, precision):
    w = _scaled(workloads.random_instance(N, K, seed=700 + 10 * N + K, complex_h=cplx, terminator=term))
    w["nsteps"], w["out_every"] = 60, 10
    g = _run(w, precision)
    o = _oracle_sites(w, N, K)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(g["pops"] - o["pops"]).max() < tp
    assert np.abs(g["eta"] - o["eta"]).max() < te
    # every stored auxiliary, relative to the largest one
    scale = np.abs(o["sites"]).max()
    assert np.abs(g["state"] - o["sites"]).max() < (1e-12 if precision == "fp64" else 1e-5) * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scaled_and_plain_paths_give_the_same_rho(precision):
    w = workloads.fmo_trap(K=4, nsteps=300)
    w["out_every"] = 50
    a = _run(w, precision)
    b = _run(_scaled(w), precision)
    tol = 1e-12 if precision == "fp64" else TOL32_POP
    assert np.abs(a["pops"] - b["pops"]).max() < tol
    assert np.abs(a["eta"] - b["eta"]).max() < tol
    # stored auxiliaries: sigma~_n = sigma_n / S(n)
    p = w["params"]
    kT = KB * p["T"] * W
    lam = np.broadcast_to(p["lam"], (7,)) * W
    gam = np.broadcast_to(p["gam"], (7,)) * W
    s = np.hypot(2 * lam * kT, lam * gam)
    multi, _, _ = heom.build_index(7, 4)
    S = np.array([math.prod(math.sqrt(math.factorial(int(k)) * s[j] ** int(k)) for j, k in enumerate(n))
                  for n in multi])
    rel = np.abs(b["state"] - a["state"] / S[:, None, None]).max() / np.abs(b["state"]).max()
    assert rel < (1e-12 if precision == "fp64" else 1e-4)


def test_scaled_launch_shapes():
    w = _scaled(workloads.random_instance(4, 3, seed=11))
    w["nsteps"], w["out_every"] = 20, 10
    o = _oracle_sites(w, 4, 3)
    with heom.Context(w["params"], "fp32") as c:
        shape = c.get_launch()
        assert shape["mode"] != 2 and shape["node_threads"] >= 3  # the default avoids shapes without a scaled kernel
    for precision in ("fp64", "fp32"):
        for shape in (dict(mode=0, team_ctas=2, block_threads=256, node_threads=4),
                      dict(mode=1, block_threads=256, node_threads=32)):
            g = _run(w, precision, shape)
            tp = TOL64 if precision == "fp64" else TOL32_POP
            assert np.abs(g["pops"] - o["pops"]).max() < tp
    for precision, shape in (("fp32", dict(node_threads=2)), ("fp64", dict(node_threads=1)),
                             ("fp32", dict(mode=2, team_ctas=1, node_threads=4))):
        with heom.Context(w["params"], precision) as c:
            c.set_launch(**shape)
            c.set_rho0(w["rho0"])
            with pytest.raises(heom.HeomError) as e:
                c.propagate(1.0, 5, 5)
            assert e.value.code == heom.EUNSUPPORTED
    with heom.Context(w["params"], "fp32") as c:
        c.set_rho0(w["rho0"])
        assert c.autotune(trial_steps=5) > 0  # shapes without a scaled kernel are skipped
        r = c.propagate(1.0, 20, 10)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL32_POP


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_of_scaled_and_plain_instances(precision):
    ws = [workloads.random_instance(3, 3, seed=900 + i) for i in range(4)]
    ws += [_scaled(workloads.random_instance(3, 3, seed=910 + i)) for i in range(4)]
    ws += [_scaled(workloads.random_instance(9, 1, seed=920))]
    with heom.Batch([w["params"] for w in ws], precision) as b:
        shape = b.get_launch(3)
        assert shape["mode"] != 2 and shape["node_threads"] >= 3  # N = 3 has scaled instances
        with pytest.raises(heom.HeomError) as e:
            b.get_launch(4)  # no instance with 4 sites
        assert e.value.code == heom.EINVAL
        b.set_rho0([w["rho0"] for w in ws])
        rs = b.propagate(1.0, 40, 10)
    tp = TOL64 if precision == "fp64" else TOL32_POP
    for w, r in zip(ws, rs):
        o = oracle.propagate(w["params"], w["rho0"], 1.0, 40, 10)
        assert np.abs(r["pops"] - o["pops"]).max() < tp


def test_server_runs_scaled_requests():
    w = _scaled(workloads.random_instance(5, 3, seed=77))
    with serving.Server(device_bytes=1 << 28, streams=2) as srv:
        i = srv.submit(w["params"], w["rho0"], 1.0, 50, 10, "fp32")
        t0 = time.time()
        while srv.status(i) not in (serving.DONE, serving.FAILED):
            srv.progress()
            assert time.time() - t0 < 60, "server did not finish"
            time.sleep(1e-4)
        assert srv.status(i) == serving.DONE
        r = srv.result(i)
    o = oracle.propagate(w["params"], w["rho0"], 1.0, 50, 10)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL32_POP


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scaled_stop_rule_and_trapping_time(precision):
    """The stop rule and <t> read rho only, so the scaled hierarchy stops at the
    same step and gives the same <t> as the oracle's scaled run."""
    w = _scaled(workloads.fmo_trap(K=3))
    p = dict(w["params"], trap=np.full(7, 20.0), recomb=np.full(7, 1.0))
    w = dict(w, params=p)
    nsteps, every = 3000, 10
    o = oracle.propagate(p, w["rho0"], 1.0, nsteps, 1, stop_trace=1e-5)
    n_stop = o["steps_done"]
    assert 0 < n_stop < nsteps
    with heom.Context(p, precision) as c:
        c.set_stop(1e-5)
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, nsteps, every)
        t, n = c.trapping_time()
    assert n == n_stop
    rows = n_stop // every + 1
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(r["pops"][:rows] - o["pops"][: n_stop + 1: every]).max() < tp
    assert abs(t - o["tmean"][n_stop]) < 2 * te * n_stop


def test_scaled_batch_graph_replay_equals_direct_calls():
    import torch
    ws = [_scaled(workloads.random_instance(N, K, seed=930 + N)) for N, K in ((3, 3), (7, 2), (10, 1))]
    n, every, reps = 40, 10, 2
    nout = n // every + 1
    Ns = sum(w["params"]["N"] for w in ws)
    dev = torch.device("cuda", 0)
    out = {}
    for mode in ("direct", "graph"):
        d_pops = torch.zeros(Ns * nout, dtype=torch.float64, device=dev)
        with heom.Batch([w["params"] for w in ws], "fp32") as b:
            b.set_rho0([w["rho0"] for w in ws])
            if mode == "direct":
                for _ in range(reps):
                    b.propagate_device(1.0, n, every, d_pops)
            else:
                with b.graph(1.0, n, every, d_pops) as g:
                    for _ in range(reps):
                        g.launch()
                    b.synchronize()
            b.synchronize()
            out[mode] = (d_pops.cpu().numpy(), np.array(b.efficiency()[0]))
    for a, c in zip(out["direct"], out["graph"]):
        assert np.array_equal(a, c)
    for i, w in enumerate(ws):
        o = oracle.propagate(w["params"], w["rho0"], 1.0, reps * n, reps * n)
        assert abs(out["graph"][1][i] - o["eta"][-1]) < TOL32_ETA
