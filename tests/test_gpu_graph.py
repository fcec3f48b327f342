"""A batch propagation captured as a CUDA graph replays exactly what the
direct calls compute (same kernels, same descriptors, same summation order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def _instances():
    return [workloads.random_instance(N, K, seed=900 + N) for N, K in ((3, 3), (5, 2), (7, 3), (7, 2))]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_equals_direct_calls(precision):
    ws = _instances()
    n, every, reps = 60, 10, 3
    nout = n // every + 1
    rows = len(ws) * nout
    Ns = sum(w["params"]["N"] for w in ws)
    dev = torch.device("cuda", 0)
    out = {}
    for mode in ("direct", "graph"):
        d_pops = torch.zeros(Ns * nout, dtype=torch.float64, device=dev)
        d_el = torch.zeros(2 * rows, dtype=torch.float64, device=dev)
        with heom.Batch([w["params"] for w in ws], precision) as b:
            b.set_rho0([w["rho0"] for w in ws])
            if mode == "direct":
                for _ in range(reps):
                    b.propagate_device(1.0, n, every, d_pops, d_el)
            else:
                with b.graph(1.0, n, every, d_pops, d_el) as g:
                    for _ in range(reps):
                        g.launch()
                    b.synchronize()
            b.synchronize()
            out[mode] = (d_pops.cpu().numpy(), d_el.cpu().numpy(), b.efficiency()[0], b.trapping_time()[0])
    for a, c in zip(out["direct"], out["graph"]):
        assert np.array_equal(a, c)
    # and the replays continued the propagation: compare with the oracle after reps * n steps
    tol = 1e-10 if precision == "fp64" else 1e-4
    for i, w in enumerate(ws):
        o = oracle.propagate(w["params"], w["rho0"], 1.0, reps * n, reps * n)
        assert abs(out["graph"][2][i] - o["eta"][-1]) < tol


def test_graph_restarts_after_set_rho0():
    """set_rho0 between replays restarts the instances: replay, reset, replay
    equals one direct call from rho(0) (cluster mode, explicit shape)."""
    ws = _instances()[:2]
    n, every = 40, 10
    nout = n // every + 1
    Ns = sum(w["params"]["N"] for w in ws)
    dev = torch.device("cuda", 0)
    res = []
    for mode in ("direct", "graph"):
        d_pops = torch.zeros(Ns * nout, dtype=torch.float64, device=dev)
        with heom.Batch([w["params"] for w in ws], "fp64") as b:
            b.set_launch(mode=0, team_ctas=1, block_threads=256, node_threads=2)
            b.set_rho0([w["rho0"] for w in ws])
            if mode == "direct":
                b.propagate_device(1.0, n, every, d_pops)
            else:
                with b.graph(1.0, n, every, d_pops) as g:
                    g.launch()
                    b.synchronize()
                    b.set_rho0([w["rho0"] for w in ws])
                    g.launch()
                    b.synchronize()
            b.synchronize()
            res.append(d_pops.cpu().numpy())
    assert np.array_equal(res[0], res[1])
