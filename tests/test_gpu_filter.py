"""Filtered hierarchies on the GPU (heom_node_magnitudes, heom_filter_select,
heom_create_subset) against the oracle: the node magnitudes of a scaled
state, and a filtered context in every engine against the oracle propagating
the same node set (nodes removed from its hierarchy), element by element."""
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


def _perm(N, K):
    """library node order -> oracle node order"""
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(oracle.multi_indices(N, K).tolist())}
    return np.array([pos[tuple(m)] for m in multi.tolist()])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_node_magnitudes_match_the_oracle_state(precision):
    w = workloads.fmo_trap(K=5, nsteps=300)
    p = dict(w["params"], scaled=1)
    with heom.Context(p, precision) as c:
        c.set_rho0(w["rho0"])
        c.propagate(1.0, 300, 300)
        mags = c.node_magnitudes()
    st = oracle.propagate(p, w["rho0"], 1.0, 300, 300, want_state=True)["state"][:, :7, :7]
    ref = np.abs(st).reshape(len(st), -1).max(axis=1)[_perm(7, 5)]
    assert np.abs(mags - ref).max() < (TOL64 if precision == "fp64" else 1e-6)


@pytest.fixture(scope="module")
def pilot():
    """Filter of the FMO-like depth-5 scaled hierarchy from a 500 fs GPU pilot
    (magnitudes every 100 fs, FP64), threshold 1e-5."""
    w = workloads.fmo_trap(K=5, nsteps=400)
    p = dict(w["params"], scaled=1)
    mags = None
    with heom.Context(p, "fp64") as c:
        c.set_rho0(w["rho0"])
        for _ in range(5):
            c.propagate(1.0, 100, 100)
            m = c.node_magnitudes()
            mags = m if mags is None else np.maximum(mags, m)
    keep = heom.filter_select(7, 5, mags, 1e-5)
    assert 0.2 * len(keep) < keep.sum() < len(keep)  # a real reduction
    okeep = np.zeros(len(keep), np.uint8)
    okeep[_perm(7, 5)] = keep
    o = oracle.propagate(dict(p, keep=okeep), w["rho0"], 1.0, 400, 20, want_state=True)
    return w, p, keep, o


SHAPES = [None, dict(mode=0, team_ctas=4, block_threads=256, node_threads=8),
          dict(mode=1, team_ctas=1, block_threads=256, node_threads=32), dict(mode=3, block_threads=12 * 28)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "default" if s is None else "m%d" % s["mode"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_filtered_context_matches_the_filtered_oracle(pilot, precision, shape):
    w, p, keep, o = pilot
    with heom.Context(p, precision, keep=keep) as c:
        assert c.nodes == int(keep.sum())
        if shape:
            c.set_launch(**shape)
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 400, 20)
        state, _ = c.state()
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(r["pops"] - o["pops"]).max() < tp
    assert np.abs(r["eta"] - o["eta"]).max() < te
    kept = np.flatnonzero(keep)
    ref = o["state"][_perm(7, 5)[kept]][:, :7, :7]
    assert state.shape == ref.shape
    assert np.abs(state - ref).max() < (TOL64 if precision == "fp64" else 1e-5)


def test_filtered_run_stays_close_to_the_full_hierarchy(pilot):
    w, p, keep, _ = pilot
    with heom.Context(p, "fp32", keep=keep) as c:
        c.set_rho0(w["rho0"])
        f = c.propagate(1.0, 3000, 30)
    with heom.Context(p, "fp32") as c:
        c.set_rho0(w["rho0"])
        g = c.propagate(1.0, 3000, 30)
    assert np.abs(f["pops"] - g["pops"]).max() < 1e-4
    assert np.abs(f["eta"] - g["eta"]).max() < 1e-4


def test_filtered_context_rejects_bad_node_sets():
    w = workloads.fmo_trap(K=3, nsteps=10)
    M = heom.num_nodes(7, 3)
    no_root = np.ones(M, np.uint8)
    no_root[0] = 0
    with pytest.raises(heom.HeomError) as e:
        heom.Context(w["params"], "fp32", keep=no_root)
    assert e.value.code == heom.EINVAL
    open_set = np.zeros(M, np.uint8)
    open_set[0] = 1
    open_set[M - 1] = 1  # a deepest node without its lower neighbours
    with pytest.raises(heom.HeomError) as e:
        heom.Context(w["params"], "fp32", keep=open_set)
    assert e.value.code == heom.EINVAL
    with pytest.raises(heom.HeomError) as e:
        heom.Context(dict(w["params"], terminator=1), "fp32", keep=np.ones(M, np.uint8))
    assert e.value.code == heom.EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_filtered_batch_matches_the_filtered_oracle(pilot, precision):
    """A batch mixing a filtered instance, the same instance unfiltered and a
    filtered instance of another size, in the batch's default launch."""
    w, p, keep, o = pilot
    w3 = workloads.random_instance(4, 4, seed=31)
    p3 = dict(w3["params"], scaled=1)
    M3 = heom.num_nodes(4, 4)
    keep3 = heom.filter_select(4, 4, np.linspace(1.0, 0.0, M3), 0.5)  # the shallower half, closed downwards
    with heom.Batch([p, p, p3], precision, keep=[keep, None, keep3]) as b:
        assert b.num_nodes(0) == int(keep.sum()) and b.num_nodes(1) == heom.num_nodes(7, 5)
        b.set_rho0([w["rho0"], w["rho0"], w3["rho0"]])
        res = b.propagate(1.0, 400, 20)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(res[0]["pops"] - o["pops"]).max() < tp
    assert np.abs(res[0]["eta"] - o["eta"]).max() < te
    full = oracle.propagate(p, w["rho0"], 1.0, 400, 20)
    assert np.abs(res[1]["pops"] - full["pops"]).max() < tp
    ok3 = np.zeros(M3, np.uint8)
    ok3[_perm(4, 4)] = keep3
    o3 = oracle.propagate(dict(p3, keep=ok3), w3["rho0"], 1.0, 400, 20)
    assert np.abs(res[2]["pops"] - o3["pops"]).max() < tp
    assert np.abs(res[2]["eta"] - o3["eta"]).max() < te


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kept_nodes_propagated_unscaled_match_the_oracle(pilot, precision):
    """The node set chosen from the scaled magnitudes, propagated in the
    unscaled representation (same auxiliaries, same rho; the batched and
    large-hierarchy kernels of that form are the fast ones)."""
    w, p, keep, o_scaled = pilot
    pu = dict(p, scaled=0)
    ok = np.zeros(len(keep), np.uint8)
    ok[_perm(7, 5)] = keep
    o = oracle.propagate(dict(pu, keep=ok), w["rho0"], 1.0, 400, 20)
    with heom.Context(pu, precision, keep=keep) as c:
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 400, 20)
    tp, te = (TOL64, TOL64) if precision == "fp64" else (TOL32_POP, TOL32_ETA)
    assert np.abs(r["pops"] - o["pops"]).max() < tp
    assert np.abs(r["eta"] - o["eta"]).max() < te
    # the same physics as the scaled filtered run
    assert np.abs(o["pops"] - o_scaled["pops"]).max() < 1e-12


def test_filtered_depth8_runs_several_nodes_per_thread():
    """A filtered depth-8 hierarchy of about 4000 kept nodes: too many for one
    node per thread of the dataflow engine, so the default carries several;
    every kept node against the oracle on the same node set."""
    w = workloads.fmo_trap(K=8, nsteps=30)
    p = w["params"]
    M = heom.num_nodes(7, 8)
    keep = heom.filter_select(7, 8, np.linspace(1.0, 0.0, M), 0.38)  # the first ~62 %, closed downwards
    assert 3000 < keep.sum() < 5000
    with heom.Context(p, "fp32", keep=keep) as c:
        L = c.get_launch()
        assert L["mode"] == 3 and L["team_ctas"] > 1, L
        c.set_rho0(w["rho0"])
        r = c.propagate(1.0, 30, 10)
        st, _ = c.state()
    okeep = np.zeros(M, np.uint8)
    okeep[_perm(7, 8)] = keep
    o = oracle.propagate(dict(p, keep=okeep), w["rho0"], 1.0, 30, 10, want_state=True)
    assert np.abs(r["pops"] - o["pops"]).max() < TOL32_POP
    assert np.abs(r["eta"] - o["eta"]).max() < TOL32_ETA
    kept = np.flatnonzero(keep)
    ref = o["state"][_perm(7, 8)][kept][:, :7, :7]
    assert np.abs(st - ref).max() < 1e-5
