"""The filtered hierarchy on the host (no GPU): the node selection of
heom_filter_select (threshold, root, closure downwards) against a brute-force
closure, and the oracle's filtered propagation (nodes removed from the
hierarchy) against the full hierarchy: identical when nothing is removed, and
an error that shrinks with the threshold when small scaled auxiliaries are
removed (the scaled HEOM needing fewer auxiliaries, the paper's
introduction)."""
import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def test_selection_is_the_threshold_closed_downwards():
    N, K = 4, 5
    multi, _, _ = heom.build_index(N, K)
    rng = np.random.default_rng(3)
    mags = 10.0 ** rng.uniform(-9, -1, size=len(multi))
    for delta in (0.0, 1e-6, 1e-4, 1e-2, np.inf):
        keep = heom.filter_select(N, K, mags, delta).astype(bool)
        # brute force: a node is kept iff it is the root or some node above the
        # threshold dominates it componentwise (n - e_j steps reach it)
        above = multi[mags >= delta]
        expect = np.array([i == 0 or bool(np.any(np.all(above >= m, axis=1))) for i, m in enumerate(multi)])
        assert np.array_equal(keep, expect), delta
        assert keep[0]
    assert heom.filter_select(N, K, mags, 0.0).all()
    assert heom.filter_select(N, K, mags, np.inf).sum() == 1
    # monotone in the threshold
    a = heom.filter_select(N, K, mags, 1e-6).astype(bool)
    b = heom.filter_select(N, K, mags, 1e-4).astype(bool)
    assert np.all(a >= b) and a.sum() > b.sum()


def test_selection_rejects_bad_input():
    with pytest.raises(heom.HeomError) as e:
        heom.filter_select(3, 2, np.zeros(10), -1.0)
    assert e.value.code == heom.EINVAL
    with pytest.raises(ValueError):
        heom.filter_select(3, 2, np.zeros(3), 1e-6)


def _to_oracle_order(keep, N, K):
    multi, _, _ = heom.build_index(N, K)
    pos = {tuple(m): i for i, m in enumerate(oracle.multi_indices(N, K).tolist())}
    out = np.zeros(len(multi), np.uint8)
    for i, m in enumerate(multi.tolist()):
        out[pos[tuple(m)]] = keep[i]
    return out


def test_oracle_filtered_hierarchy_keeping_every_node_is_the_full_one():
    w = workloads.fmo_trap(K=4, nsteps=300)
    p = dict(w["params"], scaled=1)
    a = oracle.propagate(p, w["rho0"], 1.0, 300, 30)
    b = oracle.propagate(dict(p, keep=np.ones(oracle.num_nodes(7, 4), np.uint8)), w["rho0"], 1.0, 300, 30)
    assert np.array_equal(a["pops"], b["pops"]) and np.array_equal(a["eta"], b["eta"])


def test_oracle_filtered_error_shrinks_with_the_threshold():
    """Pilot (500 fs of the full scaled hierarchy, magnitudes every 100 fs),
    selection, then 3 ps of the filtered hierarchy against the full one."""
    N, K = 7, 5
    w = workloads.fmo_trap(K=K)
    p = dict(w["params"], scaled=1)
    multi, _, _ = heom.build_index(N, K)
    om = oracle.multi_indices(N, K)
    pos = {tuple(m): i for i, m in enumerate(om.tolist())}
    perm = np.array([pos[tuple(m)] for m in multi.tolist()])  # library order -> oracle order
    mags = np.zeros(len(multi))
    for t in (100, 200, 300, 400, 500):
        st = oracle.propagate(p, w["rho0"], 1.0, t, t, want_state=True)["state"][:, :N, :N]
        mags = np.maximum(mags, np.abs(st).reshape(len(om), -1).max(axis=1)[perm])
    full = oracle.propagate(p, w["rho0"], 1.0, 3000, 30)
    errs, kept = [], []
    for delta in (1e-4, 1e-5, 1e-6):
        keep = heom.filter_select(N, K, mags, delta)
        f = oracle.propagate(dict(p, keep=_to_oracle_order(keep, N, K)), w["rho0"], 1.0, 3000, 30)
        errs.append(max(np.abs(f["pops"] - full["pops"]).max(), np.abs(f["eta"] - full["eta"]).max()))
        kept.append(int(keep.sum()))
    assert kept[0] < kept[1] <= kept[2] <= len(multi)
    assert kept[0] < 0.8 * len(multi)  # a real reduction at the coarsest threshold
    assert errs[0] < 1e-3 and errs[1] < 1e-4
    assert errs[2] <= errs[1] <= errs[0]
