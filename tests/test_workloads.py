"""The seeded synthetic inputs follow the recipe the design notes state:
shapes, ranges, seeds and the Poisson arrival process of the serving trace."""
import numpy as np

from paper_1012_4382_gb300 import workloads


def _is_hermitian(H):
    return np.allclose(H, np.conj(H.T), atol=0.0)


def test_fmo_like_workload():
    w = workloads.fmo_trap()
    p = w["params"]
    assert (p["N"], p["K"], w["nsteps"], w["dt"], w["out_every"]) == (7, 6, 10000, 1.0, 10)
    H = p["H"]
    assert _is_hermitian(H) and np.all(H.imag == 0)
    assert np.all((H.real.diagonal() >= 12100) & (H.real.diagonal() <= 12600))
    off = H.real[np.triu_indices(7, 1)]
    assert 5.0 < off.std() < 100.0  # couplings of tens of cm^-1
    assert np.array_equal(p["trap"], np.eye(7)[2])  # 1 ps^-1 on index 2 (BChl 3)
    assert np.all(p["recomb"] == 1e-3)
    assert np.all(p["lam"] == 35.0) and np.all(p["gam"] == 106.0) and p["T"] == 300.0
    assert w["rho0"][0, 0] == 1.0 and np.abs(w["rho0"]).sum() == 1.0
    # seeded: the same call gives the same model, another seed another one
    assert np.array_equal(workloads.fmo_trap()["params"]["H"], H)
    assert not np.array_equal(workloads.fmo_trap(seed=5)["params"]["H"], H)


def test_batched_scan_recipe():
    ws = workloads.batched_scan()
    assert len(ws) == 256
    K = np.array([w["params"]["K"] for w in ws])
    lam = np.array([w["params"]["lam"][0] for w in ws])
    T = np.array([w["params"]["T"] for w in ws])
    assert set(K) == set(range(4, 9))
    assert lam.min() >= 2.0 and lam.max() <= 200.0 and lam.std() > 30.0
    assert T.min() >= 77.0 and T.max() <= 300.0
    assert all(w["nsteps"] == 5000 and w["params"]["N"] == 7 for w in ws)
    # per-instance Hamiltonians
    assert not np.array_equal(ws[0]["params"]["H"], ws[1]["params"]["H"])


def test_serving_trace_is_poisson_with_the_stated_mix():
    tr = workloads.serving_trace()
    assert len(tr) == 2000
    t = np.array([w["arrival_s"] for w in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps of mean 1/200 s: mean and coefficient of variation near 1/200 and 1
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.08
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    N = np.array([w["params"]["N"] for w in tr])
    K = np.array([w["params"]["K"] for w in tr])
    ps = np.array([w["nsteps"] for w in tr]) / 1000.0
    assert set(N) == set(range(2, 9)) and set(K) == set(range(3, 9))
    assert ps.min() >= 1.0 and ps.max() <= 20.0
    for w in tr[:50]:
        n = w["params"]["N"]
        assert w["params"]["trap"][min(2, n - 1)] == 1.0 and w["params"]["trap"].sum() == 1.0
        assert _is_hermitian(w["params"]["H"])
    slow = workloads.serving_trace(count=400, rate_per_s=12.0)
    assert abs(np.diff([w["arrival_s"] for w in slow]).mean() * 12.0 - 1.0) < 0.15


def test_large_trimer_block_structure():
    w = workloads.large_trimer()
    p = w["params"]
    assert (p["N"], p["K"], w["nsteps"]) == (24, 4, 2000)
    assert p["trap"] is None and p["recomb"] is None
    H = p["H"].real
    blk = np.arange(24) // 8
    same = blk[:, None] == blk[None, :]
    iu = np.triu_indices(24, 1)
    intra = H[iu][same[iu]]
    inter = H[iu][~same[iu]]
    assert 25.0 < intra.std() < 60.0 and 2.5 < inter.std() < 8.0
