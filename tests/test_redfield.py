"""The secular Redfield comparison model (oracle/redfield.c; the paper's
App. A1) against what fixes it: the Hermitian eigendecomposition, detailed
balance of its rates, the closed-form zero-frequency rate, relaxation to the
Gibbs state, probability conservation with trapping, the coherent limit
lambda = 0 (equal to the HEOM oracle there), and agreement with the HEOM
oracle in the weak-coupling limit, where both methods must describe the same
relaxation (the test also shows that a rate normalisation off by pi, the
paper's printed 2 pi J, would fail it)."""
import numpy as np
import pytest

import oracle
from oracle import redfield
from paper_1012_4382_gb300 import workloads

CM = 2 * np.pi * 2.99792458e-5  # cm^-1 -> rad/fs
KB = 0.6950348004  # cm^-1 / K


def test_spectrum_is_the_eigendecomposition():
    for w in (workloads.fmo_trap(), workloads.random_instance(6, 2, seed=3, complex_h=True)):
        p = w["params"]
        H = np.asarray(p["H"], dtype=complex) * CM
        E, C = redfield.spectrum(p)
        assert np.all(np.diff(E) >= 0)
        assert np.abs(E - np.linalg.eigvalsh(H)).max() < 1e-13
        assert np.abs(C.conj().T @ C - np.eye(p["N"])).max() < 1e-12
        assert np.abs(C @ np.diag(E) @ C.conj().T - H).max() < 1e-13


def test_rates_obey_detailed_balance_and_the_zero_frequency_form():
    p = dict(workloads.random_instance(5, 2, seed=11)["params"])
    kT = KB * p["T"] * CM
    E, _ = redfield.spectrum(p)
    W, g0 = redfield.rates(p, redfield.BOSE)
    Wh, g0h = redfield.rates(p, redfield.HIGH_T)
    lam, gam = np.asarray(p["lam"]) * CM, np.asarray(p["gam"]) * CM
    assert np.allclose(g0, 4 * lam * kT / gam, rtol=1e-13)
    assert np.allclose(g0h, g0, rtol=1e-13)
    for M in range(5):
        for K in range(5):
            if M == K:
                assert W[M, K] == 0.0
                continue
            om = E[M] - E[K]  # jump K -> M
            # Bose-Einstein rates: exactly the Boltzmann factor
            assert W[M, K] / W[K, M] == pytest.approx(np.exp(-om / kT), rel=1e-12)
            # high-temperature bath: (2 kT - omega) / (2 kT + omega), site by site
            assert Wh[M, K] / Wh[K, M] == pytest.approx((2 * kT - om) / (2 * kT + om), rel=1e-12)
            assert W[M, K] > 0


def test_relaxes_to_the_gibbs_state_without_trap():
    w = workloads.random_instance(4, 2, seed=21, trap=False)
    p = dict(w["params"])
    kT = KB * p["T"] * CM
    E, C = redfield.spectrum(p)
    W, _ = redfield.rates(p, redfield.BOSE)
    # the rate matrix's stationary vector is the Boltzmann distribution
    G = W - np.diag(W.sum(axis=0))
    boltz = np.exp(-(E - E[0]) / kT)
    boltz /= boltz.sum()
    assert np.abs(G @ boltz).max() < 1e-15
    # and a long propagation gets there (site populations of the exciton Gibbs
    # state): 100 ps are 24 times the slowest relaxation time of this model
    slowest = -1.0 / np.sort(np.linalg.eigvals(G).real)[-2]
    assert 2.0 * 50000 > 20 * slowest
    r = redfield.propagate(p, w["rho0"], 2.0, 50000, 50000)
    site_eq = (np.abs(C) ** 2) @ boltz
    assert np.abs(r["pops"][-1] - site_eq).max() < 1e-8


def test_probability_is_conserved_with_trap_and_decay():
    w = workloads.fmo_trap(nsteps=3000)
    r = redfield.propagate(w["params"], w["rho0"], 1.0, 3000, 100)
    assert np.abs(r["trace"] + r["eta"] + r["loss"] - 1.0).max() < 1e-12
    assert r["eta"][-1] > 0.05 and np.all(np.diff(r["eta"]) >= -1e-15)


def test_lambda_zero_is_the_coherent_limit_of_the_heom():
    """Without bath both methods reduce to -i[H, rho] plus the trap/decay
    terms: the Redfield model and the HEOM oracle (depth 0) agree to
    round-off (the same RK4 on the same linear system)."""
    w = workloads.fmo_trap(K=0, nsteps=800)
    p = dict(w["params"], lam=np.zeros(7))
    r = redfield.propagate(p, w["rho0"], 1.0, 800, 20)
    h = oracle.propagate(p, w["rho0"], 1.0, 800, 20)
    assert np.abs(r["pops"] - h["pops"]).max() < 1e-12
    assert np.abs(r["eta"] - h["eta"]).max() < 1e-12
    assert np.abs(r["loss"] - h["loss"]).max() < 1e-12


def _relaxation_mismatch(w, lam, K, rate_scale=1.0, steps=6000, every=200):
    """max |P_HEOM - P_Redfield| over the run, divided by the change of the
    HEOM populations, starting from the highest exciton state (no
    coherences, so the dropped Lamb shift does not enter)."""
    p = dict(w["params"], lam=np.full(w["params"]["N"], lam), K=K)
    _, C = redfield.spectrum(p)
    v = C[:, -1]
    rho0 = np.outer(v, v.conj())
    h = oracle.propagate(p, rho0, 1.0, steps, every)
    # Redfield rates are proportional to lambda: rate_scale multiplies them all
    pr = dict(p, lam=np.full(p["N"], lam * rate_scale))
    r = redfield.propagate(pr, rho0, 1.0, steps, every, bath_form=redfield.HIGH_T)
    effect = np.abs(h["pops"] - h["pops"][0]).max()
    return np.abs(h["pops"] - r["pops"]).max() / effect, np.abs(h["eta"] - r["eta"]).max()


@pytest.mark.parametrize("case", ["N3", "N4_trap"])
def test_weak_coupling_agrees_with_the_heom(case):
    w = (workloads.random_instance(3, 4, seed=5, trap=False) if case == "N3"
         else workloads.random_instance(4, 4, seed=8, trap=True))
    K = 6 if case == "N3" else 5
    strong, _ = _relaxation_mismatch(w, 2.0, K)
    weak, deta = _relaxation_mismatch(w, 0.5, K)
    assert weak < 0.05, weak  # a few per cent of the relaxation at lambda = 0.5 cm^-1
    assert weak < 0.7 * strong, (weak, strong)  # and the mismatch shrinks with the coupling
    assert deta < 5e-3
    # rates off by pi (2 pi J in place of 2 J) are clearly seen
    wrong, _ = _relaxation_mismatch(w, 0.5, K, rate_scale=np.pi)
    assert wrong > 5 * weak and wrong > 0.2, (wrong, weak)


def test_fmo_trapping_time_has_no_optimal_lambda():
    """The paper's FMO setting (Table-1 Hamiltonian, trapping from BChl 3 and 4
    at 1/(2.5 ps), radiative decay 1/(250 ps), 300 K, 1/gamma = 166 fs): it
    states that secular Redfield gives no local minimum of the trapping time
    in lambda, only a plateau (Sec. "Trapping time for different
    reorganization energies").  From BChl 1, <t> = int t d(eta) up to the
    paper's t_max (site population below 1e-5) decreases with lambda at every
    step of the grid, by less and less."""
    import os
    H = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "fmo_table1.txt"), comments="#")
    N = 7
    trap = np.zeros(N)
    trap[2] = trap[3] = 1.0 / 2.5
    rho0 = np.zeros((N, N), complex)
    rho0[0, 0] = 1.0
    tmean = []
    for lam in (10.0, 20.0, 55.0, 150.0, 300.0):
        p = dict(N=N, H=H.astype(complex), lam=np.full(N, lam), gam=np.full(N, 1.0 / (166.0 * CM)), T=300.0,
                 trap=trap, recomb=np.full(N, 1.0 / 250.0))
        r = redfield.propagate(p, rho0, 2.5, 40000, 4)  # the paper's 2.5 fs steps, rows every 10 fs
        site = r["pops"].sum(axis=1)
        end = int(np.argmax(site < 1e-5)) if (site < 1e-5).any() else len(site) - 1
        t = np.arange(end + 1) * 10.0
        eta = r["eta"][: end + 1]
        tmean.append(np.sum(0.5 * (t[1:] + t[:-1]) * np.diff(eta)) / 1000.0)
    d = np.diff(tmean)
    assert np.all(d < 0), tmean
    assert np.all(np.diff(-d) < 0), tmean  # the decrease flattens towards a plateau
