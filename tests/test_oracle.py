"""Pins the FP64 CPU oracle to results fixed by the paper and by mathematics.

Each test below checks the oracle against something that is not the oracle:
counts printed in the paper, closed-form solutions of special cases, exact
invariants of the equations, and a dense matrix exponential of the generator.
A dropped term, a wrong sign or a swapped site index anywhere in the
right-hand side fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_1012_4382_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C_CM_PER_FS = 2.99792458e-5
KB = 0.6950348004  # cm^-1 / K
W = 2.0 * math.pi * C_CM_PER_FS  # cm^-1 -> rad/fs


def _load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


# ----------------------------------------------------------------------------
# Hierarchy size and structure (App. B: N_tot = (N+N_max)!/(N! N_max!))
# ----------------------------------------------------------------------------

def test_node_counts_match_paper_table():
    for N, K, nodes in _load_table("table2_node_counts.txt").astype(int):
        assert oracle.num_nodes(N, K) == nodes
        assert math.comb(N + K, K) == nodes


@pytest.mark.parametrize("N,K", [(1, 0), (1, 5), (2, 4), (3, 3), (4, 2), (5, 0)])
def test_multi_indices_brute_force(N, K):
    got = oracle.multi_indices(N, K)
    brute = sorted(t for t in itertools.product(range(K + 1), repeat=N) if sum(t) <= K)
    assert len(got) == len(brute) == math.comb(N + K, K)
    assert sorted(map(tuple, got.tolist())) == brute
    # root first, levels non-decreasing
    assert tuple(got[0]) == (0,) * N
    assert np.all(np.diff(got.sum(axis=1)) >= 0)


# ----------------------------------------------------------------------------
# Closed forms
# ----------------------------------------------------------------------------

def test_rabi_oscillation_lambda_zero():
    """lambda = 0: the auxiliaries stay zero and the dimer oscillates coherently,
    P_1(t) = 1 - (4 J^2 / Omega^2) sin^2(Omega t / 2), Omega = sqrt(Delta^2 + 4 J^2)."""
    w = workloads.dimer()
    p = dict(w["params"])
    p["lam"] = np.zeros(2)
    r1 = oracle.propagate(p, w["rho0"], 1.0, 1000, 1)
    r2 = oracle.propagate(p, w["rho0"], 0.5, 2000, 2)
    t = np.arange(1001) * 1.0
    om = math.sqrt(100.0 ** 2 + 4 * 100.0 ** 2) * W
    p1 = 1.0 - (4 * 100.0 ** 2 / (100.0 ** 2 + 4 * 100.0 ** 2)) * np.sin(om * t / 2) ** 2
    e1 = np.abs(r1["pops"][:, 0] - p1).max()
    e2 = np.abs(r2["pops"][:, 0] - p1).max()
    assert e1 < 1e-6
    assert 12.0 < e1 / e2 < 20.0  # RK4: error ~ dt^4
    assert np.abs(r1["trace"] - 1.0).max() < 1e-13


def _pure_dephasing_exact(lam, gam, T, e1, e2, t):
    """Two uncoupled sites, one Drude bath each: the (1,2) element of the
    hierarchy decouples into a scalar chain whose infinite-depth solution is
    rho_12(t) = rho_12(0) exp(-i(e1-e2)t - (a1 - i b1) f1(t) - (a2 + i b2) f2(t)),
    a = 2 lambda k_B T, b = lambda gamma, f(t) = (gamma t - 1 + exp(-gamma t)) / gamma^2."""
    a = 2 * lam * W * KB * T * W
    b = lam * gam * W * W
    g = gam * W
    f = (g * t - 1 + np.exp(-g * t)) / g ** 2
    return np.exp(-1j * (e1 - e2) * W * t - (a[0] - 1j * b[0]) * f[0] - (a[1] + 1j * b[1]) * f[1])


def test_pure_dephasing_closed_form():
    lam = np.array([35.0, 10.0])
    gam = np.array([106.0, 60.0])
    H = np.diag([0.0, 150.0]).astype(complex)
    p = dict(N=2, K=30, H=H, lam=lam, gam=gam, T=300.0)
    rho0 = np.full((2, 2), 0.5, dtype=complex)
    exact = 0.5 * _pure_dephasing_exact(lam, gam, 300.0, 0.0, 150.0, 200.0)
    r1 = oracle.propagate(p, rho0, 1.0, 200, 200)
    r2 = oracle.propagate(p, rho0, 0.5, 400, 400)
    e1 = abs(r1["rho"][0, 1] - exact) / abs(exact)
    e2 = abs(r2["rho"][0, 1] - exact) / abs(exact)
    assert e1 < 2e-6
    assert 10.0 < e1 / e2 < 22.0
    # populations do not move without inter-site coupling
    assert np.abs(r1["pops"] - 0.5).max() < 1e-14


def _matsubara_rate(lam_cm, gam_cm, T):
    """sum_{k>=1} c_k / nu_k of the Drude-Lorentz Matsubara terms by direct
    summation (rad/fs): c_k / nu_k = 4 lambda gamma kT / (nu_k^2 - gamma^2),
    nu_k = 2 pi k kT; 10^6 terms plus the 1/k^2 tail."""
    lam, gam, kT = lam_cm * W, gam_cm * W, KB * T * W
    k = np.arange(1, 1_000_001, dtype=np.float64)
    nu = 2.0 * math.pi * k * kT
    s = np.sum(4.0 * lam * gam * kT / (nu * nu - gam * gam))
    return s + lam * gam / (math.pi ** 2 * kT * k[-1])


@pytest.mark.parametrize("T", [300.0, 77.0])
def test_low_temperature_correction_dephasing(T):
    """The lowest-order quantum correction adds -sum_j c_j V_j^x V_j^x sigma_n,
    c_j the Markovian weight of the Matsubara terms.  On the pure-dephasing
    case it damps every node's (1,2) element by exp(-(c_1 + c_2) t) on top of
    the high-temperature solution; c_j is computed here by summing the series."""
    lam = np.array([35.0, 10.0])
    gam = np.array([106.0, 60.0])
    H = np.diag([0.0, 150.0]).astype(complex)
    rho0 = np.full((2, 2), 0.5, dtype=complex)
    c = sum(_matsubara_rate(lam[j], gam[j], T) for j in range(2))
    assert c > 0
    base = oracle.propagate(dict(N=2, K=30, H=H, lam=lam, gam=gam, T=T), rho0, 0.5, 400, 400)
    ltc = oracle.propagate(dict(N=2, K=30, H=H, lam=lam, gam=gam, T=T, low_temp=1), rho0, 0.5, 400, 400)
    ratio = ltc["rho"][0, 1] / base["rho"][0, 1]
    # equal up to the RK4 error of the two runs (a few 1e-9 at dt = 0.5 fs); a
    # 1e-6 relative error in c_j would show as 1e-7 here
    assert abs(ratio - math.exp(-c * 200.0)) < 2e-8
    # the correction does not touch populations
    assert np.abs(ltc["pops"] - 0.5).max() < 1e-14


def test_markov_terminator_reduces_truncation_error():
    lam = np.array([35.0, 10.0])
    gam = np.array([106.0, 60.0])
    H = np.diag([0.0, 150.0]).astype(complex)
    rho0 = np.full((2, 2), 0.5, dtype=complex)
    exact = 0.5 * _pure_dephasing_exact(lam, gam, 300.0, 0.0, 150.0, 200.0)
    for K in (2, 4, 6):
        errs = []
        for term in (0, 1):
            p = dict(N=2, K=K, H=H, lam=lam, gam=gam, T=300.0, terminator=term)
            r = oracle.propagate(p, rho0, 0.5, 400, 400)
            errs.append(abs(r["rho"][0, 1] - exact))
        assert errs[1] < errs[0] / 2


@pytest.mark.parametrize("K", [0, 1, 2, 3, 4])
def test_markov_terminator_keeps_the_exact_long_time_rate(K):
    """One bath (on site 1) and two uncoupled sites: the (1,2) elements form
    the chain x_n' = -n g x_n + i x_{n+1} + n c x_{n-1}, c = i a + b, whose
    infinite-depth solution decays at long times with the Markov rate
    lambda = i c / g (the t/g term of f(t) in the closed form above).  The
    vector x_n = (c/g)^n is an exact eigenvector of the infinite chain for
    that rate, and at the last level the terminator's
    (n_1 + 1) c x_n / (n_1 g + g) equals its next entry, so a chain cut at any
    depth K with the terminator keeps the exact rate; without it the rate is
    off by about (|c|/g^2)^(K+1) g.  Checked on x_0(t2)/x_0(t1) at times where
    the faster modes (rates near -g, -2g, ...) have died out, against the RK4
    amplification of that rate.  The (n_j + 1)
    factor and the sum_k n_k g_k of the denominator enter at every K >= 1."""
    lam = np.array([2.0, 0.0])
    gam = np.array([106.0, 60.0])
    H = np.diag([0.0, 150.0]).astype(complex)
    rho0 = np.full((2, 2), 0.5, dtype=complex)
    t1, t2 = 1000, 2000
    a = 2 * lam[0] * W * KB * 300.0 * W
    b = lam[0] * gam[0] * W * W
    g = gam[0] * W
    # the rate of x_0 (phase of the site-energy difference included); classic RK4
    # advances an eigenvector of a linear system by the degree-4 Taylor polynomial
    # P(h lambda) per step exactly, so the expected ratio carries no time-step error
    rate = -1j * (0.0 - 150.0) * W - (a - 1j * b) / g
    z = rate * 1.0
    markov = (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24) ** (t2 - t1)
    assert abs(markov - np.exp(rate * (t2 - t1))) < 1e-6  # and it is the continuous rate to RK4 accuracy
    ratios = []
    for term in (1, 0):
        p = dict(N=2, K=K, H=H, lam=lam, gam=gam, T=300.0, terminator=term)
        x1 = oracle.propagate(p, rho0, 1.0, t1, t1)["rho"][0, 1]
        x2 = oracle.propagate(p, rho0, 1.0, t2, t2)["rho"][0, 1]
        ratios.append(x2 / x1)
    assert abs(ratios[0] - markov) < 1e-8 * abs(markov)
    # the plain truncation misses it by far more at every depth here
    assert abs(ratios[1] - markov) > 1e-6 * abs(markov)


def test_single_site_trap_and_decay_closed_form():
    """One site with trap rate G_t and radiative rate G_r (ps^-1): the bath
    cannot act (V^x vanishes on a 1x1 block), so rho_11 = exp(-(G_t+G_r) t),
    eta = G_t/(G_t+G_r) (1 - exp(-(G_t+G_r) t)), loss likewise with G_r."""
    gt, gr = 0.8, 0.05
    p = dict(N=1, K=3, H=np.array([[12345.0]]), lam=35.0, gam=106.0, T=300.0,
             trap=np.array([gt]), recomb=np.array([gr]))
    r = oracle.propagate(p, np.array([[1.0]]), 1.0, 3000, 100)
    t = np.arange(r["pops"].shape[0]) * 100.0
    g = (gt + gr) * 1e-3
    assert np.abs(r["pops"][:, 0] - np.exp(-g * t)).max() < 1e-12
    assert np.abs(r["eta"] - gt / (gt + gr) * (1 - np.exp(-g * t))).max() < 1e-12
    assert np.abs(r["loss"] - gr / (gt + gr) * (1 - np.exp(-g * t))).max() < 1e-12


def test_trapping_time_single_site_closed_form():
    """Eq. trappingtime for one site: d eta/dt = G_t exp(-g t), so
    <t>(T) = G_t / g^2 (1 - exp(-g T) (1 + g T)), g = G_t + G_r (fs^-1)."""
    gt, gr = 0.8, 0.05
    p = dict(N=1, K=2, H=np.array([[12345.0]]), lam=35.0, gam=106.0, T=300.0,
             trap=np.array([gt]), recomb=np.array([gr]))
    r = oracle.propagate(p, np.array([[1.0]]), 1.0, 6000, 250)
    t = np.arange(r["tmean"].shape[0]) * 250.0
    g, G = (gt + gr) * 1e-3, gt * 1e-3
    exact = G / g**2 * (1.0 - np.exp(-g * t) * (1.0 + g * t))
    assert r["tmean"][0] == 0.0
    assert np.abs(r["tmean"] - exact).max() < 1e-9 * exact.max()
    # the running value tends to the mean trapping time G_t / g^2 times eta(inf)
    assert abs(r["tmean"][-1] - G / g**2) < 0.05 * G / g**2


def test_trapping_time_nonhermitian_dimer_quadrature():
    """Without a bath the trapped flux is sum_m Gamma_m |psi_m(t)|^2 with
    psi(t) = expm(-i H_eff t) psi(0); <t> by Gauss-Legendre quadrature of
    t times that flux must match the oracle's value within the RK4 error."""
    H = np.array([[0.0, 80.0], [80.0, 120.0]], dtype=complex)
    trap = np.array([0.0, 1.5])
    p = dict(N=2, K=2, H=H, lam=0.0, gam=106.0, T=300.0, trap=trap)
    T = 2000.0
    r = oracle.propagate(p, workloads.pure_state(2, 0), 0.5, int(T / 0.5), int(T / 0.5))
    heff = H * W - 0.5j * np.diag(trap * 1e-3)
    x, wq = np.polynomial.legendre.leggauss(64)
    total = 0.0
    for k in range(40):  # 40 panels of 50 fs
        a, b = k * T / 40, (k + 1) * T / 40
        for xi, wi in zip(x, wq):
            t = 0.5 * (b - a) * xi + 0.5 * (a + b)
            psi = expm(-1j * heff * t) @ np.array([1.0, 0.0])
            total += 0.5 * (b - a) * wi * t * np.sum(trap * 1e-3 * np.abs(psi) ** 2)
    assert abs(r["tmean"][-1] - total) < 1e-6 * total


def test_stop_rule_ends_at_t_max():
    """Sec. "Trapping time": propagation stops once the site population is
    below the threshold.  For one site RK4 multiplies the population by
    P(-g h) = 1 - x + x^2/2 - x^3/6 + x^4/24 (x = g h) per step, so the stop
    step is known exactly; later output rows are NaN."""
    gt = 5.0
    p = dict(N=1, K=1, H=np.array([[0.0]]), lam=35.0, gam=106.0, T=300.0, trap=np.array([gt]))
    x = gt * 1e-3 * 2.0
    f = 1 - x + x**2 / 2 - x**3 / 6 + x**4 / 24
    s_stop = int(np.ceil(np.log(1e-5) / np.log(f)))
    assert f ** s_stop < 1e-5 <= f ** (s_stop - 1)
    r = oracle.propagate(p, np.array([[1.0]]), 2.0, 5000, 1, stop_trace=1e-5)
    assert r["steps_done"] == s_stop
    assert np.isfinite(r["pops"][: s_stop + 1]).all() and np.isnan(r["pops"][s_stop + 1:]).all()
    assert abs(r["pops"][s_stop, 0] - f ** s_stop) < 1e-15
    full = oracle.propagate(p, np.array([[1.0]]), 2.0, 5000, 1)
    assert full["steps_done"] == 5000
    assert np.array_equal(full["tmean"][: s_stop + 1], r["tmean"][: s_stop + 1])


def test_nonhermitian_dimer_without_bath():
    """lambda = 0 with a trap: a pure state evolves with the non-Hermitian
    H_eff = H - (i/2) diag(Gamma), so rho(t) = psi psi^+ with
    psi = expm(-i H_eff t) psi(0), and eta = 1 - |psi|^2 (all loss goes to RC)."""
    H = np.array([[0.0, 80.0], [80.0, 120.0]], dtype=complex)
    trap = np.array([0.0, 1.5])
    p = dict(N=2, K=2, H=H, lam=0.0, gam=106.0, T=300.0, trap=trap)
    r = oracle.propagate(p, workloads.pure_state(2, 0), 0.5, 4000, 100)
    heff = H * W - 0.5j * np.diag(trap * 1e-3)
    for o, t in enumerate(np.arange(r["pops"].shape[0]) * 50.0):
        psi = expm(-1j * heff * t) @ np.array([1.0, 0.0])
        # RK4 error at dt = 0.5 fs over 2 ps is a few 1e-9 here
        assert np.abs(r["pops"][o] - np.abs(psi) ** 2).max() < 1e-8
        assert abs(r["eta"][o] - (1.0 - np.vdot(psi, psi).real)) < 1e-8


# ----------------------------------------------------------------------------
# Invariants
# ----------------------------------------------------------------------------

def test_hermiticity_and_probability_conservation():
    w = workloads.random_instance(3, 3, seed=11, trap=True)
    p = w["params"]
    r = oracle.propagate(p, w["rho0"], 1.0, 300, 10, want_state=True)
    st = r["state"]
    herm = np.abs(st - np.conj(np.transpose(st, (0, 2, 1)))).max()
    assert herm < 1e-14
    total = r["trace"] + r["eta"] + r["loss"]
    assert np.abs(total - 1.0).max() < 1e-13
    assert r["eta"][-1] > 1e-3  # the trap is active


def test_no_trap_means_no_efficiency():
    w = workloads.random_instance(3, 3, seed=5, trap=False)
    r = oracle.propagate(w["params"], w["rho0"], 1.0, 300, 10)
    assert np.all(r["eta"] == 0.0) and np.all(r["loss"] == 0.0)
    assert np.abs(r["trace"] - 1.0).max() < 1e-13


# ----------------------------------------------------------------------------
# RK4 against the dense generator of the dimer hierarchy
# ----------------------------------------------------------------------------

def test_rk4_equals_taylor_polynomial_and_approaches_expm():
    w = workloads.dimer()
    p = dict(w["params"])
    p["trap"] = np.array([0.0, 0.7])
    p["recomb"] = np.array([0.01, 0.01])
    N, K = 2, 4
    nodes = oracle.num_nodes(N, K)
    D = N + 2
    dim = nodes * D * D
    L = np.zeros((dim, dim), dtype=complex)
    for k in range(dim):
        e = np.zeros(dim, dtype=complex)
        e[k] = 1.0
        L[:, k] = oracle.rhs(p, e.reshape(nodes, D, D)).reshape(-1)
    y0 = np.zeros((nodes, D, D), dtype=complex)
    y0[0, :N, :N] = w["rho0"]
    y0 = y0.reshape(-1)
    h, n = 1.0, 200
    x = h * L
    P = np.eye(dim) + x + x @ x / 2 + x @ x @ x / 6 + x @ x @ x @ x / 24
    y_poly = np.linalg.matrix_power(P, n) @ y0
    r = oracle.propagate(p, w["rho0"], h, n, n, want_state=True)
    y_rk4 = r["state"].reshape(-1)
    assert np.abs(y_rk4 - y_poly).max() < 1e-12
    y_exact = expm(L * h * n) @ y0
    err1 = np.abs(y_rk4 - y_exact).max()
    r2 = oracle.propagate(p, w["rho0"], h / 2, 2 * n, 2 * n, want_state=True)
    err2 = np.abs(r2["state"].reshape(-1) - y_exact).max()
    assert err1 < 1e-7
    assert 10.0 < err1 / err2 < 22.0
    # ground and RC entries never feed back into the site block (why the
    # trap and the radiative decay act like an anti-Hermitian part of H)
    idx = np.arange(dim).reshape(nodes, D, D)
    site_rows = idx[:, :N, :N].reshape(-1)
    outside = np.setdiff1d(np.arange(dim), site_rows)
    assert np.all(L[np.ix_(site_rows, outside)] == 0.0)


# ----------------------------------------------------------------------------
# Scaled hierarchy (the "scaled version of the HEOM" of the introduction):
# sigma~_n = sigma_n / S(n), S(n) = prod_j sqrt(n_j! s_j^{n_j}), s_j = |c_j|
# ----------------------------------------------------------------------------

def _scale_of_nodes(p, multi):
    """S(n) per node, from the multi-indices and s_j = |2 lambda kT - i lambda gamma| (rad^2/fs^2)."""
    N = int(p["N"])
    lam = np.broadcast_to(np.asarray(p["lam"], dtype=float), (N,)) * W
    gam = np.broadcast_to(np.asarray(p["gam"], dtype=float), (N,)) * W
    kT = KB * p["T"] * W
    s = np.hypot(2.0 * lam * kT, lam * gam)
    s = np.where(s > 0, s, 1.0)
    return np.array([math.prod(math.sqrt(math.factorial(int(k)) * s[j] ** int(k)) for j, k in enumerate(n))
                     for n in multi])


@pytest.mark.parametrize("term", [0, 1])
def test_scaled_generator_is_a_diagonal_similarity(term):
    """L~ = S^-1 L S node block by node block: every up weight sqrt((n_j+1) s_j)
    and down weight sqrt(n_j / s_j) is pinned against the unscaled generator."""
    w = workloads.dimer()
    p = dict(w["params"], trap=np.array([0.0, 0.7]), recomb=np.array([0.01, 0.01]), terminator=term,
             lam=np.array([35.0, 80.0]), gam=np.array([106.0, 50.0]), low_temp=1)
    N, K = 2, 4
    nodes = oracle.num_nodes(N, K)
    D = N + 2
    dim = nodes * D * D

    def generator(q):
        L = np.zeros((dim, dim), dtype=complex)
        for k in range(dim):
            e = np.zeros(dim, dtype=complex)
            e[k] = 1.0
            L[:, k] = oracle.rhs(q, e.reshape(nodes, D, D)).reshape(-1)
        return L

    L = generator(p)
    Ls = generator(dict(p, scaled=1))
    S = np.repeat(_scale_of_nodes(p, oracle.multi_indices(N, K)), D * D)
    assert S[0] == 1.0 and S.max() / S.min() > 10.0
    ref = L * S[None, :] / S[:, None]
    assert np.abs(Ls - ref).max() <= 1e-14 * np.abs(L).max()
    assert np.abs(Ls - L).max() > 1e-3 * np.abs(L).max()  # the rescaling did change the links


def test_scaled_propagation_gives_the_same_rho_and_rescaled_auxiliaries():
    N = 3
    H = workloads.fmo_like_hamiltonian(N, 1234)
    p = dict(N=N, K=3, H=H, lam=np.array([35.0, 20.0, 60.0]), gam=np.array([106.0, 80.0, 150.0]), T=150.0,
             trap=np.array([0.0, 0.0, 1.0]), recomb=np.full(N, 1e-3), terminator=1)
    rho0 = workloads.pure_state(N, 0)
    a = oracle.propagate(p, rho0, 1.0, 300, 50, want_state=True)
    b = oracle.propagate(dict(p, scaled=1), rho0, 1.0, 300, 50, want_state=True)
    for k in ("pops", "eta", "loss", "tmean"):
        assert np.abs(a[k] - b[k]).max() < 1e-13, k
    S = _scale_of_nodes(p, a["multi"])
    assert np.abs(b["state"] - a["state"] / S[:, None, None]).max() < 1e-13 * np.abs(a["state"] / S[:, None, None]).max()
    # the rescaled auxiliaries are of comparable size across levels
    lev = a["multi"].sum(axis=1)
    mag = lambda st, l: np.abs(st[lev == l]).max()
    spread_plain = max(mag(a["state"], l) for l in range(4)) / min(mag(a["state"], l) for l in range(4))
    spread_scaled = max(mag(b["state"], l) for l in range(4)) / min(mag(b["state"], l) for l in range(4))
    assert spread_scaled < spread_plain


# ----------------------------------------------------------------------------
# Physics: long-time state of the isolated dimer is close to Gibbs
# (Sec. "Trapping time for different temperatures": agreement above 100 K)
# ----------------------------------------------------------------------------

def test_isolated_dimer_relaxes_near_gibbs_state():
    w = workloads.dimer()
    p = dict(w["params"])
    p["K"] = 6
    r = oracle.propagate(p, w["rho0"], 1.0, 4000, 1000)
    Hr = p["H"].real
    beta = 1.0 / (KB * p["T"])
    ev, U = np.linalg.eigh(Hr)
    rho_th = U @ np.diag(np.exp(-beta * ev)) @ U.T
    rho_th /= np.trace(rho_th)
    # stationary
    assert np.abs(r["pops"][-1] - r["pops"][-2]).max() < 1e-5
    assert np.abs(r["pops"][-1] - np.diag(rho_th)).max() < 0.03


def test_depth_convergence_of_efficiency():
    """Truncation converges: the change of eta from depth K to K+1 shrinks."""
    w = workloads.fmo_trap()
    p = dict(w["params"])
    # three sites keep this quick: the first three of the FMO-like model
    H = p["H"][:3, :3]
    base = dict(N=3, H=H, lam=p["lam"][:3], gam=p["gam"][:3], T=300.0, trap=np.array([0.0, 0.0, 1.0]),
                recomb=np.full(3, 1e-3))
    etas = []
    for K in (1, 2, 3, 4, 5):
        r = oracle.propagate(dict(base, K=K), workloads.pure_state(3, 0), 2.0, 500, 500)
        etas.append(r["eta"][-1])
    d = np.abs(np.diff(etas))
    assert d[-1] < d[0]
    assert d[-1] < 1e-3


def test_fmo_table_fixture_is_hermitian():
    H = _load_table("fmo_table1.txt")
    assert H.shape == (7, 7)
    assert np.array_equal(H, H.T)
