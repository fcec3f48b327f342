"""Seeded synthetic inputs for the five benchmark workloads.

This module only draws numbers: it holds none of the method's arithmetic (no
unit conversion, no hierarchy, no propagation).  Both the CUDA path's tests and
benchmark and the oracle's tests take their inputs from here.

All values are in the paper's units: energies and couplings in cm^-1, rates in
ps^-1, temperatures in K, times in fs.  Site indices are 0-based, so the
paper's BChl_3 (the site next to the reaction centre, Sec. "Model") is index 2.

The shapes follow the paper's FMO model (Table 1: N = 7, site energies
12210-12630 cm^-1, couplings of tens of cm^-1; Sec. "Trapping time ...":
lambda = 35 cm^-1, gamma^-1 = 50 fs, i.e. gamma = 106 cm^-1, T = 300 K), with
seeded random Hamiltonians in place of the table's values.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1234


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def fmo_like_hamiltonian(N: int, seed: int) -> np.ndarray:
    """Real symmetric N x N: diagonal ~ U(12100, 12600), off-diagonal ~ N(0, 40)."""
    g = _rng(seed)
    eps = g.uniform(12100.0, 12600.0, size=N)
    J = g.normal(0.0, 40.0, size=(N, N))
    J = np.triu(J, 1)
    H = np.diag(eps) + J + J.T
    return H.astype(np.complex128)


def block_trimer_hamiltonian(blocks: int, block_size: int, seed: int) -> np.ndarray:
    """`blocks` FMO-like blocks; intra-block couplings N(0, 40), inter-block N(0, 5)."""
    g = _rng(seed)
    N = blocks * block_size
    eps = g.uniform(12100.0, 12600.0, size=N)
    H = np.diag(eps)
    for a in range(N):
        for b in range(a + 1, N):
            same = (a // block_size) == (b // block_size)
            v = g.normal(0.0, 40.0 if same else 5.0)
            H[a, b] = v
            H[b, a] = v
    return H.astype(np.complex128)


def pure_state(N: int, site: int) -> np.ndarray:
    rho = np.zeros((N, N), dtype=np.complex128)
    rho[site, site] = 1.0
    return rho


def _params(H, K, lam, gam, T, trap=None, recomb=None, terminator=0, add_reorg=0):
    N = H.shape[0]
    return {
        "N": int(N),
        "K": int(K),
        "H": np.asarray(H, dtype=np.complex128),
        "lam": np.full(N, float(lam)) if np.isscalar(lam) else np.asarray(lam, dtype=np.float64),
        "gam": np.full(N, float(gam)) if np.isscalar(gam) else np.asarray(gam, dtype=np.float64),
        "T": float(T),
        "trap": None if trap is None else np.asarray(trap, dtype=np.float64),
        "recomb": None if recomb is None else np.asarray(recomb, dtype=np.float64),
        "terminator": int(terminator),
        "add_reorg": int(add_reorg),
    }


def dimer() -> dict:
    """Dimer: energies 0 and 100 cm^-1, coupling 100 cm^-1, lambda 35, gamma 106,
    300 K, depth 4 (15 nodes), rho(0) = |0><0|, dt 1 fs, 1000 steps, no trap."""
    H = np.array([[0.0, 100.0], [100.0, 100.0]], dtype=np.complex128)
    return {"params": _params(H, 4, 35.0, 106.0, 300.0), "rho0": pure_state(2, 0), "dt": 1.0, "nsteps": 1000,
            "out_every": 1}


def fmo_trap(K: int = 6, seed: int = SEED_BASE, nsteps: int = 10000) -> dict:
    """FMO-like N = 7 with trap: trap 1 ps^-1 on index 2, recombination 1 ns^-1 on all
    sites, lambda 35, gamma 106, 300 K, depth 6 (1716 nodes), dt 1 fs, 10 ps."""
    N = 7
    H = fmo_like_hamiltonian(N, seed)
    trap = np.zeros(N)
    trap[2] = 1.0
    recomb = np.full(N, 1e-3)
    return {"params": _params(H, K, 35.0, 106.0, 300.0, trap, recomb), "rho0": pure_state(N, 0), "dt": 1.0,
            "nsteps": int(nsteps), "out_every": 10}


def batched_scan(count: int = 256, nsteps: int = 5000) -> list:
    """`count` seeded N = 7 trap models: lambda ~ U(2, 200), T ~ U(77, 300),
    depth ~ U{4..8}; the rest as fmo_trap; 5 ps each at 1 fs."""
    out = []
    for i in range(count):
        seed = SEED_BASE + i
        g = _rng(seed + 1_000_000)
        lam = g.uniform(2.0, 200.0)
        T = g.uniform(77.0, 300.0)
        K = int(g.integers(4, 9))
        w = fmo_trap(K=K, seed=seed, nsteps=nsteps)
        w["params"]["lam"] = np.full(7, lam)
        w["params"]["T"] = float(T)
        w["out_every"] = 10
        out.append(w)
    return out


def serving_trace(count: int = 2000, rate_per_s: float = 200.0, seed: int = SEED_BASE) -> list:
    """Poisson arrivals: returns dicts with arrival time (s), N ~ U{2..8},
    K ~ U{3..8}, FMO-like H, length ~ U(1, 20) ps at dt = 1 fs; trap 1 ps^-1 on
    index min(2, N-1), recombination 1 ns^-1 on all sites."""
    g = _rng(seed + 2_000_000)
    t = 0.0
    out = []
    for i in range(count):
        t += g.exponential(1.0 / rate_per_s)
        N = int(g.integers(2, 9))
        K = int(g.integers(3, 9))
        length_ps = g.uniform(1.0, 20.0)
        H = fmo_like_hamiltonian(N, SEED_BASE + 10_000 + i)
        trap = np.zeros(N)
        trap[min(2, N - 1)] = 1.0
        recomb = np.full(N, 1e-3)
        out.append({
            "arrival_s": t,
            "params": _params(H, K, 35.0, 106.0, 300.0, trap, recomb),
            "rho0": pure_state(N, 0),
            "dt": 1.0,
            "nsteps": int(round(length_ps * 1000.0)),
            "out_every": 100,
        })
    return out


def large_trimer(nsteps: int = 2000, seed: int = SEED_BASE) -> dict:
    """24 sites as three 8-site FMO-like blocks, lambda 35, gamma 106, 300 K,
    depth 4 (20475 nodes), no trap, rho(0) = |0><0|, dt 1 fs, 2 ps."""
    H = block_trimer_hamiltonian(3, 8, seed)
    return {"params": _params(H, 4, 35.0, 106.0, 300.0), "rho0": pure_state(24, 0), "dt": 1.0,
            "nsteps": int(nsteps), "out_every": 10}


def random_instance(N: int, K: int, seed: int, trap: bool = True, complex_h: bool = False,
                    terminator: int = 0) -> dict:
    """Small random model for parity tests: FMO-like H (optionally with an
    imaginary Hermitian part), per-site lambda, gamma, rates."""
    g = _rng(seed)
    H = fmo_like_hamiltonian(N, seed + 7)
    if complex_h:
        Ji = g.normal(0.0, 20.0, size=(N, N))
        Ji = np.triu(Ji, 1)
        H = H + 1j * (Ji - Ji.T)
    lam = g.uniform(10.0, 120.0, size=N)
    gam = g.uniform(40.0, 200.0, size=N)
    T = g.uniform(77.0, 300.0)
    tr = g.uniform(0.1, 2.0, size=N) * (g.uniform(size=N) < 0.5) if trap else None
    rc = np.full(N, 2e-3) if trap else None
    rho0 = pure_state(N, int(g.integers(0, N)))
    return {"params": _params(H, K, lam, gam, T, tr, rc, terminator), "rho0": rho0, "dt": 1.0, "nsteps": 50,
            "out_every": 5}
