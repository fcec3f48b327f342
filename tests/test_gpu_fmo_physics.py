"""The paper's FMO results for the trapping time (Sec. "Trapping time for
different reorganization energies", Eq. trappingtime, lower panel of Fig.
"reorg") from the CUDA path: the Table-1 Hamiltonian, trapping from BChl 3
and 4 at 1/(2.5 ps), radiative decay at 1/(250 ps), 300 K, 1/gamma = 166 fs,
depth 8 with the low-temperature correction (reading R6), each run until the
site population is below 1e-5 (the paper's t_max).  The text prints the
optimal reorganisation energy and trapping time for the two pathways
(fixture tests/golden/fig_reorg_optima.txt); the minimum over a grid of
lambda must sit at the printed lambda_opt, and <t> there must be within
0.3 ps of the printed value (the depth and the reading of the quantum
correction move it by about 0.1 ps).  The grid also shows the decrease of
<t> with lambda below 50 cm^-1 that the text describes."""
import math
import os

import numpy as np
import pytest

from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LAMBDAS = (20.0, 35.0, 55.0, 85.0, 150.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def _trapping_time_ps(lam, start):
    H = np.array(_load("fmo_table1.txt"))
    N = 7
    gam = 1.0 / (166.0 * 2.0 * math.pi * 2.99792458e-5)  # 1/(166 fs) in cm^-1
    trap = np.zeros(N)
    trap[2] = trap[3] = 1.0 / 2.5
    p = dict(N=N, K=8, H=H.astype(complex), lam=np.full(N, lam), gam=np.full(N, gam), T=300.0, trap=trap,
             recomb=np.full(N, 1.0 / 250.0), low_temp=1)
    rho0 = np.zeros((N, N), complex)
    rho0[start, start] = 1.0
    with heom.Context(p, "fp32") as c:
        c.set_stop(1e-5)
        c.set_rho0(rho0)
        c.propagate(1.0, 150000, 150000)
        t_fs, steps = c.trapping_time()
        eta, _ = c.efficiency()
    assert steps < 150000  # t_max reached
    assert 0.95 < eta < 1.0
    return t_fs / 1000.0


@pytest.mark.parametrize("row", _load("fig_reorg_optima.txt"), ids=lambda r: "site%d" % r[0])
def test_optimal_reorganisation_energy_and_trapping_time(row):
    site, lam_opt, t_opt = int(row[0]), row[1], row[2]
    t = {lam: _trapping_time_ps(lam, site - 1) for lam in LAMBDAS}
    best = min(t, key=t.get)
    assert best == lam_opt, t
    assert abs(t[best] - t_opt) < 0.3, t
    assert t[20.0] > t[35.0] > t[55.0]  # below 50 cm^-1 the bath assists the transfer
