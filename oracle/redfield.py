"""Python access to the secular Redfield comparison model (``redfield.c``).

TEST AND COMPARISON INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the
model the paper compares its HEOM with (App. A1, "Secular Redfield
approximation"; Born-Markov and secular approximations, rates from the
Drude-Lorentz spectral density and the Bose function, Lamb shift dropped),
propagated on the CPU with classic RK4.  Parameters are the dicts of
:mod:`oracle` (N, H, lam, gam, T, trap, recomb, add_reorg).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "redfield.c")
_LIB = os.path.join(_HERE, "libredfield.so")
_FLAGS = ["-O3", "-std=c11", "-fPIC", "-shared"]
_lock = threading.Lock()
_lib = None

BOSE, HIGH_T = 0, 1  # bath_form: the paper's Bose-Einstein rates; the HEOM's high-temperature bath


def build(force: bool = False) -> str:
    """Compiles the model with gcc (ISO C: no floating-point contraction)."""
    stamp = _LIB + ".flags"
    changed = not os.path.exists(stamp) or open(stamp).read() != " ".join(_FLAGS)
    if force or changed or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc"] + _FLAGS + [_SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(" ".join(_FLAGS))
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("H", ctypes.POINTER(ctypes.c_double)),
                ("lam", ctypes.POINTER(ctypes.c_double)), ("gam", ctypes.POINTER(ctypes.c_double)),
                ("T", ctypes.c_double), ("trap", ctypes.POINTER(ctypes.c_double)),
                ("recomb", ctypes.POINTER(ctypes.c_double)), ("add_reorg", ctypes.c_int),
                ("bath_form", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.redfield_spectrum.argtypes = [ctypes.POINTER(_Params), dp, dp]
            L.redfield_rates.argtypes = [ctypes.POINTER(_Params), dp, dp]
            L.redfield_propagate.argtypes = [ctypes.POINTER(_Params), dp, ctypes.c_double, ctypes.c_longlong,
                                             ctypes.c_longlong, dp, dp, dp, dp]
            for f in (L.redfield_spectrum, L.redfield_rates, L.redfield_propagate):
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctypes.c_double))
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Keep:
    def __init__(self, p, bath_form):
        N = int(p["N"])
        H = np.asarray(p["H"], dtype=np.complex128).reshape(N, N)
        self.H = np.ascontiguousarray(H).view(np.float64).reshape(-1).copy()
        self.lam = np.ascontiguousarray(np.broadcast_to(np.asarray(p["lam"], float), (N,)))
        self.gam = np.ascontiguousarray(np.broadcast_to(np.asarray(p["gam"], float), (N,)))
        self.trap = None if p.get("trap") is None else np.ascontiguousarray(np.asarray(p["trap"], float))
        self.recomb = None if p.get("recomb") is None else np.ascontiguousarray(np.asarray(p["recomb"], float))
        self.c = _Params(N, _dp(self.H), _dp(self.lam), _dp(self.gam), float(p["T"]), _dp(self.trap),
                         _dp(self.recomb), int(p.get("add_reorg", 0)), int(bath_form))


def spectrum(params: dict, bath_form: int = BOSE):
    """Exciton energies (rad/fs, ascending) and C[m, M] = c_m(M) (site m of exciton M)."""
    k = _Keep(params, bath_form)
    N = int(params["N"])
    E = np.zeros(N)
    V = np.zeros(2 * N * N)
    if _load().redfield_spectrum(ctypes.byref(k.c), _dp(E), _dp(V)) != 0:
        raise RuntimeError("redfield_spectrum failed")
    return E, V.view(np.complex128).reshape(N, N)


def rates(params: dict, bath_form: int = BOSE):
    """W[M, K]: rate (1/fs) of the jump K -> M in the exciton basis; gamma_m(0) per site."""
    k = _Keep(params, bath_form)
    N = int(params["N"])
    W = np.zeros(N * N)
    d = np.zeros(N)
    if _load().redfield_rates(ctypes.byref(k.c), _dp(W), _dp(d)) != 0:
        raise RuntimeError("redfield_rates failed")
    return W.reshape(N, N), d


def propagate(params: dict, rho0, dt_fs: float, nsteps: int, out_every: int = 1, bath_form: int = BOSE) -> dict:
    """Secular Redfield propagation from rho(0) (site basis); rows every out_every steps."""
    k = _Keep(params, bath_form)
    N = int(params["N"])
    nout = int(nsteps) // int(out_every) + 1
    pops, trace, eta, loss = np.zeros((nout, N)), np.zeros(nout), np.zeros(nout), np.zeros(nout)
    r0 = np.ascontiguousarray(np.asarray(rho0, dtype=np.complex128).reshape(N, N)).view(np.float64).reshape(-1).copy()
    rc = _load().redfield_propagate(ctypes.byref(k.c), _dp(r0), float(dt_fs), int(nsteps), int(out_every), _dp(pops),
                                    _dp(trace), _dp(eta), _dp(loss))
    if rc != 0:
        raise RuntimeError("redfield_propagate failed (%d)" % rc)
    return {"pops": pops, "trace": trace, "eta": eta, "loss": loss}
