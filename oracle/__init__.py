"""Python access to the FP64 CPU oracle (``oracle/heom_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA path of the
package never imports this module.

The oracle integrates the ME-HEOM hierarchy of Kreisbeck et al.
(arXiv:1012.4382, App. A2, Eqs. labsevena and lab8) with classic RK4 (App. B)
on the (N+2)-dimensional space of sites, ground state and reaction centre,
with trapping and radiative decay in Lindblad form (App. A1, Eqs. lab2, lab3)
and eta = <RC|rho|RC> (Eq. eta).  See the header of heom_oracle.c for the
readings of the paper it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heom_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


_FLAGS = ["-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc: -O3, OpenMP over nodes.  ISO C mode
    (-std=c11) keeps floating-point contraction off, so the optimisation
    level changes no result; no -march=native, so the x86 and Arm builds
    compute the same numbers."""
    stamp = _LIB + ".flags"
    flags_changed = not os.path.exists(stamp) or open(stamp).read() != " ".join(_FLAGS)
    if force or flags_changed or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc"] + _FLAGS + [_SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(" ".join(_FLAGS))
    from . import redfield  # the secular Redfield comparison model, same flags
    redfield.build()
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("H", ctypes.POINTER(ctypes.c_double)),
        ("lam", ctypes.POINTER(ctypes.c_double)),
        ("gam", ctypes.POINTER(ctypes.c_double)),
        ("T", ctypes.c_double),
        ("trap", ctypes.POINTER(ctypes.c_double)),
        ("recomb", ctypes.POINTER(ctypes.c_double)),
        ("terminator", ctypes.c_int32),
        ("add_reorg", ctypes.c_int32),
        ("low_temp", ctypes.c_int32),
        ("scaled", ctypes.c_int32),
        ("keep", ctypes.POINTER(ctypes.c_ubyte)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_num_nodes.restype = ctypes.c_longlong
            lib.oracle_num_nodes.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_multi_indices.restype = ctypes.c_int
            lib.oracle_multi_indices.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.oracle_rhs.restype = ctypes.c_int
            lib.oracle_rhs.argtypes = [ctypes.POINTER(_Params), dp, dp]
            lib.oracle_propagate.restype = ctypes.c_int
            lib.oracle_propagate.argtypes = [ctypes.POINTER(_Params), dp, ctypes.c_double, ctypes.c_longlong,
                                             ctypes.c_longlong, dp, dp, dp, dp, dp, dp]
            lib.oracle_propagate_ex.restype = ctypes.c_int
            lib.oracle_propagate_ex.argtypes = [ctypes.POINTER(_Params), dp, ctypes.c_double, ctypes.c_longlong,
                                                ctypes.c_longlong, ctypes.c_double, dp, dp, dp, dp, dp, dp, dp,
                                                ctypes.POINTER(ctypes.c_longlong)]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _dptr(a):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctypes.c_double))
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and out.size != n:
        raise ValueError("expected %d values, got %d" % (n, out.size))
    return out


def _cplx_interleaved(m, N):
    m = np.asarray(m, dtype=np.complex128).reshape(N, N)
    return np.ascontiguousarray(m).view(np.float64).reshape(-1).copy()


class _Keep:
    """Holds the numpy buffers a ctypes parameter block points into."""

    def __init__(self, p):
        N = int(p["N"])
        self.H = _cplx_interleaved(p["H"], N)
        self.lam = _f64(np.broadcast_to(np.asarray(p["lam"], dtype=np.float64), (N,)), N)
        self.gam = _f64(np.broadcast_to(np.asarray(p["gam"], dtype=np.float64), (N,)), N)
        self.trap = _f64(p.get("trap"), N)
        self.recomb = _f64(p.get("recomb"), N)
        # keep: optional boolean flags per node in the order of multi_indices(N, K) (the filtered hierarchy)
        self.keep = None
        if p.get("keep") is not None:
            self.keep = np.ascontiguousarray(np.asarray(p["keep"], dtype=np.uint8))
            if self.keep.size != num_nodes(N, int(p["K"])):
                raise ValueError("keep needs one flag per node")
        keep_ptr = (self.keep.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)) if self.keep is not None
                    else ctypes.cast(None, ctypes.POINTER(ctypes.c_ubyte)))
        self.c = _Params(N, int(p["K"]), _dptr(self.H), _dptr(self.lam), _dptr(self.gam), float(p["T"]),
                         _dptr(self.trap), _dptr(self.recomb), int(p.get("terminator", 0)),
                         int(p.get("add_reorg", 0)), int(p.get("low_temp", 0)), int(p.get("scaled", 0)), keep_ptr)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def num_nodes(N: int, K: int) -> int:
    return int(_load().oracle_num_nodes(int(N), int(K)))


def multi_indices(N: int, K: int) -> np.ndarray:
    n = num_nodes(N, K)
    out = np.zeros((n, N), dtype=np.int32)
    if _load().oracle_multi_indices(int(N), int(K), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))) != 0:
        raise RuntimeError("oracle_multi_indices failed")
    return out


def rhs(params: dict, state: np.ndarray) -> np.ndarray:
    """One application of the right-hand side to a full state.

    ``state`` has shape (nodes, N+2, N+2) complex, node order of
    :func:`multi_indices`, basis sites then |0> then |RC>.
    """
    keep = _Keep(params)
    N = int(params["N"])
    s = np.ascontiguousarray(np.asarray(state, dtype=np.complex128))
    if s.shape != (num_nodes(N, int(params["K"])), N + 2, N + 2):
        raise ValueError("bad state shape %r" % (s.shape,))
    out = np.zeros_like(s)
    rc = _load().oracle_rhs(ctypes.byref(keep.c), _dptr(s.view(np.float64)), _dptr(out.view(np.float64)))
    if rc != 0:
        raise RuntimeError("oracle_rhs failed")
    return out


def propagate(params: dict, rho0, dt_fs: float, nsteps: int, out_every: int = 1, want_state: bool = False,
              stop_trace: float = 0.0) -> dict:
    """Classic RK4 propagation; see oracle_propagate_ex in heom_oracle.c.

    ``params`` keys: N, K, H (N x N complex, cm^-1), lam, gam (cm^-1, scalar or
    per site), T (K), trap, recomb (ps^-1 per site, optional), terminator
    (0/1), add_reorg (0/1), low_temp (0/1: low-temperature correction),
    scaled (0/1: rescaled auxiliaries; the state then holds sigma~_n), keep (optional
    flags per node in the order of :func:`multi_indices`: nodes flagged 0 are removed).
    Returns a dict with pops [nout, N], trace [nout], eta [nout], loss [nout],
    tmean [nout] (trapping time <t> up to each row, fs), steps_done,
    rho [N, N] complex, and with ``want_state`` the full final state
    [nodes, N+2, N+2] plus the node multi-indices.  ``stop_trace`` > 0 ends
    the run after the first step whose site population is below it (rows
    after the stop are NaN).
    """
    keep = _Keep(params)
    N, K = int(params["N"]), int(params["K"])
    nout = int(nsteps) // int(out_every) + 1
    pops = np.zeros((nout, N))
    trace = np.zeros(nout)
    eta = np.zeros(nout)
    loss = np.zeros(nout)
    tmean = np.zeros(nout)
    done = ctypes.c_longlong(0)
    rho = np.zeros((N, N), dtype=np.complex128)
    r0 = _cplx_interleaved(rho0, N)
    state = None
    if want_state:
        state = np.zeros((num_nodes(N, K), N + 2, N + 2), dtype=np.complex128)
    rc = _load().oracle_propagate_ex(ctypes.byref(keep.c), _dptr(r0), float(dt_fs), int(nsteps), int(out_every),
                                     float(stop_trace), _dptr(pops), _dptr(trace), _dptr(eta), _dptr(loss),
                                     _dptr(tmean), _dptr(rho.view(np.float64)),
                                     _dptr(state.view(np.float64)) if state is not None else _dptr(None),
                                     ctypes.byref(done))
    if rc != 0:
        raise RuntimeError("oracle_propagate failed (bad input or out of memory)")
    out = {"pops": pops, "trace": trace, "eta": eta, "loss": loss, "tmean": tmean, "steps_done": done.value,
           "rho": rho}
    if want_state:
        out["state"] = state
        out["multi"] = multi_indices(N, K)
    return out
