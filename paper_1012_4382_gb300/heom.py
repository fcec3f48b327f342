"""ctypes binding of libheom (include/heom.h).

Argument marshalling only: every step of the propagation runs in the CUDA
kernels of libheom.so.  There is no CPU fallback; if the library is missing
or cannot load, :func:`lib` raises.

Parameters are passed as dicts with the keys used by
:mod:`paper_1012_4382_gb300.workloads` (N, K, H, lam, gam, T, trap, recomb,
terminator, add_reorg) in the paper's units (cm^-1, ps^-1, K, fs).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libheom.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ENONFINITE, EINTERNAL = 0, 1, 2, 3, 4, 5, 6, 7
FP64, FP32_MIXED = 0, 1
FLAG_LOW_TEMP = 1  # heom_params.flags: low-temperature correction
FLAG_SCALED = 2  # heom_params.flags: scaled hierarchy (auxiliaries divided by prod_j sqrt(n_j! s_j^n_j))
TERM_NONE, TERM_MARKOV = 0, 1
MAX_SITES = 24

_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class HeomError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libheom error %d: %s" % (code, msg))
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("H", _dp),
        ("lam", _dp),
        ("gam", _dp),
        ("T", ctypes.c_double),
        ("trap", _dp),
        ("recomb", _dp),
        ("precision", ctypes.c_int32),
        ("terminator", ctypes.c_int32),
        ("add_reorg", ctypes.c_int32),
        ("flags", ctypes.c_int32),
    ]


def lib() -> ctypes.CDLL:
    """Loads libheom.so (built by ``paper_1012_4382_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libheom.so is missing (%s); build it with python -m paper_1012_4382_gb300.build"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        sig = {
            "heom_num_nodes": [ctypes.c_int32, ctypes.c_int32, _i64p],
            "heom_build_index": [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p],
            "heom_check_node_tables": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)],
            "heom_set_allocator": [ALLOC_FN, FREE_FN, vp],
            "heom_create": [ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)],
            "heom_set_rho0": [vp, _dp],
            "heom_set_rho0_device": [vp, vp],
            "heom_propagate": [vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _dp, _dp, _dp],
            "heom_propagate_device": [vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, vp, vp],
            "heom_synchronize": [vp],
            "heom_efficiency": [vp, _dp, _dp],
            "heom_trapping_time": [vp, _dp, _i64p],
            "heom_set_stop": [vp, ctypes.c_double],
            "heom_get_rho": [vp, _dp],
            "heom_get_state": [vp, _dp, _dp],
            "heom_set_state": [vp, _dp, _dp],
            "heom_ctx_num_nodes": [vp, _i64p],
            "heom_set_launch": [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
            "heom_get_launch": [vp, _i32p, _i32p, _i32p, _i32p],
            "heom_autotune": [vp, ctypes.c_int64, _dp],
            "heom_batch_create": [ctypes.POINTER(_Params), ctypes.c_int32, vp, ctypes.POINTER(vp)],
            "heom_batch_count": [vp, _i32p],
            "heom_batch_set_rho0": [vp, _dp],
            "heom_batch_propagate": [vp, _dp, _i64p, ctypes.c_int64, _dp, _dp],
            "heom_batch_propagate_device": [vp, _dp, _i64p, ctypes.c_int64, vp, vp],
            "heom_batch_graph_create": [vp, _dp, _i64p, ctypes.c_int64, vp, vp, ctypes.POINTER(vp)],
            "heom_graph_launch": [vp],
            "heom_batch_synchronize": [vp],
            "heom_batch_efficiency": [vp, _dp, _dp],
            "heom_batch_trapping_time": [vp, _dp, _i64p],
            "heom_batch_set_stop": [vp, ctypes.c_double],
            "heom_batch_get_rho": [vp, ctypes.c_int32, _dp],
            "heom_batch_set_launch": [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
            "heom_batch_get_launch": [vp, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p],
            "heom_batch_autotune": [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)],
            "heom_node_magnitudes": [vp, _dp],
            "heom_filter_select": [ctypes.c_int32, ctypes.c_int32, _dp, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_uint8)],
            "heom_create_subset": [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_uint8), vp, ctypes.POINTER(vp)],
            "heom_batch_create_subset": [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.POINTER(ctypes.c_uint8)),
                                         ctypes.c_int32, vp, ctypes.POINTER(vp)],
            "heom_batch_num_nodes": [vp, ctypes.c_int32, _i64p],
            "heom_batch_node_magnitudes": [vp, ctypes.c_int32, _dp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.heom_destroy.argtypes = [vp]
        L.heom_destroy.restype = None
        L.heom_batch_destroy.argtypes = [vp]
        L.heom_batch_destroy.restype = None
        L.heom_graph_destroy.argtypes = [vp]
        L.heom_graph_destroy.restype = None
        L.heom_last_error.argtypes = []
        L.heom_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(code):
    if code != OK:
        raise HeomError(code, lib().heom_last_error().decode(errors="replace"))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return ctypes.cast(None, _dp)
    return a.ctypes.data_as(_dp)


def _cplx(m, N):
    m = np.asarray(m, dtype=np.complex128).reshape(N, N)
    return np.ascontiguousarray(m).view(np.float64).reshape(-1).copy()


def _uncplx(flat, shape):
    return np.ascontiguousarray(flat).view(np.complex128).reshape(shape)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


class _Keep:
    """Owns the arrays a ctypes heom_params points into."""

    def __init__(self, p, precision):
        N = int(p["N"])
        self.H = _cplx(p["H"], N)
        self.lam = _f64(np.broadcast_to(np.asarray(p["lam"], dtype=np.float64), (N,)))
        self.gam = _f64(np.broadcast_to(np.asarray(p["gam"], dtype=np.float64), (N,)))
        self.trap = None if p.get("trap") is None else _f64(p["trap"])
        self.recomb = None if p.get("recomb") is None else _f64(p["recomb"])
        for a in (self.trap, self.recomb):
            if a is not None and a.size != N:
                raise ValueError("rate arrays need N entries")
        self.c = _Params(N, int(p["K"]), _ptr(self.H), _ptr(self.lam), _ptr(self.gam), float(p["T"]),
                         _ptr(self.trap), _ptr(self.recomb), int(precision), int(p.get("terminator", 0)),
                         int(p.get("add_reorg", 0)),
                         (FLAG_LOW_TEMP if p.get("low_temp", 0) else 0) | (FLAG_SCALED if p.get("scaled", 0) else 0))


def _precision(precision):
    if precision in ("fp64", FP64):
        return FP64
    if precision in ("fp32", "fp32_mixed", FP32_MIXED):
        return FP32_MIXED
    raise ValueError("precision must be 'fp64' or 'fp32'")


def selftest_bounded_wait(limit_ms: float = 20.0):
    """heom_selftest_bounded_wait: returns (timed_out, waited_ms)."""
    L = lib()
    L.heom_selftest_bounded_wait.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_double)]
    L.heom_selftest_bounded_wait.restype = ctypes.c_int
    t, ms = ctypes.c_int32(), ctypes.c_double()
    _check(L.heom_selftest_bounded_wait(float(limit_ms), ctypes.byref(t), ctypes.byref(ms)))
    return bool(t.value), ms.value


def num_nodes(N: int, K: int) -> int:
    out = ctypes.c_int64(0)
    _check(lib().heom_num_nodes(int(N), int(K), ctypes.byref(out)))
    return int(out.value)


def build_index(N: int, K: int):
    """(multi, up, down) arrays of shape [nodes, N] in the library's node order."""
    M = num_nodes(N, K)
    multi = np.zeros((M, N), np.int32)
    up = np.zeros((M, N), np.int32)
    down = np.zeros((M, N), np.int32)
    p = lambda a: a.ctypes.data_as(_i32p)
    _check(lib().heom_build_index(int(N), int(K), p(multi), p(up), p(down)))
    return multi, up, down


def device_tables(N: int, K: int):
    """(up, dn, Mpad) in the device layout the kernels read, as host arrays
    [N][Mpad]: up = index of n + e_j or -1, dn = (n_j << 24) | index of n - e_j
    or -1."""
    multi, up, down = build_index(N, K)
    M = len(multi)
    Mpad = (M + 31) // 32 * 32
    u = np.full((N, Mpad), -1, np.int32)
    d = np.full((N, Mpad), -1, np.int32)
    u[:, :M] = up.T
    d[:, :M] = np.where(down.T >= 0, (multi.T.astype(np.int64) << 24) | down.T, -1).astype(np.int32)
    return u, d, Mpad


def check_node_tables(d_up, d_dn, M: int, Mpad: int, N: int) -> int:
    """Runs the device-side table check (heom_check_node_tables) on DEVICE
    int32 tensors [N][Mpad]; returns -1 when they pass, raises HeomError
    (EINVAL) naming the first offending node otherwise."""
    bad = ctypes.c_int64(-1)
    rc = lib().heom_check_node_tables(ctypes.c_void_p(d_up.data_ptr()), ctypes.c_void_p(d_dn.data_ptr()), int(M),
                                      int(Mpad), int(N), ctypes.byref(bad))
    if rc != OK:
        err = HeomError(rc, lib().heom_last_error().decode(errors="replace"))
        err.bad_node = bad.value
        raise err
    return bad.value


_hooks = None


def use_torch_allocator(enable: bool = True) -> None:
    """Routes libheom's device allocations through PyTorch's caching allocator
    (for contexts created afterwards)."""
    global _hooks
    L = lib()
    if not enable:
        _check(L.heom_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _hooks = None
        return
    import torch

    def _alloc(nbytes, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def _free(ptr, nbytes, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(L.heom_set_allocator(hooks[0], hooks[1], None))
    _hooks = hooks


def filter_select(N: int, K: int, node_max, delta: float) -> np.ndarray:
    """heom_filter_select: node flags (uint8, heom_build_index order) of the
    filtered hierarchy -- nodes with node_max >= delta, the root, closed downwards."""
    M = num_nodes(N, K)
    nm = _f64(node_max)
    if nm.size != M:
        raise ValueError("node_max needs one value per node (%d)" % M)
    keep = np.zeros(M, np.uint8)
    _check(lib().heom_filter_select(int(N), int(K), _ptr(nm), float(delta),
                                    keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return keep


class Context:
    """One hierarchy resident on the GPU (heom_create ... heom_destroy); with
    `keep` (flags per node of the full hierarchy, heom_build_index order) the
    filtered hierarchy over the kept nodes (heom_create_subset)."""

    def __init__(self, params: dict, precision="fp64", stream=None, keep=None):
        self._keep = _Keep(params, _precision(precision))
        self.N = int(params["N"])
        self.K = int(params["K"])
        self.precision = _precision(precision)
        self._h = ctypes.c_void_p()
        if keep is None:
            _check(lib().heom_create(ctypes.byref(self._keep.c), ctypes.c_void_p(_stream_handle(stream)),
                                     ctypes.byref(self._h)))
            self.nodes = num_nodes(self.N, self.K)
        else:
            self.keep = np.ascontiguousarray(np.asarray(keep, dtype=np.uint8))
            if self.keep.size != num_nodes(self.N, self.K):
                raise ValueError("keep needs one flag per node of the full hierarchy")
            _check(lib().heom_create_subset(ctypes.byref(self._keep.c),
                                            self.keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                            ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(self._h)))
            self.nodes = int(np.count_nonzero(self.keep))

    def node_magnitudes(self) -> np.ndarray:
        """heom_node_magnitudes: max_ab |sigma_n,ab| per node of the current state."""
        out = np.zeros(self.nodes)
        _check(lib().heom_node_magnitudes(self._h, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().heom_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_rho0(self, rho0):
        _check(lib().heom_set_rho0(self._h, _ptr(_cplx(rho0, self.N))))

    def set_rho0_device(self, d_rho0):
        """d_rho0: device tensor or pointer holding N*N complex128 (or 2*N*N float64)."""
        _check(lib().heom_set_rho0_device(self._h, ctypes.c_void_p(_dev_ptr(d_rho0))))

    def propagate(self, dt, nsteps, out_every=1):
        nout = int(nsteps) // int(out_every) + 1
        pops = np.zeros((nout, self.N))
        trace = np.zeros(nout)
        eta = np.zeros(nout)
        _check(lib().heom_propagate(self._h, float(dt), int(nsteps), int(out_every), _ptr(pops), _ptr(trace),
                                    _ptr(eta)))
        return {"pops": pops, "trace": trace, "eta": eta}

    def propagate_device(self, dt, nsteps, out_every, d_pops=None, d_eta_loss=None):
        _check(lib().heom_propagate_device(self._h, float(dt), int(nsteps), int(out_every),
                                           ctypes.c_void_p(_dev_ptr(d_pops)), ctypes.c_void_p(_dev_ptr(d_eta_loss))))

    def synchronize(self):
        _check(lib().heom_synchronize(self._h))

    def efficiency(self):
        e, l = ctypes.c_double(), ctypes.c_double()
        _check(lib().heom_efficiency(self._h, ctypes.byref(e), ctypes.byref(l)))
        return e.value, l.value

    def trapping_time(self):
        """(<t> in fs up to now, steps taken by the last propagate call)."""
        t, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().heom_trapping_time(self._h, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def set_stop(self, stop_trace):
        """Stop rule: end a propagate call once the site population drops below stop_trace (0: off)."""
        _check(lib().heom_set_stop(self._h, float(stop_trace)))

    def rho(self):
        out = np.zeros(2 * self.N * self.N)
        _check(lib().heom_get_rho(self._h, _ptr(out)))
        return _uncplx(out, (self.N, self.N))

    def state(self):
        out = np.zeros(2 * self.nodes * self.N * self.N)
        extra = np.zeros(2)
        _check(lib().heom_get_state(self._h, _ptr(out), _ptr(extra)))
        return _uncplx(out, (self.nodes, self.N, self.N)), extra

    def set_state(self, state, extra=(0.0, 0.0)):
        s = np.ascontiguousarray(np.asarray(state, dtype=np.complex128)).view(np.float64).reshape(-1).copy()
        _check(lib().heom_set_state(self._h, _ptr(s), _ptr(_f64(extra))))

    def set_launch(self, mode=-1, team_ctas=0, block_threads=0, node_threads=0):
        """heom_set_launch; in mode 3 (dataflow engine) team_ctas is the number of
        nodes each thread carries (1..6)."""
        _check(lib().heom_set_launch(self._h, int(mode), int(team_ctas), int(block_threads), int(node_threads)))

    def get_launch(self):
        v = [ctypes.c_int32() for _ in range(4)]
        _check(lib().heom_get_launch(self._h, *[ctypes.byref(x) for x in v]))
        return {"mode": v[0].value, "team_ctas": v[1].value, "block_threads": v[2].value,
                "node_threads": v[3].value}

    def autotune(self, trial_steps=200):
        us = ctypes.c_double()
        _check(lib().heom_autotune(self._h, int(trial_steps), ctypes.byref(us)))
        return us.value


class Batch:
    """Many independent hierarchies propagated in persistent launches."""

    def __init__(self, params_list, precision="fp32", stream=None, keep=None):
        """keep: None, or per instance None (full hierarchy) or node flags over its
        full hierarchy (heom_batch_create_subset)."""
        prec = _precision(precision)
        self._keeps = [_Keep(p, prec) for p in params_list]
        arr = (_Params * len(self._keeps))(*[k.c for k in self._keeps])
        self._arr = arr
        self.Ns = [int(p["N"]) for p in params_list]
        self.count = len(params_list)
        self._h = ctypes.c_void_p()
        if keep is None:
            _check(lib().heom_batch_create(arr, self.count, ctypes.c_void_p(_stream_handle(stream)),
                                           ctypes.byref(self._h)))
        else:
            self._flags = [None if k is None else np.ascontiguousarray(np.asarray(k, dtype=np.uint8)) for k in keep]
            ptrs = (ctypes.POINTER(ctypes.c_uint8) * self.count)(
                *[ctypes.cast(None, ctypes.POINTER(ctypes.c_uint8)) if f is None
                  else f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) for f in self._flags])
            self._ptrs = ptrs
            _check(lib().heom_batch_create_subset(arr, ptrs, self.count, ctypes.c_void_p(_stream_handle(stream)),
                                                  ctypes.byref(self._h)))

    def num_nodes(self, i) -> int:
        out = ctypes.c_int64()
        _check(lib().heom_batch_num_nodes(self._h, int(i), ctypes.byref(out)))
        return int(out.value)

    def node_magnitudes(self, i) -> np.ndarray:
        """heom_batch_node_magnitudes: max_ab |sigma_n,ab| per node of instance i."""
        out = np.zeros(self.num_nodes(i))
        _check(lib().heom_batch_node_magnitudes(self._h, int(i), _ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().heom_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_rho0(self, rho_list):
        flat = np.concatenate([_cplx(r, N) for r, N in zip(rho_list, self.Ns)])
        _check(lib().heom_batch_set_rho0(self._h, _ptr(flat)))

    def _steps(self, dt, nsteps):
        dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.count,)))
        ns = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int64), (self.count,)))
        return dt, ns

    def propagate(self, dt, nsteps, out_every=1):
        dt, ns = self._steps(dt, nsteps)
        nout = ns // int(out_every) + 1
        pops = np.zeros(int(np.sum(nout * np.asarray(self.Ns))))
        eta = np.zeros(int(np.sum(nout)))
        _check(lib().heom_batch_propagate(self._h, _ptr(dt), ns.ctypes.data_as(_i64p), int(out_every), _ptr(pops),
                                          _ptr(eta)))
        out, po, eo = [], 0, 0
        for i in range(self.count):
            n = int(nout[i])
            out.append({"pops": pops[po:po + n * self.Ns[i]].reshape(n, self.Ns[i]), "eta": eta[eo:eo + n]})
            po += n * self.Ns[i]
            eo += n
        return out

    def propagate_device(self, dt, nsteps, out_every, d_pops=None, d_eta_loss=None):
        dt, ns = self._steps(dt, nsteps)
        self._last = (dt, ns)
        _check(lib().heom_batch_propagate_device(self._h, _ptr(dt), ns.ctypes.data_as(_i64p), int(out_every),
                                                 ctypes.c_void_p(_dev_ptr(d_pops)),
                                                 ctypes.c_void_p(_dev_ptr(d_eta_loss))))

    def graph(self, dt, nsteps, out_every, d_pops=None, d_eta_loss=None):
        """Captures one propagate_device call as a CUDA graph (see Graph)."""
        dt, ns = self._steps(dt, nsteps)
        h = ctypes.c_void_p()
        _check(lib().heom_batch_graph_create(self._h, _ptr(dt), ns.ctypes.data_as(_i64p), int(out_every),
                                             ctypes.c_void_p(_dev_ptr(d_pops)), ctypes.c_void_p(_dev_ptr(d_eta_loss)),
                                             ctypes.byref(h)))
        return Graph(h, self)

    def synchronize(self):
        _check(lib().heom_batch_synchronize(self._h))

    def efficiency(self):
        e = np.zeros(self.count)
        l = np.zeros(self.count)
        _check(lib().heom_batch_efficiency(self._h, _ptr(e), _ptr(l)))
        return e, l

    def trapping_time(self):
        t = np.zeros(self.count)
        n = np.zeros(self.count, dtype=np.int64)
        _check(lib().heom_batch_trapping_time(self._h, _ptr(t), n.ctypes.data_as(_i64p)))
        return t, n

    def set_stop(self, stop_trace):
        _check(lib().heom_batch_set_stop(self._h, float(stop_trace)))

    def rho(self, i):
        out = np.zeros(2 * self.Ns[i] ** 2)
        _check(lib().heom_batch_get_rho(self._h, int(i), _ptr(out)))
        return _uncplx(out, (self.Ns[i], self.Ns[i]))

    def set_launch(self, mode=-1, team_ctas=0, block_threads=0, node_threads=0):
        _check(lib().heom_batch_set_launch(self._h, int(mode), int(team_ctas), int(block_threads),
                                           int(node_threads)))

    def autotune(self, trial_steps=20):
        """Times the candidate launch shapes on the whole batch and keeps the
        fastest (the state is restored); returns its time in ms."""
        ms = ctypes.c_double()
        _check(lib().heom_batch_autotune(self._h, int(trial_steps), ctypes.byref(ms)))
        return ms.value

    def get_launch(self, N):
        """Launch shape of the instances with N sites."""
        v = [ctypes.c_int32() for _ in range(4)]
        _check(lib().heom_batch_get_launch(self._h, int(N), *[ctypes.byref(x) for x in v]))
        return {"mode": v[0].value, "team_ctas": v[1].value, "block_threads": v[2].value,
                "node_threads": v[3].value}


class Graph:
    """A captured batch propagation (heom_batch_graph_create): each launch()
    runs the same persistent launch again on the batch's stream."""

    def __init__(self, h, batch):
        self._h = h
        self._batch = batch  # the batch must outlive the graph

    def launch(self):
        _check(lib().heom_graph_launch(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().heom_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
