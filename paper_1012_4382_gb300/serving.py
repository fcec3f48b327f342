"""Serving loop over libheom's continuous-batching server (heom_server_* in
include/heom.h): replays a trace of timed requests, submits each at its
arrival time, keeps calling heom_server_progress, and reports throughput and
latency percentiles.  Argument marshalling and bookkeeping only: admission,
slot management and the propagation itself run in libheom.
"""
from __future__ import annotations

import ctypes
import os
import time

# Streams of concurrent launches must not share hardware work queues (the
# default is 8 queues per process); this takes effect when the CUDA context
# is created after this import.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

from . import heom

QUEUED, RUNNING, DONE, CANCELLED, FAILED = 0, 1, 2, 3, 4

_sig_done = False


def _lib():
    global _sig_done
    L = heom.lib()
    if not _sig_done:
        vp = ctypes.c_void_p
        i64 = ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "heom_server_create": [ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(vp)],
            "heom_server_submit": [vp, ctypes.POINTER(heom._Params), dp, ctypes.c_double, i64, i64,
                                   ctypes.POINTER(i64)],
            "heom_server_progress": [vp, ctypes.POINTER(ctypes.c_int32)],
            "heom_server_status": [vp, i64, ctypes.POINTER(ctypes.c_int32)],
            "heom_server_result": [vp, i64, dp, dp, dp, dp],
            "heom_server_release": [vp, i64],
            "heom_server_cancel": [vp, i64],
            "heom_server_stats": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.heom_server_destroy.argtypes = [vp]
        L.heom_server_destroy.restype = None
        _sig_done = True
    return L


class Server:
    """Continuous-batching server: a device-memory budget, a pinned host
    buffer for results and `streams` CUDA streams (concurrent launches)."""

    def __init__(self, device_bytes: int = 4 << 30, host_bytes: int = 64 << 20, streams: int = 32):
        self._h = ctypes.c_void_p()
        heom._check(_lib().heom_server_create(int(device_bytes), int(host_bytes), int(streams),
                                              ctypes.byref(self._h)))
        self._info = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib().heom_server_destroy(self._h)
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

    def submit(self, params, rho0, dt, nsteps, out_every, precision="fp32") -> int:
        keep = heom._Keep(params, heom._precision(precision))
        N = int(params["N"])
        r0 = heom._cplx(rho0, N)
        rid = ctypes.c_int64()
        heom._check(_lib().heom_server_submit(self._h, ctypes.byref(keep.c), heom._ptr(r0), float(dt), int(nsteps),
                                              int(out_every), ctypes.byref(rid)))
        self._info[rid.value] = (N, int(nsteps) // int(out_every) + 1)
        return rid.value

    def progress(self) -> int:
        n = ctypes.c_int32()
        heom._check(_lib().heom_server_progress(self._h, ctypes.byref(n)))
        return n.value

    def status(self, rid) -> int:
        st = ctypes.c_int32()
        heom._check(_lib().heom_server_status(self._h, int(rid), ctypes.byref(st)))
        return st.value

    def result(self, rid) -> dict:
        N, nout = self._info[rid]
        pops = np.zeros((nout, N))
        eta = np.zeros(nout)
        loss = np.zeros(nout)
        times = np.zeros(2)
        heom._check(_lib().heom_server_result(self._h, int(rid), heom._ptr(pops), heom._ptr(eta), heom._ptr(loss),
                                              heom._ptr(times)))
        return {"pops": pops, "eta": eta, "loss": loss, "wait_s": times[0], "done_s": times[1]}

    def release(self, rid):
        heom._check(_lib().heom_server_release(self._h, int(rid)))
        self._info.pop(rid, None)

    def cancel(self, rid):
        heom._check(_lib().heom_server_cancel(self._h, int(rid)))

    def stats(self) -> dict:
        q, r, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        heom._check(_lib().heom_server_stats(self._h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
        return {"queued": q.value, "running": r.value, "bytes_in_use": b.value}


def run_trace(trace, precision="fp32", device_bytes=8 << 30, streams=32, keep_results=False, time_limit_s=None):
    """Replays `trace` (dicts with arrival_s, params, rho0, dt, nsteps,
    out_every) against a fresh server in real time.  Latency of a request =
    time from its scheduled arrival to the progress call that saw it finish."""
    srv = Server(device_bytes, 256 << 20, streams)
    order = sorted(range(len(trace)), key=lambda i: trace[i]["arrival_s"])
    t0 = time.perf_counter()
    nxt = 0
    live = {}
    lat, work, results = [], 0.0, {}
    done_count = 0
    max_running = 0
    while nxt < len(order) or live:
        now = time.perf_counter() - t0
        if time_limit_s is not None and now > time_limit_s:
            break
        while nxt < len(order) and trace[order[nxt]]["arrival_s"] <= now:
            w = trace[order[nxt]]
            rid = srv.submit(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], precision)
            live[rid] = order[nxt]
            nxt += 1
        if srv.progress():
            tnow = time.perf_counter() - t0
            for rid in list(live):
                st = srv.status(rid)
                if st in (DONE, FAILED):
                    i = live.pop(rid)
                    w = trace[i]
                    if st == DONE:
                        lat.append(tnow - w["arrival_s"])
                        M = heom.num_nodes(w["params"]["N"], w["params"]["K"])
                        work += M * 4.0 * w["nsteps"]
                        done_count += 1
                        if keep_results:
                            results[i] = srv.result(rid)
                    srv.release(rid)
        max_running = max(max_running, srv.stats()["running"])
        if nxt < len(order):
            wait = trace[order[nxt]]["arrival_s"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 2e-4))
        else:
            time.sleep(5e-5)
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array(lat) if lat else np.array([np.nan])
    span = trace[order[-1]]["arrival_s"] - trace[order[0]]["arrival_s"] if len(order) > 1 else 0.0
    out = {
        "requests": len(trace),
        "completed": done_count,
        "offered_req_per_s": (len(trace) - 1) / span if span > 0 else None,
        "achieved_req_per_s": done_count / wall,
        "node_rhs_per_s": work / wall,
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(np.mean(lat)),
        "wall_s": wall,
        "max_concurrent": max_running,
        "streams": streams,
        "device_bytes": device_bytes,
    }
    if keep_results:
        out["results"] = results
    return out


# ------------------------------------------------------------ JSON-configured runs
#
# python -m paper_1012_4382_gb300.serving --config run.json
#
# run.json:
#   {"precision": "fp32" | "fp64",          (default fp32)
#    "device_bytes": 8589934592, "streams": 32,
#    "trace": {"rate_per_s": 200, "count": 2000, "seed": 1234}      a seeded synthetic trace
#             or "requests.jsonl"                                    one request per line (below),
#    "results": "out.jsonl"}                 optional: per-request populations and eta
#
# A request line: {"arrival_s": 0.01, "N": 3, "K": 4, "H": [[...]] (N x N, cm^-1; real, or
# [re, im] pairs), "lam": [...], "gam": [...] (cm^-1, per site or one value), "T": 300,
# "trap": [...], "recomb": [...] (ps^-1, optional), "terminator": 0, "low_temp": 0,
# "initial_site": 0, "dt": 1.0, "nsteps": 1000, "out_every": 100}.

_PARAM_KEYS = ("N", "K", "lam", "gam", "T", "trap", "recomb", "terminator", "add_reorg", "low_temp", "scaled")


def request_from_json(d: dict) -> dict:
    """One trace entry (the form run_trace takes) from a request line."""
    N = int(d["N"])
    H = np.asarray(d["H"], dtype=np.float64)
    if H.shape == (N, N, 2):
        H = H[..., 0] + 1j * H[..., 1]
    elif H.shape != (N, N):
        raise ValueError("H must be N x N (real) or N x N x 2 ([re, im]), got %r" % (H.shape,))
    params = {"H": np.asarray(H, dtype=np.complex128)}
    for k in _PARAM_KEYS:
        if k in d:
            v = d[k]
            params[k] = np.asarray(v, dtype=np.float64) if isinstance(v, list) else v
    for k in ("lam", "gam"):
        if np.ndim(params[k]) == 0:
            params[k] = np.full(N, float(params[k]))
    s = int(d.get("initial_site", 0))
    if not 0 <= s < N:
        raise ValueError("initial_site %d outside 0..%d" % (s, N - 1))
    rho0 = np.zeros((N, N), dtype=np.complex128)
    rho0[s, s] = 1.0
    return {"arrival_s": float(d.get("arrival_s", 0.0)), "params": params, "rho0": rho0,
            "dt": float(d.get("dt", 1.0)), "nsteps": int(d["nsteps"]), "out_every": int(d.get("out_every", d["nsteps"]))}


def load_trace(cfg: dict, base_dir: str = ".") -> list:
    """The request list a run configuration names: a seeded synthetic trace
    (workloads.serving_trace) or a file of request lines."""
    tr = cfg.get("trace", {"rate_per_s": 200.0, "count": 2000})
    if isinstance(tr, dict):
        from . import workloads
        kw = {"count": int(tr.get("count", 2000)), "rate_per_s": float(tr.get("rate_per_s", 200.0))}
        if "seed" in tr:
            kw["seed"] = int(tr["seed"])
        return workloads.serving_trace(**kw)
    path = tr if os.path.isabs(tr) else os.path.join(base_dir, tr)
    out = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line:
                import json
                out.append(request_from_json(json.loads(line)))
    return out


def main(argv=None) -> int:
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Replay a request trace against the continuous-batching server.")
    ap.add_argument("--config", required=True, help="JSON run configuration (see the comment above main)")
    a = ap.parse_args(argv)
    with open(a.config) as f:
        cfg = json.load(f)
    trace = load_trace(cfg, os.path.dirname(os.path.abspath(a.config)))
    res_path = cfg.get("results")
    out = run_trace(trace, precision=cfg.get("precision", "fp32"), device_bytes=int(cfg.get("device_bytes", 8 << 30)),
                    streams=int(cfg.get("streams", 32)), keep_results=bool(res_path))
    results = out.pop("results", None)
    if res_path:
        with open(res_path, "w") as f:
            for i in sorted(results):
                r = results[i]
                f.write(json.dumps({"request": i, "pops": r["pops"].tolist(), "eta": r["eta"].tolist(),
                                    "loss": r["loss"].tolist()}) + "\n")
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
