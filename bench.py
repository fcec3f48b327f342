"""Benchmark of the HEOM RK4 hot path on one or more GB300 GPUs.

One "step" is one complete solve of the FMO-like N = 7 trap workload
(depth 6, 1716 hierarchy nodes, dt = 1 fs for 10 ps = 10 000 RK4 steps, seeded
synthetic Hamiltonian) through the library's C ABI.  The headline value is
node-RHS evaluations per second (nodes x 4 RK4 stages x steps / time) of the
mixed-precision path (float right-hand sides, float-float accumulation of
rho_0, populations and eta); the plain FP64 path is timed beside it on the
same input.  Beside it: the batched scan (256 instances in one launch) against
plain FP64 solves of the same 256 instances, the serving trace, the 24-site
large hierarchy (HBM-resident) with its own bandwidth roofline, and the depth
sweep of the paper's timing table (N = 7, depths 4-12, 1000 steps) beside the
paper's own numbers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (N > 1) runs are replicas launched by torchrun: every rank solves
its own copies of the workload; only the timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# the serving measurement runs up to 32 concurrent launches on separate streams
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1012_4382_gb300 import workloads  # noqa: E402

METRIC = "HEOM node-RHS evals/s, batched solves/s and p99 latency vs plain FP64 path"
UNIT = "node-RHS evals/s"
WORKLOAD = "FMO-like N=7 with trap: K=6 (1716 nodes), dt=1 fs for 10 ps, seed 1234"
L2_FLUSH_BYTES = 256 << 20
# the paper's table of GPU timings (Tesla C2050, FP32): N = 7, N_max = 6, 1716 matrices,
# 1000 RK4 steps in 3 s -> 1716 x 4 x 1000 / 3 node-RHS evaluations per second
PAPER_NODE_RHS_PER_S = 1716 * 4 * 1000 / 3.0
# the whole table (Table 2): N = 7, 1000 RK4 steps; N_max -> (matrices, CPU s, GPU s), the CPU an
# "Intel 2.40 GHz", the GPU a Tesla C2050 in FP32
PAPER_TABLE2 = {4: (330, 120.0, 1.0), 6: (1716, 676.0, 3.0), 8: (6435, 2636.0, 7.0), 10: (19448, 8275.0, 19.0),
                12: (50388, 21972.0, 48.0)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-scan measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-trace measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 24-site large-hierarchy measurement")
    ap.add_argument("--no-table2", action="store_true",
                    help="skip the depth sweep of the paper's timing table (N = 7, depths 4-12, 1000 steps)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the scaled-hierarchy and low-temperature variants of the headline workload")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests replayed from the serving trace (default: the full trace, 2000)")
    ap.add_argument("--cpu-sample-steps", type=int, default=0, help="RK4 steps of the oracle sample (0: auto)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline (profiling runs)")
    ap.add_argument("--autotune", action="store_true",
                    help="time every candidate launch shape first and keep the fastest (default: the library's "
                         "default shapes, the ones the full-horizon parity tests run)")
    ap.add_argument("--no-autotune", action="store_true", help="accepted for older command lines; the default")
    ap.add_argument("--launch", default="",
                    help="mode,team_ctas,block,node_threads for the mixed path instead of autotuning (profiling runs)")
    ap.add_argument("--solve-steps", type=int, default=0,
                    help="RK4 steps per solve instead of the workload's 10 000 (profiling runs; not a bench value)")
    ap.add_argument("--batched-steps", type=int, default=0,
                    help="RK4 steps of the batched scan instead of its 5000 (profiling runs; not a bench value)")
    ap.add_argument("--large-steps", type=int, default=0,
                    help="RK4 steps of the 24-site workload instead of its 2000 (profiling runs; not a bench value)")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed

def dist_init(n):
    rank, world, local = 0, 1, 0
    if n > 1 or "WORLD_SIZE" in os.environ and int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# -------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_from_profile(name):
    """DRAM bytes per launch recorded in profiles/<name> by an ncu capture,
    or None when the kernel's source file changed since (its sha256, recorded
    beside the figure, differs)."""
    import hashlib
    try:
        rec = {}
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for ln in f:
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    k = k.strip().strip("-* `")
                    if k in ("traffic_bytes_per_launch", "source_file", "source_sha256"):
                        rec[k] = v.strip().strip("`")
        with open(os.path.join(ROOT, rec["source_file"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if rec.get("source_sha256") != sha:
            return None
        return float(rec["traffic_bytes_per_launch"])
    except Exception:
        return None


def l2_copy_gbs(torch, dev):
    """Copy bandwidth over an L2-resident pair of 16 MiB buffers (read + write
    bytes / time, CUDA events, best of 5 runs of 100 copies)."""
    n = (16 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(20):
        b.copy_(a)
    best = 0.0
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(100):
            b.copy_(a)
        e1.record()
        e1.synchronize()
        best = max(best, 2.0 * 4 * n * 100 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def algorithmic_bytes_per_node_step(N, elem_bytes):
    """The implementation's own count -- Horner-form RK4 over Hermitian-packed
    nodes: stage 0 reads y and writes wa; stages 1-3 read the stage input and
    y and write the output, so a node moves 11 packed arrays of N*N reals per
    step."""
    return 11 * N * N * elem_bytes


def model_bytes_per_node_stage(N, complex_bytes):
    """The method's count, used for `frac`: classic RK4 on full complex N x N
    matrices with three stored arrays (y, z, acc) reads z, y and acc and
    writes acc and z in every stage, 5 N^2 complex numbers per node-stage;
    complex_bytes = 8 (FP32 complex) or 16 (FP64 complex).  Neighbour gathers
    are reads of other nodes' z and count as reuse."""
    return 5 * N * N * complex_bytes


def roofline_block(N, nodes, steps, launch_ms, elem_bytes, peak, peak_kind, traffic, kernel, note=None):
    """Bandwidth roofline of one launch under both byte counts: `achieved` /
    `frac` with the method's 5 N^2 s per node-stage (s = complex size), and
    `achieved_impl` / `frac_impl` with the implementation's 11 N^2 packed
    reals per node-step; `traffic` is ncu's DRAM bytes per launch."""
    model = model_bytes_per_node_stage(N, 2 * elem_bytes) * nodes * 4 * steps
    impl = algorithmic_bytes_per_node_step(N, elem_bytes) * nodes * steps
    a = model / (launch_ms * 1e-3) / 1e9
    ai = impl / (launch_ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak, "traffic": traffic,
           "peak_kind": peak_kind, "kernel": kernel, "launch_ms": launch_ms,
           "bytes_model": "5 N^2 x %d B per node-stage (classic RK4, complex y/z/acc)" % (2 * elem_bytes),
           "algorithmic_bytes_per_launch": model,
           "achieved_impl": ai, "frac_impl": ai / peak,
           "bytes_model_impl": "11 N^2 x %d B per node-step (Horner RK4, Hermitian-packed)" % elem_bytes,
           "algorithmic_bytes_per_launch_impl": impl}
    if traffic is not None:
        out["traffic_vs_impl_bytes"] = traffic / impl
    if note:
        out["note"] = note
    return out


def flops_per_node_stage(N, complex_h=False):
    """Multiply-adds of one node's right-hand side in the Hermitian-packed
    form, times 2: per off-diagonal pair the commutator with the real part
    of H (4N - 6; twice that with an imaginary part) plus 12 for damping,
    trap, up- and down-couplings; per diagonal 2(N - 1) + 3."""
    pair = (4 * N - 6) * (2 if complex_h else 1) + 12
    diag = 2 * (N - 1) + 3
    return 2.0 * (N * (N - 1) // 2 * pair + N * diag)


def fp64_peak_tflops(sm_mhz):
    """FP64 FMA peak from unit counts: a double-precision warp instruction
    occupies a sub-partition for 64 cycles, so an SM retires 4 x 32 / 64 = 2
    FMAs (4 flops) per cycle; 152 SMs."""
    return 152 * 4.0 * sm_mhz * 1e6 / 1e12


def cpu_model():
    """Host CPU model (lscpu, else /proc/cpuinfo), with the architecture."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().lower().startswith("model name"):
                return "%s (%s)" % (line.split(":", 1)[1].strip(), platform.machine())
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return "%s (%s)" % (line.split(":", 1)[1].strip(), platform.machine())
    except OSError:
        pass
    return platform.machine()


def oracle_sample(w, steps, compare=None):
    """The oracle on the first `steps` steps of workload w, timed on the host
    cores.  compare: {name: GPU population rows at the workload's output
    cadence}; the largest difference over the common rows is reported."""
    import oracle
    oracle.build()
    nodes = oracle.num_nodes(w["params"]["N"], w["params"]["K"])
    every = w["out_every"] if compare else steps
    t0 = time.perf_counter()
    r = oracle.propagate(w["params"], w["rho0"], w["dt"], steps, every)
    dt = time.perf_counter() - t0
    out = {"value": nodes * 4.0 * steps / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "cpu": cpu_model(), "sample": "%d RK4 steps of the %d-node workload (%.2f s)" % (steps, nodes, dt)}
    if compare:
        # the same oracle on one host core, on a tenth of the sample
        n1 = max(1, steps // 10)
        threads = oracle.num_threads()
        oracle.set_threads(1)
        t1 = time.perf_counter()
        oracle.propagate(w["params"], w["rho0"], w["dt"], n1, n1)
        t1 = time.perf_counter() - t1
        oracle.set_threads(threads)
        out["single_core"] = {"value": nodes * 4.0 * n1 / t1, "unit": UNIT, "cores": 1,
                              "sample": "%d RK4 steps (%.2f s)" % (n1, t1)}
        for name, pops in compare.items():
            rows = min(len(pops), len(r["pops"]))
            out["max_abs_pop_diff_%s_vs_oracle" % name] = float(np.abs(pops[:rows] - r["pops"][:rows]).max())
        out["compared_rows"] = "populations every %g fs over the sample" % (w["out_every"] * w["dt"])
    return out


# ----------------------------------------------------------------- reference

def run_reference(args):
    rank, world, _ = dist_init(args.gpus)
    if rank != 0:
        barrier(world)
        return
    w = workloads.fmo_trap()
    steps = args.cpu_sample_steps or 1000  # about 2 s of host work per timed step
    for _ in range(max(args.warmup, 0)):
        oracle_sample(w, 2)
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(w, steps))
    wall = time.perf_counter() - t_all
    v = sum(x["value"] for x in vals) / len(vals)
    nodes = w["params"]["N"]
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 1, "seq_len": None, "parallelism": "replicas",
                   "sample": "each step: %d RK4 steps of the full hierarchy on the host cores" % steps},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                         "cpu": vals[0]["cpu"], "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    barrier(world)


# ---------------------------------------------------------------------- ours

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank, world, local = dist_init(args.gpus)
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1012_4382_gb300 import build as heom_build
    heom_build.build()
    from paper_1012_4382_gb300 import heom

    w = workloads.fmo_trap()
    p = w["params"]
    N, K = p["N"], p["K"]
    nsteps, out_every, dt = w["nsteps"], w["out_every"], w["dt"]
    if args.solve_steps > 0:
        nsteps = args.solve_steps
    nodes = heom.num_nodes(N, K)
    units_per_solve = nodes * 4.0 * nsteps
    nout = nsteps // out_every + 1
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rho0_dev = torch.from_numpy(np.ascontiguousarray(w["rho0"])).to(dev)
    d_pops = torch.empty(nout * N, dtype=torch.float64, device=dev)
    d_el = torch.empty(2 * nout, dtype=torch.float64, device=dev)

    kernel_ms = []

    def timed_device(ctx, steps, warm):
        """Per-solve device time (ms) with inputs resident; L2 flushed between
        solves.  The propagation launch alone is timed too (kernel_ms)."""
        times = []
        with torch.cuda.stream(stream):
            for i in range(warm + steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                em = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.set_rho0_device(rho0_dev)
                em.record(stream)
                ctx.propagate_device(dt, nsteps, out_every, d_pops, d_el)
                e1.record(stream)
                if i >= warm:
                    times.append((e0, em, e1))
        stream.synchronize()
        ctx.synchronize()
        kernel_ms[:] = [b.elapsed_time(c) for a, b, c in times]
        return [a.elapsed_time(c) for a, b, c in times]

    results = {}
    for prec in ("fp32", "fp64"):
        ctx = heom.Context(p, prec, stream=stream)
        if args.launch and prec == "fp32":
            m, c, b, g = (int(x) for x in args.launch.split(","))
            ctx.set_launch(mode=m, team_ctas=c, block_threads=b, node_threads=g)
        elif args.autotune:
            ctx.autotune(trial_steps=200)
        results[prec] = {"ctx": ctx, "launch": ctx.get_launch()}

    # ---- timed region: mixed-precision path (headline)
    ctx = results["fp32"]["ctx"]
    timed_device(ctx, 0, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per = timed_device(ctx, args.steps, 0)
    per_kernel = list(kernel_ms)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    dev_ms = sum(per)
    dev_ms_max = allreduce_max(dev_ms, world)
    total_units = allreduce_sum(units_per_solve * args.steps, world)
    value = total_units / (dev_ms_max * 1e-3)
    pops_gpu = d_pops.view(nout, N).cpu().numpy()
    eta_gpu = d_el.view(nout, 2)[:, 0].cpu().numpy()

    # ---- e2e: host buffers through the public blocking API
    e2e_times = []
    for i in range(1 + args.steps):
        t = time.perf_counter()
        ctx.set_rho0(w["rho0"])
        r = ctx.propagate(dt, nsteps, out_every)
        if i > 0:
            e2e_times.append(time.perf_counter() - t)
    e2e_s = allreduce_max(sum(e2e_times), world)
    e2e_value = total_units / e2e_s
    t_mean_fs, _ = ctx.trapping_time()  # <t> up to 10 ps of the last solve
    h2d = 16 * N * N
    d2h = 8 * (nout * N + 2 * nout)

    # ---- plain FP64 path, same workload
    ctx64 = results["fp64"]["ctx"]
    timed_device(ctx64, 0, 1)
    per64 = timed_device(ctx64, max(1, args.steps // 2), 0)
    per64_kernel = list(kernel_ms)
    fp64_value = units_per_solve * len(per64) / (sum(per64) * 1e-3)
    pops64 = d_pops.view(nout, N).cpu().numpy()
    eta64 = d_el.view(nout, 2)[:, 0].cpu().numpy()

    # ---- variants of the headline solve: scaled hierarchy, low-temperature correction
    variants = {}
    if not args.no_variants:
        L = results["fp32"]["launch"]
        for name, key in (("scaled_hierarchy", "scaled"), ("low_temperature_correction", "low_temp")):
            cv = heom.Context(dict(p, **{key: 1}), "fp32", stream=stream)
            cv.set_launch(mode=L["mode"], team_ctas=L["team_ctas"], block_threads=L["block_threads"],
                          node_threads=L["node_threads"])
            timed_device(cv, 0, 1)
            pv = timed_device(cv, 2, 0)
            pops_v = d_pops.view(nout, N).cpu().numpy()
            v = units_per_solve * len(pv) / (sum(pv) * 1e-3)
            variants[name] = {"value": v, "unit": UNIT, "ms_per_solve": statistics.mean(pv),
                              "vs_plain_mixed": v / (value / world),
                              "max_abs_pop_diff_vs_plain_mixed": float(np.abs(pops_v - pops_gpu).max())}
            cv.close()
        # filtered scaled hierarchy: a 2 ps pilot of the full scaled hierarchy (node magnitudes every
        # 250 fs), nodes below 1e-5 left out (closed downwards), then the timed solves on the kept nodes
        ps = dict(p, scaled=1)
        pilot = heom.Context(ps, "fp32", stream=stream)
        pilot.set_rho0(w["rho0"])
        mags = None
        for _ in range(8):
            pilot.propagate(dt, 250, 250)
            m = pilot.node_magnitudes()
            mags = m if mags is None else np.maximum(mags, m)
        pilot.close()
        keep = heom.filter_select(N, K, mags, 1e-5)
        cf = heom.Context(p, "fp32", stream=stream, keep=keep)  # the kept nodes, unscaled
        timed_device(cf, 0, 1)
        pf = timed_device(cf, 2, 0)
        pops_f = d_pops.view(nout, N).cpu().numpy()
        vf = units_per_solve * len(pf) / (sum(pf) * 1e-3)
        variants["filtered_hierarchy"] = {
            "value": vf, "unit": UNIT + " (of the full hierarchy's node count)", "ms_per_solve": statistics.mean(pf),
            "vs_plain_mixed": vf / (value / world), "nodes_kept": int(keep.sum()), "nodes_full": nodes,
            "threshold": 1e-5, "pilot": "2 ps of the full scaled hierarchy, magnitudes every 250 fs; kept nodes run "
                                        "unscaled",
            "launch": cf.get_launch(), "max_abs_pop_diff_vs_plain_mixed": float(np.abs(pops_f - pops_gpu).max())}
        cf.close()
        variants["scaled_hierarchy"]["note"] = "same rho as the plain path up to float rounding"
        variants["low_temperature_correction"]["note"] = "a change of the model: the difference is its effect"

    # ---- roofline of the dominant kernel (the persistent engine launch)
    launch_ms = statistics.mean(per_kernel)
    peak, peak_kind = peaks()
    l2_gbs = l2_copy_gbs(torch, dev)
    roof = roofline_block(N, nodes, nsteps, launch_ms, 4, peak, peak_kind,
                          traffic_from_profile("flow_fmo7_k6_mixed.md" if results["fp32"]["launch"]["mode"] == 3
                                               else "engine_fmo7_k6_mixed.md"),
                          kernel_name(results["fp32"]["launch"], N, "f32"),
                          "the 1 MB working set is L2-resident: the launch is bound by the latency of its "
                          "40 000 dependent stages (one L2 exchange of stage-tagged neighbour words each), not by "
                          "a bandwidth")
    roof["l2_copy_gbs_measured"] = l2_gbs
    roof["frac_of_l2_copy"] = roof["achieved"] / l2_gbs

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_NODE_RHS_PER_S,
        "vs_baseline_note": "against the paper's N=7, N_max=6 (1716 matrices) GPU timing on a Tesla C2050 in FP32 "
                            "(1000 steps in 3 s = %.3g node-RHS/s); other hardware, context only" % PAPER_NODE_RHS_PER_S,
        "dtype": "f32 (float-float rho_0, populations and eta)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": world, "seq_len": None,
                   "parallelism": "replicas x%d" % world,
                   "l2": "flushed (256 MB write) before every solve; the 1.0 MB state is L2-resident within a solve",
                   "launch": results["fp32"]["launch"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "wall_s": wall,
        "fp64_path": {"value": fp64_value, "unit": UNIT, "ms_per_solve": statistics.mean(per64),
                      "launch": results["fp64"]["launch"],
                      "roofline": {"bound": "alu", "unit": "TFLOP/s",
                                   "achieved": flops_per_node_stage(N) * nodes * 4 * nsteps
                                   / (statistics.mean(per64_kernel) * 1e-3) / 1e12,
                                   "peak": fp64_peak_tflops(2070.0),
                                   "frac": flops_per_node_stage(N) * nodes * 4 * nsteps
                                   / (statistics.mean(per64_kernel) * 1e-3) / 1e12 / fp64_peak_tflops(2070.0),
                                   "peak_kind": "derived: 152 SMs x 4 FP64 flops/cycle x 2070 MHz",
                                   "kernel": kernel_name(results["fp64"]["launch"], N, "f64"),
                                   "hbm": roofline_block(N, nodes, nsteps, statistics.mean(per64_kernel), 8, peak,
                                                         peak_kind, None, kernel_name(results["fp64"]["launch"], N,
                                                                                      "f64"))},
                      "mixed_vs_fp64_speedup": value / world / fp64_value,
                      "max_abs_pop_diff_vs_mixed": float(np.abs(pops64 - pops_gpu).max()),
                      "abs_eta_diff_vs_mixed": float(abs(eta64[-1] - eta_gpu[-1]))},
        "roofline": roof,
        "eta_10ps": float(eta_gpu[-1]),
        "variants": variants,
        "trapping_time_10ps_fs": t_mean_fs,
    }
    if rank == 0 and not args.no_batched:
        line["batched"] = bench_batched(heom, torch, stream, args.batched_steps)
    if rank == 0 and not args.no_large:
        line["large"] = bench_large(heom, torch, stream, peak, peak_kind, args.large_steps)
    if rank == 0 and not args.no_table2:
        line["table2_sweep"] = bench_table2(heom, torch, stream)
    if rank == 0 and not args.no_serving:
        line["serving"] = bench_serving(args.serving_requests)
    if rank == 0:
        n_sample = args.cpu_sample_steps or 5000  # about 10 s of host work
        if not args.no_cpu:
            line["cpu_baseline"] = oracle_sample(w, n_sample, {"mixed": pops_gpu, "fp64": pops64})
        print(json.dumps(line), flush=True)
    for v in results.values():
        v["ctx"].close()
    barrier(world)


def kernel_name(launch, N, prec):
    mode = launch.get("mode") if isinstance(launch, dict) else None
    if N > 8:
        return "heom_large_kernel<%s>" % prec
    if mode == 2:
        return "heom_smem_kernel<%d> (distributed shared memory)" % N
    if mode == 3:
        return "heom_flow_kernel<%d, %s> (dataflow, %d threads per CTA)" % (N, prec, launch.get("block_threads", 0))
    return "heom_engine_kernel<%d, %s>%s" % (N, prec, " (cooperative grid)" if mode == 1 else "")


def bench_large(heom, torch, stream, peak, peak_kind, steps=0):
    """24-site trimer, depth 4 (20 475 nodes of 24 x 24): the state is larger
    than L2, so every stage streams it from HBM.  Times the full 2 ps (2000
    steps) in FP64 and mixed precision; roofline of the FP64 launch."""
    w = workloads.large_trimer(nsteps=steps) if steps > 0 else workloads.large_trimer()
    p = w["params"]
    N = p["N"]
    nodes = heom.num_nodes(N, p["K"])
    nout = w["nsteps"] // w["out_every"] + 1
    rho0 = torch.from_numpy(np.ascontiguousarray(w["rho0"])).to(torch.cuda.current_device())
    d_pops = torch.empty(nout * N, dtype=torch.float64, device=rho0.device)
    d_el = torch.empty(2 * nout, dtype=torch.float64, device=rho0.device)
    out = {"workload": "24-site trimer (3 x 8-site blocks), K=4, 20475 nodes, dt=1 fs for 2 ps, no trap"}
    for prec, esize in (("fp64", 8), ("fp32", 4)):
        flops = flops_per_node_stage(N) * nodes * 4 * w["nsteps"]
        ctx = heom.Context(p, prec, stream=stream)
        ms = []
        with torch.cuda.stream(stream):
            for i in range(2):
                ctx.set_rho0_device(rho0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.propagate_device(w["dt"], w["nsteps"], w["out_every"], d_pops, d_el)
                e1.record(stream)
                ms.append((e0, e1))
        stream.synchronize()
        t = ms[-1][0].elapsed_time(ms[-1][1])
        rl = roofline_block(N, nodes, w["nsteps"], t, esize, peak, peak_kind,
                            traffic_from_profile("large_trimer_%s.md" % prec), "heom_large_kernel<%s>" % prec)
        if prec == "fp64":
            # FP64 runs at 1/64 of the FP32 rate: the arithmetic, not HBM, bounds this launch
            fp = fp64_peak_tflops(2070.0)
            tf = flops / (t * 1e-3) / 1e12
            rl = {"bound": "alu", "achieved": tf, "peak": fp, "unit": "TFLOP/s", "frac": tf / fp,
                  "peak_kind": "derived: 152 SMs x 4 FP64 flops/cycle x 2070 MHz",
                  "traffic": rl["traffic"], "kernel": rl["kernel"], "algorithmic_flops_per_launch": flops,
                  "hbm": rl}
        out[prec] = {"ms_per_solve": t, "node_rhs_per_s": nodes * 4.0 * w["nsteps"] / (t * 1e-3),
                     "launch": ctx.get_launch(), "roofline": rl,
                     "pop0_end": float(d_pops.view(nout, N)[-1, 0].item())}
        ctx.close()
    # the filtered form in mixed precision: a 500 fs pilot of the full scaled hierarchy
    # (magnitudes every 100 fs), nodes below 1e-5 left out, then the timed 2 ps on the kept nodes
    pops_full = d_pops.view(nout, N).cpu().numpy()
    ps = dict(p, scaled=1)
    pilot = heom.Context(ps, "fp32", stream=stream)
    pilot.set_rho0(w["rho0"])
    mags = None
    for _ in range(5):
        pilot.propagate(w["dt"], 100, 100)
        m = pilot.node_magnitudes()
        mags = m if mags is None else np.maximum(mags, m)
    pilot.close()
    keep = heom.filter_select(N, p["K"], mags, 1e-5)
    cf = heom.Context(p, "fp32", stream=stream, keep=keep)  # the kept nodes, unscaled
    with torch.cuda.stream(stream):
        cf.set_rho0_device(rho0)
        cf.propagate_device(w["dt"], 20, 20)
        cf.set_rho0_device(rho0)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        cf.propagate_device(w["dt"], w["nsteps"], w["out_every"], d_pops, d_el)
        f1.record(stream)
    cf.synchronize()
    tf = f0.elapsed_time(f1)
    out["fp32_filtered"] = {
        "ms_per_solve": tf, "vs_unfiltered_fp32": out["fp32"]["ms_per_solve"] / tf, "nodes_kept": int(keep.sum()),
        "nodes_full": nodes, "threshold": 1e-5,
        "pilot": "500 fs of the full scaled hierarchy, magnitudes every 100 fs; kept nodes run unscaled",
        "launch": cf.get_launch(),
        "max_abs_pop_diff_vs_unfiltered": float(np.abs(d_pops.view(nout, N).cpu().numpy() - pops_full).max())}
    cf.close()
    return out


def bench_table2(heom, torch, stream, nsteps=1000):
    """The paper's timing table (Table 2) on this GPU: one FMO-like N = 7 trap
    hierarchy at depths 4, 6, 8, 10 and 12 (330 to 50 388 matrices), 1000 RK4
    steps at 1 fs, in mixed precision (the paper ran FP32) and in FP64.  Each
    depth is timed in the library's default launch shape and in the shape its
    autotuner picks on the live hierarchy; the paper's C2050 and CPU timings
    stand beside them as context (other hardware)."""
    out = {"workload": "FMO-like N=7 with trap (seed 1234), depths 4-12, %d RK4 steps at 1 fs, one hierarchy "
                       "per solve, inputs resident, CUDA events; paper: Tesla C2050 FP32 and an Intel 2.40 GHz CPU"
                       % nsteps, "rows": []}
    for K, (mats, cpu_s, gpu_s) in sorted(PAPER_TABLE2.items()):
        w = workloads.fmo_trap(K=K, nsteps=nsteps)
        nodes = heom.num_nodes(7, K)
        assert nodes == mats
        row = {"depth": K, "matrices": nodes, "paper_gpu_s": gpu_s, "paper_cpu_s": cpu_s,
               "paper_gpu_node_rhs_per_s": nodes * 4.0 * nsteps / gpu_s}
        rho0 = torch.from_numpy(np.ascontiguousarray(w["rho0"])).to(torch.cuda.current_device())
        for prec in ("fp32", "fp64"):
            ctx = heom.Context(w["params"], prec, stream=stream)
            for shape in ("default", "tuned"):
                if shape == "tuned":
                    ctx.autotune(trial_steps=20)
                ev = []
                with torch.cuda.stream(stream):
                    for i in range(3):
                        ctx.set_rho0_device(rho0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        ctx.propagate_device(1.0, nsteps, nsteps)
                        e1.record(stream)
                        ev.append((e0, e1))
                stream.synchronize()
                ms = min(a.elapsed_time(b) for a, b in ev[1:])
                row["%s_%s" % (prec, shape)] = {"ms": ms, "node_rhs_per_s": nodes * 4.0 * nsteps / (ms * 1e-3),
                                                "launch": ctx.get_launch()}
            ctx.close()
        best32 = min(row["fp32_default"]["ms"], row["fp32_tuned"]["ms"])
        row["vs_paper_gpu"] = gpu_s * 1e3 / best32
        out["rows"].append(row)
    return out


def bench_batched(heom, torch, stream, steps=0, filter_scan=True):
    """Batched scan: 256 seeded N = 7 trap instances, depth 4..8, lambda and T
    scanned, 5 ps each, mixed precision, one persistent launch."""
    ws = workloads.batched_scan(nsteps=steps) if steps > 0 else workloads.batched_scan()
    b = heom.Batch([w["params"] for w in ws], "fp32", stream=stream)
    nodes = sum(heom.num_nodes(w["params"]["N"], w["params"]["K"]) for w in ws)
    nsteps = ws[0]["nsteps"]
    b.set_rho0([w["rho0"] for w in ws])
    with torch.cuda.stream(stream):
        b.propagate_device(1.0, nsteps, nsteps)
    b.synchronize()
    b.set_rho0([w["rho0"] for w in ws])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.propagate_device(1.0, nsteps, nsteps)
        e1.record(stream)
    b.synchronize()
    ms = e0.elapsed_time(e1)
    eta, _ = b.efficiency()
    launch = b.get_launch(ws[0]["params"]["N"])  # every instance has N = 7
    b.close()
    # plain FP64 path: every one of the 256 instances solved on its own in FP64, one launch each in
    # the library's default shape for its size; the device times of the 256 timed solves are summed
    # (a 20-step call before each warms its context up)
    plain_ms = 0.0
    eta_err = 0.0
    for i, w in enumerate(ws):
        ctx = heom.Context(w["params"], "fp64", stream=stream)
        ctx.set_rho0(w["rho0"])
        with torch.cuda.stream(stream):
            ctx.propagate_device(1.0, 20, 20)
        ctx.set_rho0(w["rho0"])
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            f0.record(stream)
            ctx.propagate_device(1.0, nsteps, nsteps)
            f1.record(stream)
        ctx.synchronize()
        plain_ms += f0.elapsed_time(f1)
        e64, _ = ctx.efficiency()
        eta_err = max(eta_err, abs(e64 - eta[i]))
        ctx.close()
    # the filtered form of the same scan: a 1 ps pilot of every instance's full scaled
    # hierarchy (magnitudes every 250 fs), nodes below 1e-5 left out, then the timed 5 ps on
    # the kept nodes; eta against the unfiltered scan
    filtered = None
    if filter_scan:
        pb = heom.Batch([dict(w["params"], scaled=1) for w in ws], "fp32", stream=stream)
        pb.set_rho0([w["rho0"] for w in ws])
        mags = [None] * len(ws)
        for _ in range(4):
            pb.propagate(1.0, 250, 250)
            for i in range(len(ws)):
                m = pb.node_magnitudes(i)
                mags[i] = m if mags[i] is None else np.maximum(mags[i], m)
        pb.close()
        keeps = [heom.filter_select(7, w["params"]["K"], mags[i], 1e-5) for i, w in enumerate(ws)]
        # the kept auxiliaries are propagated unscaled (the same node set and rho), which runs the
        # batch's register-view kernels
        fb = heom.Batch([w["params"] for w in ws], "fp32", stream=stream, keep=keeps)
        fb.set_rho0([w["rho0"] for w in ws])
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            g0.record(stream)
            fb.propagate_device(1.0, nsteps, nsteps)
            g1.record(stream)
        fb.synchronize()
        fms = g0.elapsed_time(g1)
        feta, _ = fb.efficiency()
        kept = sum(int(k.sum()) for k in keeps)
        fb.close()
        filtered = {"solves_per_s": len(ws) / (fms * 1e-3), "ms": fms, "nodes_kept": kept, "nodes_full": nodes,
                    "vs_unfiltered": ms / fms, "threshold": 1e-5,
                    "pilot": "1 ps of each full scaled hierarchy, magnitudes every 250 fs; kept nodes run unscaled",
                    "max_abs_eta_diff_vs_unfiltered": float(np.abs(np.asarray(feta) - np.asarray(eta)).max())}
    solves = len(ws) / (ms * 1e-3)
    plain = len(ws) / (plain_ms * 1e-3)
    peak, peak_kind = peaks()
    roof = roofline_block(7, nodes, nsteps, ms, 4, peak, peak_kind, traffic_from_profile("engine_batched_scan.md"),
                          "heom_engine_kernel<7, f32> (batched persistent launch)")
    return {"workload": "256 x N=7 trap, K~U{4..8}, lambda~U(2,200), T~U(77,300), 5 ps, fp32 mixed",
            "solves_per_s": solves, "node_rhs_per_s": nodes * 4.0 * nsteps / (ms * 1e-3),
            "ms": ms, "total_nodes": nodes, "eta_mean": float(np.mean(eta)), "launch": launch, "roofline": roof,
            "plain_fp64_solves_per_s": plain, "vs_plain_fp64": solves / plain,
            "plain_fp64_note": "all 256 instances solved one after another in FP64, one launch each in the default "
                               "shape for its size; device times summed",
            "filtered": filtered,
            "max_abs_eta_diff_vs_fp64": eta_err}


SERVING_LOW_RATE = 12.0  # req/s, about a quarter of the measured capacity of the mix
SERVING_CAPACITY_RATE = 40.0  # req/s, just below the measured capacity (about 42 req/s)


def bench_serving(count):
    """Serving: Poisson arrivals at 200 requests/s, N ~ U{2..8}, depth ~ U{3..8},
    1-20 ps at 1 fs, mixed precision, continuous batching with memory
    admission; latency from scheduled arrival to completion."""
    from paper_1012_4382_gb300 import serving
    tr = workloads.serving_trace(count=count)
    r = serving.run_trace(tr, "fp32", device_bytes=16 << 30, streams=32, time_limit_s=120.0)
    r["workload"] = ("Poisson 200 req/s, N~U{2..8}, K~U{3..8}, 1-20 ps at 1 fs, fp32 mixed; %s" %
                     ("the full seeded trace" if count == 2000 else "first %d requests of the seeded trace" % count))
    keys = ("requests", "completed", "offered_req_per_s", "achieved_req_per_s", "node_rhs_per_s", "p50_latency_s",
            "p99_latency_s", "mean_latency_s", "wall_s", "max_concurrent")
    # the same mix offered at about the capacity, and well below it (the
    # latency of a request that does not queue)
    for name, n, rate in (("at_capacity", 400, SERVING_CAPACITY_RATE), ("below_saturation", 200, SERVING_LOW_RATE)):
        tr2 = workloads.serving_trace(count=min(n, count), rate_per_s=rate)
        r2 = serving.run_trace(tr2, "fp32", device_bytes=16 << 30, streams=32, time_limit_s=120.0)
        r[name] = {k: r2[k] for k in keys}
        r[name]["workload"] = "the same mix at Poisson %g req/s, %d requests" % (rate, min(n, count))
    return r


if __name__ == "__main__":
    main()
