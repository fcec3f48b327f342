"""Continuous-batching server: every result is the same alone and in the mix,
matches the oracle, and admission, rejection and cancellation behave as
documented.  Failures are made on the host (oversized or malformed requests,
cancellation); no GPU fault is provoked."""
import time

import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, serving, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def _requests():
    tr = workloads.serving_trace(count=10)
    for w in tr:
        w["nsteps"] = 200 + 37 * (w["params"]["N"] % 3)
        w["out_every"] = 20
    return tr


def _drain(srv, ids, timeout=120.0):
    t0 = time.time()
    while True:
        srv.progress()
        if all(srv.status(i) in (serving.DONE, serving.FAILED, serving.CANCELLED) for i in ids):
            return
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(1e-4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_results_alone_equal_results_in_the_mix(precision):
    reqs = _requests()
    alone = []
    with serving.Server(device_bytes=1 << 30, streams=1) as srv:
        for w in reqs:
            i = srv.submit(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], precision)
            _drain(srv, [i])
            alone.append(srv.result(i))
    with serving.Server(device_bytes=1 << 30, streams=8) as srv:
        ids = [srv.submit(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], precision) for w in reqs]
        seen_running = 0
        t0 = time.time()
        while not all(srv.status(i) in (serving.DONE, serving.FAILED) for i in ids):
            srv.progress()
            seen_running = max(seen_running, srv.stats()["running"])
            assert time.time() - t0 < 120
        mixed = [srv.result(i) for i in ids]
    assert seen_running > 1  # their work overlapped on the device
    for a, b in zip(alone, mixed):
        assert np.abs(a["pops"] - b["pops"]).max() <= 1e-12
        assert np.abs(a["eta"] - b["eta"]).max() <= 1e-12
    # and they are right
    tol = (1e-10, 1e-10) if precision == "fp64" else (1e-5, 1e-4)
    for w, r in list(zip(reqs, mixed))[:4]:
        o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"])
        assert np.abs(r["pops"] - o["pops"]).max() < tol[0]
        assert np.abs(r["eta"] - o["eta"]).max() < tol[1]


def test_admission_does_not_block_on_a_busy_stream():
    """One stream: the first progress call launches the head request's group
    and every later request that joins it; a request of another site count
    keeps its place and starts on the next free stream."""
    small = workloads.random_instance(3, 3, seed=71)
    other = workloads.random_instance(5, 3, seed=72)
    with serving.Server(device_bytes=1 << 30, streams=1) as srv:
        a = srv.submit(small["params"], small["rho0"], 1.0, 400, 100)
        b = srv.submit(other["params"], other["rho0"], 1.0, 400, 100)
        c = srv.submit(small["params"], small["rho0"], 1.0, 400, 100)
        srv.progress()
        assert srv.status(b) == serving.QUEUED
        assert srv.status(a) != serving.QUEUED and srv.status(c) != serving.QUEUED
        _drain(srv, [a, b, c])
        assert all(srv.status(i) == serving.DONE for i in (a, b, c))
        ra, rc = srv.result(a), srv.result(c)
        assert np.array_equal(ra["pops"], rc["pops"])


def test_admission_waits_for_memory():
    reqs = _requests()[:6]
    need = max(heom.num_nodes(w["params"]["N"], w["params"]["K"]) for w in reqs)
    # a budget that holds roughly one of the larger requests at a time
    budget = max(1 << 20, int(need * 64 * 4 * 3 * 1.6) + (1 << 18))
    with serving.Server(device_bytes=budget, streams=8) as srv:
        ids = []
        for w in reqs:
            try:
                ids.append(srv.submit(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"], "fp32"))
            except heom.HeomError as e:
                assert e.code == heom.ENOMEM
        _drain(srv, ids)
        for i in ids:
            assert srv.status(i) == serving.DONE
        assert srv.stats()["bytes_in_use"] > 0  # cached tables stay resident


def test_rejections_and_cancellation():
    w = workloads.fmo_trap(K=8)
    with serving.Server(device_bytes=1 << 20, streams=2) as srv:
        with pytest.raises(heom.HeomError) as e:  # can never fit in 1 MiB
            srv.submit(w["params"], w["rho0"], 1.0, 100, 10)
        assert e.value.code == heom.ENOMEM
        bad = dict(w["params"])
        bad["T"] = 0.0
        with pytest.raises(heom.HeomError) as e:
            srv.submit(bad, w["rho0"], 1.0, 100, 10)
        assert e.value.code == heom.EINVAL
        small = workloads.fmo_trap(K=2)
        a = srv.submit(small["params"], small["rho0"], 1.0, 50, 10)
        b = srv.submit(small["params"], small["rho0"], 1.0, 50, 10)
        c = srv.submit(small["params"], small["rho0"], 1.0, 50, 10)
        srv.cancel(c)  # still queued: no progress call yet
        assert srv.status(c) == serving.CANCELLED
        _drain(srv, [a, b])
        with pytest.raises(heom.HeomError):
            srv.cancel(a)  # finished requests cannot be cancelled
        ra, rb = srv.result(a), srv.result(b)
        assert np.array_equal(ra["pops"], rb["pops"])
        srv.release(a)
        srv.release(c)
        with pytest.raises(heom.HeomError):
            srv.status(a)


def test_trace_replay_reports_latency():
    tr = workloads.serving_trace(count=40, rate_per_s=400.0)
    for w in tr:
        w["nsteps"] = min(w["nsteps"], 1500)
    r = serving.run_trace(tr, "fp32", device_bytes=2 << 30, streams=8)
    assert r["completed"] == 40
    assert 0 < r["p50_latency_s"] <= r["p99_latency_s"]


def test_json_configured_run_matches_the_oracle(tmp_path, capsys):
    """The serving harness driven by a JSON run configuration and a file of
    request lines: every request's populations and eta, written to the
    results file, against the oracle."""
    import json
    lines = []
    for i, (N, K) in enumerate([(2, 3), (4, 3), (3, 5)]):
        w = workloads.random_instance(N, K, seed=2100 + i)
        p = w["params"]
        lines.append({"arrival_s": 0.02 * i, "N": N, "K": K,
                      "H": [[[float(z.real), float(z.imag)] for z in row] for row in p["H"]],
                      "lam": p["lam"].tolist(), "gam": p["gam"].tolist(), "T": float(p["T"]),
                      "trap": p["trap"].tolist(), "recomb": p["recomb"].tolist(), "initial_site": 0,
                      "dt": 1.0, "nsteps": 150, "out_every": 30})
    (tmp_path / "req.jsonl").write_text("\n".join(json.dumps(x) for x in lines) + "\n")
    cfg = {"precision": "fp32", "device_bytes": 1 << 30, "streams": 4, "trace": "req.jsonl",
           "results": str(tmp_path / "out.jsonl")}
    (tmp_path / "run.json").write_text(json.dumps(cfg))
    assert serving.main(["--config", str(tmp_path / "run.json")]) == 0
    summary = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert summary["completed"] == 3
    got = {r["request"]: r for r in map(json.loads, (tmp_path / "out.jsonl").read_text().splitlines())}
    for i, line in enumerate(lines):
        e = serving.request_from_json(line)
        o = oracle.propagate(e["params"], e["rho0"], 1.0, 150, 30)
        assert np.abs(np.array(got[i]["pops"]) - o["pops"]).max() < 1e-5
        assert np.abs(np.array(got[i]["eta"]) - o["eta"]).max() < 1e-4


def test_benchmark_trace_prefix_full_length_sampled_against_the_oracle():
    """The first 40 requests of the benchmark's serving trace (Poisson 200/s,
    N 2..8, depth 3..8, 1..20 ps at full length) replayed in the benchmark's
    server configuration (16 GB budget, 32 streams); every request completes,
    and the four cheapest for the host (nodes x steps) are checked against the
    oracle on every 100 fs row."""
    tr = workloads.serving_trace()[:40]
    r = serving.run_trace(tr, "fp32", device_bytes=16 << 30, streams=32, keep_results=True)
    assert r["completed"] == 40
    cost = [heom.num_nodes(w["params"]["N"], w["params"]["K"]) * w["nsteps"] for w in tr]
    for i in np.argsort(cost)[:4]:
        w = tr[i]
        o = oracle.propagate(w["params"], w["rho0"], w["dt"], w["nsteps"], w["out_every"])
        g = r["results"][int(i)]
        assert g["pops"].shape == o["pops"].shape
        assert np.abs(g["pops"] - o["pops"]).max() < 1e-5, i
        assert np.abs(g["eta"] - o["eta"]).max() < 1e-4, i
