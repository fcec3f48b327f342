"""The JSON run configuration of the serving harness (no GPU): request lines
become the trace entries the server takes, synthetic traces are the seeded
ones of workloads.serving_trace, and malformed lines are refused."""
import json

import numpy as np
import pytest

from paper_1012_4382_gb300 import serving, workloads


def test_request_line_becomes_a_trace_entry():
    H = [[0.0, 50.0, 0.0], [50.0, 120.0, 20.0], [0.0, 20.0, 300.0]]
    d = {"arrival_s": 0.25, "N": 3, "K": 4, "H": H, "lam": 35.0, "gam": [100.0, 110.0, 120.0], "T": 250,
         "trap": [0.0, 0.0, 1.0], "initial_site": 1, "dt": 0.5, "nsteps": 400, "out_every": 50}
    e = serving.request_from_json(json.loads(json.dumps(d)))
    assert e["arrival_s"] == 0.25 and e["dt"] == 0.5 and e["nsteps"] == 400 and e["out_every"] == 50
    p = e["params"]
    assert p["N"] == 3 and p["K"] == 4 and p["T"] == 250
    assert np.array_equal(p["H"], np.asarray(H, dtype=np.complex128))
    assert np.array_equal(p["lam"], np.full(3, 35.0)) and np.array_equal(p["gam"], [100.0, 110.0, 120.0])
    assert np.array_equal(p["trap"], [0.0, 0.0, 1.0]) and "recomb" not in p
    rho0 = np.zeros((3, 3), complex)
    rho0[1, 1] = 1.0
    assert np.array_equal(e["rho0"], rho0)


def test_complex_h_as_pairs_and_defaults():
    H = [[[0.0, 0.0], [40.0, 5.0]], [[40.0, -5.0], [100.0, 0.0]]]
    e = serving.request_from_json({"N": 2, "K": 2, "H": H, "lam": 20, "gam": 90, "T": 300, "nsteps": 10})
    assert e["params"]["H"][0, 1] == 40 + 5j and e["params"]["H"][1, 0] == 40 - 5j
    assert e["arrival_s"] == 0.0 and e["dt"] == 1.0 and e["out_every"] == 10 and e["rho0"][0, 0] == 1.0


@pytest.mark.parametrize("bad", [{"H": [[0.0]]}, {"initial_site": 2}])
def test_malformed_lines_are_refused(bad):
    d = {"N": 2, "K": 1, "H": [[0.0, 10.0], [10.0, 50.0]], "lam": 20, "gam": 90, "T": 300, "nsteps": 10}
    d.update(bad)
    with pytest.raises(ValueError):
        serving.request_from_json(d)


def test_trace_from_a_file_and_synthetic(tmp_path):
    lines = [{"arrival_s": 0.1 * i, "N": 2, "K": 2, "H": [[0.0, 30.0], [30.0, 80.0]], "lam": 35, "gam": 106,
              "T": 300, "nsteps": 100 + i, "out_every": 10} for i in range(3)]
    (tmp_path / "req.jsonl").write_text("\n".join(json.dumps(x) for x in lines) + "\n")
    tr = serving.load_trace({"trace": "req.jsonl"}, str(tmp_path))
    assert [t["nsteps"] for t in tr] == [100, 101, 102] and tr[2]["arrival_s"] == pytest.approx(0.2)
    syn = serving.load_trace({"trace": {"count": 5, "rate_per_s": 50.0}})
    ref = workloads.serving_trace(count=5, rate_per_s=50.0)
    assert len(syn) == 5
    for a, b in zip(syn, ref):
        assert a["arrival_s"] == b["arrival_s"] and a["nsteps"] == b["nsteps"]
        assert np.array_equal(a["params"]["H"], b["params"]["H"])
