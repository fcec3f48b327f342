"""The allocation-free entry point, heom_propagate_static, called through the
C ABI and checked against the regular context API on the same inputs.

It exists for callers that cannot call cudaMalloc (code under a device-memory
budget fixed up front, or inside a framework that owns every device
allocation); all of its working memory is one static device array that every
call reuses.  Two different problems are propagated in a row, then the first
one again, so a result that leaked state from the previous call would fail.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-10), "fp32": (1e-5, 1e-4)}


@pytest.fixture(scope="module")
def lib():
    heom_build.build()
    L = heom.lib()
    vp = ctypes.c_void_p
    L.heom_propagate_static.argtypes = [ctypes.POINTER(heom._Params), vp, ctypes.c_double, ctypes.c_int64,
                                        ctypes.c_int64, vp, vp, vp, vp]
    L.heom_propagate_static.restype = ctypes.c_int
    return L


def _static_call(L, w, precision, nsteps, out_every):
    import torch
    N = w["params"]["N"]
    keep = heom._Keep(w["params"], heom._precision(precision))
    nout = nsteps // out_every + 1
    d_rho0 = torch.from_numpy(np.ascontiguousarray(w["rho0"], dtype=np.complex128)).cuda()
    d_pops = torch.full((nout * N,), float("nan"), dtype=torch.float64, device="cuda")
    d_el = torch.full((nout * 2,), float("nan"), dtype=torch.float64, device="cuda")
    d_rho = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.heom_propagate_static(ctypes.byref(keep.c), d_rho0.data_ptr(), float(w["dt"]), int(nsteps),
                                 int(out_every), d_pops.data_ptr(), d_el.data_ptr(), d_rho.data_ptr(), stream)
    assert rc == heom.OK, L.heom_last_error().decode()
    torch.cuda.synchronize()
    el = d_el.view(nout, 2).cpu().numpy()
    return {"pops": d_pops.view(nout, N).cpu().numpy(), "eta": el[:, 0], "loss": el[:, 1],
            "rho": d_rho.cpu().numpy()}


def _context_call(w, precision, nsteps, out_every):
    with heom.Context(w["params"], precision) as c:
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], nsteps, out_every)
        r["rho"] = c.rho()
    return r


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_point_matches_context_on_consecutive_calls(lib, precision):
    tp, te = TOL[precision]
    a = workloads.fmo_trap(K=5, nsteps=300)
    b = workloads.random_instance(4, 3, seed=21, trap=True, complex_h=True, terminator=1)
    for w, nsteps, out_every in [(a, 300, 10), (b, 120, 7), (a, 300, 10)]:
        got = _static_call(lib, w, precision, nsteps, out_every)
        ref = _context_call(w, precision, nsteps, out_every)
        assert np.abs(got["pops"] - ref["pops"]).max() < tp
        assert np.abs(got["eta"] - ref["eta"]).max() < te
        assert np.abs(got["rho"] - ref["rho"]).max() < tp


def test_static_entry_point_rejects_oversized_problems(lib):
    import torch
    w = workloads.fmo_trap(K=10)  # 19 448 nodes: beyond the static area in either precision
    keep = heom._Keep(w["params"], heom.FP32_MIXED)
    d_rho0 = torch.zeros((7, 7), dtype=torch.complex128, device="cuda")
    rc = lib.heom_propagate_static(ctypes.byref(keep.c), d_rho0.data_ptr(), 1.0, 10, 10, None, None, None, None)
    assert rc == heom.EINVAL
    assert b"static area" in lib.heom_last_error()


def test_static_entry_point_rejects_scaled_hierarchies(lib):
    import torch
    w = workloads.fmo_trap(K=2)
    keep = heom._Keep(dict(w["params"], scaled=1), heom.FP64)
    d_rho0 = torch.zeros((7, 7), dtype=torch.complex128, device="cuda")
    rc = lib.heom_propagate_static(ctypes.byref(keep.c), d_rho0.data_ptr(), 1.0, 10, 10, None, None, None, None)
    assert rc == heom.EUNSUPPORTED
