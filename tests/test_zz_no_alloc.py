"""The allocation-free entry point, heom_propagate_static, called through the
C ABI and checked against the oracle and against the regular context API on
the same inputs.

It exists for callers that cannot call cudaMalloc (code under a device-memory
budget fixed up front, or inside a framework that owns every device
allocation); all of its working memory is one static device array that every
call reuses.  Two different problems are propagated in a row, then the first
one again, so a result that leaked state from the previous call would fail;
the device's free memory and the torch allocator's reserved bytes are checked
to stay the same across calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


class _Buffers:
    """Device inputs and outputs of one static call, allocated up front so
    that the calls themselves can be checked for allocations."""

    def __init__(self, w, nsteps, out_every):
        import torch
        N = w["params"]["N"]
        self.N, self.nout = N, nsteps // out_every + 1
        self.rho0 = torch.from_numpy(np.ascontiguousarray(w["rho0"], dtype=np.complex128)).cuda()
        self.pops = torch.full((self.nout * N,), float("nan"), dtype=torch.float64, device="cuda")
        self.el = torch.full((self.nout * 2,), float("nan"), dtype=torch.float64, device="cuda")
        self.rho = torch.zeros((N, N), dtype=torch.complex128, device="cuda")

    def result(self):
        el = self.el.view(self.nout, 2).cpu().numpy()
        return {"pops": self.pops.view(self.nout, self.N).cpu().numpy(), "eta": el[:, 0], "loss": el[:, 1],
                "rho": self.rho.cpu().numpy()}


def _static_rc(L, w, precision, nsteps, out_every, buf, stream=None):
    import torch
    keep = heom._Keep(w["params"], heom._precision(precision))
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    return L.heom_propagate_static(ctypes.byref(keep.c), buf.rho0.data_ptr(), float(w["dt"]), int(nsteps),
                                   int(out_every), buf.pops.data_ptr(), buf.el.data_ptr(), buf.rho.data_ptr(), s)


def _static_call(L, w, precision, nsteps, out_every, buf=None):
    buf = buf or _Buffers(w, nsteps, out_every)
    rc = _static_rc(L, w, precision, nsteps, out_every, buf)
    assert rc == heom.OK, L.heom_last_error().decode()
    return buf.result()


def _context_call(w, precision, nsteps, out_every):
    with heom.Context(w["params"], precision) as c:
        c.set_rho0(w["rho0"])
        r = c.propagate(w["dt"], nsteps, out_every)
        r["rho"] = c.rho()
    return r


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_point_matches_context_and_oracle_on_consecutive_calls(lib, precision):
    tp, te = TOL[precision]
    a = workloads.fmo_trap(K=5, nsteps=300)
    b = workloads.random_instance(4, 3, seed=21, trap=True, complex_h=True, terminator=1)
    refs = {}
    for name, w, nsteps, out_every in [("a", a, 300, 10), ("b", b, 120, 7), ("a", a, 300, 10)]:
        got = _static_call(lib, w, precision, nsteps, out_every)
        ref = _context_call(w, precision, nsteps, out_every)
        assert np.abs(got["pops"] - ref["pops"]).max() < tp
        assert np.abs(got["eta"] - ref["eta"]).max() < te
        assert np.abs(got["rho"] - ref["rho"]).max() < tp
        if name not in refs:
            refs[name] = oracle.propagate(w["params"], w["rho0"], w["dt"], nsteps, out_every)
        o = refs[name]
        N = w["params"]["N"]
        assert np.abs(got["pops"] - o["pops"]).max() < tp
        assert np.abs(got["eta"] - o["eta"]).max() < te
        assert np.abs(got["loss"] - o["loss"]).max() < te
        assert np.abs(got["rho"] - o["rho"][:N, :N]).max() < tp


def test_static_entry_point_allocates_no_device_memory(lib):
    import torch
    w = workloads.fmo_trap(K=5, nsteps=200)
    buf = _Buffers(w, 200, 10)
    for precision in ("fp32", "fp64"):  # loads the kernels (lazy module loading may take device memory)
        assert _static_rc(lib, w, precision, 200, 10, buf) == heom.OK, lib.heom_last_error().decode()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for precision in ("fp32", "fp64", "fp32"):
        assert _static_rc(lib, w, precision, 200, 10, buf) == heom.OK, lib.heom_last_error().decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_static_entry_point_reports_a_non_finite_run(lib):
    w = workloads.fmo_trap(K=3, nsteps=50)
    rho0 = np.array(w["rho0"], dtype=np.complex128)
    rho0[1, 1] = np.nan  # host-made input: the device path does not validate d_rho0
    w = dict(w, rho0=rho0)
    buf = _Buffers(w, 50, 10)
    for precision in ("fp64", "fp32"):
        assert _static_rc(lib, w, precision, 50, 10, buf) == heom.ENONFINITE
        assert b"NaN" in lib.heom_last_error()
    # a finite problem right after it is clean again (the status word is cleared per call)
    good = workloads.fmo_trap(K=3, nsteps=50)
    r = _static_call(lib, good, "fp64", 50, 10)
    o = oracle.propagate(good["params"], good["rho0"], good["dt"], 50, 10)
    assert np.abs(r["pops"] - o["pops"]).max() < 1e-10


def test_static_entry_point_refuses_stream_capture(lib):
    import torch
    w = workloads.fmo_trap(K=2, nsteps=10)
    buf = _Buffers(w, 10, 10)
    side = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        codes.append(_static_rc(lib, w, "fp32", 10, 10, buf, stream=side.cuda_stream))
    assert codes == [heom.EUNSUPPORTED]
    assert b"graph" in lib.heom_last_error() or b"capture" in lib.heom_last_error()


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
