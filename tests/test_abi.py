"""Host-side checks of libheom that need no GPU: the library loads, exports
every entry point include/heom.h declares, validates its inputs, refuses to
run without a device (no CPU fallback), and its hierarchy index builder agrees
with the oracle's independent enumeration."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "heom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(heom_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported():
    L = heom.lib()
    names = _declared_symbols()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n


def test_num_nodes_table_and_limits():
    for N, K, nodes in [(7, 4, 330), (7, 6, 1716), (7, 8, 6435), (7, 10, 19448), (7, 12, 50388), (7, 16, 245157),
                        (2, 4, 15), (24, 4, 20475)]:
        assert heom.num_nodes(N, K) == nodes
    with pytest.raises(heom.HeomError) as e:
        heom.num_nodes(0, 3)
    assert e.value.code == heom.EINVAL
    with pytest.raises(heom.HeomError):
        heom.num_nodes(25, 1)
    with pytest.raises(heom.HeomError):
        heom.num_nodes(24, 60)  # C(84, 60) is far above the node limit


@pytest.mark.parametrize("N,K", [(1, 0), (1, 4), (2, 4), (3, 5), (7, 6), (8, 3), (5, 0)])
def test_index_matches_oracle_enumeration(N, K):
    multi, up, down = heom.build_index(N, K)
    M = math.comb(N + K, K)
    assert multi.shape == (M, N)
    ref = oracle.multi_indices(N, K)
    assert sorted(map(tuple, multi.tolist())) == sorted(map(tuple, ref.tolist()))
    lev = multi.sum(axis=1)
    assert np.all(np.diff(lev) >= 0)
    assert tuple(multi[0]) == (0,) * N
    # lexicographically descending inside each level
    for L in range(K + 1):
        rows = [tuple(r) for r in multi[lev == L]]
        assert rows == sorted(rows, reverse=True)
    pos = {tuple(r): i for i, r in enumerate(multi.tolist())}
    for i, n in enumerate(multi.tolist()):
        for j in range(N):
            m = list(n)
            m[j] += 1
            exp_up = pos.get(tuple(m), -1) if sum(n) < K else -1
            assert up[i, j] == exp_up
            m[j] -= 2
            exp_dn = pos.get(tuple(m), -1) if n[j] > 0 else -1
            assert down[i, j] == exp_dn
            if up[i, j] >= 0:
                assert down[up[i, j], j] == i


def test_up_links_increase_within_a_level():
    multi, up, _ = heom.build_index(7, 6)
    lev = multi.sum(axis=1)
    for L in range(6):
        idx = np.where(lev == L)[0]
        for j in range(7):
            assert np.all(np.diff(up[idx, j]) > 0)


def test_invalid_parameters_are_rejected_before_any_device_work():
    w = workloads.dimer()
    bad = dict(w["params"])
    bad["H"] = np.array([[0, 1 + 1j], [1 + 1j, 0]])  # not Hermitian
    with pytest.raises(heom.HeomError) as e:
        heom.Context(bad)
    assert e.value.code == heom.EINVAL
    bad = dict(w["params"])
    bad["gam"] = np.array([106.0, 0.0])
    with pytest.raises(heom.HeomError) as e:
        heom.Context(bad)
    assert e.value.code == heom.EINVAL
    bad = dict(w["params"])
    bad["T"] = -1.0
    with pytest.raises(heom.HeomError):
        heom.Context(bad)
    # flags: only HEOM_FLAG_LOW_TEMP and HEOM_FLAG_SCALED exist
    keep = heom._Keep(dict(w["params"], low_temp=1, scaled=1), heom.FP64)
    keep.c.flags = heom.FLAG_LOW_TEMP | heom.FLAG_SCALED | 8
    h = heom.ctypes.c_void_p()
    assert heom.lib().heom_create(heom.ctypes.byref(keep.c), None, heom.ctypes.byref(h)) == heom.EINVAL
    assert b"unknown flags" in heom.lib().heom_last_error()


def test_no_cpu_fallback_without_a_device():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    w = workloads.dimer()
    with pytest.raises(heom.HeomError) as e:
        heom.Context(w["params"])
    assert e.value.code == heom.ECUDA
    with pytest.raises(heom.HeomError) as e:
        heom.selftest_bounded_wait(20.0)
    assert e.value.code == heom.ECUDA
