"""Device-side check of the node tables (heom_check_node_tables): the tables
of every hierarchy pass, and corrupted copies fail at the node a host
restatement of the same test names.  The corruptions are made on the host in
a copy of the tables; the check reads a linked entry only after finding its
index in range, so every read stays inside the arrays."""
import numpy as np
import pytest

from paper_1012_4382_gb300 import build as heom_build
from paper_1012_4382_gb300 import heom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    heom_build.build()


def host_first_bad(u, d, M):
    """The test of heom_check_node_tables, written out on the host: the
    smallest node that breaks it, or -1."""
    N, Mpad = u.shape
    bad = []
    for j in range(N):
        for n in range(Mpad):
            up, dn = int(u[j, n]), int(d[j, n])
            if n >= M:
                ok = up == -1 and dn == -1
            else:
                ok = dn == -1 or (dn >= 0 and (dn >> 24) >= 1 and (dn & 0xFFFFFF) < n)
                nj = dn >> 24 if dn >= 0 else 0
                if ok and dn >= 0:
                    ok = int(u[j, dn & 0xFFFFFF]) == n
                if ok and up != -1:
                    ok = n < up < M
                    if ok:
                        back = int(d[j, up])
                        ok = back >= 0 and (back & 0xFFFFFF) == n and (back >> 24) == nj + 1
            if not ok:
                bad.append(n)
    return min(bad) if bad else -1


def on_device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("N,K", [(1, 4), (2, 5), (4, 3), (7, 6), (8, 4), (24, 2)])
def test_library_tables_pass(N, K):
    u, d, Mpad = heom.device_tables(N, K)
    M = heom.num_nodes(N, K)
    assert host_first_bad(u, d, M) == -1
    assert heom.check_node_tables(on_device(u), on_device(d), M, Mpad, N) == -1


def _corruptions(u, d, M):
    """(name, up, dn) copies with one entry changed each."""
    rng = np.random.default_rng(5)
    N, Mpad = u.shape
    out = []
    for name in ("up out of range", "up backwards", "up to a wrong node", "down count", "down to a later node",
                 "down to a wrong node", "padding", "removed up link"):
        uu, dd = u.copy(), d.copy()
        while True:
            j, n = int(rng.integers(N)), int(rng.integers(1, M))
            if name.startswith("up") and u[j, n] >= 0:
                break
            if name.startswith("down") and d[j, n] >= 0:
                break
            if name == "padding" and (Mpad > M or u[j, n] >= 0):
                break
            if name == "removed up link" and u[j, n] >= 0:
                break
        if name == "up out of range":
            uu[j, n] = M + 3
        elif name == "up backwards":
            uu[j, n] = n - 1
        elif name == "up to a wrong node":
            uu[j, n] = min(M - 1, u[j, n] + 1) if u[j, n] + 1 < M else u[j, n] - 1
        elif name == "down count":
            dd[j, n] = d[j, n] + (1 << 24)
        elif name == "down to a later node":
            dd[j, n] = (d[j, n] & ~0xFFFFFF) | (n + 1)
        elif name == "down to a wrong node":
            dd[j, n] = (d[j, n] & ~0xFFFFFF) | ((d[j, n] & 0xFFFFFF) ^ 1)
        elif name == "padding":
            if Mpad > M:
                uu[j, M] = 0
            else:
                uu[j, n] = -7
        else:  # an up link dropped while its partner still points back
            uu[j, n] = -1
        out.append((name, uu, dd))
    return out


@pytest.mark.parametrize("N,K", [(4, 3), (7, 6)])
def test_corrupted_tables_fail_at_the_host_named_node(N, K):
    u, d, Mpad = heom.device_tables(N, K)
    M = heom.num_nodes(N, K)
    for name, uu, dd in _corruptions(u, d, M):
        want = host_first_bad(uu, dd, M)
        assert want >= 0, name
        with pytest.raises(heom.HeomError) as e:
            heom.check_node_tables(on_device(uu), on_device(dd), M, Mpad, N)
        assert e.value.code == heom.EINVAL, name
        assert e.value.bad_node == want, (name, e.value.bad_node, want)
    # the check leaves the device usable
    assert heom.check_node_tables(on_device(u), on_device(d), M, Mpad, N) == -1


def test_check_rejects_bad_arguments():
    u, d, Mpad = heom.device_tables(3, 2)
    M = heom.num_nodes(3, 2)
    du, dd = on_device(u), on_device(d)
    for args in [(M, M - 1, 3), (0, Mpad, 3), (M, Mpad, 0), (M, Mpad, 25)]:
        with pytest.raises(heom.HeomError) as e:
            heom.check_node_tables(du, dd, *args)
        assert e.value.code == heom.EINVAL
