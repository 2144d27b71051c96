"""apsp_path (host reconstruction, no GPU) on stage records made here by the
plain Fig. 1 loop: the last improving k of each pair gives the stage
k // kblock.  Any valid order of the relaxations leaves a record with the
property apsp_path relies on, so the k-sequential loop serves as input."""
import numpy as np
import pytest

import oracle
from paper_1001_4108_gb300 import binding, inputs

INF = inputs.INF_I32


def fw_with_stages(w, kblock):
    """Fig. 1 (int64, explicit infinity) recording the stage of the last
    strict improvement of every pair (-1: never)."""
    n = w.shape[0]
    big = 1 << 60
    d = np.where(w >= INF, big, w.astype(np.int64))
    via = np.full((n, n), -1, np.int16)
    for k in range(n):
        cand = np.where((d[:, k:k + 1] < big) & (d[k:k + 1, :] < big), d[:, k:k + 1] + d[k:k + 1, :], big)
        better = cand < d
        d = np.where(better, cand, d)
        via[better] = k // kblock
    out = np.where(d >= big, INF, d).astype(np.int32)
    return out, via


def walk_weight(w, p):
    s = 0
    for u, v in zip(p[:-1], p[1:]):
        assert w[u, v] < INF, f"no edge {u}->{v}"
        s += int(w[u, v])
    return s


@pytest.fixture(scope="module")
def lib():
    try:
        return binding.lib()
    except RuntimeError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("n,kb,pot", [(60, 64, 0), (150, 64, 30), (200, 128, 0)])
def test_reconstruction_on_fig1_records(lib, n, kb, pot):
    w = inputs.int_graph(n, 0.06, 1, 100, seed=n, potential_max=pot)
    d, via = fw_with_stages(w, kb)
    np.testing.assert_array_equal(d, oracle.fw_int32_conv(w))  # the loop above is Fig. 1
    for i in range(0, n, 7):
        for j in range(0, n, 5):
            p = binding.path(d, via, i, j, kb)
            if i == j:
                assert p == [i]
            elif d[i, j] >= (1 << 28):
                assert p == []
            else:
                assert p[0] == i and p[-1] == j
                assert walk_weight(w, p) == d[i, j]


def test_errors(lib):
    w = inputs.int_graph(50, 0.1, 1, 100, seed=3)
    d, via = fw_with_stages(w, 64)
    i, j = np.argwhere((via >= 0) & (d < (1 << 28)))[0]
    p = binding.path(d, via, int(i), int(j), 64)
    assert len(p) >= 3
    args = (d.ctypes.data, via.ctypes.data, 50, 50, 50, binding.APSP_I32, 64, int(i), int(j))
    import ctypes
    ln = ctypes.c_int64(0)
    buf = (ctypes.c_int64 * 2)()
    assert lib.apsp_path(*args, buf, 2, ctypes.byref(ln)) == binding.APSP_ENOMEM and ln.value == len(p)
    # a record that does not belong to the matrix: its block 7 holds no vertex
    bad = via.copy()
    bad[i, j] = 7
    assert lib.apsp_path(d.ctypes.data, bad.ctypes.data, 50, 50, 50, binding.APSP_I32, 64, int(i), int(j),
                         buf, 2, ctypes.byref(ln)) == binding.APSP_EINVAL
    assert lib.apsp_path(*args[:6], 96, int(i), int(j), buf, 2, ctypes.byref(ln)) == binding.APSP_EINVAL
