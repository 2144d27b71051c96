"""Path reconstruction (apsp_fw_paths + apsp_path) on the GPU.

What is unique is compared exactly: the distances equal apsp_fw's bit for
bit (and the oracle's for the integers).  The stage record and the paths are
not unique (ties), so they are checked for validity against definitions:
* via[i][j] = -1  =>  d_ij is the input weight w_ij;
* via[i][j] = b  =>  some k of k-block b, k != i, j, has d_ik + d_kj = d_ij
  (integers, exactly) and d_ij < w_ij;
* a path i -> j is a walk along edges of the input whose weight sum is d_ij
  (integers: exactly; fp32: within the fp32 tolerance of the FP64 oracle).
"""
import numpy as np
import pytest

import oracle
from paper_1001_4108_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    binding.lib()
    yield
    assert binding.device_error() == 0


def _graph(dt, n, seed):
    if dt == "f32":
        w = inputs.dense_f32(n, seed=seed)
        g = np.random.default_rng(seed)
        w[g.random((n, n)) < 0.5] = np.inf  # sparse, so that paths have several edges
        np.fill_diagonal(w, 0)
        return w
    w = inputs.int_graph(n, 0.05, 1, 1000, seed=seed, potential_max=0 if dt == "i16" else 40)
    return inputs.to_int16(np.minimum(w, inputs.INF_I32)) if dt == "i16" else w


def _solve_paths(w, kblock=0, flags=0):
    t = torch.from_numpy(w).cuda()
    via = torch.empty(w.shape, dtype=torch.int16, device="cuda")
    binding.apsp_fw_paths(t, via, kblock=kblock, flags=flags)
    torch.cuda.synchronize()
    return t.cpu().numpy(), via.cpu().numpy()


def _reach(dt, d):
    if dt == "f32":
        return np.isfinite(d)
    return d < (inputs.INF_I16 if dt == "i16" else (1 << 28))


def _check_record(dt, w, d, via, S):
    n = w.shape[0]
    reach = _reach(dt, d)
    never = via < 0
    # never improved: the input value (edge or infinity) is final
    if dt == "f32":
        assert np.array_equal(d[never], w[never])
    else:
        assert np.array_equal(d[never & reach], w[never & reach])
    # improved in stage b: a split vertex in k-block b (integers: exact)
    if dt != "f32":
        di = np.where(reach, d.astype(np.int64), 1 << 40)
        for b in np.unique(via[~never]):
            ii, jj = np.nonzero(via == b)
            ks = np.arange(b * S, min(n, (b + 1) * S))
            best = np.full(ii.shape, 1 << 41, np.int64)
            for k in ks:
                cand = di[ii, k] + di[k, jj]
                cand[(ii == k) | (jj == k)] = 1 << 41
                best = np.minimum(best, cand)
            sel = reach[ii, jj]
            assert np.array_equal(best[sel], di[ii, jj][sel]), f"stage {b}: no split vertex"


def _check_path(dt, w, d, p, i, j, d64=None):
    assert p[0] == i and p[-1] == j
    wsum = 0.0 if dt == "f32" else 0
    for u, v in zip(p[:-1], p[1:]):
        e = w[u, v]
        if dt == "f32":
            assert np.isfinite(e), f"no edge {u}->{v}"
            wsum += float(e)
        else:
            assert e < (inputs.INF_I16 if dt == "i16" else inputs.INF_I32), f"no edge {u}->{v}"
            wsum += int(e)
    if dt == "f32":
        assert abs(wsum - d64[i, j]) <= 1e-5 * max(abs(d64[i, j]), 1.0) + 1e-6 * len(p)
    else:
        assert wsum == int(d[i, j])


@pytest.mark.parametrize("dt", ["i32", "f32", "i16"])
@pytest.mark.parametrize("n,kb", [(200, 64), (700, 64), (9 * 128 + 37, 128)])
def test_paths_record_and_reconstruction(dt, n, kb):
    w = _graph(dt, n, seed=n + kb)
    d, via = _solve_paths(w, kblock=kb)
    # distances: bit-identical to the plain solve
    t = torch.from_numpy(w).cuda()
    binding.apsp_fw(t, kblock=kb)
    torch.cuda.synchronize()
    assert np.array_equal(d, t.cpu().numpy())
    d64 = None
    if dt == "f32":
        d64 = oracle.fw_f64(w)
    else:
        np.testing.assert_array_equal(d, oracle.fw_int16_conv(w) if dt == "i16" else oracle.fw_int32_conv(w))
    assert via.min() >= -1 and via.max() < (n + kb - 1) // kb
    _check_record(dt, w, d, via, kb)
    g = np.random.default_rng(n)
    reach = _reach(dt, d)
    pairs = list(zip(g.integers(0, n, 300), g.integers(0, n, 300)))
    for i, j in pairs:
        p = binding.path(d, via, int(i), int(j), kb)
        if i == j:
            assert p == [i]
        elif not reach[i, j]:
            assert p == []
        else:
            _check_path(dt, w, d, p, int(i), int(j), d64)


def test_paths_lookahead_plain_and_graph_replay_agree():
    # the stage record does not depend on the schedule: each tile sees the
    # stages in order in both
    w = _graph("i32", 1100, seed=1)
    d0, v0 = _solve_paths(w)                                    # lookahead, direct
    d1, v1 = _solve_paths(w, flags=binding.FLAG_NO_LOOKAHEAD)   # plain
    t = torch.from_numpy(w).cuda()
    via = torch.empty(w.shape, dtype=torch.int16, device="cuda")
    src = t.clone()
    for _ in range(3):  # direct, captured graph, replay (via reset every call)
        t.copy_(src)
        binding.apsp_fw_paths(t, via)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), d0) and np.array_equal(via.cpu().numpy(), v0)
    assert np.array_equal(d0, d1) and np.array_equal(v0, v1)


def test_paths_tiny_graphs():
    # n = 1 and 2 (one stage, phase 1 only) and a 2-cycle with an improvement
    for w in (np.array([[0]], np.int32), np.array([[0, 5], [inputs.INF_I32, 0]], np.int32),
              np.array([[0, 10, 1], [1, 0, inputs.INF_I32], [inputs.INF_I32, 2, 0]], np.int32)):
        d, via = _solve_paths(w)
        np.testing.assert_array_equal(d, oracle.fw_int32_conv(w))
        n = w.shape[0]
        for i in range(n):
            for j in range(n):
                p = binding.path(d, via, i, j, binding.query_config(n, binding.APSP_I32).kblock)
                if i == j:
                    assert p == [i]
                elif d[i, j] >= (1 << 28):
                    assert p == []
                else:
                    _check_path("i32", w, d, p, i, j)
    # the 3-vertex case: 0 -> 1 improves from 10 to 3 through 2 (stage 0)
    d, via = _solve_paths(np.array([[0, 10, 1], [1, 0, inputs.INF_I32], [inputs.INF_I32, 2, 0]], np.int32))
    assert d[0, 1] == 3 and via[0, 1] == 0 and via[0, 2] == -1


def test_paths_bad_arguments():
    t = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    v = torch.zeros((8, 8), dtype=torch.int16, device="cuda")
    L = binding.lib()
    opt = binding.Options(0, 0, None, 0, None, 0)
    assert L.apsp_fw_paths(t.data_ptr(), None, 8, 8, 8, binding.APSP_I32, opt, None) == binding.APSP_EINVAL
    assert L.apsp_fw_paths(t.data_ptr(), v.data_ptr(), 8, 8, 7, binding.APSP_I32, opt, None) == binding.APSP_EINVAL
    assert L.apsp_fw_paths(t.data_ptr(), v.data_ptr(), 8, 8, 8, 9, opt, None) == binding.APSP_EINVAL
