"""Parity of the CUDA path (through the C ABI) with the oracle.

int32 / int16: bit-exact.  fp32: |d_gpu - d_64| <= 1e-5 * max(|d_64|, S_ij)
where S_ij bounds the sum of |w| along a shortest path (for non-negative
weights S_ij = d_64; for the reweighted graphs the sum of |w'| along the path
is at most d_0 + 2 * max p, d_0 the distance before reweighting).  fp32 with
integer-valued weights and path sums < 2^24 is bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1001_4108_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

INF = inputs.INF_I32
FP32_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    binding.lib()
    yield
    assert binding.device_error() == 0


def gpu_solve(w: np.ndarray, n=None, **kw) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    binding.apsp_fw(t, n, **kw)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_fp32_close(d_gpu, d64, scale=None):
    d_gpu = d_gpu.astype(np.float64)
    assert np.array_equal(np.isinf(d_gpu), np.isinf(d64))
    fin = np.isfinite(d64)
    s = np.abs(d64) if scale is None else np.maximum(np.abs(d64), scale)
    err = np.abs(d_gpu[fin] - d64[fin])
    bound = FP32_RTOL * s[fin]
    worst = np.max(err - bound) if err.size else -1
    assert worst <= 0, f"max excess {worst}"


# ------------------------------------------------------------------ int32 ---

@pytest.mark.parametrize("seed", [0, 1])
def test_c1_int32_exact(seed):
    w = inputs.c1(seed=seed)
    np.testing.assert_array_equal(gpu_solve(w), oracle.fw_int32_conv(w))


@pytest.mark.parametrize("n", [1, 2, 31, 33, 63, 64, 65, 127, 128, 129, 200, 257, 1000])
@pytest.mark.parametrize("kblock", [64, 128])
def test_ragged_int32_negative_weights(n, kblock):
    w = inputs.int_graph(n, 0.2, 0, 1000, seed=n, potential_max=50)
    np.testing.assert_array_equal(gpu_solve(w, kblock=kblock), oracle.fw_int32_conv(w))


@pytest.mark.parametrize("n,ld", [(100, 104), (300, 301), (129, 160), (513, 515)])
def test_leading_dimension_and_poison(n, ld):
    # ld*4 % 16 != 0 for odd ld: the generic phase-3 kernel runs
    w = inputs.int_graph(n, 0.3, 1, 1000, seed=ld, ld=ld)
    out = gpu_solve(w, n)
    np.testing.assert_array_equal(out[:, :n], oracle.fw_int32_conv(np.ascontiguousarray(w[:, :n])))
    assert (out[:, n:] == -7).all(), "padding columns beyond n were written"


def test_int32_unreachable_and_clamp():
    # two components, one of them with negative edges: unreachable pairs must
    # come back as exactly 2^29 (clamped), reachable ones exact
    n = 300
    w = inputs.int_graph(n, 0.05, 0, 1000, seed=5, potential_max=200)
    w[:150, 150:] = INF
    d = gpu_solve(w)
    np.testing.assert_array_equal(d, oracle.fw_int32_conv(w))
    assert (d[:150, 150:] == INF).all()


def test_generic_equals_tma_int32():
    w = inputs.c1(seed=3)
    a = gpu_solve(w)
    b = gpu_solve(w, flags=binding.FLAG_GENERIC)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_phase3_order_independence(dt):
    # Sec. 3.2: the tasks of a doubly dependent block may run in any order.
    # Reversing the k order inside phase 3 must give bit-identical results.
    if dt == "i32":
        w = inputs.int_graph(700, 0.2, 0, 1000, seed=9, potential_max=30)
    else:
        w = inputs.dense_f32(700, seed=9)
    for kb in (64, 128):
        a = gpu_solve(w, kblock=kb)
        b = gpu_solve(w, kblock=kb, flags=binding.FLAG_REVERSE_K)
        c = gpu_solve(w, kblock=kb, flags=binding.FLAG_REVERSE_K | binding.FLAG_GENERIC)
        assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("n,kb", [(700, 64), (1000, 128), (2048, 128)])
def test_fp32_packed_equals_unpacked(n, kb):
    # packed f32x2 + min3 phase 3 (workspace) vs one-k-at-a-time phase 3
    w = inputs.dense_f32(n, seed=n)
    a = gpu_solve(w, kblock=kb)
    b = gpu_solve(w, kblock=kb, flags=binding.FLAG_NO_WORKSPACE)
    c = gpu_solve(w, kblock=kb, flags=binding.FLAG_GENERIC)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_fp32_user_workspace():
    n = 900
    w, _ = inputs.dense_f32(n, seed=5, reweighted=True)
    nbytes = binding.workspace_bytes(n, binding.APSP_F32)
    assert nbytes == 2 * 64 * 960 * 4  # 15 stages: two panel buffers (lookahead)
    ref = gpu_solve(w, flags=binding.FLAG_NO_WORKSPACE)
    for size in (nbytes, nbytes // 2):  # lookahead, plain schedule
        ws = torch.full((size // 4,), float("nan"), device="cuda")
        t = torch.from_numpy(w).cuda()
        binding.apsp_fw(t, workspace=ws)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), ref)
    small = torch.empty(nbytes // 8 - 1, device="cuda")
    opt = binding.Options(0, 0, None, 0, small.data_ptr(), small.numel() * 4)
    assert binding.apsp_fw_raw(t.data_ptr(), n, n, binding.APSP_F32, None, opt) == binding.APSP_EINVAL


def test_graph_replay_same_buffer():
    w = inputs.c1(seed=4, n=520)
    exp = oracle.fw_int32_conv(w)
    src = torch.from_numpy(w).cuda()
    t = torch.empty_like(src)
    for _ in range(4):  # direct launch, capture, replay, replay
        t.copy_(src)
        binding.apsp_fw(t)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), exp)


def test_capture_into_user_graph():
    w = inputs.c1(seed=6, n=300)
    src = torch.from_numpy(w).cuda()
    t = src.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        binding.apsp_fw(t, stream=s)
    t.copy_(src)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(t.cpu().numpy(), oracle.fw_int32_conv(w))


# ------------------------------------------------ closed forms on the GPU ---

@pytest.mark.parametrize("n", [300, 1100])
def test_closed_forms_on_gpu(n):
    # results the definition fixes without any oracle: a complete graph with
    # all weights c (d_ij = c), the directed cycle 0 -> 1 -> ... -> n-1 -> 0
    # with unit weights (d_ij = (j - i) mod n) and the chain with weights
    # w_i,i+1 = i + 1 (d_ij = prefix-sum difference for i < j, unreachable
    # backwards), in int32, fp32 (integer-valued: exact) and int16
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cases = []
    w = np.full((n, n), 7, np.int32)
    np.fill_diagonal(w, 0)
    cases.append((w, np.where(i == j, 0, 7)))
    w = np.full((n, n), inputs.INF_I32, np.int32)
    np.fill_diagonal(w, 0)
    w[np.arange(n), (np.arange(n) + 1) % n] = 1
    cases.append((w, (j - i) % n))
    w = np.full((n, n), inputs.INF_I32, np.int32)
    np.fill_diagonal(w, 0)
    w[np.arange(n - 1), np.arange(1, n)] = np.arange(1, n)
    pre = np.concatenate([[0], np.cumsum(np.arange(1, n))])
    cases.append((w, np.where(j >= i, pre[j] - pre[i], inputs.INF_I32)))
    for w, exp in cases:
        np.testing.assert_array_equal(gpu_solve(w), exp)
        f = np.where(w >= inputs.INF_I32, np.inf, w).astype(np.float32)
        ef = np.where(exp >= inputs.INF_I32, np.inf, exp).astype(np.float32)
        np.testing.assert_array_equal(gpu_solve(f), ef)  # integer sums < 2^24: exact
        if exp[exp < inputs.INF_I32].max() < inputs.INF_I16:
            np.testing.assert_array_equal(gpu_solve(inputs.to_int16(w)),
                                          np.where(exp >= inputs.INF_I32, inputs.INF_I16, exp).astype(np.int16))


# --------------------------------------------------- lookahead schedule ---

def _graph(dt, n, seed):
    if dt == "f32":
        return inputs.dense_f32(n, seed=seed)
    w = inputs.int_graph(n, 0.2, 0, 1000, seed=seed, potential_max=40)
    return inputs.to_int16(w) if dt == "i16" else w


def _oracle(dt, w):
    return {"f32": oracle.fw_f64, "i32": oracle.fw_int32_conv, "i16": oracle.fw_int16_conv}[dt](w)


@pytest.mark.parametrize("dt", ["f32", "i32", "i16"])
@pytest.mark.parametrize("n,kb", [(192, 64), (200, 64), (512, 64), (1100, 64), (9 * 128 + 37, 128), (8 * 128, 128),
                                  (8 * 128 + 1, 128)])
def test_lookahead_equals_plain(dt, n, kb):
    # The lookahead schedule reorders independent phase-3 tiles and overlaps
    # phases 1-2 of stage b+1 with them; results are bit-identical to the
    # plain schedule (and, for the integers, to the oracle).  The sizes cover
    # a ragged last stage whose row/column is the lookahead's cross.
    w = _graph(dt, n, seed=n + kb)
    cfg = binding.query_config(n, binding.dtype_code(w.dtype), kb)
    assert cfg.lookahead == 1
    a = gpu_solve(w, kblock=kb)
    b = gpu_solve(w, kblock=kb, flags=binding.FLAG_NO_LOOKAHEAD)
    c = gpu_solve(w, kblock=kb, flags=binding.FLAG_REVERSE_K | binding.FLAG_NO_GRAPH)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    if dt == "f32":
        assert_fp32_close(a, oracle.fw_f64(w))
    else:
        np.testing.assert_array_equal(a, _oracle(dt, w))


@pytest.mark.parametrize("dt", ["f32", "i32", "i16"])
@pytest.mark.parametrize("n", [65, 128, 129, 300, 640, 1000, 1024, 1500, 2047, 2048])
def test_one_launch_equals_multi_launch(dt, n):
    """APSP_FLAG_ONE_LAUNCH: every stage in one cooperative launch (tiles
    spread over the CTAs, ordered by per-tile flags).  Bit-identical to the
    multi-launch schedules, and to the oracle for the integers.  Stage counts
    2 to 32, whole and ragged; direct, library graph and a user's capture."""
    w = _graph(dt, n, seed=n + 7)
    cfg = binding.query_config(n, binding.dtype_code(w.dtype))
    assert cfg.kblock == 64 and 2 <= cfg.rounds <= 32
    F = binding.FLAG_ONE_LAUNCH
    one = gpu_solve(w, flags=F | binding.FLAG_NO_GRAPH)
    multi = gpu_solve(w)
    plain = gpu_solve(w, flags=binding.FLAG_NO_LOOKAHEAD)
    assert np.array_equal(one, multi) and np.array_equal(one, plain)
    if dt == "f32":
        if n <= 1024:
            assert_fp32_close(one, oracle.fw_f64(w))
    else:
        np.testing.assert_array_equal(one, _oracle(dt, w))
    src = torch.from_numpy(w).cuda()
    t = torch.empty_like(src)
    for _ in range(3):  # direct, captured graph, replay
        t.copy_(src)
        binding.apsp_fw(t, flags=F)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), one)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        binding.apsp_fw(t, stream=s, flags=F)
    t.copy_(src)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), one)
    assert binding.device_error() == 0


def test_one_launch_workspace_and_limits():
    # a caller workspace too small for the flags, or a size outside 2..32
    # stages: the multi-launch schedule runs, same result
    F = binding.FLAG_ONE_LAUNCH
    w = inputs.c1(seed=3, n=1000)
    ref = gpu_solve(w)
    np.testing.assert_array_equal(ref, oracle.fw_int32_conv(w))
    need = (3 * 16 * 16 + 16) * 4  # 16 stages
    for size in (need, need - 4):
        ws = torch.zeros(size // 4 + 1, dtype=torch.int32, device="cuda")
        t = torch.from_numpy(w).cuda()
        opt = binding.Options(0, F, None, 0, ws.data_ptr(), size)
        assert binding.apsp_fw_raw(t.data_ptr(), 1000, 1000, binding.APSP_I32,
                                   torch.cuda.current_stream().cuda_stream, opt) == binding.APSP_OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), ref)
    for n in (40, 2100):  # 1 stage, 33 stages
        x = inputs.int_graph(n, 0.05, 1, 1000, seed=n)
        np.testing.assert_array_equal(gpu_solve(x, flags=F), gpu_solve(x))


def test_lookahead_graph_replay_and_user_capture():
    n = 1100
    w = _graph("i32", n, seed=3)
    exp = oracle.fw_int32_conv(w)
    src = torch.from_numpy(w).cuda()
    s = torch.cuda.Stream()
    t = torch.empty_like(src)
    with torch.cuda.stream(s):
        for _ in range(3):  # direct launch (creates the side stream of s), library graph, replay
            t.copy_(src)
            binding.apsp_fw(t, stream=s)
            s.synchronize()
            np.testing.assert_array_equal(t.cpu().numpy(), exp)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):  # the user's capture takes the fork/join too
        binding.apsp_fw(t, stream=s)
    for _ in range(2):
        t.copy_(src)
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), exp)


def test_lookahead_concurrent_streams():
    # two host threads solving on their own streams at once: each launching
    # stream has its own side stream, fork/join events and workspace
    import threading
    ws = [_graph("i32", 1100, seed=s) for s in (5, 6)]
    exp = [oracle.fw_int32_conv(w) for w in ws]
    errors = []

    def worker(k):
        try:
            s = torch.cuda.Stream()
            src = torch.from_numpy(ws[k]).cuda()
            t = torch.empty_like(src)
            for _ in range(3):  # direct, graph capture, replay
                with torch.cuda.stream(s):
                    t.copy_(src)
                    binding.apsp_fw(t, stream=s)
                s.synchronize()
                np.testing.assert_array_equal(t.cpu().numpy(), exp[k])
        except BaseException as e:  # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors


def _status(w, flags, n=None):
    t = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    n = w.shape[0] if n is None else n
    opt = binding.Options(0, flags, None, 0, None, 0)
    st = binding.apsp_fw_raw(t.data_ptr(), n, t.stride(0), binding.dtype_code(w.dtype),
                             torch.cuda.current_stream().cuda_stream, opt)
    torch.cuda.synchronize()
    return st, t.cpu().numpy()


def test_validate_flag():
    F = binding.FLAG_VALIDATE
    w = inputs.c1(seed=0)  # n = 1024, weights 1..1000: 1023 * 1000 < 2^28
    st, d = _status(w, F)
    assert st == binding.APSP_OK
    np.testing.assert_array_equal(d, oracle.fw_int32_conv(w))
    r = inputs.int_graph(700, 0.2, 0, 1000, seed=3, potential_max=50)  # negative weights within the bound
    assert _status(r, F)[0] == binding.APSP_OK
    for (i, j, v) in [(0, 1, 300000), (3, 4, (1 << 29) + 1), (5, 6, -300000)]:
        bad = w.copy()
        bad[i, j] = v
        st, d = _status(bad, F)
        assert st == binding.APSP_EINVAL, (i, j, v)
        assert np.array_equal(d, bad), "a refused input must be left untouched"
    h = inputs.to_int16(inputs.int_graph(500, 0.1, 1, 30, seed=4))  # 499 * 30 < 16383
    assert _status(h, F)[0] == binding.APSP_OK
    for v in (-1, 40, 20000):  # negative, over the bound, above infinity
        bad = h.copy()
        bad[2, 3] = v
        assert _status(bad, F)[0] == binding.APSP_EINVAL, v
    f = inputs.dense_f32(300, seed=2)
    assert _status(f, F)[0] == binding.APSP_OK
    bad = f.copy()
    bad[7, 8] = np.nan
    assert _status(bad, F)[0] == binding.APSP_EINVAL
    # synchronizing flags are refused inside a stream capture
    t = torch.from_numpy(w).cuda()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g, stream=s):
        opt = binding.Options(0, F, None, 0, None, 0)
        codes.append(binding.apsp_fw_raw(t.data_ptr(), 1024, 1024, binding.APSP_I32, s.cuda_stream, opt))
        opt = binding.Options(0, binding.FLAG_NEGCYCLE, None, 0, None, 0)
        codes.append(binding.apsp_fw_raw(t.data_ptr(), 1024, 1024, binding.APSP_I32, s.cuda_stream, opt))
        t.add_(0)  # the refused calls enqueue nothing: keep the captured graph non-empty
    assert codes == [binding.APSP_EINVAL, binding.APSP_EINVAL]


def test_narrow_int32_through_int16():
    # APSP_FLAG_NARROW: int32 in and out, solved by the int16x2 kernels;
    # identical to the int32 path and the oracle
    N, V = binding.FLAG_NARROW, binding.FLAG_VALIDATE
    w32, _ = inputs.c3(seed=1)  # n = 2048, weights 1..7: 2047 * 7 < 16383
    exp = oracle.fw_int32_conv(w32)
    for flags in (N, N | V, N | binding.FLAG_NO_GRAPH, N | binding.FLAG_NO_LOOKAHEAD):
        np.testing.assert_array_equal(gpu_solve(w32, flags=flags), exp)
    src = torch.from_numpy(w32).cuda()
    t = torch.empty_like(src)
    for _ in range(3):  # direct, captured graph, replay
        t.copy_(src)
        binding.apsp_fw(t, flags=N)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), exp)
    # ragged n, padded leading dimension, unreachable pairs
    w = inputs.int_graph(1001, 0.01, 1, 16, seed=8, ld=1004)
    out = gpu_solve(w, 1001, flags=N)
    np.testing.assert_array_equal(out[:, :1001], oracle.fw_int32_conv(np.ascontiguousarray(w[:, :1001])))
    assert (out[:, 1001:] == -7).all()
    # inputs outside the int16 rules are refused with the check, left untouched
    for bad in (inputs.c1(seed=0), inputs.int_graph(300, 0.2, 0, 10, seed=1, potential_max=3)):
        st, d = _status(bad, N | V)
        assert st == binding.APSP_EINVAL and np.array_equal(d, bad)
    via = torch.empty((2048, 2048), dtype=torch.int16, device="cuda")
    with pytest.raises(binding.ApspError):
        binding.apsp_fw_paths(torch.from_numpy(w32).cuda(), via, flags=N)


def test_bounded_wait_gives_up_without_fault():
    # a wait on a barrier phase that nothing completes runs out after 5 ms,
    # sets the device error word and returns; the context stays usable
    assert binding.device_error() == 0
    assert binding.lib().apsp_selftest_wait(5_000_000, None) == binding.APSP_OK
    assert binding.lib().apsp_device_error(1) == 1  # kDevTimeoutTma, then cleared
    assert binding.device_error() == 0
    w = inputs.c1(seed=2, n=600)
    np.testing.assert_array_equal(gpu_solve(w), oracle.fw_int32_conv(w))
    assert binding.lib().apsp_selftest_wait(0, None) == binding.APSP_EINVAL


def test_negative_cycle_flag():
    w = np.array([[0, 1, INF], [-3, 0, 1], [INF, INF, 0]], np.int32)
    t = torch.from_numpy(w).cuda()
    st = binding.apsp_fw_raw(t.data_ptr(), 3, 3, binding.APSP_I32, torch.cuda.current_stream().cuda_stream,
                             binding.Options(0, binding.FLAG_NEGCYCLE, None, 0))
    assert st == binding.APSP_ENEGCYCLE
    w2 = inputs.c1(seed=1, n=100)
    t2 = torch.from_numpy(w2).cuda()
    st = binding.apsp_fw_raw(t2.data_ptr(), 100, 100, binding.APSP_I32, torch.cuda.current_stream().cuda_stream,
                             binding.Options(0, binding.FLAG_NEGCYCLE, None, 0))
    assert st == binding.APSP_OK


# ------------------------------------------------------------------- fp32 ---

@pytest.mark.parametrize("n", [5, 64, 100, 129, 777])
def test_fp32_integer_weights_bit_exact(n):
    w = inputs.int_graph(n, 0.3, 1, 1000, seed=n)
    wf = np.where(w == INF, np.inf, w).astype(np.float32)
    d = gpu_solve(wf)
    exp = oracle.fw_int32_conv(w).astype(np.float64)
    exp[exp == INF] = np.inf
    np.testing.assert_array_equal(d.astype(np.float64), exp)


@pytest.mark.parametrize("n", [300, 2048])
def test_c2_dense_fp32(n):
    w = inputs.dense_f32(n, seed=n)
    assert_fp32_close(gpu_solve(w), oracle.fw_f64(w))


@pytest.mark.parametrize("n", [257, 1024])
def test_c2_reweighted_fp32(n):
    w, pot = inputs.dense_f32(n, seed=n + 1, reweighted=True)
    d64 = oracle.fw_f64(w)
    d0 = d64 - pot[:, None] + pot[None, :]
    scale = np.abs(d0) + 2 * pot.max()
    assert_fp32_close(gpu_solve(w), d64, scale)


_ORACLE_F64 = {}


def _fw_f64_all_cores(key, w):
    """Fig. 1 in FP64 on every host core (bit-identical to the single-thread
    form), cached per input for the cases that solve it more than once."""
    if key not in _ORACLE_F64:
        _ORACLE_F64[key] = oracle.fw_f64_mt(w)[0]
    return _ORACLE_F64[key]


@pytest.mark.parametrize("n", [2048, 4096])
@pytest.mark.parametrize("kblock", [0, 128])
def test_c2_reweighted_fp32_config_sizes(n, kblock):
    """The negative-edge variant of the fp32 workload (w' = w + p_u - p_v) at
    its own sizes against the full FP64 oracle, on the default tile (s = 64
    here) and forced through the s = 128 packed kernels."""
    w, pot = inputs.dense_f32(n, seed=n + 2, reweighted=True)
    assert (w < 0).any()
    d64 = _fw_f64_all_cores(("rw", n), w)
    d0 = d64 - pot[:, None] + pot[None, :]
    cfg = binding.query_config(n, binding.APSP_F32, kblock)
    assert cfg.kblock == (kblock or 64)
    assert_fp32_close(gpu_solve(w, kblock=kblock), d64, np.abs(d0) + 2 * pot.max())


def test_c2_dense_fp32_n4096_full_oracle():
    n = 4096
    w = inputs.dense_f32(n, seed=n)
    assert_fp32_close(gpu_solve(w), _fw_f64_all_cores(("plain", n), w))


def _bellman_rows_f64(wt, t, rows):
    """best_ij = min(w_ij, min_k w_ik + d_kj) in FP64 for the given rows, on
    the device in column blocks (a checker of the property, not the product);
    best_ii is set to 0 (the empty path)."""
    n = t.shape[0]
    out = []
    for i in rows:
        best = wt[i].double()
        for k0 in range(0, n, 1024):
            cand = (wt[i, k0:k0 + 1024].double()[:, None] + t[k0:k0 + 1024].double()).min(0).values
            best = torch.minimum(best, cand)
        best[int(i)] = 0.0
        out.append(best.cpu().numpy())
    return np.stack(out)


def test_c2_dense_fp32_n8192_sampled():
    n = 8192
    w = inputs.dense_f32(n, seed=n)
    t = torch.from_numpy(w).cuda()
    binding.apsp_fw(t)
    torch.cuda.synchronize()
    rows = inputs.rng(81).choice(n, size=8, replace=False)
    d_rows = t[torch.from_numpy(rows).cuda()].cpu().numpy()
    exact = oracle.dijkstra_rows_f32(w, rows)
    assert_fp32_close(d_rows, exact)
    best = _bellman_rows_f64(torch.from_numpy(w).cuda(), t, rows[:2])
    assert (np.abs(d_rows[:2] - best) <= FP32_RTOL * np.abs(best)).all()
    assert (t.diagonal() == 0).all().item()


def test_c2_reweighted_fp32_full_size():
    """The negative-edge variant at n = 16384 on the bench's s = 128 packed
    kernels.  Exact rows come from the oracle's Dijkstra on the graph before
    reweighting (its weights are w' - p_u + p_v, exact, in (0,1]) and the
    closed form d'_ij = d_ij + p_i - p_j; the Bellman equation is checked on
    sampled rows, the triangle inequality on 10^6 triples, and the diagonal
    is 0.  Tolerance: 1e-5 * S_ij, S_ij = |d_ij| + 2 max p bounding the sum
    of |w'| along the path."""
    n = 16384
    w, pot = inputs.dense_f32(n, seed=3, reweighted=True)
    assert binding.query_config(n, binding.APSP_F32).kblock == 128
    t = torch.from_numpy(w).cuda()
    binding.apsp_fw(t)
    torch.cuda.synchronize()
    pmax = pot.max()
    rows = inputs.rng(82).choice(n, size=4, replace=False)
    w0 = (w.astype(np.float64) - pot[:, None] + pot[None, :]).astype(np.float32)
    assert w0[~np.eye(n, dtype=bool)].min() > 0
    d0_rows = oracle.dijkstra_rows_f32(w0, rows)
    del w0
    exact = d0_rows + pot[rows][:, None] - pot[None, :]
    d_rows = t[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_fp32_close(d_rows, exact, np.abs(d0_rows) + 2 * pmax)
    # Bellman equation: |d_ij - best_ij| <= 1e-5 (S_ij + max_k S_kj)
    best = _bellman_rows_f64(torch.from_numpy(w).cuda(), t, rows[:2])
    s_max = (t.double() - torch.from_numpy(pot).cuda()[:, None] + torch.from_numpy(pot).cuda()[None, :]).abs().max()
    s_max = float(s_max) + 2 * pmax
    s_row = np.abs(d0_rows[:2]) + 2 * pmax
    assert (np.abs(d_rows[:2].astype(np.float64) - best) <= FP32_RTOL * (s_row + s_max)).all()
    # triangle inequality on 10^6 sampled triples
    g = inputs.rng(83)
    i, j, k = (torch.from_numpy(g.integers(0, n, 1_000_000)).cuda() for _ in range(3))
    p = torch.from_numpy(pot).cuda()

    def scale(a, b):
        return (t[a, b].double() - p[a] + p[b]).abs() + 2 * pmax

    slack = FP32_RTOL * (scale(i, j) + scale(i, k) + scale(k, j))
    assert (t[i, j].double() <= t[i, k].double() + t[k, j].double() + slack).all().item()
    assert (t.diagonal() == 0).all().item()


# ------------------------------------------------------------------ int16 ---

@pytest.mark.parametrize("n", [1, 33, 130, 2048])
def test_c3_int16_exact(n):
    w32, w16 = inputs.c3(seed=n, n=n)
    d16 = gpu_solve(w16)
    d32 = gpu_solve(w32)
    np.testing.assert_array_equal(d16, oracle.fw_int16_conv(w16))
    np.testing.assert_array_equal(np.where(d16 == inputs.INF_I16, INF, d16.astype(np.int32)), d32)


@pytest.mark.parametrize("n,ld,kb", [(700, 704, 64), (1000, 1000, 128), (1030, 1032, 128), (2048, 2048, 128)])
def test_int16_packed_vs_generic_vs_oracle(n, ld, kb):
    # packed int16x2 DPX phases 2-3 (workspace) against the scalar kernels and the oracle
    w32 = inputs.int_graph(n, 0.1, 1, 7, seed=n + 3)
    w16 = np.full((n, ld), 5, np.int16)
    w16[:, :n] = inputs.to_int16(w32)
    a = gpu_solve(w16, n, kblock=kb)
    b = gpu_solve(w16, n, kblock=kb, flags=binding.FLAG_GENERIC)
    c = gpu_solve(w16, n, kblock=kb, flags=binding.FLAG_REVERSE_K)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(a[:, :n], oracle.fw_int16_conv(np.ascontiguousarray(w16[:, :n])))
    assert (a[:, n:] == 5).all()


def test_int16_large_vs_int32_and_dijkstra():
    n = 4096
    w32 = inputs.int_graph(n, 0.1, 1, 3, seed=41)
    w16 = inputs.to_int16(w32)
    d16 = gpu_solve(w16)
    d32 = gpu_solve(w32)
    np.testing.assert_array_equal(np.where(d16 == inputs.INF_I16, INF, d16.astype(np.int32)), d32)
    rows = [0, 1234, 4095]
    np.testing.assert_array_equal(d32[rows], oracle.dijkstra_rows_i32(w32, rows))


@pytest.mark.parametrize("n", [5200, 6144])
def test_int16_s128_bulk_odd_and_even_tile_counts(n):
    """s = 128 int16x2 phase 3 (deferred C tile, TMA ring) at odd and even
    tile counts per launch, ragged and whole: identical to the int32 path,
    to the reversed k order and to exact Dijkstra rows."""
    w32 = inputs.int_graph(n, 0.05, 1, 3, seed=n)
    w16 = inputs.to_int16(w32)
    assert binding.query_config(n, binding.APSP_I16).kblock == 128
    d16 = gpu_solve(w16)
    np.testing.assert_array_equal(gpu_solve(w16, flags=binding.FLAG_REVERSE_K), d16)
    d32 = gpu_solve(w32)
    np.testing.assert_array_equal(np.where(d16 == inputs.INF_I16, INF, d16.astype(np.int32)), d32)
    rows = [0, n // 2, n - 1]
    np.testing.assert_array_equal(d32[rows], oracle.dijkstra_rows_i32(w32, rows))


def test_int16_bench_workload_n16000():
    """The bench's int16x2 line at its own size (n = 16000, p = 0.1, unit
    weights: the largest weight bound with (n - 1) Wmax < 16383), in the
    launch configuration it times (s = 128, lookahead, library graph):
    every entry equal to the int32 path's on the same graph, and sampled rows
    equal to exact Dijkstra rows of the oracle."""
    n = 16000
    w32 = inputs.int_graph(n, 0.1, 1, max(1, 16382 // (n - 1)), seed=16000)
    w16 = inputs.to_int16(w32)
    cfg = binding.query_config(n, binding.APSP_I16)
    assert cfg.kblock == 128 and cfg.lookahead == 1
    d16 = gpu_solve(w16)
    d32 = gpu_solve(w32)
    np.testing.assert_array_equal(np.where(d16 == inputs.INF_I16, INF, d16.astype(np.int32)), d32)
    rows = [0, 7777, n - 1]
    np.testing.assert_array_equal(d32[rows], oracle.dijkstra_rows_i32(w32, rows))


# --------------------------------------------------------------- host path ---

def test_host_entry_point():
    w = inputs.int_graph(333, 0.2, 1, 1000, seed=2, ld=340)
    exp = oracle.fw_int32_conv(np.ascontiguousarray(w[:, :333]))
    a = w.copy()
    view = a[:, :333]
    binding.lib().apsp_fw_host(view.ctypes.data, 333, 340, binding.APSP_I32,
                               torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(a[:, :333], exp)
    assert (a[:, 333:] == -7).all()
    f = inputs.dense_f32(500, seed=3)  # rows padded to 504 on the device: pitched copies
    g = f.copy()
    binding.apsp_fw_host(g)
    assert_fp32_close(g, oracle.fw_f64(f))
    h = inputs.int_graph(520, 0.1, 1, 1000, seed=4)  # n a multiple of 8: one linear copy each way
    e = oracle.fw_int32_conv(h)
    binding.apsp_fw_host(h)
    np.testing.assert_array_equal(h, e)


@pytest.mark.parametrize("dt,n,ld", [("f32", 1024, 1024), ("i32", 768, 776), ("f32", 2048, 2048),
                                     ("i32", 1024, 1025), ("f32", 1000, 1000), ("i16", 1024, 1024)])
def test_host_entry_point_pinned(dt, n, ld):
    # Pinned host matrices: with whole tiles and 16-byte rows the first stage
    # reads its tiles from host memory and the last stage writes them back
    # (only the panels are copied); other layouts take the copying form.
    # Same results either way; padding columns untouched.
    if dt == "f32":
        w = inputs.dense_f32(n, seed=n, ld=ld)
    elif dt == "i32":
        w = inputs.int_graph(n, 0.1, 1, 1000, seed=n, ld=ld)
    else:
        w = inputs.to_int16(np.minimum(inputs.int_graph(n, 0.05, 1, 15, seed=n), inputs.INF_I32))
    h = torch.from_numpy(w).pin_memory()
    for _ in range(3):  # direct, captured graph, replay
        h.copy_(torch.from_numpy(w))
        binding.lib().apsp_fw_host(h.data_ptr(), n, ld, binding.dtype_code(w.dtype),
                                   torch.cuda.current_stream().cuda_stream)
        out = h.numpy()
        base = np.ascontiguousarray(w[:, :n])
        if dt == "f32":
            assert_fp32_close(out[:, :n], oracle.fw_f64(base))
        elif dt == "i32":
            np.testing.assert_array_equal(out[:, :n], oracle.fw_int32_conv(base))
        else:
            np.testing.assert_array_equal(out[:, :n], oracle.fw_int16_conv(base))
        if ld > n:
            assert (out[:, n:] == -7).all()
    # the pinned form equals the device solve bit for bit
    t = torch.from_numpy(w).cuda()
    binding.apsp_fw(t, n)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy()[:, :n], h.numpy()[:, :n])


# ------------------------------------------ both sides of the strip limit ---

@pytest.mark.parametrize("dt,n", [("f32", 3000), ("f32", 3072), ("f32", 3100), ("f32", 3136),
                                  ("i32", 2000), ("i32", 2048), ("i32", 2050), ("i32", 2112)])
def test_strip_limit_sizes(dt, n):
    """s = 64 solves on either side of the round count up to which the panel
    and cross launches run as strips (fp32: R <= 48, int32: R <= 32), whole
    and ragged: sampled rows against Dijkstra and the Bellman equation."""
    cfg = binding.query_config(n, binding.APSP_F32 if dt == "f32" else binding.APSP_I32)
    assert cfg.kblock == 64 and cfg.lookahead == 1
    assert cfg.strips == (cfg.rounds <= (48 if dt == "f32" else 32))
    if dt == "f32":
        w = inputs.dense_f32(n, seed=n)
        g0 = np.random.default_rng(n)
        w[g0.random((n, n)) < 0.9] = np.inf  # sparse: paths of several edges
        np.fill_diagonal(w, 0)
    else:
        w = inputs.int_graph(n, 0.05, 1, 1000, seed=n)
    t = torch.from_numpy(w).cuda()
    binding.apsp_fw(t)
    torch.cuda.synchronize()
    d = t.cpu().numpy()
    rows = inputs.rng(n).choice(n, size=24, replace=False)
    if dt == "f32":
        assert_fp32_close(d[rows], oracle.dijkstra_rows_f32(w, rows))
    else:
        np.testing.assert_array_equal(d[rows], oracle.dijkstra_rows_i32(w, rows))
    # Bellman equation d_ij = min(w_ij, min_k w_ik + d_kj) on three rows
    for i in rows[:3]:
        if dt == "f32":
            best = np.min(w[i].astype(np.float64)[:, None] + d.astype(np.float64), axis=0)
            best = np.minimum(best, w[i])
            best[i] = 0
            fin = np.isfinite(best)
            assert np.array_equal(np.isfinite(d[i]), fin)
            assert np.all(np.abs(d[i][fin] - best[fin]) <= FP32_RTOL * np.abs(best[fin]) + 1e-30)
        else:
            wi = w[i].astype(np.int64)
            dd = np.where(d < (1 << 28), d.astype(np.int64), 1 << 40)
            best = np.min(np.where(wi[:, None] < inputs.INF_I32, wi[:, None] + dd, 1 << 40), axis=0)
            best = np.minimum(best, np.where(wi < inputs.INF_I32, wi, 1 << 40))
            best[i] = 0
            best = np.where(best >= (1 << 28), inputs.INF_I32, best)
            np.testing.assert_array_equal(d[i], best)


# ------------------------------------------------------- full size, sampled ---

@pytest.mark.parametrize("dt,n", [("f32", 16384), ("i32", 16384), ("f32", 32768)])
def test_full_size_sampled(dt, n):
    """The bench's size (and the largest complete fp32 graph, n = 32768, 4 GiB):
    sampled rows against Dijkstra (exact), the Bellman equation
    d_ij = min(w_ij, min_k w_ik + d_kj) on sampled rows (with d_ii = 0 it
    holds only for the shortest-path matrix), and the triangle inequality on
    10^6 sampled triples."""
    if dt == "f32":
        w = inputs.dense_f32(n, seed=0)
    else:
        w = inputs.int_graph(n, 0.3, 1, 1000, seed=0)
    t = torch.from_numpy(w).cuda()
    binding.apsp_fw(t)
    torch.cuda.synchronize()
    g = inputs.rng(77)
    rows = g.choice(n, size=6 if n <= 16384 else 3, replace=False)
    d_rows = t[torch.from_numpy(rows).cuda()].cpu().numpy()
    if dt == "f32":
        exact = oracle.dijkstra_rows_f32(w, rows)
        assert_fp32_close(d_rows, exact)
    else:
        exact = oracle.dijkstra_rows_i32(w, rows)
        np.testing.assert_array_equal(d_rows, exact)
    # Bellman equation on two rows, in FP64 / int64 on the device (a checker, not the product)
    wt = torch.from_numpy(w).cuda()
    for i in rows[:2]:
        best = wt[i].double() if dt == "f32" else wt[i].long()
        for k0 in range(0, n, 1024):
            wk = wt[i, k0:k0 + 1024]
            dk = t[k0:k0 + 1024]
            if dt == "f32":
                cand = (wk.double()[:, None] + dk.double()).min(0).values
            else:
                fin = (wk < inputs.INF_I32)[:, None] & (dk < (1 << 28))
                cand = torch.where(fin, wk.long()[:, None] + dk.long(), torch.full_like(dk, 1 << 40, dtype=torch.long))
                cand = cand.min(0).values
            best = torch.minimum(best, cand)
        di = t[i].double() if dt == "f32" else t[i].long()
        if dt == "f32":
            assert torch.all((di - best).abs() <= 1e-5 * best.abs()).item()  # weights > 0: S_ij = d_ij
        else:
            best = torch.where(best >= (1 << 28), torch.full_like(best, inputs.INF_I32), best)
            best[i] = 0
            assert torch.equal(di, best)
    del wt
    # triangle inequality on 10^6 random triples (within fp32 rounding)
    i = torch.from_numpy(g.integers(0, n, 1_000_000)).cuda()
    j = torch.from_numpy(g.integers(0, n, 1_000_000)).cuda()
    k = torch.from_numpy(g.integers(0, n, 1_000_000)).cuda()
    dij = t[i, j].double().cpu().numpy()
    dik = t[i, k].double().cpu().numpy()
    dkj = t[k, j].double().cpu().numpy()
    slack = 1e-5 * (np.abs(dik) + np.abs(dkj)) if dt == "f32" else 0
    assert (dij <= dik + dkj + slack).all()
    assert (t.diagonal() == 0).all().item()


@pytest.mark.parametrize("n,flags", [(100, 0), (400, 0), (1100, 0), (1100, binding.FLAG_NO_LOOKAHEAD)])
def test_traced_events_per_phase(n, flags):
    # the tracing option records 5 events per stage: phase 1, phase 2 (start,
    # end) and the phase-3 launch on the call's stream (start, end)
    E = binding.EVENTS_PER_STAGE
    w = inputs.dense_f32(n, seed=12)
    t = torch.from_numpy(w).cuda()
    cfg = binding.query_config(n, binding.APSP_F32)
    lookahead = cfg.lookahead and not flags
    assert cfg.lookahead == (1 if cfg.rounds >= 3 else 0)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(E * cfg.rounds)]
    for e in evs:
        e.record()
    binding.apsp_fw(t, events=evs, flags=flags)
    torch.cuda.synchronize()

    def le(i, j):
        return evs[i].elapsed_time(evs[j]) >= 0

    R = cfg.rounds
    if not lookahead:  # one stream: every event in order
        assert all(le(i, i + 1) for i in range(len(evs) - 1))
    else:
        for r in range(R):
            assert le(E * r, E * r + 1) and le(E * r + 1, E * r + 2)   # phases 1, 2 of stage r
            assert le(E * r + 2, E * r + 3) and le(E * r + 3, E * r + 4)  # phase 3 after phase 2
            if r + 1 < R:
                assert le(E * r + 2, E * (r + 1))      # stage r+1 starts after phase 2 of stage r
                assert le(E * r + 4, E * (r + 1) + 3)  # phase-3 launches in stage order
    assert_fp32_close(t.cpu().numpy(), oracle.fw_f64(w))
