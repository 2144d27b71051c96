"""Batched form (apsp_fw_batched): many graphs of uneven n in one persistent
launch.  Integer results must be bit-identical to the oracle and to one
apsp_fw call per graph; fp32 within the parity tolerance."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1001_4108_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
INF = inputs.INF_I32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    binding.lib()
    yield
    assert binding.device_error() == 0


def _to_gpu(ws):
    return [torch.from_numpy(np.ascontiguousarray(w)).cuda() for w in ws]


def test_c4_small_batch_vs_oracle():
    ws = inputs.c4_batch(48, seed=7)
    ts = _to_gpu(ws)
    binding.apsp_fw_batched(ts)
    torch.cuda.synchronize()
    for w, t in zip(ws, ts):
        np.testing.assert_array_equal(t.cpu().numpy(), oracle.fw_int32_conv(w))


def test_c4_full_batch_equals_per_graph_launches():
    ws = inputs.c4_batch(4096, seed=8)
    a = _to_gpu(ws)
    b = _to_gpu(ws)
    binding.apsp_fw_batched(a)
    for t in b:
        binding.apsp_fw(t)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # every one of the 4096 graphs against the oracle (Fig. 1, int64 with
    # infinity flags), spread over the host cores: the oracle call releases
    # the interpreter lock
    got = [x.cpu().numpy() for x in a]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        exp = list(ex.map(oracle.fw_int32_conv, ws))
    for k, (x, e) in enumerate(zip(got, exp)):
        np.testing.assert_array_equal(x, e, err_msg=f"graph {k} (n = {ws[k].shape[0]})")
    # replay (second call of the same batch runs its CUDA graph)
    c = _to_gpu(ws[:300])
    for _ in range(3):
        for t, w in zip(c, ws[:300]):
            t.copy_(torch.from_numpy(w))
        binding.apsp_fw_batched(c)
        torch.cuda.synchronize()
        for x, y in zip(c, b[:300]):
            assert torch.equal(x, y)


def test_mixed_sizes_and_dtypes():
    g = inputs.rng(9)
    ns = [0, 1, 2, 63, 64, 65, 200, 511, 512, 513, 700]
    ws = [inputs.int_graph(n, 0.2, 0, 1000, seed=int(g.integers(1 << 30)), potential_max=40) for n in ns]
    ts = _to_gpu(ws)
    binding.apsp_fw_batched(ts)
    torch.cuda.synchronize()
    for w, t in zip(ws, ts):
        np.testing.assert_array_equal(t.cpu().numpy(), oracle.fw_int32_conv(w))
    # fp32 (reweighted, negative edges) within tolerance
    fs = [inputs.dense_f32(n, seed=n, reweighted=True) for n in (17, 130, 300)]
    tf = _to_gpu([w for w, _ in fs])
    binding.apsp_fw_batched(tf)
    torch.cuda.synchronize()
    for (w, pot), t in zip(fs, tf):
        d64 = oracle.fw_f64(w)
        d0 = d64 - pot[:, None] + pot[None, :]
        err = np.abs(t.cpu().numpy().astype(np.float64) - d64)
        assert (err <= 1e-5 * np.maximum(np.abs(d64), np.abs(d0) + 2 * pot.max())).all()
    # int16
    hs = [inputs.c3(seed=n, n=n)[1] for n in (40, 256, 400)]
    th = _to_gpu(hs)
    binding.apsp_fw_batched(th)
    torch.cuda.synchronize()
    for w, t in zip(hs, th):
        np.testing.assert_array_equal(t.cpu().numpy(), oracle.fw_int16_conv(w))


def test_batched_padded_leading_dimension():
    ws = [inputs.int_graph(n, 0.3, 1, 100, seed=n, ld=n + 5) for n in (50, 129, 333)]
    ts = _to_gpu(ws)
    binding.apsp_fw_batched(ts, ns=[50, 129, 333])
    torch.cuda.synchronize()
    for w, t, n in zip(ws, ts, (50, 129, 333)):
        out = t.cpu().numpy()
        np.testing.assert_array_equal(out[:, :n], oracle.fw_int32_conv(np.ascontiguousarray(w[:, :n])))
        assert (out[:, n:] == -7).all()


def test_autotune_and_table_roundtrip(tmp_path):
    rep = binding.autotune(binding.APSP_I32)
    assert rep["dtype"] == "i32" and len(rep["batched"]) == 5 and len(rep["kblock"]) == 5
    assert all(0 <= b["best"] < 4 and len(b["ms"]) == 4 for b in rep["batched"])
    path = str(tmp_path / "tuning.txt")
    binding.tuning_save(path)
    binding.tuning_load(path)
    # results do not depend on the chosen shapes
    ws = inputs.c4_batch(40, seed=21)
    ts = _to_gpu(ws)
    binding.apsp_fw_batched(ts)
    torch.cuda.synchronize()
    for w, t in zip(ws, ts):
        np.testing.assert_array_equal(t.cpu().numpy(), oracle.fw_int32_conv(w))


def _force_variant(tmp_path, variant, dtypes=("i32", "f32", "i16")):
    """Writes and loads a tuning file that gives every n bucket of the given
    element types the batched shape `variant`; returns the saved table's path."""
    saved = str(tmp_path / "saved.txt")
    binding.tuning_save(saved)
    lines = open(saved).read().splitlines()
    forced = [lines[0]]
    for ln in lines[1:]:
        f = ln.split()
        if f[0] in dtypes:
            i = f.index("batch_variants")
            f[i + 1:i + 6] = [str(variant)] * 5
        forced.append(" ".join(f))
    path = str(tmp_path / "forced.txt")
    open(path, "w").write("\n".join(forced) + "\n")
    binding.tuning_load(path)
    return saved


@pytest.mark.parametrize("variant", [2])
def test_fp32_batched_s64_equals_single_graph(tmp_path, variant):
    """The s = 64 batched shape runs the stages of the single-graph path at
    s = 64 with the same per-element operations, so fp32 results are
    bit-identical to apsp_fw (what lets the server pick either kernel)."""
    saved = _force_variant(tmp_path, variant, ("f32",))
    try:
        g = inputs.rng(300 + variant)
        ns = [1, 5, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 300, 384, 449, 511, 512]
        fs = []
        for n in ns:
            w, _ = inputs.dense_f32(n, seed=int(g.integers(1 << 30)), reweighted=True)
            w[g.random((n, n)) < 0.5] = np.inf
            np.fill_diagonal(w, 0)
            fs.append(w)
        tb = _to_gpu(fs)
        binding.apsp_fw_batched(tb)
        ts = _to_gpu(fs)
        for t in ts:
            binding.apsp_fw(t)
        torch.cuda.synchronize()
        for n, x, y in zip(ns, tb, ts):
            assert torch.equal(x, y), n
    finally:
        binding.tuning_load(saved)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_each_batched_shape(tmp_path, variant):
    """Every kernel shape, forced through a tuning file for all n buckets,
    gives the oracle's result (graphs of all buckets, ragged and whole tiles)."""
    saved = _force_variant(tmp_path, variant)
    try:
        g = inputs.rng(100 + variant)
        ns = [1, 17, 32, 63, 64, 100, 128, 129, 250, 256, 300, 448, 512]
        ws = [inputs.int_graph(n, 0.2, 0, 950, seed=int(g.integers(1 << 30)), potential_max=50) for n in ns]
        ts = _to_gpu(ws)
        binding.apsp_fw_batched(ts)
        torch.cuda.synchronize()
        for w, t in zip(ws, ts):
            np.testing.assert_array_equal(t.cpu().numpy(), oracle.fw_int32_conv(w))
        # padded rows: 16-byte multiples (vector copies) and not
        pads = [(130, 134), (260, 263), (333, 333), (70, 76)]
        wp = [inputs.int_graph(n, 0.2, 0, 950, seed=n + ld, potential_max=50, ld=ld) for n, ld in pads]
        tp = _to_gpu(wp)
        binding.apsp_fw_batched(tp, ns=[n for n, _ in pads])
        torch.cuda.synchronize()
        for (n, ld), w, t in zip(pads, wp, tp):
            out = t.cpu().numpy()
            np.testing.assert_array_equal(out[:, :n], oracle.fw_int32_conv(np.ascontiguousarray(w[:, :n])))
            assert (out[:, n:] == -7).all()
        fs = [inputs.dense_f32(n, seed=n) for n in (40, 200, 512)]
        tf = _to_gpu(fs)
        binding.apsp_fw_batched(tf)
        torch.cuda.synchronize()
        for w, t in zip(fs, tf):
            assert np.allclose(t.cpu().numpy(), oracle.fw_f64(w), rtol=1e-5, atol=0)
    finally:
        binding.tuning_load(saved)
