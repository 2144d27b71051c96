"""The allocation-free fp32 entry point, apsp_fw_f32_noalloc.

It exists for callers that may not allocate device memory while solving: a
plugin whose host framework owns every byte of device memory through its own
pool, or a latency-critical service that cannot absorb cudaMalloc / cudaFree
(either can fail mid-request under a fixed budget, and cudaFree synchronizes
the device).  Its scratch is one static device array shared by every call, so
these checks run it several times in a row -- each call starts from the
previous call's leftovers in the array -- and require each result to equal
apsp_fw's plain schedule bit for bit (both run the same kernels, k-block and
per-element operation order).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_1001_4108_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32_RTOL = 1e-5
ARRAY_MAX_N = 16384  # the static array holds one interleaved panel of 128 x 16384 floats


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    return binding.lib()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _noalloc(lib, t, n, ld):
    st = lib.apsp_fw_f32_noalloc(t.data_ptr(), n, ld, _stream())
    assert st == binding.APSP_OK, binding.lib().apsp_status_str(st)


def _plain(w, n):
    ref = torch.from_numpy(w).cuda()
    binding.apsp_fw(ref, n, flags=binding.FLAG_NO_LOOKAHEAD)
    return ref


def test_noalloc_equals_apsp_fw_on_consecutive_calls(lib):
    # k-block 128, then 64, then 128 again over the 64-deep leftovers
    cases = ((5000, 11, 128), (1500, 12, 64), (4700, 13, 128))
    for n, seed, kb in cases:
        assert binding.query_config(n, binding.APSP_F32).kblock == kb
        w = inputs.dense_f32(n, seed=seed)
        ref = _plain(w, n)
        t = torch.from_numpy(w).cuda()
        _noalloc(lib, t, n, n)
        torch.cuda.synchronize()
        assert torch.equal(t, ref), n
        if n == 1500:  # and against the FP64 oracle once
            d64 = oracle.fw_f64(w)
            d = t.cpu().numpy().astype(np.float64)
            assert (np.abs(d - d64) <= FP32_RTOL * np.abs(d64)).all()


def test_noalloc_at_the_array_limit(lib):
    # n = 16384 fills the array exactly (s = 128); n = 16300 is ragged in the
    # same range.  Each against apsp_fw bit for bit; the full one also against
    # exact (Dijkstra, FP64) rows of the oracle.
    for n in (ARRAY_MAX_N, 16300):
        cfg = binding.query_config(n, binding.APSP_F32)
        assert cfg.kblock == 128 and 128 * cfg.rounds * 128 == 128 * ARRAY_MAX_N
        w = inputs.dense_f32(n, seed=n)
        ref = _plain(w, n)
        t = torch.from_numpy(w).cuda()
        _noalloc(lib, t, n, n)
        torch.cuda.synchronize()
        assert torch.equal(t, ref), n
        del ref
        if n == ARRAY_MAX_N:
            rows = np.array([0, 9999, n - 1])
            exact = oracle.dijkstra_rows_f32(w, rows)
            d = t[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
            assert (np.abs(d - exact) <= FP32_RTOL * np.abs(exact)).all()
        del t
        torch.cuda.empty_cache()


def test_noalloc_unpacked_layout(lib):
    # rows of 4 * 1001 bytes are not 16-byte multiples: the unpacked kernels
    # run (no scratch); padding columns stay untouched
    n, ld = 1000, 1001
    w = inputs.dense_f32(n, seed=3, ld=ld)
    ref = _plain(w, n)
    t = torch.from_numpy(w).cuda()
    _noalloc(lib, t, n, ld)
    torch.cuda.synchronize()
    assert torch.equal(t, ref)
    assert (t[:, n:] == -7).all().item()


def test_noalloc_allocates_no_device_memory(lib):
    # after one warm-up call (module load, kernel attributes, the array's
    # address), further calls leave the device's free memory unchanged
    mats = []
    for n, seed in ((3000, 1), (700, 2), (5000, 3)):
        mats.append((n, torch.from_numpy(inputs.dense_f32(n, seed=seed)).cuda()))
    for n, t in mats:
        _noalloc(lib, t, n, n)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for n, t in mats:
            _noalloc(lib, t, n, n)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    t = torch.zeros(4, device="cuda")
    assert lib.apsp_fw_f32_noalloc(t.data_ptr(), ARRAY_MAX_N + 1, ARRAY_MAX_N + 1, _stream()) == \
        binding.APSP_EUNSUPPORTED
    assert lib.apsp_fw_f32_noalloc(t.data_ptr(), 10, 9, _stream()) == binding.APSP_EINVAL
    torch.cuda.synchronize()
    assert (t == 0).all().item()
