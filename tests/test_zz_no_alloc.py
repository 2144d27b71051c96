"""The allocation-free fp32 entry point, apsp_fw_f32_noalloc.

It exists for callers that may not allocate device memory while solving (a
plugin whose host framework owns all device memory, a latency-critical
service that cannot absorb cudaMalloc/cudaFree).  Its scratch is a static
device array shared by every call, so these checks run it several times in a
row — the later calls start from the earlier calls' leftovers — and compare
each result with apsp_fw's, within the fp32 tolerance the parity tests use.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1001_4108_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32_RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    return binding.lib()


def _close(a, ref):
    a = a.astype(np.float64)
    ref = ref.astype(np.float64)
    assert np.array_equal(np.isinf(a), np.isinf(ref))
    fin = np.isfinite(ref)
    assert (np.abs(a[fin] - ref[fin]) <= FP32_RTOL * np.abs(ref[fin])).all()


def test_noalloc_matches_apsp_fw_on_consecutive_calls(lib):
    stream = torch.cuda.current_stream().cuda_stream
    # k-block 128, then 64, then 128 again over the previous calls' leftovers
    for n, seed in ((5000, 11), (1500, 12), (4100, 13)):
        w = inputs.dense_f32(n, seed=seed)
        ref = torch.from_numpy(w).cuda()
        binding.apsp_fw(ref)
        t = torch.from_numpy(w).cuda()
        assert lib.apsp_fw_f32_noalloc(t.data_ptr(), n, n, stream) == binding.APSP_OK
        torch.cuda.synchronize()
        _close(t.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    t = torch.zeros(4, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.apsp_fw_f32_noalloc(t.data_ptr(), 16385, 16385, stream) == binding.APSP_EUNSUPPORTED
    assert lib.apsp_fw_f32_noalloc(t.data_ptr(), 10, 9, stream) == binding.APSP_EINVAL
    assert (t == 0).all().item()
