"""Serving form (apsp_server_*): continuous batching with admission by HBM
footprint.  Every result must be exactly what the same request gives alone
(the kernels depend only on (n, dtype)) and, for integers, what the oracle
gives."""
import threading
import time

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


def _mix(seed, count, nmax):
    return inputs.c5_requests(count, rate_hz=1000.0, seed=seed, nmin=8, nmax=nmax)


def test_results_same_alone_and_in_mix():
    reqs = _mix(1, 40, 1500)
    # alone: one request at a time
    alone = []
    with binding.Server(max_inflight=8) as srv:
        for r in reqs:
            alone.append(srv.wait(srv.submit(r.w)))
    # mix: all submitted together from two threads, collected out of order
    with binding.Server(max_inflight=16) as srv:
        tickets = [None] * len(reqs)

        def sub(idx):
            for i in idx:
                tickets[i] = srv.submit(reqs[i].w)
        th = [threading.Thread(target=sub, args=(range(k, len(reqs), 2),)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = {}
        while len(got) < len(reqs):
            for i, t in enumerate(tickets):
                if i not in got:
                    out = srv.poll(t)
                    if out is not None:
                        got[i] = out
            time.sleep(0.001)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0
    for i, r in enumerate(reqs):
        np.testing.assert_array_equal(got[i], alone[i])
        if r.dtype == "i32" and r.n <= 600:
            np.testing.assert_array_equal(got[i], oracle.fw_int32_conv(r.w))
        if r.dtype == "f32" and r.n <= 600:
            d64 = oracle.fw_f64(r.w)
            assert (np.abs(got[i].astype(np.float64) - d64) <= 1e-5 * np.abs(d64)).all()


def test_admission_respects_hbm_budget():
    n = 700
    w = inputs.int_graph(n, 0.1, 1, 100, seed=3)
    per = n * 704 * 4  # device rows padded to 16 bytes
    budget = int(per * 2.5)
    with binding.Server(max_inflight=64, hbm_budget_bytes=budget) as srv:
        tickets = [srv.submit(w) for _ in range(12)]
        peak = 0
        while True:
            st = srv.stats()
            peak = max(peak, st["bytes_resident"])
            if st["completed"] == 12:
                break
            time.sleep(0.0005)
        assert 0 < peak <= budget
        ref = oracle.fw_int32_conv(w)
        for t in tickets:
            np.testing.assert_array_equal(srv.wait(t), ref)
        with pytest.raises(binding.ApspError) as e:
            srv.submit(inputs.int_graph(1200, 0.1, 1, 100, seed=4))  # larger than the whole budget
        assert e.value.status == binding.APSP_ENOMEM


def test_poll_pending_and_wait_timeout():
    big = inputs.dense_f32(6144, seed=5)
    with binding.Server() as srv:
        t = srv.submit(big)
        assert srv.poll(t) is None or True  # may already be done on a fast GPU
        out = srv.wait(t, timeout_s=60)
        assert out is not None and out.shape == (6144, 6144)
        t2 = srv.submit(big)
        assert srv.wait(t2, timeout_s=0) is None  # still running
        assert srv.wait(t2) is not None
        # empty matrix completes at once
        assert srv.wait(srv.submit(np.zeros((0, 0), np.int32))).shape == (0, 0)


def test_device_matrices_in_and_out():
    # a request may come from device memory and be delivered into device
    # memory (or host memory); same values as a solve in place
    reqs = [inputs.c1(seed=2, n=300), inputs.dense_f32(700, seed=3), inputs.int_graph(1500, 0.05, 1, 100, seed=4)]
    with binding.Server(max_inflight=8) as srv:
        for w in reqs:
            src = torch.from_numpy(w).cuda()
            ref = src.clone()
            binding.apsp_fw(ref)
            t = srv.submit(src)
            src.fill_(0)  # the server copied it before submit returned
            out = torch.empty_like(ref)
            assert srv.wait(t, out=out) is out
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
            t2 = srv.submit(ref.cpu())  # a host tensor, delivered into a host tensor
            out_h = torch.empty(ref.shape, dtype=ref.dtype)
            srv.wait(t2, out=out_h)
            assert torch.equal(out_h, ref.cpu())
