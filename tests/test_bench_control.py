"""Control flow of bench.py's serving sweep with a fake server (no GPU): every
request is submitted, collected and timed, and the run ends."""
import threading
import time

import numpy as np

import bench


class FakeServer:
    """Solves nothing: returns the input after a short delay, like a server
    whose results arrive asynchronously."""

    def __init__(self):
        self._lock = threading.Lock()
        self._res = {}
        self._t = 0
        self._lat = []

    def submit(self, a):
        with self._lock:
            self._t += 1
            self._res[self._t] = (time.perf_counter(), a.copy())
            return self._t

    def wait(self, t, timeout_s=None):
        t0, a = self._res.pop(t)
        time.sleep(0.0005)
        self._lat.append((time.perf_counter() - t0) * 1e3)
        return a

    def stats(self):
        v = sorted(self._lat)
        return {"p50_ms": v[len(v) // 2], "p99_ms": v[-1], "graphs_per_s": 1000.0}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        pass


def test_serving_sweep_terminates_with_fake_server():
    r = bench.bench_serving(count=30, rates=(0.5, 1.0), server_factory=FakeServer,
                            solve_host=lambda a: a, time_limit_s=60)
    assert r["same_results_as_plain"] is True
    assert [s["fraction_of_saturation"] for s in r["sweep"]] == [0.5, 1.0]
    assert all(s["server"]["p99_ms"] >= s["server"]["p50_ms"] for s in r["sweep"])


def test_serving_surfaces_submit_errors():
    class Broken(FakeServer):
        def submit(self, a):
            raise RuntimeError("boom")
    try:
        bench.bench_serving(count=5, rates=(1.0,), server_factory=Broken, solve_host=lambda a: a, time_limit_s=30)
    except RuntimeError as e:
        assert "boom" in str(e)
    else:
        raise AssertionError("expected the submit error")


def test_cpu_baseline_all_cores_and_single_thread():
    # the oracle timed on every host core and on one thread, for each dtype
    for dt in ("f32", "i32", "i16"):
        r = bench.cpu_baseline(dt, n_sample=96)
        assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0
        assert r["single_thread"]["cores"] == 1 and r["single_thread"]["value"] > 0
