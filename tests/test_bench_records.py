"""Host-side pieces of bench.py's JSON line (no GPU): the nvidia-smi clock
record and its per-step windows, the measured-traffic record, the whole-job
throughput."""
import json
import time

import bench


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = lines
    return s


def test_clock_record_and_step_windows():
    t = time.perf_counter()
    s = _sampler([
        (t + 0.0, "0, 2070, 2070, 610.5, 0x0, Not Active, Not Active, Not Active, Not Active"),
        (t + 0.2, "0, 1980, 2070, 640.0, 0x4, Not Active, Not Active, Not Active, Active"),
        (t + 0.4, "0, 2070, 2070, 655.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
        (t + 0.5, "not a sample"),
        (t + 0.6, "0, [N/A], 2070, 600.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
    ])
    # a step spanning the first two samples, one spanning the third, one with none
    assert s.window_mhz(t - 0.01, t + 0.25) == (2070 + 1980) / 2
    assert s.window_mhz(t + 0.3, t + 0.45) == 2070
    assert s.window_mhz(t + 0.7, t + 0.9) is None
    rec = s.stop()
    assert rec["samples"] == 3 and rec["sm_mhz"] == 2070 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["sw_power_cap"] and rec["power_w_max"] == 655.0


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler(0)
    rec = s.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_record_scales_by_tiles_and_tracks_sources():
    rec = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    f = rec["f32"]
    per_tile = f["bytes_per_launch"] / f["tiles_per_launch"]
    # each dtype's entry names the sources it was taken with and their hash
    for dt in ("f32", "i32", "i16"):
        assert tuple(rec[dt]["kernel_sources"]) == tuple(
            "paper_1001_4108_gb300/csrc/" + x for x in bench.KERNEL_SOURCES_BY_DTYPE[dt])
    if bench.kernel_source_hash("f32") == f["kernel_sources_sha256"]:
        got = bench._measured_traffic("f32", 16384, 128, 15876)
        assert abs(got - per_tile * 15876) < 1.0
        # the record is for s = 128 only; no figure for another tile side or a single-tile matrix
        assert bench._measured_traffic("f32", 4096, 64, 100) is None
        assert bench._measured_traffic("f32", 128, 128, 0) is None
    else:
        assert bench._measured_traffic("f32", 16384, 128, 15876) is None
    # C read + write once per stage is the floor the measured bytes are compared with
    assert per_tile <= 2 * 128 * 128 * 4 * 1.05


def test_job_value_is_whole_job_throughput():
    assert bench.job_value(10.0, 4, 2.0) == 20.0
    assert bench.job_value(8.0, 1, 0.5) == 16.0


def test_nvml_clock_record_and_fallback():
    c = bench.NvmlClock(0)
    if c._lib is None:  # no NVML here: every reading is None and the record says so
        assert c.read() == (None, None)
        rec = c.stop()
        assert rec["sm_mhz"] is None and rec["reasons"] == ["nvml unavailable"]
    # the record from planted samples: per-window medians and the slowdown bits
    c = bench.NvmlClock(0)
    c._lib = True  # as if loaded; no thread is started
    c.samples = [(1.0, 2070.0, 0x0), (2.0, 1980.0, 0x4), (3.0, None, None), (4.0, 2070.0, 0x1)]
    assert c.window_mhz(0.5, 2.5) == (2070.0 + 1980.0) / 2
    assert c.window_mhz(2.5, 3.5) is None
    rec = c.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]  # 0x1 (idle) is not a slowdown


def test_source_hash_ignores_comments_only():
    assert bench._code_only("int a; // note\n/* block\n comment */ int b;\n\n  // only a comment\n") == "int a;\n int b;"
    # a changed statement changes the code text, a changed comment does not
    assert bench._code_only("x = 1; // one") == bench._code_only("x = 1; // uno")
    assert bench._code_only("x = 1;") != bench._code_only("x = 2;")
