"""The C-ABI library loads and exports every symbol include/apsp.h declares;
host-side argument checks (no GPU work is issued by any call here)."""
import ctypes
import re

import pytest

from paper_1001_4108_gb300 import binding, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def _declared_functions():
    text = open(binding.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*APSP_API\s+(?:const\s+)?\w+\s*\*?\s*(apsp_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_what_binding_lists():
    assert _declared_functions() == sorted(binding.EXPORTS)


def test_every_declared_symbol_is_exported(L):
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_no_other_symbols_leak():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    apsp_syms = sorted({l.split()[-1] for l in out.splitlines() if " T apsp_" in l})
    assert apsp_syms == sorted(binding.EXPORTS)


def test_status_strings(L):
    assert binding.status_str(0) == "APSP_OK"
    assert binding.status_str(8) == "APSP_ENEGCYCLE"
    assert binding.status_str(99) == "APSP_UNKNOWN"
    assert L.apsp_version() >= 100


@pytest.mark.parametrize("ptr,n,ld,dt", [
    (0x1000, -1, 4, binding.APSP_I32),      # negative n
    (0x1000, 8, 7, binding.APSP_I32),       # ld < n
    (0, 8, 8, binding.APSP_F32),            # null matrix
    (0x1000, 8, 8, 7),                      # unknown dtype
])
def test_bad_arguments_rejected_synchronously(L, ptr, n, ld, dt):
    assert binding.apsp_fw_raw(ptr, n, ld, dt, None) == binding.APSP_EINVAL


def test_bad_kblock_rejected(L):
    opt = binding.Options(96, 0, None, 0)
    assert binding.apsp_fw_raw(0x1000, 8, 8, binding.APSP_I32, None, opt) == binding.APSP_EINVAL


def test_empty_matrix_is_a_noop(L):
    assert binding.apsp_fw_raw(0, 0, 0, binding.APSP_I32, None) == binding.APSP_OK


def test_query_config(L):
    c = binding.query_config(16384, binding.APSP_F32)
    assert c.kblock == 128 and c.rounds == 128 and c.phase3_tma == 1 and c.phase3_threads == 256
    assert c.phase3_relax_per_round == (16384 - 128) ** 2 * 128
    c = binding.query_config(1000, binding.APSP_I32)
    assert c.kblock == 64 and c.rounds == 16
    assert binding.query_config(4096, binding.APSP_F32).kblock == 64
    assert binding.query_config(4608, binding.APSP_F32).kblock == 128
    assert binding.query_config(4095, binding.APSP_I32).kblock == 64
    assert binding.query_config(4096, binding.APSP_I32).kblock == 128
    assert binding.query_config(5119, binding.APSP_I16).kblock == 64
    assert binding.query_config(5120, binding.APSP_I16).kblock == 128
    c = binding.query_config(1000, binding.APSP_I16, 128)
    assert c.kblock == 128 and c.rounds == 8 and c.phase3_tma == 1
    cfg = binding.Config()
    assert L.apsp_query_config(10, 1, 100, ctypes.byref(cfg)) == binding.APSP_EINVAL


def test_query_config_strips(L):
    # strips: s = 64 panel/cross launches of up to 48 (fp32) / 32 (int32) stages
    q = binding.query_config
    assert [q(n, binding.APSP_F32).strips for n in (64, 65, 1024, 3072, 3073, 4096, 16384)] == [0, 1, 1, 1, 0, 0, 0]
    assert [q(n, binding.APSP_I32).strips for n in (100, 2048, 2049, 4096)] == [1, 1, 0, 0]
    assert q(1024, binding.APSP_I16).strips == 0
    assert q(1024, binding.APSP_F32, 128).strips == 0


def test_batched_bad_arguments(L):
    import ctypes as C
    P = (C.c_void_p * 2)(0x1000, 0)
    N = (C.c_int64 * 2)(4, 4)
    LD = (C.c_int64 * 2)(4, 4)
    # second matrix is null with n > 0
    assert L.apsp_fw_batched(P, N, LD, 2, binding.APSP_I32, None) == binding.APSP_EINVAL
    assert L.apsp_fw_batched(P, N, LD, -1, binding.APSP_I32, None) == binding.APSP_EINVAL
    assert L.apsp_fw_batched(None, None, None, 0, binding.APSP_I32, None) == binding.APSP_OK


def test_tuning_file_validation(L, tmp_path):
    bad = tmp_path / "bad.txt"
    bad.write_text("apsp-tuning 1\ni32 kblock_crossover 4096 batch_variants 0 2 2 9 2 tuned 0\n")
    assert L.apsp_tuning_load(str(bad).encode()) == binding.APSP_EINVAL
    good = tmp_path / "good.txt"
    assert L.apsp_tuning_save(str(good).encode()) == binding.APSP_OK
    assert L.apsp_tuning_load(str(good).encode()) == binding.APSP_OK
    assert "batch_variants" in good.read_text()
    assert L.apsp_tuning_load(str(tmp_path / "missing.txt").encode()) == binding.APSP_EINVAL


def test_server_bad_config(L):
    h = ctypes.c_void_p()
    cfg = binding.ServerConfig(0, 0, 1 << 20, 0, 0, 1024)  # no slots
    assert L.apsp_server_create(ctypes.byref(h), ctypes.byref(cfg)) == binding.APSP_EINVAL
    cfg = binding.ServerConfig(0, 4, 0, 0, 0, 1024)  # no memory
    assert L.apsp_server_create(ctypes.byref(h), ctypes.byref(cfg)) == binding.APSP_EINVAL
    assert L.apsp_poll(None, 1, None, 0) == binding.APSP_EINVAL
    assert L.apsp_server_destroy(None) == binding.APSP_EINVAL
