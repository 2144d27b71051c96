"""ctypes binding of libapsp (include/apsp.h): argument marshalling only.

Every computation happens in the CUDA library.  ``lib()`` loads the in-tree
``_lib/libapsp.so`` and raises if it is missing -- there is no fallback.
Torch tensors are accepted for convenience: their data pointer, row stride
and current CUDA stream are passed through unchanged.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libapsp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "apsp.h")

APSP_I32, APSP_F32, APSP_I16 = 0, 1, 2
APSP_OK, APSP_EINVAL, APSP_ENOMEM, APSP_EUNSUPPORTED, APSP_ECUDA = 0, 1, 2, 3, 4
APSP_ETIMEOUT, APSP_EBUSY, APSP_EPENDING, APSP_ENEGCYCLE = 5, 6, 7, 8
FLAG_NO_GRAPH, FLAG_GENERIC, FLAG_REVERSE_K, FLAG_NEGCYCLE, FLAG_NO_WORKSPACE = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_NO_LOOKAHEAD = 0x20
FLAG_VALIDATE = 0x40
FLAG_NARROW = 0x80
FLAG_ONE_LAUNCH = 0x100
EVENTS_PER_STAGE = 5
INF_I32 = 1 << 29
INF_I16 = 16383

# Every symbol include/apsp.h declares (checked by the tests).
EXPORTS = ["apsp_status_str", "apsp_version", "apsp_fw", "apsp_fw_ex", "apsp_fw_host",
           "apsp_workspace_bytes", "apsp_query_config", "apsp_device_error", "apsp_ubench_minplus",
           "apsp_fw_f32_noalloc", "apsp_fw_batched", "apsp_autotune", "apsp_tuning_save",
           "apsp_tuning_load", "apsp_server_create", "apsp_submit", "apsp_poll", "apsp_wait",
           "apsp_server_stats", "apsp_server_destroy", "apsp_fw_paths", "apsp_path", "apsp_selftest_wait"]


class Options(ctypes.Structure):
    _fields_ = [("kblock", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("events", ctypes.POINTER(ctypes.c_void_p)), ("n_events", ctypes.c_int64),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_int64)]


class Config(ctypes.Structure):
    _fields_ = [("kblock", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("phase3_tma", ctypes.c_int32), ("phase3_threads", ctypes.c_int32),
                ("phase3_relax_per_round", ctypes.c_int64), ("lookahead", ctypes.c_int32),
                ("strips", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("max_n", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("inflight", ctypes.c_int64), ("bytes_resident", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("graphs_per_s", ctypes.c_double)]


class ApspError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)}")


_lock = threading.Lock()
_lib = None
_path = LIB_PATH


def use_library(path: str):
    """Select another build of libapsp.so (a tuning variant) before first use."""
    global _path
    assert _lib is None, "library already loaded"
    _path = path


def lib() -> ctypes.CDLL:
    """Load libapsp.so (built by ``paper_1001_4108_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_path):
                raise RuntimeError(f"libapsp.so not built ({_path}); run "
                                   "`python -m paper_1001_4108_gb300.build`")
            L = ctypes.CDLL(_path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.apsp_status_str.argtypes = [i32]
            L.apsp_status_str.restype = ctypes.c_char_p
            L.apsp_version.restype = i32
            L.apsp_fw.argtypes = [vp, i64, i64, i32, vp]
            L.apsp_fw_ex.argtypes = [vp, i64, i64, i32, ctypes.POINTER(Options), vp]
            L.apsp_fw_host.argtypes = [vp, i64, i64, i32, vp]
            L.apsp_fw_f32_noalloc.argtypes = [vp, i64, i64, vp]
            L.apsp_fw_paths.argtypes = [vp, vp, i64, i64, i64, i32, ctypes.POINTER(Options), vp]
            L.apsp_path.argtypes = [vp, vp, i64, i64, i64, i32, ctypes.c_int32, i64, i64,
                                    ctypes.POINTER(ctypes.c_int64), i64, ctypes.POINTER(ctypes.c_int64)]
            L.apsp_autotune.argtypes = [i32, vp, ctypes.c_char_p, i64]
            L.apsp_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ServerConfig)]
            L.apsp_submit.argtypes = [vp, vp, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
            L.apsp_poll.argtypes = [vp, ctypes.c_uint64, vp, i64]
            L.apsp_wait.argtypes = [vp, ctypes.c_uint64, vp, i64, i64]
            L.apsp_server_stats.argtypes = [vp, ctypes.POINTER(Stats), i32]
            L.apsp_server_destroy.argtypes = [vp]
            L.apsp_tuning_save.argtypes = [ctypes.c_char_p]
            L.apsp_tuning_load.argtypes = [ctypes.c_char_p]
            L.apsp_fw_batched.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64), i64, i32, vp]
            L.apsp_query_config.argtypes = [i64, i32, ctypes.c_int32, ctypes.POINTER(Config)]
            L.apsp_workspace_bytes.argtypes = [i64, i32, ctypes.c_int32]
            L.apsp_workspace_bytes.restype = i64
            L.apsp_device_error.argtypes = [i32]
            L.apsp_selftest_wait.argtypes = [i64, vp]
            L.apsp_ubench_minplus.argtypes = [i32, i64, i32, i32, vp, vp, ctypes.POINTER(ctypes.c_double)]
            for name in EXPORTS:
                getattr(L, name).restype = getattr(L, name).restype or i32
            L.apsp_status_str.restype = ctypes.c_char_p
            _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().apsp_status_str(int(status)).decode()


def _check(status: int, what: str):
    if status != APSP_OK:
        raise ApspError(status, what)


def dtype_code(t) -> int:
    """Map a torch/numpy dtype (or its name) to apsp_dtype."""
    name = str(t).split(".")[-1]
    return {"int32": APSP_I32, "float32": APSP_F32, "int16": APSP_I16}[name]


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _matrix_args(d, n):
    """(ptr, n, ld, dtype) of a 2-D CUDA tensor whose leading n x n block is
    the matrix (row stride = ld, unit column stride)."""
    assert d.dim() == 2, "2-D matrix expected"
    n = d.shape[0] if n is None else n
    if n == 0:
        return d.data_ptr(), 0, 0, dtype_code(d.dtype)
    assert d.stride(1) == 1, "row-major matrix with unit column stride expected"
    assert d.shape[0] >= n and d.shape[1] >= n
    return d.data_ptr(), n, d.stride(0), dtype_code(d.dtype)


def apsp_fw(d, n: int | None = None, *, kblock: int = 0, flags: int = 0, events=None, stream=None,
            workspace=None):
    """In-place all-pairs shortest paths on a CUDA tensor (int32/float32/int16).
    ``workspace``: optional CUDA tensor used as the device workspace."""
    ptr, n, ld, dt = _matrix_args(d, n)
    s = _stream_handle(stream)
    if kblock == 0 and flags == 0 and events is None and workspace is None:
        _check(lib().apsp_fw(ptr, n, ld, dt, s), "apsp_fw")
        return d
    opt = Options(kblock, flags, None, 0, None, 0)
    if workspace is not None:
        opt.workspace = workspace.data_ptr()
        opt.workspace_bytes = workspace.numel() * workspace.element_size()
    if events is not None:
        handles = [e.cuda_event for e in events]
        if not all(handles):
            raise ValueError("events must be created (recorded once) before they are passed in")
        arr = (ctypes.c_void_p * len(events))(*handles)
        opt.events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
        opt.n_events = len(events)
    _check(lib().apsp_fw_ex(ptr, n, ld, dt, ctypes.byref(opt), s), "apsp_fw_ex")
    return d


def apsp_fw_paths(d, via, n: int | None = None, *, kblock: int = 0, flags: int = 0, stream=None):
    """apsp_fw plus the stage record: ``via`` is an int16 CUDA tensor (n x n or
    wider) that receives, per pair, the stage of the last improvement (-1:
    never improved).  Returns (d, via)."""
    import torch
    ptr, n, ld, dt = _matrix_args(d, n)
    assert via.is_cuda and via.dtype == torch.int16 and via.dim() == 2 and via.stride(1) == 1
    assert via.shape[0] >= n and via.shape[1] >= n
    opt = Options(kblock, flags, None, 0, None, 0)
    _check(lib().apsp_fw_paths(ptr, via.data_ptr(), n, ld, via.stride(0), dt, ctypes.byref(opt),
                               _stream_handle(stream)), "apsp_fw_paths")
    return d, via


def path(dist, via, i: int, j: int, kblock: int) -> list:
    """One shortest path i -> j (list of vertices; [] if unreachable) from
    host (numpy) copies of a solved matrix and its stage record."""
    import numpy as np
    assert dist.ndim == 2 and via.ndim == 2 and via.dtype == np.int16
    assert dist.strides[1] == dist.itemsize and via.strides[1] == 2
    n = dist.shape[0]
    cap = ctypes.c_int64(0)
    ln = ctypes.c_int64(0)
    args = (dist.ctypes.data, via.ctypes.data, n, dist.strides[0] // dist.itemsize, via.strides[0] // 2,
            dtype_code(dist.dtype), kblock, i, j)
    st = lib().apsp_path(*args, None, 0, ctypes.byref(ln))
    if st == APSP_OK and ln.value == 0:
        return []
    if st != APSP_ENOMEM:
        _check(st, "apsp_path")
    buf = (ctypes.c_int64 * ln.value)()
    _check(lib().apsp_path(*args, buf, ln.value, ctypes.byref(ln)), "apsp_path")
    return list(buf[:ln.value])


def apsp_fw_batched(mats, stream=None, ns=None):
    """Many graphs in one call: ``mats`` is a list of 2-D CUDA tensors of one
    dtype (each solved in place on its leading n x n block)."""
    if not mats:
        return mats
    ptrs, nn, lds, dts = [], [], [], set()
    for i, m in enumerate(mats):
        p, n, ld, dt = _matrix_args(m, None if ns is None else ns[i])
        ptrs.append(p); nn.append(n); lds.append(ld); dts.add(dt)
    assert len(dts) == 1, "one dtype per batch"
    cnt = len(mats)
    P = (ctypes.c_void_p * cnt)(*ptrs)
    N = (ctypes.c_int64 * cnt)(*nn)
    LD = (ctypes.c_int64 * cnt)(*lds)
    _check(lib().apsp_fw_batched(P, N, LD, cnt, dts.pop(), _stream_handle(stream)), "apsp_fw_batched")
    return mats


def apsp_fw_raw(ptr: int, n: int, ld: int, dtype: int, stream: int | None, opt: Options | None = None) -> int:
    """Direct call returning the status code (used by argument-check tests)."""
    if opt is None:
        return lib().apsp_fw(ptr, n, ld, dtype, stream)
    return lib().apsp_fw_ex(ptr, n, ld, dtype, ctypes.byref(opt), stream)


def apsp_fw_host(a, stream=None):
    """All-pairs shortest paths on a host (CPU) numpy array or torch tensor,
    in place, through the library's host entry point (H2D, solve, D2H)."""
    import numpy as np
    if isinstance(a, np.ndarray):
        assert a.ndim == 2 and a.strides[1] == a.itemsize
        n, ld, dt, ptr = a.shape[0], a.strides[0] // a.itemsize, dtype_code(a.dtype), a.ctypes.data
    else:
        assert not a.is_cuda and a.stride(1) == 1
        n, ld, dt, ptr = a.shape[0], a.stride(0), dtype_code(a.dtype), a.data_ptr()
    _check(lib().apsp_fw_host(ptr, n, ld, dt, _stream_handle(stream)), "apsp_fw_host")
    return a


def workspace_bytes(n: int, dtype, kblock: int = 0) -> int:
    dt = dtype if isinstance(dtype, int) else dtype_code(dtype)
    return int(lib().apsp_workspace_bytes(n, dt, kblock))


def autotune(dtype, stream=None) -> dict:
    """Time the batched kernel shapes and the k-block crossover on this GPU and
    use the winners from now on (see apsp_autotune).  Returns the report."""
    import json
    dt = dtype if isinstance(dtype, int) else dtype_code(dtype)
    buf = ctypes.create_string_buffer(1 << 14)
    _check(lib().apsp_autotune(dt, _stream_handle(stream), buf, len(buf)), "apsp_autotune")
    return json.loads(buf.value.decode())


def tuning_save(path: str):
    _check(lib().apsp_tuning_save(path.encode()), "apsp_tuning_save")


def tuning_load(path: str):
    _check(lib().apsp_tuning_load(path.encode()), "apsp_tuning_load")


def query_config(n: int, dtype, kblock: int = 0) -> Config:
    cfg = Config()
    dt = dtype if isinstance(dtype, int) else dtype_code(dtype)
    _check(lib().apsp_query_config(n, dt, kblock, ctypes.byref(cfg)), "apsp_query_config")
    return cfg


def device_error(reset: bool = True) -> int:
    return lib().apsp_device_error(1 if reset else 0)


def ubench(form: int, iters: int, sink, blocks: int = 0, threads: int = 256, stream=None) -> float:
    out = ctypes.c_double(0.0)
    _check(lib().apsp_ubench_minplus(form, iters, blocks, threads, sink.data_ptr(),
                                     _stream_handle(stream), ctypes.byref(out)), "apsp_ubench_minplus")
    return out.value


class Server:
    """Serving handle (apsp_server_*): submit host matrices, poll / wait for
    the distances.  Use as a context manager or call close()."""

    def __init__(self, device: int = 0, max_inflight: int = 64, hbm_budget_bytes: int = 8 << 30,
                 streams: int = 4, max_n: int = 16384):
        self._h = ctypes.c_void_p()
        cfg = ServerConfig(device, max_inflight, hbm_budget_bytes, streams, 0, max_n)
        _check(lib().apsp_server_create(ctypes.byref(self._h), ctypes.byref(cfg)), "apsp_server_create")
        self._shapes = {}

    def submit(self, a) -> int:
        """Queue a matrix -- a numpy array or a (CUDA or CPU) torch tensor,
        copied before return; returns the ticket."""
        import numpy as np
        t = ctypes.c_uint64()
        n = a.shape[0]
        if isinstance(a, np.ndarray):
            assert a.ndim == 2
            if n:
                assert a.strides[1] == a.itemsize, "row-major matrix with unit column stride expected"
            ptr, ld, dt = a.ctypes.data, (a.strides[0] // a.itemsize if n else 0), a.dtype
        else:
            assert a.dim() == 2 and (n == 0 or a.stride(1) == 1), "row-major matrix expected"
            ptr, ld, dt = a.data_ptr(), (a.stride(0) if n else 0), a.dtype
        _check(lib().apsp_submit(self._h, ptr, n, ld, dtype_code(dt), 0, ctypes.byref(t)), "apsp_submit")
        self._shapes[t.value] = (n, np.dtype(str(dt).split(".")[-1]))
        return t.value

    def _out(self, ticket, out):
        import numpy as np
        if out is not None:
            assert out.dim() == 2 and out.stride(1) == 1
            return out, out.data_ptr(), out.stride(0)
        n, dt = self._shapes[ticket]
        a = np.empty((n, n), dtype=dt)
        return a, a.ctypes.data, n

    def poll(self, ticket: int, out=None):
        """The result if finished, else None: a new numpy array, or `out` (a
        torch tensor in host or device memory) filled in place."""
        res, ptr, ld = self._out(ticket, out)
        st = lib().apsp_poll(self._h, ticket, ptr, ld)
        if st == APSP_EPENDING:
            return None
        self._shapes.pop(ticket, None)
        _check(st, "apsp_poll")
        return res

    def wait(self, ticket: int, timeout_s: float | None = None, out=None):
        res, ptr, ld = self._out(ticket, out)
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        st = lib().apsp_wait(self._h, ticket, ptr, ld, us)
        if st == APSP_ETIMEOUT:
            return None
        self._shapes.pop(ticket, None)
        _check(st, "apsp_wait")
        return res

    def stats(self, reset: bool = False) -> dict:
        s = Stats()
        _check(lib().apsp_server_stats(self._h, ctypes.byref(s), 1 if reset else 0), "apsp_server_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def close(self):
        if self._h:
            lib().apsp_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
