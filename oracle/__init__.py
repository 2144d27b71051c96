"""Oracle for all-pairs shortest paths -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations of what the GPU library
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` may import this package.  It shares no
code with the CUDA path and never imports it.

What is computed (Sec. 3.1, Fig. 1 of Lund & Smith): for a directed graph with
weights w_ij (infinity for a missing edge, 0 on the diagonal, no negative
cycle), d_ij = length of a shortest path from v_i to v_j.  The blocked method
of Sec. 3.2 (Fig. 2) is a reordering of the same relaxations, so for integer
weights it reaches exactly this result, and for fp32 weights it reaches it up
to the rounding of fp32 additions.

Functions
---------
fw_int(w, absent)        Fig. 1 in int64 with an explicit "infinity" flag.
fw_int32_conv(w32)       fw_int on the int32 I/O convention of the library
                         (absent edge = 2**29 on input, unreachable = 2**29
                         on output) -- the decoding/encoding is done here, the
                         arithmetic in int64 with flags.
fw_int16_conv(w16)       the same for the int16 convention (absent = 16383).
fw_f64(w)                Fig. 1 in double precision, +inf for a missing edge.
fw_f64_mt, fw_int32_conv_mt
                         the same loops with the rows of each iteration k
                         shared among host threads (all cores by default);
                         bit-identical to the single-thread forms.
bellman_ford_*           textbook single-source algorithm (independent pin).
dijkstra_rows_*          textbook single-source algorithm for non-negative
                         weights, on the stored input matrix (large-n rows).
brute_force_paths(...)   enumeration of all simple paths (n <= 8).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Input/output conventions of the library under test, restated here from its
# documented interface (not imported from it).
ABSENT_I32 = 1 << 29
ABSENT_I16 = 16383


def build(force: bool = False) -> str:
    """Compile fw_oracle.c into a shared library with plain gcc -O2."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_fw_i64.argtypes = [p, p, i64]
            lib.oracle_fw_f64.argtypes = [p, i64]
            lib.oracle_fw_i64_mt.argtypes = [p, p, i64, ctypes.c_int]
            lib.oracle_fw_i64_mt.restype = ctypes.c_int
            lib.oracle_fw_f64_mt.argtypes = [p, i64, ctypes.c_int]
            lib.oracle_fw_f64_mt.restype = ctypes.c_int
            lib.oracle_bellman_ford_i64.argtypes = [p, p, i64, i64, p, p]
            lib.oracle_bellman_ford_i64.restype = ctypes.c_int
            lib.oracle_bellman_ford_f64.argtypes = [p, i64, i64, p]
            lib.oracle_bellman_ford_f64.restype = ctypes.c_int
            lib.oracle_dijkstra_f32in.argtypes = [p, i64, i64, i64, p]
            lib.oracle_dijkstra_i32in.argtypes = [p, i64, i64, i64, ctypes.c_int32, p, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


# ---------------------------------------------------------------- Fig. 1 ---

def fw_int(w: np.ndarray, absent: np.ndarray):
    """Fig. 1 on integer weights.  Returns (d int64, unreachable bool)."""
    n = w.shape[0]
    d = np.ascontiguousarray(w, dtype=np.int64).copy()
    inf = np.ascontiguousarray(absent, dtype=np.uint8).copy()
    d[inf.astype(bool)] = 0
    if n:
        _load().oracle_fw_i64(_ptr(d), _ptr(inf), n)
    return d, inf.astype(bool)


def fw_int32_conv(w32: np.ndarray) -> np.ndarray:
    """Input: int32 n x n, 2**29 = missing edge.  Output: int32 distances,
    2**29 for every unreachable pair (the library's output convention)."""
    w32 = np.asarray(w32)
    d, unreach = fw_int(w32.astype(np.int64), w32 == ABSENT_I32)
    out = d.copy()
    out[unreach] = ABSENT_I32
    return out.astype(np.int32)


def fw_int16_conv(w16: np.ndarray) -> np.ndarray:
    """Input: int16 n x n, 16383 = missing edge.  Output: int16 distances,
    16383 for every unreachable pair."""
    w16 = np.asarray(w16)
    d, unreach = fw_int(w16.astype(np.int64), w16 == ABSENT_I16)
    out = d.copy()
    out[unreach] = ABSENT_I16
    return out.astype(np.int16)


def fw_f64(w: np.ndarray) -> np.ndarray:
    """Fig. 1 in double precision (+inf = missing edge).  Input is widened
    exactly to float64 (fp32 -> fp64 is exact)."""
    d = np.ascontiguousarray(w, dtype=np.float64).copy()
    if d.shape[0]:
        _load().oracle_fw_f64(_ptr(d), d.shape[0])
    return d


def fw_int32_conv_mt(w32: np.ndarray, threads: int = 0):
    """fw_int32_conv on `threads` host threads (0 = all cores).  Returns
    (distances, threads used)."""
    w32 = np.asarray(w32)
    n = w32.shape[0]
    absent = w32 == ABSENT_I32
    d = np.ascontiguousarray(w32, dtype=np.int64).copy()
    inf = np.ascontiguousarray(absent, dtype=np.uint8).copy()
    d[absent] = 0
    used = _load().oracle_fw_i64_mt(_ptr(d), _ptr(inf), n, int(threads)) if n else 1
    d[inf.astype(bool)] = ABSENT_I32
    return d.astype(np.int32), used


def fw_f64_mt(w: np.ndarray, threads: int = 0):
    """fw_f64 on `threads` host threads (0 = all cores).  Returns (distances,
    threads used)."""
    d = np.ascontiguousarray(w, dtype=np.float64).copy()
    used = _load().oracle_fw_f64_mt(_ptr(d), d.shape[0], int(threads)) if d.shape[0] else 1
    return d, used


# -------------------------------------------------- independent pins -------

def bellman_ford_int(w: np.ndarray, absent: np.ndarray, src: int):
    """Single-source Bellman-Ford.  Returns (dist int64, unreachable bool,
    negative_cycle bool)."""
    n = w.shape[0]
    wi = np.ascontiguousarray(w, dtype=np.int64)
    ab = np.ascontiguousarray(absent, dtype=np.uint8)
    dist = np.zeros(n, np.int64)
    unr = np.zeros(n, np.uint8)
    neg = _load().oracle_bellman_ford_i64(_ptr(wi), _ptr(ab), n, src, _ptr(dist), _ptr(unr))
    return dist, unr.astype(bool), bool(neg)


def bellman_ford_f64(w: np.ndarray, src: int):
    n = w.shape[0]
    wd = np.ascontiguousarray(w, dtype=np.float64)
    dist = np.zeros(n, np.float64)
    neg = _load().oracle_bellman_ford_f64(_ptr(wd), n, src, _ptr(dist))
    return dist, bool(neg)


def dijkstra_rows_f32(w32: np.ndarray, sources) -> np.ndarray:
    """Exact (fp64) shortest-path rows for the given sources of an fp32
    matrix with non-negative weights.  w32 may be a strided view (leading
    dimension = its row stride)."""
    w32 = np.asarray(w32)
    assert w32.dtype == np.float32 and w32.strides[1] == 4
    n = w32.shape[0]
    ld = w32.strides[0] // 4
    out = np.empty((len(sources), n), np.float64)
    lib = _load()
    for r, s in enumerate(sources):
        lib.oracle_dijkstra_f32in(w32.ctypes.data, n, ld, int(s), out[r].ctypes.data)
    return out


def dijkstra_rows_i32(w32: np.ndarray, sources) -> np.ndarray:
    """Exact rows for an int32 matrix (2**29 = missing edge, other weights
    >= 0), returned in the library's output convention (2**29 unreachable)."""
    w32 = np.asarray(w32)
    assert w32.dtype == np.int32 and w32.strides[1] == 4
    n = w32.shape[0]
    ld = w32.strides[0] // 4
    out = np.empty((len(sources), n), np.int32)
    lib = _load()
    dist = np.zeros(n, np.int64)
    unr = np.zeros(n, np.uint8)
    for r, s in enumerate(sources):
        lib.oracle_dijkstra_i32in(w32.ctypes.data, n, ld, int(s), ABSENT_I32,
                                  _ptr(dist), _ptr(unr))
        row = dist.copy()
        row[unr.astype(bool)] = ABSENT_I32
        out[r] = row.astype(np.int32)
    return out


def brute_force_paths(w: np.ndarray, absent: np.ndarray):
    """Shortest simple-path lengths by enumerating every simple path with a
    depth-first search (n <= 8).  With no negative cycle the shortest walk is a
    simple path, so this is the definition of d_ij (Sec. 3.1).  Returns
    (d as object array of Python numbers or None for unreachable)."""
    n = w.shape[0]
    assert n <= 8
    assert all(not absent[v, v] and w[v, v] == 0 for v in range(n)), "zero diagonal expected"
    zero = w.dtype.type(0)
    best = [[None] * n for _ in range(n)]
    for s in range(n):
        best[s][s] = zero  # the empty path; no negative cycle can beat it
        visited = [False] * n
        visited[s] = True

        def dfs(u, length):
            for v in range(n):
                if v == u or absent[u, v] or visited[v]:
                    continue
                cand = length + w[u, v]
                if best[s][v] is None or cand < best[s][v]:
                    best[s][v] = cand
                visited[v] = True
                dfs(v, cand)
                visited[v] = False

        dfs(s, zero)
    return best
