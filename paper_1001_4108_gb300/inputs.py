"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module only draws random graphs in the library's input conventions; it
holds none of the shortest-path arithmetic, so both the oracle side and the
CUDA side can take their inputs from here.

Conventions (the problem statement of Sec. 3.1: w_ij = infinity for a missing
edge, w_ii = 0, no negative cycle):
  * int32: a missing edge is stored as 2**29;
  * int16: a missing edge is stored as 16383;
  * fp32 : a missing edge is +inf.

The paper names no dataset and no generator (it only says "any graph with
single precision edge weights"), so the workloads are synthetic:

  c1   n=1024, each off-diagonal edge present with probability 0.3,
       int32 weights uniform in {1..1000}.
  c2   complete directed graph, fp32 weights uniform in (0,1] (= 1 - U[0,1)
       drawn in fp32), n in {2048 ... 32768}.  Variant ``reweighted``: integer
       multiples of 2**-23 for w and for potentials p_v in [0, 0.5], and
       w'_uv = w_uv + p_u - p_v, which is then exact in fp32 (|w'| < 2), so the
       graph has negative edges but no negative cycle.
  c3   n=2048, edge probability 0.1, int weights uniform in {1..7}
       ((n-1) * 7 = 14329 < 16383), in both int32 and int16 encodings.
  c4   batches of graphs with n uniform in {16..512}, edge probability 0.2,
       w = b + p_u - p_v with b uniform in {0..950} and integer potentials p_v
       uniform in {0..50} (weights in [-50, 1000], no negative cycle).
  c5   request streams: Poisson arrivals, n log-uniform in [32, 4096], half
       int32 (weights {1..1000}, edge probability uniform in [0.05, 0.5]) and
       half complete fp32 graphs with weights in (0,1].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

INF_I32 = 1 << 29
INF_I16 = 16383


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def int_graph(n: int, p: float, wlo: int, whi: int, seed: int, ld: int | None = None,
              potential_max: int = 0) -> np.ndarray:
    """Random directed graph, int32, missing edges = 2**29, diagonal 0.

    Each off-diagonal edge is present independently with probability p and
    gets a weight uniform in {wlo..whi}.  With potential_max > 0, integer
    potentials p_v uniform in {0..potential_max} are drawn and each present
    weight becomes w + p_u - p_v (no negative cycle can appear because every
    cycle keeps its original, non-negative sum).  With ld > n the rows are
    padded to ld columns; the padding holds a poison value (-7) that callers can
    check is left untouched."""
    g = rng(seed)
    ld = n if ld is None else ld
    present = g.random((n, n), dtype=np.float32) < np.float32(p)
    w = g.integers(wlo, whi + 1, size=(n, n), dtype=np.int32)
    if potential_max > 0:
        pot = g.integers(0, potential_max + 1, size=n, dtype=np.int32)
        w = w + pot[:, None] - pot[None, :]
    w = np.where(present, w, np.int32(INF_I32)).astype(np.int32)
    np.fill_diagonal(w, 0)
    if ld == n:
        return w
    out = np.full((n, ld), -7, np.int32)
    out[:, :n] = w
    return out


def dense_f32(n: int, seed: int, reweighted: bool = False, ld: int | None = None):
    """Complete directed fp32 graph.  Returns w (n x ld, float32) or, with
    reweighted=True, (w', p) where p are the float64 potentials."""
    g = rng(seed)
    ld = n if ld is None else ld
    if not reweighted:
        w = np.float32(1.0) - g.random((n, n), dtype=np.float32)
        np.fill_diagonal(w, 0.0)
        pot = None
    else:
        q = 2.0 ** -23
        k = g.integers(0, 1 << 23, size=(n, n), dtype=np.int64)
        m = g.integers(0, (1 << 22) + 1, size=n, dtype=np.int64)
        # all in integer units of 2**-23: w = 2**23 - k, p = m
        units = (1 << 23) - k + m[:, None] - m[None, :]
        w = (units.astype(np.float64) * q).astype(np.float32)
        np.fill_diagonal(w, 0.0)
        pot = m.astype(np.float64) * q
    if ld != n:
        out = np.full((n, ld), np.float32(-7.0), np.float32)
        out[:, :n] = w
        w = out
    return w if pot is None else (w, pot)


def c1(seed: int = 0, n: int = 1024) -> np.ndarray:
    return int_graph(n, 0.3, 1, 1000, seed)


def c3(seed: int = 0, n: int = 2048):
    """Returns (w32, w16): the same graph in both integer encodings."""
    w32 = int_graph(n, 0.1, 1, 7, seed)
    return w32, to_int16(w32)


def to_int16(w32: np.ndarray) -> np.ndarray:
    """Re-encode an int32 graph (2**29 = missing) as int16 (16383 = missing).
    Weights must already fit."""
    w16 = np.where(w32 == INF_I32, INF_I16, w32)
    assert w16.min() >= -16384 and w16.max() <= INF_I16
    return w16.astype(np.int16)


def c4_batch(count: int, seed: int, nmin: int = 16, nmax: int = 512, p: float = 0.2):
    """List of int32 graphs for the batched form (weights in [-50, 1000])."""
    g = rng(seed)
    ns = g.integers(nmin, nmax + 1, size=count)
    seeds = g.integers(0, 2 ** 62, size=count)
    return [int_graph(int(n), p, 0, 950, int(s), potential_max=50) for n, s in zip(ns, seeds)]


@dataclass
class Request:
    t_arrival: float   # seconds from the start of the stream
    n: int
    dtype: str         # "i32" or "f32"
    w: np.ndarray


def c5_requests(count: int, rate_hz: float, seed: int, nmin: int = 32, nmax: int = 4096):
    """Poisson request stream for the serving form."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for r in range(count):
        n = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
        s = int(g.integers(0, 2 ** 62))
        if r % 2 == 0:
            pe = float(g.uniform(0.05, 0.5))
            reqs.append(Request(float(t[r]), n, "i32", int_graph(n, pe, 1, 1000, s)))
        else:
            reqs.append(Request(float(t[r]), n, "f32", dense_f32(n, s)))
    return reqs
