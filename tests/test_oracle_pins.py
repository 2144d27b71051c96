"""Pins of the oracle against facts that do not come from the oracle itself.

The paper prints no worked example and no distance values, so the pins are:
hand-derived fixtures (tests/golden), brute-force enumeration of simple paths,
two independent textbook algorithms (Bellman-Ford, Dijkstra), closed forms
(uniform complete graph, directed cycle, chain, empty graph), exact
invariances (vertex relabeling, potential reweighting) and the optimality
conditions of a distance matrix.  ``test_mutants_are_caught`` plants plausible
mistakes in a copy of Fig. 1 and checks that these pins reject each of them.
"""
import glob
import math
import os

import numpy as np
import pytest

import oracle
from paper_1001_4108_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = inputs.INF_I32


def _parse_golden(path):
    kind = n = None
    rows_in, rows_out, cur = [], [], None
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        if line.startswith("kind"):
            kind = line.split()[1]
        elif line.startswith("n "):
            n = int(line.split()[1])
        elif line == "input":
            cur = rows_in
        elif line == "expected":
            cur = rows_out
        else:
            cur.append(line.split())
    assert len(rows_in) == n and len(rows_out) == n
    return kind, n, rows_in, rows_out


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "g*.txt"))),
                         ids=lambda p: os.path.basename(p))
def test_golden_hand_derived(path):
    kind, n, rin, rout = _parse_golden(path)
    if kind == "int":
        w = np.array([[INF if t == "inf" else int(t) for t in r] for r in rin], np.int32)
        exp = np.array([[INF if t == "inf" else int(t) for t in r] for r in rout], np.int32)
        np.testing.assert_array_equal(oracle.fw_int32_conv(w), exp)
        # the flag-based entry point agrees on reachability and lengths
        d, unr = oracle.fw_int(w.astype(np.int64), w == INF)
        np.testing.assert_array_equal(unr, exp == INF)
        np.testing.assert_array_equal(d[~unr], exp[~unr])
        # the double-precision entry point on the same integer graph
        wf = np.where(w == INF, np.inf, w.astype(np.float64))
        ef = np.where(exp == INF, np.inf, exp.astype(np.float64))
        np.testing.assert_array_equal(oracle.fw_f64(wf), ef)
        # and the brute-force enumeration of simple paths
        bd, bunr = _brute_as_arrays(oracle.brute_force_paths(w.astype(np.int64), w == INF))
        np.testing.assert_array_equal(bunr, exp == INF)
        np.testing.assert_array_equal(bd[~bunr], exp[~bunr])
    else:
        w = np.array([[np.inf if t == "inf" else float(t) for t in r] for r in rin])
        exp = np.array([[np.inf if t == "inf" else float(t) for t in r] for r in rout])
        np.testing.assert_array_equal(oracle.fw_f64(w), exp)


# ------------------------------------------------------------ generators ---

def _rand_int_graph(g, n, p, lo, hi, pot):
    present = g.random((n, n)) < p
    w = g.integers(lo, hi + 1, size=(n, n)).astype(np.int64)
    if pot:
        pv = g.integers(0, pot + 1, size=n)
        w = w + pv[:, None] - pv[None, :]
    absent = ~present
    np.fill_diagonal(absent, False)
    np.fill_diagonal(w, 0)
    w[absent] = 0
    return w, absent


def _brute_as_arrays(best):
    n = len(best)
    d = np.zeros((n, n), np.int64)
    unr = np.zeros((n, n), bool)
    for i in range(n):
        for j in range(n):
            if best[i][j] is None:
                unr[i, j] = True
            else:
                d[i, j] = best[i][j]
    return d, unr


# ------------------------------------------------------------ brute force ---

def test_brute_force_int_negative_weights():
    g = inputs.rng(101)
    for trial in range(300):
        n = int(g.integers(1, 8))
        w, absent = _rand_int_graph(g, n, float(g.uniform(0.1, 0.9)), 0, 20, pot=int(g.integers(0, 15)))
        d, unr = oracle.fw_int(w, absent)
        bd, bunr = _brute_as_arrays(oracle.brute_force_paths(w, absent))
        np.testing.assert_array_equal(unr, bunr, err_msg=f"trial {trial}")
        np.testing.assert_array_equal(d[~unr], bd[~bunr], err_msg=f"trial {trial}")


def test_brute_force_real_dyadic():
    # dyadic weights (multiples of 1/64, |w| < 8): every path sum is exact, so
    # the comparison is exact whatever the order of the additions
    g = inputs.rng(102)
    for trial in range(200):
        n = int(g.integers(2, 8))
        pv = g.integers(0, 64, size=n) / 64.0
        w = g.integers(1, 256, size=(n, n)) / 64.0 + pv[:, None] - pv[None, :]
        absent = g.random((n, n)) > 0.6
        np.fill_diagonal(absent, False)
        np.fill_diagonal(w, 0.0)
        wf = np.where(absent, np.inf, w)
        d = oracle.fw_f64(wf)
        best = oracle.brute_force_paths(w, absent)
        for i in range(n):
            for j in range(n):
                exp = np.inf if best[i][j] is None else best[i][j]
                assert d[i, j] == exp, (trial, i, j)


# ------------------------------------------------ independent algorithms ---

@pytest.mark.parametrize("n", [1, 2, 17, 64, 97])
def test_bellman_ford_int(n):
    g = inputs.rng(200 + n)
    w, absent = _rand_int_graph(g, n, 0.15, 0, 1000, pot=60)
    d, unr = oracle.fw_int(w, absent)
    for s in range(n):
        bd, bunr, neg = oracle.bellman_ford_int(w, absent, s)
        assert not neg
        np.testing.assert_array_equal(unr[s], bunr)
        np.testing.assert_array_equal(d[s][~unr[s]], bd[~bunr])


def test_bellman_ford_detects_negative_cycle():
    # sanity of the pin itself: a 2-cycle of length -1
    w = np.array([[0, 1], [-2, 0]], np.int64)
    _, _, neg = oracle.bellman_ford_int(w, np.zeros((2, 2), bool), 0)
    assert neg


def test_bellman_ford_real():
    g = inputs.rng(300)
    n = 80
    pv = g.integers(0, 32, size=n) / 64.0
    w = g.integers(1, 64, size=(n, n)) / 64.0 + pv[:, None] - pv[None, :]
    np.fill_diagonal(w, 0.0)
    w[g.random((n, n)) > 0.3] = np.inf
    np.fill_diagonal(w, 0.0)
    d = oracle.fw_f64(w)
    for s in range(0, n, 7):
        bd, neg = oracle.bellman_ford_f64(w, s)
        assert not neg
        np.testing.assert_array_equal(d[s], bd)


def test_dijkstra_rows_match():
    w32 = inputs.int_graph(300, 0.05, 1, 1000, seed=7)
    d = oracle.fw_int32_conv(w32)
    src = [0, 5, 123, 299]
    np.testing.assert_array_equal(oracle.dijkstra_rows_i32(w32, src), d[src])
    wf = inputs.dense_f32(200, seed=8)
    df = oracle.fw_f64(wf)
    rows = oracle.dijkstra_rows_f32(wf, [0, 77, 199])
    # different summation orders: equal to within a few ulps of the path length
    np.testing.assert_allclose(rows, df[[0, 77, 199]], rtol=1e-14, atol=0)


def test_dijkstra_strided_view():
    w = inputs.dense_f32(100, seed=9, ld=104)
    view = w[:, :100]
    rows = oracle.dijkstra_rows_f32(view, [3])
    np.testing.assert_allclose(rows[0], oracle.fw_f64(np.ascontiguousarray(view))[3], rtol=1e-14)


# ------------------------------------------------------------ closed forms ---

@pytest.mark.parametrize("n", [1, 3, 40])
def test_uniform_complete_graph(n):
    c = 37
    w = np.full((n, n), c, np.int32)
    np.fill_diagonal(w, 0)
    exp = np.full((n, n), c, np.int32)
    np.fill_diagonal(exp, 0)
    np.testing.assert_array_equal(oracle.fw_int32_conv(w), exp)
    wf = np.full((n, n), 0.375)
    np.fill_diagonal(wf, 0.0)
    ef = np.full((n, n), 0.375)
    np.fill_diagonal(ef, 0.0)
    np.testing.assert_array_equal(oracle.fw_f64(wf), ef)


@pytest.mark.parametrize("n", [2, 9, 64])
def test_directed_cycle(n):
    w = np.full((n, n), INF, np.int32)
    np.fill_diagonal(w, 0)
    for i in range(n):
        w[i, (i + 1) % n] = 1
    i, j = np.indices((n, n))
    np.testing.assert_array_equal(oracle.fw_int32_conv(w), ((j - i) % n).astype(np.int32))


@pytest.mark.parametrize("n", [2, 33])
def test_chain_prefix_sums(n):
    g = inputs.rng(400 + n)
    steps = g.integers(-30, 100, size=n - 1)
    w = np.full((n, n), INF, np.int32)
    np.fill_diagonal(w, 0)
    for i in range(n - 1):
        w[i, i + 1] = steps[i]
    pref = np.concatenate([[0], np.cumsum(steps)])
    exp = np.full((n, n), INF, np.int64)
    for i in range(n):
        for j in range(i, n):
            exp[i, j] = pref[j] - pref[i]
    np.testing.assert_array_equal(oracle.fw_int32_conv(w), exp.astype(np.int32))
    # the same chain with real weights that are integers: exact in double
    wf = np.where(w == INF, np.inf, w.astype(np.float64))
    np.testing.assert_array_equal(oracle.fw_f64(wf), np.where(exp == INF, np.inf, exp))


def test_empty_graph():
    n = 12
    w = np.full((n, n), INF, np.int32)
    np.fill_diagonal(w, 0)
    np.testing.assert_array_equal(oracle.fw_int32_conv(w), w)
    assert oracle.fw_int32_conv(np.zeros((0, 0), np.int32)).shape == (0, 0)


# ---------------------------------------------------------- invariances ---

def test_relabeling():
    w = inputs.int_graph(70, 0.1, 1, 1000, seed=11, potential_max=40)
    perm = inputs.rng(12).permutation(70)
    d = oracle.fw_int32_conv(w)
    dp = oracle.fw_int32_conv(w[np.ix_(perm, perm)])
    np.testing.assert_array_equal(dp, d[np.ix_(perm, perm)])


def test_potential_reweighting_int():
    base = inputs.int_graph(90, 0.08, 0, 1000, seed=13)
    pot = inputs.rng(14).integers(0, 500, size=90)
    rew = base.astype(np.int64)
    present = base != INF
    rew[present] = (rew + pot[:, None] - pot[None, :])[present]
    rew = np.where(present, rew, INF).astype(np.int32)
    d = oracle.fw_int32_conv(base)
    dr = oracle.fw_int32_conv(rew)
    reach = d != INF
    np.testing.assert_array_equal(dr != INF, reach)
    exp = d.astype(np.int64) + pot[:, None] - pot[None, :]
    np.testing.assert_array_equal(dr[reach], exp[reach])


def test_potential_reweighting_f64_generator():
    n = 96
    w = inputs.dense_f32(n, seed=15, reweighted=False)
    wr, pot = inputs.dense_f32(n, seed=15, reweighted=True)
    assert (wr < 0).any()
    d = oracle.fw_f64(wr)
    # reweighted graph: d' = d0 + p_i - p_j with d0 the distances of the
    # un-reweighted integer-unit graph; recover d0 and check it is the fixed
    # point of the Bellman equation on that graph
    w0 = wr.astype(np.float64) - pot[:, None] + pot[None, :]
    np.fill_diagonal(w0, 0.0)
    assert (w0 > 0)[~np.eye(n, dtype=bool)].all()
    d0 = oracle.fw_f64(w0)
    np.testing.assert_allclose(d, d0 + pot[:, None] - pot[None, :], rtol=0, atol=1e-12)
    assert w.shape == wr.shape


# --------------------------------------------------- optimality conditions ---

def check_optimality_int(w, d):
    """Conditions that together characterise the distance matrix (with no
    zero- or negative-length cycle): d_ii = 0, d_ij <= w_ij, the triangle
    inequality, and tightness d_ij = min(w_ij, min_k w_ik + d_kj) for i != j.
    Works on int64 arrays with np.inf-free encoding: unreachable = INF."""
    n = w.shape[0]
    big = np.int64(1) << 40
    wi = np.where(w == INF, big, w.astype(np.int64))
    di = np.where(d == INF, big, d.astype(np.int64))
    ok = True
    def add(a, b):  # a + b with "big" absorbing, whatever the sign of the other term
        return np.where((a == big) | (b == big), big, a + b)

    ok &= bool((np.diag(di) == 0).all())
    ok &= bool((di <= wi).all())
    for k in range(n):
        ok &= bool((di <= add(di[:, k:k + 1], di[k:k + 1, :])).all())
    tight = np.minimum(wi, np.min(add(wi[:, :, None], di[None, :, :]), axis=1))
    np.fill_diagonal(tight, 0)
    ok &= bool((tight == di).all())
    return ok


def test_optimality_conditions_hold():
    for seed in range(5):
        w = inputs.int_graph(48, 0.1, 1, 50, seed=500 + seed, potential_max=10)
        assert check_optimality_int(w, oracle.fw_int32_conv(w))


# -------------------------------------------------------------- mutants ---

def _fw_variant(w, absent, mutation):
    """Fig. 1 with a planted mistake (numpy, on the CPU)."""
    n = w.shape[0]
    big = np.int64(1) << 40
    d = np.where(absent, big, w.astype(np.int64))
    if mutation == "k_innermost":          # loop order i, j, k (wrong)
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    d[i, j] = min(d[i, j], d[i, k] + d[k, j])
    else:
        for k in range(n - 1 if mutation == "drop_last_k" else n):
            if mutation == "transposed":
                cand = d[k, :][:, None] + d[:, k][None, :]
            elif mutation == "wrong_sign":
                cand = d[:, k:k + 1] - d[k:k + 1, :]
            elif mutation == "wrong_index":
                kk = (k + 1) % n
                cand = d[:, k:k + 1] + d[kk:kk + 1, :]
            else:
                cand = d[:, k:k + 1] + d[k:k + 1, :]
            if mutation == "no_min":
                d = np.where(cand < big, cand, d)
            else:
                d = np.minimum(d, cand)
    d = np.where(d >= big // 2, INF, d)
    return d


@pytest.mark.parametrize("mutation", ["k_innermost", "drop_last_k", "transposed",
                                      "wrong_sign", "wrong_index", "no_min"])
def test_mutants_are_caught(mutation):
    caught = False
    g = inputs.rng(600)
    for trial in range(40):
        n = int(g.integers(3, 8))
        w, absent = _rand_int_graph(g, n, 0.5, 1, 30, pot=5)
        dm = _fw_variant(w, absent, mutation)
        bd, bunr = _brute_as_arrays(oracle.brute_force_paths(w, absent))
        ref = np.where(bunr, INF, bd)
        w32 = np.where(absent, INF, w).astype(np.int32)
        if not np.array_equal(dm, ref) or not check_optimality_int(w32, dm.astype(np.int32)):
            caught = True
            break
    assert caught, mutation
    # and the unmutated variant passes the same pins
    for trial in range(10):
        n = int(g.integers(3, 8))
        w, absent = _rand_int_graph(g, n, 0.5, 1, 30, pot=5)
        dm = _fw_variant(w, absent, "none")
        bd, bunr = _brute_as_arrays(oracle.brute_force_paths(w, absent))
        np.testing.assert_array_equal(dm, np.where(bunr, INF, bd))


# ------------------------------------------- the all-core Fig. 1 loops ---

def test_multithreaded_fig1_equals_serial():
    """fw_int32_conv_mt / fw_f64_mt share the rows of each iteration k among
    threads; with no negative cycle they read what the serial loop reads, so
    they must equal the pinned serial forms bit for bit (negative edges,
    unreachable pairs, thread counts above n included)."""
    g = inputs.rng(700)
    for trial in range(12):
        n = int(g.integers(1, 90))
        w = inputs.int_graph(n, float(g.uniform(0.02, 0.6)), 0, 1000, seed=700 + trial,
                             potential_max=int(g.integers(0, 60)))
        exp = oracle.fw_int32_conv(w)
        for threads in (1, 2, 3, 0):
            d, used = oracle.fw_int32_conv_mt(w, threads)
            np.testing.assert_array_equal(d, exp, err_msg=f"trial {trial} threads {threads}")
            assert used >= 1 and (threads == 0 or used == threads)
        f, pot = inputs.dense_f32(n, seed=800 + trial, reweighted=True)
        f[g.random((n, n)) < 0.3] = np.inf
        np.fill_diagonal(f, 0)
        e64 = oracle.fw_f64(f)
        for threads in (1, 4, 0):
            np.testing.assert_array_equal(oracle.fw_f64_mt(f, threads)[0], e64)


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "g*.txt"))),
                         ids=lambda p: os.path.basename(p))
def test_multithreaded_fig1_golden(path):
    kind, n, rin, rout = _parse_golden(path)
    if kind == "int":
        w = np.array([[INF if t == "inf" else int(t) for t in r] for r in rin], np.int32)
        exp = np.array([[INF if t == "inf" else int(t) for t in r] for r in rout], np.int32)
        np.testing.assert_array_equal(oracle.fw_int32_conv_mt(w, 3)[0], exp)
    else:
        w = np.array([[np.inf if t == "inf" else float(t) for t in r] for r in rin])
        exp = np.array([[np.inf if t == "inf" else float(t) for t in r] for r in rout])
        np.testing.assert_array_equal(oracle.fw_f64_mt(w, 3)[0], exp)


def test_multithreaded_fig1_brute_force():
    g = inputs.rng(701)
    for trial in range(100):
        n = int(g.integers(1, 8))
        w, absent = _rand_int_graph(g, n, float(g.uniform(0.1, 0.9)), 0, 20, pot=int(g.integers(0, 15)))
        w32 = np.where(absent, INF, w).astype(np.int32)
        bd, bunr = _brute_as_arrays(oracle.brute_force_paths(w, absent))
        np.testing.assert_array_equal(oracle.fw_int32_conv_mt(w32, 2)[0], np.where(bunr, INF, bd))


# --------------------------------------------------- library conventions ---

def test_int16_convention():
    w32, w16 = inputs.c3(seed=3, n=96)
    d32 = oracle.fw_int32_conv(w32)
    d16 = oracle.fw_int16_conv(w16)
    np.testing.assert_array_equal(np.where(d16 == inputs.INF_I16, INF, d16.astype(np.int32)), d32)


def test_generators_are_deterministic_and_shaped():
    a = inputs.c1(seed=5, n=64)
    b = inputs.c1(seed=5, n=64)
    np.testing.assert_array_equal(a, b)
    assert a.dtype == np.int32 and (np.diag(a) == 0).all()
    frac = (a != INF).mean()
    assert 0.2 < frac < 0.45
    f = inputs.dense_f32(64, seed=1)
    assert f.dtype == np.float32 and (f[~np.eye(64, dtype=bool)] > 0).all() and f.max() <= 1.0
    padded = inputs.int_graph(10, 0.5, 1, 9, seed=2, ld=16)
    assert padded.shape == (10, 16) and (padded[:, 10:] == -7).all()
    batch = inputs.c4_batch(8, seed=3)
    assert all(16 <= g.shape[0] <= 512 for g in batch)
    assert min(int(g[g != INF].min()) for g in batch) >= -50
    reqs = inputs.c5_requests(6, 100.0, seed=4, nmax=300)
    assert [r.dtype for r in reqs] == ["i32", "f32"] * 3
    assert all(32 <= r.n <= 300 for r in reqs)
    assert math.isclose(reqs[0].t_arrival, 0.0)
