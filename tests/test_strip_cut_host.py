"""The strip cut of the s = 64 panel and cross launches (fw_strip), restated
on the host: for every stage of small tile grids, each strip CTA's read and
write sets, from the same block-index mapping the kernel uses.  Within one
launch no strip writes a cell another strip reads or writes, and the strips
together write exactly the launch's tiles.  (Cells are (row, column) of a
matrix of R x R tiles of side S; the k-block is b.)"""
import itertools

import pytest

S = 64
Q = S // 4  # strip width


def skip_pivot(t, b):
    return t if t < b else t + 1


def rect(r0, nr, c0, nc):
    return {(r, c) for r in range(r0, r0 + nr) for c in range(c0, c0 + nc)}


def strip_sets(It, Jt, q, b, panel):
    """(reads, writes) of strip q of tile (It, Jt) in stage b."""
    I0, J0, K0 = It * S, Jt * S, b * S
    if panel and Jt == b:  # column panel: 16 x 64 row strip, x_ij <- min_k x_ik + D_kj
        r0, nr, c0, nc = I0 + q * Q, Q, J0, S
    else:                  # 64 x 16 column strip
        r0, nr, c0, nc = I0, S, J0 + q * Q, Q
    a = rect(r0, nr, K0, S)      # rows of the strip, the k-block's columns
    bb = rect(K0, S, c0, nc)     # the k-block's rows, columns of the strip
    c = rect(r0, nr, c0, nc)
    return a | bb | c, c


def panel_launch(R, b):
    for blk in range(4 * 2 * (R - 1)):
        t, q = divmod(blk, 4)
        rp = t < R - 1
        It = b if rp else skip_pivot(t - (R - 1), b)
        Jt = skip_pivot(t, b) if rp else b
        yield It, Jt, q


def cross_launch(R, b):
    # row and column b+1 without the pivot row/column b (the lookahead's cross(b))
    tiles = [(b + 1, j) for j in range(R) if j != b] + [(i, b + 1) for i in range(R) if i not in (b, b + 1)]
    for (It, Jt), q in itertools.product(tiles, range(4)):
        yield It, Jt, q


def check(launch, panel, expect_tiles):
    sets = [strip_sets(It, Jt, q, b_, panel) for (It, Jt, q), b_ in launch]
    written = set()
    for i, (_, w) in enumerate(sets):
        assert not (written & w), "two strips write the same cell"
        written |= w
    for i, (_, w) in enumerate(sets):
        for j, (rd, _) in enumerate(sets):
            if i != j:
                assert not (w & rd), "a strip reads a cell another strip writes"
    assert written == set().union(*(rect(I * S, S, J * S, S) for I, J in expect_tiles))


@pytest.mark.parametrize("R", [2, 3, 5])
def test_panel_strips_are_independent(R):
    for b in range(R):
        launch = [(x, b) for x in panel_launch(R, b)]
        tiles = {(b, j) for j in range(R) if j != b} | {(i, b) for i in range(R) if i != b}
        check(launch, True, tiles)


@pytest.mark.parametrize("R", [3, 4, 6])
def test_cross_strips_are_independent(R):
    for b in range(R - 1):
        launch = [(x, b) for x in cross_launch(R, b)]
        tiles = {(b + 1, j) for j in range(R) if j != b} | {(i, b + 1) for i in range(R) if i not in (b, b + 1)}
        check(launch, False, tiles)


def test_cut_along_rows_would_race():
    # the check above is not vacuous: 16 x 64 row strips of a row-panel tile
    # (b, J) read the tile's k rows that other strips of the same tile write
    b, J = 0, 1
    sets = []
    for q in range(4):
        r0, c0, K0 = b * S + q * Q, J * S, b * S
        reads = rect(r0, Q, K0, S) | rect(K0, S, c0, S) | rect(r0, Q, c0, S)
        sets.append((reads, rect(r0, Q, c0, S)))
    assert any(sets[i][1] & sets[j][0] for i in range(4) for j in range(4) if i != j)
