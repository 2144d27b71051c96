// Sets of phase-3 tiles of one stage, numbered by a CTA's linear index.
//
// Phase 3 of stage b updates every tile (I, J) with I != b and J != b
// (Fig. 2).  With the lookahead schedule it is split in two launches:
//   cross(b): row b+1 and column b+1 (the tiles that phases 1 and 2 of stage
//             b+1 read), launched first on the side stream, right before them;
//   rest(b):  all other tiles, on the caller's stream, while phases 1 and 2 of
//             stage b+1 run beside it.
// The order of the two does not matter for the result: the tiles of one stage
// are independent of each other (Sec. 3.2).  A set may further be restricted
// to the interior tiles (every row and column inside the matrix) or to the
// edge tiles of a ragged matrix (last tile row or column), for kernels that
// drop the bounds masks on interior tiles.
//
// Plain C++ so that the host test harness can enumerate the sets.
#pragma once

#if defined(__CUDACC__)
#define APSP_HD __host__ __device__ __forceinline__
#else
#define APSP_HD inline
#endif

namespace apsp {

constexpr int kTileNone = 1 << 30;

// A rectangle of tiles.  A fixed row (col >= 0) is one tile index; an
// enumerated one (-1) runs over [0, hi) without e0 and e1 (e0 < e1, either
// may be kTileNone), in increasing order.
struct TileSeg {
  int row, col, hi, e0, e1;
};

struct TileSet {
  int nseg;
  TileSeg seg[3];
  int count[3];  // CTAs of each segment

  APSP_HD static int span(const TileSeg &s) { return s.hi - (s.e0 < s.hi ? 1 : 0) - (s.e1 < s.hi ? 1 : 0); }
  APSP_HD static int pick(int x, const TileSeg &s) {
    if (x >= s.e0) ++x;
    if (x >= s.e1) ++x;
    return x;
  }
  APSP_HD int total() const {
    int t = 0;
    for (int i = 0; i < nseg; ++i) t += count[i];
    return t;
  }
  // Tile of CTA t (0 <= t < total()); consecutive t share a tile row.
  // Segments are picked with constant indices only, so that a kernel
  // parameter of this type is read in place (no local-memory copy).
  APSP_HD void tile(int t, int &I, int &J) const {
    TileSeg s = seg[0];
    if (nseg > 1 && t >= count[0]) {
      t -= count[0];
      s = seg[1];
      if (nseg > 2 && t >= count[1]) {
        t -= count[1];
        s = seg[2];
      }
    }
    if (s.row >= 0 && s.col >= 0) {
      I = s.row;
      J = s.col;
    } else if (s.row >= 0) {
      I = s.row;
      J = pick(t, s);
    } else if (s.col >= 0) {
      I = pick(t, s);
      J = s.col;
    } else {
      const int m = span(s);
      const int ti = t / m;
      I = pick(ti, s);
      J = pick(t - ti * m, s);
    }
  }
  void add(int row, int col, int hi, int e0, int e1) {
    if (e1 < e0) {
      const int x = e0;
      e0 = e1;
      e1 = x;
    }
    TileSeg s{row, col, hi, e0, e1};
    const int m = span(s);
    const int c = (row >= 0 ? 1 : m) * (col >= 0 ? 1 : m);
    if (c <= 0) return;
    seg[nseg] = s;
    count[nseg] = c;
    ++nseg;
  }
};

enum TileKind { kTilesAll = 0, kTilesCross = 1, kTilesRest = 2 };
enum TilePart { kPartAny = 0, kPartInterior = 1, kPartEdge = 2 };

// The tiles of `kind` for stage b of an R x R tile grid whose last tile row
// and column are partial when `ragged`, restricted to `part`.  Stage b must
// have a full k-block (b < R - 1 when ragged); cross and rest need b + 1 < R.
inline TileSet make_tileset(int kind, int part, int b, int R, bool ragged) {
  TileSet ts{};
  const int c = b + 1;
  const int N = kTileNone;
  const int Ri = ragged ? R - 1 : R;  // interior tile rows / columns
  const int E = R - 1;                // the ragged edge
  if (part == kPartAny) {
    if (kind == kTilesAll) ts.add(-1, -1, R, b, N);
    if (kind == kTilesCross) {
      ts.add(c, -1, R, b, N);
      ts.add(-1, c, R, b, c);
    }
    if (kind == kTilesRest) ts.add(-1, -1, R, b, c);
  } else if (part == kPartInterior) {
    if (kind == kTilesAll) ts.add(-1, -1, Ri, b, N);
    if (kind == kTilesCross && c < Ri) {
      ts.add(c, -1, Ri, b, N);
      ts.add(-1, c, Ri, b, c);
    }
    if (kind == kTilesRest) ts.add(-1, -1, Ri, b, c < Ri ? c : N);
  } else if (ragged) {
    const bool c_edge = c == E;
    if (kind == kTilesAll || (kind == kTilesCross && c_edge)) {
      ts.add(E, -1, Ri, b, N);
      ts.add(-1, E, R, b, N);
    }
    if (kind == kTilesCross && !c_edge) {
      ts.add(c, E, R, N, N);
      ts.add(E, c, R, N, N);
    }
    if (kind == kTilesRest && !c_edge) {
      ts.add(E, -1, Ri, b, c);
      ts.add(-1, E, R, b, c);
    }
  }
  return ts;
}

}  // namespace apsp
