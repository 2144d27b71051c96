// Host check of the phase-3 tile sets: for every tile grid R x R (ragged or
// not) and stage b, each set enumerates its tiles exactly once, and
//   cross(b) + rest(b) = all(b) = {(I, J) : I != b, J != b},
//   interior + edge = any, interior tiles inside, edge tiles on the edge.
// Exit status 0 when every check holds; the first failure is printed.
#include <cstdio>
#include <vector>

#include "../../paper_1001_4108_gb300/csrc/tileset.h"

using apsp::make_tileset;
using apsp::TileSet;

static int fails = 0;
#define CHECK(c, ...)                                   \
  do {                                                  \
    if (!(c)) {                                         \
      if (fails++ == 0) std::printf(__VA_ARGS__);       \
    }                                                   \
  } while (0)

// counts[I*R+J] += 1 for every CTA of ts
static void mark(const TileSet &ts, int R, std::vector<int> &counts, int &bad) {
  for (int t = 0; t < ts.total(); ++t) {
    int I = -1, J = -1;
    ts.tile(t, I, J);
    if (I < 0 || I >= R || J < 0 || J >= R) {
      ++bad;
      continue;
    }
    counts[I * R + J] += 1;
  }
}

int main() {
  for (int R = 2; R <= 41; ++R)
    for (int rg = 0; rg < 2; ++rg) {
      const bool ragged = rg == 1;
      const int Ri = ragged ? R - 1 : R, E = R - 1;
      const int bmax = ragged ? R - 2 : R - 1;
      for (int b = 0; b <= bmax; ++b) {
        const int c = b + 1;
        const int kinds = c < R ? 3 : 1;
        std::vector<std::vector<int>> any(3, std::vector<int>(R * R, 0));
        for (int kind = 0; kind < kinds; ++kind) {
          std::vector<int> a(R * R, 0), in(R * R, 0), ed(R * R, 0);
          int bad = 0;
          mark(make_tileset(kind, apsp::kPartAny, b, R, ragged), R, a, bad);
          mark(make_tileset(kind, apsp::kPartInterior, b, R, ragged), R, in, bad);
          mark(make_tileset(kind, apsp::kPartEdge, b, R, ragged), R, ed, bad);
          CHECK(bad == 0, "R=%d ragged=%d b=%d kind=%d: tile out of range\n", R, rg, b, kind);
          for (int I = 0; I < R; ++I)
            for (int J = 0; J < R; ++J) {
              const int x = I * R + J;
              bool want = I != b && J != b;
              if (kind == 1) want = want && (I == c || J == c);
              if (kind == 2) want = want && I != c && J != c;
              CHECK(a[x] == (want ? 1 : 0), "R=%d ragged=%d b=%d kind=%d: tile (%d,%d) x%d\n", R, rg, b, kind,
                    I, J, a[x]);
              CHECK(in[x] + ed[x] == a[x], "R=%d ragged=%d b=%d kind=%d: parts at (%d,%d)\n", R, rg, b, kind, I,
                    J);
              if (in[x]) CHECK(I < Ri && J < Ri, "R=%d b=%d kind=%d: interior (%d,%d)\n", R, b, kind, I, J);
              if (ed[x]) CHECK(ragged && (I == E || J == E), "R=%d b=%d kind=%d: edge (%d,%d)\n", R, b, kind, I, J);
              any[kind][x] = a[x];
            }
        }
        if (kinds == 3)
          for (int x = 0; x < R * R; ++x)
            CHECK(any[1][x] + any[2][x] == any[0][x], "R=%d ragged=%d b=%d: cross + rest != all\n", R, rg, b);
      }
    }
  if (fails) std::printf("%d failed checks\n", fails);
  else std::printf("ok\n");
  return fails ? 1 : 0;
}
