// Path reconstruction from the distances and the stage record of
// apsp_fw_paths (host code; the paper computes distances only).
//
// via[i][j] = b >= 0 says that the last strict improvement of d_ij happened
// in stage b, through some k of k-block b: d_ij = d_ik + d_kj at that moment.
// Later stages only lower values, and the final matrix satisfies
// d_ij <= d_ik + d_kj, so at the end d_ij = d_ik + d_kj still holds with the
// final d_ik and d_kj (integers: exactly).  Searching block b for such a k
// and recursing on (i, k) and (k, j) yields a shortest path; via[i][j] = -1
// means d_ij was never improved: the edge i -> j itself.
#include <cmath>
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/apsp.h"

namespace {

struct Dist {
  const void *d;
  int64_t ld;
  int dtype;
  // value of d_ij as int64 (integers) or double (fp32), and reachability
  bool reach(int64_t i, int64_t j) const {
    switch (dtype) {
      case APSP_I32: return static_cast<const int32_t *>(d)[i * ld + j] < (1 << 28);
      case APSP_I16: return static_cast<const int16_t *>(d)[i * ld + j] < 16383;
      default: return std::isfinite(static_cast<const float *>(d)[i * ld + j]);
    }
  }
  int64_t ival(int64_t i, int64_t j) const {
    return dtype == APSP_I32 ? static_cast<const int32_t *>(d)[i * ld + j]
                             : static_cast<const int16_t *>(d)[i * ld + j];
  }
  float fval(int64_t i, int64_t j) const { return static_cast<const float *>(d)[i * ld + j]; }
};

// A k of block b (k != i, j) with d_ik + d_kj = d_ij; fp32: the one whose
// rounded sum is closest to d_ij.  Among equal candidates one whose two
// halves were last improved in stage b or before is preferred: the k that
// made the last improvement is such a vertex, and with zero-weight edges a
// tie could otherwise lead back to a later pair.  -1 if none.
int64_t split_vertex(const Dist &D, const int16_t *via, int64_t via_ld, int64_t n, int S, int b, int64_t i,
                     int64_t j) {
  const int64_t k0 = (int64_t)b * S, k1 = std::min<int64_t>(n, k0 + S);
  int64_t best = -1;
  double best_err = INFINITY;
  bool best_early = false;
  for (int64_t k = k0; k < k1; ++k) {
    if (k == i || k == j || !D.reach(i, k) || !D.reach(k, j)) continue;
    double err;
    if (D.dtype == APSP_F32) {
      const float sum = D.fval(i, k) + D.fval(k, j);  // rounded as in the kernels
      err = std::fabs((double)sum - (double)D.fval(i, j));
    } else {
      if (D.ival(i, k) + D.ival(k, j) != D.ival(i, j)) continue;
      err = 0;
    }
    const bool early = via[i * via_ld + k] <= b && via[k * via_ld + j] <= b;
    if (err < best_err || (err == best_err && early && !best_early)) {
      best = k;
      best_err = err;
      best_early = early;
      if (err == 0 && early) break;
    }
  }
  return best;
}

}  // namespace

extern "C" int apsp_path(const void *dist, const int16_t *via, int64_t n, int64_t ld, int64_t via_ld, int dtype,
                         int32_t kblock, int64_t i, int64_t j, int64_t *path, int64_t cap, int64_t *len) {
  if (!len) return APSP_EINVAL;
  *len = 0;
  if (dtype != APSP_I32 && dtype != APSP_F32 && dtype != APSP_I16) return APSP_EINVAL;
  if (n <= 0 || !dist || !via || ld < n || via_ld < n || (kblock != 64 && kblock != 128)) return APSP_EINVAL;
  if (i < 0 || i >= n || j < 0 || j >= n || cap < 0 || (cap > 0 && !path)) return APSP_EINVAL;
  const Dist D{dist, ld, dtype};
  std::vector<int64_t> out{i};
  if (i != j) {
    if (!D.reach(i, j)) return APSP_OK;  // unreachable: empty path
    // in-order expansion of the segments (u, v) with an explicit stack
    std::vector<std::pair<int64_t, int64_t>> stack{{i, j}};
    int64_t steps = 0;
    while (!stack.empty()) {
      const auto [u, v] = stack.back();
      stack.pop_back();
      if (++steps > 4 * n) return APSP_EINVAL;  // inconsistent record (not from this solve)
      const int b = via[u * via_ld + v];
      if (b < 0) {
        out.push_back(v);  // the edge u -> v
        continue;
      }
      const int64_t k = split_vertex(D, via, via_ld, n, kblock, b, u, v);
      if (k < 0) return APSP_EINVAL;
      stack.push_back({k, v});
      stack.push_back({u, k});
    }
  }
  *len = (int64_t)out.size();
  if ((int64_t)out.size() > cap) return APSP_ENOMEM;
  for (size_t t = 0; t < out.size(); ++t) path[t] = out[t];
  return APSP_OK;
}
