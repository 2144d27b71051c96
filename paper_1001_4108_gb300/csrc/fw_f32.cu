// fp32 instantiation: INF = +inf, fp32 add then exact min, TMA-staged phase 3.
#include "fw_host.cuh"

namespace apsp {
int run_f32(const RunArgs &a) { return run_any<float, true>(a); }
}  // namespace apsp
