// int32 instantiation: INF = 2^29, DPX add-min, TMA-staged phase 3.
#include "fw_host.cuh"

namespace apsp {
int run_i32(const RunArgs &a) { return run_any<int32_t, true>(a); }
}  // namespace apsp
