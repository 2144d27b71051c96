// int16 instantiation (scalar kernels, int32 arithmetic, INF = 16383).
#include "fw_host.cuh"

namespace apsp {
int run_i16(const RunArgs &a) { return run_any<int16_t, false>(a); }
}  // namespace apsp
