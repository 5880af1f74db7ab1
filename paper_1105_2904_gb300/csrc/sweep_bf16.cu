// Instantiation of the sweep family for bfloat16 scaled deviations storage (FP32 arithmetic).
#include "sweep.cuh"

namespace lbmp {
const KernelTable* kernels_bf16() { return make_table<__nv_bfloat16>(); }
}  // namespace lbmp
