// Instantiation of the sweep family for FP32 deviations storage (FP32 arithmetic).
#include "sweep.cuh"

namespace lbmp {
const KernelTable* kernels_f32() { return make_table<float>(); }
}  // namespace lbmp
