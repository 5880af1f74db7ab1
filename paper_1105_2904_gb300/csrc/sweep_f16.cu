// Instantiation of the sweep family for half-precision scaled deviations storage (FP32 arithmetic).
#include "sweep.cuh"

namespace lbmp {
const KernelTable* kernels_f16() { return make_table<__half>(); }
}  // namespace lbmp
