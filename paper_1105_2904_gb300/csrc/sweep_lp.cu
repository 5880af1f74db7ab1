// Reduced-storage instantiations of the sweep family: FP32 deviations, and half / bfloat16
// scaled deviations, all with FP32 arithmetic.
#include "sweep.cuh"

namespace lbmp {
const KernelTable* kernels_f32() { return make_table<float>(); }
const KernelTable* kernels_f16() { return make_table<__half>(); }
const KernelTable* kernels_bf16() { return make_table<__nv_bfloat16>(); }
}  // namespace lbmp
