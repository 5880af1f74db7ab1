// FP64 instantiations of the sweep family. Built with -fmad=false: every expression is
// evaluated as written (no fused multiply-add contraction), which makes the FP64 path
// reproduce a plain FP64 implementation of the same equations bit for bit.
#include "sweep.cuh"

namespace lbmp {
const KernelTable* kernels_f64() { return make_table<double>(); }
}  // namespace lbmp
