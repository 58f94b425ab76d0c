// Kernel instantiations for FP64 arithmetic (one translation unit per arithmetic
// family keeps the parallel build short).
#include "cg_kernels.cuh"
namespace mwk {
KernelTable table_fp64() { return make_table<mw::FP64>(); }
}  // namespace mwk
