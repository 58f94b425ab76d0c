// Kernel instantiations for QQF, four FP32 words with power-of-two-scaled CG.
#include "cg_float.cuh"

namespace mwk {
KernelTable table_qqf() { return make_table_qqf(); }
}  // namespace mwk
