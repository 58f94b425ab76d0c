// Kernel instantiations for double-word (DW) arithmetic.
#include "cg_kernels.cuh"
namespace mwk {
KernelTable table_dw() { return make_table<mw::DW, mw::DW_S>(); }
}  // namespace mwk
