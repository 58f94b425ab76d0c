// Kernel instantiations for quadruple-word arithmetic (QW).
#include "cg_kernels.cuh"
#include "mw_device4.cuh"

namespace mwk {
KernelTable table_qw() { return make_table<mw::QW>(); }
}  // namespace mwk
