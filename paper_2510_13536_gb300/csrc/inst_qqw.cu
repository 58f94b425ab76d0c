// Kernel instantiations for quasi quadruple-word arithmetic, normalised and not.
#include "cg_kernels.cuh"
#include "mw_device4.cuh"

namespace mwk {
KernelTable table_qqw() { return make_table<mw::QQW>(); }
KernelTable table_qqw_nn() { return make_table<mw::QQW_NN>(); }
}  // namespace mwk
