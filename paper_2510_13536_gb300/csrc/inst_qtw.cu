// Kernel instantiations for quasi triple-word arithmetic, normalised and not.
#include "cg_kernels.cuh"
namespace mwk {
KernelTable table_qtw() { return make_table<mw::QTW, mw::QTW_S>(); }
KernelTable table_qtw_nn() { return make_table<mw::QTW_NN, mw::QTW_NN_S>(); }
}  // namespace mwk
