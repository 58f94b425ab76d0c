// Kernel instantiations for quasi double-word arithmetic, normalised and not.
#include "cg_kernels.cuh"
namespace mwk {
KernelTable table_qdw() { return make_table<mw::QDW, mw::QDW_S>(); }
KernelTable table_qdw_nn() { return make_table<mw::QDW_NN, mw::QDW_NN_S>(); }
}  // namespace mwk
