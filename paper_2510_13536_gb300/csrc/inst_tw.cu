// Kernel instantiations for triple-word (TW) arithmetic.
#include "cg_kernels.cuh"
namespace mwk {
KernelTable table_tw() { return make_table<mw::TW>(); }
}  // namespace mwk
