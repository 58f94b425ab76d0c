// Kernel instantiations for QF: QQF renormalised after every operation, with
// the same power-of-two-scaled CG.
#include "cg_float.cuh"

namespace mwk {
KernelTable table_qf() { return make_table_qqf<mw::QF>(); }
}  // namespace mwk
