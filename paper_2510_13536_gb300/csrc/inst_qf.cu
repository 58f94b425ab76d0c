// Kernel instantiations for QF: QQF renormalised after every operation, with
// the same power-of-two-scaled CG and BiCGStab.
#include "bicg_float.cuh"
#include "cg_float.cuh"

namespace mwk {
KernelTable table_qf() { return make_table_qqf<mw::QF>(); }
BiTable bitable_qf() { return make_bitable_qqf<mw::QF>(); }
}  // namespace mwk
