// Kernel instantiations for QQF, four FP32 words with power-of-two-scaled CG
// and BiCGStab.
#include "bicg_float.cuh"
#include "cg_float.cuh"

namespace mwk {
KernelTable table_qqf() { return make_table_qqf<mw::QQF>(); }
BiTable bitable_qqf() { return make_bitable_qqf<mw::QQF>(); }
// ||b|| and the first scale: FP64 work only, shared by QQF and QF.
const void* qqf_init_pre() { return (const void*)&k_qqf_bnorm<mw::QQF>; }
}  // namespace mwk
