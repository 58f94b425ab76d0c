// BiCGStab kernel instantiations: FP64, DW, QDW, QDW-NN.
#include "bicg_kernels.cuh"

namespace mwk {
BiTable bitable_fp64() { return make_bitable<mw::FP64>(); }
BiTable bitable_dw() { return make_bitable<mw::DW>(); }
BiTable bitable_qdw() { return make_bitable<mw::QDW>(); }
BiTable bitable_qdw_nn() { return make_bitable<mw::QDW_NN>(); }
}  // namespace mwk
