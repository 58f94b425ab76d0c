// BiCGStab kernel instantiations: TW, QTW, QTW-NN.
#include "bicg_kernels.cuh"

namespace mwk {
BiTable bitable_tw() { return make_bitable<mw::TW>(); }
BiTable bitable_qtw() { return make_bitable<mw::QTW>(); }
BiTable bitable_qtw_nn() { return make_bitable<mw::QTW_NN>(); }
}  // namespace mwk
