// BiCGStab kernel instantiations: QW, QQW, QQW-NN.
#include "bicg_kernels.cuh"
#include "mw_device4.cuh"

namespace mwk {
BiTable bitable_qw() { return make_bitable<mw::QW>(); }
BiTable bitable_qqw() { return make_bitable<mw::QQW>(); }
BiTable bitable_qqw_nn() { return make_bitable<mw::QQW_NN>(); }
}  // namespace mwk
