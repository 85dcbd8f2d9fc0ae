// FP32-bulk instantiation: fields, stencils and DCTs in FP32; SAV inner
// products, the 5x5 solve and all scalar updates in FP64.
#include "sim_impl.cuh"
namespace ccm {
SimBase* make_sim_f32(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err) {
    return make_sim<float>(p, N, flags, s, err);
}
}  // namespace ccm
