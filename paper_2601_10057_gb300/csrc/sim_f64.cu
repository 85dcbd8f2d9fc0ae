// FP64 instantiation: every field operation and reduction in FP64.
#include "sim_impl.cuh"
namespace ccm {
SimBase* make_sim_f64(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err) {
    return make_sim<double>(p, N, flags, s, err);
}
}  // namespace ccm
