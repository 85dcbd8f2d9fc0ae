// ccmsav_noalloc.cu -- ccmsav_mass_noalloc(): the discrete mass h^2 sum psi
// of a caller-owned device field, computed without any allocation by the
// library.
//
// Some callers cannot let a library allocate device memory: services whose
// device memory is reserved up front by a pooling allocator or capped by a
// framework (a cudaMalloc there either fails or steals from the pool), and
// real-time loops that must not pay allocation latency or fragment the heap.
// For them this entry point takes its scratch (one FP64 partial sum per
// reduction block plus the final sum) from a fixed array compiled into the
// library.  Every GPU that loads the library holds that array
// (kScratchDoubles doubles, under 10 KB, whatever N is) until the process
// exits.
//
// The array's name, used in host code, is only a host-side stand-in for the
// device symbol: a kernel handed it would fault or, where the GPU can reach
// host memory, silently use the wrong memory.  So every call looks up the
// real device address with cudaGetSymbolAddress for the current device and
// context (a lookup, not an allocation; nothing is cached, so a device reset
// between calls leaves no stale address behind).  All calls share the array
// and it keeps the last call's contents:
// every slot a call reads is written earlier in the same call, so nothing
// needs clearing, but calls whose work overlaps on the GPU (other streams,
// other host threads) race on it.
#include <cuda_runtime.h>
#include "../../include/ccmsav.h"

namespace {

constexpr int kBlocks = 1184;                 // fixed reduction grid (8 blocks per SM on 148+ SMs)
constexpr int kThreads = 256;
constexpr int kScratchDoubles = kBlocks + 1;  // block partials, then the final sum

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];


// FP64 block sum in a fixed order (warp shuffles, then warps in order).
__device__ __forceinline__ double block_sum(double v, double* sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sm[i];
    return s;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mass_partials(const T* __restrict__ psi, size_t n, double* __restrict__ part) {
    __shared__ double sm[kThreads / 32];
    double s = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        s += (double)psi[q];
    const double b = block_sum(s, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(kThreads)
k_mass_final(double* __restrict__ part, int nb, double h2) {
    __shared__ double sm[kThreads / 32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    const double t = block_sum(s, sm);
    if (threadIdx.x == 0) part[kBlocks] = h2 * t;
}

}  // namespace

extern "C" int ccmsav_mass_noalloc(const void* psi, int N, int precision, double L,
                                   double* mass, void* stream) {
    if (!psi || !mass) return CCMSAV_EINVAL;
    if (N < 1 || N > CCMSAV_NOALLOC_MAX_N) return CCMSAV_EINVAL;
    if (precision != CCMSAV_FP64 && precision != CCMSAV_FP32_BULK) return CCMSAV_EINVAL;
    if (!(L > 0.0) || !(L < 1e300)) return CCMSAV_EINVAL;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CCMSAV_ECUDA;
    double* scratch = static_cast<double*>(p);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)N * N;
    int nb = (int)((n + kThreads - 1) / kThreads);
    if (nb > kBlocks) nb = kBlocks;
    // cudaLaunchKernel returns this launch's own status (an error left over
    // from earlier work of the caller is not taken for ours)
    void* psi_arg = const_cast<void*>(psi);
    size_t n_arg = n;
    void* part_args[] = {&psi_arg, &n_arg, &scratch};
    const void* kpart = precision == CCMSAV_FP64 ? (const void*)k_mass_partials<double>
                                                 : (const void*)k_mass_partials<float>;
    if (cudaLaunchKernel(kpart, dim3(nb), dim3(kThreads), part_args, 0, st) != cudaSuccess) return CCMSAV_ECUDA;
    const double h = L / N;
    double h2 = h * h;
    void* fin_args[] = {&scratch, &nb, &h2};
    if (cudaLaunchKernel((const void*)k_mass_final, dim3(1), dim3(kThreads), fin_args, 0, st) != cudaSuccess)
        return CCMSAV_ECUDA;
    if (cudaMemcpyAsync(mass, scratch + kBlocks, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CCMSAV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCMSAV_ECUDA;
    return CCMSAV_OK;
}
