// bounds.cuh -- optional index checks of the step kernels' global accesses.
//
// Built with -DCCMSAV_BOUNDS (paper_2601_10057_gb300.build with bounds=True,
// a separate libccmsav_bounds.so), every checked access verifies that its
// element index lies inside the array it addresses.  An index outside
// records a bit in a device flag (read and cleared by ccmsav_bounds_flag())
// and the access is redirected to element 0 (loads) or dropped (stores), so
// the kernel neither faults nor waits on anything.  Without the macro the
// checks compile to the plain access.  Bits: 1 a load, 2 a store.
#pragma once
#include <cstddef>

namespace ccm {
#ifdef CCMSAV_BOUNDS
static __device__ unsigned int g_oob_flag;
// w consecutive elements from index i inside an array of n
__device__ __forceinline__ size_t oob_ix(size_t i, size_t w, size_t n) {
    if (i + w <= n) return i;
    atomicOr(&g_oob_flag, 1u);
    return 0;
}
__device__ __forceinline__ bool oob_ok(size_t i, size_t w, size_t n) {
    if (i + w <= n) return true;
    atomicOr(&g_oob_flag, 2u);
    return false;
}
#define CCM_IX(i, n) ::ccm::oob_ix((size_t)(i), 1, (size_t)(n))
#define CCM_IXW(i, w, n) ::ccm::oob_ix((size_t)(i), (size_t)(w), (size_t)(n))
#define CCM_OK(i, n) ::ccm::oob_ok((size_t)(i), 1, (size_t)(n))
#define CCM_OKW(i, w, n) ::ccm::oob_ok((size_t)(i), (size_t)(w), (size_t)(n))
#else
#define CCM_IX(i, n) (i)
#define CCM_IXW(i, w, n) (i)
#define CCM_OK(i, n) true
#define CCM_OKW(i, w, n) true
#endif
}  // namespace ccm
