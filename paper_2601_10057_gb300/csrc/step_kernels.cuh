// step_kernels.cuh -- kernels of one CC-MSAV time step (templated on the
// field precision T = float or double).
//
// One step n -> n+1 (Sec. 3.2 of the paper, solved as in Appendix B) is
// computed in increment form: with the reference levels
//   phi_bar = (4 phi^n - phi^{n-1})/3   (BDF1 start step: phi_bar = phi^n),
//   X_bar   = (4 X^n - X^{n-1})/3 for each SAV X in V, U, W, Z (BDF1: X^n),
// the unknowns are d_phi = phi^{n+1} - phi_bar, d_psi = psi^{n+1} - psi_bar
// and the SAV increments.  The scheme's equations are unchanged: since
// chi phi_bar = C1 phi_bar - C2 Lap phi_bar + C3 Lap^2 phi_bar and C1 contains
// 3/(2 dt), the explicit right-hand sides of Appendix B Step 2 become
//   chi d_phi = f0' - sum_j c_j X_j^{n+1} F_j,
//     f0' = -beta' phi_bar - M_phi theta~ Lap phi* + C2 Lap phi_bar - C3 Lap^2 phi_bar,
//   zeta d_psi = g0' + Z^{n+1} LP,   g0' = lam Lap(psi_bar - psi*),
// and the SAV updates (eqs. V_BDF2 .. Z_BDF2) become X^{n+1} = X_bar +
// (F, d_phi) (+ (P, d_psi) for Z): 3 phi^{n+1} - 4 phi^n + phi^{n-1} = 3 d_phi.
// The 5x5 matrix of Step 4 is the same; only its right-hand side changes.
// In exact arithmetic this is the paper's step; in finite precision it keeps
// O(1) fields out of the transforms and the SAV algebra, so nothing of size
// (1/dt) phi or (F, phi) has to cancel.
//
//   k_stencil     phi*, phi_bar, psi*, psi_bar and the unnormalised fields
//                   f0', g0' (above),
//                   S  = phi*(phi*^2 - 1 - beta)/eps
//                   H  = 3 sqrt2/4 [(phi*^3 - phi*)/eps - eps Lap phi*]
//                   Q  = 6[phi*|grad phi*|^2 - div(phi*^2 grad phi*)]
//                        + (phi*^3 - phi*)(3 phi*^2 - 1)/eps^2
//                   K  = p'(phi*)(f_in - f_out)/2
//                   P  = [g_in(1+p)(psi*-psi_in) + g_out(1-p)(psi*-psi_out)]/2
//                   LP = div(M_psi(A phi*) grad P)           (eq. mobility_flux)
//                 plus per-block partial sums of the SAV radicands, the minimum
//                 face mobility and the sums of psi^n, psi^{n-1};
//   k_rowdct_T    forward DCT-II along x of the 8 fields, written transposed;
//   k_coldct_gram forward DCT-II along y (now contiguous), spectral Gram sums
//                 (Parseval: (u, chi^{-1} v)_h = h^2 sum_k u^ v^ / sigma_k) and
//                 the spectra needed for recovery;
//   k_solve       FP64 reduction of the partials, the 5x5 system (Appendix B
//                 Step 4), the SAV update and the recovery coefficients;
//   k_comb_icolT  recovery in spectral space
//                   d_phi^ = (f0'^ - aS S^ - aH H^ - aQ Q^ - aK K^) / sigma,
//                   d_psi^ = (g0'^ + aL LP^) / tau,
//                 inverse DCT along y, written transposed;
//   k_irow        inverse DCT along x and phi^{n+1} = phi_bar + d_phi,
//                 psi^{n+1} = psi_bar + d_psi.
#pragma once
#include <type_traits>
#include "dct_device.cuh"
#include "warp_fft.cuh"
#include "bounds.cuh"

namespace ccm {

enum { NRED1 = 10 };   // k_stencil partials: IV IW IZ sum(psi^n) sum(psi^{n-1}) (3 unused) minM (pad)
enum { NRED2 = 17 };   // gram partials: 15 chi pairs (a <= b over f0' S H Q K), PG, PL
enum { NF = 8 };       // fields out of k_stencil: f0' S H Q K P g0' LP

// Coefficients of k_stencil in the field precision T (converted once on the
// host: per-thread FP64 conversions would run on GB300's narrow FP64 pipe).
template <typename T>
struct StencilCoef {
    int bdf1;             // 1: start step (phi* = phi_bar = phi^n)
    T inv_h, inv_h2;
    T eps, inv_eps, inv_eps2, beta, quarter_inv_eps;
    T Mth;                // M_phi * theta~
    T C2, C3, betap;      // chi coefficients; betap = M_phi gamma_surf 3 sqrt2 beta / (4 eps)
    T lam;
    T gin, gout, hgin, hgout, psin, psout, bin, bout;
    T M0;
};

struct SpecCoef {          // sigma = C1 + C2 s + C3 s^2, tau = Ct + lam s, s = ev[kx] + ev[ky]
    double C1, C2, C3, Ct, lam;
};

// Device-resident scalar state of one simulation.
struct DevScalars {
    double V, U, W, Z;            // level n
    double Vo, Uo, Wo, Zo;        // level n-1
    double A;                     // target arc length
    double lamsum;                // sum_{j>=2} dt/2 ||d^j||^2
    double steps;                 // steps taken
    double mass_mode;             // conserved mean of psi (FP64) that the FP32 path keeps
    double alpha[5];              // recovery coefficients aS aH aQ aK aL
    double anchor;                // FP32 path: mean correction added to psi^{n+1}
    double dc_col;                // FP32 path: sum over y of the inverse column pass of the
                                  // zero-mean psi increment at kx = 0 (its DC leakage)
    double last[6];               // IV IW IZ minM and diagnostics of the last step
    int status;                   // 0 or a CCMSAV_E* code set on the device
    unsigned int solve_arrivals;  // blocks of k_solve done with their slice (reset by the last)
};

struct SolveCoef {
    double h2, cgs, cga, cgb, cgo;
    double inv_NN;                // 1 / points per field (exact: a power of two)
    int bdf1;
    int anchor;                   // FP32 path: compute the psi mean correction
    int nb1, nb2;                 // number of partial rows
};

struct SpecCoefF {        // FP32 copy of SpecCoef for the FP32 spectral kernels
    float C1, C2, C3, Ct, lam;
};

// Grouped launches (FP32 warp path): one launch of a step kernel serves
// several simulations of the same N.  blockIdx.x = simulation * bps + the
// block index the kernel has in a launch of its own (bps = that launch's
// gridDim.x), and the kernel takes from ga.a[simulation] the pointers and
// coefficients it otherwise receives as arguments.  Each simulation's blocks
// do exactly what its own launch does, so the results are the same bits.
// The records travel in the kernel parameters (__grid_constant__: read in
// place from the parameter bank, with a CTA-uniform index, so they cost no
// more registers than ordinary arguments); the kernels take a template flag
// GRP, and without it ga is an empty struct and the code is that of the
// plain kernel.
struct BatchArgs {
    const float* phn; const float* pho; const float* psn; const float* pso;   // levels n, n-1
    float* phi_new; float* psi_new;                                           // level n+1
    float* bufA; float* bufB;                                                 // the two field buffers
    double* part1; double* part2; double* part3;                              // partial rows, solve slices
    DevScalars* sc;
    const cplx<float>* tw2;                                                   // four-step twiddles
    wf::PairTwTab twF, twI;                                                   // DCT pair twiddles
    const float* evf; const float4* evp;                                      // FP32 eigenvalues
    StencilCoef<float> c;
    SpecCoefF sf;
    SolveCoef so;
};

// Simulations per grouped launch: 64 records of 328 bytes stay well inside
// the 32764 bytes of kernel parameters.
constexpr int kMaxGroup = 64;
template <bool GRP> struct GroupArgs { int unused = 0; };
template <> struct GroupArgs<true> { BatchArgs a[kMaxGroup]; };

// ------------------------------------------------------------------ helpers
template <typename T> __device__ __forceinline__ void sincospi_(T x, T* s, T* c);
// FP32: x = j + r with j = rint(x) and |r| <= 1/2 (exact), sin(pi r) =
// r P(r^2) and cos(pi r) = Q(r^2) with P, Q of degree 4 and 5 fitted in FP64
// by least squares at Chebyshev nodes (sinpi_fit.py in this package), then
// the sign (-1)^j.  Error within 2 ulp of 1; about half the instructions of
// the library routine, which also handles arguments of any size.
template <> __device__ __forceinline__ void sincospi_<float>(float x, float* s, float* c) {
    const float j = rintf(x);
    const float r = x - j, q = r * r;
    float ps = fmaf(q, 0.0776576623f, -0.598291278f);
    ps = fmaf(q, ps, 2.55007744f);
    ps = fmaf(q, ps, -5.1677103f);
    ps = fmaf(q, ps, 3.14159274f);
    float pc = fmaf(q, -0.0243963245f, 0.23493731f);
    pc = fmaf(q, pc, -1.33521199f);
    pc = fmaf(q, pc, 4.05870914f);
    pc = fmaf(q, pc, -4.93480206f);
    pc = fmaf(q, pc, 1.0f);
    const float sg = (static_cast<int>(j) & 1) ? -1.0f : 1.0f;
    *s = sg * (r * ps);
    *c = sg * pc;
}
template <> __device__ __forceinline__ void sincospi_<double>(double x, double* s, double* c) { sincospi(x, s, c); }

// bytes (a multiple of 16) at a 16-byte aligned global address into L2.
// The row-transform kernel prefetches the rows of the CTA one residency
// ahead (block id + resident CTAs): when that CTA starts on a freed slot its
// loads hit L2 instead of waiting for DRAM.  (Measured: a gain there; a loss
// in the other tiled kernels, whose first loads overlap better already.)
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p), "r"(bytes) : "memory");
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NV per-thread values over the block: the T-precision warp sum
// (FP32 for the FP32 path: at most 32 terms), then FP64 across warps.
// Writes NV doubles to out (one row of the partials array).
template <int NV, typename T>
__device__ void block_sum_store(T (&v)[NV], double* out, double* sm) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;     // blocks may be 2D
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T s = warp_sum(v[i]);
        if (lane == 0) sm[warp * NV + i] = (double)s;
    }
    __syncthreads();
    if (tid < NV) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sm[w * NV + tid];
        out[tid] = s;
    }
    __syncthreads();
}


// Warp sum carried as an unevaluated pair hi + lo (error-free transformation
// TwoSum of Knuth / Dekker double-length arithmetic), so that a warp of FP32
// values sums to ~2^-44 relative accuracy without FP64 per element.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ double warp_sum_exact(float x) {
    float hi = x, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, ohi, s, e);
        e += lo + olo;
        hi = s + e;                       // renormalise (Fast2Sum, |s| >= |e|)
        lo = e - (hi - s);
    }
    return (double)hi + (double)lo;
}
__device__ __forceinline__ double warp_sum_exact(double x) { return warp_sum(x); }

// Double-float (TwoSum) accumulation of FP32 values, then a sum over the G
// lanes of one lane group (xor offsets below G stay inside the group).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

// (hi, lo) += (bh, bl) in double-float arithmetic (TwoSum of the high parts)
__device__ __forceinline__ void df_add2(float& hi, float& lo, float bh, float bl) {
    float s, e;
    two_sum(hi, bh, s, e);
    e += lo + bl;
    hi = s + e;
    lo = e - (hi - s);
}
template <int G>
__device__ __forceinline__ double group_sum_exact(float hi, float lo) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, ohi, s, e);
        e += lo + olo;
        hi = s + e;
        lo = e - (hi - s);
    }
    return (double)hi + (double)lo;
}

// The same group sum kept as an unevaluated pair (no FP64 instruction)
template <int G>
__device__ __forceinline__ float2 group_sum_df(float hi, float lo) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
        df_add2(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
    return make_float2(hi, lo);
}

// Partial-sum rows read by k_solve: FP64 on the FP64 path; on the FP32 path
// unevaluated float pairs (hi, lo), formed without FP64 instructions (FP64
// issues at a small fraction of the FP32 rate on GB300), 8 bytes like a double.
template <typename T> struct PartialOf { using type = double; };
template <> struct PartialOf<float> { using type = float2; };

// block_sum_store into a partial row of the precision's type: for FP32 the
// T-precision warp sums are added over the warps in double-float.
template <int NV, typename T>
__device__ void block_sum_store_part(T (&v)[NV], typename PartialOf<T>::type* out, double* sm) {
    if constexpr (std::is_same<T, double>::value) {
        block_sum_store<NV, T>(v, out, sm);
    } else {
        float* smf = reinterpret_cast<float*>(sm);
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int nthr = blockDim.x * blockDim.y;
        const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float sw = warp_sum(v[i]);
            if (lane == 0) smf[warp * NV + i] = sw;
        }
        __syncthreads();
        if (tid < NV) {
            float hi = 0.f, lo = 0.f;
            for (int w = 0; w < nw; ++w) df_add(hi, lo, smf[w * NV + tid]);
            out[tid] = make_float2(hi, lo);
        }
        __syncthreads();
    }
}

// Per-thread accumulator of a field sum: double-float for FP32 fields, plain
// FP64 for FP64 fields.
template <typename T> struct ExactSum;
template <> struct ExactSum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) { df_add(hi, lo, x); }
    __device__ __forceinline__ double warp_total() { return group_sum_exact<32>(hi, lo); }
    __device__ __forceinline__ float2 warp_pair() { return group_sum_df<32>(hi, lo); }
};
template <> struct ExactSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double warp_total() { return warp_sum(s); }
};

// Neumann ghost cells by even reflection about the boundary face:
// index -1 -> 0, -2 -> 1, N -> N-1, N+1 -> N-2 (for halo 1 this is the
// mirror phi_0 = phi_1 of Appendix D; for halo 2 it makes Lap phi at a ghost
// cell equal the mirror of Lap phi, i.e. Lap^2 = Lap o Lap with mirrored ghosts).
// Tile cells farther out than that (the tile's far side on grids smaller than
// the tile) feed only results outside the grid, which are never stored; they
// are clamped into the grid so that every load stays inside the field.
__device__ __forceinline__ int reflect(int i, int N) {
    i = i < 0 ? -1 - i : (i >= N ? 2 * N - 1 - i : i);
    return min(max(i, 0), N - 1);
}

// Counter-based 32-bit hash (the "lowbias32" integer mixer: xor-shifts and
// odd multipliers) of a point index and a step key.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ uint32_t dither_key(uint32_t step, uint32_t idx) {
    return mix32(idx * 0x9e3779b9u ^ mix32(step + 0x632be5abu));
}

// Round s + r (|r| below about one ulp of s, r the exact residual) to a
// neighbouring float with probability proportional to closeness: adds a
// uniform dither of one ulp before rounding to nearest.  The stored FP32
// value is then unbiased and its rounding error uncorrelated between points,
// even where a whole region holds the same value, so a sub-ulp mean
// correction shifts the stored mass as intended.
__device__ __forceinline__ float dither_round(float s, float r, uint32_t key) {
    const int ex = (__float_as_int(s) >> 23) & 0xff;
    const float ulp = ex > 24 ? __int_as_float((ex - 23) << 23) : 1.17549435e-38f * 2.0f;
    // u in (-1/2, 1/2), never +-1/2: a float input with r = 0 is returned unchanged
    const float u = ((float)(key >> 8) + 0.5f) * (1.0f / 16777216.0f) - 0.5f;
    return s + fmaf(u, ulp, r);
}

// u^{n+1} = u_bar + du (+ anchor) with u_bar = u^n + (u^n - u^{n-1})/3
// (BDF1: u^n).  FP32: the two roundings are compensated (FMA residual and
// TwoSum), so the stored value is the correctly rounded u_bar + du + anchor
// and a sub-ulp anchor shifts the stored mean without bias.
// dither: 0 = round to nearest, else the key of dither_round.
__device__ __forceinline__ float bar_add(float a, float b, float du, float anc, bool bdf1, uint32_t dither = 0) {
    float t1 = a, e1 = 0.f;
    if (!bdf1) {
        const float d = a - b;
        t1 = fmaf(d, 1.0f / 3.0f, a);
        e1 = fmaf(d, 1.0f / 3.0f, a - t1);
    }
    float s, e2;
    two_sum(t1, du, s, e2);
    const float r = (e1 + e2) + anc;
    return dither ? dither_round(s, r, dither) : s + r;
}
// The same sum rounded to nearest with error feedback: carry (the exact
// rounding error of this thread's earlier values, value minus stored) is
// added before rounding and replaced by the new error (TwoSum), so the
// stored values of one thread sum to the exact values within half an ulp.
__device__ __forceinline__ float bar_add_fb(float a, float b, float du, float anc, bool bdf1, float& carry) {
    float t1 = a, e1 = 0.f;
    if (!bdf1) {
        const float d = a - b;
        t1 = fmaf(d, 1.0f / 3.0f, a);
        e1 = fmaf(d, 1.0f / 3.0f, a - t1);
    }
    float s, e2;
    two_sum(t1, du, s, e2);
    const float r = ((e1 + e2) + anc) + carry;
    float out;
    two_sum(s, r, out, carry);
    return out;
}
__device__ __forceinline__ double bar_add(double a, double b, double du, double anc, bool bdf1, uint32_t = 0) {
    return (bdf1 ? a : a + (a - b) / 3.0) + du + anc;
}

// ------------------------------------------------------------------ k_stencil
// Tile of TX x TYB cells per block of TX x TY threads (each thread handles
// TYB / TY cells of one column).  Shared-memory tiles: phi_bar with a
// two-cell halo (for Lap^2 phi_bar), and phi*, psi* (overwritten in place by
// the P numerator), psi_bar - psi* and Lap phi_bar with a one-cell halo.  Partial sums are
// accumulated per thread over its cells, then reduced once per block.
//
// FP32 fields: phi_bar = phi^n + (phi^n - phi^{n-1})/3 is kept as an
// unevaluated pair hi + lo (hi the FMA-rounded value, lo its exact residual,
// the same pair the final update u^{n+1} = u_bar + du forms), and lo enters
// Lap phi_bar, Lap^2 phi_bar and the beta' phi_bar term of f0'.  The linear
// part of f0' (C2 Lap - C3 Lap^2 - beta') phi_bar is nearly cancelled by the
// implicit operator in the recovery; with phi_bar rounded to FP32 here but
// not in the final update, the mismatch was fed back into phi every step
// (measured: 4.0e-5 max-norm deviation from the FP64 path after 1000 steps
// at N = 2048 with the rounded phi_bar, 2.6e-6 with phi_bar exact in f0').
constexpr int TX = 64, TY = 4, TYB = 32;
template <typename T> constexpr bool kBarLo = std::is_same<T, float>::value;

template <typename T, bool GRP = false>
__global__ void __launch_bounds__(TX * TY)
k_stencil(const T* __restrict__ phn, const T* __restrict__ pho,
          const T* __restrict__ psn, const T* __restrict__ pso,
          T* __restrict__ out, double* __restrict__ part, int N, StencilCoef<T> c,
          const __grid_constant__ GroupArgs<GRP> ga, int bps) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int W2 = TX + 4, W1 = TX + 2, H1 = TYB + 2;
    T* sbar = reinterpret_cast<T*>(smraw);              // [TYB+4][W2]
    T* sph = sbar + (TYB + 4) * W2;                     // [H1][W1] each below
    T* sps = sph + H1 * W1;
    T* sP = sps;              // the P numerator replaces psi* in the one-halo pass
    T* sdq = sps + H1 * W1;
    T* slb = sdq + H1 * W1;
    T* slo = slb + H1 * W1;   // FP32 only: [TYB+4][W2] low parts of phi_bar
    __shared__ double sred[(TX * TY / 32) * 4];
    __shared__ double smean[2][TX * TY / 32];
    __shared__ T smin[TX * TY / 32];
    int bx = blockIdx.x, gx = gridDim.x;
    if constexpr (GRP) {          // grouped launch (FP32)
        static_assert(std::is_same<T, float>::value, "grouped launches are FP32");
        const int sim = blockIdx.x / bps;
        bx = blockIdx.x - sim * bps;
        gx = bps;
        const BatchArgs& A = ga.a[sim];
        phn = A.phn; pho = A.pho; psn = A.psn; pso = A.pso; out = A.bufA; part = A.part1; c = A.c;
    }
    const int i0 = bx * TX, j0 = blockIdx.y * TYB;
    const int tid = threadIdx.y * TX + threadIdx.x;
    // with d = u^n - u^{n-1} (exact for nearby values): u* = u^n + d,
    // u_bar = u^n + d/3, u_bar - u* = -2d/3 (BDF1: u* = u_bar = u^n)
    const T kst = c.bdf1 ? (T)0 : (T)1, kbar = c.bdf1 ? (T)0 : (T)(1.0 / 3.0), kq = c.bdf1 ? (T)0 : (T)(-2.0 / 3.0);
    const T ih = c.inv_h, ih2 = c.inv_h2;
    const size_t NN = (size_t)N * N;
    ExactSum<T> sum_n, sum_o;
    // Halo load: thread (cx, ty) = (tid mod TX, tid / TX) takes tile column cx
    // in rows ty, ty + TY, ... (so its column, its reflection and its column
    // tests are fixed); the four right-hand halo columns TX .. TX + 3 are one
    // more item of the first 4 (TYB + 4) threads.  The global loads of NB
    // items are issued before any of them is used.  The sums of psi^n and
    // psi^{n-1} over the block's own cells are taken here, from the loaded
    // values.
    {
        constexpr int NT = TX * TY, RH = TYB + 4, NR = RH / TY, NI = NR + 1, NB = (NI + 1) / 2;
        static_assert(RH % TY == 0 && 4 * RH <= NT, "halo load mapping");
        const int cx = tid % TX, ty = tid / TX;
        const int gxc = reflect(i0 + cx - 2, N);
        const int ex_r = tid >> 2, ex_c = TX + (tid & 3);
        const bool ex_on = tid < 4 * RH;
        const int gxe = reflect(i0 + ex_c - 2, N);
#pragma unroll
        for (int u0 = 0; u0 < NI; u0 += NB) {
            T ra[NB], rb[NB], rc[NB], rd[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int u = u0 + b;
                ra[b] = rb[b] = rc[b] = rd[b] = (T)0;
                const bool ex = u == NR;
                if (u < NI && (!ex || ex_on)) {
                    const int lj = ex ? ex_r : ty + TY * u, li = ex ? ex_c : cx;
                    const size_t g = (size_t)reflect(j0 + lj - 2, N) * N + (ex ? gxe : gxc);
                    ra[b] = phn[CCM_IX(g, NN)];
                    rb[b] = pho[CCM_IX(g, NN)];
                    if (lj >= 1 && lj <= TYB + 2 && li >= 1 && li <= TX + 2) {
                        rc[b] = psn[CCM_IX(g, NN)];
                        rd[b] = pso[CCM_IX(g, NN)];
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int u = u0 + b;
                const bool ex = u == NR;
                if (u < NI && (!ex || ex_on)) {
                    const int lj = ex ? ex_r : ty + TY * u, li = ex ? ex_c : cx;
                    const T a = ra[b], da = a - rb[b];
                    if constexpr (kBarLo<T>) {
                        const T t1 = fmaf(da, kbar, a);
                        sbar[lj * W2 + li] = t1;
                        slo[lj * W2 + li] = fmaf(da, kbar, a - t1);
                    } else {
                        sbar[lj * W2 + li] = a + kbar * da;
                    }
                    if (lj >= 1 && lj <= TYB + 2 && li >= 1 && li <= TX + 2) {
                        const int o = (lj - 1) * W1 + (li - 1);
                        const T du = rc[b] - rd[b];
                        sph[o] = a + kst * da;
                        sps[o] = rc[b] + kst * du;
                        sdq[o] = kq * du;
                        if (lj >= 2 && lj <= TYB + 1 && li >= 2 && li <= TX + 1
                            && i0 + li - 2 < N && j0 + lj - 2 < N) {
                            sum_n.add(rc[b]);
                            sum_o.add(rd[b]);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    // One-halo region: Lap phi_bar (sums of neighbour differences: each
    // difference of nearby values is exact, so the rounding is relative to
    // the Laplacian, not to the field), p(phi*) = sin(pi phi*/2) once per
    // cell, the P numerator, and on the block's own cells K and the I_Z term.
    T acc2 = 0;
    for (int q = tid; q < W1 * H1; q += TX * TY) {
        const int lj1 = q / W1, li1 = q % W1;
        const T* b = sbar + (lj1 + 1) * W2 + li1 + 1;
        const T C = b[0];
        if constexpr (kBarLo<T>) {
            const T* bl = slo + (lj1 + 1) * W2 + li1 + 1;
            const T Cl = bl[0];
            const T lapl = ((bl[1] - Cl) + (bl[-1] - Cl)) + ((bl[W2] - Cl) + (bl[-W2] - Cl));
            slb[q] = ((((b[1] - C) + (b[-1] - C)) + ((b[W2] - C) + (b[-W2] - C))) + lapl) * ih2;
        } else {
            slb[q] = (((b[1] - C) + (b[-1] - C)) + ((b[W2] - C) + (b[-W2] - C))) * ih2;
        }
        const T ph = sph[q], ps = sps[q];
        T sp, cp;
        sincospi_<T>((T)0.5 * ph, &sp, &cp);
        sP[q] = (T)0.5 * (c.gin * ((T)1 + sp) * (ps - c.psin) + c.gout * ((T)1 - sp) * (ps - c.psout));
        const int gi = i0 + li1 - 1, gj = j0 + lj1 - 1;
        if (lj1 >= 1 && lj1 <= TYB && li1 >= 1 && li1 <= TX && gi < N && gj < N &&
            CCM_OK(4 * NN + (size_t)gj * N + gi, 8 * NN)) {
            const T fin = c.hgin * (ps - c.psin) * (ps - c.psin) + c.bin;
            const T fout = c.hgout * (ps - c.psout) * (ps - c.psout) + c.bout;
            out[4 * NN + (size_t)gj * N + gi] = (T)0.5 * ((T)1.5707963267948966192 * cp) * (fin - fout);
            acc2 += ((T)1 + sp) * fin + ((T)1 - sp) * fout;
        }
    }
    __syncthreads();
    T acc0 = 0, acc1 = 0;
    T mm = (T)1e30;
    const int gi = i0 + threadIdx.x;
    const int li = threadIdx.x + 1;
    for (int jj = threadIdx.y; jj < TYB; jj += TY) {
        const int lj = jj + 1, gj = j0 + jj;
        const bool inside = gi < N && gj < N;   // tiles overhang grids smaller than the tile
        const size_t g = inside ? (size_t)gj * N + gi : 0;
        const int o = lj * W1 + li;
        const T pC = sph[o], pE = sph[o + 1], pW = sph[o - 1], pN = sph[o + W1], pS = sph[o - W1];
        const T lapp = (((pE - pC) + (pW - pC)) + ((pN - pC) + (pS - pC))) * ih2;
        const T dC = sdq[o];
        const T lapd = (((sdq[o + 1] - dC) + (sdq[o - 1] - dC)) + ((sdq[o + W1] - dC) + (sdq[o - W1] - dC))) * ih2;
        const T lbC = slb[o];
        const T lap2b = (((slb[o + 1] - lbC) + (slb[o - 1] - lbC)) + ((slb[o + W1] - lbC) + (slb[o - W1] - lbC))) * ih2;
        const T p2 = pC * pC, p3m = pC * (p2 - (T)1);
        // face gradients (zero on boundary faces through the mirrored ghosts)
        const T gE = (pE - pC) * ih, gW = (pC - pW) * ih, gN = (pN - pC) * ih, gS = (pC - pS) * ih;
        const T gbar = (T)0.5 * (gE * gE + gW * gW) + (T)0.5 * (gN * gN + gS * gS);
        const T divp2g = (((T)0.5 * (p2 + pE * pE)) * gE - ((T)0.5 * (p2 + pW * pW)) * gW
                          + ((T)0.5 * (p2 + pN * pN)) * gN - ((T)0.5 * (p2 + pS * pS)) * gS) * ih;
        const T Snum = pC * (p2 - (T)1 - c.beta) * c.inv_eps;
        const T Hv = (T)1.0606601717798212866 * (p3m * c.inv_eps - c.eps * lapp);   // 3 sqrt2 / 4
        const T Qnum = (T)6 * (pC * gbar - divp2g) + p3m * ((T)3 * p2 - (T)1) * c.inv_eps2;
        const T PC = sP[o];
        // face mobilities M(A phi*) and the flux divergence of P
        auto mob = [&](T a) { T s = a * a - (T)1; return (T)1 - c.M0 * s * s; };
        const T mE = mob((T)0.5 * (pC + pE)), mW = mob((T)0.5 * (pC + pW));
        const T mN = mob((T)0.5 * (pC + pN)), mS = mob((T)0.5 * (pC + pS));
        const T LP = (mE * (sP[o + 1] - PC) - mW * (PC - sP[o - 1])
                      + mN * (sP[o + W1] - PC) - mS * (PC - sP[o - W1])) * ih2;
        const T bC = sbar[(lj + 1) * W2 + li + 1];
        T f0 = c.C2 * lbC - c.C3 * lap2b - c.Mth * lapp - c.betap * bC;
        if constexpr (kBarLo<T>) f0 = fmaf(-c.betap, slo[(lj + 1) * W2 + li + 1], f0);
        const T g0 = c.lam * lapd;
        if (inside && CCM_OK(7 * NN + g, 8 * NN)) {
            out[0 * NN + g] = f0;
            out[1 * NN + g] = Snum;
            out[2 * NN + g] = Hv;
            out[3 * NN + g] = Qnum;
            out[5 * NN + g] = PC;
            out[6 * NN + g] = g0;
            out[7 * NN + g] = LP;
            const T vv = p2 - (T)1 - c.beta;
            acc0 += vv * vv * c.quarter_inv_eps;
            acc1 += (T)6 * p2 * gbar + p3m * p3m * c.inv_eps2;
            // minimum face mobility over interior faces: each interior face
            // is the east or north face of exactly one cell (boundary faces
            // carry no flux)
            if (gi + 1 < N) mm = min(mm, mE);
            if (gj + 1 < N) mm = min(mm, mN);
        }
    }
    const size_t prow_i = (size_t)(blockIdx.y * gx + bx) * NRED1;
    const int lane = tid & 31, wp = tid >> 5;
    const T w0 = warp_sum(acc0), w1 = warp_sum(acc1), w2 = warp_sum(acc2);
    mm = warp_min(mm);
    if constexpr (std::is_same<T, float>::value) {
        // partial row of float pairs: I_V, I_W, I_Z, sum psi^n, sum psi^{n-1}, ..., min mobility
        float* sf = reinterpret_cast<float*>(sred);      // 8 floats per warp (sred holds 4 doubles per warp)
        const float2 sn = sum_n.warp_pair(), so = sum_o.warp_pair();
        if (lane == 0) {
            sf[wp * 8 + 0] = w0; sf[wp * 8 + 1] = w1; sf[wp * 8 + 2] = w2; sf[wp * 8 + 3] = sn.x;
            sf[wp * 8 + 4] = sn.y; sf[wp * 8 + 5] = so.x; sf[wp * 8 + 6] = so.y; sf[wp * 8 + 7] = mm;
        }
        __syncthreads();
        float2* prow = reinterpret_cast<float2*>(part) + prow_i;
        if (tid < 5) {
            float hi = 0.f, lo = 0.f;
            for (int w = 0; w < TX * TY / 32; ++w) {
                if (tid < 3) df_add(hi, lo, sf[w * 8 + tid]);
                else df_add2(hi, lo, sf[w * 8 + 3 + 2 * (tid - 3)], sf[w * 8 + 4 + 2 * (tid - 3)]);
            }
            prow[tid] = make_float2(hi, lo);
        } else if (tid == 5) {
            float m = sf[7];
            for (int w = 1; w < TX * TY / 32; ++w) m = fminf(m, sf[w * 8 + 7]);
            prow[5] = prow[6] = prow[7] = prow[9] = make_float2(0.f, 0.f);
            prow[8] = make_float2(m, 0.f);
        }
    } else {
        double* prow = part + prow_i;
        const double sn = sum_n.warp_total(), so = sum_o.warp_total();
        if (lane == 0) {
            sred[wp * 4 + 0] = (double)w0; sred[wp * 4 + 1] = (double)w1; sred[wp * 4 + 2] = (double)w2;
            smean[0][wp] = sn; smean[1][wp] = so; smin[wp] = mm;
        }
        __syncthreads();
        if (tid == 0) {
            double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
            T m = smin[0];
            for (int w = 0; w < TX * TY / 32; ++w) {
                a0 += sred[w * 4]; a1 += sred[w * 4 + 1]; a2 += sred[w * 4 + 2];
                a3 += smean[0][w]; a4 += smean[1][w];
                m = min(m, smin[w]);
            }
            prow[0] = a0; prow[1] = a1; prow[2] = a2; prow[3] = a3; prow[4] = a4;
            prow[5] = 0; prow[6] = 0; prow[7] = 0;
            prow[8] = (double)m; prow[9] = 0;
        }
    }
}

template <typename T> __host__ __device__ constexpr size_t stencil_smem_bytes() {
    return ((size_t)(kBarLo<T> ? 2 : 1) * (TYB + 4) * (TX + 4) + 4 * (size_t)(TYB + 2) * (TX + 2)) * sizeof(T);
}

// The pair k (0 <= k <= M/2) of the line transforms touches the modes
// k, N-k, M-k, M+k; u indexes them.  Each mode belongs to exactly one
// (k, u): N-0 does not exist, M-0 = M+0 and, at k = M/2, M-k = k and
// M+k = N-k.
__device__ __forceinline__ bool pair_mode_valid(int u, int k, int M) {
    switch (u) {
        case 0: return true;
        case 1: return k > 0;
        case 2: return k < M / 2;
        default: return k > 0 && k < M / 2;
    }
}

// ------------------------------------------------------------------ DCT geometry
struct Geo {
    int N, M;
    int ldc;            // padded complex line length
};

// ------------------------------------------------------------------ k_rowdct_T
// Forward DCT-II along x of RT rows (y0 .. y0+RT-1) of field blockIdx.y, then
// a transposed write: out[f][kx][y0 + r] = X_r[kx].
template <typename T>
__global__ void __launch_bounds__(512)
k_rowdct_T(const T* __restrict__ in, T* __restrict__ out, int N, int RT, int lds,
           const cplx<T>* __restrict__ twM, const PostTw<T>* __restrict__ twP) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = N / 2, ldc = padded_len(M);
    const int E = M < 8 ? M : 8, G = M / E, P = blockDim.x / G;
    T* stage = reinterpret_cast<T*>(smraw);                                   // RT x lds
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw + (((size_t)RT * lds * sizeof(T) + 15) & ~(size_t)15));
    const size_t NN = (size_t)N * N;
    const int f = blockIdx.y;
    const int y0 = blockIdx.x * RT;
    const T* src = in + f * NN;
    const T cn0 = (T)sqrt(1.0 / N), cn = (T)sqrt(2.0 / N);
    for (int r0 = 0; r0 < RT; r0 += P) {
        const int nr = min(P, RT - r0);
        // pack nr rows
        for (int q = threadIdx.x; q < nr * (M / 2); q += blockDim.x) {
            const int r = q / (M / 2), m = q % (M / 2);
            pack4(fb + (size_t)r * ldc, M, m, ld4(src + CCM_IXW((size_t)(y0 + r0 + r) * N + 4 * m, 4, NN)));
        }
        __syncthreads();
        fft_lines<T, false>(fb, ldc, nr, M, twM);
        for (int q = threadIdx.x; q < nr * (M / 2 + 1); q += blockDim.x) {
            const int r = q / (M / 2 + 1), k = q % (M / 2 + 1);
            Quad<T> X = post_forward(fb + (size_t)r * ldc, M, k, twP[k], cn0, cn);
            T* srow = stage + (size_t)(r0 + r) * lds;
            srow[k] = X.xk;
            if (pair_mode_valid(1, k, M)) srow[N - k] = X.xNk;
            if (pair_mode_valid(2, k, M)) srow[M - k] = X.xMk;
            if (pair_mode_valid(3, k, M)) srow[M + k] = X.xMpk;
        }
        __syncthreads();
    }
    T* dst = out + f * NN;
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q % RT, kx = q / RT;
        if (CCM_OK((size_t)kx * N + y0 + r, NN)) dst[(size_t)kx * N + y0 + r] = stage[(size_t)r * lds + kx];
    }
}

// ------------------------------------------------------------------ k_coldct_gram
// One spectral row kx per block: forward DCT-II along y of the 8 transposed
// fields, Gram partial sums, and the spectra spec[f][kx][ky] (slots in the
// order f0 S H Q K P g0 LP; slot 5 (P) is only written when the fields are
// transformed in groups, because P^ enters the Gram sums only).
// FG = number of field lines that fit in shared memory at once (8, 4, 2, 1).
template <typename T>
__device__ __forceinline__ void gram_accumulate(T (&acc)[NRED2], const T (&v)[NF], T isig, T itau) {
    int p = 0;
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = a; b < 5; ++b) acc[p++] += v[a] * v[b] * isig;
    acc[15] += v[5] * v[6] * itau;
    acc[16] += v[5] * v[7] * itau;
}

template <typename T>
__global__ void __launch_bounds__(512)
k_coldct_gram(const T* __restrict__ in, T* __restrict__ spec, double* __restrict__ part, int N, int FG,
              const cplx<T>* __restrict__ twM, const PostTw<T>* __restrict__ twP,
              const double* __restrict__ ev, SpecCoef sc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double sred[16 * NRED2];
    const int M = N / 2, ldc = padded_len(M);
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw);
    const size_t NN = (size_t)N * N;
    const int kx = blockIdx.x;
    const T cn0 = (T)sqrt(1.0 / N), cn = (T)sqrt(2.0 / N);
    T acc[NRED2];
#pragma unroll
    for (int i = 0; i < NRED2; ++i) acc[i] = 0;
    const double evx = ev[kx];
    for (int fg0 = 0; fg0 < NF; fg0 += FG) {
        for (int q = threadIdx.x; q < FG * (M / 2); q += blockDim.x) {
            const int f = q / (M / 2), m = q % (M / 2);
            pack4(fb + (size_t)f * ldc, M, m, ld4(in + CCM_IXW((fg0 + f) * NN + (size_t)kx * N + 4 * m, 4, NF * NN)));
        }
        __syncthreads();
        fft_lines<T, false>(fb, ldc, FG, M, twM);
        if (FG == NF) {
            for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) {
                Quad<T> X[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) X[f] = post_forward(fb + (size_t)f * ldc, M, k, twP[k], cn0, cn);
                const int kys[4] = {k, N - k, M - k, M + k};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!pair_mode_valid(u, k, M)) continue;
                    const int ky = kys[u];
                    const double s = evx + ev[ky];
                    const T isig = (T)(1.0 / (sc.C1 + sc.C2 * s + sc.C3 * s * s));
                    const T itau = (T)(1.0 / (sc.Ct + sc.lam * s));
                    T v[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        v[f] = (u == 0) ? X[f].xk : (u == 1) ? X[f].xNk : (u == 2) ? X[f].xMk : X[f].xMpk;
                    gram_accumulate(acc, v, isig, itau);
                    const size_t o = (size_t)kx * N + ky;
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        if (f != 5 && CCM_OK(f * NN + o, NF * NN)) spec[f * NN + o] = v[f];
                }
            }
        } else {
            for (int q = threadIdx.x; q < FG * (M / 2 + 1); q += blockDim.x) {
                const int f = q / (M / 2 + 1), k = q % (M / 2 + 1);
                Quad<T> X = post_forward(fb + (size_t)f * ldc, M, k, twP[k], cn0, cn);
                if (!CCM_OK((fg0 + f) * NN + (size_t)kx * N + (M + k < N ? M + k : N - 1), NF * NN)) continue;
                T* row = spec + (fg0 + f) * NN + (size_t)kx * N;
                row[k] = X.xk;
                if (pair_mode_valid(1, k, M)) row[N - k] = X.xNk;
                if (pair_mode_valid(2, k, M)) row[M - k] = X.xMk;
                if (pair_mode_valid(3, k, M)) row[M + k] = X.xMpk;
            }
        }
        __syncthreads();
    }
    if (FG != NF) {
        // Gram sums from the row just written (visible to the block after the barrier)
        for (int ky = threadIdx.x; ky < N; ky += blockDim.x) {
            const double s = evx + ev[ky];
            const T isig = (T)(1.0 / (sc.C1 + sc.C2 * s + sc.C3 * s * s));
            const T itau = (T)(1.0 / (sc.Ct + sc.lam * s));
            T v[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) v[f] = spec[CCM_IX(f * NN + (size_t)kx * N + ky, NF * NN)];
            gram_accumulate(acc, v, isig, itau);
        }
    }
    block_sum_store_part<NRED2, T>(acc, reinterpret_cast<typename PartialOf<T>::type*>(part) + (size_t)kx * NRED2, sred);
}

// ------------------------------------------------------------------ k_solve
// Single block: FP64 reduction of both partial arrays in a fixed order, then
// (thread 0) the scalar algebra of Appendix B Steps 1 and 4.
__device__ inline bool finite_(double x) { return isfinite(x); }

// kSolveBlocks blocks of kSolveThreads.  FP64 instructions issue at a small
// fraction of the FP32 rate on GB300 (about one warp instruction per 64-80
// cycles per SM sub-partition, dependent or not), so this kernel is laid out
// to execute few of them:
//  - the per-column sums run with one column per lane: block b adds its
//    slice of the partial rows; the block that finishes last (an atomic
//    arrival count; nothing waits) adds the slices, split over its warps;
//  - the minimum column (minimum face mobility) is reduced through
//    order-preserving integer keys;
//  - one warp solves the 5x5 system of Appendix B Step 4 holding one entry
//    of the augmented matrix per lane (Gauss-Jordan elimination with partial
//    pivoting, pivots compared as integer magnitudes).
// Every sum runs in a fixed order, so the result is deterministic.
enum { NRQ = NRED1 + NRED2, kSolveThreads = 128, kSolveBlocks = 128, kSolveMinCol = 8 };
static_assert(NRQ <= 32, "one column per lane");
static_assert(kSolveBlocks == 32 * (kSolveThreads / 32), "32 slices per warp in the last block");

// total order of doubles as signed 64-bit integers
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double from_order_key(long long k) {
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffLL);
}

// rows [b * per, min(n, (b + 1) * per)) of an n-row array belong to block b
__device__ __forceinline__ void solve_slice(int n, int b, int& r0, int& cnt) {
    const int per = (n + kSolveBlocks - 1) / kSolveBlocks;
    r0 = min(n, b * per);
    cnt = min(n, r0 + per) - r0;
}

template <typename P, bool GRP = false>
__global__ void __launch_bounds__(kSolveThreads)
k_solve(const P* __restrict__ p1, int nb1, const P* __restrict__ p2, int nb2,
        double* __restrict__ slices, DevScalars* sc, SolveCoef co,
        const __grid_constant__ GroupArgs<GRP> ga, int bps) {
    constexpr int NR = NRQ;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ double fin_[NR];
    __shared__ double part[kSolveThreads / 32][NR];
    __shared__ double s_state[10];       // V U W Z at n and n-1, conserved mean, steps
    __shared__ int s_status, is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int bx = blockIdx.x, gx = gridDim.x;
    if constexpr (GRP) {                 // grouped launch (FP32)
        static_assert(std::is_same<P, float2>::value, "grouped launches are FP32");
        const int sim = blockIdx.x / bps;
        bx = blockIdx.x - sim * bps;
        gx = bps;
        const BatchArgs& A = ga.a[sim];
        p1 = reinterpret_cast<const P*>(A.part1); p2 = reinterpret_cast<const P*>(A.part2);
        nb1 = A.so.nb1; nb2 = A.so.nb2; slices = A.part3; sc = A.sc; co = A.so;
    }
    if (threadIdx.x == 32) {             // the scalar state, read while warp 0 streams
        s_state[0] = sc->V; s_state[1] = sc->U; s_state[2] = sc->W; s_state[3] = sc->Z;
        s_state[4] = sc->Vo; s_state[5] = sc->Uo; s_state[6] = sc->Wo; s_state[7] = sc->Zo;
        s_state[8] = sc->mass_mode; s_state[9] = sc->steps; s_status = sc->status;
    }
    // this block's slice: lane c of warp 0 adds column c
    if (warp == 0 && lane < NR) {
        const int c = lane;
        const bool in1 = c < NRED1;
        const P* col = in1 ? p1 + c : p2 + (c - NRED1);
        const int stride = in1 ? NRED1 : NRED2;
        int r0, cnt;
        solve_slice(in1 ? nb1 : nb2, bx, r0, cnt);
        double acc = 0.0;
        long long kmin = 0x7fffffffffffffffLL;
        if constexpr (std::is_same<P, float2>::value) {
            // FP32 path: float pairs added in double-float, one conversion per column
            float hi = 0.f, lo = 0.f, fm = 3.0e38f;
            for (int r = 0; r < cnt; r += 16) {
                float2 v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = (r + u < cnt) ? col[(size_t)(r0 + r + u) * stride] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (r + u >= cnt) break;
                    if (c == kSolveMinCol) fm = fminf(fm, v[u].x);
                    else df_add2(hi, lo, v[u].x, v[u].y);
                }
            }
            if (c == kSolveMinCol) kmin = order_key((double)fm);
            else acc = (double)hi + (double)lo;
        } else {
            for (int r = 0; r < cnt; r += 8) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = (r + u < cnt) ? col[(size_t)(r0 + r + u) * stride] : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (r + u >= cnt) break;
                    if (c == kSolveMinCol) kmin = min(kmin, order_key(v[u]));
                    else acc += v[u];
                }
            }
        }
        slices[(size_t)bx * NR + c] = (c == kSolveMinCol) ? __longlong_as_double(kmin) : acc;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&sc->solve_arrivals, 1u) == (unsigned)gx - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // last block: warp w adds slices 32 w .. 32 w + 31 of every column
    if (lane < NR) {
        const int c = lane;
        double v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = __ldcg(slices + (size_t)(32 * warp + q) * NR + c);
        // four independent FP64 chains (a dependent FP64 add waits ~30 ns on this GPU)
        double a4[4] = {0.0, 0.0, 0.0, 0.0};
        long long kmin = 0x7fffffffffffffffLL;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            if (c == kSolveMinCol) kmin = min(kmin, __double_as_longlong(v[q]));
            else a4[q & 3] += v[q];
        }
        part[warp][c] = (c == kSolveMinCol) ? __longlong_as_double(kmin) : (a4[0] + a4[1]) + (a4[2] + a4[3]);
    }
    if (threadIdx.x == 0) sc->solve_arrivals = 0u;
    __syncthreads();
    if (warp != 0) return;
    if (lane < NR) {
        const int c = lane;
        if (c == kSolveMinCol) {
            long long kmin = __double_as_longlong(part[0][c]);
#pragma unroll
            for (int w = 1; w < kSolveThreads / 32; ++w) kmin = min(kmin, __double_as_longlong(part[w][c]));
            fin_[c] = from_order_key(kmin);
        } else {
            double acc = part[0][c];
#pragma unroll
            for (int w = 1; w < kSolveThreads / 32; ++w) acc += part[w][c];
            fin_[c] = acc;
        }
    }
    __syncwarp();
    if (s_status != 0) return;
    const double* r = fin_;
    const double IV = r[0], IW = r[1], IZ = r[2], sum_n = r[3], sum_o = r[4], minM = r[kSolveMinCol];
    const double* Gm = r + NRED1;
    const bool fin_ok = __all_sync(FULL, lane >= NR || finite_(r[lane < NR ? lane : 0]));
    if (!(fin_ok && IV > 0 && IW > 0 && IZ > 0 && minM > 0)) {
        if (lane == 0) sc->status = -5;
        return;
    }
    const double h2 = co.h2;
    // normalisations 1/(2 sqrt I_V), 1/sqrt I_W, 1/sqrt I_Z (lanes 0, 1, 2)
    const double rr = rsqrt(h2 * (lane == 0 ? IV : lane == 1 ? IW : IZ));
    const double nS = 0.5 * __shfl_sync(FULL, rr, 0), nQ = __shfl_sync(FULL, rr, 1), nK = __shfl_sync(FULL, rr, 2);
    // reference SAVs X_bar (Step 1 with the increments taken about phi_bar), lane q < 4
    constexpr double third = 1.0 / 3.0;
    const int q4 = lane & 3;
    const double x0q = s_state[q4], xpq = s_state[4 + q4];
    const double xbq = co.bdf1 ? x0q : (4.0 * x0q - xpq) * third;
    auto nrm_of = [&](int q) { return q == 0 ? nS : q == 1 ? 1.0 : q == 2 ? nQ : nK; };
    auto cc_of = [&](int q) { return q == 0 ? co.cgs : q == 1 ? co.cga : q == 2 ? co.cgb : co.cgo; };
    const double wq = cc_of(q4) * xbq * nrm_of(q4);
    double xb[4], w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { xb[q] = __shfl_sync(FULL, xbq, q); w[q] = __shfl_sync(FULL, wq, q); }
    // Gram entry (a, b) over (f0', S, H, Q, K), stored for a <= b row by row
    auto G = [&](int ga, int gb) -> double {
        const int lo = ga < gb ? ga : gb, hi = ga < gb ? gb : ga;
        return Gm[lo * 5 - lo * (lo - 1) / 2 + (hi - lo)];
    };
    // entry (i, j) of the augmented matrix [A | b] on lane 6 i + j
    const int l = lane < 30 ? lane : 29;
    const int i = l / 6, j = l % 6;
    double a;
    if (i < 4) {
        const double ni = nrm_of(i);
        if (j < 5) {
            const double nj = j < 4 ? nrm_of(j) : nK, cj = j < 4 ? cc_of(j) : co.cgo;
            a = (i == j ? 1.0 : 0.0) + cj * (h2 * ni * nj * G(i + 1, j < 4 ? j + 1 : 4));
        } else {
            double bi = G(0, i + 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) bi -= w[q] * G(i + 1, q + 1);
            a = h2 * ni * bi;
        }
    } else {
        const double PL = h2 * nK * nK * Gm[16];
        a = j == 3 ? -PL : j == 4 ? 1.0 - PL : j == 5 ? h2 * nK * Gm[15] + xb[3] * PL : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const unsigned long long mag = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
        unsigned long long best = __shfl_sync(FULL, mag, 6 * k + k);
        int piv = k;
#pragma unroll
        for (int rr2 = k + 1; rr2 < 5; ++rr2) {
            const unsigned long long m = __shfl_sync(FULL, mag, 6 * rr2 + k);
            if (m > best) { best = m; piv = rr2; }
        }
        if (best == 0ull) {
            if (lane == 0) sc->status = -5;
            return;
        }
        a = __shfl_sync(FULL, a, i == k ? 6 * piv + j : i == piv ? 6 * k + j : l);
        const double rinv = 1.0 / __shfl_sync(FULL, a, 6 * k + k);
        const double akj = __shfl_sync(FULL, a, 6 * k + j) * rinv;
        const double aik = __shfl_sync(FULL, a, 6 * i + k);
        a = (i == k) ? akj : a - aik * akj;
    }
    double x[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) x[q] = __shfl_sync(FULL, a, 6 * q + 5);
    if (lane != 0) return;
    const double V0 = s_state[0], U0 = s_state[1], W0 = s_state[2], Z0 = s_state[3];
    const double Vn = xb[0] + x[0], Un = xb[1] + x[1], Wn = xb[2] + x[2], Zn = xb[3] + x[3] + x[4];
    bool ok2 = finite_(Vn) && finite_(Un) && finite_(Wn) && finite_(Zn);
    if (!ok2) { sc->status = -5; return; }
    sc->Vo = V0; sc->Uo = U0; sc->Wo = W0; sc->Zo = Z0;
    sc->V = Vn; sc->U = Un; sc->W = Wn; sc->Z = Zn;
    sc->alpha[0] = co.cgs * Vn * nS;
    sc->alpha[1] = co.cga * Un;
    sc->alpha[2] = co.cgb * Wn * nQ;
    sc->alpha[3] = co.cgo * Zn * nK;
    sc->alpha[4] = Zn * nK;
    // FP32 path: psi^{n+1} = psi_bar + d_psi + anchor keeps the stored mean at
    // the conserved value (means of the stored levels summed to ~1e-13)
    if (co.anchor) {
        const double mn = sum_n * co.inv_NN, mo = sum_o * co.inv_NN;
        const double mbar = co.bdf1 ? mn : mn + (mn - mo) * third;
        sc->anchor = s_state[8] - mbar;
    } else {
        sc->anchor = 0.0;
    }
    sc->last[0] = IV; sc->last[1] = IW; sc->last[2] = IZ; sc->last[3] = minM;
    sc->steps = s_state[9] + 1.0;
}

// ------------------------------------------------------------------ k_comb_icolT
// Rows kx0 .. kx0+RT-1 of the spectra: recovery combination, inverse DCT
// along ky (DCT-III), transposed write out[f][y][kx] for f = phi, psi.
template <typename T>
__global__ void __launch_bounds__(512)
k_comb_icolT(const T* __restrict__ spec, T* __restrict__ out, int N, int RT, int lds,
             const cplx<T>* __restrict__ twM, const PostTw<T>* __restrict__ twP,
             const double* __restrict__ ev, SpecCoef sc, const DevScalars* __restrict__ dsc,
             int anchor_mass) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = N / 2, ldc = padded_len(M);
    const int E = M < 8 ? M : 8, G = M / E, P = blockDim.x / G;
    T* stage = reinterpret_cast<T*>(smraw);                                   // 2 RT x lds
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw + (((size_t)2 * RT * lds * sizeof(T) + 15) & ~(size_t)15));
    const size_t NN = (size_t)N * N;
    const int kx0 = blockIdx.x * RT;
    const T inv0 = (T)(1.0 / (M * sqrt(1.0 / N))), inv = (T)(1.0 / (M * sqrt(2.0 / N)));
    const T aS = (T)dsc->alpha[0], aH = (T)dsc->alpha[1], aQ = (T)dsc->alpha[2], aK = (T)dsc->alpha[3], aL = (T)dsc->alpha[4];
    const int nlines = 2 * RT;   // line l: row r = l / 2, field f = l % 2
    for (int l0 = 0; l0 < nlines; l0 += P) {
        const int nl = min(P, nlines - l0);
        for (int q = threadIdx.x; q < nl * (M / 2 + 1); q += blockDim.x) {
            const int l = l0 + q / (M / 2 + 1), k = q % (M / 2 + 1);
            const int r = l >> 1, f = l & 1;
            const int kx = kx0 + r;
            const double evx = ev[kx];
            const int kys[4] = {k, N - k, M - k, M + k};
            T vals[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int ky = kys[u];
                if (u == 1 && k == 0) { vals[u] = 0; continue; }
                const double s = evx + ev[ky];
                const size_t o = CCM_IX((size_t)kx * N + ky, NN);
                if (f == 0) {
                    const T isig = (T)(1.0 / (sc.C1 + sc.C2 * s + sc.C3 * s * s));
                    vals[u] = (spec[0 * NN + o] - aS * spec[1 * NN + o] - aH * spec[2 * NN + o]
                               - aQ * spec[3 * NN + o] - aK * spec[4 * NN + o]) * isig;
                } else {
                    const T itau = (T)(1.0 / (sc.Ct + sc.lam * s));
                    vals[u] = (spec[6 * NN + o] + aL * spec[7 * NN + o]) * itau;
                    // d_psi has zero mean (mass conservation); the FP32 path sets the zero
                    // mode exactly and keeps the stored mean with the anchor in k_irow
                    if (anchor_mass && kx == 0 && ky == 0) vals[u] = (T)0;
                }
            }
            Quad<T> X{vals[0], vals[1], vals[2], vals[3]};
            cplx<T> zk, zMk;
            pre_inverse(X, k, twP[k], inv0, inv, zk, zMk);
            cplx<T>* z = fb + (size_t)(l - l0) * ldc;
            z[padc(k)] = zk;
            if (k > 0) z[padc(M - k)] = zMk;
        }
        __syncthreads();
        fft_lines<T, true>(fb, ldc, nl, M, twM);
        for (int q = threadIdx.x; q < nl * (M / 2); q += blockDim.x) {
            const int l = l0 + q / (M / 2), m = q % (M / 2);
            vec4<T> v = unpack4(fb + (size_t)(l - l0) * ldc, M, m);
            const int r = l >> 1, f = l & 1;
            T* srow = stage + (size_t)(f * RT + r) * lds + 4 * m;
            srow[0] = v.a; srow[1] = v.b; srow[2] = v.c; srow[3] = v.d;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < 2 * RT * N; q += blockDim.x) {
        const int r = q % RT, rest = q / RT;
        const int y = rest % N, f = rest / N;
        if (CCM_OK(f * NN + (size_t)y * N + kx0 + r, 2 * NN))
            out[f * NN + (size_t)y * N + kx0 + r] = stage[(size_t)(f * RT + r) * lds + y];
    }
}

// ------------------------------------------------------------------ k_irow
// Inverse DCT along x of PR rows (2 fields each) of the transposed buffer:
// in[f][y][kx] -> phi_new / psi_new [y][x].
template <typename T>
__global__ void __launch_bounds__(512)
k_irow(const T* __restrict__ in, T* __restrict__ phi_new, T* __restrict__ psi_new, int N, int PR,
       const cplx<T>* __restrict__ twM, const PostTw<T>* __restrict__ twP,
       const T* __restrict__ phn, const T* __restrict__ pho, const T* __restrict__ psn, const T* __restrict__ pso,
       int bdf1, const DevScalars* __restrict__ dsc, int anchor_mass) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = N / 2, ldc = padded_len(M);
    const int E = M < 8 ? M : 8, G = M / E, P = blockDim.x / G;
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw);
    const size_t NN = (size_t)N * N;
    const int y0 = blockIdx.x * PR;
    const T inv0 = (T)(1.0 / (M * sqrt(1.0 / N))), inv = (T)(1.0 / (M * sqrt(2.0 / N)));
    const int nlines = 2 * PR;
    const T anc = anchor_mass ? (T)dsc->anchor : (T)0;
    const uint32_t step = (uint32_t)dsc->steps;         // dither key
    for (int l0 = 0; l0 < nlines; l0 += P) {
        const int nl = min(P, nlines - l0);
        for (int q = threadIdx.x; q < nl * (M / 2 + 1); q += blockDim.x) {
            const int l = l0 + q / (M / 2 + 1), k = q % (M / 2 + 1);
            const int r = l >> 1, f = l & 1;
            const T* row = in + CCM_IXW(f * NN + (size_t)(y0 + r) * N, N, 2 * NN);
            Quad<T> X{row[k], k > 0 ? row[N - k] : (T)0, row[M - k], row[M + k]};
            cplx<T> zk, zMk;
            pre_inverse(X, k, twP[k], inv0, inv, zk, zMk);
            cplx<T>* z = fb + (size_t)(l - l0) * ldc;
            z[padc(k)] = zk;
            if (k > 0) z[padc(M - k)] = zMk;
        }
        __syncthreads();
        fft_lines<T, true>(fb, ldc, nl, M, twM);
        for (int q = threadIdx.x; q < nl * (M / 2); q += blockDim.x) {
            const int l = l0 + q / (M / 2), m = q % (M / 2);
            const int r = l >> 1, f = l & 1;
            const size_t off = CCM_IXW((size_t)(y0 + r) * N + 4 * m, 4, NN);
            vec4<T> v = unpack4(fb + (size_t)(l - l0) * ldc, M, m);
            const vec4<T> a = ld4((f == 0 ? phn : psn) + off), b = ld4((f == 0 ? pho : pso) + off);
            const T an = (f == 1) ? anc : (T)0;
            const bool dth = (f == 1) && anchor_mass;
            const uint32_t i0 = (uint32_t)off;
            v.a = bar_add(a.a, b.a, v.a, an, bdf1 != 0, dth ? dither_key(step, i0) | 1u : 0u);
            v.b = bar_add(a.b, b.b, v.b, an, bdf1 != 0, dth ? dither_key(step, i0 + 1) | 1u : 0u);
            v.c = bar_add(a.c, b.c, v.c, an, bdf1 != 0, dth ? dither_key(step, i0 + 2) | 1u : 0u);
            v.d = bar_add(a.d, b.d, v.d, an, bdf1 != 0, dth ? dither_key(step, i0 + 3) | 1u : 0u);
            st4((f == 0 ? phi_new : psi_new) + off, v);
        }
        __syncthreads();
    }
}

}  // namespace ccm
