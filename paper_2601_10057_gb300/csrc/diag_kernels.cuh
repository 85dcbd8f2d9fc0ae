// diag_kernels.cuh -- FP64 reductions outside the time step: initial SAVs,
// mass, the modified discrete energy and physical energy components, and
// the lambda-sum increment ||d^{n+1}||^2 of the modified energy.
#pragma once
#include "step_kernels.cuh"

namespace ccm {

enum { NDIAG = 14 };
// Sums (times h^2 where noted by the host):
//  0 (a^2-1-beta)^2/(4 eps)   1 6 a^2 gbar + (a^3-a)^2/eps^2   2 (1+p)f_in + (1-p)f_out
//  3 g(a)                     4 face sum (D a)^2               5 (Lap a)^2
//  6 (2 Lap a - Lap b)^2      7 face sum (D(2a-b))^2           8 face sum (D(a-b))^2
//  9 a^2                      10 (2a-b)^2                       11 ((a^3-a)/eps - eps Lap a)^2
//  12 f_osm                   13 psi
struct DiagCoef {
    double inv_h, inv_h2, eps, inv_eps, beta;
    double gin, gout, psin, psout, bin, bout;
};

template <typename T>
__device__ __forceinline__ double at(const T* u, int N, int i, int j) {
    i = i < 0 ? 0 : (i >= N ? N - 1 : i);
    j = j < 0 ? 0 : (j >= N ? N - 1 : j);
    return (double)u[(size_t)j * N + i];
}

// Blocks of 32 x 8 threads cover 32 x (8 kDiagRows) cells: each thread adds
// kDiagRows cells before the block reduction.
enum { kDiagRows = 8 };

template <typename T>
__global__ void __launch_bounds__(256)
k_diag(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ psi,
       double* __restrict__ part, int N, DiagCoef c) {
    __shared__ double sred[8 * NDIAG];
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    double v[NDIAG];
    for (int q = 0; q < NDIAG; ++q) v[q] = 0.0;
    for (int rr = 0; rr < kDiagRows; ++rr) {
        const int j = blockIdx.y * 8 * kDiagRows + 8 * rr + (threadIdx.x >> 5);
        if (i < N && j < N) {
            const double aC = at(a, N, i, j), aE = at(a, N, i + 1, j), aW = at(a, N, i - 1, j);
            const double aN = at(a, N, i, j + 1), aS = at(a, N, i, j - 1);
            const double bC = at(b, N, i, j), bE = at(b, N, i + 1, j), bW = at(b, N, i - 1, j);
            const double bN = at(b, N, i, j + 1), bS = at(b, N, i, j - 1);
            const double la = (aE + aW + aN + aS - 4 * aC) * c.inv_h2;
            const double lb = (bE + bW + bN + bS - 4 * bC) * c.inv_h2;
            const double gE = (aE - aC) * c.inv_h, gW = (aC - aW) * c.inv_h, gN = (aN - aC) * c.inv_h, gS = (aC - aS) * c.inv_h;
            const double gbar = 0.5 * (gE * gE + gW * gW) + 0.5 * (gN * gN + gS * gS);
            const double vv = aC * aC - 1.0 - c.beta;
            const double a3 = aC * aC * aC - aC;
            const double ps = (double)psi[(size_t)j * N + i];
            double sp, cp;
            sincospi(0.5 * aC, &sp, &cp);
            const double fin = 0.5 * c.gin * (ps - c.psin) * (ps - c.psin) + c.bin;
            const double fout = 0.5 * c.gout * (ps - c.psout) * (ps - c.psout) + c.bout;
            v[0] += vv * vv * 0.25 * c.inv_eps;
            v[1] += 6.0 * aC * aC * gbar + a3 * a3 * c.inv_eps * c.inv_eps;
            v[2] += (1.0 + sp) * fin + (1.0 - sp) * fout;
            v[3] += 0.25 * (aC * aC - 1.0) * (aC * aC - 1.0);
            // interior faces owned by this cell: east (i+1/2) and north (j+1/2)
            const double cE = 2 * aC - bC, cEe = 2 * aE - bE, cNn = 2 * aN - bN;
            const double dC = aC - bC, dEe = aE - bE, dNn = aN - bN;
            if (i + 1 < N) {
                v[4] += gE * gE;
                v[7] += (cEe - cE) * (cEe - cE) * c.inv_h2;
                v[8] += (dEe - dC) * (dEe - dC) * c.inv_h2;
            }
            if (j + 1 < N) {
                v[4] += gN * gN;
                v[7] += (cNn - cE) * (cNn - cE) * c.inv_h2;
                v[8] += (dNn - dC) * (dNn - dC) * c.inv_h2;
            }
            v[5] += la * la;
            v[6] += (2 * la - lb) * (2 * la - lb);
            v[9] += aC * aC;
            v[10] += cE * cE;
            const double w = a3 * c.inv_eps - c.eps * la;
            v[11] += w * w;
            v[12] += 0.5 * (1.0 + sp) * fin + 0.5 * (1.0 - sp) * fout;
            v[13] += ps;
        }
    }
    block_sum_store<NDIAG, double>(v, part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NDIAG, sred);
}

// ||d||^2 / (lam^2 h^2): sum over interior faces of (D w)^2 / M_psi(A phi*),
// w = psi^{n+1} - psi*, phi* = 2 phi^n - phi^{n-1}, psi* = 2 psi^n - psi^{n-1}.
template <typename T>
__global__ void __launch_bounds__(256)
k_dnorm(const T* __restrict__ phn, const T* __restrict__ pho, const T* __restrict__ psnew,
        const T* __restrict__ psn, const T* __restrict__ pso, double* __restrict__ part, int N, double M0) {
    __shared__ double sred[8];
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    double v[1] = {0.0};
    for (int rr = 0; rr < kDiagRows; ++rr) {
        const int j = blockIdx.y * 8 * kDiagRows + 8 * rr + (threadIdx.x >> 5);
        if (i < N && j < N) {
            auto ph = [&](int ii, int jj) { return 2.0 * at(phn, N, ii, jj) - at(pho, N, ii, jj); };
            auto w = [&](int ii, int jj) { return at(psnew, N, ii, jj) - (2.0 * at(psn, N, ii, jj) - at(pso, N, ii, jj)); };
            const double pC = ph(i, j), wC = w(i, j);
            auto mob = [&](double x) { double s = x * x - 1.0; return 1.0 - M0 * s * s; };
            if (i + 1 < N) { double d = w(i + 1, j) - wC; v[0] += d * d / mob(0.5 * (pC + ph(i + 1, j))); }
            if (j + 1 < N) { double d = w(i, j + 1) - wC; v[0] += d * d / mob(0.5 * (pC + ph(i, j + 1))); }
        }
    }
    block_sum_store<1, double>(v, part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x), sred);
}

// The five sums set_state needs for the initial SAVs and the arc length
// (columns 0-4 of k_diag; the other columns are written as 0) for FP32
// fields, in the FP32 arithmetic of the step's own stencil (sin/cos by the
// same polynomials) with double-float accumulation per thread.  k_diag
// evaluates every cell in FP64, whose issue rate on GB300 makes it a
// millisecond at N = 2048; this pass costs about as much as reading the two
// fields.
struct InitCoefF { float inv_h, eps, inv_eps, beta, gin, gout, psin, psout, bin, bout; };

static __global__ void __launch_bounds__(256)
k_init_sums_f32(const float* __restrict__ a, const float* __restrict__ psi, double* __restrict__ part, int N,
                InitCoefF c) {
    __shared__ double sred[8 * NDIAG];
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    float hi[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, lo[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    auto ld = [&](int ii, int jj) {
        ii = ii < 0 ? 0 : (ii >= N ? N - 1 : ii);
        jj = jj < 0 ? 0 : (jj >= N ? N - 1 : jj);
        return a[(size_t)jj * N + ii];
    };
    for (int rr = 0; rr < kDiagRows; ++rr) {
        const int j = blockIdx.y * 8 * kDiagRows + 8 * rr + (threadIdx.x >> 5);
        if (i < N && j < N) {
            const float aC = ld(i, j), aE = ld(i + 1, j), aW = ld(i - 1, j), aN = ld(i, j + 1), aS = ld(i, j - 1);
            const float gE = (aE - aC) * c.inv_h, gW = (aC - aW) * c.inv_h, gN = (aN - aC) * c.inv_h, gS = (aC - aS) * c.inv_h;
            const float gbar = 0.5f * (gE * gE + gW * gW) + 0.5f * (gN * gN + gS * gS);
            const float a2 = aC * aC, vv = a2 - 1.0f - c.beta, a3 = aC * (a2 - 1.0f);
            const float ps = psi[(size_t)j * N + i];
            float sp, cp;
            sincospi_<float>(0.5f * aC, &sp, &cp);
            const float fin = 0.5f * c.gin * (ps - c.psin) * (ps - c.psin) + c.bin;
            const float fout = 0.5f * c.gout * (ps - c.psout) * (ps - c.psout) + c.bout;
            float face = 0.f;
            if (i + 1 < N) face += gE * gE;
            if (j + 1 < N) face += gN * gN;
            const float v[5] = {vv * vv * 0.25f * c.inv_eps, 6.0f * a2 * gbar + a3 * a3 * c.inv_eps * c.inv_eps,
                                (1.0f + sp) * fin + (1.0f - sp) * fout, 0.25f * (a2 - 1.0f) * (a2 - 1.0f), face};
#pragma unroll
            for (int q = 0; q < 5; ++q) df_add(hi[q], lo[q], v[q]);
        }
    }
    double v[NDIAG];
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) v[q] = q < 5 ? (double)hi[q] + (double)lo[q] : 0.0;
    block_sum_store<NDIAG, double>(v, part + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NDIAG, sred);
}

// lamsum += scale * sum(part[0..nb)) in a fixed order (one block).
static __global__ void __launch_bounds__(256)
k_add_lamsum(const double* __restrict__ part, int nb, double scale, DevScalars* sc) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0 && sc->status == 0) sc->lamsum += scale * red[0];
}

// Upload of one FP64 field into the field precision T (FP32 psi: the
// dithered rounding of dither_round, so its stored mass carries no coherent
// rounding error), with a flag for non-finite values and, when
// part is given, per-block compensated (Neumaier) partial sums of the FP64
// values (part[2 b] + part[2 b + 1]), 256 threads per block.
template <typename T, bool DITHER>
__global__ void __launch_bounds__(256) k_upload(const double* __restrict__ in, T* __restrict__ out, size_t n,
                                                unsigned* __restrict__ bad, double* __restrict__ part) {
    double s = 0.0, c = 0.0;
    bool nonfinite = false;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const double x = in[q];
        nonfinite |= !isfinite(x);
        if constexpr (DITHER) {
            const float f = (float)x;
            out[q] = dither_round(f, (float)(x - (double)f), dither_key(0xffffffffu, (uint32_t)q) | 1u);
        } else {
            out[q] = (T)x;
        }
        if (part) {
            const double t = s + x;
            c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
            s = t;
        }
    }
    if (__any_sync(0xffffffffu, nonfinite) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
    if (part) {
        // (s, c) pairs added with TwoSum of the high parts, over the warp, then the warps
        __shared__ double ws[2][8];
        for (int o = 16; o > 0; o >>= 1) {
            const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
            const double t = s + s2, bb = t - s;
            c += c2 + ((s - (t - bb)) + (s2 - bb));
            s = t;
        }
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) { ws[0][w] = s; ws[1][w] = c; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double S = ws[0][0], C = ws[1][0];
            for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                const double t = S + ws[0][k], bb = t - S;
                C += ws[1][k] + ((S - (t - bb)) + (ws[0][k] - bb));
                S = t;
            }
            part[2 * blockIdx.x] = S;
            part[2 * blockIdx.x + 1] = C;
        }
    }
}

template <typename Tsrc, typename Tdst>
__global__ void k_convert(const Tsrc* __restrict__ in, Tdst* __restrict__ out, size_t n) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        out[q] = (Tdst)in[q];
}

}  // namespace ccm
