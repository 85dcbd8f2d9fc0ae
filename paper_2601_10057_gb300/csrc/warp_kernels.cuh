// warp_kernels.cuh -- FP32 step kernels built on the warp-level line FFT
// (N = 2M in 128 .. 2048).  Same data flow as the block-FFT kernels of
// step_kernels.cuh:
//   kw_rowdct_T    forward DCT-II along x, transposed write (RT rows per CTA)
//   kw_coldct_gram forward DCT-II along y of the 8 fields of KC spectral rows,
//                  Gram partial sums and the spectra (post-processed from all
//                  8 line buffers at once, so no staging copy)
//   kw_comb_icolT  recovery combination, inverse DCT along y, transposed write
//   kw_irow        inverse DCT along x, with the FP32 conserved mean of psi
//                  added back per point
// Every warp owns one line buffer per lane group (32 / G lines per warp).
#pragma once
#include "step_kernels.cuh"
#include "warp_fft.cuh"

namespace ccm {

struct SpecCoefF {        // FP32 copy of SpecCoef for the FP32 spectral kernels
    float C1, C2, C3, Ct, lam;
};

constexpr int kWarps = 8;

// Double-float (TwoSum) accumulation of FP32 values, then a sum over the G
// lanes of one line group (xor offsets below G stay inside the group).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
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

template <int M> struct WGeo {
    static constexpr int E = wf::Shape<M>::E, G = wf::Shape<M>::G;
    static constexpr int LPW = 32 / G;                  // lines per warp
    static constexpr int SLOTS = kWarps * LPW;          // line buffers per CTA
    static constexpr int BUF = wf::buf_len<M>();        // complex per buffer
    static constexpr size_t buf_bytes() { return (size_t)SLOTS * BUF * sizeof(cplx<float>); }
};

// ------------------------------------------------------------------ kw_rowdct_T
template <int M>
__global__ void __launch_bounds__(kWarps * 32)
kw_rowdct_T(const float* __restrict__ in, float* __restrict__ out, int RT, int lds,
            const cplx<float>* __restrict__ tw2, const PostTw<float>* __restrict__ twP) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    float* stage = reinterpret_cast<float*>(smraw + Gm::buf_bytes());
    const size_t NN = (size_t)N * N;
    const int f = blockIdx.y, y0 = blockIdx.x * RT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / G, n2 = lane % G;
    const int slot = warp * Gm::LPW + grp;
    cplx<float>* buf = bufs + (size_t)slot * Gm::BUF;
    const float cn0 = sqrtf(1.0f / N), cn = sqrtf(2.0f / N);
    for (int l0 = 0; l0 < RT; l0 += Gm::SLOTS) {
        const int l = l0 + slot;
        const bool act = l < RT;
        const float* x = in + f * NN + (size_t)(y0 + (act ? l : 0)) * N;
        cplx<float> v[E];
        wf::pack_fwd_global<M>(x, v, n2);
        wf::fourstep<float, M, false>(v, buf, tw2, n2);
        if (act) {
            float* srow = stage + (size_t)l * lds;
            for (int k = n2; k <= M / 2; k += G) {
                const Quad<float> X = wf::post_pair(buf[k], buf[(M - k) & (M - 1)], k, twP[k], cn0, cn);
                srow[k] = X.xk;
                if (pair_mode_valid(1, k, M)) srow[N - k] = X.xNk;
                if (pair_mode_valid(2, k, M)) srow[M - k] = X.xMk;
                if (pair_mode_valid(3, k, M)) srow[M + k] = X.xMpk;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    float* dst = out + f * NN;
    const int R4 = RT / 4;
    for (int q = threadIdx.x; q < R4 * N; q += blockDim.x) {
        const int r4 = q % R4, kx = q / R4;
        const float* s = stage + (size_t)(4 * r4) * lds + kx;
        *reinterpret_cast<float4*>(dst + (size_t)kx * N + y0 + 4 * r4) =
            make_float4(s[0], s[lds], s[2 * lds], s[3 * lds]);
    }
}

// ------------------------------------------------------------------ kw_coldct_gram
template <int M>
__global__ void __launch_bounds__(kWarps * 32)
kw_coldct_gram(const float* __restrict__ in, float* __restrict__ spec, double* __restrict__ part,
               const cplx<float>* __restrict__ tw2, const PostTw<float>* __restrict__ twP,
               const float* __restrict__ evf, SpecCoefF sc) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E, KC = Gm::SLOTS / NF;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double sred[kWarps * NRED2];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    const int kx0 = blockIdx.x * KC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / G, n2 = lane % G;
    const int slot = warp * Gm::LPW + grp;               // line = (kc, field)
    const int kc = slot / NF, f = slot % NF;
    {
        cplx<float> v[E];
        wf::pack_fwd_global<M>(in + f * NN + (size_t)(kx0 + kc) * N, v, n2);
        wf::fourstep<float, M, false>(v, bufs + (size_t)slot * Gm::BUF, tw2, n2);
    }
    __syncthreads();
    const float cn0 = sqrtf(1.0f / N), cn = sqrtf(2.0f / N);
    float acc[NRED2];
#pragma unroll
    for (int i = 0; i < NRED2; ++i) acc[i] = 0.f;
    for (int q = threadIdx.x; q < KC * (M / 2 + 1); q += blockDim.x) {
        const int c = q / (M / 2 + 1), k = q % (M / 2 + 1);
        const int kx = kx0 + c;
        Quad<float> X[NF];
#pragma unroll
        for (int g = 0; g < NF; ++g) {
            const cplx<float>* b = bufs + (size_t)(c * NF + g) * Gm::BUF;
            X[g] = wf::post_pair(b[k], b[(M - k) & (M - 1)], k, twP[k], cn0, cn);
        }
        const float evx = evf[kx];
        const int kys[4] = {k, N - k, M - k, M + k};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!pair_mode_valid(u, k, M)) continue;
            const int ky = kys[u];
            const float s = evx + evf[ky];
            const float isig = 1.0f / (sc.C1 + s * (sc.C2 + sc.C3 * s));
            const float itau = 1.0f / (sc.Ct + sc.lam * s);
            float v[NF];
#pragma unroll
            for (int g = 0; g < NF; ++g)
                v[g] = (u == 0) ? X[g].xk : (u == 1) ? X[g].xNk : (u == 2) ? X[g].xMk : X[g].xMpk;
            gram_accumulate(acc, v, isig, itau);
            const size_t o = (size_t)kx * N + ky;
#pragma unroll
            for (int g = 0; g < NF; ++g)
                if (g != 5) spec[g * NN + o] = v[g];
        }
    }
    block_sum_store<NRED2, float>(acc, part + (size_t)blockIdx.x * NRED2, sred);
}

// ------------------------------------------------------------------ kw_comb_icolT
// RT spectral rows per CTA, two lines (phi^, psi^) per row.
template <int M>
__global__ void __launch_bounds__(kWarps * 32)
kw_comb_icolT(const float* __restrict__ spec, float* __restrict__ out, int RT, int lds,
              const cplx<float>* __restrict__ tw2, const PostTw<float>* __restrict__ twP,
              const float* __restrict__ evf, SpecCoefF sc, DevScalars* __restrict__ dsc,
              int anchor_mass) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    float* stage = reinterpret_cast<float*>(smraw + Gm::buf_bytes());     // [2][RT][lds]
    const size_t NN = (size_t)N * N;
    const int kx0 = blockIdx.x * RT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / G, n2 = lane % G;
    const int slot = warp * Gm::LPW + grp;
    cplx<float>* buf = bufs + (size_t)slot * Gm::BUF;
    const float inv0 = 1.0f / (M * sqrtf(1.0f / N)), inv = 1.0f / (M * sqrtf(2.0f / N));
    const float aS = (float)dsc->alpha[0], aH = (float)dsc->alpha[1], aQ = (float)dsc->alpha[2];
    const float aK = (float)dsc->alpha[3], aL = (float)dsc->alpha[4];
    const int nlines = 2 * RT;
    for (int l0 = 0; l0 < nlines; l0 += Gm::SLOTS) {
        const int l = l0 + slot;
        const bool act = l < nlines;
        const int r = (act ? l : 0) >> 1, fld = (act ? l : 0) & 1;
        const int kx = kx0 + r;
        const float evx = evf[kx];
        for (int k = n2; k <= M / 2; k += G) {
            const int kys[4] = {k, N - k, M - k, M + k};
            float vals[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u == 1 && k == 0) { vals[u] = 0.f; continue; }
                const int ky = kys[u];
                const float s = evx + evf[ky];
                const size_t o = (size_t)kx * N + ky;
                if (fld == 0) {
                    const float isig = 1.0f / (sc.C1 + s * (sc.C2 + sc.C3 * s));
                    vals[u] = (spec[o] - aS * spec[NN + o] - aH * spec[2 * NN + o]
                               - aQ * spec[3 * NN + o] - aK * spec[4 * NN + o]) * isig;
                } else {
                    const float itau = 1.0f / (sc.Ct + sc.lam * s);
                    vals[u] = (spec[6 * NN + o] + aL * spec[7 * NN + o]) * itau;
                    if (anchor_mass && kx == 0 && ky == 0) vals[u] = 0.f;
                }
            }
            cplx<float> zk, zMk;
            pre_inverse(Quad<float>{vals[0], vals[1], vals[2], vals[3]}, k, twP[k], inv0, inv, zk, zMk);
            buf[k] = zk;
            if (k > 0) buf[M - k] = zMk;
        }
        __syncwarp();
        cplx<float> v[E];
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) v[n1] = buf[G * n1 + n2];
        __syncwarp();
        wf::fourstep<float, M, true>(v, buf, tw2, n2);
        float dhi = 0.f, dlo = 0.f;
        if (act) {
            float* srow = stage + (size_t)(fld * RT + r) * lds;
            for (int m = n2; m < M / 2; m += G) {
                const cplx<float> a = buf[m], b = buf[M - 1 - m];
                *reinterpret_cast<float4*>(srow + 4 * m) = make_float4(a.x, b.y, a.y, b.x);
                df_add(dhi, dlo, a.x); df_add(dhi, dlo, b.y); df_add(dhi, dlo, a.y); df_add(dhi, dlo, b.x);
            }
        }
        // FP32 path: the zero-mean psi increment's kx = 0 column should sum to 0
        // over y; record what the FP32 transform left (removed in kw_irow)
        const double dsum = group_sum_exact<G>(dhi, dlo);
        if (anchor_mass && act && fld == 1 && kx == 0 && n2 == 0) dsc->dc_col = dsum;
        __syncwarp();
    }
    __syncthreads();
    const int R4 = RT / 4;
    for (int q = threadIdx.x; q < 2 * R4 * N; q += blockDim.x) {
        const int r4 = q % R4, rest = q / R4;
        const int y = rest % N, fld = rest / N;
        const float* s = stage + (size_t)(fld * RT + 4 * r4) * lds + y;
        *reinterpret_cast<float4*>(out + fld * NN + (size_t)y * N + kx0 + 4 * r4) =
            make_float4(s[0], s[lds], s[2 * lds], s[3 * lds]);
    }
}

// ------------------------------------------------------------------ kw_irow
// RI rows per CTA, two lines (phi, psi) per row.
template <int M>
__global__ void __launch_bounds__(kWarps * 32)
kw_irow(const float* __restrict__ in, float* __restrict__ phi_new, float* __restrict__ psi_new, int RI,
        const cplx<float>* __restrict__ tw2, const PostTw<float>* __restrict__ twP,
        const float* __restrict__ phn, const float* __restrict__ pho,
        const float* __restrict__ psn, const float* __restrict__ pso, int bdf1,
        const DevScalars* __restrict__ dsc, int anchor_mass, uint32_t step) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    const int y0 = blockIdx.x * RI;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / G, n2 = lane % G;
    const int slot = warp * Gm::LPW + grp;
    cplx<float>* buf = bufs + (size_t)slot * Gm::BUF;
    const float inv0 = 1.0f / (M * sqrtf(1.0f / N)), inv = 1.0f / (M * sqrtf(2.0f / N));
    const double anc_d = anchor_mass ? dsc->anchor - sqrt((double)N) * dsc->dc_col / ((double)N * N) : 0.0;
    const int nlines = 2 * RI;
    for (int l0 = 0; l0 < nlines; l0 += Gm::SLOTS) {
        const int l = l0 + slot;
        const bool act = l < nlines;
        const int r = (act ? l : 0) >> 1, fld = (act ? l : 0) & 1;
        const float* row = in + fld * NN + (size_t)(y0 + r) * N;
        const float x0 = row[0];                  // the line's DC coefficient
        for (int k = n2; k <= M / 2; k += G) {
            const Quad<float> X{row[k], k > 0 ? row[N - k] : 0.f, row[M - k], row[M + k]};
            cplx<float> zk, zMk;
            pre_inverse(X, k, twP[k], inv0, inv, zk, zMk);
            buf[k] = zk;
            if (k > 0) buf[M - k] = zMk;
        }
        __syncwarp();
        cplx<float> v[E];
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) v[n1] = buf[G * n1 + n2];
        __syncwarp();
        wf::fourstep<float, M, true>(v, buf, tw2, n2);
        // FP32 path, psi: the row's increments should sum to sqrt(N) x0; the
        // residual of the FP32 transform is removed (with the anchor) in the
        // compensated final rounding, so the stored mass stays conserved
        float rhi = 0.f, rlo = 0.f;
        if (anchor_mass && fld == 1)
            for (int m = n2; m < M / 2; m += G) {
                const cplx<float> a = buf[m], b = buf[M - 1 - m];
                df_add(rhi, rlo, a.x); df_add(rhi, rlo, b.y); df_add(rhi, rlo, a.y); df_add(rhi, rlo, b.x);
            }
        const double rsum = group_sum_exact<G>(rhi, rlo);
        if (act) {
            const size_t roff = (size_t)(y0 + r) * N;
            float* dst = (fld == 0 ? phi_new : psi_new) + roff;
            const float4* un = reinterpret_cast<const float4*>((fld == 0 ? phn : psn) + roff);
            const float4* uo = reinterpret_cast<const float4*>((fld == 0 ? pho : pso) + roff);
            const float an = (fld == 1 && anchor_mass)
                                 ? (float)(anc_d + (sqrt((double)N) * (double)x0 - rsum) / (double)N) : 0.f;
            const bool b1 = bdf1 != 0;
            const bool dth = (fld == 1) && anchor_mass;
            for (int m = n2; m < M / 2; m += G) {
                const cplx<float> a = buf[m], b = buf[M - 1 - m];
                const float4 p = __ldg(un + m), q = __ldg(uo + m);
                const uint32_t i0 = (uint32_t)(roff + 4 * m);
                float4 o;
                o.x = bar_add(p.x, q.x, a.x, an, b1, dth ? dither_key(step, i0) | 1u : 0u);
                o.y = bar_add(p.y, q.y, b.y, an, b1, dth ? dither_key(step, i0 + 1) | 1u : 0u);
                o.z = bar_add(p.z, q.z, a.y, an, b1, dth ? dither_key(step, i0 + 2) | 1u : 0u);
                o.w = bar_add(p.w, q.w, b.x, an, b1, dth ? dither_key(step, i0 + 3) | 1u : 0u);
                *reinterpret_cast<float4*>(dst + 4 * m) = o;
            }
        }
        __syncwarp();
    }
}

}  // namespace ccm
