// warp_kernels.cuh -- FP32 step kernels built on the warp-level line FFT
// (N = 2M in 128 .. 8192).  Same data flow as the block-FFT kernels of
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

constexpr int kWarps = 8;

// Exact (double-float) sum over the G lanes of one line: inside the warp for
// G <= 32; for G = 32 W each of the W warps sums its part, the parts go
// through `sm` (W float2 per line slot) and every warp adds them in the same
// order.
template <int G>
__device__ __forceinline__ double line_sum_exact(float hi, float lo, int slot, float2* sm) {
    if constexpr (G <= 32) {
        return group_sum_exact<G>(hi, lo);
    } else {
        constexpr int W = G / 32;
        const float2 h = group_sum_df<32>(hi, lo);
        const int part = (threadIdx.x >> 5) % W;
        if ((threadIdx.x & 31) == 0) sm[W * slot + part] = h;
        wf::line_sync<G>(slot);
        float2 a = sm[W * slot];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            const float2 b = sm[W * slot + w];
            df_add2(a.x, a.y, b.x, b.y);
        }
        wf::line_sync<G>(slot);        // the slots may be written again by a later call
        return (double)a.x + (double)a.y;
    }
}



// Pair-ordered spectra of the warp path: for each spectral row kx and each
// of the 7 stored fields (f0', S, H, Q, K, g0', L_P), the float4 of modes
// (k, N-k, M-k, M+k) for each pair k = 0 .. M/2, i.e. a row of
// RS = 4 (M/2 + 1) = N + 4 floats (16-byte aligned).  The layout is kx-major:
// the 7 field rows of one kx are contiguous (stride KS = 7 RS), so the
// recovery kernel reads each CTA's rows as one contiguous block and the
// column kernel writes each kx as one.
template <int M> struct SpecRow {
    static constexpr int RS = 4 * (M / 2 + 1);
    static constexpr size_t FO = (size_t)RS;          // next field, same kx
    static constexpr size_t KS = (size_t)7 * RS;      // next kx
};

template <int M, int S = 0, int WARPS = kWarps> struct WGeo {
    static constexpr int E = wf::Shape<M, S>::E, G = wf::Shape<M, S>::G;
    static constexpr int WPL = G > 32 ? G / 32 : 1;     // warps per line
    static constexpr int LPW = G > 32 ? 1 : 32 / G;     // lines per warp (one line spans WPL warps)
    static constexpr int SLOTS = WARPS * LPW / WPL;     // line buffers per CTA
    // complex per buffer: unpadded, XOR-swizzled transpose (M + 2), so that
    // three 8-line CTAs of the forward kernels fit the 196 KB shared-memory
    // configuration; padded rows (G + 1 values) for the recovery kernel (two
    // CTAs per SM, measured faster than three)
    static constexpr int BUF = wf::buf_len<M, true, S>();
    static constexpr int BUFP = wf::buf_len<M, false, S>();
    static constexpr size_t buf_bytes() { return (size_t)SLOTS * BUF * sizeof(cplx<float>); }
    static constexpr size_t bufp_bytes() { return (size_t)SLOTS * BUFP * sizeof(cplx<float>); }
};

// ------------------------------------------------------------------ kw_rowdct_T
// SLOTS rows of field blockIdx.y per CTA (one line per lane group).  Each
// line's natural-order half-length spectrum stays in its buffer; the DCT
// post-process reads it from there pair by pair while writing the transposed
// output, so the buffers double as the staging area of that write.
template <int M, bool GRP = false>
__global__ void __launch_bounds__(kWarps * 32, M <= 1024 ? 3 : 1)
kw_rowdct_T(const float* __restrict__ in, float* __restrict__ out,
            const cplx<float>* __restrict__ tw2, wf::PairTwTab twF, int ahead,
            const __grid_constant__ GroupArgs<GRP> ga, int bps) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, E = Gm::E, RT = Gm::SLOTS;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    int bx = blockIdx.x;
    if constexpr (GRP) {          // grouped launch (no prefetch ahead)
        const int sim = blockIdx.x / bps;
        bx = blockIdx.x - sim * bps;
        const BatchArgs& A = ga.a[sim];
        in = A.bufA; out = A.bufB; tw2 = A.tw2; twF = A.twF; ahead = 0;
    }
    const int f = blockIdx.y, y0 = bx * RT;
    {   // rows of the CTA one residency ahead
        const int t = blockIdx.y * gridDim.x + blockIdx.x + ahead;
        if (ahead > 0 && t < (int)(gridDim.x * gridDim.y) && threadIdx.x < RT)
            prefetch_l2(in + (t / gridDim.x) * NN + (size_t)((t % gridDim.x) * RT + threadIdx.x) * N, N * sizeof(float));
    }
    int n2, slot;
    wf::lane_geo<M>(n2, slot);
    cplx<float>* buf = bufs + (size_t)slot * Gm::BUF;
    {
        cplx<float> v[E];
        wf::pack_fwd_global<M>(in + CCM_IXW(f * NN + (size_t)(y0 + slot) * N, N, NF * NN), v, n2);
        wf::fourstep<float, M, false, true>(v, buf, tw2, n2, slot);
    }
    __syncthreads();
    // DCT post-process fused into the transposed write.  Item (r4, k) takes
    // the pair k (slots k and M-k of the natural-order spectra) of the rows
    // 4 r4 .. 4 r4 + 3 and writes its four modes k, N-k, M-k, M+k, each as one
    // float4 of the four rows; the item k = 0 also takes the pair M/2, so
    // that every item loads eight slots and stores four float4 (pair 0 gives
    // the modes 0 and M, pair M/2 the modes M/2 and 3M/2).  Consecutive
    // threads take the two halves of one 32-byte row segment when R4 = 2.
    const float2* stage = reinterpret_cast<const float2*>(bufs);
    constexpr int BC = Gm::BUF;                      // float2 per line buffer
    float* dst = out + f * NN + y0;
    constexpr int R4 = RT / 4;
    static_assert(RT % 4 == 0, "rows of a CTA in groups of four");
    auto put = [&](int mode, int r4, float a, float b, float c, float d) {
        if (CCM_OKW(f * NN + y0 + (size_t)mode * N + 4 * r4, 4, NF * NN))
            *reinterpret_cast<float4*>(dst + (size_t)mode * N + 4 * r4) = make_float4(a, b, c, d);
    };
    for (int q = threadIdx.x; q < R4 * (M / 2); q += blockDim.x) {
        const int r4 = q % R4, k = q / R4;
        const float2* sp = stage + (size_t)(4 * r4) * BC;
        const int ka = k == 0 ? M / 2 : M - k;       // second slot: M - k, or the pair M/2
        cplx<float> A[4], B[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float2 a = sp[(size_t)r * BC + k], b = sp[(size_t)r * BC + ka];
            A[r] = mk(a.x, a.y);
            B[r] = mk(b.x, b.y);
        }
        if (k == 0) {
            const wf::PairTw t0 = wf::load_pair_tw<false>(twF, 0), th = wf::load_pair_tw<false>(twF, M / 2);
            Quad<float> X[4], Y[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                X[r] = wf::post_pair_lean(A[r], A[r], t0);
                Y[r] = wf::post_pair_lean(B[r], B[r], th);
            }
            put(0, r4, X[0].xk, X[1].xk, X[2].xk, X[3].xk);
            put(M, r4, X[0].xMk, X[1].xMk, X[2].xMk, X[3].xMk);
            put(M / 2, r4, Y[0].xk, Y[1].xk, Y[2].xk, Y[3].xk);
            put(N - M / 2, r4, Y[0].xNk, Y[1].xNk, Y[2].xNk, Y[3].xNk);
        } else {
            const wf::PairTw t = wf::load_pair_tw<false>(twF, k);
            Quad<float> X[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) X[r] = wf::post_pair_lean(A[r], B[r], t);
            put(k, r4, X[0].xk, X[1].xk, X[2].xk, X[3].xk);
            put(N - k, r4, X[0].xNk, X[1].xNk, X[2].xNk, X[3].xNk);
            put(M - k, r4, X[0].xMk, X[1].xMk, X[2].xMk, X[3].xMk);
            put(M + k, r4, X[0].xMpk, X[1].xMpk, X[2].xMpk, X[3].xMpk);
        }
    }
}

// ------------------------------------------------------------------ kw_coldct_gram
template <int M, bool GRP = false>
__global__ void __launch_bounds__(kWarps * 32, M <= 1024 ? 3 : 1)
kw_coldct_gram(const float* __restrict__ in, float* __restrict__ spec, double* __restrict__ part,
               const cplx<float>* __restrict__ tw2, wf::PairTwTab twF,
               const float* __restrict__ evf, const float4* __restrict__ evp, SpecCoefF sc,
               const __grid_constant__ GroupArgs<GRP> ga, int bps) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E, KC = Gm::SLOTS / NF;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    int bx = blockIdx.x;
    if constexpr (GRP) {          // grouped launch
        const int sim = blockIdx.x / bps;
        bx = blockIdx.x - sim * bps;
        const BatchArgs& A = ga.a[sim];
        in = A.bufB; spec = A.bufA; part = A.part2; tw2 = A.tw2; twF = A.twF; evf = A.evf; evp = A.evp; sc = A.sf;
    }
    const int kx0 = bx * KC;
    static_assert(G <= 32, "lines of one warp at most; longer lines take kw_coldct_gram_split");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int n2, slot;                                        // line = (kc, field)
    wf::lane_geo<M>(n2, slot);
    const int kc = slot / NF, f = slot % NF;
    {
        cplx<float> v[E];
        wf::pack_fwd_global<M>(in + CCM_IXW(f * NN + (size_t)(kx0 + kc) * N, N, NF * NN), v, n2);
        wf::fourstep<float, M, false, true>(v, bufs + (size_t)slot * Gm::BUF, tw2, n2, slot);
    }
    __syncthreads();
    float acc[NRED2];
#pragma unroll
    for (int i = 0; i < NRED2; ++i) acc[i] = 0.f;
    static_assert(KC * NF <= 32, "one lane per (column, field) of the pair M/2");
    if (warp == kWarps - 1) {
        // pair M/2 (modes M/2 and 3M/2 only) of every column by the last warp,
        // one lane per (column, field), so that the loop below gives every
        // thread the same number of pairs; lane 8c adds the column's Gram terms
        const int c = lane >> 3, g = lane & 7;
        float xm = 0.f, x3 = 0.f;
        if (c < KC) {
            const cplx<float>* b = bufs + (size_t)(c * NF + g) * Gm::BUF;
            const Quad<float> X = wf::post_pair_lean(b[M / 2], b[M / 2], wf::load_pair_tw<false>(twF, M / 2));
            xm = X.xk;
            x3 = X.xNk;
            if (g != 5)
                *reinterpret_cast<float4*>(spec + (size_t)(kx0 + c) * SpecRow<M>::KS + (size_t)(g < 5 ? g : g - 1) * SpecRow<M>::FO +
                                           4 * (M / 2)) = make_float4(xm, x3, xm, x3);
        }
#pragma unroll 1
        for (int mode = 0; mode < 2; ++mode) {       // M/2, then 3M/2
            float v[NF];
#pragma unroll
            for (int u = 0; u < NF; ++u) v[u] = __shfl_sync(0xffffffffu, mode ? x3 : xm, (lane & ~7) + u);
            if (g == 0 && c < KC) {
                const float4 eh = evp[M / 2];
                const float sm = evf[kx0 + c] + (mode ? eh.y : eh.x);
                gram_accumulate(acc, v, __frcp_rn(sc.C1 + sm * (sc.C2 + sc.C3 * sm)), __frcp_rn(sc.Ct + sc.lam * sm));
            }
        }
    }
    for (int q = threadIdx.x; q < KC * (M / 2); q += blockDim.x) {
        const int c = q / (M / 2), k = q % (M / 2);
        const int kx = kx0 + c;
        Quad<float> X[NF];
        const wf::PairTw tw = wf::load_pair_tw<false>(twF, k);
#pragma unroll
        for (int g = 0; g < NF; ++g) {
            const cplx<float>* b = bufs + (size_t)(c * NF + g) * Gm::BUF;
            X[g] = wf::post_pair_lean(b[k], b[(M - k) & (M - 1)], tw);
        }
        const float evx = evf[kx];
        const float4 e4 = evp[k];
        const float ev_u[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!pair_mode_valid(u, k, M)) continue;
            const float s = evx + ev_u[u];
            // correctly rounded reciprocals (the same values as 1.0f / x)
            const float isig = __frcp_rn(sc.C1 + s * (sc.C2 + sc.C3 * s));
            const float itau = __frcp_rn(sc.Ct + sc.lam * s);
            float v[NF];
#pragma unroll
            for (int g = 0; g < NF; ++g)
                v[g] = (u == 0) ? X[g].xk : (u == 1) ? X[g].xNk : (u == 2) ? X[g].xMk : X[g].xMpk;
            gram_accumulate(acc, v, isig, itau);
        }
        // spectra in pair order: slot u of pair k holds mode k, N-k, M-k, M+k
        // (k = 0: no mode N, slot 3 repeats mode M; k = M/2, above: slots 2, 3
        // repeat modes M/2, 3M/2), one float4 per field
        float* dst = spec + (size_t)kx * SpecRow<M>::KS + 4 * k;
#pragma unroll
        for (int g = 0; g < NF; ++g) {
            if (g == 5) continue;
            if (!CCM_OKW((size_t)kx * SpecRow<M>::KS + 4 * k + (size_t)(g < 5 ? g : g - 1) * SpecRow<M>::FO, 4,
                         (size_t)N * SpecRow<M>::KS)) continue;
            float4 o = make_float4(X[g].xk, k == 0 ? 0.f : X[g].xNk, X[g].xMk, X[g].xMpk);
            if (k == 0) o.w = o.z;
            *reinterpret_cast<float4*>(dst + (size_t)(g < 5 ? g : g - 1) * SpecRow<M>::FO) = o;
        }
    }
    __syncthreads();       // the line buffers are free: their start holds the block reduction
    block_sum_store_part<NRED2, float>(acc, reinterpret_cast<float2*>(part) + (size_t)bx * NRED2,
                                       reinterpret_cast<double*>(smraw));
}

// ------------------------------------------------------------------ kw_coldct_gram_split
// The column pass for lines too long to keep all eight fields of a column on
// chip (M = 4096: 32 KB per line).  The Gram sums have no terms across the
// two groups {f0', S, H, Q, K} (the 15 chi entries) and {P, g0', LP} (the
// two zeta entries), so one CTA per (column kx, group): blockIdx.y = 0 takes
// the five fields (ten warps, two per line), blockIdx.y = 1 the three (six
// warps; its other four warps only join the block barriers).  Each writes its
// own columns of the column's partial row and its fields' spectra (P is not
// stored).
constexpr int kSplitWarps = 10;

template <int M>
__global__ void __launch_bounds__(kSplitWarps * 32, 1)
kw_coldct_gram_split(const float* __restrict__ in, float* __restrict__ spec, double* __restrict__ part,
                     const cplx<float>* __restrict__ tw2, wf::PairTwTab twF,
                     const float* __restrict__ evf, const float4* __restrict__ evp, SpecCoefF sc) {
    using Gm = WGeo<M>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E;
    static_assert(G == 64, "two warps per line");
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    const int kx = blockIdx.x, grp = blockIdx.y;
    const int nf = grp == 0 ? 5 : 3, f0 = grp == 0 ? 0 : 5;
    int n2, slot;
    wf::lane_geo<M>(n2, slot);                           // slot 0 .. 4
    if (slot < nf) {                                     // both warps of a line take the same branch
        cplx<float> v[E];
        wf::pack_fwd_global<M>(in + CCM_IXW((f0 + slot) * NN + (size_t)kx * N, N, NF * NN), v, n2);
        wf::fourstep<float, M, false, true>(v, bufs + (size_t)slot * Gm::BUF, tw2, n2, slot);
    }
    __syncthreads();
    float acc[NRED2];
#pragma unroll
    for (int i = 0; i < NRED2; ++i) acc[i] = 0.f;
    const float evx = evf[kx];
    for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) {
        const wf::PairTw tw = wf::load_pair_tw<false>(twF, k);
        Quad<float> X[5];
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            if (g >= nf) continue;
            const cplx<float>* b = bufs + (size_t)g * Gm::BUF;
            X[g] = wf::post_pair_lean(b[k], b[(M - k) & (M - 1)], tw);
        }
        const float4 e4 = evp[k];
        const float ev_u[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!pair_mode_valid(u, k, M)) continue;
            const float s = evx + ev_u[u];
            const float isig = __frcp_rn(sc.C1 + s * (sc.C2 + sc.C3 * s));
            const float itau = __frcp_rn(sc.Ct + sc.lam * s);
            float v[NF];
#pragma unroll
            for (int g = 0; g < NF; ++g) v[g] = 0.f;
#pragma unroll
            for (int g = 0; g < 5; ++g) {
                if (g >= nf) continue;
                const float x = (u == 0) ? X[g].xk : (u == 1) ? X[g].xNk : (u == 2) ? X[g].xMk : X[g].xMpk;
                v[f0 + g] = x;
            }
            gram_accumulate(acc, v, isig, itau);
        }
        // spectra in pair order (the layout of kw_coldct_gram)
        float* dst = spec + (size_t)kx * SpecRow<M>::KS + 4 * k;
#pragma unroll
        for (int g = 0; g < 5; ++g) {
            if (g >= nf) continue;
            const int f = f0 + g;
            if (f == 5) continue;
            const size_t o = (size_t)kx * SpecRow<M>::KS + 4 * k + (size_t)(f < 5 ? f : f - 1) * SpecRow<M>::FO;
            if (!CCM_OKW(o, 4, (size_t)N * SpecRow<M>::KS)) continue;
            float4 w = make_float4(X[g].xk, k == 0 ? 0.f : X[g].xNk, X[g].xMk, X[g].xMpk);
            if (k == 0) w.w = w.z;
            *reinterpret_cast<float4*>(dst + (size_t)(f < 5 ? f : f - 1) * SpecRow<M>::FO) = w;
        }
    }
    __syncthreads();       // the line buffers are free: their start holds the block reduction
    // block sums of this group's Gram columns (float pairs, as block_sum_store_part)
    float* smf = reinterpret_cast<float*>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NRED2; ++i) {
        const float sw = warp_sum(acc[i]);
        if (lane == 0) smf[warp * NRED2 + i] = sw;
    }
    __syncthreads();
    const int c0 = grp == 0 ? 0 : 15, c1 = grp == 0 ? 15 : NRED2;
    if (threadIdx.x >= c0 && threadIdx.x < c1) {
        float hi = 0.f, lo = 0.f;
        for (int w = 0; w < kSplitWarps; ++w) df_add(hi, lo, smf[w * NRED2 + threadIdx.x]);
        reinterpret_cast<float2*>(part)[(size_t)kx * NRED2 + threadIdx.x] = make_float2(hi, lo);
    }
}

// ------------------------------------------------------------------ kw_comb_icolT
// RT = SLOTS/2 spectral rows per CTA, two lines (d_phi^, d_psi^) per row.
// Phase 1 (all threads): gather the spectra, combine, divide, pre-process
// into the line buffers.  Phase 2 (per line): inverse four-step FFT and
// unpack in place.  Phase 3: transposed write from the buffers.
// Line shapes of the inverse transforms (variant 1: 32 values per lane):
// 2048- and 4096-point lines over two and four warps in both inverse
// kernels; the other lines are shaped as in the forward transforms.  The
// recovery kernel runs sixteen warps per CTA at 4096 points, so that a CTA
// still holds two spectral rows (8-byte transposed stores).
template <int M> __host__ __device__ constexpr int comb_shape() { return M == 2048 || M == 4096 ? 1 : 0; }
template <int M> __host__ __device__ constexpr int irow_shape() { return M == 2048 || M == 4096 ? 1 : 0; }
template <int M> __host__ __device__ constexpr int comb_warps() { return M == 4096 ? 16 : kWarps; }

template <int M, bool GRP = false>
__global__ void __launch_bounds__(comb_warps<M>() * 32)
kw_comb_icolT(const float* __restrict__ spec, float* __restrict__ out,
              const cplx<float>* __restrict__ tw2, wf::PairTwTab twI,
              const float* __restrict__ evf, const float4* __restrict__ evp, SpecCoefF sc,
              DevScalars* __restrict__ dsc, int anchor_mass,
              const __grid_constant__ GroupArgs<GRP> ga, int bps) {
    constexpr int SV = comb_shape<M>();
    using Gm = WGeo<M, SV, comb_warps<M>()>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E, RT = Gm::SLOTS / 2, NU = (M / 2 + G - 1) / G;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    int bx = blockIdx.x;
    if constexpr (GRP) {          // grouped launch
        const int sim = blockIdx.x / bps;
        bx = blockIdx.x - sim * bps;
        const BatchArgs& A = ga.a[sim];
        spec = A.bufA; out = A.bufB; tw2 = A.tw2; twI = A.twI; evf = A.evf; evp = A.evp; sc = A.sf; dsc = A.sc;
    }
    const int kx0 = bx * RT;
    const float aS = (float)dsc->alpha[0], aH = (float)dsc->alpha[1], aQ = (float)dsc->alpha[2];
    const float aK = (float)dsc->alpha[3], aL = (float)dsc->alpha[4];
    constexpr int PAIRS = M / 2 + 1;
    // one item = one spectral row and one pair index k: the four modes
    // k, N-k, M-k, M+k of both lines (d_phi^ from five spectra, d_psi^ from
    // two), one float4 per spectrum in the pair-ordered layout
#pragma unroll 4
    for (int q = threadIdx.x; q < RT * PAIRS; q += blockDim.x) {
        const int r = q / PAIRS, k = q % PAIRS;
        const int kx = kx0 + r;
        const float evx = evf[kx];
        const float4 e4 = evp[k];
        const float* src = spec + CCM_IXW((size_t)kx * SpecRow<M>::KS + 4 * k, 6 * SpecRow<M>::FO + 4,
                                          (size_t)N * SpecRow<M>::KS);
        constexpr size_t FS = SpecRow<M>::FO;
        const float4 f0 = __ldg(reinterpret_cast<const float4*>(src));
        const float4 f1 = __ldg(reinterpret_cast<const float4*>(src + FS));
        const float4 f2 = __ldg(reinterpret_cast<const float4*>(src + 2 * FS));
        const float4 f3 = __ldg(reinterpret_cast<const float4*>(src + 3 * FS));
        const float4 f4 = __ldg(reinterpret_cast<const float4*>(src + 4 * FS));
        const float4 f6 = __ldg(reinterpret_cast<const float4*>(src + 5 * FS));
        const float4 f7 = __ldg(reinterpret_cast<const float4*>(src + 6 * FS));
        auto comb = [&](float a0, float a1, float a2, float a3, float a4, float a6, float a7, float ev,
                        float& vp, float& vq) {
            const float s = evx + ev;
            vp = (a0 - aS * a1 - aH * a2 - aQ * a3 - aK * a4) * __frcp_rn(sc.C1 + s * (sc.C2 + sc.C3 * s));
            vq = (a6 + aL * a7) * __frcp_rn(sc.Ct + sc.lam * s);
        };
        float vp[4], vq[4];
        comb(f0.x, f1.x, f2.x, f3.x, f4.x, f6.x, f7.x, e4.x, vp[0], vq[0]);
        comb(f0.y, f1.y, f2.y, f3.y, f4.y, f6.y, f7.y, e4.y, vp[1], vq[1]);
        comb(f0.z, f1.z, f2.z, f3.z, f4.z, f6.z, f7.z, e4.z, vp[2], vq[2]);
        comb(f0.w, f1.w, f2.w, f3.w, f4.w, f6.w, f7.w, e4.w, vp[3], vq[3]);
        // d_psi has zero mean (mass conservation); the FP32 path sets the
        // zero mode exactly and keeps the stored mean with the anchor
        if (anchor_mass && kx == 0 && k == 0) vq[0] = 0.f;
        const wf::PairTw tw = wf::load_pair_tw<true>(twI, k);
        cplx<float> zk, zMk;
        cplx<float>* b = bufs + (size_t)(2 * r) * Gm::BUFP;
        wf::pre_pair_lean(Quad<float>{vp[0], vp[1], vp[2], vp[3]}, tw, zk, zMk);
        b[k] = zk;
        if (k > 0) b[M - k] = zMk;
        b += Gm::BUFP;
        wf::pre_pair_lean(Quad<float>{vq[0], vq[1], vq[2], vq[3]}, tw, zk, zMk);
        b[k] = zk;
        if (k > 0) b[M - k] = zMk;
    }
    __syncthreads();
    __shared__ float2 lsum[4 * Gm::SLOTS];
    int n2, slot;                                        // line = slot: row slot/2, field slot%2
    wf::lane_geo<M, SV>(n2, slot);
    cplx<float>* buf = bufs + (size_t)slot * Gm::BUFP;
    {
        cplx<float> v[E];
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) v[n1] = buf[G * n1 + n2];
        wf::line_sync<G>(slot);
        wf::fourstep<float, M, true, false, SV>(v, buf, tw2, n2, slot);
    }
    float dhi = 0.f, dlo = 0.f;
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        const int m = n2 + G * i;
        const cplx<float> a = buf[m], b = buf[M - 1 - m];
        df_add(dhi, dlo, a.x); df_add(dhi, dlo, b.y); df_add(dhi, dlo, a.y); df_add(dhi, dlo, b.x);
    }
    // FP32 path: the zero-mean psi increment's kx = 0 column should sum to 0
    // over y; record what the FP32 transform left (removed in kw_irow)
    const double dsum = line_sum_exact<G>(dhi, dlo, slot, lsum);
    if (anchor_mass && (slot & 1) == 1 && kx0 + (slot >> 1) == 0 && n2 == 0) dsc->dc_col = dsum;
    __syncthreads();
    // transposed write straight from the line buffers: after the inverse
    // transform slot m holds the samples y = 4m, 4m+2 and slot M-1-m the
    // samples y = 4m+3, 4m+1 (the even/odd reordering undone in the indexing)
    const float2* stage = reinterpret_cast<const float2*>(bufs);
    constexpr int BC = Gm::BUFP;                     // float2 per line buffer
    if constexpr (RT < 4) {
        // two rows per CTA (4096-point lines): 8-byte stores of the row pair
        static_assert(RT == 2, "two or a multiple of four rows per CTA");
        for (int q = threadIdx.x; q < 2 * (M / 2); q += blockDim.x) {
            const int m = q % (M / 2), fld = q / (M / 2);
            const float2* sp = stage + (size_t)fld * BC;       // row 0: buffer fld, row 1: buffer 2 + fld
            const float2 a0 = sp[m], a1 = sp[2 * BC + m];
            const float2 b0 = sp[M - 1 - m], b1 = sp[2 * BC + M - 1 - m];
            if (!CCM_OKW(fld * NN + (size_t)(4 * m + 3) * N + kx0, 2, 2 * NN)) continue;
            float* d = out + fld * NN + (size_t)(4 * m) * N + kx0;
            *reinterpret_cast<float2*>(d) = make_float2(a0.x, a1.x);
            *reinterpret_cast<float2*>(d + N) = make_float2(b0.y, b1.y);
            *reinterpret_cast<float2*>(d + 2 * (size_t)N) = make_float2(a0.y, a1.y);
            *reinterpret_cast<float2*>(d + 3 * (size_t)N) = make_float2(b0.x, b1.x);
        }
        return;
    }
    constexpr int R4 = RT / 4;
    for (int q = threadIdx.x; q < 2 * R4 * (M / 2); q += blockDim.x) {
        const int m = q % (M / 2), rest = q / (M / 2);
        const int r4 = rest % R4, fld = rest / R4;
        // line of row 4 r4 + i and field fld is buffer 2 (4 r4 + i) + fld
        const float2* sp = stage + (size_t)(8 * r4 + fld) * BC;
        const float2 a0 = sp[m], a1 = sp[2 * BC + m], a2 = sp[4 * BC + m], a3 = sp[6 * BC + m];
        const float2 b0 = sp[M - 1 - m], b1 = sp[2 * BC + M - 1 - m], b2 = sp[4 * BC + M - 1 - m], b3 = sp[6 * BC + M - 1 - m];
        if (!CCM_OKW(fld * NN + (size_t)(4 * m + 3) * N + kx0 + 4 * r4, 4, 2 * NN)) continue;
        float* d = out + fld * NN + (size_t)(4 * m) * N + kx0 + 4 * r4;
        *reinterpret_cast<float4*>(d) = make_float4(a0.x, a1.x, a2.x, a3.x);
        *reinterpret_cast<float4*>(d + N) = make_float4(b0.y, b1.y, b2.y, b3.y);
        *reinterpret_cast<float4*>(d + 2 * (size_t)N) = make_float4(a0.y, a1.y, a2.y, a3.y);
        *reinterpret_cast<float4*>(d + 3 * (size_t)N) = make_float4(b0.x, b1.x, b2.x, b3.x);
    }
}

// ------------------------------------------------------------------ kw_irow
// InvGeo<M>::LINES lines per CTA, line = 2 y + field (phi, psi of row y), so
// that 3 CTAs per SM hold every line of an N = 2048 field at once (one round,
// no tail).  Phase 1 (all threads): pre-process the transposed rows into
// the line buffers; phase 2 (per line): inverse four-step FFT, then
// u^{n+1} = u_bar + du with the compensated (and, for psi on the FP32 path,
// error-feedback and mass-anchored) final rounding.
// Warps per CTA of the inverse row kernel: 9 at M = 1024 (3 CTAs of 9 lines
// per SM hold all 4096 lines of N = 2048: one round); 4 at M = 2048 (3 CTAs
// per SM); fewer at small M so that the grid still has >= 128 CTAs.
template <int M> __host__ __device__ constexpr int inv_warps() {
    return M == 1024 ? 9 : M >= 2048 ? 4 : M == 512 ? 4 : M == 256 ? 2 : 1;
}
template <int M> __host__ __device__ constexpr int inv_min_ctas() {
    return M == 2048 || M == 4096 ? 4 : M == 1024 ? 3 : 4;
}

template <int M> struct InvGeo {
    using W = WGeo<M, irow_shape<M>()>;
    static constexpr int WARPS = inv_warps<M>();
    static constexpr int LINES = WARPS * W::LPW / W::WPL;     // lines per CTA
    static constexpr int BUF = wf::buf_len<M, true, irow_shape<M>()>();   // swizzled or split-row transpose
    static constexpr size_t smem_bytes() { return (size_t)LINES * BUF * sizeof(cplx<float>); }
};

template <int M, bool GRP = false>
__global__ void __launch_bounds__(inv_warps<M>() * 32, inv_min_ctas<M>())
kw_irow(const float* __restrict__ in, float* __restrict__ phi_new, float* __restrict__ psi_new,
        const cplx<float>* __restrict__ tw2, wf::PairTwTab twI,
        const float* __restrict__ phn, const float* __restrict__ pho,
        const float* __restrict__ psn, const float* __restrict__ pso, int bdf1,
        const DevScalars* __restrict__ dsc, int anchor_mass,
        const __grid_constant__ GroupArgs<GRP> ga, int bps) {
    constexpr int SV = irow_shape<M>();
    using Gm = WGeo<M, SV>;
    constexpr int N = 2 * M, G = Gm::G, E = Gm::E, L = InvGeo<M>::LINES, NU = (M / 2 + G - 1) / G;
    int bx = blockIdx.x;
    if constexpr (GRP) {          // grouped launch
        const int sim = blockIdx.x / bps;
        bx = blockIdx.x - sim * bps;
        const BatchArgs& A = ga.a[sim];
        in = A.bufB; phi_new = A.phi_new; psi_new = A.psi_new; tw2 = A.tw2; twI = A.twI;
        phn = A.phn; pho = A.pho; psn = A.psn; pso = A.pso; dsc = A.sc;
    }
    const uint32_t step = (uint32_t)dsc->steps;         // dither key (graph replays read it here)
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<float>* bufs = reinterpret_cast<cplx<float>*>(smraw);
    const size_t NN = (size_t)N * N;
    const int l0 = bx * L;                               // first line of this CTA
    constexpr int PAIRS = M / 2 + 1;
    constexpr int UNR = M >= 2048 ? 8 : 4;    // loads in flight per thread in the pre-process
#pragma unroll UNR
    for (int q = threadIdx.x; q < L * PAIRS; q += blockDim.x) {
        const int l = q / PAIRS, k = q % PAIRS;
        const int gl = l0 + l;
        if (gl >= 2 * N) continue;
        const float* row = in + CCM_IXW((gl & 1) * NN + (size_t)(gl >> 1) * N, N, 2 * NN);
        const Quad<float> X{__ldg(row + k), k > 0 ? __ldg(row + N - k) : 0.f, __ldg(row + M - k), __ldg(row + M + k)};
        cplx<float> zk, zMk;
        wf::pre_pair_lean(X, wf::load_pair_tw<true>(twI, k), zk, zMk);
        cplx<float>* b = bufs + (size_t)l * InvGeo<M>::BUF;
        b[k] = zk;
        if (k > 0) b[M - k] = zMk;
    }
    __syncthreads();
    __shared__ float2 lsum[4 * L];
    int n2, slot;
    wf::lane_geo<M, SV>(n2, slot);
    const int gl = l0 + slot;
    const bool valid = gl < 2 * N;                       // the last CTA has fewer lines
    const int fld = gl & 1;
    cplx<float>* buf = bufs + (size_t)slot * InvGeo<M>::BUF;
    {
        cplx<float> v[E];
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) v[n1] = buf[G * n1 + n2];
        wf::line_sync<G>(slot);
        wf::fourstep<float, M, true, true, SV>(v, buf, tw2, n2, slot);
    }
    const size_t roff = valid ? (size_t)(gl >> 1) * N : 0;
    // FP32 path, psi: the row's increments should sum to sqrt(N) x0 (x0 the
    // row's DC coefficient); the residual of the FP32 transform and the
    // column residual dc_col are removed, with the mean anchor, in the final
    // rounding, so the stored mass stays conserved
    const bool psi_line = valid && fld == 1 && anchor_mass;
    float rhi = 0.f, rlo = 0.f;
    if (psi_line)
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            const int m = n2 + G * i;
            const cplx<float> a = buf[m], b = buf[M - 1 - m];
            df_add(rhi, rlo, a.x); df_add(rhi, rlo, b.y); df_add(rhi, rlo, a.y); df_add(rhi, rlo, b.x);
        }
    const double rsum = line_sum_exact<G>(rhi, rlo, slot, lsum);
    float an = 0.f;
    if (psi_line) {
        const double x0 = (double)__ldg(in + fld * NN + roff);
        const double sN = sqrt((double)N);
        an = (float)(dsc->anchor - sN * dsc->dc_col / ((double)N * N) + (sN * x0 - rsum) / (double)N);
    }
    float* dst = (fld == 0 ? phi_new : psi_new) + roff;
    const float4* un = reinterpret_cast<const float4*>((fld == 0 ? phn : psn) + roff);
    const float4* uo = reinterpret_cast<const float4*>((fld == 0 ? pho : pso) + roff);
    const bool b1 = bdf1 != 0;
    // psi on the FP32 path: rounding with error feedback along each lane's
    // values, then the lanes' remaining errors (summed exactly over the row)
    // are folded into the row's first value with one dithered rounding, so
    // the stored row sums to its exact value within about one ulp.  Every
    // lane takes part in the group sum (the carry stays 0 on other lines).
    float carry = 0.f;
    float first = 0.f;
#pragma unroll
    for (int i = 0; i < NU; ++i) {
        const int m = n2 + G * i;
        const cplx<float> a = buf[m], b = buf[M - 1 - m];
        if (!valid) continue;
        if (!CCM_OKW(roff + 4 * m, 4, NN)) continue;
        const float4 p = __ldg(un + m), q = __ldg(uo + m);
        float4 o;
        if (psi_line) {
            o.x = bar_add_fb(p.x, q.x, a.x, an, b1, carry);
            o.y = bar_add_fb(p.y, q.y, b.y, an, b1, carry);
            o.z = bar_add_fb(p.z, q.z, a.y, an, b1, carry);
            o.w = bar_add_fb(p.w, q.w, b.x, an, b1, carry);
        } else {
            o.x = bar_add(p.x, q.x, a.x, 0.f, b1);
            o.y = bar_add(p.y, q.y, b.y, 0.f, b1);
            o.z = bar_add(p.z, q.z, a.y, 0.f, b1);
            o.w = bar_add(p.w, q.w, b.x, 0.f, b1);
        }
        if (i == 0) first = o.x;
        *reinterpret_cast<float4*>(dst + 4 * m) = o;
    }
    const double rest = line_sum_exact<G>(carry, 0.f, slot, lsum);
    if (psi_line && n2 == 0) dst[0] = dither_round(first, (float)rest, dither_key(step, (uint32_t)roff) | 1u);
}

}  // namespace ccm
