// dct_device.cuh -- CTA-level real DCT-II / DCT-III of whole grid lines.
//
// The elliptic solves of the CC-MSAV step (Appendix C of the paper: forward
// 2D DCT, divide by the closed-form Neumann eigenvalues, inverse DCT) apply
// a length-N orthonormal DCT along every line of an N x N field.  Each line
// transform follows Makhoul's construction:
//   forward  x -> even/odd reordered v -> length-N/2 complex FFT of
//            z[m] = v[2m] + i v[2m+1] -> split into the length-N spectrum of v
//            -> post-twiddle by exp(-i pi k / 2N) -> X[k], X[N-k] together;
//   inverse  the same steps backwards.
// The complex FFT is a radix-8/4/2 Stockham transform kept in shared memory,
// with each thread holding E = min(8, M) values of its line in registers per
// stage (load all, barrier, butterflies, store, barrier).
//
// Layout of a line buffer in shared memory: M = N/2 complex values at padded
// positions pad(i) = i + i/8 (one spare slot per 8 values breaks the
// power-of-two strides of the early Stockham stages across banks).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccm {

template <typename T> struct cplx { T x, y; };

template <typename T> __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> c; c.x = a; c.y = b; return c; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {   // a * conj(b)
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ cplx<T> conj_(cplx<T> a) { return mk(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cplx<T> scale(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) {
    return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

__device__ __forceinline__ int padc(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int padded_len(int M) { return M + (M >> 3) + 1; }

// ---------------------------------------------------------------- radix kernels
// In-register DFTs of size 2, 4, 8 (exact constants; INV selects exp(+i...)).

template <typename T, bool INV> __device__ __forceinline__ void dft2(cplx<T>& a, cplx<T>& b) {
    cplx<T> t = a; a = t + b; b = t - b;
}

template <typename T, bool INV> __device__ __forceinline__ void dft4(cplx<T>* v) {
    // X0 = (v0+v2) + (v1+v3); X2 = (v0+v2) - (v1+v3); X1 = (v0-v2) -/+ i(v1-v3); X3 = (v0-v2) +/- i(v1-v3)
    cplx<T> s02 = v[0] + v[2], d02 = v[0] - v[2], s13 = v[1] + v[3], d13 = v[1] - v[3];
    cplx<T> r = mul_mi<T, INV>(d13);
    v[0] = s02 + s13; v[2] = s02 - s13; v[1] = d02 + r; v[3] = d02 - r;
}

template <typename T, bool INV> __device__ __forceinline__ void dft8(cplx<T>* v) {
    const T h = (T)0.70710678118654752440;   // cos(pi/4)
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<T, INV>(e);
    dft4<T, INV>(o);
    // twiddles W8^k for k = 0..3 applied to the odd half
    cplx<T> o1 = INV ? mk(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                     : mk(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    cplx<T> o2 = mul_mi<T, INV>(o[2]);
    cplx<T> o3 = INV ? mk(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                     : mk(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = e[0] + o[0]; v[4] = e[0] - o[0];
    v[1] = e[1] + o1;   v[5] = e[1] - o1;
    v[2] = e[2] + o2;   v[6] = e[2] - o2;
    v[3] = e[3] + o3;   v[7] = e[3] - o3;
}

// ---------------------------------------------------------------- Stockham FFT
// One radix-R Stockham stage for a thread holding NB butterflies of one line.
// Butterfly j (= t + G b) reads x[j + r M/R], twiddles by W_{Ns R}^{r k}
// (k = j mod Ns), and writes x[(j - k) R + k + r Ns].
template <typename T, bool INV, int R, int NB>
__device__ __forceinline__ void stockham_stage(cplx<T>* x, bool active, int t, int G, int M, int Ns,
                                               const cplx<T>* __restrict__ twM) {
    cplx<T> v[R * NB];
    const int MR = M / R;
    if (active) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = x[padc(t + G * b + r * MR)];
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + G * b;
            const int k = j & (Ns - 1);
            cplx<T>* w = v + b * R;
            if (Ns > 1) {
                const int step = k * (M / (Ns * R));
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    cplx<T> tw = twM[r * step];
                    w[r] = INV ? cmulc(w[r], tw) : cmul(w[r], tw);
                }
            }
            if (R == 8) dft8<T, INV>(w);
            else if (R == 4) dft4<T, INV>(w);
            else dft2<T, INV>(w[0], w[1]);
            const int i0 = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) x[padc(i0 + r * Ns)] = w[r];
        }
    }
    __syncthreads();
}

// Transforms `nrows` lines of M complex values (line r at buf + r * ldc, padded
// layout) in place.  All threads of the CTA must call it (it contains
// __syncthreads).  twM[t] = exp(-2 pi i t / M), t < M, in global memory.
// Each thread holds E = min(8, M) values of one line; G = M / E threads
// share a line and P = blockDim.x / G lines are transformed at once.
template <typename T, bool INV>
__device__ void fft_lines(cplx<T>* buf, int ldc, int nrows, int M, const cplx<T>* __restrict__ twM) {
    const int E = M < 8 ? M : 8;
    const int G = M / E;
    const int P = blockDim.x / G;
    const int tid = threadIdx.x;
    const int t = tid % G;
    const int pl = tid / G;
    for (int r0 = 0; r0 < nrows; r0 += P) {
        const int row = r0 + pl;
        const bool active = (pl < P) && (row < nrows);
        cplx<T>* x = buf + (size_t)(active ? row : 0) * ldc;
        for (int Ns = 1; Ns < M;) {
            const int rem = M / Ns;
            if (rem >= 8) { stockham_stage<T, INV, 8, 1>(x, active, t, G, M, Ns, twM); Ns *= 8; }
            else if (rem == 4) {
                if (E == 8) stockham_stage<T, INV, 4, 2>(x, active, t, G, M, Ns, twM);
                else stockham_stage<T, INV, 4, 1>(x, active, t, G, M, Ns, twM);
                Ns *= 4;
            } else { stockham_stage<T, INV, 2, 4>(x, active, t, G, M, Ns, twM); Ns *= 2; }
        }
    }
}

// ---------------------------------------------------------------- line packing
// Forward pack: real line x (global, N values, 16-byte aligned) into the
// complex FFT input z[m] = v[2m] + i v[2m+1], v the Makhoul reorder
// (v[n] = x[2n], v[N-1-n] = x[2n+1]).  Reading x in groups of four,
// x[4m..4m+3] gives z[m] = (x[4m], x[4m+2]) and z[M-1-m] = (x[4m+3], x[4m+1]).
template <typename T> struct vec4 { T a, b, c, d; };

template <typename T> __device__ __forceinline__ vec4<T> ld4(const T* p);
template <> __device__ __forceinline__ vec4<float> ld4<float>(const float* p) {
    float4 q = __ldg(reinterpret_cast<const float4*>(p));
    return {q.x, q.y, q.z, q.w};
}
template <> __device__ __forceinline__ vec4<double> ld4<double>(const double* p) {
    double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
    double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return {q0.x, q0.y, q1.x, q1.y};
}
template <typename T> __device__ __forceinline__ void st4(T* p, vec4<T> v);
template <> __device__ __forceinline__ void st4<float>(float* p, vec4<float> v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.a, v.b, v.c, v.d);
}
template <> __device__ __forceinline__ void st4<double>(double* p, vec4<double> v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v.a, v.b);
    reinterpret_cast<double2*>(p)[1] = make_double2(v.c, v.d);
}

// Pack from 4 values that the caller already holds (x[4m..4m+3]).
template <typename T> __device__ __forceinline__ void pack4(cplx<T>* z, int M, int m, vec4<T> q) {
    z[padc(m)] = mk(q.a, q.c);
    z[padc(M - 1 - m)] = mk(q.d, q.b);
}

// Inverse unpack: z (IDFT output) -> x[4m..4m+3].
template <typename T> __device__ __forceinline__ vec4<T> unpack4(const cplx<T>* z, int M, int m) {
    cplx<T> a = z[padc(m)], b = z[padc(M - 1 - m)];
    return {a.x, b.y, a.y, b.x};
}

// ---------------------------------------------------------------- post/pre twiddles
// Per-size table entry k in [0, M/2]: cos/sin(2 pi k/N) and cos/sin(pi k/(2N)).
template <typename T> struct PostTw { T cN, sN, c4, s4; };

// Forward post-process of the pair (k, M-k), 0 <= k <= M/2, from the FFT
// output Z.  Produces X[k], X[N-k], X[M-k], X[M+k] (orthonormal DCT-II;
// X[N] for k = 0 is not produced).  cn0 = sqrt(1/N), cn = sqrt(2/N).
template <typename T> struct Quad { T xk, xNk, xMk, xMpk; };

template <typename T>
__device__ __forceinline__ Quad<T> post_forward(const cplx<T>* Z, int M, int k, PostTw<T> tw, T cn0, T cn) {
    const T h = (T)0.70710678118654752440;
    cplx<T> A = Z[padc(k)];
    cplx<T> B = Z[padc(k == 0 ? 0 : M - k)];
    cplx<T> WN = mk(tw.cN, -tw.sN), W4 = mk(tw.c4, -tw.s4);
    cplx<T> E = scale(A + conj_(B), (T)0.5);
    cplx<T> D = scale(A - conj_(B), (T)0.5);          // O = -i D
    cplx<T> O = mk(D.y, -D.x);
    cplx<T> W = cmul(W4, E + cmul(WN, O));
    // mode M-k: E' = conj(E), O' = -i (B - conj A)/2 = -i * (-conj(D)) = i conj(D)
    cplx<T> Dc = conj_(D);
    cplx<T> O2 = mk(-Dc.y, Dc.x);
    cplx<T> WN2 = mk(-WN.x, WN.y);                    // -conj(WN)
    cplx<T> W4c = conj_(W4);
    cplx<T> W42 = mk(h * (W4c.x + W4c.y), h * (W4c.y - W4c.x));   // exp(-i pi/4) * conj(W4)
    cplx<T> W2 = cmul(W42, conj_(E) + cmul(WN2, O2));
    Quad<T> q;
    q.xk = (k == 0 ? cn0 : cn) * W.x;
    q.xNk = -cn * W.y;
    q.xMk = cn * W2.x;
    q.xMpk = -cn * W2.y;
    return q;
}

// Inverse pre-process of the pair (k, M-k), 0 <= k <= M/2: from the
// orthonormal coefficients X[k], X[N-k] (0 for k = 0), X[M-k], X[M+k]
// builds Zin[k] and Zin[M-k] (the latter unused for k = 0) such that the
// unnormalised inverse FFT of Zin followed by unpack4 gives the DCT-III.
// inv0 = 1/(M sqrt(1/N)), inv = 1/(M sqrt(2/N)).
template <typename T>
__device__ __forceinline__ void pre_inverse(Quad<T> X, int k, PostTw<T> tw, T inv0, T inv,
                                            cplx<T>& zk, cplx<T>& zMk) {
    const T h = (T)0.70710678118654752440;
    T Uk = X.xk * (k == 0 ? inv0 : inv);
    T UNk = (k == 0) ? (T)0 : X.xNk * inv;
    T UMk = X.xMk * inv, UMpk = X.xMpk * inv;
    cplx<T> W4 = mk(tw.c4, -tw.s4);
    cplx<T> WN = mk(tw.cN, -tw.sN);
    // V_k = conj(W4) (U_k - i U_{N-k}); V_{M-k} = exp(i pi/4) W4 (U_{M-k} - i U_{M+k})
    cplx<T> Vk = cmul(conj_(W4), mk(Uk, -UNk));
    cplx<T> e4W4 = mk(h * (W4.x - W4.y), h * (W4.x + W4.y));
    cplx<T> Vm = cmul(e4W4, mk(UMk, -UMpk));
    cplx<T> s = scale(Vk + conj_(Vm), (T)0.5);
    cplx<T> d = scale(Vk - conj_(Vm), (T)0.5);
    cplx<T> t = cmul(d, conj_(WN));
    zk = mk(s.x - t.y, s.y + t.x);                    // s + i t
    cplx<T> s2 = scale(Vm + conj_(Vk), (T)0.5);
    cplx<T> d2 = scale(Vm - conj_(Vk), (T)0.5);
    cplx<T> WNm = mk(-WN.x, WN.y);                    // W_N^{M-k} = -conj(WN)
    cplx<T> t2 = cmul(d2, conj_(WNm));
    zMk = mk(s2.x - t2.y, s2.y + t2.x);
}

}  // namespace ccm
