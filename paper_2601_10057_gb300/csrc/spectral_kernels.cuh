// spectral_kernels.cuh -- kernels of the standalone constant-coefficient
// spectral solver and of the initial-condition smoother.
//
// The solver computes u = (c0 - c1 Lap_h + c2 Lap_h^2)^{-1} f on an N x N
// cell-centred grid (Appendix C of the paper: forward transform, divide by
// the closed-form eigenvalues, inverse transform), for three boundary rules
// of the 5-point Laplacian Lap_h:
//   Neumann    mirror ghosts u_{-1} = u_0 (Appendix D):       orthonormal
//              DCT-II / DCT-III, eigenvalues of -Lap_h (4/h^2)(sin^2(pi k/2N)
//              + sin^2(pi l/2N));
//   Dirichlet  odd ghosts u_{-1} = -u_0 (u = 0 on the boundary faces):
//              DST-II / DST-III, computed as the DCT of (-1)^{i+j} u (the
//              DCT's mode N-1-k is the DST's mode k), so the eigenvalue at DCT
//              index k is (4/h^2) sin^2(pi (N-k)/2N) = (4/h^2) cos^2(pi k/2N);
//   periodic   wrapped ghosts u_{-1} = u_{N-1}: the complex DFT of length N
//              along both axes, eigenvalues (4/h^2)(sin^2(pi k/N) + sin^2(pi l/N)).
// The paper names the DST and FFT solvers as the fast solvers for Dirichlet
// and periodic boundaries (Sec. 5, limitations and scope).
//
// The DCT/DST kernels transform gridDim.y fields at once (field f at offset
// f * fstride of every array); a field whose dskip[f] is set is left alone
// (iterations of a solver that has converged), and dcoef, if given, holds
// the coefficients c0, c1, c2 on the device.
//
// Data flow of one solve (three kernels):
//   k_ss_row_fwd    transform along x of RT rows, written transposed (line kx
//                   of the scratch holds the column-x spectra over y);
//   k_ss_col_solve  transform along y of each line, divide, inverse transform
//                   along y, written back in place;
//   k_ss_row_inv    transposed read of RT rows, inverse transform along x,
//                   output in natural layout.
// The DCT lines use Makhoul's half-length complex FFT (dct_device.cuh); the
// periodic lines a full-length complex FFT.
#pragma once
#include "dct_device.cuh"

namespace ccm {
namespace ss {

enum { BC_NEUMANN = 0, BC_DIRICHLET = 1, BC_PERIODIC = 2 };

// (-1)^(i+j) for the Dirichlet transform
template <typename T> __device__ __forceinline__ T alt(int i) { return (i & 1) ? (T)-1 : (T)1; }

// ------------------------------------------------------------------ DCT / DST lines
// Forward DCT-II along x of rows y0 .. y0+RT-1 (DST: of (-1)^(i+j) u), written
// transposed: out[kx * N + y].
template <typename T, bool DST>
__global__ void __launch_bounds__(512)
k_ss_row_fwd(const T* __restrict__ in, T* __restrict__ out, int N, int RT, int lds,
             const cplx<T>* __restrict__ twM, const PostTw<T>* __restrict__ twP,
             const int* __restrict__ dskip, size_t fstride) {
    if (dskip && dskip[blockIdx.y]) return;
    in += blockIdx.y * fstride;
    out += blockIdx.y * fstride;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = N / 2, ldc = padded_len(M);
    const int E = M < 8 ? M : 8, G = M / E, P = blockDim.x / G;
    T* stage = reinterpret_cast<T*>(smraw);                                   // RT x lds
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw + (((size_t)RT * lds * sizeof(T) + 15) & ~(size_t)15));
    const int y0 = blockIdx.x * RT;
    const T cn0 = (T)sqrt(1.0 / N), cn = (T)sqrt(2.0 / N);
    for (int r0 = 0; r0 < RT; r0 += P) {
        const int nr = min(P, RT - r0);
        for (int q = threadIdx.x; q < nr * (M / 2); q += blockDim.x) {
            const int r = q / (M / 2), m = q % (M / 2);
            const int y = y0 + r0 + r;
            vec4<T> v = ld4(in + (size_t)y * N + 4 * m);
            if (DST) {   // x = 4m is even: signs (+, -, +, -) times (-1)^y
                const T s = alt<T>(y);
                v.a *= s; v.b *= -s; v.c *= s; v.d *= -s;
            }
            pack4(fb + (size_t)r * ldc, M, m, v);
        }
        __syncthreads();
        fft_lines<T, false>(fb, ldc, nr, M, twM);
        for (int q = threadIdx.x; q < nr * (M / 2 + 1); q += blockDim.x) {
            const int r = q / (M / 2 + 1), k = q % (M / 2 + 1);
            const Quad<T> X = post_forward(fb + (size_t)r * ldc, M, k, twP[k], cn0, cn);
            T* srow = stage + (size_t)(r0 + r) * lds;
            srow[k] = X.xk;
            if (k > 0) srow[N - k] = X.xNk;
            if (k < M / 2) srow[M - k] = X.xMk;
            if (k > 0 && k < M / 2) srow[M + k] = X.xMpk;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q % RT, kx = q / RT;
        out[(size_t)kx * N + y0 + r] = stage[(size_t)r * lds + kx];
    }
}

// Lines kx0 .. kx0+RC-1 of the transposed buffer (contiguous over y): forward
// DCT-II along y, divide each mode by c0 + c1 s + c2 s^2 (s = ev[kx] + ev[ky],
// the eigenvalue of -Lap_h), inverse DCT-III, written back in place.  Each
// pair (k, M-k) of the half-length FFT is post-processed, divided and
// pre-processed by one thread in the slots it read, so the line buffer is
// reused in place.
template <typename T>
__global__ void __launch_bounds__(512)
k_ss_col_solve(T* __restrict__ data, int N, int RC, const cplx<T>* __restrict__ twM,
               const PostTw<T>* __restrict__ twP, const double* __restrict__ ev,
               double c0, double c1, double c2, const double* __restrict__ dcoef,
               const int* __restrict__ dskip, size_t fstride) {
    if (dskip && dskip[blockIdx.y]) return;
    data += blockIdx.y * fstride;
    if (dcoef) { c0 = dcoef[0]; c1 = dcoef[1]; c2 = dcoef[2]; }   // coefficients formed on the device
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = N / 2, ldc = padded_len(M);
    const int E = M < 8 ? M : 8, G = M / E, P = blockDim.x / G;
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw);
    const int kx0 = blockIdx.x * RC;
    const T cn0 = (T)sqrt(1.0 / N), cn = (T)sqrt(2.0 / N);
    const T inv0 = (T)(1.0 / (M * sqrt(1.0 / N))), inv = (T)(1.0 / (M * sqrt(2.0 / N)));
    for (int l0 = 0; l0 < RC; l0 += P) {
        const int nl = min(P, RC - l0);
        for (int q = threadIdx.x; q < nl * (M / 2); q += blockDim.x) {
            const int l = q / (M / 2), m = q % (M / 2);
            pack4(fb + (size_t)l * ldc, M, m, ld4(data + (size_t)(kx0 + l0 + l) * N + 4 * m));
        }
        __syncthreads();
        fft_lines<T, false>(fb, ldc, nl, M, twM);
        for (int q = threadIdx.x; q < nl * (M / 2 + 1); q += blockDim.x) {
            const int l = q / (M / 2 + 1), k = q % (M / 2 + 1);
            cplx<T>* z = fb + (size_t)l * ldc;
            Quad<T> X = post_forward(z, M, k, twP[k], cn0, cn);
            const double ex = ev[kx0 + l0 + l];
            auto div = [&](T v, int ky) {
                const double s = ex + ev[ky];
                return (T)((double)v / (c0 + s * (c1 + c2 * s)));
            };
            X.xk = div(X.xk, k);
            X.xNk = k > 0 ? div(X.xNk, N - k) : (T)0;
            X.xMk = div(X.xMk, M - k);
            X.xMpk = div(X.xMpk, M + k);
            cplx<T> zk, zMk;
            pre_inverse(X, k, twP[k], inv0, inv, zk, zMk);
            z[padc(k)] = zk;
            if (k > 0) z[padc(M - k)] = zMk;
        }
        __syncthreads();
        fft_lines<T, true>(fb, ldc, nl, M, twM);
        for (int q = threadIdx.x; q < nl * (M / 2); q += blockDim.x) {
            const int l = q / (M / 2), m = q % (M / 2);
            st4(data + (size_t)(kx0 + l0 + l) * N + 4 * m, unpack4(fb + (size_t)l * ldc, M, m));
        }
        __syncthreads();
    }
}

// Rows y0 .. y0+RT-1: transposed read in[kx * N + y], inverse DCT-III along
// x (DST: times (-1)^(i+j)), natural-layout output.
template <typename T, bool DST>
__global__ void __launch_bounds__(512)
k_ss_row_inv(const T* __restrict__ in, T* __restrict__ out, int N, int RT, int lds,
             const cplx<T>* __restrict__ twM, const PostTw<T>* __restrict__ twP,
             const int* __restrict__ dskip, size_t fstride) {
    if (dskip && dskip[blockIdx.y]) return;
    in += blockIdx.y * fstride;
    out += blockIdx.y * fstride;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = N / 2, ldc = padded_len(M);
    const int E = M < 8 ? M : 8, G = M / E, P = blockDim.x / G;
    T* stage = reinterpret_cast<T*>(smraw);                                   // RT x lds
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw + (((size_t)RT * lds * sizeof(T) + 15) & ~(size_t)15));
    const int y0 = blockIdx.x * RT;
    const T inv0 = (T)(1.0 / (M * sqrt(1.0 / N))), inv = (T)(1.0 / (M * sqrt(2.0 / N)));
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q % RT, kx = q / RT;
        stage[(size_t)r * lds + kx] = in[(size_t)kx * N + y0 + r];
    }
    __syncthreads();
    for (int r0 = 0; r0 < RT; r0 += P) {
        const int nr = min(P, RT - r0);
        for (int q = threadIdx.x; q < nr * (M / 2 + 1); q += blockDim.x) {
            const int r = q / (M / 2 + 1), k = q % (M / 2 + 1);
            const T* srow = stage + (size_t)(r0 + r) * lds;
            const Quad<T> X{srow[k], k > 0 ? srow[N - k] : (T)0, srow[M - k], srow[M + k]};
            cplx<T> zk, zMk;
            pre_inverse(X, k, twP[k], inv0, inv, zk, zMk);
            cplx<T>* z = fb + (size_t)r * ldc;
            z[padc(k)] = zk;
            if (k > 0) z[padc(M - k)] = zMk;
        }
        __syncthreads();
        fft_lines<T, true>(fb, ldc, nr, M, twM);
        for (int q = threadIdx.x; q < nr * (M / 2); q += blockDim.x) {
            const int r = q / (M / 2), m = q % (M / 2);
            const int y = y0 + r0 + r;
            vec4<T> v = unpack4(fb + (size_t)r * ldc, M, m);
            if (DST) {
                const T s = alt<T>(y);
                v.a *= s; v.b *= -s; v.c *= s; v.d *= -s;
            }
            st4(out + (size_t)y * N + 4 * m, v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ periodic lines
// Full-length complex FFT of RT real rows (imaginary part 0), written
// transposed as complex values: outc[kx * N + y].
template <typename T>
__global__ void __launch_bounds__(1024)
k_ss_row_fwd_p(const T* __restrict__ in, cplx<T>* __restrict__ outc, int N, int RT,
               const cplx<T>* __restrict__ twN) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ldc = padded_len(N);
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw);     // RT lines
    const int y0 = blockIdx.x * RT;
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q / N, i = q % N;
        fb[(size_t)r * ldc + padc(i)] = mk(in[(size_t)(y0 + r) * N + i], (T)0);
    }
    __syncthreads();
    fft_lines<T, false>(fb, ldc, RT, N, twN);
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q % RT, kx = q / RT;
        outc[(size_t)kx * N + y0 + r] = fb[(size_t)r * ldc + padc(kx)];
    }
}

// Complex lines kx0 .. kx0+RC-1 (contiguous over y): FFT, divide by
// c0 + c1 s + c2 s^2 (s = evp[kx] + evp[ky]), inverse FFT, in place.
template <typename T>
__global__ void __launch_bounds__(1024)
k_ss_col_solve_p(cplx<T>* __restrict__ data, int N, int RC, const cplx<T>* __restrict__ twN,
                 const double* __restrict__ evp, double c0, double c1, double c2) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ldc = padded_len(N);
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw);
    const int kx0 = blockIdx.x * RC;
    for (int q = threadIdx.x; q < RC * N; q += blockDim.x) {
        const int l = q / N, i = q % N;
        fb[(size_t)l * ldc + padc(i)] = data[(size_t)(kx0 + l) * N + i];
    }
    __syncthreads();
    fft_lines<T, false>(fb, ldc, RC, N, twN);
    for (int q = threadIdx.x; q < RC * N; q += blockDim.x) {
        const int l = q / N, ky = q % N;
        const double s = evp[kx0 + l] + evp[ky];
        const T d = (T)(1.0 / (c0 + s * (c1 + c2 * s)));
        cplx<T>& z = fb[(size_t)l * ldc + padc(ky)];
        z = scale(z, d);
    }
    __syncthreads();
    fft_lines<T, true>(fb, ldc, RC, N, twN);
    for (int q = threadIdx.x; q < RC * N; q += blockDim.x) {
        const int l = q / N, i = q % N;
        data[(size_t)(kx0 + l) * N + i] = fb[(size_t)l * ldc + padc(i)];
    }
}

// Rows y0 .. y0+RT-1: transposed complex read, inverse FFT along x, the real
// part divided by N^2 (the unnormalised forward and inverse FFTs along both
// axes multiply by N twice), natural-layout real output.
template <typename T>
__global__ void __launch_bounds__(1024)
k_ss_row_inv_p(const cplx<T>* __restrict__ inc, T* __restrict__ out, int N, int RT,
               const cplx<T>* __restrict__ twN) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ldc = padded_len(N);
    cplx<T>* fb = reinterpret_cast<cplx<T>*>(smraw);
    const int y0 = blockIdx.x * RT;
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q % RT, kx = q / RT;
        fb[(size_t)r * ldc + padc(kx)] = inc[(size_t)kx * N + y0 + r];
    }
    __syncthreads();
    fft_lines<T, true>(fb, ldc, RT, N, twN);
    const T sc = (T)(1.0 / ((double)N * (double)N));
    for (int q = threadIdx.x; q < RT * N; q += blockDim.x) {
        const int r = q / N, i = q % N;
        out[(size_t)(y0 + r) * N + i] = fb[(size_t)r * ldc + padc(i)].x * sc;
    }
}

// ------------------------------------------------------------------ smoother (Appendix F)
// Ghost index of the boundary rule (one cell beyond the grid) and its sign.
__device__ __forceinline__ int ghost_idx(int i, int N, int bc, float& sgn) {
    sgn = 1.f;
    if (i >= 0 && i < N) return i;
    if (bc == BC_PERIODIC) return i < 0 ? i + N : i - N;
    if (bc == BC_DIRICHLET) sgn = -1.f;
    return i < 0 ? 0 : N - 1;
}

// Right-hand side of one semi-implicit step of the constant-mobility
// Cahn-Hilliard smoother: r = phi / dt + Mob Lap_h g(phi), g = (phi^3 - phi)/eps
// (g is odd, so the Dirichlet ghost of g is -g of the mirrored cell).
template <typename T>
__global__ void k_smooth_rhs(const T* __restrict__ phi, T* __restrict__ r, int N, int bc,
                             double inv_dt, double mob_inv_h2, double inv_eps) {
    const size_t NN = (size_t)N * N;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % N), j = (int)(q / N);
        auto g = [&](int ii, int jj) -> double {
            float si, sj;
            const int gi = ghost_idx(ii, N, bc, si), gj = ghost_idx(jj, N, bc, sj);
            const double p = (double)phi[(size_t)gj * N + gi];
            return (double)(si * sj) * (p * p * p - p) * inv_eps;
        };
        const double gc = g(i, j);
        const double lap = (g(i + 1, j) - gc) + (g(i - 1, j) - gc) + ((g(i, j + 1) - gc) + (g(i, j - 1) - gc));
        r[q] = (T)((double)phi[q] * inv_dt + mob_inv_h2 * lap);
    }
}

// ------------------------------------------------------------------ launch geometry
// Threads per CTA, rows per CTA of the row kernels (RT), lines per CTA of the
// column kernel (RC) and the dynamic shared memory of each, for N x N fields
// of precision T (periodic: full-length complex lines).
struct Geo {
    int threads = 256, RT = 1, RC = 1, lds = 0;
    size_t sm_fwd = 0, sm_col = 0, sm_inv = 0;
};

template <typename T> inline Geo geometry(int N, bool periodic) {
    constexpr size_t cap = 200 * 1024;
    Geo g;
    const int M = periodic ? N : N / 2;                // complex line length
    const int E = M < 8 ? M : 8, G = M / E;
    g.threads = G > 256 ? G : 256;                     // <= 512 for DCT lines, <= 1024 periodic
    const int P = g.threads / G;                       // lines transformed at once
    const size_t line = (size_t)padded_len(M) * sizeof(cplx<T>);
    if (periodic) {
        int rt = 8;
        while (rt > 1 && ((size_t)rt * line > cap || N % rt)) rt /= 2;
        if (rt > N) rt = N;
        g.RT = g.RC = rt;
        g.sm_fwd = g.sm_col = g.sm_inv = (size_t)rt * line;
    } else {
        g.lds = N + 1;
        auto rows_bytes = [&](int rt) {
            return (((size_t)rt * g.lds * sizeof(T) + 15) & ~(size_t)15) + (size_t)(rt < P ? rt : P) * line;
        };
        int rt = 16;
        while (rt > 1 && (rows_bytes(rt) > cap || N % rt)) rt /= 2;
        if (rt > N) rt = N;
        g.RT = rt;
        g.sm_fwd = g.sm_inv = rows_bytes(rt);
        int rc = P < 8 ? P : 8;
        while (rc > 1 && ((size_t)rc * line > cap || N % rc)) rc /= 2;
        g.RC = rc;
        g.sm_col = (size_t)rc * line;
    }
    return g;
}

// Opt a kernel in to the largest dynamic shared memory a block can take (the
// attribute is per kernel and process-wide, so it must not depend on one
// grid size); fails if that is below `bytes`.
inline int optin_smem(const void* fn, size_t bytes) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
        return -3;   // CCMSAV_ECUDA
    const int lim = optin - (int)fa.sharedSizeBytes;
    if (lim < 0 || (size_t)lim < bytes) return -1;   // CCMSAV_EINVAL
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess ? 0 : -3;
}

// Opt in every DCT/DST kernel of precision T (Neumann and Dirichlet) or every
// periodic one.
template <typename T> inline int optin_all(const Geo& g, bool periodic) {
    int r = 0;
    if (periodic) {
        if ((r = optin_smem((const void*)k_ss_row_fwd_p<T>, g.sm_fwd)) ||
            (r = optin_smem((const void*)k_ss_col_solve_p<T>, g.sm_col)) ||
            (r = optin_smem((const void*)k_ss_row_inv_p<T>, g.sm_inv)))
            return r;
    } else {
        if ((r = optin_smem((const void*)k_ss_row_fwd<T, false>, g.sm_fwd)) ||
            (r = optin_smem((const void*)k_ss_row_fwd<T, true>, g.sm_fwd)) ||
            (r = optin_smem((const void*)k_ss_col_solve<T>, g.sm_col)) ||
            (r = optin_smem((const void*)k_ss_row_inv<T, false>, g.sm_inv)) ||
            (r = optin_smem((const void*)k_ss_row_inv<T, true>, g.sm_inv)))
            return r;
    }
    return 0;
}

// phi <- max(-1, min(1, phi)) (the final step of Appendix F)
template <typename T>
__global__ void k_clamp(T* __restrict__ phi, size_t n) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        phi[q] = fmin(fmax(phi[q], (T)-1), (T)1);
}

}  // namespace ss
}  // namespace ccm
