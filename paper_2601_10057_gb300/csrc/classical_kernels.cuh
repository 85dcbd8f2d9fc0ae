// classical_kernels.cuh -- the Cahn-Hilliard part of the classical MSAV
// scheme (the baseline of Sec. 3.5.2 of the paper; Appendix B remarks on the
// Classical-MSAV-BDF2 / BDF1 schemes), solved by DCT-preconditioned
// conjugate gradients on the GPU.
//
// In the classical scheme the Cahn-Hilliard stabilisation sits inside the
// chemical potential, nu^{n+1} = lam (psi^{n+1} - psi*) + Z^{n+1} P, so its
// operator has the variable mobility:
//   zeta_c u = a u - lam div(M_psi(A phi*) grad u),   a = 3/(2 dt) (BDF1: 1/dt).
// In the increment form psi^{n+1} = psi_bar + d_psi the step needs
//   y1 = zeta_c^{-1} g0c,  g0c = lam div(M grad(psi_bar - psi*)),
//   y2 = zeta_c^{-1} LP,   LP  = div(M grad P)      (the stencil's output),
// then d_psi = y1 + aL y2 with the recovery coefficient aL of the 5x5 solve,
// whose psi entries are the physical inner products (P, y1) and (P, y2).
// Both systems are solved together by preconditioned CG (the operator is
// symmetric positive definite); the preconditioner is the constant-
// coefficient operator a - lam Mbar Lap_h (Mbar: the mean interior face
// mobility), inverted by DCT (spectral_kernels.cuh), as in the paper's
// Classical+DCT-PCG.  Every inner product is a per-block partial sum plus a
// last-block-done reduction in a fixed order (no spin-wait); the CG scalars
// stay on the device.
#pragma once
#include "step_kernels.cuh"

namespace ccm {

// Device state of the two conjugate-gradient solves.
struct PcgScalars {
    double rho[2], alpha[2], beta[2], rr0[2], rr[2];
    double coef[3];        // preconditioner: c0 = a, c1 = lam Mbar, c2 = 0
    double ip[2];          // sum_ij P y1, sum_ij P y2
    double rtol2;          // converged when ||r||^2 <= rtol2 ||b||^2
    int conv[2];           // 1: system s has converged (its later kernels return at once)
    int iters[2];          // iterations taken by system s in this step
    unsigned arrivals;     // blocks done with the current reduction (reset by the last)
};

constexpr int kClThreads = 256;

// Fixed-order block sum of NV values, then the last block to arrive adds the
// block sums (in block order) and runs fin(total) on thread 0.
template <int NV, typename Fin>
__device__ __forceinline__ void cl_reduce(double (&v)[NV], double* __restrict__ red, PcgScalars* pc, Fin fin) {
    __shared__ double sm[kClThreads / 32][NV];
    __shared__ int last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sm[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int q = 0; q < kClThreads / 32; ++q) s += sm[q][threadIdx.x];
        red[(size_t)blockIdx.x * NV + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&pc->arrivals, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(red + (size_t)b * NV + threadIdx.x);
        sm[0][threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = sm[0][k];
        fin(tot);
        pc->arrivals = 0u;
    }
}

__device__ __forceinline__ double mob_face(double a, double M0) {
    const double s = a * a - 1.0;
    return 1.0 - M0 * s * s;
}

// Face mobilities of phi* (east face of cell i in Mx, north face in My; 0 on
// boundary faces, which carry no flux), the right-hand side g0c, the
// preconditioner coefficients from the mean interior face mobility, and the
// reset of the CG state.
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_prep(const T* __restrict__ phn, const T* __restrict__ pho, const T* __restrict__ psn,
          const T* __restrict__ pso, int bdf1, T* __restrict__ Mx, T* __restrict__ My, T* __restrict__ b1,
          double* __restrict__ red, PcgScalars* __restrict__ pc, int N, double a, double lam,
          double M0, double inv_h2, double rtol) {
    const size_t NN = (size_t)N * N;
    double msum = 0.0;
    auto phs = [&](int i, int j) {
        const size_t q = (size_t)j * N + i;
        return bdf1 ? (double)phn[q] : 2.0 * (double)phn[q] - (double)pho[q];
    };
    auto dq = [&](int i, int j) {   // psi_bar - psi* = -(2/3)(psi^n - psi^{n-1}) (0 for BDF1)
        const size_t q = (size_t)j * N + i;
        return bdf1 ? 0.0 : -2.0 / 3.0 * ((double)psn[q] - (double)pso[q]);
    };
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % N), j = (int)(q / N);
        const double pc0 = phs(i, j);
        const double mE = i + 1 < N ? mob_face(0.5 * (pc0 + phs(i + 1, j)), M0) : 0.0;
        const double mW = i > 0 ? mob_face(0.5 * (pc0 + phs(i - 1, j)), M0) : 0.0;
        const double mN = j + 1 < N ? mob_face(0.5 * (pc0 + phs(i, j + 1)), M0) : 0.0;
        const double mS = j > 0 ? mob_face(0.5 * (pc0 + phs(i, j - 1)), M0) : 0.0;
        Mx[q] = (T)mE;
        My[q] = (T)mN;
        msum += mE + mN;
        const double d0 = dq(i, j);
        double g = 0.0;
        if (i + 1 < N) g += mE * (dq(i + 1, j) - d0);
        if (i > 0) g -= mW * (d0 - dq(i - 1, j));
        if (j + 1 < N) g += mN * (dq(i, j + 1) - d0);
        if (j > 0) g -= mS * (d0 - dq(i, j - 1));
        b1[q] = (T)(lam * g * inv_h2);
    }
    double v[1] = {msum};
    cl_reduce<1>(v, red, pc, [&](const double* t) {
        const double mbar = t[0] / (2.0 * (double)N * (double)(N - 1));
        pc->coef[0] = a; pc->coef[1] = lam * mbar; pc->coef[2] = 0.0;
        pc->rtol2 = rtol * rtol;
        for (int s = 0; s < 2; ++s) { pc->conv[s] = 0; pc->iters[s] = 0; pc->alpha[s] = pc->beta[s] = 0.0; }
    });
}

// x = 0, p = 0, r = b for both systems (b = (b1, b2)), ||b||^2.
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_init(const T* __restrict__ b1, const T* __restrict__ b2, T* __restrict__ x, T* __restrict__ r,
          T* __restrict__ p, double* __restrict__ red, PcgScalars* __restrict__ pc, size_t NN) {
    double v[2] = {0.0, 0.0};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        const T u1 = b1[q], u2 = b2[q];
        x[q] = (T)0; x[NN + q] = (T)0;
        p[q] = (T)0; p[NN + q] = (T)0;
        r[q] = u1; r[NN + q] = u2;
        v[0] += (double)u1 * (double)u1;
        v[1] += (double)u2 * (double)u2;
    }
    cl_reduce<2>(v, red, pc, [&](const double* t) {
        for (int s = 0; s < 2; ++s) {
            pc->rr0[s] = t[s];
            pc->rr[s] = t[s];
            if (!(t[s] > 0.0)) pc->conv[s] = 1;          // zero right-hand side: y = 0
        }
    });
}

// rho_new = (r, z); first: rho = rho_new, beta = 0; else beta = rho_new / rho.
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_dot_rz(const T* __restrict__ r, const T* __restrict__ z, double* __restrict__ red,
            PcgScalars* __restrict__ pc, size_t NN, int first) {
    const int c0 = pc->conv[0], c1 = pc->conv[1];
    double v[2] = {0.0, 0.0};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        if (!c0) v[0] += (double)r[q] * (double)z[q];
        if (!c1) v[1] += (double)r[NN + q] * (double)z[NN + q];
    }
    cl_reduce<2>(v, red, pc, [&](const double* t) {
        for (int s = 0; s < 2; ++s) {
            if (pc->conv[s]) continue;
            pc->beta[s] = first ? 0.0 : t[s] / pc->rho[s];
            pc->rho[s] = t[s];
        }
    });
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_pupdate(const T* __restrict__ z, T* __restrict__ p, const PcgScalars* __restrict__ pc, size_t NN) {
    for (int s = 0; s < 2; ++s) {
        if (pc->conv[s]) continue;
        const T b = (T)pc->beta[s];
        const T* zs = z + s * NN;
        T* ps = p + s * NN;
        for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x)
            ps[q] = zs[q] + b * ps[q];
    }
}

// q = zeta_c p and (p, q); alpha = rho / (p, q).
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_apply(const T* __restrict__ p, const T* __restrict__ Mx, const T* __restrict__ My, T* __restrict__ qv,
           double* __restrict__ red, PcgScalars* __restrict__ pc, int N, double a, double lam_inv_h2) {
    const size_t NN = (size_t)N * N;
    const int cv[2] = {pc->conv[0], pc->conv[1]};
    double v[2] = {0.0, 0.0};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % N), j = (int)(q / N);
        const double mE = (double)Mx[q], mN = (double)My[q];
        const double mW = i > 0 ? (double)Mx[q - 1] : 0.0, mS = j > 0 ? (double)My[q - N] : 0.0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (cv[s]) continue;
            const T* ps = p + s * NN;
            const double c = (double)ps[q];
            double d = 0.0;
            if (i + 1 < N) d += mE * ((double)ps[q + 1] - c);
            if (i > 0) d -= mW * (c - (double)ps[q - 1]);
            if (j + 1 < N) d += mN * ((double)ps[q + N] - c);
            if (j > 0) d -= mS * (c - (double)ps[q - N]);
            const double Av = a * c - lam_inv_h2 * d;
            qv[s * NN + q] = (T)Av;
            v[s] += c * Av;
        }
    }
    cl_reduce<2>(v, red, pc, [&](const double* t) {
        for (int s = 0; s < 2; ++s)
            if (!pc->conv[s]) pc->alpha[s] = pc->rho[s] / t[s];
    });
}

// x += alpha p, r -= alpha q, ||r||^2; convergence test on the last block.
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ qv,
            double* __restrict__ red, PcgScalars* __restrict__ pc, size_t NN) {
    const int cv[2] = {pc->conv[0], pc->conv[1]};
    const T al[2] = {(T)pc->alpha[0], (T)pc->alpha[1]};
    double v[2] = {0.0, 0.0};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (cv[s]) continue;
            const size_t o = s * NN + q;
            x[o] += al[s] * p[o];
            const T rn = r[o] - al[s] * qv[o];
            r[o] = rn;
            v[s] += (double)rn * (double)rn;
        }
    }
    cl_reduce<2>(v, red, pc, [&](const double* t) {
        for (int s = 0; s < 2; ++s) {
            if (pc->conv[s]) continue;
            pc->rr[s] = t[s];
            pc->iters[s] += 1;
            if (t[s] <= pc->rtol2 * pc->rr0[s]) pc->conv[s] = 1;
        }
    });
}

// sum_ij P y1 and sum_ij P y2 (the psi entries of the 5x5 system, before the h^2 factor).
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_pdot(const T* __restrict__ P, const T* __restrict__ y, double* __restrict__ red,
          PcgScalars* __restrict__ pc, size_t NN) {
    double v[2] = {0.0, 0.0};
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x) {
        const double pv = (double)P[q];
        v[0] += pv * (double)y[q];
        v[1] += pv * (double)y[NN + q];
    }
    cl_reduce<2>(v, red, pc, [&](const double* t) { pc->ip[0] = t[0]; pc->ip[1] = t[1]; });
}

// Replace the spectral psi entries (columns 15, 16) of the Gram partial rows
// by the conjugate-gradient inner products: row 0 holds them, the other rows 0.
template <typename P>
__global__ void k_cl_inject(P* __restrict__ part2, int nb2, const PcgScalars* __restrict__ pc) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nb2; r += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const double v = r == 0 ? pc->ip[c] : 0.0;
            if constexpr (std::is_same<P, float2>::value) {
                const float hi = (float)v;
                part2[(size_t)r * NRED2 + 15 + c] = make_float2(hi, (float)(v - (double)hi));
            } else {
                part2[(size_t)r * NRED2 + 15 + c] = v;
            }
        }
}

// psi^{n+1} = psi_bar + y1 + aL y2 (overwrites the spectral recovery of psi).
template <typename T>
__global__ void __launch_bounds__(kClThreads)
k_cl_psi(const T* __restrict__ psn, const T* __restrict__ pso, const T* __restrict__ y,
         const DevScalars* __restrict__ dsc, int bdf1, T* __restrict__ psi_new, size_t NN) {
    const T aL = (T)dsc->alpha[4];
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NN; q += (size_t)gridDim.x * blockDim.x)
        psi_new[q] = bar_add(psn[q], pso[q], y[q] + aL * y[NN + q], (T)0, bdf1 != 0);
}

}  // namespace ccm
