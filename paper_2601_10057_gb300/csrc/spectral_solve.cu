// spectral_solve.cu -- the standalone constant-coefficient spectral solver
// (Neumann DCT, Dirichlet DST, periodic FFT; Appendix C of the paper and its
// closing remarks on other boundaries) and the initial-condition smoother of
// Appendix F, behind the ccmsav_solver_* entry points of include/ccmsav.h.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include "../../include/ccmsav.h"
#include "spectral_kernels.cuh"

struct ccmsav_solver {
    int N = 0, bc = 0, precision = 0;
    double L = 1.0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    void* scratch = nullptr;       // N*N of T (DCT/DST) or of cplx<T> (periodic)
    void* rhs = nullptr;           // N*N of T: smoother right-hand side
    void* tw = nullptr;            // FFT twiddles: M = N/2 (DCT/DST) or N (periodic) values
    void* twP = nullptr;           // DCT post/pre-processing twiddles (M/2 + 1)
    double* ev = nullptr;          // 1D eigenvalues of -Lap_h in the transform's index order
    double smin = 0.0;             // smallest 2D eigenvalue of -Lap_h
    int threads = 256, RT = 1, RC = 1, lds = 0;
    size_t sm_fwd = 0, sm_col = 0, sm_inv = 0;
    long long launches = 0;
};

namespace {

using ccm::cplx;
using ccm::PostTw;
namespace ss = ccm::ss;

// Launch geometry and tables of one solver (precision T).
template <typename T> int setup(ccmsav_solver* s) {
    const int N = s->N;
    const double h = s->L / N;
    const bool per = s->bc == CCMSAV_BC_PERIODIC;
    const int M = per ? N : N / 2;                     // complex line length
    const size_t NN = (size_t)N * N;
    const ss::Geo g = ss::geometry<T>(N, per);
    s->threads = g.threads; s->RT = g.RT; s->RC = g.RC; s->lds = g.lds;
    s->sm_fwd = g.sm_fwd; s->sm_col = g.sm_col; s->sm_inv = g.sm_inv;
    if (const int r = ss::optin_all<T>(g, per)) return r;
    // tables, computed on the host in FP64 and rounded to T
    std::vector<cplx<T>> hw(M);
    for (int t = 0; t < M; ++t) {
        const double a = 2.0 * M_PI * t / M;
        hw[t].x = (T)std::cos(a); hw[t].y = (T)(-std::sin(a));
    }
    std::vector<double> he(N);
    for (int k = 0; k < N; ++k) {
        const double a = per ? M_PI * k / N : M_PI * k / (2.0 * N);
        const double t = s->bc == CCMSAV_BC_DIRICHLET ? std::cos(a) : std::sin(a);
        he[k] = 4.0 * t * t / (h * h);
    }
    s->smin = 2.0 * (s->bc == CCMSAV_BC_DIRICHLET ? he[N - 1] : 0.0);
    if (cudaMalloc(&s->tw, M * sizeof(cplx<T>)) != cudaSuccess) return CCMSAV_ENOMEM;
    if (cudaMalloc(&s->ev, N * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
    if (cudaMalloc(&s->scratch, NN * (per ? sizeof(cplx<T>) : sizeof(T))) != cudaSuccess) return CCMSAV_ENOMEM;
    if (cudaMalloc(&s->rhs, NN * sizeof(T)) != cudaSuccess) return CCMSAV_ENOMEM;
    if (cudaMemcpyAsync(s->tw, hw.data(), M * sizeof(cplx<T>), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
        cudaMemcpyAsync(s->ev, he.data(), N * sizeof(double), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
        return CCMSAV_ECUDA;
    if (!per) {
        std::vector<PostTw<T>> hp(M / 2 + 1);
        for (int k = 0; k <= M / 2; ++k) {
            const double a = 2.0 * M_PI * k / N, b = M_PI * k / (2.0 * N);
            hp[k].cN = (T)std::cos(a); hp[k].sN = (T)std::sin(a);
            hp[k].c4 = (T)std::cos(b); hp[k].s4 = (T)std::sin(b);
        }
        if (cudaMalloc(&s->twP, (M / 2 + 1) * sizeof(PostTw<T>)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMemcpyAsync(s->twP, hp.data(), (M / 2 + 1) * sizeof(PostTw<T>), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
            return CCMSAV_ECUDA;
    }
    return cudaStreamSynchronize(s->st) == cudaSuccess ? CCMSAV_OK : CCMSAV_ECUDA;
}

template <typename T> int solve(ccmsav_solver* s, const double c[3], const T* f, T* u) {
    const int N = s->N;
    const dim3 b(s->threads);
    const cplx<T>* tw = static_cast<const cplx<T>*>(s->tw);
    if (s->bc == CCMSAV_BC_PERIODIC) {
        cplx<T>* sc = static_cast<cplx<T>*>(s->scratch);
        ss::k_ss_row_fwd_p<T><<<N / s->RT, b, s->sm_fwd, s->st>>>(f, sc, N, s->RT, tw);
        ss::k_ss_col_solve_p<T><<<N / s->RC, b, s->sm_col, s->st>>>(sc, N, s->RC, tw, s->ev, c[0], c[1], c[2]);
        ss::k_ss_row_inv_p<T><<<N / s->RT, b, s->sm_inv, s->st>>>(sc, u, N, s->RT, tw);
    } else {
        T* sc = static_cast<T*>(s->scratch);
        const PostTw<T>* tp = static_cast<const PostTw<T>*>(s->twP);
        if (s->bc == CCMSAV_BC_DIRICHLET)
            ss::k_ss_row_fwd<T, true><<<N / s->RT, b, s->sm_fwd, s->st>>>(f, sc, N, s->RT, s->lds, tw, tp, nullptr, 0);
        else
            ss::k_ss_row_fwd<T, false><<<N / s->RT, b, s->sm_fwd, s->st>>>(f, sc, N, s->RT, s->lds, tw, tp, nullptr, 0);
        ss::k_ss_col_solve<T><<<N / s->RC, b, s->sm_col, s->st>>>(sc, N, s->RC, tw, tp, s->ev, c[0], c[1], c[2],
                                                                   nullptr, nullptr, 0);
        if (s->bc == CCMSAV_BC_DIRICHLET)
            ss::k_ss_row_inv<T, true><<<N / s->RT, b, s->sm_inv, s->st>>>(sc, u, N, s->RT, s->lds, tw, tp, nullptr, 0);
        else
            ss::k_ss_row_inv<T, false><<<N / s->RT, b, s->sm_inv, s->st>>>(sc, u, N, s->RT, s->lds, tw, tp, nullptr, 0);
    }
    s->launches += 3;
    return cudaPeekAtLastError() == cudaSuccess ? CCMSAV_OK : CCMSAV_ECUDA;
}

template <typename T> int smooth(ccmsav_solver* s, double eps, double mob, double dt, int nsteps, T* phi) {
    const int N = s->N;
    const double h = s->L / N;
    const double c[3] = {1.0 / dt, 0.0, mob * eps};      // (1/dt + Mob eps Lap^2) phi^{n+1} = r
    T* r = static_cast<T*>(s->rhs);
    const int nb = (int)(((size_t)N * N + 255) / 256 < 4096 ? ((size_t)N * N + 255) / 256 : 4096);
    for (int n = 0; n < nsteps; ++n) {
        ss::k_smooth_rhs<T><<<nb, 256, 0, s->st>>>(phi, r, N, s->bc, 1.0 / dt, mob / (h * h), 1.0 / eps);
        ++s->launches;
        int e = solve<T>(s, c, r, phi);
        if (e) return e;
    }
    ss::k_clamp<T><<<nb, 256, 0, s->st>>>(phi, (size_t)N * N);
    ++s->launches;
    return cudaPeekAtLastError() == cudaSuccess ? CCMSAV_OK : CCMSAV_ECUDA;
}

void release(ccmsav_solver* s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    cudaFree(s->scratch); cudaFree(s->rhs); cudaFree(s->tw); cudaFree(s->twP); cudaFree(s->ev);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
}

}  // namespace

extern "C" int ccmsav_solver_create(ccmsav_solver_t** out, int N, double L, int bc, int precision, void* stream) {
    if (!out) return CCMSAV_EINVAL;
    *out = nullptr;
    if (N < 8 || N > 8192 || (N & (N - 1))) return CCMSAV_EINVAL;
    if (!(std::isfinite(L) && L > 0.0)) return CCMSAV_EINVAL;
    if (bc != CCMSAV_BC_NEUMANN && bc != CCMSAV_BC_DIRICHLET && bc != CCMSAV_BC_PERIODIC) return CCMSAV_EINVAL;
    if (precision != CCMSAV_FP64 && precision != CCMSAV_FP32_BULK) return CCMSAV_EINVAL;
    ccmsav_solver* s = new (std::nothrow) ccmsav_solver();
    if (!s) return CCMSAV_ENOMEM;
    s->N = N; s->L = L; s->bc = bc; s->precision = precision;
    s->st = (cudaStream_t)stream;
    if (!s->st) {
        if (cudaStreamCreate(&s->st) != cudaSuccess) { delete s; return CCMSAV_ECUDA; }
        s->own_stream = true;
    }
    const int r = precision == CCMSAV_FP64 ? setup<double>(s) : setup<float>(s);
    if (r != CCMSAV_OK) { release(s); return r; }
    *out = s;
    return CCMSAV_OK;
}

extern "C" int ccmsav_solver_solve(ccmsav_solver_t* s, const double coef[3], const void* f, void* u) {
    if (!s || !coef || !f || !u) return CCMSAV_EINVAL;
    for (int i = 0; i < 3; ++i) if (!std::isfinite(coef[i])) return CCMSAV_EINVAL;
    if (coef[1] < 0.0 || coef[2] < 0.0) return CCMSAV_EINVAL;
    if (!(coef[0] + s->smin * (coef[1] + coef[2] * s->smin) > 0.0)) return CCMSAV_EINVAL;
    return s->precision == CCMSAV_FP64
               ? solve<double>(s, coef, static_cast<const double*>(f), static_cast<double*>(u))
               : solve<float>(s, coef, static_cast<const float*>(f), static_cast<float*>(u));
}

extern "C" int ccmsav_solver_smooth(ccmsav_solver_t* s, double eps, double mobility, double dt, int nsteps, void* phi) {
    if (!s || !phi || nsteps < 0) return CCMSAV_EINVAL;
    if (!(std::isfinite(eps) && eps > 0.0 && std::isfinite(mobility) && mobility >= 0.0 && std::isfinite(dt) && dt > 0.0))
        return CCMSAV_EINVAL;
    return s->precision == CCMSAV_FP64 ? smooth<double>(s, eps, mobility, dt, nsteps, static_cast<double*>(phi))
                                       : smooth<float>(s, eps, mobility, dt, nsteps, static_cast<float*>(phi));
}

extern "C" int ccmsav_solver_sync(ccmsav_solver_t* s) {
    if (!s) return CCMSAV_EINVAL;
    return cudaStreamSynchronize(s->st) == cudaSuccess ? CCMSAV_OK : CCMSAV_ECUDA;
}

extern "C" long long ccmsav_solver_launch_count(ccmsav_solver_t* s) { return s ? s->launches : 0; }

extern "C" void ccmsav_solver_destroy(ccmsav_solver_t* s) { release(s); }
