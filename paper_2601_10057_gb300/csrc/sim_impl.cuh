// sim_impl.cuh -- host orchestration of one simulation in precision T.
//
// Device memory per simulation (T = field precision):
//   phi[3], psi[3]   three time levels in rotation (n+1 is written into the
//                    spare level, so n-1 stays readable for the optional
//                    lambda-sum reduction)
//   bufA             8 N x N fields: stencil outputs, later the spectra
//   bufB             8 N x N fields: row-transformed (transposed) fields,
//                    later the two inverse-column-transformed fields
//   part1/part2      FP64 per-block partial sums of the stencil and Gram
//                    reductions (reduced in a fixed order by k_solve)
//   twM, twP, ev     FFT twiddles, DCT pre/post twiddles and the 1D Laplacian
//                    eigenvalues 4 sin^2(pi k / 2N) / h^2 (computed on the host
//                    in FP64)
//   sc               DevScalars (SAVs, recovery coefficients, status)
#pragma once
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstddef>
#include <vector>
#include "sim.h"
#include "diag_kernels.cuh"
#include "warp_kernels.cuh"
#include "spectral_kernels.cuh"
#include "classical_kernels.cuh"
#include <type_traits>
#include <map>
#include <mutex>

namespace ccm {

template <typename T> struct TuneTable {
    static std::mutex& mu() { static std::mutex m; return m; }
    static std::map<int, TuneChoice>& table() { static std::map<int, TuneChoice> t; return t; }
};

#define CCM_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return CCMSAV_ECUDA;     \
    } while (0)

static inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
static const size_t kSmemMax = 227 * 1024;

template <typename T>
class SimImpl : public SimBase {
public:
    ccmsav_params p{};
    int flags = 0;
    cudaStream_t st = nullptr;
    int M = 0;
    size_t NN = 0;
    T* phi[3] = {nullptr, nullptr, nullptr};
    T* psi[3] = {nullptr, nullptr, nullptr};
    int cur = 0, prev = 1, spare = 2;
    T* bufA = nullptr;
    T* bufB = nullptr;
    double* part1 = nullptr;
    double* part2 = nullptr;
    double* partd = nullptr;
    double* part3 = nullptr;         // k_solve slices (kSolveBlocks x NRQ)
    cplx<T>* twM = nullptr;
    PostTw<T>* twP = nullptr;
    double* ev = nullptr;
    DevScalars* sc = nullptr;
    // FP32 warp-FFT path (N = 128 .. 2048): twiddle matrix W_M^{n2 k1} and FP32 eigenvalues
    bool warp_path = false;
    cplx<float>* tw2 = nullptr;
    cplx<float>* tw2i = nullptr;   // table of the inverse kernels' variant line shape (or tw2)
    float* evf = nullptr;
    float4* evp = nullptr;   // eigenvalues in the pair order of the warp-path spectra
    float4* twF = nullptr;       // forward / inverse pair twiddles of the warp path
    float4* twI = nullptr;       // (wn, a) per pair; b of pair 0 in twF0 / twI0
    float2 twF0{}, twI0{};
    wf::PairTwTab pair_tab(const float4* t) const { return wf::PairTwTab{t, t == twF ? twF0 : twI0}; }
    int wRT = 8, wlds = 0, wRT4 = 4, wlds4 = 0, wKC = 1, wRI = 4;
    int ahead_rt = 0;   // L2 prefetch distance of the row kernel (0: none)
    size_t wsm_rt = 0, wsm_col = 0, wsm_comb = 0, wsm_irow = 0;
    DevScalars* sc_host = nullptr;   // pinned
    double* h_part = nullptr;        // pinned, diag partial rows
    void* tmp64 = nullptr;           // FP64 staging for host I/O
    static constexpr int kUpBlocks = 1024;   // blocks of the upload kernels
    unsigned* d_upbad = nullptr;     // upload: non-finite flag, then 2 kUpBlocks partial sums
    double* h_up = nullptr;          // pinned mirror of the same
    bool have_state = false, poisoned = false;
    long long steps_taken = 0;
    long long nlaunch = 0;
    // launch geometry
    dim3 g_st, b_st;
    int nb1 = 0;
    int RT = 1, lds_rt = 0; size_t sm_rt = 0;
    int FG = 8; size_t sm_col = 0;
    int RT4 = 1, lds_c = 0; size_t sm_comb = 0;
    int PR = 1; size_t sm_irow = 0;
    dim3 g_dg;
    int nbd = 0;
    // CUDA graphs of three BDF2 steps, one per phase of the three-level rotation
    cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t gexec1[3] = {nullptr, nullptr, nullptr};   // one BDF2 step per phase
    bool own_stream = false;
    bool graphs_failed = false;
    // tracing: event marks between the kernels of traced steps
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;        // kernel slot of the interval that ends at this mark (-1: step start)
    size_t ev_used = 0;
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long prof_steps = 0;
    // classical MSAV (CCMSAV_CLASSICAL): conjugate-gradient Cahn-Hilliard solves
    bool classical = false;
    T* cl = nullptr;                 // Mx My b1 (1 field each), x r p zq scratch (2 fields each)
    PcgScalars* pcg = nullptr;
    PcgScalars* pcg_host = nullptr;  // pinned
    double* cl_red = nullptr;        // per-block partial sums
    int cl_nb = 0;
    ss::Geo cl_geo;
    double pcg_rtol = 1e-10;
    int pcg_max_it = 200;
    double pcg_last[3] = {0, 0, 0};  // iterations, residuals of the last step
    long long pcg_total = 0;

    ~SimImpl() override {
        if (st) cudaStreamSynchronize(st); else cudaDeviceSynchronize();
        cudaFree(tune_snap);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        for (int i = 0; i < 3; ++i) if (gexec[i]) cudaGraphExecDestroy(gexec[i]);
        for (int i = 0; i < 3; ++i) if (gexec1[i]) cudaGraphExecDestroy(gexec1[i]);
        release();
        if (own_stream && st) cudaStreamDestroy(st);
    }

    // Three consecutive steps as direct launches on st while the stream is
    // being captured: nothing executes, so the host counters are restored
    // (three steps rotate the three levels back to the same phase).
    int queue_steps_captured(int n3) override {
        if (n3 != 3) return CCMSAV_EINVAL;
        const long long s0 = steps_taken, l0 = nlaunch;
        int r = CCMSAV_OK;
        for (int i = 0; i < 3 && r == CCMSAV_OK; ++i) r = queue_one_step();
        steps_taken = s0; nlaunch = l0;
        return r;
    }

    long long launches_per_step() const { return 6 + ((flags & CCMSAV_TRACK_ENERGY) ? 2 : 0); }

    void count_steps(int n3) override { steps_taken += n3; nlaunch += n3 * launches_per_step(); }
    void count_steps_grouped(int n3) override { steps_taken += n3; }

    // ---- grouped launches -------------------------------------------------
    // FP32 warp path with one warp or less per line (N <= 2048), BDF2 steps (not
    // CCMSAV_BDF1_ALWAYS), no classical mode, no energy tracking: simulations of
    // the same M share each kernel launch.
    int group_key() const override {
        if constexpr (std::is_same<T, float>::value)
            if (warp_path && !classical && !(flags & (CCMSAV_TRACK_ENERGY | CCMSAV_BDF1_ALWAYS)) && M >= 64 && M <= 1024)
                return M;
        return 0;
    }
    size_t batch_args_bytes() const override { return sizeof(BatchArgs); }
    int fill_batch_args(int i, void* rec) const override {
        if constexpr (std::is_same<T, float>::value) {
            if (i < 0 || i > 2 || !rec) return CCMSAV_EINVAL;
            int c0 = cur, p0 = prev, s0 = spare;
            for (int k = 0; k < i; ++k) { const int nw = s0; s0 = p0; p0 = c0; c0 = nw; }
            StencilCoef<float> c;
            SpecCoef sp;
            SolveCoef so;
            step_coefs(false, c, sp, so);
            so.anchor = 1;
            so.nb2 = N / wKC;
            BatchArgs a;
            a.phn = phi[c0]; a.pho = phi[p0]; a.psn = psi[c0]; a.pso = psi[p0];
            a.phi_new = phi[s0]; a.psi_new = psi[s0];
            a.bufA = reinterpret_cast<float*>(bufA); a.bufB = reinterpret_cast<float*>(bufB);
            a.part1 = part1; a.part2 = part2; a.part3 = part3; a.sc = sc;
            a.tw2 = tw2; a.twF = pair_tab(twF); a.twI = pair_tab(twI); a.evf = evf; a.evp = evp;
            a.c = c;
            a.sf = SpecCoefF{(float)sp.C1, (float)sp.C2, (float)sp.C3, (float)sp.Ct, (float)sp.lam};
            a.so = so;
            std::memcpy(rec, &a, sizeof a);
            return CCMSAV_OK;
        }
        return CCMSAV_EINVAL;
    }
    int max_group() const override { return kMaxGroup; }
    template <int MM> void group_launch(const GroupArgs<true>& ga, int n, cudaStream_t s) {
        const int bst = g_st.x, brt = N / wRT, bcol = N / wKC, bcomb = N / wRT4;
        const int birow = (2 * N + InvGeo<MM>::LINES - 1) / InvGeo<MM>::LINES;
        k_stencil<float, true><<<dim3(bst * n, g_st.y), b_st, stencil_smem_bytes<float>(), s>>>(
            nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, N, StencilCoef<float>{}, ga, bst);
        kw_rowdct_T<MM, true><<<dim3(brt * n, NF), kWarps * 32, wsm_rt, s>>>(nullptr, nullptr, nullptr, wf::PairTwTab{}, 0,
                                                                         ga, brt);
        kw_coldct_gram<MM, true><<<bcol * n, kWarps * 32, wsm_col, s>>>(nullptr, nullptr, nullptr, nullptr, wf::PairTwTab{},
                                                                       nullptr, nullptr, SpecCoefF{}, ga, bcol);
        k_solve<float2, true><<<kSolveBlocks * n, kSolveThreads, 0, s>>>(nullptr, 0, nullptr, 0, nullptr, nullptr,
                                                                         SolveCoef{}, ga, kSolveBlocks);
        kw_comb_icolT<MM, true><<<bcomb * n, comb_warps<MM>() * 32, wsm_comb, s>>>(nullptr, nullptr, nullptr, wf::PairTwTab{},
                                                                        nullptr, nullptr, SpecCoefF{}, nullptr, 1, ga, bcomb);
        kw_irow<MM, true><<<birow * n, InvGeo<MM>::WARPS * 32, wsm_irow, s>>>(nullptr, nullptr, nullptr, nullptr,
            wf::PairTwTab{}, nullptr, nullptr, nullptr, nullptr, 0, nullptr, 1, ga, birow);
    }
    // recs: host records, three blocks of `stride` (one per step), of which
    // this group's n are at the start of each block; copied into the launch
    // parameters (so a stream capture keeps them with the graph)
    int queue_group_steps(const void* recs, int n, int stride, cudaStream_t s) override {
        if constexpr (std::is_same<T, float>::value) {
            if (!recs || n < 2 || n > kMaxGroup || stride < n || group_key() == 0) return CCMSAV_EINVAL;
            std::vector<GroupArgs<true>> ga(1);
            for (int i = 0; i < 3; ++i) {
                std::memcpy(ga[0].a, static_cast<const unsigned char*>(recs) + (size_t)i * stride * sizeof(BatchArgs),
                            (size_t)n * sizeof(BatchArgs));
                switch (M) {
                    case 64: group_launch<64>(ga[0], n, s); break;
                    case 128: group_launch<128>(ga[0], n, s); break;
                    case 256: group_launch<256>(ga[0], n, s); break;
                    case 512: group_launch<512>(ga[0], n, s); break;
                    case 1024: group_launch<1024>(ga[0], n, s); break;
                    default: return CCMSAV_EINVAL;
                }
            }
            CCM_CUDA(cudaGetLastError());
            return CCMSAV_OK;
        }
        return CCMSAV_EINVAL;
    }
    cudaStream_t stream() const override { return st; }
    int phase() const override { return cur; }
    bool batchable() const override { return have_state && !poisoned && steps_taken > 0 && !prof && !classical; }

    // Captures three consecutive BDF2 steps starting at the current rotation
    // phase into this simulation's graph for that phase.
    int capture_phase() {
        const int ph = cur;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCMSAV_ECUDA;
        const int r = queue_steps_captured(3);
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (r != CCMSAV_OK || e != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); return CCMSAV_ECUDA; }
        const cudaError_t e2 = cudaGraphInstantiate(&gexec[ph], g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) { gexec[ph] = nullptr; return CCMSAV_ECUDA; }
        return CCMSAV_OK;
    }

    // One BDF2 step from the current phase into gexec1[phase] (nothing
    // executes while capturing: counters and the level rotation are restored).
    int capture_single() {
        const int ph = cur, c0 = cur, p0 = prev, s0r = spare;
        const long long s0 = steps_taken, l0 = nlaunch;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCMSAV_ECUDA;
        const int r = queue_one_step();
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        steps_taken = s0; nlaunch = l0; cur = c0; prev = p0; spare = s0r;
        if (r != CCMSAV_OK || e != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); return CCMSAV_ECUDA; }
        const cudaError_t e2 = cudaGraphInstantiate(&gexec1[ph], g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) { gexec1[ph] = nullptr; return CCMSAV_ECUDA; }
        return CCMSAV_OK;
    }

    int mark(int kind) {
        if (!prof) return CCMSAV_OK;
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e;
            CCM_CUDA(cudaEventCreate(&e));
            ev_pool.push_back(e);
            ev_kind.push_back(kind);
        }
        ev_kind[ev_used] = kind;
        CCM_CUDA(cudaEventRecord(ev_pool[ev_used], st));
        ++ev_used;
        return CCMSAV_OK;
    }

    int profile_flush() {
        if (ev_used == 0) return CCMSAV_OK;
        CCM_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 1; i < ev_used; ++i) {
            if (ev_kind[i] < 0) continue;
            float ms = 0.f;
            CCM_CUDA(cudaEventElapsedTime(&ms, ev_pool[i - 1], ev_pool[i]));
            prof_ms[ev_kind[i]] += ms;
        }
        ev_used = 0;
        return CCMSAV_OK;
    }

    int profile(bool enable) override {
        int r = profile_flush();
        prof = enable;
        return r;
    }

    int profile_read(double ms[8], long long* nsteps) override {
        int r = profile_flush();
        for (int i = 0; i < 8; ++i) { ms[i] = prof_ms[i]; prof_ms[i] = 0; }
        *nsteps = prof_steps;
        prof_steps = 0;
        return r;
    }

    void release() {
        for (int i = 0; i < 3; ++i) { cudaFree(phi[i]); cudaFree(psi[i]); phi[i] = psi[i] = nullptr; }
        cudaFree(bufA); cudaFree(bufB); cudaFree(part1); cudaFree(part2); cudaFree(partd); cudaFree(part3);
        cudaFree(twM); cudaFree(twP); cudaFree(ev); cudaFree(sc); cudaFree(tmp64);
        if (tw2i && tw2i != tw2) cudaFree(tw2i);
        cudaFree(tw2); cudaFree(evf); cudaFree(evp); cudaFree(twF); cudaFree(twI);
        cudaFree(cl); cudaFree(pcg); cudaFree(cl_red);
        if (pcg_host) cudaFreeHost(pcg_host);
        cl = nullptr; pcg = nullptr; cl_red = nullptr; pcg_host = nullptr;
        tw2 = nullptr; tw2i = nullptr; evf = nullptr; evp = nullptr; twF = nullptr; twI = nullptr;
        if (sc_host) cudaFreeHost(sc_host);
        if (h_part) cudaFreeHost(h_part);
        if (h_up) cudaFreeHost(h_up);
        cudaFree(d_upbad);
        h_up = nullptr; d_upbad = nullptr;
        bufA = bufB = nullptr; part1 = part2 = partd = part3 = nullptr; twM = nullptr; twP = nullptr;
        ev = nullptr; sc = nullptr; tmp64 = nullptr; sc_host = nullptr; h_part = nullptr;
    }

    // max_carveout: take the whole unified L1 as shared memory (kernels whose
    // occupancy is set by their tiles; the others keep L1 for cached loads)
    // carveout: preferred shared-memory share of the unified L1 in percent
    // (-1: the driver's choice; 100: all of it)
    static int set_smem_limit(const void* fn, size_t needed, int carveout = -1) {
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 1;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 1;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 1;
        const int lim = optin - (int)fa.sharedSizeBytes;
        if ((size_t)lim < needed) return 1;
        if (carveout >= 0 && cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carveout) != cudaSuccess)
            return 1;
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess;
    }

    static int lines_per_batch(int M_) { int E = M_ < 8 ? M_ : 8; return 512 / (M_ / E); }

    int init(const ccmsav_params& pp, int N_, int flags_, cudaStream_t s) {
        p = pp; N = N_; flags = flags_; st = s;
        if (!st) {
            // NULL: a stream owned by the handle; it is a blocking stream, so it
            // stays ordered with work on the legacy default stream
            if (cudaStreamCreate(&st) != cudaSuccess) return CCMSAV_ECUDA;
            own_stream = true;
        }
        M = N / 2; NN = (size_t)N * N;
        const size_t fb = NN * sizeof(T);
        for (int i = 0; i < 3; ++i) {
            if (cudaMalloc(&phi[i], fb) != cudaSuccess) return CCMSAV_ENOMEM;
            if (cudaMalloc(&psi[i], fb) != cudaSuccess) return CCMSAV_ENOMEM;
        }
        if (cudaMalloc(&bufA, 8 * fb) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&bufB, 8 * fb) != cudaSuccess) return CCMSAV_ENOMEM;
        b_st = dim3(TX, TY);
        g_st = dim3((N + TX - 1) / TX, (N + TYB - 1) / TYB);
        nb1 = g_st.x * g_st.y;
        g_dg = dim3((N + 31) / 32, (N + 8 * kDiagRows - 1) / (8 * kDiagRows));
        nbd = g_dg.x * g_dg.y;
        if (cudaMalloc(&part1, (size_t)nb1 * NRED1 * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&part2, (size_t)N * NRED2 * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&partd, (size_t)nbd * NDIAG * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&part3, (size_t)kSolveBlocks * NRQ * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&tmp64, 2 * NN * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&d_upbad, (1 + 2 * kUpBlocks) * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaHostAlloc(&h_up, (1 + 2 * kUpBlocks) * sizeof(double), cudaHostAllocDefault) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&sc, sizeof(DevScalars)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaHostAlloc(&sc_host, sizeof(DevScalars), cudaHostAllocDefault) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaHostAlloc(&h_part, (size_t)nbd * NDIAG * sizeof(double), cudaHostAllocDefault) != cudaSuccess) return CCMSAV_ENOMEM;
        std::memset(sc_host, 0, sizeof(DevScalars));
        CCM_CUDA(cudaMemcpyAsync(sc, sc_host, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
        // tables (FP64 on the host, rounded to T)
        std::vector<cplx<T>> hM(M);
        for (int t = 0; t < M; ++t) {
            const double a = 2.0 * M_PI * t / M;
            hM[t].x = (T)std::cos(a); hM[t].y = (T)(-std::sin(a));
        }
        std::vector<PostTw<T>> hP(M / 2 + 1);
        for (int k = 0; k <= M / 2; ++k) {
            const double a = 2.0 * M_PI * k / N, b = M_PI * k / (2.0 * N);
            hP[k].cN = (T)std::cos(a); hP[k].sN = (T)std::sin(a);
            hP[k].c4 = (T)std::cos(b); hP[k].s4 = (T)std::sin(b);
        }
        std::vector<double> hE(N);
        const double h = p.L / N;
        for (int k = 0; k < N; ++k) { const double s = std::sin(M_PI * k / (2.0 * N)); hE[k] = 4.0 * s * s / (h * h); }
        if (cudaMalloc(&twM, M * sizeof(cplx<T>)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&twP, (M / 2 + 1) * sizeof(PostTw<T>)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&ev, N * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        CCM_CUDA(cudaMemcpyAsync(twM, hM.data(), M * sizeof(cplx<T>), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(twP, hP.data(), (M / 2 + 1) * sizeof(PostTw<T>), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(ev, hE.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
        // DCT kernel geometry
        const int P = lines_per_batch(M);
        const size_t ldc = padded_len(M);
        const size_t lsz = ldc * sizeof(cplx<T>);
        RT = (int)std::min<size_t>(64 / sizeof(T), std::max<size_t>(1, 131072 / (N * sizeof(T))));
        if (RT > N) RT = N;
        lds_rt = N + 1;
        sm_rt = align16((size_t)RT * lds_rt * sizeof(T)) + (size_t)std::min(P, RT) * lsz;
        FG = 8;
        while (FG > 1 && (size_t)FG * lsz + 16 * NRED2 * sizeof(double) > kSmemMax) FG /= 2;
        sm_col = (size_t)FG * lsz;
        RT4 = (int)std::max<size_t>(1, std::min<size_t>(64 / sizeof(T), 65536 / (N * sizeof(T))));
        if (RT4 > N) RT4 = N;
        lds_c = N + 1;
        sm_comb = align16((size_t)2 * RT4 * lds_c * sizeof(T)) + (size_t)std::min(P, 2 * RT4) * lsz;
        PR = std::max(1, std::min(4, N / 8));
        sm_irow = (size_t)std::min(P, 2 * PR) * lsz;
        if (sm_rt > kSmemMax || sm_col > kSmemMax || sm_comb > kSmemMax || sm_irow > kSmemMax) return CCMSAV_EINVAL;
        // opt in to the largest dynamic shared memory each kernel can take (the
        // per-block opt-in limit minus the kernel's static shared memory); the
        // attribute is per kernel, so it must not depend on this simulation's N
        // FP32: 72 % of 228 KB, rounded up by the driver to the 196 KB
        // configuration: three 55.5 KB tiles per SM (the low part of phi_bar
        // is a second two-halo tile) and 60 KB of L1 for the halo re-reads
        // (faster than four tiles at 228 KB with a 28 KB L1); FP64 tiles are
        // twice the size of the FP32 ones without the low part
        if (set_smem_limit((const void*)k_stencil<T>, stencil_smem_bytes<T>(), std::is_same<T, float>::value ? 72 : 100))
            return CCMSAV_ECUDA;
        if constexpr (std::is_same<T, float>::value)
            if (set_smem_limit((const void*)k_stencil<float, true>, stencil_smem_bytes<float>(), 72))
                return CCMSAV_ECUDA;
        if (set_smem_limit((const void*)k_rowdct_T<T>, sm_rt) || set_smem_limit((const void*)k_coldct_gram<T>, sm_col) ||
            set_smem_limit((const void*)k_comb_icolT<T>, sm_comb) || set_smem_limit((const void*)k_irow<T>, sm_irow))
            return CCMSAV_ECUDA;
        if (flags & CCMSAV_CLASSICAL) {
            int r = init_classical();
            if (r) return r;
        }
        const char* force_block = std::getenv("CCMSAV_FORCE_BLOCK_FFT");   // test switch: block-FFT kernels only
        if (std::is_same<T, float>::value && M >= 64 && M <= 4096 && !(force_block && force_block[0] == '1')) {
            int r = init_warp_path();
            if (r) return r;
        }
        CCM_CUDA(cudaStreamSynchronize(st));
        return CCMSAV_OK;
    }

    int init_classical() {
        classical = true;
        graphs_failed = true;            // the host reads convergence flags inside a step
        pcg_rtol = std::is_same<T, float>::value ? 1e-6 : 1e-10;
        if (cudaMalloc(&cl, 13 * NN * sizeof(T)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&pcg, sizeof(PcgScalars)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaHostAlloc(&pcg_host, sizeof(PcgScalars), cudaHostAllocDefault) != cudaSuccess) return CCMSAV_ENOMEM;
        CCM_CUDA(cudaMemsetAsync(pcg, 0, sizeof(PcgScalars), st));
        const size_t nbw = (NN + kClThreads - 1) / kClThreads;
        cl_nb = (int)(nbw < 1216 ? nbw : 1216);
        if (cudaMalloc(&cl_red, (size_t)cl_nb * 2 * sizeof(double)) != cudaSuccess) return CCMSAV_ENOMEM;
        cl_geo = ss::geometry<T>(N, false);
        if (cl_geo.sm_fwd > kSmemMax || cl_geo.sm_col > kSmemMax || cl_geo.sm_inv > kSmemMax) return CCMSAV_EINVAL;
        if (ss::optin_all<T>(cl_geo, false)) return CCMSAV_ECUDA;
        return CCMSAV_OK;
    }

    // z = M^{-1} r for both systems (DCT solve of a - lam Mbar Lap_h with the
    // coefficients on the device); converged systems are skipped.
    void cl_precond(const T* r, T* z, T* scr) {
        const dim3 g1(N / cl_geo.RT, 2), g2(N / cl_geo.RC, 2), b(cl_geo.threads);
        // device addresses of the convergence flags and the coefficients
        const int* conv = reinterpret_cast<const int*>(reinterpret_cast<const char*>(pcg) + offsetof(PcgScalars, conv));
        const double* coef = reinterpret_cast<const double*>(reinterpret_cast<const char*>(pcg) + offsetof(PcgScalars, coef));
        ss::k_ss_row_fwd<T, false><<<g1, b, cl_geo.sm_fwd, st>>>(r, scr, N, cl_geo.RT, cl_geo.lds, twM, twP, conv, NN);
        ss::k_ss_col_solve<T><<<g2, b, cl_geo.sm_col, st>>>(scr, N, cl_geo.RC, twM, twP, ev, 0.0, 0.0, 0.0,
                                                           coef, conv, NN);
        ss::k_ss_row_inv<T, false><<<g1, b, cl_geo.sm_inv, st>>>(scr, z, N, cl_geo.RT, cl_geo.lds, twM, twP, conv, NN);
        nlaunch += 3;
    }

    // The classical scheme's two Cahn-Hilliard solves y1 = zeta_c^{-1} g0c and
    // y2 = zeta_c^{-1} LP by preconditioned CG, then (P, y1) and (P, y2).
    // Reads the stencil's P and LP (bufA fields 5 and 7) before the column
    // transforms overwrite bufA.
    int queue_classical_ch(bool bdf1) {
        T* Mx = cl;
        T* My = cl + NN;
        T* b1 = cl + 2 * NN;
        T* x = cl + 3 * NN;
        T* r = cl + 5 * NN;
        T* pv = cl + 7 * NN;
        T* zq = cl + 9 * NN;
        T* scr = cl + 11 * NN;
        const double a = bdf1 ? 1.0 / p.dt : 1.5 / p.dt;
        const double h2i = 1.0 / (h() * h());
        k_cl_prep<T><<<cl_nb, kClThreads, 0, st>>>(phi[cur], phi[prev], psi[cur], psi[prev], bdf1 ? 1 : 0, Mx, My, b1,
                                                   cl_red, pcg, N, a, p.lam, p.M0, h2i, pcg_rtol);
        k_cl_init<T><<<cl_nb, kClThreads, 0, st>>>(b1, bufA + 7 * NN, x, r, pv, cl_red, pcg, NN);
        nlaunch += 2;
        cl_precond(r, zq, scr);
        k_cl_dot_rz<T><<<cl_nb, kClThreads, 0, st>>>(r, zq, cl_red, pcg, NN, 1);
        k_cl_pupdate<T><<<cl_nb, kClThreads, 0, st>>>(zq, pv, pcg, NN);
        nlaunch += 2;
        for (int it = 1; it <= pcg_max_it; ++it) {
            k_cl_apply<T><<<cl_nb, kClThreads, 0, st>>>(pv, Mx, My, zq, cl_red, pcg, N, a, p.lam * h2i);
            k_cl_update<T><<<cl_nb, kClThreads, 0, st>>>(x, r, pv, zq, cl_red, pcg, NN);
            nlaunch += 2;
            cl_precond(r, zq, scr);
            k_cl_dot_rz<T><<<cl_nb, kClThreads, 0, st>>>(r, zq, cl_red, pcg, NN, 0);
            k_cl_pupdate<T><<<cl_nb, kClThreads, 0, st>>>(zq, pv, pcg, NN);
            nlaunch += 2;
            if (it % 4 == 0 || it == pcg_max_it) {
                CCM_CUDA(cudaGetLastError());
                CCM_CUDA(cudaMemcpyAsync(pcg_host, pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
                CCM_CUDA(cudaStreamSynchronize(st));
                if (pcg_host->conv[0] && pcg_host->conv[1]) break;
            }
        }
        k_cl_pdot<T><<<cl_nb, kClThreads, 0, st>>>(bufA + 5 * NN, x, cl_red, pcg, NN);
        ++nlaunch;
        CCM_CUDA(cudaGetLastError());
        CCM_CUDA(cudaMemcpyAsync(pcg_host, pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        const int itmax = pcg_host->iters[0] > pcg_host->iters[1] ? pcg_host->iters[0] : pcg_host->iters[1];
        pcg_last[0] = itmax;
        for (int s = 0; s < 2; ++s)
            pcg_last[1 + s] = pcg_host->rr0[s] > 0 ? std::sqrt(pcg_host->rr[s] / pcg_host->rr0[s]) : 0.0;
        pcg_total += itmax;
        return CCMSAV_OK;
    }

    int set_pcg(double rtol, int max_iter) override {
        if (!classical) return CCMSAV_EINVAL;
        if (!(std::isfinite(rtol) && rtol > 0.0) || max_iter < 1) return CCMSAV_EINVAL;
        pcg_rtol = rtol;
        pcg_max_it = max_iter;
        return CCMSAV_OK;
    }

    // ---- autotuner --------------------------------------------------------
    template <int MM> static const void* coldct_fn() {
        if constexpr (WGeo<MM>::WPL > 1) return (const void*)kw_coldct_gram_split<MM>;
        else return (const void*)kw_coldct_gram<MM>;
    }
    template <int MM> int apply_carveout_M(int c) {
        if (cudaFuncSetAttribute((const void*)kw_rowdct_T<MM>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
            cudaFuncSetAttribute(coldct_fn<MM>(), cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
            cudaFuncSetAttribute((const void*)kw_comb_icolT<MM>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess)
            return CCMSAV_ECUDA;
        if constexpr (WGeo<MM>::WPL == 1)
            if (cudaFuncSetAttribute((const void*)kw_rowdct_T<MM, true>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
                cudaFuncSetAttribute((const void*)kw_coldct_gram<MM, true>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess ||
                cudaFuncSetAttribute((const void*)kw_comb_icolT<MM, true>, cudaFuncAttributePreferredSharedMemoryCarveout, c) != cudaSuccess)
                return CCMSAV_ECUDA;
        return CCMSAV_OK;
    }
    int apply_carveout(int c) {
        if constexpr (std::is_same<T, float>::value) {
            switch (M) {
                case 64: return apply_carveout_M<64>(c);
                case 128: return apply_carveout_M<128>(c);
                case 256: return apply_carveout_M<256>(c);
                case 512: return apply_carveout_M<512>(c);
                case 1024: return apply_carveout_M<1024>(c);
                case 2048: return apply_carveout_M<2048>(c);
                case 4096: return apply_carveout_M<4096>(c);
            }
        }
        return CCMSAV_OK;
    }
    void drop_graphs() {
        if (st) cudaStreamSynchronize(st);
        for (int i = 0; i < 3; ++i) {
            if (gexec[i]) cudaGraphExecDestroy(gexec[i]);
            if (gexec1[i]) cudaGraphExecDestroy(gexec1[i]);
            gexec[i] = gexec1[i] = nullptr;
        }
    }
    // Apply a schedule (the warp path only where it was set up).
    int apply_choice(const TuneChoice& c) {
        drop_graphs();
        warp_path = have_warp && c.warp;
        return have_warp ? apply_carveout(c.carveout) : CCMSAV_OK;
    }
    bool have_warp = false;
    static constexpr double kTuneMargin = 0.02;

    // State saved while the autotuner times candidate schedules: the four
    // levels, the scalars and the host counters.
    T* tune_snap = nullptr;
    DevScalars tune_sc{};
    int tune_cur = 0, tune_prev = 1, tune_spare = 2;
    long long tune_steps = 0;

    int tune_save() override {
        if (!have_state || poisoned || classical) return CCMSAV_ESTATE;
        if (!tune_snap && cudaMalloc(&tune_snap, 4 * NN * sizeof(T)) != cudaSuccess) return CCMSAV_ENOMEM;
        tune_cur = cur; tune_prev = prev; tune_spare = spare; tune_steps = steps_taken;
        T* lv[4] = {phi[cur], psi[cur], phi[prev], psi[prev]};
        for (int q = 0; q < 4; ++q)
            CCM_CUDA(cudaMemcpyAsync(tune_snap + q * NN, lv[q], NN * sizeof(T), cudaMemcpyDeviceToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(&tune_sc, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        return CCMSAV_OK;
    }

    int tune_load() override {
        if (!tune_snap) return CCMSAV_ESTATE;
        cur = tune_cur; prev = tune_prev; spare = tune_spare; steps_taken = tune_steps;
        T* dst[4] = {phi[cur], psi[cur], phi[prev], psi[prev]};
        for (int q = 0; q < 4; ++q)
            CCM_CUDA(cudaMemcpyAsync(dst[q], tune_snap + q * NN, NN * sizeof(T), cudaMemcpyDeviceToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(sc, &tune_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        poisoned = false;
        return CCMSAV_OK;
    }

    void tune_free() override {
        cudaFree(tune_snap);
        tune_snap = nullptr;
    }

    bool tune_has_warp() const override { return have_warp; }

    int tune_apply(int warp, int carveout) override {
        TuneChoice c;
        c.warp = warp; c.carveout = carveout;
        return apply_choice(c);
    }

    int tune_record(int warp, int carveout, double ms, double ms_default) override {
        TuneChoice c;
        c.warp = warp; c.carveout = carveout; c.ms = ms; c.ms_default = ms_default;
        int r = apply_choice(c);
        std::lock_guard<std::mutex> lk(TuneTable<T>::mu());
        TuneTable<T>::table()[N] = c;
        return r;
    }

    // Times `k` steps (a multiple of three, after three warm-up steps that
    // capture the graphs) of each candidate schedule of this simulation
    // alone, from the same saved state; keeps the fastest (the default unless
    // another is kTuneMargin faster), restores the state and records the
    // choice for this (N, precision).  out = {warp, carveout, best ms/step,
    // ms/step of the default schedule}.
    int autotune(int k, double out[4]) override {
        if (k < 3) k = 3;
        k = (k + 2) / 3 * 3;
        int r = tune_save();
        if (r) return r;
        const std::vector<TuneChoice> cand = tune_candidates(have_warp);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = CCMSAV_ECUDA;
        double best = 1e300, dflt = 0.0;
        size_t bi = 0;
        for (size_t i = 0; i < cand.size() && !r; ++i) {
            if ((r = tune_apply(cand[i].warp, cand[i].carveout)) || (r = tune_load())) break;
            if (steps_taken == 0) { if ((r = queue_steps(1))) break; }   // start step outside the timing
            if ((r = queue_steps(3))) break;
            if (cudaEventRecord(e0, st) != cudaSuccess) { r = CCMSAV_ECUDA; break; }
            if ((r = queue_steps(k))) break;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { r = CCMSAV_ECUDA; break; }
            if ((r = device_status())) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / k;
            if (i == 0) dflt = per;
            if (per < best) { best = per; bi = i; }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (bi != 0 && best > (1.0 - kTuneMargin) * dflt) { bi = 0; best = dflt; }
        if (!r) r = tune_record(cand[bi].warp, cand[bi].carveout, best, dflt);
        const int r2 = tune_load();
        tune_free();
        if (r) return r;
        if (r2) return r2;
        out[0] = cand[bi].warp && have_warp ? 1.0 : 0.0; out[1] = cand[bi].carveout; out[2] = best; out[3] = dflt;
        return CCMSAV_OK;
    }

    int autotune_apply_cached() override {
        TuneChoice c;
        {
            std::lock_guard<std::mutex> lk(TuneTable<T>::mu());
            auto it = TuneTable<T>::table().find(N);
            if (it == TuneTable<T>::table().end()) return CCMSAV_OK;
            c = it->second;
        }
        return apply_choice(c);
    }

    int autotune_report(double out[4]) override {
        TuneChoice c;
        c.carveout = kRowCarveout;
        {
            std::lock_guard<std::mutex> lk(TuneTable<T>::mu());
            auto it = TuneTable<T>::table().find(N);
            if (it != TuneTable<T>::table().end()) c = it->second;
        }
        out[0] = warp_path ? 1.0 : 0.0; out[1] = c.carveout; out[2] = c.ms; out[3] = c.ms_default;
        return CCMSAV_OK;
    }

    int bounds_flag() override {
#ifdef CCMSAV_BOUNDS
        unsigned v = 0, z = 0;
        CCM_CUDA(cudaStreamSynchronize(st));
        CCM_CUDA(cudaMemcpyFromSymbol(&v, g_oob_flag, sizeof(v)));
        CCM_CUDA(cudaMemcpyToSymbol(g_oob_flag, &z, sizeof(z)));
        return (int)v;
#else
        return CCMSAV_EINVAL;
#endif
    }

    int pcg_stats(double out[4]) override {
        if (!classical) return CCMSAV_EINVAL;
        CCM_CUDA(cudaStreamSynchronize(st));
        out[0] = pcg_last[0]; out[1] = (double)pcg_total; out[2] = pcg_last[1]; out[3] = pcg_last[2];
        return CCMSAV_OK;
    }

    // Shared-memory share (percent of 228 KB) of the 8-line transform kernels;
    // the driver rounds it up to a supported size: 72 % -> 196 KB, three of
    // the forward kernels' 65 KB CTAs (swizzled line buffers) or two of the
    // recovery kernel's 68 KB ones at N = 2048, and 60 KB of L1 for the
    // twiddle and eigenvalue tables (the full 228 KB leaves 28 KB).
    static constexpr int kRowCarveout = 72;
    static constexpr int kColCarveout = 72;
    static constexpr int kCombCarveout = 72;
    // four-step twiddle table W_M^{n2 k1} of an E x G line shape, entry k1 G + n2
    int make_tw2(int MM, int E, int G, cplx<float>** out) {
        std::vector<cplx<float>> h2((size_t)MM);
        for (int k1 = 0; k1 < E; ++k1)
            for (int n2 = 0; n2 < G; ++n2) {
                const double a = 2.0 * M_PI * (double)((long)n2 * k1 % MM) / MM;
                h2[(size_t)k1 * G + n2].x = (float)std::cos(a);
                h2[(size_t)k1 * G + n2].y = (float)(-std::sin(a));
            }
        if (cudaMalloc(out, MM * sizeof(cplx<float>)) != cudaSuccess) { *out = nullptr; return CCMSAV_ENOMEM; }
        CCM_CUDA(cudaMemcpyAsync(*out, h2.data(), MM * sizeof(cplx<float>), cudaMemcpyHostToDevice, st));
        return CCMSAV_OK;
    }
    template <int MM> int setup_warp() {
        using Gm = WGeo<MM>;
        using Gc = WGeo<MM, comb_shape<MM>(), comb_warps<MM>()>;   // the recovery kernel's geometry
        using Gv = WGeo<MM, 1>;                     // the variant of the inverse kernels
        if (int r = make_tw2(MM, Gm::E, Gm::G, &tw2)) return r;
        if constexpr (comb_shape<MM>() != 0 || irow_shape<MM>() != 0) {
            if (int r = make_tw2(MM, Gv::E, Gv::G, &tw2i)) return r;
        } else {
            tw2i = tw2;
        }
        const size_t bb = Gm::buf_bytes();
        wRT = Gm::SLOTS; wsm_rt = bb;
        wKC = Gm::SLOTS / NF; wsm_col = bb;
        if constexpr (Gm::WPL > 1) {     // two-warp lines: column pass split into the two field groups, one column per CTA
            wKC = 1;
            wsm_col = (size_t)5 * Gm::BUF * sizeof(cplx<float>);
        }
        wRT4 = Gc::SLOTS / 2; wsm_comb = Gc::bufp_bytes();
        wsm_irow = InvGeo<MM>::smem_bytes();
        if (set_smem_limit((const void*)kw_rowdct_T<MM>, wsm_rt, kRowCarveout) || set_smem_limit(coldct_fn<MM>(), wsm_col, kColCarveout) ||
            set_smem_limit((const void*)kw_comb_icolT<MM>, wsm_comb, kCombCarveout) || set_smem_limit((const void*)kw_irow<MM>, wsm_irow))
            return CCMSAV_ECUDA;
        // the grouped-launch instantiations (one warp or less per line)
        if constexpr (WGeo<MM>::WPL == 1)
            if (set_smem_limit((const void*)kw_rowdct_T<MM, true>, wsm_rt, kRowCarveout) ||
                set_smem_limit((const void*)kw_coldct_gram<MM, true>, wsm_col, kColCarveout) ||
                set_smem_limit((const void*)kw_comb_icolT<MM, true>, wsm_comb, kCombCarveout) ||
                set_smem_limit((const void*)kw_irow<MM, true>, wsm_irow))
                return CCMSAV_ECUDA;
        // L2 prefetch one residency ahead only where few CTAs fit per SM (one
        // at N = 4096); with three per SM (N <= 2048) it evicts rows before
        // their use and costs time (73.3 vs 71.5 us at N = 2048)
        {
            int dev = 0, nsm = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return CCMSAV_ECUDA;
            const int res = resident_ctas((const void*)kw_rowdct_T<MM>, kWarps * 32, wsm_rt);
            ahead_rt = res >= 3 * nsm ? 0 : res;
        }
        return CCMSAV_OK;
    }

    // CTAs of a kernel resident on the whole device at once (0 if unknown)
    static int resident_ctas(const void* fn, int threads, size_t smem) {
        int dev = 0, nsm = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) return 0;
        return nsm * per_sm;
    }

    int init_warp_path() {
        std::vector<float> he(N), hp;
        std::vector<wf::PairTw> hf, hi;
        const double hh = p.L / N;
        for (int k = 0; k < N; ++k) { const double s = std::sin(M_PI * k / (2.0 * N)); he[k] = (float)(4.0 * s * s / (hh * hh)); }
        if (cudaMalloc(&evf, N * sizeof(float)) != cudaSuccess) return CCMSAV_ENOMEM;
        CCM_CUDA(cudaMemcpyAsync(evf, he.data(), N * sizeof(float), cudaMemcpyHostToDevice, st));
        // pair k: modes k, N-k (k > 0), M-k, M+k
        const int Mh = N / 2;
        hp.assign(4 * (size_t)(Mh / 2 + 1), 0.f);
        for (int k = 0; k <= Mh / 2; ++k) {
            hp[4 * k + 0] = he[k];
            hp[4 * k + 1] = k > 0 ? he[N - k] : 0.f;
            hp[4 * k + 2] = he[Mh - k];
            hp[4 * k + 3] = he[Mh + k];
        }
        if (cudaMalloc(&evp, hp.size() * sizeof(float)) != cudaSuccess) return CCMSAV_ENOMEM;
        CCM_CUDA(cudaMemcpyAsync(evp, hp.data(), hp.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        // pair twiddles (FP64 closed forms, see wf::PairTw)
        hf.assign(Mh / 2 + 1, wf::PairTw{});
        hi.assign(Mh / 2 + 1, wf::PairTw{});
        const double c0 = std::sqrt(1.0 / N), c1 = std::sqrt(2.0 / N);
        const double s0 = 1.0 / (Mh * c0), s1 = 1.0 / (Mh * c1);
        for (int k = 0; k <= Mh / 2; ++k) {
            const double a = 2.0 * M_PI * k / N, th = M_PI * k / (2.0 * N), q = M_PI / 4.0;
            const double ck = k == 0 ? c0 : c1, sk = k == 0 ? s0 : s1;
            wf::PairTw f{}, v{};
            f.wnx = v.wnx = (float)std::cos(a);
            f.wny = v.wny = (float)(-std::sin(a));
            f.ax = (float)(0.5 * ck * std::cos(th)); f.ay = (float)(-0.5 * ck * std::sin(th));
            f.bx = (float)(0.5 * c1 * std::cos(th - q)); f.by = (float)(0.5 * c1 * std::sin(th - q));
            v.ax = (float)(0.5 * sk * std::cos(th)); v.ay = (float)(0.5 * sk * std::sin(th));
            v.bx = (float)(0.5 * s1 * std::cos(q - th)); v.by = (float)(0.5 * s1 * std::sin(q - th));
            hf[k] = f; hi[k] = v;
        }
        const int np = Mh / 2 + 1;
        std::vector<float4> pf(np), pi(np);
        for (int k = 0; k < np; ++k) {
            pf[k] = make_float4(hf[k].wnx, hf[k].wny, hf[k].ax, hf[k].ay);
            pi[k] = make_float4(hi[k].wnx, hi[k].wny, hi[k].ax, hi[k].ay);
        }
        twF0 = make_float2(hf[0].bx, hf[0].by);
        twI0 = make_float2(hi[0].bx, hi[0].by);
        if (cudaMalloc(&twF, pf.size() * sizeof(float4)) != cudaSuccess) return CCMSAV_ENOMEM;
        if (cudaMalloc(&twI, pi.size() * sizeof(float4)) != cudaSuccess) return CCMSAV_ENOMEM;
        CCM_CUDA(cudaMemcpyAsync(twF, pf.data(), pf.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(twI, pi.data(), pi.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        int r = CCMSAV_EINVAL;
        if constexpr (std::is_same<T, float>::value)
        switch (M) {
            case 64: r = setup_warp<64>(); break;
            case 128: r = setup_warp<128>(); break;
            case 256: r = setup_warp<256>(); break;
            case 512: r = setup_warp<512>(); break;
            case 1024: r = setup_warp<1024>(); break;
            case 2048: r = setup_warp<2048>(); break;
            case 4096: r = setup_warp<4096>(); break;
        }
        if (r == CCMSAV_OK) warp_path = have_warp = true;
        if (r == CCMSAV_OK) {   // a schedule the autotuner chose for this N
            std::lock_guard<std::mutex> lk(TuneTable<T>::mu());
            auto it = TuneTable<T>::table().find(N);
            if (it != TuneTable<T>::table().end()) {
                warp_path = it->second.warp != 0;
                r = apply_carveout(it->second.carveout);
            }
        }
        return r;
    }

    // The FFT kernels of one step on the warp path (FP32 only).
    template <int MM>
    void launch_warp_ffts(const SpecCoef& s, int anchor) {
        SpecCoefF sf{(float)s.C1, (float)s.C2, (float)s.C3, (float)s.Ct, (float)s.lam};
        const float* fin = reinterpret_cast<const float*>(bufA);
        float* fB = reinterpret_cast<float*>(bufB);
        const cplx<float>* t2 = tw2;
        kw_rowdct_T<MM><<<dim3(N / wRT, NF), kWarps * 32, wsm_rt, st>>>(fin, fB, t2, pair_tab(twF), ahead_rt, GroupArgs<false>{}, 0);
        mark(1);
        if constexpr (WGeo<MM>::WPL > 1)
            kw_coldct_gram_split<MM><<<dim3(N, 2), kSplitWarps * 32, wsm_col, st>>>(fB, reinterpret_cast<float*>(bufA), part2,
                                                                                  t2, pair_tab(twF), evf, evp, sf);
        else
            kw_coldct_gram<MM><<<N / wKC, kWarps * 32, wsm_col, st>>>(fB, reinterpret_cast<float*>(bufA), part2, t2, pair_tab(twF), evf, evp, sf,
                                                                     GroupArgs<false>{}, 0);
        mark(2);
    }
    int bdf1_launch = 0;
    template <int MM>
    void launch_warp_inverse(const SpecCoef& s, int anchor) {
        SpecCoefF sf{(float)s.C1, (float)s.C2, (float)s.C3, (float)s.Ct, (float)s.lam};
        kw_comb_icolT<MM><<<N / wRT4, comb_warps<MM>() * 32, wsm_comb, st>>>(reinterpret_cast<const float*>(bufA),
            reinterpret_cast<float*>(bufB), comb_shape<MM>() ? tw2i : tw2, pair_tab(twI), evf, evp, sf, sc, anchor,
            GroupArgs<false>{}, 0);
        mark(4);
        kw_irow<MM><<<(2 * N + InvGeo<MM>::LINES - 1) / InvGeo<MM>::LINES, InvGeo<MM>::WARPS * 32, wsm_irow, st>>>(
            reinterpret_cast<const float*>(bufB),
            reinterpret_cast<float*>(phi[spare]), reinterpret_cast<float*>(psi[spare]), irow_shape<MM>() ? tw2i : tw2,
            pair_tab(twI),
            reinterpret_cast<const float*>(phi[cur]), reinterpret_cast<const float*>(phi[prev]),
            reinterpret_cast<const float*>(psi[cur]), reinterpret_cast<const float*>(psi[prev]),
            bdf1_launch, sc, anchor, GroupArgs<false>{}, 0);
        mark(5);
    }
    void warp_forward(const SpecCoef& s, int anchor) {
        if constexpr (std::is_same<T, float>::value)
        switch (M) {
            case 64: launch_warp_ffts<64>(s, anchor); break;
            case 128: launch_warp_ffts<128>(s, anchor); break;
            case 256: launch_warp_ffts<256>(s, anchor); break;
            case 512: launch_warp_ffts<512>(s, anchor); break;
            case 1024: launch_warp_ffts<1024>(s, anchor); break;
            case 2048: launch_warp_ffts<2048>(s, anchor); break;
            default: launch_warp_ffts<4096>(s, anchor); break;
        }
    }
    void warp_inverse(const SpecCoef& s, int anchor) {
        if constexpr (std::is_same<T, float>::value)
        switch (M) {
            case 64: launch_warp_inverse<64>(s, anchor); break;
            case 128: launch_warp_inverse<128>(s, anchor); break;
            case 256: launch_warp_inverse<256>(s, anchor); break;
            case 512: launch_warp_inverse<512>(s, anchor); break;
            case 1024: launch_warp_inverse<1024>(s, anchor); break;
            case 2048: launch_warp_inverse<2048>(s, anchor); break;
            default: launch_warp_inverse<4096>(s, anchor); break;
        }
    }

    double h() const { return p.L / N; }
    double theta_tilde() const { return p.theta + p.gamma_bend * 3.0 * M_SQRT2 / (4.0 * p.eps); }

    DiagCoef diag_coef() const {
        DiagCoef c;
        c.inv_h = 1.0 / h(); c.inv_h2 = 1.0 / (h() * h()); c.eps = p.eps; c.inv_eps = 1.0 / p.eps; c.beta = p.beta;
        c.gin = p.gamma_in; c.gout = p.gamma_out; c.psin = p.psi_in; c.psout = p.psi_out; c.bin = p.beta_in; c.bout = p.beta_out;
        return c;
    }

    // Runs k_diag on (a, b, psi) and returns the NDIAG sums (FP64, fixed order).
    int diag_sums(const T* a, const T* b, const T* ps, double out[NDIAG]) {
        k_diag<T><<<g_dg, 256, 0, st>>>(a, b, ps, partd, N, diag_coef());
        ++nlaunch;
        CCM_CUDA(cudaGetLastError());
        CCM_CUDA(cudaMemcpyAsync(h_part, partd, (size_t)nbd * NDIAG * sizeof(double), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < NDIAG; ++q) out[q] = 0.0;
        for (int bk = 0; bk < nbd; ++bk)
            for (int q = 0; q < NDIAG; ++q) out[q] += h_part[(size_t)bk * NDIAG + q];
        return CCMSAV_OK;
    }

    // Uploads the four levels (FP64 host arrays; a missing previous level is
    // a device copy of level n) through the FP64 staging buffer; the upload kernels flag non-finite values and sum psi0 with
    // compensated partial sums, so the host touches no field value.  One
    // synchronisation at the end (the copies and kernels are stream-ordered).
    int upload_levels(const double* phi0, const double* psi0, const double* phi1, const double* psi1, double* psi_sum) {
        double* d = (double*)tmp64;
        const size_t nb = NN * sizeof(double);
        double* dpart = reinterpret_cast<double*>(d_upbad) + 1;
        CCM_CUDA(cudaMemsetAsync(d_upbad, 0, sizeof(double), st));
        const double* src[4] = {phi0, psi0, phi1, psi1};
        T* dst[4] = {phi[cur], psi[cur], phi[prev], psi[prev]};
        for (int q = 0; q < 4; ++q) {
            if (!src[q]) {   // no previous level given: the same values (and rounding) as level n
                CCM_CUDA(cudaMemcpyAsync(dst[q], dst[q - 2], NN * sizeof(T), cudaMemcpyDeviceToDevice, st));
                continue;
            }
            double* stage = d + (q & 1) * NN;
            CCM_CUDA(cudaMemcpyAsync(stage, src[q], nb, cudaMemcpyHostToDevice, st));
            double* part = q == 1 ? dpart : nullptr;
            if (std::is_same<T, float>::value && (q & 1))
                k_upload<float, true><<<kUpBlocks, 256, 0, st>>>(stage, reinterpret_cast<float*>(dst[q]), NN, d_upbad, part);
            else
                k_upload<T, false><<<kUpBlocks, 256, 0, st>>>(stage, dst[q], NN, d_upbad, part);
            ++nlaunch;
            CCM_CUDA(cudaGetLastError());
        }
        CCM_CUDA(cudaMemcpyAsync(h_up, d_upbad, (1 + 2 * kUpBlocks) * sizeof(double), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        if (*reinterpret_cast<const unsigned*>(h_up) != 0u) return CCMSAV_ENONFINITE;
        // conserved mass: the blocks' compensated partials added in a fixed
        // order (Neumaier), accurate to a few ulps of the sum; a plain running
        // sum of 10^6..10^8 positive values can be off by 1e-11 relative,
        // which the FP32 path would then conserve
        double ssum = 0.0, scomp = 0.0;
        for (int k = 0; k < 2 * kUpBlocks; ++k) {
            const double x = h_up[1 + k], t = ssum + x;
            scomp += std::fabs(ssum) >= std::fabs(x) ? (ssum - t) + x : (x - t) + ssum;
            ssum = t;
        }
        *psi_sum = ssum + scomp;
        return CCMSAV_OK;
    }

    int init_scalars_from_fields(double psi_sum_fp64) {
        double s[NDIAG];
        int r = CCMSAV_OK;
        if constexpr (std::is_same<T, float>::value) {
            // FP32 fields: the five sums in the step's FP32 arithmetic
            const double hh = h();
            InitCoefF ic{(float)(1.0 / hh), (float)p.eps, (float)(1.0 / p.eps), (float)p.beta, (float)p.gamma_in,
                         (float)p.gamma_out, (float)p.psi_in, (float)p.psi_out, (float)p.beta_in, (float)p.beta_out};
            k_init_sums_f32<<<g_dg, 256, 0, st>>>(phi[cur], psi[cur], partd, N, ic);
            ++nlaunch;
            CCM_CUDA(cudaGetLastError());
            CCM_CUDA(cudaMemcpyAsync(h_part, partd, (size_t)nbd * NDIAG * sizeof(double), cudaMemcpyDeviceToHost, st));
            CCM_CUDA(cudaStreamSynchronize(st));
            for (int q = 0; q < NDIAG; ++q) s[q] = 0.0;
            for (int bk = 0; bk < nbd; ++bk)
                for (int q = 0; q < 5; ++q) s[q] += h_part[(size_t)bk * NDIAG + q];
        } else {
            r = diag_sums(phi[cur], phi[cur], psi[cur], s);
        }
        if (r) return r;
        const double h2 = h() * h();
        std::memset(sc_host, 0, sizeof(DevScalars));
        sc_host->V = sc_host->Vo = std::sqrt(h2 * s[0]);
        sc_host->W = sc_host->Wo = std::sqrt(h2 * s[1]);
        sc_host->Z = sc_host->Zo = std::sqrt(h2 * s[2]);
        const double arc = 3.0 * M_SQRT2 / 4.0 * (h2 * s[3] / p.eps + 0.5 * p.eps * h2 * s[4]);
        sc_host->A = arc;
        sc_host->U = sc_host->Uo = 0.0;
        sc_host->mass_mode = psi_sum_fp64 / ((double)N * N);
        sc_host->status = 0;
        if (!(s[0] > 0 && s[1] > 0 && s[2] > 0) || !std::isfinite(arc)) return CCMSAV_ENONFINITE;
        CCM_CUDA(cudaMemcpyAsync(sc, sc_host, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        return CCMSAV_OK;
    }

    int set_state_host(const double* phi0, const double* psi0, const double* phi1, const double* psi1) override {
        cur = 0; prev = 1; spare = 2;
        double psum = 0.0;
        int r = upload_levels(phi0, psi0, phi1, psi1, &psum);
        if (r == CCMSAV_OK) r = init_scalars_from_fields(psum);
        if (r) { have_state = false; return r; }   // the levels were overwritten: no state
        have_state = true; poisoned = false;
        steps_taken = (phi1 && psi1) ? 1 : 0;   // two given levels: continue with BDF2
        return CCMSAV_OK;
    }

    int set_state_device(const void* dphi, const void* dpsi) override {
        cur = 0; prev = 1; spare = 2;
        const size_t fb = NN * sizeof(T);
        CCM_CUDA(cudaMemcpyAsync(phi[cur], dphi, fb, cudaMemcpyDeviceToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(psi[cur], dpsi, fb, cudaMemcpyDeviceToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(phi[prev], dphi, fb, cudaMemcpyDeviceToDevice, st));
        CCM_CUDA(cudaMemcpyAsync(psi[prev], dpsi, fb, cudaMemcpyDeviceToDevice, st));
        double s[NDIAG];
        int r = diag_sums(phi[cur], phi[cur], psi[cur], s);
        if (r) return r;
        for (int q = 0; q < NDIAG; ++q) if (!std::isfinite(s[q])) return CCMSAV_ENONFINITE;
        r = init_scalars_from_fields(s[13]);
        if (r) return r;
        have_state = true; poisoned = false; steps_taken = 0;
        return CCMSAV_OK;
    }

    // Coefficients of one step's kernels (BDF1 start step or BDF2).
    void step_coefs(bool bdf1, StencilCoef<T>& c, SpecCoef& s, SolveCoef& so) const {
        const double dt = p.dt;
        c.bdf1 = bdf1 ? 1 : 0;
        c.inv_h = (T)(1.0 / h()); c.inv_h2 = (T)(1.0 / (h() * h()));
        c.eps = (T)p.eps; c.inv_eps = (T)(1.0 / p.eps); c.inv_eps2 = (T)(1.0 / (p.eps * p.eps));
        c.beta = (T)p.beta; c.quarter_inv_eps = (T)(0.25 / p.eps);
        c.Mth = (T)(p.M_phi * theta_tilde()); c.lam = (T)p.lam;
        c.C2 = (T)(p.M_phi * (p.gamma_surf * 3.0 * M_SQRT2 * p.eps / 4.0 + p.theta));
        c.C3 = (T)(p.M_phi * p.gamma_bend * 3.0 * M_SQRT2 * p.eps / 8.0);
        c.betap = (T)(p.M_phi * p.gamma_surf * 3.0 * M_SQRT2 * p.beta / (4.0 * p.eps));
        c.gin = (T)p.gamma_in; c.gout = (T)p.gamma_out; c.hgin = (T)(0.5 * p.gamma_in); c.hgout = (T)(0.5 * p.gamma_out);
        c.psin = (T)p.psi_in; c.psout = (T)p.psi_out;
        c.bin = (T)p.beta_in; c.bout = (T)p.beta_out; c.M0 = (T)p.M0;
        const double a = bdf1 ? 1.0 / dt : 1.5 / dt;
        s.C1 = a + p.M_phi * p.gamma_surf * 3.0 * M_SQRT2 * p.beta / (4.0 * p.eps);
        s.C2 = p.M_phi * (p.gamma_surf * 3.0 * M_SQRT2 * p.eps / 4.0 + p.theta);
        s.C3 = p.M_phi * p.gamma_bend * 3.0 * M_SQRT2 * p.eps / 8.0;
        s.Ct = a; s.lam = p.lam;
        so.h2 = h() * h();
        so.cgs = p.M_phi * p.gamma_surf * 3.0 * M_SQRT2 / 2.0;
        so.cga = p.M_phi * p.gamma_area;
        so.cgb = p.M_phi * p.gamma_bend * 3.0 * M_SQRT2 / (8.0 * p.eps);
        so.cgo = p.M_phi;
        so.bdf1 = bdf1 ? 1 : 0;
        so.nb1 = nb1; so.nb2 = N;
        so.inv_NN = 1.0 / (double)NN;
    }

    int queue_one_step() {
        const bool bdf1 = (steps_taken == 0) || (flags & CCMSAV_BDF1_ALWAYS);
        const double dt = p.dt;
        StencilCoef<T> c;
        SpecCoef s;
        SolveCoef so;
        step_coefs(bdf1, c, s, so);
        const int anchor = (sizeof(T) == sizeof(float)) ? 1 : 0;
        so.anchor = anchor;

        if (prof && ev_used + 16 > 4096) { int r = profile_flush(); if (r) return r; }
        mark(-1);
        k_stencil<T><<<g_st, b_st, stencil_smem_bytes<T>(), st>>>(phi[cur], phi[prev], psi[cur], psi[prev], bufA, part1, N, c,
                                                              GroupArgs<false>{}, 0);
        mark(0);
        if (classical) {
            int r = queue_classical_ch(bdf1);
            if (r) return r;
            mark(7);
        }
        if (warp_path) {
            warp_forward(s, anchor);
            so.nb2 = N / wKC;
        } else {
            k_rowdct_T<T><<<dim3(N / RT, NF), 512, sm_rt, st>>>(bufA, bufB, N, RT, lds_rt, twM, twP);
            mark(1);
            k_coldct_gram<T><<<N, 512, sm_col, st>>>(bufB, bufA, part2, N, FG, twM, twP, ev, s);
            mark(2);
        }
        {   // partial rows: FP64, or float pairs on the FP32 path
            using P = typename PartialOf<T>::type;
            if (classical) {   // the psi entries from the conjugate-gradient solves
                k_cl_inject<P><<<(so.nb2 + 255) / 256, 256, 0, st>>>(reinterpret_cast<P*>(part2), so.nb2, pcg);
                ++nlaunch;
            }
            k_solve<P><<<kSolveBlocks, kSolveThreads, 0, st>>>(reinterpret_cast<const P*>(part1), so.nb1,
                                                               reinterpret_cast<const P*>(part2), so.nb2, part3, sc, so,
                                                               GroupArgs<false>{}, 0);
        }
        mark(3);
        if (warp_path) {
            bdf1_launch = so.bdf1;
            warp_inverse(s, anchor);
        } else {
            k_comb_icolT<T><<<N / RT4, 512, sm_comb, st>>>(bufA, bufB, N, RT4, lds_c, twM, twP, ev, s, sc, anchor);
            mark(4);
            k_irow<T><<<N / PR, 512, sm_irow, st>>>(bufB, phi[spare], psi[spare], N, PR, twM, twP,
                                                    phi[cur], phi[prev], psi[cur], psi[prev], so.bdf1, sc, anchor);
            mark(5);
        }
        nlaunch += 6;
        if (classical) {
            k_cl_psi<T><<<cl_nb, kClThreads, 0, st>>>(psi[cur], psi[prev], cl + 3 * NN, sc, bdf1 ? 1 : 0, psi[spare], NN);
            ++nlaunch;
        }
        if (!bdf1 && (flags & CCMSAV_TRACK_ENERGY)) {
            k_dnorm<T><<<g_dg, 256, 0, st>>>(phi[cur], phi[prev], psi[spare], psi[cur], psi[prev], partd, N, p.M0);
            k_add_lamsum<<<1, 256, 0, st>>>(partd, nbd, 0.5 * dt * p.lam * p.lam, sc);
            mark(6);
            nlaunch += 2;
        }
        if (prof) ++prof_steps;
        CCM_CUDA(cudaGetLastError());
        const int nw = spare;
        spare = prev; prev = cur; cur = nw;
        ++steps_taken;
        return CCMSAV_OK;
    }

    int queue_steps(int nsteps) override {
        if (!have_state) return CCMSAV_ESTATE;
        if (poisoned) return CCMSAV_ENONFINITE;
        int r;
        // the BDF1 start step and traced steps are launched directly
        while (nsteps > 0 && (steps_taken == 0 || prof || graphs_failed)) {
            if ((r = queue_one_step())) return r;
            --nsteps;
        }
        // BDF2 steps in groups of three from CUDA graphs (the rotation of the
        // three levels has period three, so one graph per phase)
        const long long per_step = launches_per_step();
        while (nsteps >= 3 && !graphs_failed) {
            const int ph = cur;
            if (!gexec[ph] && capture_phase() != CCMSAV_OK) { graphs_failed = true; break; }
            CCM_CUDA(cudaGraphLaunch(gexec[ph], st));
            steps_taken += 3;
            nlaunch += 3 * per_step;
            nsteps -= 3;
        }
        // the remaining one or two steps from single-step graphs (one launch
        // each instead of six; step-at-a-time callers take this path)
        while (nsteps > 0 && !graphs_failed) {
            const int ph = cur;
            if (!gexec1[ph] && capture_single() != CCMSAV_OK) { graphs_failed = true; break; }
            CCM_CUDA(cudaGraphLaunch(gexec1[ph], st));
            const int nw = spare;
            spare = prev; prev = cur; cur = nw;
            steps_taken += 1;
            nlaunch += per_step;
            --nsteps;
        }
        while (nsteps-- > 0)
            if ((r = queue_one_step())) return r;
        return CCMSAV_OK;
    }

    int device_status() override {
        // one wait: the copy into the pinned mirror is ordered after the queued steps
        CCM_CUDA(cudaMemcpyAsync(sc_host, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        if (sc_host->status != 0) { poisoned = true; return sc_host->status; }
        return CCMSAV_OK;
    }

    int get_fields(double* ph, double* ps, bool previous) override {
        if (!have_state) return CCMSAV_ESTATE;
        int r = device_status();
        if (r) return r;
        double* d = (double*)tmp64;
        const int lv = previous ? prev : cur;
        k_convert<T, double><<<1024, 256, 0, st>>>(phi[lv], d, NN);
        k_convert<T, double><<<1024, 256, 0, st>>>(psi[lv], d + NN, NN);
        nlaunch += 2;
        CCM_CUDA(cudaGetLastError());
        CCM_CUDA(cudaMemcpyAsync(ph, d, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaMemcpyAsync(ps, d + NN, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        return CCMSAV_OK;
    }

    int energy(double out[8]) override {
        if (!have_state) return CCMSAV_ESTATE;
        int r = device_status();
        if (r) return r;
        double s[NDIAG];
        if ((r = diag_sums(phi[cur], phi[prev], psi[cur], s))) return r;
        const double h2 = h() * h();
        const DevScalars& q = *sc_host;
        const double cb = p.gamma_bend * 3.0 * M_SQRT2 * p.eps / 8.0;
        const double cs = p.gamma_surf * 3.0 * M_SQRT2 * p.eps / 4.0 + p.theta;
        const double cbeta = p.gamma_surf * 3.0 * M_SQRT2 * p.beta / (4.0 * p.eps);
        const double tt = theta_tilde();
        if (flags & CCMSAV_BDF1_ALWAYS) {
            // one-level energy of the first-order scheme (the BDF1 energy balance)
            double E1 = 0.5 * cb * h2 * s[5] + 0.5 * (cs - tt) * h2 * s[4] + 0.5 * cbeta * h2 * s[9];
            E1 += 0.5 * p.gamma_surf * 3.0 * M_SQRT2 / 2.0 * q.V * q.V + 0.5 * p.gamma_area * q.U * q.U;
            E1 += 0.5 * p.gamma_bend * 3.0 * M_SQRT2 / (8.0 * p.eps) * q.W * q.W + 0.5 * q.Z * q.Z;
            out[0] = E1;
        }
        double E = 0.5 * cb * h2 * (s[5] + s[6]);
        E += 0.5 * cs * h2 * (s[4] + s[7]);
        E -= 0.5 * tt * h2 * (s[4] + s[7] - 2.0 * s[8]);
        E += 0.5 * cbeta * h2 * (s[9] + s[10]);
        E += 0.5 * p.gamma_surf * 3.0 * M_SQRT2 / 2.0 * (q.V * q.V + (2 * q.V - q.Vo) * (2 * q.V - q.Vo));
        E += 0.5 * p.gamma_area * (q.U * q.U + (2 * q.U - q.Uo) * (2 * q.U - q.Uo));
        E += 0.5 * p.gamma_bend * 3.0 * M_SQRT2 / (8.0 * p.eps) * (q.W * q.W + (2 * q.W - q.Wo) * (2 * q.W - q.Wo));
        E += 0.5 * (q.Z * q.Z + (2 * q.Z - q.Zo) * (2 * q.Z - q.Zo));
        E -= q.lamsum;
        const double arc = 3.0 * M_SQRT2 / 4.0 * (h2 * s[3] / p.eps + 0.5 * p.eps * h2 * s[4]);
        const double Fs = p.gamma_surf * arc;
        const double Fb = p.gamma_bend * 3.0 * M_SQRT2 / (16.0 * p.eps) * h2 * s[11];
        const double Fa = 0.5 * p.gamma_area * (arc - q.A) * (arc - q.A);
        const double Fo = h2 * s[12];
        if (!(flags & CCMSAV_BDF1_ALWAYS)) out[0] = E;
        out[1] = Fs; out[2] = Fb; out[3] = Fa; out[4] = Fo; out[5] = arc;
        out[6] = q.lamsum; out[7] = Fs + Fb + Fa + Fo;
        return CCMSAV_OK;
    }

    int mass(double* m) override {
        if (!have_state) return CCMSAV_ESTATE;
        int r = device_status();
        if (r) return r;
        double s[NDIAG];
        if ((r = diag_sums(phi[cur], phi[cur], psi[cur], s))) return r;
        *m = h() * h() * s[13];
        return CCMSAV_OK;
    }

    int get_aux(double aux[12]) override {
        if (!have_state) return CCMSAV_ESTATE;
        int r = device_status();
        if (r && r != CCMSAV_ENONFINITE) return r;
        const DevScalars& q = *sc_host;
        aux[0] = q.V; aux[1] = q.U; aux[2] = q.W; aux[3] = q.Z;
        aux[4] = q.Vo; aux[5] = q.Uo; aux[6] = q.Wo; aux[7] = q.Zo;
        aux[8] = q.A; aux[9] = q.lamsum; aux[10] = (double)steps_taken; aux[11] = q.mass_mode;
        return r;
    }

    // the first twelve doubles of DevScalars are aux[0..11] in order
    int get_aux_async(double aux[12]) override {
        static_assert(offsetof(DevScalars, mass_mode) == 11 * sizeof(double), "aux layout");
        if (!have_state) return CCMSAV_ESTATE;
        CCM_CUDA(cudaMemcpyAsync(aux, sc, 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
        return CCMSAV_OK;
    }

    int set_aux(const double aux[12]) override {
        if (!have_state) return CCMSAV_ESTATE;
        for (int i = 0; i < 11; ++i) if (!std::isfinite(aux[i])) return CCMSAV_ENONFINITE;
        int r = device_status();
        if (r && r != CCMSAV_ENONFINITE) return r;
        DevScalars q = *sc_host;
        q.V = aux[0]; q.U = aux[1]; q.W = aux[2]; q.Z = aux[3];
        q.Vo = aux[4]; q.Uo = aux[5]; q.Wo = aux[6]; q.Zo = aux[7];
        q.A = aux[8]; q.lamsum = aux[9]; q.steps = aux[10]; q.status = 0;
        if (aux[11] != 0.0 && std::isfinite(aux[11])) q.mass_mode = aux[11];
        *sc_host = q;
        CCM_CUDA(cudaMemcpyAsync(sc, sc_host, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
        CCM_CUDA(cudaStreamSynchronize(st));
        steps_taken = (long long)aux[10];
        poisoned = false;
        return CCMSAV_OK;
    }

    bool has_state() const override { return have_state; }
    bool in_error() const override { return poisoned; }
    long long launches() const override { return nlaunch; }
};

template <typename T>
SimBase* make_sim(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err) {
    SimImpl<T>* sim = new SimImpl<T>();
    int r = sim->init(p, N, flags, s);
    if (r != CCMSAV_OK) { delete sim; *err = r; return nullptr; }
    *err = CCMSAV_OK;
    return sim;
}

}  // namespace ccm
