// ccmsav_api.cu -- the extern "C" entry points declared in include/ccmsav.h.
#include <cmath>
#include <new>
#include <vector>
#include "sim.h"

// A handle with several simulations gives each its own stream, ordered with
// the caller's stream by events around every call (fork: the simulations
// wait for the caller's stream; join: the caller's stream waits for them), so
// independent simulations run concurrently.  Their BDF2 steps run from one
// graph per rotation phase holding three steps of every simulation as
// parallel branches: one launch per three steps for the whole batch.
struct ccmsav {
    std::vector<ccm::SimBase*> sims;
    cudaStream_t stream = nullptr;        // the caller's stream
    int precision = 0;
    int flags = 0;
    long long extra_launches = 0;
    cudaStream_t cap = nullptr;           // capture origin of the batch graphs
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    cudaGraphExec_t bexec[3] = {nullptr, nullptr, nullptr};
    bool batch_failed = false;
};

namespace {

bool valid_params(const ccmsav_params& p) {
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    auto nonneg = [](double x) { return std::isfinite(x) && x >= 0.0; };
    return pos(p.eps) && pos(p.dt) && pos(p.L) && pos(p.lam) && pos(p.M_phi) &&
           nonneg(p.theta) && nonneg(p.beta) && nonneg(p.gamma_surf) && nonneg(p.gamma_bend) &&
           nonneg(p.gamma_area) && nonneg(p.gamma_in) && nonneg(p.gamma_out) &&
           std::isfinite(p.psi_in) && std::isfinite(p.psi_out) && std::isfinite(p.beta_in) &&
           std::isfinite(p.beta_out) && std::isfinite(p.M0) && p.M0 > 0.0 && p.M0 < 1.0;
}

bool valid_N(int N) { return N >= 8 && N <= 8192 && (N & (N - 1)) == 0; }

bool batched(const ccmsav* h) { return h->sims.size() > 1; }

// the simulations' streams wait for work queued so far on `from`
int fork_from(ccmsav* h, cudaStream_t from) {
    if (cudaEventRecord(h->fork_ev, from) != cudaSuccess) return CCMSAV_ECUDA;
    for (ccm::SimBase* s : h->sims)
        if (cudaStreamWaitEvent(s->stream(), h->fork_ev, 0) != cudaSuccess) return CCMSAV_ECUDA;
    return CCMSAV_OK;
}

// `into` waits for work queued so far on every simulation's stream
int join_into(ccmsav* h, cudaStream_t into) {
    for (size_t k = 0; k < h->sims.size(); ++k) {
        if (cudaEventRecord(h->join_ev[k], h->sims[k]->stream()) != cudaSuccess) return CCMSAV_ECUDA;
        if (cudaStreamWaitEvent(into, h->join_ev[k], 0) != cudaSuccess) return CCMSAV_ECUDA;
    }
    return CCMSAV_OK;
}

// every simulation takes a BDF2 step next, in the same rotation phase
bool uniform_phase(const ccmsav* h) {
    const int ph = h->sims[0]->phase();
    for (ccm::SimBase* s : h->sims)
        if (!s->batchable() || s->phase() != ph) return false;
    return true;
}

// One graph: three steps of every simulation, each on its own stream.
int capture_batch(ccmsav* h, int ph) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCMSAV_ECUDA;
    int r = fork_from(h, h->cap);
    for (size_t k = 0; k < h->sims.size() && r == CCMSAV_OK; ++k) r = h->sims[k]->queue_steps_captured(3);
    if (r == CCMSAV_OK) r = join_into(h, h->cap);
    const cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (r != CCMSAV_OK || e != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); return CCMSAV_ECUDA; }
    const cudaError_t e2 = cudaGraphInstantiate(&h->bexec[ph], g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) { h->bexec[ph] = nullptr; return CCMSAV_ECUDA; }
    return CCMSAV_OK;
}

int step_batched(ccmsav* h, int nsteps) {
    int r = fork_from(h, h->stream);
    if (r) return r;
    // start steps (BDF1) and any simulation out of phase: direct, per simulation
    while (nsteps > 0 && !uniform_phase(h)) {
        for (ccm::SimBase* s : h->sims)
            if ((r = s->queue_steps(1))) return r;
        --nsteps;
    }
    if (nsteps >= 3 && !h->batch_failed) {
        if ((r = join_into(h, h->stream))) return r;
        while (nsteps >= 3) {
            const int ph = h->sims[0]->phase();
            if (!h->bexec[ph] && capture_batch(h, ph) != CCMSAV_OK) { h->batch_failed = true; break; }
            if (cudaGraphLaunch(h->bexec[ph], h->stream) != cudaSuccess) return CCMSAV_ECUDA;
            for (ccm::SimBase* s : h->sims) s->count_steps(3);
            nsteps -= 3;
        }
        if ((r = fork_from(h, h->stream))) return r;
    }
    for (ccm::SimBase* s : h->sims)
        if ((r = s->queue_steps(nsteps))) return r;
    return join_into(h, h->stream);
}

ccm::SimBase* get(ccmsav_t* h, int sim) {
    if (!h || sim < 0 || sim >= (int)h->sims.size()) return nullptr;
    return h->sims[sim];
}

}  // namespace

extern "C" {

int ccmsav_create(ccmsav_t** out, const ccmsav_params* params, int n_sims, const int* N,
                  const ccmsav_params* per_sim, int precision, int flags, void* stream) {
    if (!out) return CCMSAV_EINVAL;
    *out = nullptr;
    if (n_sims < 1 || !N || (!params && !per_sim)) return CCMSAV_EINVAL;
    if (precision != CCMSAV_FP64 && precision != CCMSAV_FP32_BULK) return CCMSAV_EINVAL;
    if (flags & ~(CCMSAV_TRACK_ENERGY | CCMSAV_BDF1_ALWAYS | CCMSAV_CLASSICAL)) return CCMSAV_EINVAL;
    for (int s = 0; s < n_sims; ++s) {
        if (!valid_N(N[s])) return CCMSAV_EINVAL;
        if (!valid_params(per_sim ? per_sim[s] : *params)) return CCMSAV_EINVAL;
    }
    ccmsav* h = new (std::nothrow) ccmsav();
    if (!h) return CCMSAV_ENOMEM;
    h->stream = (cudaStream_t)stream;
    h->precision = precision;
    h->flags = flags;
    if (n_sims > 1) {
        if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
            ccmsav_destroy(h);
            return CCMSAV_ECUDA;
        }
        h->join_ev.assign(n_sims, nullptr);
        for (int s = 0; s < n_sims; ++s)
            if (cudaEventCreateWithFlags(&h->join_ev[s], cudaEventDisableTiming) != cudaSuccess) {
                ccmsav_destroy(h);
                return CCMSAV_ECUDA;
            }
    }
    for (int s = 0; s < n_sims; ++s) {
        int err = 0;
        const ccmsav_params& p = per_sim ? per_sim[s] : *params;
        // several simulations: each on a stream of its own (see struct ccmsav)
        cudaStream_t ss = n_sims > 1 ? nullptr : h->stream;
        ccm::SimBase* sim = (precision == CCMSAV_FP64) ? ccm::make_sim_f64(p, N[s], flags, ss, &err)
                                                       : ccm::make_sim_f32(p, N[s], flags, ss, &err);
        if (!sim) { ccmsav_destroy(h); return err ? err : CCMSAV_ENOMEM; }
        sim->N = N[s];
        h->sims.push_back(sim);
    }
    *out = h;
    return CCMSAV_OK;
}

int ccmsav_set_state(ccmsav_t* h, int sim, const double* phi, const double* psi) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !phi || !psi) return CCMSAV_EINVAL;
    return s->set_state_host(phi, psi, nullptr, nullptr);
}

int ccmsav_set_state_levels(ccmsav_t* h, int sim, const double* phi, const double* psi,
                            const double* phi_prev, const double* psi_prev) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !phi || !psi || !phi_prev || !psi_prev) return CCMSAV_EINVAL;
    return s->set_state_host(phi, psi, phi_prev, psi_prev);
}

int ccmsav_set_state_device(ccmsav_t* h, int sim, const void* phi, const void* psi) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !phi || !psi) return CCMSAV_EINVAL;
    return s->set_state_device(phi, psi);
}

int ccmsav_step(ccmsav_t* h, int nsteps) {
    if (!h || nsteps < 0) return CCMSAV_EINVAL;
    for (ccm::SimBase* s : h->sims) {
        if (!s->has_state()) return CCMSAV_ESTATE;
        if (s->in_error()) return CCMSAV_ESTATE;
    }
    if (batched(h)) return step_batched(h, nsteps);
    return h->sims[0]->queue_steps(nsteps);
}

int ccmsav_sync(ccmsav_t* h) {
    if (!h) return CCMSAV_EINVAL;
    int first = CCMSAV_OK;
    for (ccm::SimBase* s : h->sims) {
        if (!s->has_state()) continue;
        int r = s->device_status();
        if (r && !first) first = r;
    }
    return first;
}

int ccmsav_get_state(ccmsav_t* h, int sim, double* phi, double* psi) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !phi || !psi) return CCMSAV_EINVAL;
    return s->get_fields(phi, psi, false);
}

int ccmsav_get_prev_state(ccmsav_t* h, int sim, double* phi, double* psi) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !phi || !psi) return CCMSAV_EINVAL;
    return s->get_fields(phi, psi, true);
}

int ccmsav_energy(ccmsav_t* h, int sim, double out[8]) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !out) return CCMSAV_EINVAL;
    return s->energy(out);
}

int ccmsav_mass(ccmsav_t* h, int sim, double* mass) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !mass) return CCMSAV_EINVAL;
    return s->mass(mass);
}

int ccmsav_get_aux(ccmsav_t* h, int sim, double aux[12]) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !aux) return CCMSAV_EINVAL;
    return s->get_aux(aux);
}

int ccmsav_get_aux_async(ccmsav_t* h, int sim, double aux[12]) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !aux) return CCMSAV_EINVAL;
    return s->get_aux_async(aux);
}

int ccmsav_set_aux(ccmsav_t* h, int sim, const double aux[12]) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !aux) return CCMSAV_EINVAL;
    return s->set_aux(aux);
}

int ccmsav_set_pcg(ccmsav_t* h, double rtol, int max_iter) {
    if (!h || !(h->flags & CCMSAV_CLASSICAL)) return CCMSAV_EINVAL;
    for (ccm::SimBase* s : h->sims) {
        const int r = s->set_pcg(rtol, max_iter);
        if (r) return r;
    }
    return CCMSAV_OK;
}

int ccmsav_pcg_stats(ccmsav_t* h, int sim, double out[4]) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !out) return CCMSAV_EINVAL;
    return s->pcg_stats(out);
}

int ccmsav_autotune(ccmsav_t* h, int steps, double* report) {
    if (!h || steps < 1 || steps > 3000) return CCMSAV_EINVAL;
    if (h->flags & CCMSAV_CLASSICAL) return CCMSAV_EINVAL;
    int r = ccmsav_sync(h);
    if (r) return r;
    for (ccm::SimBase* s : h->sims)
        if (!s->has_state()) return CCMSAV_ESTATE;
    if (!batched(h)) {
        double row[4];
        if ((r = h->sims[0]->autotune(steps, row))) return r;
        if (report) for (int i = 0; i < 4; ++i) report[i] = row[i];
        return CCMSAV_OK;
    }
    // Several simulations: every candidate schedule is applied to all of
    // them and the batched step of the whole handle is timed, since that is
    // what the handle runs (a schedule that is faster for one simulation
    // alone can be slower when the simulations share the GPU).
    const int k = (steps < 3 ? 3 : steps + 2) / 3 * 3;
    bool any_warp = false;
    for (ccm::SimBase* s : h->sims) {
        if ((r = s->tune_save())) return r;
        any_warp = any_warp || s->tune_has_warp();
    }
    const std::vector<ccm::TuneChoice> cand = ccm::tune_candidates(any_warp);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = CCMSAV_ECUDA;
    double best = 1e300, dflt = 0.0;
    size_t bi = 0;
    auto drop_batch = [&]() {
        for (int i = 0; i < 3; ++i) if (h->bexec[i]) { cudaGraphExecDestroy(h->bexec[i]); h->bexec[i] = nullptr; }
    };
    for (size_t i = 0; i < cand.size() && !r; ++i) {
        for (ccm::SimBase* s : h->sims) {
            if ((r = s->tune_apply(cand[i].warp, cand[i].carveout)) || (r = s->tune_load())) break;
        }
        if (r) break;
        drop_batch();
        if ((r = ccmsav_step(h, 3))) break;
        if (cudaEventRecord(e0, h->stream) != cudaSuccess) { r = CCMSAV_ECUDA; break; }
        if ((r = ccmsav_step(h, k))) break;
        if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { r = CCMSAV_ECUDA; break; }
        if ((r = ccmsav_sync(h))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / k;
        if (i == 0) dflt = per;
        if (per < best) { best = per; bi = i; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (bi != 0 && best > 0.98 * dflt) { bi = 0; best = dflt; }
    for (ccm::SimBase* s : h->sims) {
        int e = r ? CCMSAV_OK : s->tune_record(cand[bi].warp, cand[bi].carveout, best, dflt);
        const int e2 = s->tune_load();
        s->tune_free();
        if (!r) r = e ? e : e2;
    }
    drop_batch();
    if (r) return r;
    if (report)
        for (size_t q = 0; q < h->sims.size(); ++q)
            if ((r = h->sims[q]->autotune_report(report + 4 * q))) return r;
    return CCMSAV_OK;
}

int ccmsav_bounds_flag(ccmsav_t* h) {
    if (!h) return CCMSAV_EINVAL;
    int acc = 0;
    for (ccm::SimBase* s : h->sims) {
        const int r = s->bounds_flag();
        if (r < 0) return r;
        acc |= r;
    }
    return acc;
}

int ccmsav_grid_size(ccmsav_t* h, int sim) {
    ccm::SimBase* s = get(h, sim);
    if (!s) return CCMSAV_EINVAL;
    return s->N;
}

long long ccmsav_launch_count(ccmsav_t* h) {
    if (!h) return 0;
    long long n = h->extra_launches;
    for (ccm::SimBase* s : h->sims) n += s->launches();
    return n;
}

int ccmsav_profile(ccmsav_t* h, int enable) {
    if (!h) return CCMSAV_EINVAL;
    for (ccm::SimBase* s : h->sims) {
        int r = s->profile(enable != 0);
        if (r) return r;
    }
    return CCMSAV_OK;
}

int ccmsav_profile_read(ccmsav_t* h, int sim, double ms[8], long long* nsteps) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !ms || !nsteps) return CCMSAV_EINVAL;
    return s->profile_read(ms, nsteps);
}

const char* ccmsav_strerror(int status) {
    switch (status) {
        case CCMSAV_OK: return "ok";
        case CCMSAV_EINVAL: return "invalid argument";
        case CCMSAV_ENOMEM: return "out of memory";
        case CCMSAV_ECUDA: return "CUDA runtime error";
        case CCMSAV_ESTATE: return "call out of order (no state set, or simulation in error)";
        case CCMSAV_ENONFINITE: return "non-finite state, non-positive SAV radicand or non-positive face mobility";
        case CCMSAV_ETIMEOUT: return "a bounded device-side wait gave up";
        default: return "unknown status";
    }
}

void ccmsav_destroy(ccmsav_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    for (ccm::SimBase* s : h->sims) delete s;
    for (cudaGraphExec_t& g : h->bexec) if (g) cudaGraphExecDestroy(g);
    for (cudaEvent_t e : h->join_ev) if (e) cudaEventDestroy(e);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

}  // extern "C"
