// ccmsav_api.cu -- the extern "C" entry points declared in include/ccmsav.h.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <vector>
#include "sim.h"

// A handle with several simulations gives each its own stream, ordered with
// the caller's stream by events around every call (fork: the simulations
// wait for the caller's stream; join: the caller's stream waits for them), so
// independent simulations run concurrently.  Their BDF2 steps run from one
// graph per rotation phase holding three steps of every simulation as
// parallel branches: one launch per three steps for the whole batch.
// Default size of a launch group: simulations of the same N are grouped
// until a group holds about this many grid points; several groups run on
// different streams, so their phases still overlap.  Measured (64 FP32
// simulations, ms per batched step, no grouping -> 2^21): N = 128 0.222 ->
// 0.114, N = 256 0.351 -> 0.286, the mixed 128/256/512 batch 0.549 ->
// 0.484; at N = 512 and 1024 grouping gains nothing (0.252 -> 0.263 for 16
// at N = 512), so the autotuner also times the group size per handle.
constexpr long long kGroupPoints = 1LL << 21;

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
    // grouped launches of the graph of each rotation phase: which
    // simulations are grouped, and how many kernel launches one replay makes
    // for the groups
    std::vector<char> grouped[3];
    long long group_launches[3] = {0, 0, 0};
    long long group_points = kGroupPoints;   // grid points per launch group (0: no grouping)
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

// One graph: three steps of every simulation.  Simulations that can share
// launches (the same line length on the FP32 warp path) are grouped: each
// group's six kernels per step run as one launch each on the stream of its
// first member; every other simulation runs its own launches on its own
// stream.  The groups' argument records go into the launch parameters, so
// the graph keeps its own copy.
int capture_batch(ccmsav* h, int ph) {
    const size_t n = h->sims.size();
    std::map<int, std::vector<size_t>> bykey;
    if (h->group_points > 0)
        for (size_t k = 0; k < n; ++k)
            if (const int key = h->sims[k]->group_key()) bykey[key].push_back(k);
    // launch groups: consecutive members of one key, about group_points grid
    // points each; a group of one runs its own launches
    std::vector<std::vector<size_t>> groups;
    for (auto& kv : bykey) {
        const long long pts = (long long)h->sims[kv.second[0]]->N * h->sims[kv.second[0]]->N;
        const size_t cap = (size_t)std::min<long long>(h->sims[kv.second[0]]->max_group(),
                                                       std::max(1LL, h->group_points / pts));
        for (size_t i = 0; i < kv.second.size(); i += cap) {
            std::vector<size_t> g(kv.second.begin() + i, kv.second.begin() + std::min(kv.second.size(), i + cap));
            if (g.size() >= 2) groups.push_back(g);
        }
    }
    h->grouped[ph].assign(n, 0);
    h->group_launches[ph] = 0;
    size_t ng = 0;
    for (auto& g : groups) ng += g.size();
    std::vector<unsigned char> host;
    if (ng > 0) {
        const size_t rb = h->sims[groups[0][0]]->batch_args_bytes();
        host.assign(3 * ng * rb, 0);
        size_t pos = 0;
        for (auto& g : groups)
            for (size_t k : g) {
                for (int i = 0; i < 3; ++i) {
                    const int e = h->sims[k]->fill_batch_args(i, host.data() + ((size_t)i * ng + pos) * rb);
                    if (e) return e;
                }
                h->grouped[ph][k] = 1;
                ++pos;
            }
        h->group_launches[ph] = 3 * 6 * (long long)groups.size();
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCMSAV_ECUDA;
    int r = fork_from(h, h->cap);
    for (size_t k = 0; k < n && r == CCMSAV_OK; ++k)
        if (!h->grouped[ph][k]) r = h->sims[k]->queue_steps_captured(3);
    size_t pos = 0;
    for (size_t gi = 0; gi < groups.size() && r == CCMSAV_OK; ++gi) {
        ccm::SimBase* lead = h->sims[groups[gi][0]];
        const size_t rb = lead->batch_args_bytes();
        r = lead->queue_group_steps(host.data() + pos * rb, (int)groups[gi].size(), (int)ng, lead->stream());
        pos += groups[gi].size();
    }
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
            for (size_t k = 0; k < h->sims.size(); ++k) {
                if (h->grouped[ph].size() == h->sims.size() && h->grouped[ph][k]) h->sims[k]->count_steps_grouped(3);
                else h->sims[k]->count_steps(3);
            }
            h->extra_launches += h->group_launches[ph];
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
    auto drop_batch = [&]() {
        for (int i = 0; i < 3; ++i) if (h->bexec[i]) { cudaGraphExecDestroy(h->bexec[i]); h->bexec[i] = nullptr; }
    };
    // ms per batched step from the kept state (three warm-up steps, then k)
    auto time_batch = [&](double& per) -> int {
        int q;
        for (ccm::SimBase* s : h->sims)
            if ((q = s->tune_load())) return q;
        drop_batch();
        h->batch_failed = false;
        if ((q = ccmsav_step(h, 3))) return q;
        if (cudaEventRecord(e0, h->stream) != cudaSuccess) return CCMSAV_ECUDA;
        if ((q = ccmsav_step(h, k))) return q;
        if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return CCMSAV_ECUDA;
        if ((q = ccmsav_sync(h))) return q;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        per = ms / k;
        return CCMSAV_OK;
    };
    double best = 1e300, dflt = 0.0;
    size_t bi = 0;
    for (size_t i = 0; i < cand.size() && !r; ++i) {
        for (ccm::SimBase* s : h->sims)
            if ((r = s->tune_apply(cand[i].warp, cand[i].carveout))) break;
        double per = 0.0;
        if (r || (r = time_batch(per))) break;
        if (i == 0) dflt = per;
        if (per < best) { best = per; bi = i; }
    }
    if (bi != 0 && best > 0.98 * dflt) { bi = 0; best = dflt; }
    // second stage, with the chosen schedule: the size of the launch groups
    // (grid points per group; the handle's current value first)
    bool groupable = false;
    for (ccm::SimBase* s : h->sims) {
        if (!r) r = s->tune_apply(cand[bi].warp, cand[bi].carveout);
        groupable = groupable || s->group_key() != 0;
    }
    if (!r && groupable) {
        const long long g0 = h->group_points;
        std::vector<long long> gc{g0};
        for (long long g : {0LL, 1LL << 17, 1LL << 18, 1LL << 19, 1LL << 20, 1LL << 21, 1LL << 22, 1LL << 26})
            if (g != g0) gc.push_back(g);
        double gbest = 1e300, gdflt = 0.0;
        size_t gi = 0;
        for (size_t i = 0; i < gc.size() && !r; ++i) {
            h->group_points = gc[i];
            double per = 0.0;
            if ((r = time_batch(per))) break;
            if (i == 0) gdflt = per;
            if (per < gbest) { gbest = per; gi = i; }
        }
        if (gi != 0 && gbest > 0.98 * gdflt) { gi = 0; gbest = gdflt; }
        h->group_points = gc[gi];
        if (!r && gbest < best) best = gbest;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
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

int ccmsav_set_group_points(ccmsav_t* h, long long points) {
    if (!h || points < 0) return CCMSAV_EINVAL;
    int r = ccmsav_sync(h);
    if (r) return r;
    h->group_points = points;
    for (cudaGraphExec_t& g : h->bexec) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    h->batch_failed = false;
    return CCMSAV_OK;
}

long long ccmsav_group_points(ccmsav_t* h) { return h ? h->group_points : -1; }

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
