// ccmsav_api.cu -- the extern "C" entry points declared in include/ccmsav.h.
#include <cmath>
#include <new>
#include <vector>
#include "sim.h"

struct ccmsav {
    std::vector<ccm::SimBase*> sims;
    cudaStream_t stream = nullptr;
    int precision = 0;
    int flags = 0;
    long long extra_launches = 0;
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
    if (flags & ~CCMSAV_TRACK_ENERGY) return CCMSAV_EINVAL;
    for (int s = 0; s < n_sims; ++s) {
        if (!valid_N(N[s])) return CCMSAV_EINVAL;
        if (!valid_params(per_sim ? per_sim[s] : *params)) return CCMSAV_EINVAL;
    }
    ccmsav* h = new (std::nothrow) ccmsav();
    if (!h) return CCMSAV_ENOMEM;
    h->stream = (cudaStream_t)stream;
    h->precision = precision;
    h->flags = flags;
    for (int s = 0; s < n_sims; ++s) {
        int err = 0;
        const ccmsav_params& p = per_sim ? per_sim[s] : *params;
        ccm::SimBase* sim = (precision == CCMSAV_FP64) ? ccm::make_sim_f64(p, N[s], flags, h->stream, &err)
                                                       : ccm::make_sim_f32(p, N[s], flags, h->stream, &err);
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
    for (int i = 0; i < nsteps; ++i)
        for (ccm::SimBase* s : h->sims) {
            int r = s->queue_steps(1);
            if (r) return r;
        }
    return CCMSAV_OK;
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

int ccmsav_set_aux(ccmsav_t* h, int sim, const double aux[12]) {
    ccm::SimBase* s = get(h, sim);
    if (!s || !aux) return CCMSAV_EINVAL;
    return s->set_aux(aux);
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
    delete h;
}

}  // extern "C"
