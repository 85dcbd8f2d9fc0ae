// sim.h -- precision-independent interface between the C ABI and the
// per-precision implementations of one simulation.
#pragma once
#include <cuda_runtime.h>
#include "../../include/ccmsav.h"

namespace ccm {

class SimBase {
public:
    virtual ~SimBase() {}
    // phi_prev/psi_prev may be NULL (both levels set to phi/psi; next step is BDF1).
    virtual int set_state_host(const double* phi, const double* psi,
                               const double* phi_prev, const double* psi_prev) = 0;
    virtual int set_state_device(const void* phi, const void* psi) = 0;
    virtual int queue_steps(int nsteps) = 0;
    virtual int get_fields(double* phi, double* psi, bool previous) = 0;
    virtual int energy(double out[8]) = 0;
    virtual int mass(double* m) = 0;
    virtual int get_aux(double aux[12]) = 0;
    virtual int get_aux_async(double aux[12]) = 0;   // queued copy, no wait
    virtual int set_aux(const double aux[12]) = 0;
    virtual int device_status() = 0;      // synchronises the stream
    virtual bool has_state() const = 0;
    virtual bool in_error() const = 0;
    virtual long long launches() const = 0;
    virtual int profile(bool enable) = 0;
    virtual int profile_read(double ms[8], long long* nsteps) = 0;
    // batched stepping of several simulations (one graph for all of them)
    virtual cudaStream_t stream() const = 0;
    virtual int phase() const = 0;                 // rotation phase of the three levels
    virtual bool batchable() const = 0;            // next step is BDF2; no tracing, no error
    virtual int queue_steps_captured(int n3) = 0;  // three steps as direct launches (for a
                                                   // stream capture); host counters unchanged
    virtual void count_steps(int n3) = 0;          // host counters after three batched steps
    // classical MSAV (CCMSAV_CLASSICAL): conjugate-gradient settings and statistics
    virtual int set_pcg(double rtol, int max_iter) = 0;
    virtual int pcg_stats(double out[4]) = 0;
    // autotuner of the line-transform schedule (see ccmsav_autotune)
    virtual int autotune(int k, double out[4]) = 0;
    virtual int autotune_apply_cached() = 0;       // take this N's recorded schedule
    virtual int autotune_report(double out[4]) = 0; // {warp path, carveout, best ms, default ms}
    // index-check flag of a bounds-checked build (-DCCMSAV_BOUNDS), read and cleared
    virtual int bounds_flag() = 0;
    int N = 0;
};

SimBase* make_sim_f32(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err);
SimBase* make_sim_f64(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err);

}  // namespace ccm
