// sim.h -- precision-independent interface between the C ABI and the
// per-precision implementations of one simulation.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "../../include/ccmsav.h"

namespace ccm {

// Schedule chosen by the autotuner for one (grid size, precision): the FFT
// path of the line transforms (warp-level four-step FFT or CTA-level Stockham
// FFT) and the shared-memory carveout of the three 8-line warp-FFT kernels.
// Process-wide, so handles created later with the same N start from it.
struct TuneChoice { int warp = 1; int carveout = 72; double ms = 0.0, ms_default = 0.0; };
// Candidate schedules, the default first: warp-FFT kernels at carveouts of
// 72, 58 and 100 percent (where the warp path exists), then the block FFT.
inline std::vector<TuneChoice> tune_candidates(bool have_warp) {
    std::vector<TuneChoice> c;
    if (have_warp)
        for (int cv : {72, 58, 100}) { TuneChoice t; t.warp = 1; t.carveout = cv; c.push_back(t); }
    TuneChoice b; b.warp = 0; b.carveout = 72; c.push_back(b);
    return c;
}

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
    virtual int tune_save() = 0;                   // keep the state while schedules are timed
    virtual int tune_load() = 0;                   // back to the kept state
    virtual void tune_free() = 0;
    virtual bool tune_has_warp() const = 0;
    virtual int tune_apply(int warp, int carveout) = 0;
    virtual int tune_record(int warp, int carveout, double ms, double ms_default) = 0;
    virtual int autotune_apply_cached() = 0;       // take this N's recorded schedule
    virtual int autotune_report(double out[4]) = 0; // {warp path, carveout, best ms, default ms}
    // index-check flag of a bounds-checked build (-DCCMSAV_BOUNDS), read and cleared
    virtual int bounds_flag() = 0;
    // grouped launches: the BDF2 steps of several simulations of the same
    // line length from one launch per kernel (see BatchArgs in the kernels)
    virtual int group_key() const = 0;                 // line length M, or 0: not groupable
    virtual size_t batch_args_bytes() const = 0;       // size of one simulation's argument record
    virtual int fill_batch_args(int i, void* rec) const = 0;   // record of the i-th step (0..2) from now
    // queues three steps of the n simulations (2 <= n <= max_group()) whose
    // host records (three blocks of `stride` records, one per step) start at
    // recs; called on one member
    virtual int max_group() const = 0;
    virtual int queue_group_steps(const void* recs, int n, int stride, cudaStream_t s) = 0;
    virtual void count_steps_grouped(int n3) = 0;      // host counters after grouped steps
    int N = 0;
};

SimBase* make_sim_f32(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err);
SimBase* make_sim_f64(const ccmsav_params& p, int N, int flags, cudaStream_t s, int* err);

}  // namespace ccm
