#!/usr/bin/env python
"""Throughput benchmark of the CC-MSAV time step on GB300.

Workload: three seeded perturbed-circle vesicles on an N = 2048 grid
(FP32-bulk precision, dt = 1e-5), the configuration the throughput metric is
quoted on.  A "step" is one full CC-MSAV time step over the grid.  The
metric is grid-point-steps per second (N^2 per step), whole job over all
ranks.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank advances its own independent simulation
(replicas: the step has no data exchange between GPUs); the time is the
maximum over ranks.  ``--impl reference`` times the CPU FP64 oracle on the
host cores instead (rank 0 only), on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
# Field passes (N x N reads + writes) per launch of each step kernel as
# implemented (the stencil's 8 outputs are written and re-read by the row
# transform; the inverse-row kernel reads the four levels of the increment form).
PASSES = {
    "k_stencil": 12, "k_rowdct_T": 16, "k_coldct_gram": 15, "k_solve": 0,
    "k_comb_icolT": 9, "k_irow": 8,
}
# The dependency-minimal schedule of one step (40 field passes): its phases,
# the kernels that implement each phase here, and the phase's algorithmic
# passes (K1 reads 4 levels and writes 8 row-transformed fields; K2 reads 8
# and writes 7 spectra; K4 reads 7 and writes 2; K5 reads 2 and writes 2).
PHASES = {
    "K1 stencil + row DCT": (("k_stencil", "k_rowdct_T"), 12),
    "K2 column DCT + Gram": (("k_coldct_gram",), 15),
    "K3 5x5 solve": (("k_solve",), 0),
    "K4 recovery + inverse column DCT": (("k_comb_icolT",), 9),
    "K5 inverse row DCT": (("k_irow",), 4),
}
STEP_PASSES_MIN_SCHEDULE = sum(p for _, p in PHASES.values())   # 40
# FP64 step at N = 2048: FP64 operations per grid point and step (2 DFMA + DADD
# + DMUL thread instructions of the six step kernels, one ncu capture) and the
# nominal FP64 peak, 152 SMs x 2 FP64 FMA/clock x 2 x 2.07 GHz
FP64_FLOP_PER_POINT_N2048 = 1042.0
FP64_PEAK_TFLOPS = 1.25
# Files holding the step kernels' device code (the DRAM traffic of a
# committed ncu capture stays valid while these are unchanged)
KERNEL_SOURCES = ("bounds.cuh", "dct_device.cuh", "step_kernels.cuh", "warp_fft.cuh", "warp_kernels.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=2048)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--accuracy-steps", type=int, default=1000,
                    help="steps of the FP32-vs-FP64 accuracy run on the headline workload")
    ap.add_argument("--dct-sweep", action="store_true",
                    help="only the sweep over N of the line-transform kernels (warp path) and of the "
                         "step with the warp-FFT against the block-FFT kernels; one JSON line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary workloads (batch of 64, N=4096, N=8192)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def code_text(src):
    """C++/CUDA source without comments and with whitespace collapsed: what
    the compiler sees, so that editing a comment keeps a profile's key."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return re.sub(r"\s+", " ", src).strip()


def source_hash():
    """Hash of the step kernels' code (comments and layout ignored)."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2601_10057_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f not in KERNEL_SOURCES:
            continue
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(f.encode() + code_text(fh.read()).encode())
    return h.hexdigest()[:12]


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None if missing or taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != source_hash():
            return None
        return d["workloads"][workload][kernel]["dram_bytes_per_launch"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed regions."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smmax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smmax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def aggregate(local_seconds, local_units, world):
    """Whole-job throughput: sum of units over ranks / max time over ranks."""
    if world == 1:
        return local_units / local_seconds, local_seconds, local_units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


ORACLE_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
from oracle import ccmsav_oracle as O
from paper_2601_10057_gb300 import inputs as I
kind = sys.argv[5] if len(sys.argv) > 5 else "three_vesicles"
w = (I.three_vesicles(N=int(sys.argv[2]), seed=int(sys.argv[3])) if kind == "three_vesicles"
     else I.workload(kind, N=int(sys.argv[2])))
seconds = float(sys.argv[4])
m = O.Model.from_params(w.N, w.params)
s = O.step(O.initial_state(w.phi0, w.psi0, m), m)   # the BDF1 start step, untimed
n, t0 = 0, time.perf_counter()
while True:
    s = O.step(s, m)
    n += 1
    el = time.perf_counter() - t0
    if el >= seconds:
        break
print(json.dumps({"value": w.N * w.N * n / el, "steps": n, "seconds": el}))
"""


def cpu_oracle_sample(N, seed, seconds, threads=None, kind="three_vesicles"):
    """Time the FP64 oracle (as it stands) on the host cores in a child
    process (no GPU use): all cores, or `threads` BLAS/OpenMP threads."""
    env = dict(os.environ)
    if threads:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", ORACLE_SAMPLE, ROOT, str(N), str(seed), str(seconds), kind],
                       capture_output=True, text=True, env=env, timeout=20 * seconds + 600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def accuracy_vs_fp64(ws, steps, sh):
    """FP32-bulk against the FP64 GPU path (which matches the oracle to
    1e-12) after `steps` steps from the same initial states: phi and psi
    max-abs error relative to the FP64 field's max-norm and RMS error
    relative to its RMS (maxima over the simulations), and the relative
    drift of the stored mass h^2 sum psi in both precisions."""
    import numpy as np
    from paper_2601_10057_gb300 import ccmsav as cc
    out = {}
    for prec in ("fp64", "fp32"):
        sim = cc.Simulation(None if len(ws) > 1 else ws[0].params, [w.N for w in ws],
                            per_sim=[w.params for w in ws] if len(ws) > 1 else None, precision=prec, stream=sh)
        for j, w in enumerate(ws):
            sim.set_state(w.phi0, w.psi0, sim=j)
        sim.step(steps)
        sim.sync()
        out[prec] = [(*sim.state(sim=j), sim.mass(sim=j)) for j in range(len(ws))]
        sim.close()
    e = {"steps": steps, "phi_max": 0.0, "phi_l2": 0.0, "psi_max": 0.0, "psi_l2": 0.0,
         "mass_drift_fp32": 0.0, "mass_drift_fp64": 0.0}
    for j, w in enumerate(ws):
        (p64, q64, m64), (p32, q32, m32) = out["fp64"][j], out["fp32"][j]
        m0 = (w.params.L / w.N) ** 2 * math.fsum(w.psi0.ravel().tolist())
        e["phi_max"] = max(e["phi_max"], float(np.abs(p32 - p64).max() / np.abs(p64).max()))
        e["psi_max"] = max(e["psi_max"], float(np.abs(q32 - q64).max() / np.abs(q64).max()))
        e["phi_l2"] = max(e["phi_l2"], float(np.sqrt(np.mean((p32 - p64) ** 2) / np.mean(p64 ** 2))))
        e["psi_l2"] = max(e["psi_l2"], float(np.sqrt(np.mean((q32 - q64) ** 2) / np.mean(q64 ** 2))))
        e["mass_drift_fp32"] = max(e["mass_drift_fp32"], abs(m32 - m0) / abs(m0))
        e["mass_drift_fp64"] = max(e["mass_drift_fp64"], abs(m64 - m0) / abs(m0))
    e = {k: (float(f"{v:.3g}") if isinstance(v, float) else v) for k, v in e.items()}
    e["reference"] = "FP64 GPU path (itself within 1e-12 of the oracle)"
    return e


def bench_config(w, precision, world):
    """The config object of the JSON line (both arms carry the same one)."""
    return {"workload": f"three_vesicles_N{w.N}", "N": w.N, "precision":
            ("fp32-bulk/fp64-reductions" if precision == "fp32" else "fp64"),
            "dt": w.params.dt, "vesicles": 3, "parallelism": f"replicas{world}",
            "l2": "per-step working set > L2 (no flush needed)"}


def run_reference(args, world, rank):
    from paper_2601_10057_gb300 import inputs as I
    if rank != 0:
        return
    w = I.workload("three_vesicles", N=args.N)
    budget = 150.0
    t0 = time.perf_counter()
    from oracle import ccmsav_oracle as O
    m = O.Model.from_params(w.N, w.params)
    s = O.initial_state(w.phi0, w.psi0, m)
    s = O.step(s, m)
    t_one = time.perf_counter() - t0
    warm = max(1, min(args.warmup, int(60.0 / max(t_one, 1e-3))))   # the requested warm-up, within ~60 s
    for _ in range(warm):
        s = O.step(s, m)
    k = max(1, min(args.steps, int(budget / max(t_one, 1e-3))))
    t1 = time.perf_counter()
    for _ in range(k):
        s = O.step(s, m)
    el = time.perf_counter() - t1
    value = w.N * w.N * k / el
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "grid-point-steps/s", "value": value, "unit": "grid-point-steps/s",
        "n_gpus": args.gpus, "steps": k, "warmup": warm, "ms_per_step": 1e3 * el / k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(w, args.precision, world),
        "cpu_baseline": {"value": value, "unit": "grid-point-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{k} BDF2 steps of the FP64 CPU oracle at N={w.N} (of {args.steps} "
                                   f"requested; bounded to ~{budget:.0f} s), after {warm} warm-up step(s)"},
        "e2e": {"value": value, "unit": "grid-point-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def extra_workloads(sh, stream):
    """Batching form (64 simulations of N in {128, 256, 512} in one handle:
    one stream each or one launch per kernel for a group of simulations of
    the same N, BDF2 steps from one graph for the batch) and the larger
    single grids (N = 4096 three vesicles, N = 8192 sixteen vesicles), FP32,
    device-timed with events on the caller's stream after 6 warm-up steps."""
    import torch
    from paper_2601_10057_gb300 import ccmsav as cc
    from paper_2601_10057_gb300 import inputs as I

    def run(ws, k, tune=False):
        sim = cc.Simulation(None if len(ws) > 1 else ws[0].params, [w.N for w in ws],
                            per_sim=[w.params for w in ws] if len(ws) > 1 else None,
                            precision="fp32", stream=sh)
        for j, w in enumerate(ws):
            sim.set_state(w.phi0, w.psi0, sim=j)
        sim.step(6)
        sim.sync()
        tuned = None
        if tune:   # the autotuner's schedule per grid size, before the timed steps
            rep = sim.autotune(12)
            tuned = {}
            for w, r in zip(ws, rep):
                tuned.setdefault(str(w.N), {"path": "warp" if r[0] else "block", "carveout": int(r[1]),
                                            "best_ms_per_step": round(float(r[2]), 4),
                                            "default_ms_per_step": round(float(r[3]), 4)})
            tuned["launch_group_points"] = sim.group_points()
        l0 = sim.launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        secs = e0.elapsed_time(e1) / 1e3
        pts = sum(w.N * w.N for w in ws)
        out = {"value": pts * k / secs, "unit": "grid-point-steps/s", "ms_per_step": 1e3 * secs / k,
               "steps": k, "points_per_step": pts, "gpu_launches": sim.launches() - l0}
        if tuned:
            out["autotune"] = tuned
        sim.close()
        return out

    res = {}
    for name, make, k, ka in (("batch64_N128-512", lambda: I.batch_64(), 60, 200),
                              ("three_vesicles_N4096", lambda: [I.three_vesicles(N=4096)], 30, 100),
                              ("lattice16_N8192", lambda: [I.lattice_16(N=8192)], 12, 20)):
        try:
            ws = make()
            res[name] = run(ws, k, tune=len(ws) > 1)
            res[name]["accuracy"] = accuracy_vs_fp64(ws, ka, sh)
            if len(ws) > 1:
                res[name]["sizes"] = {str(n): sum(1 for w in ws if w.N == n) for n in sorted({w.N for w in ws})}
        except Exception as e:             # reported, not fatal: the headline line still prints
            res[name] = {"error": str(e)}
    return res


def classical_comparison(sh, stream, N=2048, steps=10):
    """The paper's structural comparison (Sec. 3.5.2) on this GPU: the same
    workload stepped by CC-MSAV (DCT solves for both subsystems) and by the
    classical MSAV scheme (its variable-mobility Cahn-Hilliard operator by
    DCT-preconditioned conjugate gradients, the Allen-Cahn part as in
    CC-MSAV), device-timed after 3 warm-up steps; both precisions."""
    import torch
    from paper_2601_10057_gb300 import ccmsav as cc
    from paper_2601_10057_gb300 import inputs as I
    w = I.three_vesicles(N=N)
    out = {"workload": f"three_vesicles_N{N}", "steps": steps}
    for prec in ("fp64", "fp32"):
        rec = {}
        for kind in ("cc", "classical"):
            sim = cc.Simulation(w.params, N, precision=prec, stream=sh, classical=(kind == "classical"))
            sim.set_state(w.phi0, w.psi0)
            sim.step(3)
            sim.sync()
            it0 = sim.pcg_stats()[1] if kind == "classical" else 0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            sim.sync()
            rec[kind + "_ms_per_step"] = round(e0.elapsed_time(e1) / steps, 4)
            if kind == "classical":
                st = sim.pcg_stats()
                rec["pcg_iterations_per_step"] = round((st[1] - it0) / steps, 2)
                rec["pcg_rtol"] = 1e-10 if prec == "fp64" else 1e-6
            sim.close()
        rec["cc_speedup"] = round(rec["classical_ms_per_step"] / rec["cc_ms_per_step"], 2)
        out[prec] = rec
    out["note"] = ("classical steps launch directly and read the convergence flags every four iterations; "
                   "they also run the CC step's spectral psi work that the classical recovery then replaces")
    return out


ALG_BYTES_FP32 = {"k_rowdct_T": 64, "k_coldct_gram": 60, "k_comb_icolT": 36, "k_irow": 32}


def phase_roofline(per_launch, NN, esize, peak, peak_kind, workload):
    """Roofline of the dominant phase of the 40-pass schedule: the phase's
    algorithmic bytes per step (its passes x N^2 x element size) over the
    summed event times of the kernels that implement it, against the measured
    copy bandwidth; traffic = the ncu DRAM bytes of those kernels per step
    (null when the committed capture is of other kernel sources)."""
    times = {ph: sum(per_launch[k] for k in ks) for ph, (ks, _) in PHASES.items()}
    dom = max((ph for ph in PHASES if PHASES[ph][1] > 0), key=lambda ph: times[ph])
    ks, passes = PHASES[dom]
    alg = passes * NN * esize
    achieved = alg / (times[dom] * 1e-3) / 1e9
    tr = [ncu_traffic(k, workload) for k in ks]
    traffic = sum(tr) if all(t is not None for t in tr) else None
    step_tr = [ncu_traffic(k, workload) for k in PASSES]
    step_traffic = sum(step_tr) if all(t is not None for t in step_tr) else None
    phases = {ph: {"us": round(1e3 * times[ph], 2), "alg_passes": p,
                   "frac": (round(p * NN * esize / (times[ph] * 1e-3) / 1e9 / peak, 4) if p and times[ph] > 0 else None)}
              for ph, (_, p) in PHASES.items()}
    return {"bound": "hbm", "unit": "GB/s", "phase": dom, "kernels": list(ks),
            "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
            "frac": round(achieved / peak, 4), "traffic": traffic, "alg_bytes_per_launch": alg,
            "traffic_ratio_step": (round(step_traffic / (STEP_PASSES_MIN_SCHEDULE * NN * esize), 3)
                                   if step_traffic else None),
            "phases": phases,
            "timing": "per-kernel CUDA events recorded between the kernels of traced steps (direct launches, "
                      "no graph); their sum exceeds the graph-launched step time by the gaps between launches"}


def dct_sweep():
    """Per N (128 .. 8192, FP32): the line-transform kernels' event times and
    algorithmic GB/s on the warp-FFT path, and the step time with the
    warp-FFT kernels against the block-FFT kernels (the library takes the
    warp path wherever it exists)."""
    import torch
    from paper_2601_10057_gb300 import build as B
    from paper_2601_10057_gb300 import ccmsav as cc
    from paper_2601_10057_gb300 import inputs as I
    B.build()
    cc.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    peak, peak_kind = measured_peaks()
    rows = []
    for N in (128, 256, 512, 1024, 2048, 4096, 8192):
        w = I.three_vesicles(N=N) if N >= 1024 else I.workload("ellipse_shrink", N=N)
        k = 300 if N <= 512 else (100 if N <= 2048 else (30 if N <= 4096 else 9))
        rec = {"N": N, "steps": k}
        for path in ("warp", "block"):
            os.environ["CCMSAV_FORCE_BLOCK_FFT"] = "1" if path == "block" else "0"
            sim = cc.Simulation(w.params, N, precision="fp32", stream=sh)
            sim.set_state(w.phi0, w.psi0)
            sim.step(6)
            sim.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            sim.sync()
            rec[path + "_ms_per_step"] = round(e0.elapsed_time(e1) / k, 5)
            if path == "warp":
                cc.ccmsav_profile(sim.h, True)
                sim.step(min(k, 60))
                _, ms, nst = cc.ccmsav_profile_read(sim.h, 0)
                cc.ccmsav_profile(sim.h, False)
                sim.sync()
                kern = {}
                for i, name in enumerate(cc.KERNEL_NAMES):
                    if name in ALG_BYTES_FP32 and nst:
                        t = ms[i] / nst
                        gbs = ALG_BYTES_FP32[name] * N * N / (t * 1e-3) / 1e9
                        kern[name] = {"us": round(1e3 * t, 2), "alg_GBps": round(gbs, 1), "frac": round(gbs / peak, 3)}
                rec["transforms"] = kern
            sim.close()
        rec["warp_speedup"] = round(rec["block_ms_per_step"] / rec["warp_ms_per_step"], 2)
        rows.append(rec)
    os.environ.pop("CCMSAV_FORCE_BLOCK_FFT", None)
    print(json.dumps({"dct_sweep": rows, "peak_GBps": peak, "peak_kind": peak_kind, "precision": "fp32",
                      "workloads": "ellipse_shrink (N <= 512), three_vesicles (N >= 1024)"}), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2601_10057_gb300 import build as B
    from paper_2601_10057_gb300 import ccmsav as cc
    from paper_2601_10057_gb300 import inputs as I

    B.build()
    cc.load()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()          # a dedicated stream: the library captures CUDA graphs on it
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    w = I.three_vesicles(N=args.N, seed=1003 + rank, precision=args.precision)
    NN = w.N * w.N
    esize = 4 if args.precision == "fp32" else 8

    def make(prec):
        sim = cc.Simulation(w.params, w.N, precision=prec, stream=sh)
        sim.set_state(w.phi0, w.psi0)
        return sim

    clocks = ClockSampler(local)
    sim = make(args.precision)
    sim.step(max(args.warmup, 3))
    sim.sync()
    # ---- timed region: K steps, device events on the launching stream
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    l0 = sim.launches()
    # five windows with an event between them (each a multiple of three steps
    # but the last, so the same graphs run as for one call of K steps); the
    # value is the whole region, the windows give the median per-step time
    nwin = 5 if args.steps >= 30 else 1
    base = (args.steps // nwin) // 3 * 3
    sizes = [base] * (nwin - 1) + [args.steps - base * (nwin - 1)]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(nwin + 1)]
    evs[0].record(stream)
    for i, kw in enumerate(sizes):
        sim.step(kw)
        evs[i + 1].record(stream)
    e0, e1 = evs[0], evs[-1]
    torch.cuda.synchronize()
    barrier(world)
    secs = e0.elapsed_time(e1) / 1e3
    win_ms = [evs[i].elapsed_time(evs[i + 1]) / kw for i, kw in enumerate(sizes)]
    launches = sim.launches() - l0
    sim.sync()
    value, tmax, units = aggregate(secs, NN * args.steps, world)
    # ---- per-kernel device times (second pass with event marks between kernels)
    kprof = min(args.steps, 200)
    cc.ccmsav_profile(sim.h, True)
    sim.step(kprof)
    st, ms, nst = cc.ccmsav_profile_read(sim.h, 0)
    cc.ccmsav_profile(sim.h, False)
    sim.sync()
    per_launch = {cc.KERNEL_NAMES[i]: ms[i] / max(nst, 1) for i in (0, 1, 2, 3, 4, 5)}
    peak, peak_kind = measured_peaks()
    roof = phase_roofline(per_launch, NN, esize, peak, peak_kind, f"three_vesicles_N{w.N}_{args.precision}")
    kernels = {k: {"ms_per_launch": round(v, 5), "share": round(v / sum(per_launch.values()), 4),
                   "impl_passes": PASSES[k],
                   "impl_GBps": (round(PASSES[k] * NN * esize / (v * 1e-3) / 1e9, 1) if v > 0 and PASSES[k] else None)}
               for k, v in per_launch.items()}
    sim.close()
    # ---- FP64 step on the same workload (secondary)
    fp64 = None
    if not args.no_fp64 and args.precision == "fp32":
        s64 = make("fp64")
        s64.step(3)
        s64.sync()
        k64 = min(args.steps, 60)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.step(k64)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = f0.elapsed_time(f1) / 1e3
        s64.sync()
        s64.close()
        fp64 = {"value": NN * k64 / t64, "ms_per_step": 1e3 * t64 / k64, "steps": k64,
                "speedup_fp32_over_fp64": (NN * args.steps / secs) / (NN * k64 / t64)}
        if w.N == 2048:
            ach = FP64_FLOP_PER_POINT_N2048 * NN * k64 / t64 / 1e12     # t64: seconds for k64 steps
            fp64["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": round(ach, 3),
                                "peak": FP64_PEAK_TFLOPS, "peak_kind": "nominal FP64 (152 SMs x 2 DFMA/clk x 2 x 2.07 GHz)",
                                "frac": round(ach / FP64_PEAK_TFLOPS, 3),
                                "flop_per_point": FP64_FLOP_PER_POINT_N2048,
                                "hbm_frac": round(2289e6 * k64 / t64 / 1e9 / measured_peaks()[0], 4)}
    # ---- accuracy of the timed precision against the FP64 GPU path (1000 steps: the precision target)
    acc = None
    if args.precision == "fp32" and not args.no_fp64 and rank == 0 and args.accuracy_steps > 0:
        acc = accuracy_vs_fp64([w], args.accuracy_steps, sh)
    # ---- the method's other workloads, device-timed (secondary lines)
    extra = None
    if not args.no_extra and rank == 0 and world == 1 and args.precision == "fp32":
        extra = extra_workloads(sh, stream)
        try:
            extra["classical_vs_cc"] = classical_comparison(sh, stream, N=w.N)
        except Exception as e:             # reported, not fatal
            extra["classical_vs_cc"] = {"error": str(e)}
    # ---- end to end through the C ABI with pinned host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory().numpy()
    phi_h, psi_h = pin(w.phi0), pin(w.psi0)
    out_phi, out_psi = pin(np.zeros_like(w.phi0)), pin(np.zeros_like(w.psi0))
    e2e_sim = cc.Simulation(w.params, w.N, precision=args.precision, stream=sh)
    e2e_sim.set_state(phi_h, psi_h)
    e2e_sim.step(3)
    e2e_sim.sync()
    k_e2e = min(args.steps, 200)
    barrier(world)
    torch.cuda.synchronize()
    aux_h = torch.zeros((k_e2e, 12), dtype=torch.float64).pin_memory().numpy()
    t0 = time.perf_counter()
    e2e_sim.set_state(phi_h, psi_h)
    for j in range(k_e2e):
        e2e_sim.step(1)
        e2e_sim.aux_async(aux_h[j])          # every step's scalars to the host, without a stall
    st = cc.load().ccmsav_get_state(e2e_sim.h, 0, cc._ptr(out_phi), cc._ptr(out_psi))
    t_e2e = time.perf_counter() - t0
    if st != cc.CCMSAV_OK or [int(a[10]) for a in aux_h] != list(range(1, k_e2e + 1)):
        raise RuntimeError("end-to-end run: a step's scalars did not come back")
    barrier(world)
    clk = clocks.stop()
    e2e_sim.close()
    e2e_value, _, _ = aggregate(t_e2e, NN * k_e2e, world)
    h2d = 2 * NN * 8 / k_e2e
    d2h = 12 * 8 + 2 * NN * 8 / k_e2e
    # ---- CPU baseline (oracle on the host cores, rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        seed = 1003 + rank
        allc = cpu_oracle_sample(w.N, seed, args.cpu_seconds)
        one = cpu_oracle_sample(w.N, seed, args.cpu_seconds, threads=1)
        cpu = {"value": allc["value"], "unit": "grid-point-steps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{allc['steps']} BDF2 step(s) of the FP64 CPU oracle on the same N={w.N} workload "
                         f"({allc['seconds']:.1f} s; numpy with OpenBLAS on all {os.cpu_count()} host cores; "
                         f"its DCT is the O(N^3) cosine-matrix product, O(N) per coefficient)",
               "one_thread": {"value": one["value"], "cores": 1,
                              "sample": f"{one['steps']} BDF2 step(s), {one['seconds']:.1f} s, "
                                        "OPENBLAS_NUM_THREADS=OMP_NUM_THREADS=1"},
               "complexity": "O(N^3) per 2D transform (cosine-matrix DCT), 14 one-way transforms per step"}
        # the oracle at the small configurations' sizes too (where it runs whole workloads)
        per = {}
        for n_s, kind in ((64, "one_vesicle"), (512, "ellipse_shrink")):
            sec = min(args.cpu_seconds, 3.0)
            a = cpu_oracle_sample(n_s, seed, sec, kind=kind)
            o = cpu_oracle_sample(n_s, seed, sec, threads=1, kind=kind)
            per[f"{kind}_N{n_s}"] = {"all_cores": round(a["value"]), "one_thread": round(o["value"]),
                                     "ms_per_step_all_cores": round(1e3 * a["seconds"] / a["steps"], 2),
                                     "ms_per_step_one_thread": round(1e3 * o["seconds"] / o["steps"], 2),
                                     "unit": "grid-point-steps/s"}
        cpu["other_sizes"] = per
    if rank != 0:
        return
    line = {
        "metric": "grid-point-steps/s", "value": value, "unit": "grid-point-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": bench_config(w, args.precision, world),
        "timing_windows": {"steps": sizes, "ms_per_step": [round(x, 5) for x in win_ms],
                           "median_ms_per_step": round(sorted(win_ms)[len(win_ms) // 2], 5),
                           "what": "this rank's timed region split by events into windows (value and ms_per_step "
                                   "cover the whole region)"},
        "roofline": roof,
        "step_roofline": {"alg_bytes_per_point": STEP_PASSES_MIN_SCHEDULE * esize,
                          "achieved_GBps": round(value / world * STEP_PASSES_MIN_SCHEDULE * esize / 1e9, 1),
                          "peak": peak, "frac": round(value / world * STEP_PASSES_MIN_SCHEDULE * esize / 1e9 / peak, 4),
                          "floor_frac": round(value / world * 6 * esize / 1e9 / peak, 4),
                          "what": "whole step against the 40-pass dependency-minimal schedule (160 B/pt FP32); "
                                  "floor_frac against the 6-pass floor (read 4 levels, write 2)"},
        "kernels": kernels,
        "fp64": fp64,
        "accuracy": acc,
        "workloads": extra,
        "e2e": {"value": e2e_value, "unit": "grid-point-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": k_e2e,
                "what": "set_state from pinned host FP64 arrays, per step ccmsav_step(1) + ccmsav_get_aux_async "
                        "(each step's twelve scalars copied to pinned host memory, checked after the run), final "
                        "ccmsav_get_state to pinned host arrays"},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.dct_sweep:
        if rank == 0:
            dct_sweep()
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
