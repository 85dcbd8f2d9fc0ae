"""The step with every field, spectrum and level access index-checked: the
library built with -DCCMSAV_BOUNDS (libccmsav_bounds.so) runs the small and
ragged grids (N = 8 ... 256, FP64 and FP32, block- and warp-FFT paths, start
and BDF2 steps, graph-launched steps, the classical and BDF1 modes, a batched
handle with grouped launches; and N = 4096, 8192 on the two-warp-line kernels) in a
child process; no access may leave its array (ccmsav_bounds_flag() = 0) and
the results stay those of the oracle (the shrinking ellipse: the single
perturbed circle at N = 256 amplifies a 1e-10 perturbation to 1e-5 within
50 steps, too sensitive for an FP32 comparison).  compute-sanitizer is not available
for this purpose, so the checks are compiled into the kernels."""
import json
import os
import subprocess
import sys

import pytest

from paper_2601_10057_gb300 import build as B

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2601_10057_gb300 import ccmsav as cc
from paper_2601_10057_gb300 import inputs as I
from oracle import ccmsav_oracle as O
cc.load(cc.LIB_BOUNDS_PATH)
out = []
cases = [(N, prec, mode) for N in (8, 16, 32, 64, 128, 256) for prec in ("fp64", "fp32")
         for mode in ("cc", "bdf1", "classical")]
for N, prec, mode in cases:
    w = I.workload("ellipse_shrink", N=N)
    sim = cc.Simulation(w.params, N, precision=prec, bdf1_always=(mode == "bdf1"), classical=(mode == "classical"))
    if mode == "classical":
        sim.set_pcg(1e-13 if prec == "fp64" else 1e-6, 400)
    sim.set_state(w.phi0, w.psi0)
    sim.step(1)
    sim.step(7)          # graph-launched BDF2 steps (direct for the classical mode)
    phi, psi = sim.state()
    flag = cc.ccmsav_bounds_flag(sim.h)
    sim.close()
    m = O.Model.from_params(N, w.params)
    s = O.run(O.initial_state(w.phi0, w.psi0, m), m, 8, bdf1=(True if mode == "bdf1" else None),
              classical=(mode == "classical"))
    e = max(float(np.abs(phi - s.phi).max() / np.abs(s.phi).max()), float(np.abs(psi - s.psi).max() / np.abs(s.psi).max()))
    out.append({"N": N, "precision": prec, "mode": mode, "flag": flag, "err": e})
# the FP32 warp path with lines over two warps (2048- and 4096-point lines),
# against FP64 on the GPU
for NB, w in ((4096, I.three_vesicles(N=4096)), (8192, I.lattice_16(N=8192))):
    res = {}
    for prec in ("fp64", "fp32"):
        sim = cc.Simulation(w.params, NB, precision=prec)
        sim.set_state(w.phi0, w.psi0)
        sim.step(1)
        sim.step(3)
        res[prec] = sim.state()
        flag = cc.ccmsav_bounds_flag(sim.h) if prec == "fp32" else 0
        sim.close()
    e = max(float(np.abs(res["fp32"][0] - res["fp64"][0]).max() / np.abs(res["fp64"][0]).max()),
            float(np.abs(res["fp32"][1] - res["fp64"][1]).max() / np.abs(res["fp64"][1]).max()))
    out.append({"N": NB, "precision": "fp32", "mode": "cc-vs-fp64", "flag": flag, "err": e})
# a batched handle with grouped launches (three N = 128 and two N = 256 FP32
# simulations sharing each kernel launch, an N = 64 one on its own), against
# each simulation run alone in the same library
ws = [I.workload("one_vesicle", N=128, dt=1e-5), I.workload("ellipse_shrink", N=128),
      I.workload("one_vesicle", N=128, dt=2e-5), I.workload("ellipse_shrink", N=256),
      I.workload("one_vesicle", N=256, dt=1e-5), I.workload("one_vesicle", N=64, dt=1e-5)]
sim = cc.Simulation(None, [x.N for x in ws], per_sim=[x.params for x in ws], precision="fp32")
for k, x in enumerate(ws):
    sim.set_state(x.phi0, x.psi0, sim=k)
sim.step(1)
sim.step(9)
got = [sim.state(sim=k) for k in range(len(ws))]
flag = cc.ccmsav_bounds_flag(sim.h)
sim.close()
e = 0.0
for k, x in enumerate(ws):
    solo = cc.Simulation(x.params, x.N, precision="fp32")
    solo.set_state(x.phi0, x.psi0)
    solo.step(10)
    a, b = solo.state()
    solo.close()
    e = max(e, float(np.abs(got[k][0] - a).max()), float(np.abs(got[k][1] - b).max()))
out.append({"N": 256, "precision": "fp32", "mode": "grouped-vs-solo", "flag": flag, "err": e})
print(json.dumps(out))
"""


def test_bounds_checked_build_small_grids():
    B.build(bounds=True)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for c in res:
        print(c)
    assert all(c["flag"] == 0 for c in res), [c for c in res if c["flag"]]
    tol = {"fp64": 1e-11, "fp32": 2e-5}      # N = 4096, 8192: FP32 against FP64 after 4 steps
    bad = [c for c in res if c["err"] > (0.0 if c["mode"] == "grouped-vs-solo" else tol[c["precision"]])]
    assert not bad, bad
