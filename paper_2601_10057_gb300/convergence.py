"""Convergence studies of the CC-MSAV step on the GPU (Sec. 4.1 of the
paper): temporal (Cauchy errors at a fixed grid), spatial (successive grids at
a small fixed step) and the refinement path dt = C h, all at final time
T = 5e-3, run through the C ABI.  The refinement path takes C = 0.0005 (the
paper's 0.002 with this ellipse and stiffness puts the coarse levels at
steps above 3e-6, where the temporal study shows the error is not yet in
its asymptotic range).  Errors between grids restrict the finer
solution to the coarser cell centres with the 4-point Lagrange stencil
(-1, 9, 9, -1)/16 per axis (the paper interpolates with cubics; a coarse
centre is the midpoint of two fine centres, and this stencil is the cubic
through the four nearest fine values), with mirrored ghosts at the walls.

  python -m paper_2601_10057_gb300.convergence [--precision fp64] [--out FILE]

prints (and writes) one JSON object with the errors and rates."""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import ccmsav as cc
from . import inputs as I

T_FINAL = 5e-3


def restrict(u: np.ndarray) -> np.ndarray:
    """Fine field (2N x 2N) to the N x N coarse centres."""
    def along(v, axis):
        v = np.moveaxis(v, axis, 0)
        g = np.concatenate([v[:1], v, v[-1:]], axis=0)
        i = np.arange(0, v.shape[0], 2)
        return np.moveaxis((-g[i] + 9 * g[i + 1] + 9 * g[i + 2] - g[i + 3]) / 16.0, 0, axis)
    return along(along(u, 0), 1)


def l2(u: np.ndarray, h: float) -> float:
    return math.sqrt(h * h * float(np.sum(u * u)))


def run(N: int, dt: float, precision: str):
    w = I.convergence_ellipse(N, dt=dt)
    n = int(round(T_FINAL / dt))
    sim = cc.Simulation(w.params, N, precision=precision)
    sim.set_state(w.phi0, w.psi0)
    sim.step(n)
    phi, psi = sim.state()
    sim.close()
    return phi, psi, w.params.L / N, n


def rates(errs):
    return [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]


def study(kind: str, precision: str = "fp64", Ns=(128, 256, 512, 1024, 2048), N_time: int = 512,
          dts=(5e-6, 2.5e-6, 1.25e-6, 6.25e-7, 3.125e-7), C: float = 0.0005, dt_space: float = 1e-6):
    """One of "temporal", "spatial", "refinement"; returns a dict with the
    per-level errors of phi, psi and the combined error, and their rates."""
    levels = []
    if kind == "temporal":
        sols = [run(N_time, dt, precision) for dt in dts]
        for k in range(len(dts) - 1):
            a, b = sols[k], sols[k + 1]
            levels.append({"N": N_time, "dt": dts[k], "steps": a[3],
                           "phi": l2(a[0] - b[0], a[2]), "psi": l2(a[1] - b[1], a[2])})
    else:
        sols = {}
        for N in Ns:
            dt = C / N if kind == "refinement" else dt_space      # dt = C h with L = 1
            sols[N] = run(N, dt, precision)
        for N in Ns[:-1]:
            a, b = sols[N], sols[2 * N]
            levels.append({"N": N, "dt": C / N if kind == "refinement" else dt_space, "steps": a[3],
                           "phi": l2(a[0] - restrict(b[0]), a[2]), "psi": l2(a[1] - restrict(b[1]), a[2])})
    for lv in levels:
        lv["combined"] = math.hypot(lv["phi"], lv["psi"])
    out = {"study": kind, "precision": precision, "T": T_FINAL, "levels": levels}
    for key in ("phi", "psi", "combined"):
        out["rate_" + key] = rates([lv[key] for lv in levels])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--studies", default="temporal,spatial,refinement")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import build as B
    B.build()
    cc.load()
    res = {"workload": "convergence ellipse (semi-axes 0.3, 0.2, L = 1, eps = 0.03125, "
                       "(gamma_in, gamma_out, gamma_area) = (100, 100, 100), shrinkage column)",
           "studies": [study(k, args.precision) for k in args.studies.split(",")]}
    txt = json.dumps(res, indent=1)
    print(txt)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
