"""Run a few CC-MSAV steps of one workload with direct kernel launches (the
handle's tracing mode), for profilers such as ncu that capture individual
launches:

  python -m paper_2601_10057_gb300.profile_step N {fp32,fp64} STEPS [classical]

The workload is the three-vesicle one for N >= 1024 and the shrinking
ellipse below; the start step runs first, then STEPS BDF2 steps, so each
step kernel launches 1 + STEPS times."""
import sys

from . import build as B
from . import ccmsav as cc
from . import inputs as I


def main(argv):
    N, prec, steps = int(argv[0]), argv[1], int(argv[2])
    classical = len(argv) > 3 and argv[3] == "classical"
    B.build()
    cc.load()
    w = I.three_vesicles(N=N) if N >= 1024 else I.workload("ellipse_shrink", N=N)
    sim = cc.Simulation(w.params, N, precision=prec, classical=classical)
    sim.set_state(w.phi0, w.psi0)
    cc.ccmsav_profile(sim.h, True)
    sim.step(1 + steps)
    sim.sync()
    print("ok", N, prec, steps, sim.launches())
    sim.close()


if __name__ == "__main__":
    main(sys.argv[1:])
