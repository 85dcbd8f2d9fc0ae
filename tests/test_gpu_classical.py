"""The classical MSAV baseline on the GPU (CCMSAV_CLASSICAL: variable-
mobility Cahn-Hilliard solves by DCT-preconditioned conjugate gradients)
against the oracle's classical scheme (sparse direct solves), and against the
CC-MSAV step where the two schemes coincide (constant mobility)."""
import numpy as np
import pytest

from oracle import ccmsav_oracle as O
from paper_2601_10057_gb300 import build as B
from paper_2601_10057_gb300 import ccmsav as cc
from paper_2601_10057_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return cc.load()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def run_classical(w, nsteps, precision="fp64", rtol=1e-13, max_iter=400):
    sim = cc.Simulation(w.params, w.N, precision=precision, classical=True)
    sim.set_pcg(rtol, max_iter)
    sim.set_state(w.phi0, w.psi0)
    sim.step(nsteps)
    phi, psi = sim.state()
    aux, stats, mass = sim.aux(), sim.pcg_stats(), sim.mass()
    sim.close()
    return phi, psi, aux, stats, mass


@pytest.mark.parametrize("wl,N,steps", [("one_vesicle", 16, 4), ("one_vesicle", 64, 6),
                                        ("ellipse_shrink", 128, 6), ("ellipse_shrink", 256, 3)])
def test_classical_fp64_against_oracle(wl, N, steps):
    """FP64, conjugate gradients to a relative residual of 1e-13: fields within
    1e-10 of the oracle's sparse direct solves (the CG solution error is
    bounded by the residual times the operator's condition number, a few
    hundred here), SAVs within 1e-10, mass conserved to 1e-12."""
    w = I.workload(wl, N=N, dt=1e-5)
    phi, psi, aux, stats, mass = run_classical(w, steps)
    m = O.Model.from_params(w.N, w.params)
    s = O.run(O.initial_state(w.phi0, w.psi0, m), m, steps, classical=True)
    e = (rel(phi, s.phi), rel(psi, s.psi))
    savs = np.array([s.V, s.U, s.W, s.Z])
    scale = np.array([abs(s.V), abs(s.A), abs(s.W), abs(s.Z)])
    e_sav = float((np.abs(aux[:4] - savs) / scale).max())
    m0 = O.mass(w.psi0, m)
    print(wl, N, "classical fp64", e, e_sav, "pcg", stats)
    assert max(e) <= 1e-10 and e_sav <= 1e-10, (e, e_sav)
    assert abs(mass - m0) <= 1e-12 * abs(m0)
    assert 1 <= stats[0] <= 400


def test_classical_equals_cc_at_constant_mobility():
    """With M0 -> 0 (1e-12: the ABI takes 0 < M0 < 1) the classical step and
    the CC-MSAV step agree to the CG tolerance."""
    w = I.workload("ellipse_shrink", N=128, dt=1e-5)
    p = w.params.replace(M0=1e-12)
    wc = I.Workload(w.name, w.N, p, w.phi0, w.psi0, w.steps, w.precision)
    phi_c, psi_c, _, _, _ = run_classical(wc, 5)
    sim = cc.Simulation(p, w.N)
    sim.set_state(w.phi0, w.psi0)
    sim.step(5)
    phi, psi = sim.state()
    sim.close()
    e = (rel(phi_c, phi), rel(psi_c, psi))
    print("classical vs cc at M0=1e-12", e)
    assert max(e) <= 1e-10, e


def test_classical_fp32_against_fp64():
    """FP32 fields and transforms, CG to a relative residual of 1e-6: within
    1e-5 of the FP64 classical step after 5 steps."""
    w = I.workload("ellipse_shrink", N=256, dt=1e-5)
    p64, q64, _, _, _ = run_classical(w, 5)
    p32, q32, _, st32, _ = run_classical(w, 5, precision="fp32", rtol=1e-6)
    e = (rel(p32, p64), rel(q32, q64))
    print("classical fp32 vs fp64", e, st32)
    assert max(e) <= 1e-5, e


def test_pcg_settings_validated():
    w = I.workload("one_vesicle", N=16, dt=1e-5)
    sim = cc.Simulation(w.params, w.N)
    assert cc.ccmsav_set_pcg(sim.h, 1e-8, 50) == cc.CCMSAV_EINVAL      # not a classical handle
    assert cc.ccmsav_pcg_stats(sim.h, 0)[0] == cc.CCMSAV_EINVAL
    sim.close()
    sim = cc.Simulation(w.params, w.N, classical=True)
    assert cc.ccmsav_set_pcg(sim.h, 0.0, 50) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_set_pcg(sim.h, 1e-8, 0) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_set_pcg(sim.h, 1e-8, 50) == cc.CCMSAV_OK
    sim.close()
