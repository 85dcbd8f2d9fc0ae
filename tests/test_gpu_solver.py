"""GPU parity of the standalone spectral solver (Neumann DCT, Dirichlet DST,
periodic FFT) and of the initial-condition smoother of Appendix F, through
the C ABI, against the CPU oracle; then the smoothed sharp shapes of the
robustness runs stepped through the CC-MSAV step."""
import math

import numpy as np
import pytest

from oracle import ccmsav_oracle as O
from paper_2601_10057_gb300 import build as B
from paper_2601_10057_gb300 import ccmsav as cc
from paper_2601_10057_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BOUND = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return cc.load()


def dev(a, precision):
    import torch
    return torch.tensor(a, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", O.BCS)
@pytest.mark.parametrize("N", [8, 16, 64, 256, 1024])
def test_solver_against_oracle(N, bc, precision):
    """A random right-hand side, several line counts per CTA and the ragged
    smallest grids; FP64 within 1e-12 of the oracle's max-norm, FP32 within
    2e-5 (a few FP32 roundings per FFT stage)."""
    L = 1.7
    h = L / N
    coef = (0.0 if bc == "dirichlet" else 2.5, 0.3, 1e-4 * h * h)
    f = np.random.default_rng(N + 7 * O.BCS.index(bc)).standard_normal((N, N))
    s = cc.SpectralSolver(N, L, bc, precision)
    u = s.solve(coef, dev(f, precision))
    s.sync()
    ref = O.spectral_solve_bc(f, coef, h, bc)
    e = rel(host(u), ref)
    print(N, bc, precision, e)
    assert e <= BOUND[precision], e
    assert s.launches() == 3
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", O.BCS)
def test_solver_eigenmode_at_N8192(bc, precision):
    """The largest grid: a single eigenfunction of Lap_h with the boundary
    rule (a cosine, sine or periodic mode) is returned divided by
    c0 + c1 s + c2 s^2 (closed form), at every point; in place (u = f).
    The transforms' rounding noise lands on every mode and is divided by
    that mode's own factor (about 1 at the low modes), the signal by about
    80 here; with the reference's own cosines at arguments up to 4e3 the
    FP64 bound is 5e-11 (measured 3.4e-12 and 9.5e-12 in two cases)."""
    import torch
    N, L = 8192, 2.0
    h = L / N
    x = (torch.arange(N, dtype=torch.float64, device="cuda") + 0.5) * h
    k, l = 37, 1201
    if bc == "neumann":
        fx, fy = torch.cos(math.pi * k * x / L), torch.cos(math.pi * l * x / L)
        s_k, s_l = (4 / h ** 2 * math.sin(math.pi * q / (2 * N)) ** 2 for q in (k, l))
    elif bc == "dirichlet":
        fx, fy = torch.sin(math.pi * (k + 1) * x / L), torch.sin(math.pi * (l + 1) * x / L)
        s_k, s_l = (4 / h ** 2 * math.sin(math.pi * (q + 1) / (2 * N)) ** 2 for q in (k, l))
    else:
        fx, fy = torch.cos(2 * math.pi * k * x / L + 0.3), torch.cos(2 * math.pi * l * x / L - 1.1)
        s_k, s_l = (4 / h ** 2 * math.sin(math.pi * q / N) ** 2 for q in (k, l))
    f = torch.outer(fy, fx)
    coef = (1.0, 2e-5, 1e-12)
    s = s_k + s_l
    want = f / (coef[0] + coef[1] * s + coef[2] * s * s)
    g = f.clone() if precision == "fp64" else f.float()
    sol = cc.SpectralSolver(N, L, bc, precision)
    sol.solve(coef, g, out=g)
    sol.sync()
    e = float((g.double() - want).abs().max() / want.abs().max())
    print(bc, precision, e)
    assert e <= (5e-11 if precision == "fp64" else 5e-5), e
    sol.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", I.SHARP_SHAPES)
def test_smoother_against_oracle(shape, precision):
    """Appendix F on the sharp shapes at N = 256 (eps = 4 h, Mob = 0.01,
    dt = 1e-6, ten steps, then the clamp) against the oracle's smoother."""
    N, L = 256, 1.0
    h = L / N
    eps = 4 * h
    sharp = I.sharp_shape(shape, N, L)
    ref = O.smooth_initial(sharp, h, eps, 0.01, 1e-6, 10)
    s = cc.SpectralSolver(N, L, "neumann", precision)
    phi = dev(sharp, precision)
    s.smooth(phi, eps, 0.01, 1e-6, 10)
    s.sync()
    e = rel(host(phi), ref)
    print(shape, precision, e)
    assert e <= BOUND[precision], e
    assert np.abs(host(phi)).max() <= 1.0
    assert s.launches() == 10 * 4 + 1
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,grows", [("triangle", True), ("star", True), ("triangle", False),
                                         ("hexagon", False), ("star", False), ("crescent", False)])
def test_smoothed_shapes_step_with_conserved_mass(shape, grows, precision):
    """The robustness runs at reduced size: a smoothed sharp shape (growth or
    shrinkage column with the runs' (gamma_bend, theta)), N = 256, eps = 4 h,
    100 CC-MSAV steps at dt = 5e-6: the stored mass stays within 5e-11 of the
    initial mass and the modified energy does not increase over the BDF2 steps."""
    N, L = 256, 1.0
    h = L / N
    p = I.robustness_params(grows, N=N, L=L, eps=4 * h, dt=5e-6)
    s = cc.SpectralSolver(N, L, "neumann", "fp64")
    phi_t = dev(I.sharp_shape(shape, N, L), "fp64")
    s.smooth(phi_t, p.eps, 0.01, 1e-6, 10)
    s.sync()
    phi0 = host(phi_t)
    s.close()
    psi0 = I.concentration([phi0], [1.3 if grows else 0.8])
    m0 = h * h * math.fsum(psi0.ravel().tolist())
    sim = cc.Simulation(p, N, precision=precision, track_energy=True)
    sim.set_state(phi0, psi0)
    sim.step(1)
    E = []
    for _ in range(10):
        sim.step(10)
        E.append(sim.energy()[0])
        drift = abs(sim.mass() - m0) / abs(m0)
        assert drift < 5e-11, drift
    print(shape, grows, precision, "E", E[0], E[-1])
    if precision == "fp64":
        assert all(b <= a + 1e-12 * abs(a) for a, b in zip(E, E[1:])), E
    sim.close()


@pytest.mark.slow
@pytest.mark.parametrize("shape", ["star", "crescent"])
def test_robustness_run_at_paper_size(shape):
    """Sec. 4.4 at full size: the smoothed star and crescent in the
    shrinkage setting ((gamma_bend, theta) = (0.1, 30), eps = 0.01,
    N = 2048 on the unit square, dt = 5e-6), 400 FP64 steps: the relative
    mass error stays below 5e-11, the modified energy does not increase and
    the arc length stays within 5 % of its initial value (the paper reports
    deviations below 3.5 % for its own, unstated, shapes; measured here
    3.5 % for the star and 3.1 % for the crescent)."""
    N, L = 2048, 1.0
    p = I.robustness_params(False, N=N, L=L)
    s = cc.SpectralSolver(N, L, "neumann", "fp64")
    phi_t = dev(I.sharp_shape(shape, N, L), "fp64")
    s.smooth(phi_t, p.eps, 0.01, 1e-6, 10)
    s.sync()
    phi0 = host(phi_t)
    s.close()
    psi0 = I.concentration([phi0], [0.8])
    h = L / N
    m0 = h * h * math.fsum(psi0.ravel().tolist())
    sim = cc.Simulation(p, N, track_energy=True)
    sim.set_state(phi0, psi0)
    sim.step(1)
    arc0 = sim.energy()[5]
    E, arcs = [], []
    for _ in range(8):
        sim.step(50)
        e = sim.energy()
        E.append(e[0])
        arcs.append(e[5])
        assert abs(sim.mass() - m0) / abs(m0) < 5e-11
    print(shape, "E", E[0], E[-1], "arc", arc0, min(arcs), max(arcs))
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(E, E[1:])), E
    assert max(abs(a - arc0) for a in arcs) <= 0.05 * arc0
    sim.close()
