"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64: every field and SAV within 1e-12 relative to the oracle's max-norm
(the target stated for the FP64 step) over short runs; the FFT-based DCT,
the spectral (Parseval) Gram sums and the oracle's cosine-matrix products and
physical inner products round differently, so results are not bit-identical.
Over hundreds of steps this stiff system amplifies any change of rounding
order: the oracle itself, with its DCT evaluated by scipy's FFT-based
routine instead of the cosine matrix, moves by 3.8e-12 (N = 64, 200 steps).
Long runs are therefore bounded by twice that measured spread of the oracle
(rounding_spread below), never by less than 1e-12.
FP32-bulk: within bounds derived from FP32 rounding (see each test).
"""
import math

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


def run_gpu(w, nsteps, precision="fp64", track=False, chunks=None):
    sim = cc.Simulation(w.params, w.N, precision=precision, track_energy=track)
    sim.set_state(w.phi0, w.psi0)
    for n in (chunks or [nsteps]):
        sim.step(n)
    sim.sync()
    phi, psi = sim.state()
    aux = sim.aux()
    return sim, phi, psi, aux


def run_oracle(w, nsteps):
    m = O.Model.from_params(w.N, w.params)
    s = O.initial_state(w.phi0, w.psi0, m)
    for _ in range(nsteps):
        s = O.step(s, m)
    return m, s


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def savs(s):
    return np.array([s.V, s.U, s.W, s.Z, s.V_old, s.U_old, s.W_old, s.Z_old])


def sav_err(sav, s):
    """SAV differences on the scale of each SAV (U, a small difference of
    O(A) quantities, on the scale of A)."""
    scale = np.array([abs(s.V), abs(s.A), abs(s.W), abs(s.Z)] * 2)
    return float((np.abs(np.asarray(sav) - savs(s)) / np.maximum(scale, 1e-300)).max())


def rounding_spread(w, nsteps, s_ref):
    """How far the oracle moves when only the rounding order of its DCT
    changes: the same oracle run with scipy's FFT-based orthonormal DCT in
    place of the cosine-matrix products.  Returns (phi, psi, sav) spreads."""
    import scipy.fft as sfft
    d2, i2 = O.dct2d, O.idct2d
    try:
        O.dct2d = lambda u: sfft.dctn(u, type=2, norm="ortho")
        O.idct2d = lambda U: sfft.idctn(U, type=2, norm="ortho")
        _, s2 = run_oracle(w, nsteps)
    finally:
        O.dct2d, O.idct2d = d2, i2
    return rel(s2.phi, s_ref.phi), rel(s2.psi, s_ref.psi), sav_err(savs(s2), s_ref)


def check_fp64(w, nsteps, tol=1e-12, spread=False):
    """GPU FP64 against the oracle: fields and SAVs within tol relative to
    the max-norm (SAVs on their own scale); with spread=True the bound of
    each quantity is max(tol, 2 x the oracle's own rounding spread)."""
    sim, phi, psi, aux = run_gpu(w, nsteps)
    m, s = run_oracle(w, nsteps)
    e_phi, e_psi, e_sav = rel(phi, s.phi), rel(psi, s.psi), sav_err(aux[:8], s)
    b_phi = b_psi = b_sav = tol
    msg = f"N={w.N} steps={nsteps} phi {e_phi:.3e} psi {e_psi:.3e} sav {e_sav:.3e}"
    if spread:
        r_phi, r_psi, r_sav = rounding_spread(w, nsteps, s)
        b_phi, b_psi, b_sav = max(tol, 2 * r_phi), max(tol, 2 * r_psi), max(tol, 2 * r_sav)
        msg += f" | oracle rounding spread phi {r_phi:.3e} psi {r_psi:.3e} sav {r_sav:.3e}"
    print(msg)
    assert e_phi <= b_phi and e_psi <= b_psi, msg
    assert e_sav <= b_sav, msg
    assert aux[10] == nsteps
    sim.close()
    return e_phi, e_psi


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128])
def test_fp64_bdf1_then_bdf2_small_grids(N):
    """Few steps at grids from the smallest (one tile, N = 8) to several tiles."""
    w = I.workload("one_vesicle", N=N, dt=1e-5)
    check_fp64(w, 4)


def test_fp64_start_step_only():
    w = I.workload("ellipse_shrink", N=64, dt=1e-5)
    check_fp64(w, 1)


def test_fp64_one_vesicle_N64_200_steps():
    """The small workload: one vesicle, N = 64, 200 steps at dt = 1e-4.
    Measured on GB300: phi 3.0e-12, psi 4.0e-13 against the oracle, while
    the oracle with another DCT rounding order moves by 3.8e-12 / 6.2e-13:
    the bound is twice that spread."""
    w = I.workload("one_vesicle", N=64)
    assert w.params.dt == 1e-4 and w.steps == 200
    check_fp64(w, 200, spread=True)


@pytest.mark.slow
def test_fp64_ellipse_N512_1000_steps():
    """The shrinking-ellipse workload at full length: N = 512, 1000 steps at
    dt = 1e-5 against the oracle, bounded by twice the oracle's own rounding
    spread over the same run (measured on GB300: GPU phi 5.1e-11, psi
    3.9e-11; the oracle takes about a minute per run on 16 Arm cores)."""
    w = I.workload("ellipse_shrink", N=512)
    assert w.params.dt == 1e-5 and w.steps == 1000
    check_fp64(w, 1000, spread=True)


@pytest.mark.slow
def test_fp64_lattice_N8192_two_steps():
    """The largest grid (sixteen vesicles, N = 8192, lines of 4096 complex
    values in the block FFT): the start step and the first BDF2 step against
    the oracle at every point, within 1e-12 (measured 6.4e-14; the oracle
    takes about two minutes on 16 Arm cores)."""
    w = I.workload("lattice16", N=8192)
    check_fp64(w, 2)


def test_fp64_ellipse_N256_30_steps():
    w = I.workload("ellipse_shrink", N=256)
    check_fp64(w, 30)


def test_fp64_three_vesicles_N2048_two_steps():
    """Full size of the throughput workload: the BDF1 start step and the
    first BDF2 step against the oracle at every grid point."""
    w = I.workload("three_vesicles", N=2048)
    check_fp64(w, 2)


def test_fp32_bulk_against_oracle_N128():
    """FP32 fields: per-step rounding of ~6e-8 relative, amplified by the
    stiff osmotic coupling over 20 steps; bound 2e-5 of the max-norm."""
    w = I.workload("ellipse_shrink", N=128)
    _, phi, psi, aux = run_gpu(w, 20, precision="fp32")
    _, s = run_oracle(w, 20)
    print("fp32 rel", rel(phi, s.phi), rel(psi, s.psi))
    assert rel(phi, s.phi) < 2e-5 and rel(psi, s.psi) < 2e-5


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_fp32_bulk_small_grids_block_fft(N):
    """The FP32 path on the grids below the warp-FFT kernels (N = 8 .. 64:
    block-level FFT lines of 4 .. 32 points, one tile up to a few tiles),
    BDF1 start then BDF2, 4 steps against the FP64 oracle, bound 5e-6 of the
    max-norm."""
    w = I.workload("one_vesicle", N=N, dt=1e-5)
    _, phi, psi, aux = run_gpu(w, 4, precision="fp32")
    _, s = run_oracle(w, 4)
    e = (rel(phi, s.phi), rel(psi, s.psi))
    print("fp32 block", N, e)
    assert max(e) < 5e-6, e


@pytest.mark.parametrize("N", [128, 256, 512, 1024, 2048])
def test_fp32_bulk_against_oracle_all_fft_shapes(N):
    """The FP32 path at every line length of its FFT kernels (N = 128 .. 2048):
    3 steps against the FP64 oracle, bound 5e-6 of the max-norm (a few FP32
    roundings per step through the transforms)."""
    w = I.workload("three_vesicles", N=N) if N >= 1024 else I.workload("ellipse_shrink", N=N)
    _, phi, psi, aux = run_gpu(w, 3, precision="fp32")
    _, s = run_oracle(w, 3)
    e = (rel(phi, s.phi), rel(psi, s.psi))
    print("fp32", N, e)
    assert max(e) < 5e-6, e


@pytest.mark.parametrize("precision,N,bound", [("fp64", 256, 1e-13), ("fp32", 256, 5e-10),
                                               ("fp32", 2048, 5e-11)])
def test_mass_conservation(precision, N, bound):
    """Relative mass drift over 100 steps.  The paper bounds it by 5e-11; in
    FP32 each stored value of psi (about 0.5) rounds by up to 3e-8, so the
    stored mass carries a random error of about 3e-8 / (sqrt(3) N) relative:
    1e-10 at N = 256, 1e-11 at N = 2048."""
    w = I.workload("ellipse_shrink", N=N) if N < 1024 else I.workload("three_vesicles", N=N)
    sim = cc.Simulation(w.params, w.N, precision=precision)
    sim.set_state(w.phi0, w.psi0)
    m0 = float(np.sum(w.psi0)) * (w.params.L / w.N) ** 2
    drift = []
    for _ in range(10):
        sim.step(10)
        drift.append(abs(sim.mass() - m0) / abs(m0))
    print(precision, "mass drift", max(drift))
    assert max(drift) < bound


def test_energy_diagnostics_match_oracle():
    w = I.workload("one_vesicle", N=64, dt=1e-5)
    sim, phi, psi, aux = run_gpu(w, 6, track=True)
    E = sim.energy()
    m = O.Model.from_params(w.N, w.params)
    s = O.initial_state(w.phi0, w.psi0, m)
    for _ in range(6):
        s = O.step(s, m)
    Eo = O.modified_energy(s, m)
    phys = O.physical_energy(s.phi, s.psi, m, s.A)
    assert E[0] == pytest.approx(Eo, rel=1e-10)
    assert E[6] == pytest.approx(s.lam_sum, rel=1e-10)
    assert E[5] == pytest.approx(phys["arc_length"], rel=1e-11)
    assert E[2] == pytest.approx(phys["bend"], rel=1e-10)
    assert E[4] == pytest.approx(phys["osm"], rel=1e-11)


def test_modified_energy_decreases_on_gpu():
    w = I.workload("one_vesicle", N=128, dt=1e-5)
    sim = cc.Simulation(w.params, w.N, track_energy=True)
    sim.set_state(w.phi0, w.psi0)
    sim.step(1)
    E = []
    for _ in range(15):
        sim.step(1)
        E.append(sim.energy()[0])
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(E, E[1:]))


def test_negative_mobility_is_reported_not_faulted():
    """dt = 1e-3 overshoots |phi| past the mobility root after the start step:
    the solve kernel flags the state and the handle refuses further steps."""
    w = I.workload("one_vesicle", N=32, dt=1e-3)
    sim = cc.Simulation(w.params, w.N)
    sim.set_state(w.phi0, w.psi0)
    sim.step(4)
    assert cc.ccmsav_sync(sim.h) == cc.CCMSAV_ENONFINITE
    assert cc.ccmsav_step(sim.h, 1) == cc.CCMSAV_ESTATE
    sim.set_state(w.phi0, w.psi0)         # set_state clears the error
    sim.step(1)
    sim.sync()


def test_nonfinite_input_rejected():
    w = I.workload("one_vesicle", N=16)
    sim = cc.Simulation(w.params, w.N)
    bad = w.phi0.copy()
    bad[3, 4] = np.nan
    assert cc.ccmsav_set_state(sim.h, 0, bad, w.psi0) == cc.CCMSAV_ENONFINITE
    assert cc.ccmsav_step(sim.h, 1) == cc.CCMSAV_ESTATE


@pytest.mark.parametrize("precision,N", [("fp64", 64), ("fp32", 64), ("fp32", 2048)])
def test_uploaded_conserved_mean_is_exact_sum(precision, N):
    """set_state sums psi on the device while uploading it (compensated
    per-thread sums, TwoSum merges, a fixed-order host pass): the conserved
    mean it keeps equals the exactly rounded mean of the FP64 input."""
    import math
    w = I.workload("three_vesicles", N=N) if N >= 1024 else I.workload("one_vesicle", N=N)
    sim = cc.Simulation(w.params, w.N, precision=precision)
    sim.set_state(w.phi0, w.psi0)
    aux = sim.aux()
    exact = math.fsum(w.psi0.ravel().tolist()) / (N * N)
    assert abs(aux[11] - exact) <= 1e-14 * abs(exact), (aux[11], exact)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resume_is_bit_exact(precision):
    w = I.workload("one_vesicle", N=64, dt=1e-5)
    _, phi_a, psi_a, aux_a = run_gpu(w, 10, precision=precision)
    sim = cc.Simulation(w.params, w.N, precision=precision)
    sim.set_state(w.phi0, w.psi0)
    sim.step(5)
    phi5, psi5 = sim.state()
    phiP, psiP = sim.state(prev=True)
    aux5 = sim.aux()
    sim.close()
    sim2 = cc.Simulation(w.params, w.N, precision=precision)
    sim2.set_levels(phi5, psi5, phiP, psiP)
    sim2.set_aux(aux5)
    sim2.step(5)
    phi_b, psi_b = sim2.state()
    assert np.array_equal(phi_a, phi_b) and np.array_equal(psi_a, psi_b)
    assert np.array_equal(aux_a[:8], sim2.aux()[:8])


def test_deterministic_runs():
    w = I.workload("ellipse_shrink", N=128)
    _, p1, q1, a1 = run_gpu(w, 7, precision="fp32")
    _, p2, q2, a2 = run_gpu(w, 7, precision="fp32")
    assert np.array_equal(p1, p2) and np.array_equal(q1, q2) and np.array_equal(a1, a2)


def test_uneven_batch_matches_single_runs():
    """Several simulations of different N and parameters in one handle give
    the same bits as each simulation alone."""
    ws = [I.workload("one_vesicle", N=32, dt=1e-5), I.workload("ellipse_shrink", N=64),
          I.workload("one_vesicle", N=16, dt=2e-5)]
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws])
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    sim.step(6)
    for k, w in enumerate(ws):
        phi, psi = sim.state(sim=k)
        _, phi1, psi1, _ = run_gpu(w, 6)
        assert np.array_equal(phi, phi1) and np.array_equal(psi, psi1)


@pytest.mark.parametrize("caller_stream", [False, True])
def test_batched_graph_steps_match_single_runs(caller_stream):
    """Several simulations in one handle step concurrently (one stream each,
    BDF2 steps from one graph per rotation phase for the whole batch); over
    15 steps in uneven chunks every phase's graph runs, and each simulation
    ends bit-identical to a run of its own."""
    torch = pytest.importorskip("torch")
    ws = [I.workload("one_vesicle", N=32, dt=1e-5), I.workload("ellipse_shrink", N=64),
          I.workload("one_vesicle", N=128, dt=1e-5), I.workload("ellipse_shrink", N=256)]
    stream = torch.cuda.Stream() if caller_stream else None
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32",
                        stream=None if stream is None else stream.cuda_stream)
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    for chunk in (1, 10, 4):
        sim.step(chunk)
    sim.sync()
    for k, w in enumerate(ws):
        phi, psi = sim.state(sim=k)
        solo = cc.Simulation(w.params, w.N, precision="fp32")
        solo.set_state(w.phi0, w.psi0)
        solo.step(15)
        phi1, psi1 = solo.state()
        solo.close()
        assert np.array_equal(phi, phi1) and np.array_equal(psi, psi1), f"simulation {k} (N={w.N})"
    assert all(sim.aux(sim=k)[10] == 15 for k in range(len(ws)))
    sim.close()


def test_grouped_launches_match_single_runs():
    """FP32 simulations of the same N share each kernel launch of the batch
    graph (three at N = 128, two at N = 256, with different parameters and
    states); an N = 64 simulation (block-FFT kernels) runs its own launches
    beside them.  The launch count shows the grouping (six launches per step
    per group and per ungrouped simulation) and every simulation ends
    bit-identical to a run of its own."""
    ws = [I.workload("one_vesicle", N=128, dt=1e-5), I.workload("ellipse_shrink", N=128),
          I.one_vesicle_circle(N=128, seed=77, dt=2e-5, precision="fp32", ratio=0.8),
          I.workload("one_vesicle", N=256, dt=1e-5), I.workload("ellipse_shrink", N=256),
          I.workload("one_vesicle", N=64, dt=1e-5)]
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32")
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    sim.step(1)
    l0 = sim.launches()
    sim.step(12)
    sim.sync()
    assert sim.launches() - l0 == 12 * 6 * 3, sim.launches() - l0   # groups N = 128, 256 and the N = 64 run
    for k, w in enumerate(ws):
        phi, psi = sim.state(sim=k)
        solo = cc.Simulation(w.params, w.N, precision="fp32")
        solo.set_state(w.phi0, w.psi0)
        solo.step(13)
        phi1, psi1 = solo.state()
        a1, a2 = sim.aux(sim=k), solo.aux()
        solo.close()
        assert np.array_equal(phi, phi1) and np.array_equal(psi, psi1), f"simulation {k} (N={w.N})"
        assert np.array_equal(a1, a2), f"simulation {k} scalars"
    sim.close()


def test_launch_group_size_does_not_change_results():
    """The same batch (four N = 128 and two N = 256 FP32 simulations) with
    no grouping, groups of two (2^15 points) and whole-size groups ends with
    the same bits, and the launch count follows the grouping."""
    ws = ([I.one_vesicle_circle(N=128, seed=300 + i, dt=1e-5, precision="fp32") for i in range(4)]
          + [I.workload("ellipse_shrink", N=256), I.workload("one_vesicle", N=256, dt=1e-5)])
    out, launches = {}, {}
    for pts in (0, 1 << 15, 1 << 26):
        sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32")
        sim.set_group_points(pts)
        assert sim.group_points() == pts
        for k, w in enumerate(ws):
            sim.set_state(w.phi0, w.psi0, sim=k)
        sim.step(1)
        l0 = sim.launches()
        sim.step(6)
        launches[pts] = sim.launches() - l0
        out[pts] = [sim.state(sim=k) for k in range(len(ws))]
        sim.close()
    for pts in (1 << 15, 1 << 26):
        for k in range(len(ws)):
            assert np.array_equal(out[pts][k][0], out[0][k][0]) and np.array_equal(out[pts][k][1], out[0][k][1])
    # six launches per step for each group and each simulation outside one:
    # no grouping (6 simulations); 2^15 points (two N = 128 pairs, the two
    # N = 256 grids of 2^16 points each run alone); 2^26 (one group per N)
    assert launches == {0: 6 * 6 * 6, 1 << 15: 6 * 6 * 4, 1 << 26: 6 * 6 * 2}, launches


def test_group_points_changed_between_steps():
    """Grouping switched off and on again between steps (the batch graphs are
    captured anew each time) leaves every simulation bit-identical to a run
    of its own."""
    ws = [I.one_vesicle_circle(N=256, seed=500 + i, dt=1e-5, precision="fp32") for i in range(3)]
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32")
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    for pts, n in ((1 << 21, 4), (0, 2), (1 << 21, 5)):
        sim.set_group_points(pts)
        sim.step(n)
    sim.sync()
    for k, w in enumerate(ws):
        phi, psi = sim.state(sim=k)
        solo = cc.Simulation(w.params, w.N, precision="fp32")
        solo.set_state(w.phi0, w.psi0)
        solo.step(11)
        phi1, psi1 = solo.state()
        solo.close()
        assert np.array_equal(phi, phi1) and np.array_equal(psi, psi1), f"simulation {k}"
    sim.close()


def test_largest_launch_group():
    """65 FP32 simulations of N = 128 with no limit on the group's points: the
    first 64 (the most one launch's parameter block carries) share every
    launch and the last runs its own, so a graph-launched step is 12
    launches; members across the group, and the one outside it, end
    bit-identical to runs of their own."""
    ws = [I.one_vesicle_circle(N=128, seed=900 + i, dt=1e-5, precision="fp32", ratio=0.8 + 0.01 * i)
          for i in range(65)]
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32")
    sim.set_group_points(1 << 30)
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    sim.step(1)
    l0 = sim.launches()
    sim.step(6)           # two graph launches of three steps each
    sim.sync()
    assert sim.launches() - l0 == 6 * 6 * 2, sim.launches() - l0
    for k in (0, 1, 31, 62, 63, 64):
        w = ws[k]
        phi, psi = sim.state(sim=k)
        solo = cc.Simulation(w.params, w.N, precision="fp32")
        solo.set_state(w.phi0, w.psi0)
        solo.step(7)
        phi1, psi1 = solo.state()
        solo.close()
        assert np.array_equal(phi, phi1) and np.array_equal(psi, psi1), f"simulation {k}"
    sim.close()


def test_bdf1_mode_batch_matches_single_runs():
    """A batched handle in the BDF1 product mode (CCMSAV_BDF1_ALWAYS: every
    step first order, so its simulations stay out of the grouped launches,
    which take BDF2 steps) gives each simulation's own bits."""
    ws = [I.workload("one_vesicle", N=128, dt=1e-5), I.workload("ellipse_shrink", N=128)]
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32",
                        bdf1_always=True)
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    sim.step(7)
    for k, w in enumerate(ws):
        phi, psi = sim.state(sim=k)
        solo = cc.Simulation(w.params, w.N, precision="fp32", bdf1_always=True)
        solo.set_state(w.phi0, w.psi0)
        solo.step(7)
        phi1, psi1 = solo.state()
        solo.close()
        assert np.array_equal(phi, phi1) and np.array_equal(psi, psi1), f"simulation {k}"
    sim.close()


_FP32_1000 = {}


def fp32_vs_fp64_1000_steps():
    """Errors of the FP32-bulk path against the FP64 path after 1000 steps
    at N = 2048 (three vesicles, dt = 1e-5), computed once per session."""
    if _FP32_1000:
        return dict(_FP32_1000)
    w = I.workload("three_vesicles", N=2048)
    res = {}
    for prec in ("fp64", "fp32"):
        sim = cc.Simulation(w.params, w.N, precision=prec)
        sim.set_state(w.phi0, w.psi0)
        sim.step(1000)
        sim.sync()
        res[prec] = (*sim.state(), sim.mass())
        sim.close()
    (p64, q64, m64), (p32, q32, m32) = res["fp64"], res["fp32"]
    m0 = float(np.sum(w.psi0)) * (w.params.L / w.N) ** 2
    e = {"phi_max": rel(p32, p64), "psi_max": rel(q32, q64),
         "phi_l2": float(np.sqrt(np.mean((p32 - p64) ** 2) / np.mean(p64 ** 2))),
         "psi_l2": float(np.sqrt(np.mean((q32 - q64) ** 2) / np.mean(q64 ** 2))),
         "mass32": abs(m32 - m0) / m0, "mass64": abs(m64 - m0) / m0}
    _FP32_1000.update(e)
    return dict(e)


@pytest.mark.slow
def test_fp32_against_fp64_after_1000_steps_N2048():
    """The precision form at full size: three vesicles, N = 2048, 1000 steps
    at dt = 1e-5, FP32-bulk against the FP64 GPU path (itself within 1e-12 of
    the oracle).  Measured: phi max 3.5e-6 / L2 2.0e-7, psi max 7.0e-7
    relative to the max-norm / RMS of the FP64 fields (with phi_bar rounded
    to FP32 inside the stencil, as before the stencil kept its low part:
    phi max 4.1e-5 / L2 1.9e-6); the bounds below are regression bounds at
    about twice the measured values.  Stored mass of both paths within 5e-11
    of the initial mass."""
    e = fp32_vs_fp64_1000_steps()
    print("fp32 vs fp64 after 1000 steps", e)
    assert e["phi_l2"] < 5e-7 and e["psi_l2"] < 5e-7, e
    assert e["phi_max"] < 8e-6 and e["psi_max"] < 2e-6, e
    assert e["mass32"] < 5e-11 and e["mass64"] < 5e-11, e


@pytest.mark.slow
def test_fp32_meets_1e5_max_norm_target_after_1000_steps_N2048():
    """The precision target as stated: phi and psi within 1e-5 of the FP64
    path in the max-norm after 1000 steps at N = 2048 (three vesicles,
    dt = 1e-5)."""
    e = fp32_vs_fp64_1000_steps()
    assert e["phi_max"] <= 1e-5 and e["psi_max"] <= 1e-5, e


@pytest.mark.slow
def test_fp64_with_fp32_storage_after_1000_steps_N2048():
    """What FP32 storage of the levels alone costs: the FP64 path with phi
    and psi (both levels) rounded to FP32 after every step, through the
    checkpoint calls (get_state / get_prev_state / get_aux, set_state_levels
    / set_aux), against plain FP64.  Measured: phi max 1.0e-6, psi max
    9.7e-7, a third of the FP32-bulk path's phi error (3.5e-6): most of the
    FP32 path's deviation is storage, the rest its FP32 arithmetic."""
    w = I.workload("three_vesicles", N=2048)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    ref = cc.Simulation(w.params, w.N, precision="fp64")
    ref.set_state(f32(w.phi0), f32(w.psi0))
    ref.step(1000)
    p64, q64 = ref.state()
    ref.close()
    sim = cc.Simulation(w.params, w.N, precision="fp64")
    sim.set_state(f32(w.phi0), f32(w.psi0))
    for _ in range(1000):
        sim.step(1)
        a, b = sim.state()
        c, d = sim.state(prev=True)
        aux = sim.aux()
        sim.set_levels(f32(a), f32(b), f32(c), f32(d))
        sim.set_aux(aux)
    p, q = sim.state()
    sim.close()
    e = (rel(p, p64), rel(q, q64))
    print("fp64 with fp32 storage after 1000 steps", e)
    assert max(e) < 3e-6, e


def test_fp32_warp_path_N4096_against_fp64():
    """Line length M = 2048 of the FP32 warp FFTs (64 values per lane): three
    vesicles at N = 4096, 3 steps against the FP64 path (block FFTs, the same
    code that matches the oracle at N <= 2048); bound 5e-6 of the max-norm
    as for the other line lengths."""
    w = I.workload("three_vesicles", N=4096)
    out = {}
    for prec in ("fp64", "fp32"):
        sim = cc.Simulation(w.params, w.N, precision=prec)
        sim.set_state(w.phi0, w.psi0)
        sim.step(3)
        sim.sync()
        out[prec] = sim.state()
        sim.close()
    e = (rel(out["fp32"][0], out["fp64"][0]), rel(out["fp32"][1], out["fp64"][1]))
    print("fp32 N=4096 vs fp64", e)
    assert max(e) < 5e-6, e


def test_largest_grid_N8192_fp32_against_fp64():
    """The largest grid the library takes (N = 8192, sixteen vesicles): two
    steps of the FP32 path against the FP64 path (bound 5e-6 of the
    max-norm) and the FP32 stored mass against the initial mass."""
    w = I.workload("lattice16", N=8192)
    m0 = float(np.sum(w.psi0)) * (w.params.L / w.N) ** 2
    out = {}
    for prec in ("fp64", "fp32"):
        sim = cc.Simulation(w.params, w.N, precision=prec)
        sim.set_state(w.phi0, w.psi0)
        sim.step(2)
        sim.sync()
        out[prec] = (*sim.state(), sim.mass())
        sim.close()
    e = (rel(out["fp32"][0], out["fp64"][0]), rel(out["fp32"][1], out["fp64"][1]))
    drift = abs(out["fp32"][2] - m0) / m0
    print("fp32 N=8192 vs fp64", e, "mass drift", drift)
    assert max(e) < 5e-6, e
    assert drift < 5e-11, drift


def test_async_aux_matches_synchronous_read():
    """ccmsav_get_aux_async queues a copy of the twelve scalars behind the
    queued steps: after a sync the buffers hold each step's values, equal
    to ccmsav_get_aux at that point."""
    w = I.workload("one_vesicle", N=64, dt=1e-5)
    sim = cc.Simulation(w.params, w.N, precision="fp32")
    sim.set_state(w.phi0, w.psi0)
    bufs = np.zeros((5, 12), np.float64)
    for k in range(5):
        sim.step(1)
        sim.aux_async(bufs[k])
    sim.sync()
    assert [int(b[10]) for b in bufs] == [1, 2, 3, 4, 5]
    assert np.array_equal(bufs[-1], sim.aux())
    sim.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_bdf1_mode_against_oracle(precision, tol):
    """CCMSAV_BDF1_ALWAYS: every step is the CC-MSAV-BDF1 scheme (graph-
    launched after the first); 10 steps at N = 128 against the oracle run
    with bdf1=True, and the one-level BDF1 energy against its definition."""
    w = I.workload("ellipse_shrink", N=128)
    sim = cc.Simulation(w.params, w.N, precision=precision, bdf1_always=True)
    sim.set_state(w.phi0, w.psi0)
    sim.step(1)
    sim.step(9)
    phi, psi = sim.state()
    aux = sim.aux()
    E = sim.energy()
    sim.close()
    m = O.Model.from_params(w.N, w.params)
    s = O.run(O.initial_state(w.phi0, w.psi0, m), m, 10, bdf1=True)
    e = (rel(phi, s.phi), rel(psi, s.psi), sav_err(aux[:8], s))
    print("bdf1 mode", precision, e)
    assert max(e) <= tol, e
    if precision == "fp64":
        SQ2 = math.sqrt(2.0)
        h = m.h
        cb = m.gamma_bend * 3 * SQ2 * m.eps / 8
        cs = m.gamma_surf * 3 * SQ2 * m.eps / 4 + m.theta
        cbeta = m.gamma_surf * 3 * SQ2 * m.beta / (4 * m.eps)
        La = O.lap(s.phi, h)
        E1 = (0.5 * cb * O.ip(La, La, h) + 0.5 * (cs - m.theta_tilde) * O.grad_norm2(s.phi, h)
              + 0.5 * cbeta * O.ip(s.phi, s.phi, h) + 0.5 * m.gamma_surf * 3 * SQ2 / 2 * s.V ** 2
              + 0.5 * m.gamma_area * s.U ** 2 + 0.5 * m.gamma_bend * 3 * SQ2 / (8 * m.eps) * s.W ** 2
              + 0.5 * s.Z ** 2)
        assert E[0] == pytest.approx(E1, rel=1e-10)


def test_autotune_keeps_state_and_records_schedule():
    """ccmsav_autotune times the candidate schedules from the current state
    and restores it: the fields and scalars after tuning are bit-identical to
    those before, the report names a schedule per simulation (sizes tuned
    once), and stepping on agrees with an untuned run (FP32: the warp and
    block paths round differently, within 5e-6)."""
    ws = [I.workload("one_vesicle", N=128, dt=1e-5), I.workload("ellipse_shrink", N=256),
          I.workload("one_vesicle", N=128, dt=2e-5)]
    sim = cc.Simulation(None, [w.N for w in ws], per_sim=[w.params for w in ws], precision="fp32")
    for k, w in enumerate(ws):
        sim.set_state(w.phi0, w.psi0, sim=k)
    sim.step(4)
    before = [(*sim.state(sim=k), sim.state(sim=k, prev=True), sim.aux(sim=k)) for k in range(3)]
    rep = sim.autotune(6)
    print("autotune report", rep)
    for k in range(3):
        phi, psi = sim.state(sim=k)
        prev = sim.state(sim=k, prev=True)
        assert np.array_equal(phi, before[k][0]) and np.array_equal(psi, before[k][1])
        assert np.array_equal(prev[0], before[k][2][0]) and np.array_equal(prev[1], before[k][2][1])
        assert np.array_equal(sim.aux(sim=k)[:10], before[k][3][:10])
    assert rep.shape == (3, 4) and all(r[1] in (58, 72, 100) for r in rep)
    assert rep[0][0] == rep[2][0] and rep[0][1] == rep[2][1]          # same size, same schedule
    assert sim.group_points() in {0, 1 << 26} | {1 << q for q in range(17, 23)}, sim.group_points()
    assert all(r[2] > 0 and r[3] > 0 for r in rep[:2])
    sim.step(5)
    for k, w in enumerate(ws):
        ref = cc.Simulation(w.params, w.N, precision="fp32")
        ref.set_state(w.phi0, w.psi0)
        ref.step(9)
        a, b = ref.state()
        ref.close()
        phi, psi = sim.state(sim=k)
        assert max(rel(phi, a), rel(psi, b)) <= 5e-6
    sim.close()


def test_autotune_single_simulation():
    """One simulation: its candidate schedules timed alone; state kept."""
    w = I.workload("ellipse_shrink", N=256)
    sim = cc.Simulation(w.params, w.N, precision="fp32")
    sim.set_state(w.phi0, w.psi0)
    sim.step(2)
    phi0, psi0 = sim.state()
    rep = sim.autotune(6)
    phi1, psi1 = sim.state()
    assert np.array_equal(phi0, phi1) and np.array_equal(psi0, psi1)
    assert rep.shape == (1, 4) and rep[0][1] in (58, 72, 100) and rep[0][2] > 0 and rep[0][3] > 0
    sim.step(3)
    sim.sync()
    sim.close()
