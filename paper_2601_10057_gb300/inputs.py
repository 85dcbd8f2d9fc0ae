"""Seeded synthetic workloads for the CC-MSAV vesicle step.

This module only builds inputs: the parameter sets of the paper's parameter
table (Appendix G, Table "Parameter values used in benchmark simulations")
and seeded diffuse-interface initial states.  It holds none of the scheme's
arithmetic, so both the CUDA path's tests/benchmark and the CPU oracle can
take their inputs from here without sharing any of the method.

Conventions
-----------
* Fields are ``float64`` arrays of shape ``(N, N)``, row-major, ``a[j, i]``
  with ``j`` the y index and ``i`` the x index.  Cell ``(i, j)`` has its
  centre at ``((i + 1/2) h, (j + 1/2) h)`` with ``h = L / N``.
* The phase field of one vesicle is ``tanh((R(theta) - r) / (sqrt(2) eps))``
  (+1 inside, -1 outside).  Several vesicles are united by a pointwise max.
* The concentration follows the paper's benchmark profiles (Sec. 4.2):
  ``psi0 = -0.35 phi0 + 0.45`` for growth and ``psi0 = -0.1 phi0 + 0.7`` for
  shrinkage, i.e. 0.8 outside and 0.1 (growth) or 0.6 (shrinkage) inside.
  A workload's concentration ratio ``r`` labels each vesicle: ``r >= 1`` is
  a growing vesicle, ``r < 1`` a shrinking one.  With several vesicles,
  ``psi0 = 0.8 + sum_k (inside_k - 0.8) (1 + phi_k) / 2``.
* The random draws use ``numpy.random.Generator(PCG64(seed))`` in a fixed
  order, so a (workload, seed) pair always gives the same arrays.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Params", "growth_params", "shrinkage_params", "Workload",
    "vesicle_phi", "concentration", "workload", "WORKLOADS",
    "SHARP_SHAPES", "sharp_shape", "robustness_params",
]


@dataclasses.dataclass
class Params:
    """Model and scheme parameters (names follow the paper's symbols).

    The defaults are the growth column of the paper's parameter table
    (Appendix G); ``L`` is the side of the square domain (the paper does not
    state it; the workloads below use ``2 pi``) and ``eps`` is usually set to
    ``4 h``.
    """
    gamma_surf: float = 1.0
    gamma_bend: float = 0.05
    gamma_area: float = 5.0e4
    gamma_in: float = 1.0e5
    gamma_out: float = 1.0e5
    psi_in: float = 0.65
    psi_out: float = 0.8
    beta_in: float = 0.0
    beta_out: float = 0.0
    eps: float = 0.03125
    M_phi: float = 1.0
    M0: float = 0.5
    theta: float = 1.5
    beta: float = 0.0
    lam: float = 1.0e5
    dt: float = 1.0e-6
    L: float = 1.0

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    def as_tuple(self):
        return dataclasses.astuple(self)


def growth_params(**kw) -> Params:
    """Growth column of the parameter table (gamma_bend = 0.05, psi_in = 0.65)."""
    return Params(**kw)


def shrinkage_params(**kw) -> Params:
    """Shrinkage column of the parameter table (gamma_bend = 1, psi_in = 0.1)."""
    base = dict(gamma_bend=1.0, psi_in=0.1)
    base.update(kw)
    return Params(**base)


def _cell_centres(N: int, L: float):
    h = L / N
    c = (np.arange(N, dtype=np.float64) + 0.5) * h
    X, Y = np.meshgrid(c, c, indexing="xy")   # X[j, i] = x_i, Y[j, i] = y_j
    return X, Y


def vesicle_phi(N: int, L: float, eps: float, centre, radius_fn) -> np.ndarray:
    """``tanh((R(theta) - r) / (sqrt 2 eps))`` around ``centre``.

    ``radius_fn`` maps the polar angle array to the boundary radius R(theta).
    """
    X, Y = _cell_centres(N, L)
    dx, dy = X - centre[0], Y - centre[1]
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    return np.tanh((radius_fn(th) - r) / (math.sqrt(2.0) * eps))


def _compose(N: int, L: float, eps: float, vesicles):
    """phi = max_k phi_k and psi = 0.8 + sum_k (inside_k - 0.8)(1 + phi_k)/2 for
    vesicles ``(centre, radius_fn, rmax, ratio)``.  Each phi_k is evaluated
    only where r < rmax + 20 sqrt(2) eps: beyond that the tanh argument is
    below -20 and phi_k is exactly -1 in double precision, so the result is
    bitwise that of evaluating every vesicle on the whole grid (same
    elementwise operations in the same order), without a full-grid array per
    vesicle."""
    h = L / N
    phi = np.full((N, N), -1.0)
    psi = np.full((N, N), PSI_OUTSIDE)
    for centre, radius_fn, rmax, ratio in vesicles:
        reach = rmax + 20.0 * math.sqrt(2.0) * eps
        i0 = max(0, int(math.floor((centre[0] - reach) / h)) - 1)
        i1 = min(N, int(math.ceil((centre[0] + reach) / h)) + 1)
        j0 = max(0, int(math.floor((centre[1] - reach) / h)) - 1)
        j1 = min(N, int(math.ceil((centre[1] + reach) / h)) + 1)
        X, Y = np.meshgrid((np.arange(i0, i1, dtype=np.float64) + 0.5) * h,
                           (np.arange(j0, j1, dtype=np.float64) + 0.5) * h, indexing="xy")
        dx, dy = X - centre[0], Y - centre[1]
        pk = np.tanh((radius_fn(np.arctan2(dy, dx)) - np.hypot(dx, dy)) / (math.sqrt(2.0) * eps))
        win = (slice(j0, j1), slice(i0, i1))
        phi[win] = np.maximum(phi[win], pk)
        inside = PSI_INSIDE_GROWTH if ratio >= 1.0 else PSI_INSIDE_SHRINK
        psi[win] = psi[win] + (inside - PSI_OUTSIDE) * (1.0 + pk) / 2.0
    return phi, psi


PSI_OUTSIDE = 0.8          # outside value of both benchmark profiles
PSI_INSIDE_GROWTH = 0.1    # -0.35 * 1 + 0.45
PSI_INSIDE_SHRINK = 0.6    # -0.1 * 1 + 0.7


def concentration(phis: Sequence[np.ndarray], ratios: Sequence[float]) -> np.ndarray:
    """``0.8 + sum_k (inside_k - 0.8)(1 + phi_k)/2`` with ``inside_k`` the
    benchmark growth (0.1) or shrinkage (0.6) inside value chosen by the
    ratio label of vesicle ``k``."""
    psi = np.full_like(phis[0], PSI_OUTSIDE)
    for ph, r in zip(phis, ratios):
        inside = PSI_INSIDE_GROWTH if r >= 1.0 else PSI_INSIDE_SHRINK
        psi = psi + (inside - PSI_OUTSIDE) * (1.0 + ph) / 2.0
    return psi


def _perturbed(R0: float, amps, phases):
    amps = np.asarray(amps, dtype=np.float64)
    phases = np.asarray(phases, dtype=np.float64)
    ms = np.arange(2, 2 + len(amps))

    def fn(th):
        s = np.ones_like(th)
        for m, a, p in zip(ms, amps, phases):
            s = s + a * np.cos(m * th + p)
        return R0 * s
    return fn


@dataclasses.dataclass
class Workload:
    """One simulation: its parameters, initial state and run length."""
    name: str
    N: int
    params: Params
    phi0: np.ndarray
    psi0: np.ndarray
    steps: int
    precision: str          # "fp64" or "fp32"

    @property
    def points(self) -> int:
        return self.N * self.N


def _params_for(ratios, N, L, dt, eps=None, **kw) -> Params:
    # Growth column when any vesicle grows (ratio >= 1), shrinkage otherwise.
    grows = any(r >= 1.0 for r in ratios)
    mk = growth_params if grows else shrinkage_params
    return mk(eps=4.0 * L / N if eps is None else eps, dt=dt, L=L, **kw)


# Interface width of the multi-vesicle workloads: 4 cells up to N = 2048; the
# larger grids keep the physical width of the N = 2048 interface (8 and 16
# cells at N = 4096 and 8192).  With eps = 4 h the explicit nonlinear terms
# stiffen like 1/eps, and the largest stable step shrinks about as h^4 (a
# 1/16 of the step per doubling of N), so eps = 4 h at N = 4096 or 8192 is
# unstable at the workloads' dt = 1e-5 and 5e-6.
def _multi_vesicle_eps(N: int, L: float) -> float:
    return 4.0 * L / min(N, 2048)


def one_vesicle_circle(N: int = 64, seed: int = 1001, dt: float = 1e-4,
                       steps: int = 200, ratio: float = 1.2,
                       precision: str = "fp64", L: float = 2 * math.pi,
                       R0: float = math.pi / 3, name: str = "one_vesicle") -> Workload:
    """Perturbed circle: R(theta) = R0 (1 + sum_{m=2..6} a_m cos(m theta + p_m)),
    a_m ~ U(0, 0.03), p_m ~ U(0, 2 pi), centred in the domain."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amps = rng.uniform(0.0, 0.03, 5)
    phases = rng.uniform(0.0, 2 * math.pi, 5)
    p = _params_for([ratio], N, L, dt)
    phi = vesicle_phi(N, L, p.eps, (L / 2, L / 2), _perturbed(R0, amps, phases))
    psi = concentration([phi], [ratio])
    return Workload(name, N, p, phi, psi, steps, precision)


def ellipse_shrink(N: int = 512, seed: int = 1002, dt: float = 1e-5,
                   steps: int = 1000, ratio: float = 0.8,
                   precision: str = "fp64", L: float = 2 * math.pi) -> Workload:
    """Ellipse with semi-axes 0.9 pi/2 and 0.6 pi/2 whose polar radius is
    scaled by (1 + sum_{m=2..8} a_m cos(m theta + p_m)), a_m ~ U(0, 0.02)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    amps = rng.uniform(0.0, 0.02, 7)
    phases = rng.uniform(0.0, 2 * math.pi, 7)
    a, b = 0.9 * math.pi / 2, 0.6 * math.pi / 2
    pert = _perturbed(1.0, amps, phases)

    def radius(th):
        return a * b / np.sqrt((b * np.cos(th)) ** 2 + (a * np.sin(th)) ** 2) * pert(th)

    p = _params_for([ratio], N, L, dt)
    phi = vesicle_phi(N, L, p.eps, (L / 2, L / 2), radius)
    psi = concentration([phi], [ratio])
    return Workload("ellipse_shrink", N, p, phi, psi, steps, precision)


def _place(rng, n, rmin, rmax, L, gap, margin_extra, max_tries=100000):
    placed = []
    tries = 0
    while len(placed) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place vesicles without overlap")
        R = rng.uniform(rmin, rmax)
        m = R * 1.15 + margin_extra
        if 2 * m >= L:
            continue
        cx, cy = rng.uniform(m, L - m, 2)
        ok = all(math.hypot(cx - x, cy - y) >= R * 1.15 + r * 1.15 + gap
                 for (x, y, r) in placed)
        if ok:
            placed.append((cx, cy, R))
    return placed


def three_vesicles(N: int = 2048, seed: int = 1003, dt: float = 1e-5,
                   steps: int = 1000, ratio: float = 1.3,
                   precision: str = "fp32", L: float = 2 * math.pi) -> Workload:
    """Three perturbed circles, R ~ U(0.5, 1.0), centres by rejection sampling
    (gap >= 8 eps between perturbed outlines, wall margin >= R + 8 eps)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = _multi_vesicle_eps(N, L)
    placed = _place(rng, 3, 0.5, 1.0, L, 8 * eps, 8 * eps)
    ves = []
    for (cx, cy, R) in placed:
        amps = rng.uniform(0.0, 0.03, 5)
        phases = rng.uniform(0.0, 2 * math.pi, 5)
        ves.append(((cx, cy), _perturbed(R, amps, phases), R * (1.0 + float(np.sum(amps))), ratio))
    phi, psi = _compose(N, L, eps, ves)
    p = _params_for([ratio], N, L, dt, eps=eps)
    return Workload(f"three_vesicles_N{N}", N, p, phi, psi, steps, precision)


def lattice_16(N: int = 8192, seed: int = 1005, dt: float = 5e-6,
               steps: int = 200, precision: str = "fp32",
               L: float = 2 * math.pi) -> Workload:
    """16 perturbed circles, R ~ U(0.2, 0.4), on a jittered 4 x 4 lattice with
    concentration ratios alternating 0.8 / 1.25."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = _multi_vesicle_eps(N, L)
    cell = L / 4
    ves, ratios = [], []
    for k in range(16):
        gx, gy = k % 4, k // 4
        R = rng.uniform(0.2, 0.4)
        jit = (cell / 2 - R * 1.15 - 4 * eps)
        jx, jy = rng.uniform(-jit, jit, 2) if jit > 0 else (0.0, 0.0)
        cx, cy = (gx + 0.5) * cell + jx, (gy + 0.5) * cell + jy
        amps = rng.uniform(0.0, 0.03, 5)
        phases = rng.uniform(0.0, 2 * math.pi, 5)
        ratios.append(0.8 if k % 2 == 0 else 1.25)
        ves.append(((cx, cy), _perturbed(R, amps, phases), R * (1.0 + float(np.sum(amps))), ratios[-1]))
    phi, psi = _compose(N, L, eps, ves)
    p = _params_for(ratios, N, L, dt, eps=eps)
    return Workload(f"lattice16_N{N}", N, p, phi, psi, steps, precision)


def batch_64(seed: int = 1004, n_sims: int = 64, steps: int = 500,
             dt: float = 1e-5, sizes=(128, 256, 512),
             L: float = 2 * math.pi) -> List[Workload]:
    """64 independent single-vesicle simulations with N drawn from ``sizes``,
    concentration ratio ~ U(0.7, 1.4), eps = 4 h each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(n_sims):
        N = int(rng.choice(np.asarray(sizes)))
        ratio = float(rng.uniform(0.7, 1.4))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        w = one_vesicle_circle(N=N, seed=sub, dt=dt, steps=steps, ratio=ratio,
                               precision="fp32", L=L, name=f"batch{s}_N{N}")
        out.append(w)
    return out


WORKLOADS = {
    "one_vesicle_N64": lambda: one_vesicle_circle(),
    "ellipse_shrink_N512": lambda: ellipse_shrink(),
    "three_vesicles_N2048": lambda: three_vesicles(N=2048),
    "three_vesicles_N4096": lambda: three_vesicles(N=4096),
    "lattice16_N8192": lambda: lattice_16(),
}


def workload(name: str, N: Optional[int] = None, **kw) -> Workload:
    """Build a named workload; ``N`` (and other keywords) override its size."""
    if name.startswith("one_vesicle"):
        return one_vesicle_circle(N=N or 64, **kw)
    if name.startswith("ellipse_shrink"):
        return ellipse_shrink(N=N or 512, **kw)
    if name.startswith("three_vesicles"):
        return three_vesicles(N=N or 2048, **kw)
    if name.startswith("lattice16"):
        return lattice_16(N=N or 8192, **kw)
    raise KeyError(name)


# ---------------------------------------------------------------------------
# Sharp initial shapes of the robustness runs (the paper names a triangle, a
# star, an incomplete hexagon and a crescent but gives no dimensions; these
# are this package's definitions).  phi = +1 at cell centres inside the
# shape, -1 outside; the smoother of Appendix F turns them into diffuse
# interfaces before a run.
# ---------------------------------------------------------------------------

SHARP_SHAPES = ("triangle", "star", "hexagon", "crescent")


def _polygon_radius(theta, verts):
    """Distance from the origin to the boundary of a polygon that is
    star-shaped about the origin, along the rays at angles theta; verts are
    (n, 2) vertices in counter-clockwise order of increasing angle."""
    ang = np.mod(np.arctan2(verts[:, 1], verts[:, 0]), 2 * math.pi)
    order = np.argsort(ang)
    verts, ang = verts[order], ang[order]
    th = np.mod(theta, 2 * math.pi)
    k = np.searchsorted(ang, th, side="right") - 1          # edge k: vertex k -> k+1 (wrapping)
    a = verts[k % len(verts)]
    b = verts[(k + 1) % len(verts)]
    d = b - a
    ux, uy = np.cos(th), np.sin(th)
    cross_ad = a[..., 0] * d[..., 1] - a[..., 1] * d[..., 0]
    cross_ud = ux * d[..., 1] - uy * d[..., 0]
    return cross_ad / cross_ud


def sharp_shape(kind: str, N: int, L: float = 1.0, R: Optional[float] = None) -> np.ndarray:
    """Sharp phase field of one centred shape of circumradius R (default
    L/4): an equilateral triangle with a vertex up; a five-pointed star (inner
    radius 0.45 R); a regular hexagon with one of its six sectors removed;
    a crescent (a disc of radius R minus a disc of radius 0.8 R whose centre
    is shifted by 0.45 R)."""
    R = L / 4 if R is None else R
    X, Y = _cell_centres(N, L)
    x, y = X - L / 2, Y - L / 2
    r, th = np.hypot(x, y), np.arctan2(y, x)
    if kind == "triangle":
        a = math.pi / 2 + 2 * math.pi * np.arange(3) / 3
        inside = r < _polygon_radius(th, R * np.stack([np.cos(a), np.sin(a)], 1))
    elif kind == "star":
        a = math.pi / 2 + math.pi * np.arange(10) / 5
        rad = np.where(np.arange(10) % 2 == 0, R, 0.45 * R)
        inside = r < _polygon_radius(th, np.stack([rad * np.cos(a), rad * np.sin(a)], 1))
    elif kind == "hexagon":
        a = 2 * math.pi * np.arange(6) / 6
        hexa = r < _polygon_radius(th, R * np.stack([np.cos(a), np.sin(a)], 1))
        sector = (np.mod(th, 2 * math.pi) < 2 * math.pi / 6)   # the sector between vertices 0 and 1
        inside = hexa & ~sector
    elif kind == "crescent":
        inside = (r < R) & (np.hypot(x - 0.45 * R, y) > 0.8 * R)
    else:
        raise KeyError(kind)
    return np.where(inside, 1.0, -1.0)


def robustness_params(grows: bool, N: int = 2048, L: float = 1.0, eps: float = 0.01,
                      dt: float = 5e-6) -> Params:
    """Parameters of the robustness runs: the table's growth or shrinkage
    column with (gamma_bend, theta) = (0.05, 10) for growth and (0.1, 30)
    for shrinkage, eps = 0.01, N = 2048, dt = 5e-6 on the unit square (about
    twenty cells across the interface)."""
    if grows:
        return growth_params(gamma_bend=0.05, theta=10.0, eps=eps, dt=dt, L=L)
    return shrinkage_params(gamma_bend=0.1, theta=30.0, eps=eps, dt=dt, L=L)


def convergence_ellipse(N: int, L: float = 1.0, eps: float = 0.03125, dt: float = 1e-6,
                        a: float = 0.3, b: float = 0.2) -> Workload:
    """Smooth ellipse of the convergence studies (semi-axes a, b, centred in
    the unit square; the paper's ellipse is not given): phi =
    tanh((R(theta) - r)/(sqrt2 eps)), the shrinkage profile of psi, the
    shrinkage column with the studies' moderate stiffness (gamma_in,
    gamma_out, gamma_area) = (100, 100, 100) and eps fixed across grids."""
    def radius(th):
        return a * b / np.sqrt((b * np.cos(th)) ** 2 + (a * np.sin(th)) ** 2)
    p = shrinkage_params(eps=eps, dt=dt, L=L, gamma_in=100.0, gamma_out=100.0, gamma_area=100.0)
    phi = vesicle_phi(N, L, eps, (L / 2, L / 2), radius)
    psi = concentration([phi], [0.8])
    return Workload(f"convergence_ellipse_N{N}", N, p, phi, psi, 0, "fp64")
