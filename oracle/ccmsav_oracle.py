"""CPU FP64 oracle of one CC-MSAV time step (test infrastructure only).

This module is the slow, plain reference that the CUDA path is checked
against.  It is test infrastructure: only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA path and imports nothing from it.

It follows the paper's own formulation in physical space:

* grid, ghost cells, difference/averaging operators, inner products and
  norms of the cell-centred staggered grid (Appendix D);
* energy densities, SAVs and their variational derivatives S, H, Q, K, P
  (Sec. 2.1 eq. energy_densities; Sec. 2.2 eqs. aux_vars and the formulas
  for S, H, Q, K, P), with the nonlinear terms discretised as in Sec. 3.4.1
  (eq. mobility_flux and the nonlocal bending term);
* the CC-MSAV-BDF2 step (Sec. 3.2 eqs. AC_BDF2 ... Z_BDF2) solved by the
  paper's procedure (Appendix B, Steps 1-4 and Algorithm "BDF2 MSAV Solution
  Procedure"): explicit right-hand sides f^n and g^n, seven constant-
  coefficient solves with chi (eq. chi_operator) and zeta, a dense 5x5 system
  for (B, C, D, E, G), field recovery by eqs. decoupled_AC / decoupled_CH and
  the SAV updates;
* the first step is the CC-MSAV-BDF1 variant (Appendix B, remark on the BDF1
  scheme);
* the elliptic solves are the DCT solver of Appendix C: an orthonormal 2D
  DCT-II written out as its defining cosine sum (a dense cosine matrix applied
  along both axes), a division by the closed-form eigenvalues, and the
  transposed (DCT-III) matrix;
* the modified discrete energy of eq. modified_discrete_energy and the
  numerical dissipation K^n of eq. K_n_explicit (Appendix A).

Readings where the paper is silent or ambiguous (they are listed with the
reasons in the design notes):

* the face average in the nonlocal bending term is arithmetic,
  ``A_x(phi^2) = (phi_i^2 + phi_{i+1}^2)/2``, and the discrete
  ``6 phi^2 |grad phi|^2`` inside W is ``6 sum_faces A(phi^2) (D phi)^2``,
  which makes Q exactly the discrete gradient of W;
* the target arc length A in U is the initial arc length, so U^0 = 0;
* the zero mode is divided like any other (sigma_00 = C1 > 0 and
  tau_00 = 3/(2 dt) > 0), never set to zero;
* the first step (0 -> 1) is CC-MSAV-BDF1; BDF2 is used from n = 1 on and
  the lambda-sum of the modified energy starts with the first BDF2 step.

Arrays are ``float64`` of shape ``(N, N)`` indexed ``u[j, i]`` (j: y, i: x).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np

SQ2 = math.sqrt(2.0)


# --------------------------------------------------------------------------
# Parameters (Appendix G table; Appendix B Step 3 constants)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Model:
    """Parameter set plus grid size; constants derived as in Appendix B."""
    N: int
    gamma_surf: float
    gamma_bend: float
    gamma_area: float
    gamma_in: float
    gamma_out: float
    psi_in: float
    psi_out: float
    beta_in: float
    beta_out: float
    eps: float
    M_phi: float
    M0: float
    theta: float
    beta: float
    lam: float
    dt: float
    L: float

    @classmethod
    def from_params(cls, N: int, p) -> "Model":
        d = {f.name: getattr(p, f.name) for f in dataclasses.fields(p)}
        return cls(N=N, **d)

    @property
    def h(self) -> float:
        return self.L / self.N

    # Step 3: coefficients of chi (BDF2; BDF1 replaces 3/(2dt) by 1/dt).
    def C1(self, bdf1: bool = False) -> float:
        a = 1.0 / self.dt if bdf1 else 3.0 / (2.0 * self.dt)
        return a + self.M_phi * self.gamma_surf * 3 * SQ2 * self.beta / (4 * self.eps)

    @property
    def C2(self) -> float:
        return self.M_phi * (self.gamma_surf * 3 * SQ2 * self.eps / 4 + self.theta)

    @property
    def C3(self) -> float:
        return self.M_phi * self.gamma_bend * 3 * SQ2 * self.eps / 8

    # Step 3: the four coupling constants c_gs, c_ga, c_gb, c_go.
    @property
    def c_gs(self) -> float:
        return self.M_phi * self.gamma_surf * 3 * SQ2 / 2

    @property
    def c_ga(self) -> float:
        return self.M_phi * self.gamma_area

    @property
    def c_gb(self) -> float:
        return self.M_phi * self.gamma_bend * 3 * SQ2 / (8 * self.eps)

    @property
    def c_go(self) -> float:
        return self.M_phi

    # theta-tilde of eq. modified_discrete_energy: theta + gamma_bend 3 sqrt2/(4 eps).
    @property
    def theta_tilde(self) -> float:
        return self.theta + self.gamma_bend * 3 * SQ2 / (4 * self.eps)


# --------------------------------------------------------------------------
# Grid operators (Appendix D)
# --------------------------------------------------------------------------

def ghost(u: np.ndarray) -> np.ndarray:
    """Ghost-extended field: phi_0 = phi_1, phi_{m+1} = phi_m (Appendix D,
    boundary conditions)."""
    return np.pad(u, 1, mode="edge")


def Dx(u: np.ndarray, h: float) -> np.ndarray:
    """(D_x u)_{i+1/2, j} on all east-west faces i = 0..m; shape (N, N+1)."""
    g = ghost(u)[1:-1, :]
    return (g[:, 1:] - g[:, :-1]) / h


def Dy(u: np.ndarray, h: float) -> np.ndarray:
    """(D_y u)_{i, j+1/2} on all north-south faces j = 0..n; shape (N+1, N)."""
    g = ghost(u)[:, 1:-1]
    return (g[1:, :] - g[:-1, :]) / h


def Ax(u: np.ndarray) -> np.ndarray:
    """(A_x u)_{i+1/2, j} = (u_i + u_{i+1})/2 on east-west faces."""
    g = ghost(u)[1:-1, :]
    return 0.5 * (g[:, 1:] + g[:, :-1])


def Ay(u: np.ndarray) -> np.ndarray:
    """(A_y u)_{i, j+1/2} = (u_j + u_{j+1})/2 on north-south faces."""
    g = ghost(u)[:, 1:-1]
    return 0.5 * (g[1:, :] + g[:-1, :])


def dx(f: np.ndarray, h: float) -> np.ndarray:
    """(d_x f)_{i, j} = (f_{i+1/2} - f_{i-1/2}) / h (edge-to-centre)."""
    return (f[:, 1:] - f[:, :-1]) / h


def dy(g: np.ndarray, h: float) -> np.ndarray:
    """(d_y g)_{i, j} = (g_{j+1/2} - g_{j-1/2}) / h."""
    return (g[1:, :] - g[:-1, :]) / h


def lap(u: np.ndarray, h: float) -> np.ndarray:
    """Delta_h u = d_x D_x u + d_y D_y u (5-point, ghost-mirrored)."""
    return dx(Dx(u, h), h) + dy(Dy(u, h), h)


def ip(u: np.ndarray, v: np.ndarray, h: float) -> float:
    """Cell inner product (u, v)_h = h^2 sum u v."""
    return float(h * h * np.sum(u * v))


def face_ip(fx: np.ndarray, gx: np.ndarray, fy: np.ndarray, gy: np.ndarray,
            h: float) -> float:
    """[f, g]_ew + [f, g]_ns: each interior face counts once (weight h^2),
    each boundary face half (weight h^2/2), as in Appendix D."""
    wx = np.ones(fx.shape[1]); wx[0] = wx[-1] = 0.5
    wy = np.ones(fy.shape[0]); wy[0] = wy[-1] = 0.5
    return float(h * h * (np.sum(fx * gx * wx[None, :]) + np.sum(fy * gy * wy[:, None])))


def grad_norm2(u: np.ndarray, h: float) -> float:
    """||grad_h u||^2 = [D_x u, D_x u]_ew + [D_y u, D_y u]_ns."""
    ux, uy = Dx(u, h), Dy(u, h)
    return face_ip(ux, ux, uy, uy, h)


def div_mobility_grad(phi: np.ndarray, nu: np.ndarray, m: Model) -> np.ndarray:
    """d_x(M_psi(A_x phi) D_x nu) + d_y(M_psi(A_y phi) D_y nu), eq. mobility_flux,
    with M_psi(phi) = 1 - M0 (phi^2 - 1)^2 evaluated at the face average."""
    h = m.h
    Mx = mobility(Ax(phi), m)
    My = mobility(Ay(phi), m)
    return dx(Mx * Dx(nu, h), h) + dy(My * Dy(nu, h), h)


def mobility(phi_face: np.ndarray, m: Model) -> np.ndarray:
    """M_psi(phi) = 1 - M0 (phi^2 - 1)^2 (Sec. 2.1)."""
    return 1.0 - m.M0 * (phi_face ** 2 - 1.0) ** 2


# --------------------------------------------------------------------------
# Energy densities and SAV functionals (Secs. 2.1-2.2)
# --------------------------------------------------------------------------

def p_fun(phi):
    """Interpolation p(phi) = sin(pi phi / 2)."""
    return np.sin(0.5 * math.pi * phi)


def dp_fun(phi):
    """p'(phi) = (pi/2) cos(pi phi / 2)."""
    return 0.5 * math.pi * np.cos(0.5 * math.pi * phi)


def f_in(psi, m: Model):
    """f^in(psi) = gamma_in/2 (psi - psi_in)^2 + beta_in."""
    return 0.5 * m.gamma_in * (psi - m.psi_in) ** 2 + m.beta_in


def f_out(psi, m: Model):
    """f^out(psi) = gamma_out/2 (psi - psi_out)^2 + beta_out."""
    return 0.5 * m.gamma_out * (psi - m.psi_out) ** 2 + m.beta_out


def g_dw(phi):
    """Double well g(phi) = (phi^2 - 1)^2 / 4."""
    return 0.25 * (phi * phi - 1.0) ** 2


def bending_face_term(phi: np.ndarray, h: float) -> np.ndarray:
    """Per-cell share of sum_faces A(phi^2)(D phi)^2: phi_ij^2 times the cell
    average of the squared face gradients (each face split half/half between
    its two cells).  Summed over cells this is the face sum itself."""
    gx2 = Dx(phi, h) ** 2
    gy2 = Dy(phi, h) ** 2
    gbar = 0.5 * (gx2[:, 1:] + gx2[:, :-1]) + 0.5 * (gy2[1:, :] + gy2[:-1, :])
    return phi * phi * gbar


def I_V(phi, m: Model) -> float:
    """Radicand of V (eq. aux_VW): int (phi^2 - 1 - beta)^2 / (4 eps)."""
    return ip((phi * phi - 1.0 - m.beta) ** 2 / (4.0 * m.eps), np.ones_like(phi), m.h)


def I_W(phi, m: Model) -> float:
    """Radicand of W (eq. aux_VW): int 6 phi^2|grad phi|^2 + (phi^3-phi)^2/eps^2,
    with the gradient part as the face sum 6 sum A(phi^2)(D phi)^2."""
    cell = 6.0 * bending_face_term(phi, m.h) + (phi ** 3 - phi) ** 2 / m.eps ** 2
    return ip(cell, np.ones_like(phi), m.h)


def I_Z(phi, psi, m: Model) -> float:
    """Radicand of Z (eq. aux_ZU): 2 int f_osm = int (1+p) f_in + (1-p) f_out."""
    pp = p_fun(phi)
    return ip((1 + pp) * f_in(psi, m) + (1 - pp) * f_out(psi, m), np.ones_like(phi), m.h)


def surface_integral(phi, m: Model) -> float:
    """int f_surf = 3 sqrt2/4 ( (1/eps) int g(phi) + (eps/2) ||grad_h phi||^2 )."""
    return 3 * SQ2 / 4 * (ip(g_dw(phi), np.ones_like(phi), m.h) / m.eps
                          + 0.5 * m.eps * grad_norm2(phi, m.h))


def V_of(phi, m):
    return math.sqrt(I_V(phi, m))


def W_of(phi, m):
    return math.sqrt(I_W(phi, m))


def Z_of(phi, psi, m):
    return math.sqrt(I_Z(phi, psi, m))


def U_of(phi, m, A):
    return surface_integral(phi, m) - A


def S_fun(phi, m: Model) -> np.ndarray:
    """S(phi) = phi(phi^2 - 1 - beta)/eps / (2 sqrt(int (phi^2-1-beta)^2/(4 eps)))."""
    return phi * (phi * phi - 1.0 - m.beta) / m.eps / (2.0 * math.sqrt(I_V(phi, m)))


def H_fun(phi, m: Model) -> np.ndarray:
    """H(phi) = 3 sqrt2/4 [ phi(phi^2-1)/eps - eps Delta_h phi ]."""
    return 3 * SQ2 / 4 * (phi * (phi * phi - 1.0) / m.eps - m.eps * lap(phi, m.h))


def Q_fun(phi, m: Model) -> np.ndarray:
    """Q(phi) = {6[phi|grad phi|^2 - div(phi^2 grad phi)] + (phi^3-phi)(3phi^2-1)/eps^2}
    / sqrt(I_W), with both bending terms discretised as in Sec. 3.4.1."""
    h = m.h
    gx2 = Dx(phi, h) ** 2
    gy2 = Dy(phi, h) ** 2
    phi_grad2 = phi * (0.5 * (gx2[:, 1:] + gx2[:, :-1]) + 0.5 * (gy2[1:, :] + gy2[:-1, :]))
    p2 = phi * phi
    div_p2g = dx(Ax(p2) * Dx(phi, h), h) + dy(Ay(p2) * Dy(phi, h), h)
    num = 6.0 * (phi_grad2 - div_p2g) + (phi ** 3 - phi) * (3 * phi * phi - 1.0) / m.eps ** 2
    return num / math.sqrt(I_W(phi, m))


def K_fun(phi, psi, m: Model) -> np.ndarray:
    """K(phi, psi) = p'(phi)(f_in - f_out) / (2 sqrt(I_Z))."""
    return dp_fun(phi) * (f_in(psi, m) - f_out(psi, m)) / (2.0 * math.sqrt(I_Z(phi, psi, m)))


def P_fun(phi, psi, m: Model) -> np.ndarray:
    """P(phi, psi) = [gamma_in(1+p)(psi-psi_in) + gamma_out(1-p)(psi-psi_out)]
    / (2 sqrt(I_Z))."""
    pp = p_fun(phi)
    num = m.gamma_in * (1 + pp) * (psi - m.psi_in) + m.gamma_out * (1 - pp) * (psi - m.psi_out)
    return num / (2.0 * math.sqrt(I_Z(phi, psi, m)))


# --------------------------------------------------------------------------
# DCT fast direct solver (Appendix C)
# --------------------------------------------------------------------------

_DCT_CACHE: Dict[int, np.ndarray] = {}


def dct_matrix(N: int) -> np.ndarray:
    """Orthonormal DCT-II matrix C[k, n] = c_k cos(pi k (2n+1) / (2N)),
    c_0 = sqrt(1/N), c_k = sqrt(2/N); its transpose is the DCT-III."""
    C = _DCT_CACHE.get(N)
    if C is None:
        k = np.arange(N, dtype=np.float64)[:, None]
        n = np.arange(N, dtype=np.float64)[None, :]
        C = np.cos(math.pi * k * (2 * n + 1) / (2 * N))
        C[0, :] *= math.sqrt(1.0 / N)
        C[1:, :] *= math.sqrt(2.0 / N)
        _DCT_CACHE[N] = C
    return C


def dct2d(u: np.ndarray) -> np.ndarray:
    """Forward 2D orthonormal DCT-II (along x and along y)."""
    C = dct_matrix(u.shape[0])
    return C @ u @ C.T


def idct2d(U: np.ndarray) -> np.ndarray:
    """Inverse 2D transform (orthonormal DCT-III)."""
    C = dct_matrix(U.shape[0])
    return C.T @ U @ C


def laplacian_eigenvalues(N: int, h: float) -> np.ndarray:
    """lambda_{kl} = -(4/h^2)[sin^2(pi k/(2N)) + sin^2(pi l/(2N))] (Appendix C)."""
    s = np.sin(math.pi * np.arange(N) / (2 * N)) ** 2
    return -(4.0 / (h * h)) * (s[:, None] + s[None, :])


def chi_spectrum(m: Model, bdf1: bool = False) -> np.ndarray:
    """sigma_{kl} = C1 - C2 lambda_{kl} + C3 lambda_{kl}^2."""
    lam = laplacian_eigenvalues(m.N, m.h)
    return m.C1(bdf1) - m.C2 * lam + m.C3 * lam * lam


def zeta_spectrum(m: Model, bdf1: bool = False) -> np.ndarray:
    """tau_{kl} = 3/(2 dt) - lambda lambda_{kl} (1/dt for BDF1)."""
    lam = laplacian_eigenvalues(m.N, m.h)
    a = 1.0 / m.dt if bdf1 else 3.0 / (2.0 * m.dt)
    return a - m.lam * lam


def solve_spectral(rhs: np.ndarray, spectrum: np.ndarray) -> np.ndarray:
    """DCT -> divide by the operator's eigenvalues -> inverse DCT."""
    return idct2d(dct2d(rhs) / spectrum)


# --------------------------------------------------------------------------
# State and the time step (Sec. 3.2; Appendix B)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class State:
    """Two time levels of the fields and of the SAVs, plus bookkeeping."""
    phi: np.ndarray           # phi^n
    psi: np.ndarray           # psi^n
    phi_old: np.ndarray       # phi^{n-1} (equal to phi^n before the first step)
    psi_old: np.ndarray
    V: float
    U: float
    W: float
    Z: float
    V_old: float
    U_old: float
    W_old: float
    Z_old: float
    A: float                  # target arc length inside U
    n: int = 0                # number of steps taken
    lam_sum: float = 0.0      # sum_{j>=2} dt/2 ||d^j||^2

    def copy(self) -> "State":
        return dataclasses.replace(self, phi=self.phi.copy(), psi=self.psi.copy(),
                                   phi_old=self.phi_old.copy(), psi_old=self.psi_old.copy())


def initial_state(phi0: np.ndarray, psi0: np.ndarray, m: Model,
                  A: Optional[float] = None) -> State:
    """SAV initial values (eq. msav_ic) with A := int f_surf(phi0) unless given."""
    phi0 = np.array(phi0, dtype=np.float64)
    psi0 = np.array(psi0, dtype=np.float64)
    if A is None:
        A = surface_integral(phi0, m)
    V, W, Z = V_of(phi0, m), W_of(phi0, m), Z_of(phi0, psi0, m)
    U = U_of(phi0, m, A)
    return State(phi0, psi0, phi0.copy(), psi0.copy(), V, U, W, Z, V, U, W, Z, A)


@dataclasses.dataclass
class StepInfo:
    """Intermediate quantities of one step (for tests)."""
    Mmat: np.ndarray
    bvec: np.ndarray
    sol: np.ndarray
    gram: np.ndarray          # (F_i, chi^{-1} F_j), i, j over S, H, Q, K
    bdf1: bool


def step(s: State, m: Model, return_info: bool = False, bdf1: Optional[bool] = None,
         classical: bool = False):
    """One CC-MSAV step n -> n+1: BDF1 when s.n == 0, BDF2 afterwards; with
    bdf1=True every step is the CC-MSAV-BDF1 scheme (Appendix B, remark on
    the BDF1 scheme).  classical=True takes the classical MSAV scheme
    instead (Appendix B, remarks on the Classical-MSAV-BDF2 / BDF1 schemes):
    the Cahn-Hilliard stabilisation sits in the chemical potential, so
    g = (4 psi^n - psi^{n-1})/(2 dt) + div(M_psi(phi*) grad nu~) with
    nu~ = -lam psi* + a_Z P, and both Cahn-Hilliard solves use the
    variable-coefficient operator 3/(2 dt) - lam div(M_psi(phi*) grad),
    solved here by a sparse direct factorisation (the paper's
    Classical+Direct baseline)."""
    bdf1 = (s.n == 0) if bdf1 is None else bool(bdf1)
    h = m.h
    # Stage 1: extrapolations (BDF1 uses level n).
    if bdf1:
        phis, psis = s.phi, s.psi
    else:
        phis = 2.0 * s.phi - s.phi_old
        psis = 2.0 * s.psi - s.psi_old
    # Basis functions at the extrapolated state.
    S = S_fun(phis, m)
    H = H_fun(phis, m)
    Q = Q_fun(phis, m)
    K = K_fun(phis, psis, m)
    P = P_fun(phis, psis, m)
    # Step 1: known parts of the new SAVs,
    #   BDF2: V^{n+1} = (4V^n - V^{n-1} + (S, -4phi^n + phi^{n-1}))/3 + (S, phi^{n+1})
    #   BDF1: V^{n+1} = V^n + (S, -phi^n) + (S, phi^{n+1})
    if bdf1:
        wphi, wpsi = -s.phi, -s.psi
        aV = s.V + ip(S, wphi, h)
        aU = s.U + ip(H, wphi, h)
        aW = s.W + ip(Q, wphi, h)
        aZ = s.Z + ip(K, wphi, h) + ip(P, wpsi, h)
        f = s.phi / m.dt
        g = s.psi / m.dt
    else:
        wphi = -4.0 * s.phi + s.phi_old
        wpsi = -4.0 * s.psi + s.psi_old
        aV = (4 * s.V - s.V_old + ip(S, wphi, h)) / 3.0
        aU = (4 * s.U - s.U_old + ip(H, wphi, h)) / 3.0
        aW = (4 * s.W - s.W_old + ip(Q, wphi, h)) / 3.0
        aZ = (4 * s.Z - s.Z_old + ip(K, wphi, h) + ip(P, wpsi, h)) / 3.0
        f = (4.0 * s.phi - s.phi_old) / (2.0 * m.dt)
        g = (4.0 * s.psi - s.psi_old) / (2.0 * m.dt)
    # Step 2: explicit right-hand sides f^n and g^n.
    f = f - m.M_phi * (m.theta_tilde * lap(phis, h)
                       + m.gamma_surf * 3 * SQ2 / 2 * aV * S
                       + m.gamma_area * aU * H
                       + m.gamma_bend * 3 * SQ2 / (8 * m.eps) * aW * Q
                       + aZ * K)
    nu_tilde = aZ * P
    if classical:
        g = g + div_mobility_grad(phis, nu_tilde - m.lam * psis, m)
    else:
        g = g - m.lam * lap(psis, h) + div_mobility_grad(phis, nu_tilde, m)
    # Step 3: the seven constant-coefficient solves.
    sig = chi_spectrum(m, bdf1)
    tau = zeta_spectrum(m, bdf1)
    f_hat = solve_spectral(f, sig)
    S_hat = solve_spectral(S, sig)
    H_hat = solve_spectral(H, sig)
    Q_hat = solve_spectral(Q, sig)
    K_hat = solve_spectral(K, sig)
    if classical:
        zeta_c = classical_zeta_matrix(phis, m, bdf1)
        g_hat = sparse_solve(zeta_c, g)
        Lam_P = sparse_solve(zeta_c, div_mobility_grad(phis, P, m))
    else:
        g_hat = solve_spectral(g, tau)
        Lam_P = solve_spectral(div_mobility_grad(phis, P, m), tau)
    # Step 4: the 5x5 system for B, C, D, E, G.
    F = [S, H, Q, K]
    hats = [S_hat, H_hat, Q_hat, K_hat]
    coef = [m.c_gs, m.c_ga, m.c_gb, m.c_go]
    gram = np.array([[ip(Fi, Fj_hat, h) for Fj_hat in hats] for Fi in F])
    Mmat = np.zeros((5, 5))
    for i in range(4):
        for j in range(4):
            Mmat[i, j] = coef[j] * gram[i, j]
        Mmat[i, i] += 1.0
        Mmat[i, 4] = m.c_go * gram[i, 3]
    PL = ip(P, Lam_P, h)
    Mmat[4, 3] = -PL
    Mmat[4, 4] = 1.0 - PL
    bvec = np.array([ip(Fi, f_hat, h) for Fi in F] + [ip(P, g_hat, h)])
    sol = np.linalg.solve(Mmat, bvec)
    Bt, Ct, Dt, Et, Gt = sol
    # Field recovery (eqs. decoupled_AC, decoupled_CH).
    phi_new = (f_hat - m.c_gs * Bt * S_hat - m.c_ga * Ct * H_hat
               - m.c_gb * Dt * Q_hat - m.c_go * (Et + Gt) * K_hat)
    psi_new = g_hat + (Et + Gt) * Lam_P
    # SAV update.
    V_new, U_new, W_new, Z_new = Bt + aV, Ct + aU, Dt + aW, Et + Gt + aZ
    lam_sum = s.lam_sum
    if not bdf1:
        lam_sum += 0.5 * m.dt * d_norm2(phis, psis, psi_new, m)
    out = State(phi_new, psi_new, s.phi.copy(), s.psi.copy(),
                V_new, U_new, W_new, Z_new, s.V, s.U, s.W, s.Z,
                s.A, s.n + 1, lam_sum)
    if return_info:
        return out, StepInfo(Mmat, bvec, sol, gram, bdf1)
    return out


def run(s: State, m: Model, nsteps: int, bdf1: Optional[bool] = None,
        classical: bool = False) -> State:
    for _ in range(nsteps):
        s = step(s, m, bdf1=bdf1, classical=classical)
    return s


def mobility_operator_matrix(phis: np.ndarray, m: Model):
    """Sparse N^2 x N^2 matrix of nu -> div(M_psi(A phis) grad nu) (eq.
    mobility_flux): each interior face couples its two cells with weight
    M_face / h^2; boundary faces carry no flux (row-major cell index j N + i)."""
    import scipy.sparse as sp
    N, h = phis.shape[0], m.h
    Mx = mobility(Ax(phis), m)[:, 1:-1] / (h * h)     # interior east-west faces, (N, N-1)
    My = mobility(Ay(phis), m)[1:-1, :] / (h * h)     # interior north-south faces, (N-1, N)
    idx = np.arange(N * N).reshape(N, N)
    rows, cols, vals = [], [], []
    for a, b, w in ((idx[:, :-1], idx[:, 1:], Mx), (idx[:-1, :], idx[1:, :], My)):
        a, b, w = a.ravel(), b.ravel(), w.ravel()
        rows += [a, b, a, b]
        cols += [b, a, a, b]
        vals += [w, w, -w, -w]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N * N, N * N))


def classical_zeta_matrix(phis: np.ndarray, m: Model, bdf1: bool = False):
    """The classical scheme's Cahn-Hilliard operator 3/(2 dt) - lam div(M grad)
    (1/dt for BDF1) as a sparse matrix."""
    import scipy.sparse as sp
    a = 1.0 / m.dt if bdf1 else 1.5 / m.dt
    N = phis.shape[0]
    return (a * sp.identity(N * N, format="csr") - m.lam * mobility_operator_matrix(phis, m)).tocsc()


def sparse_solve(A, rhs: np.ndarray) -> np.ndarray:
    """Direct sparse solve (LU of scipy's SuperLU)."""
    import scipy.sparse.linalg as spla
    return spla.spsolve(A, rhs.ravel()).reshape(rhs.shape)


# --------------------------------------------------------------------------
# Diagnostics: mass, modified discrete energy, physical energy (Sec. 3.3, 3.4)
# --------------------------------------------------------------------------

def mass(psi: np.ndarray, m: Model) -> float:
    """Discrete mass h^2 sum psi (Sec. 3.4.2 remark on mass conservation)."""
    return ip(psi, np.ones_like(psi), m.h)


def d_norm2(phis, psis, psi_new, m: Model) -> float:
    """||d^{n+1}||^2 with d = lambda D(psi^{n+1} - psi*)/sqrt(M_psi(A phi*)) on faces."""
    h = m.h
    w = psi_new - psis
    Mx, My = mobility(Ax(phis), m), mobility(Ay(phis), m)
    wx, wy = Dx(w, h), Dy(w, h)
    return m.lam ** 2 * face_ip(wx, wx / Mx, wy, wy / My, h)


def modified_energy(s: State, m: Model) -> float:
    """E^{n+1,n}_mod of eq. modified_discrete_energy for the two stored levels
    (s.phi = level n+1, s.phi_old = level n)."""
    h = m.h
    a, b = s.phi, s.phi_old
    La, Lb = lap(a, h), lap(b, h)
    cb = m.gamma_bend * 3 * SQ2 * m.eps / 8
    cs = m.gamma_surf * 3 * SQ2 * m.eps / 4 + m.theta
    cbeta = m.gamma_surf * 3 * SQ2 * m.beta / (4 * m.eps)
    gn = grad_norm2
    E = 0.5 * cb * (ip(La, La, h) + ip(2 * La - Lb, 2 * La - Lb, h))
    E += 0.5 * cs * (gn(a, h) + gn(2 * a - b, h))
    E -= 0.5 * m.theta_tilde * (gn(a, h) + gn(2 * a - b, h) - 2 * gn(a - b, h))
    E += 0.5 * cbeta * (ip(a, a, h) + ip(2 * a - b, 2 * a - b, h))
    E += 0.5 * m.gamma_surf * 3 * SQ2 / 2 * (s.V ** 2 + (2 * s.V - s.V_old) ** 2)
    E += 0.5 * m.gamma_area * (s.U ** 2 + (2 * s.U - s.U_old) ** 2)
    E += 0.5 * m.gamma_bend * 3 * SQ2 / (8 * m.eps) * (s.W ** 2 + (2 * s.W - s.W_old) ** 2)
    E += 0.5 * (s.Z ** 2 + (2 * s.Z - s.Z_old) ** 2)
    E -= s.lam_sum
    return float(E)


def dissipation_K(s_new: State, s_prev: State, m: Model) -> float:
    """K^n of eq. K_n_explicit for levels (n+1, n, n-1) = (s_new.phi,
    s_new.phi_old = s_prev.phi, s_prev.phi_old)."""
    h = m.h
    a = s_new.phi - 2 * s_prev.phi + s_prev.phi_old
    La = lap(a, h)
    cb = m.gamma_bend * 3 * SQ2 * m.eps / 8
    cs = m.gamma_surf * 3 * SQ2 * m.eps / 4 + m.theta
    cbeta = m.gamma_surf * 3 * SQ2 * m.beta / (4 * m.eps)
    K = 0.5 * cb * ip(La, La, h)
    K += 0.5 * cs * grad_norm2(a, h)
    K += 1.5 * m.theta_tilde * grad_norm2(a, h)
    K += 0.5 * cbeta * ip(a, a, h)
    dd = lambda x1, x0, xm: x1 - 2 * x0 + xm
    K += 0.5 * m.gamma_surf * 3 * SQ2 / 2 * dd(s_new.V, s_prev.V, s_prev.V_old) ** 2
    K += 0.5 * m.gamma_area * dd(s_new.U, s_prev.U, s_prev.U_old) ** 2
    K += 0.5 * m.gamma_bend * 3 * SQ2 / (8 * m.eps) * dd(s_new.W, s_prev.W, s_prev.W_old) ** 2
    K += 0.5 * dd(s_new.Z, s_prev.Z, s_prev.Z_old) ** 2
    return float(K)


def physical_energy(phi, psi, m: Model, A: float) -> Dict[str, float]:
    """Energy components of eq. energy_functional with discrete norms."""
    h = m.h
    surf = surface_integral(phi, m)
    w = (phi ** 3 - phi) / m.eps - m.eps * lap(phi, h)
    bend = m.gamma_bend * 3 * SQ2 / (16 * m.eps) * ip(w, w, h)
    pp = p_fun(phi)
    osm = ip(0.5 * (1 + pp) * f_in(psi, m) + 0.5 * (1 - pp) * f_out(psi, m), np.ones_like(phi), h)
    area = 0.5 * m.gamma_area * (surf - A) ** 2
    return {"surf": m.gamma_surf * surf, "bend": bend, "area": area, "osm": osm,
            "arc_length": surf, "total": m.gamma_surf * surf + bend + area + osm}


# --------------------------------------------------------------------------
# Other boundary rules for the constant-coefficient solve (the paper's closing
# remarks: DST for Dirichlet, FFT for periodic boundaries) and the
# initial-condition smoother (Appendix F)
# --------------------------------------------------------------------------

BCS = ("neumann", "dirichlet", "periodic")


def ghost_bc(u: np.ndarray, bc: str) -> np.ndarray:
    """One ghost layer by the boundary rule: mirror (u_{-1} = u_0), odd
    (u_{-1} = -u_0, i.e. u = 0 on the boundary face) or periodic wrap."""
    if bc == "neumann":
        return np.pad(u, 1, mode="edge")
    if bc == "dirichlet":
        g = np.pad(u, 1, mode="edge")
        g[0, :] *= -1.0
        g[-1, :] *= -1.0
        g[:, 0] *= -1.0
        g[:, -1] *= -1.0
        return g
    if bc == "periodic":
        return np.pad(u, 1, mode="wrap")
    raise ValueError(bc)


def lap_bc(u: np.ndarray, h: float, bc: str) -> np.ndarray:
    """5-point Laplacian with the ghost layer of the boundary rule."""
    g = ghost_bc(u, bc)
    return (g[1:-1, 2:] + g[1:-1, :-2] + g[2:, 1:-1] + g[:-2, 1:-1] - 4.0 * u) / (h * h)


def transform_matrix(N: int, bc: str) -> np.ndarray:
    """Orthonormal (unitary) 1D transform that diagonalises the 1D Laplacian
    of the boundary rule, written out from its defining sum: DCT-II
    (Neumann), DST-II C[k, n] = c_k sin(pi (k+1)(2n+1)/(2N)) with
    c_{N-1} = sqrt(1/N), c_k = sqrt(2/N) otherwise (Dirichlet), and the DFT
    exp(-2 pi i k n / N)/sqrt(N) (periodic)."""
    k = np.arange(N, dtype=np.float64)[:, None]
    n = np.arange(N, dtype=np.float64)[None, :]
    if bc == "neumann":
        return dct_matrix(N)
    if bc == "dirichlet":
        S = np.sin(math.pi * (k + 1) * (2 * n + 1) / (2 * N))
        S[:-1, :] *= math.sqrt(2.0 / N)
        S[-1, :] *= math.sqrt(1.0 / N)
        return S
    if bc == "periodic":
        return np.exp(-2j * math.pi * k * n / N) / math.sqrt(N)
    raise ValueError(bc)


def bc_eigenvalues(N: int, h: float, bc: str) -> np.ndarray:
    """Eigenvalues of -Lap_h (1D) in the order of transform_matrix:
    (4/h^2) sin^2(pi k/(2N)), sin^2(pi (k+1)/(2N)), sin^2(pi k/N)."""
    k = np.arange(N, dtype=np.float64)
    if bc == "neumann":
        a = math.pi * k / (2 * N)
    elif bc == "dirichlet":
        a = math.pi * (k + 1) / (2 * N)
    elif bc == "periodic":
        a = math.pi * k / N
    else:
        raise ValueError(bc)
    return 4.0 / (h * h) * np.sin(a) ** 2


def spectral_solve_bc(f: np.ndarray, coef, h: float, bc: str) -> np.ndarray:
    """u = (c0 - c1 Lap_h + c2 Lap_h^2)^{-1} f: forward transform along both
    axes, division by c0 + c1 s + c2 s^2 (s = s_k + s_l), inverse transform."""
    N = f.shape[0]
    C = transform_matrix(N, bc)
    e = bc_eigenvalues(N, h, bc)
    s = e[:, None] + e[None, :]
    F = C @ f @ C.T
    U = F / (coef[0] + coef[1] * s + coef[2] * s * s)
    u = C.conj().T @ U @ C.conj()
    return np.real(u) if bc == "periodic" else u


def smooth_initial(phi: np.ndarray, h: float, eps: float, mobility: float, dt: float,
                   nsteps: int, bc: str = "neumann") -> np.ndarray:
    """Appendix F: nsteps of the constant-mobility Cahn-Hilliard equation
    phi_t = Mob Lap((phi^3 - phi)/eps - eps Lap phi), first order in time
    with the nonlinear term explicit and the biharmonic term implicit,
        (1/dt + Mob eps Lap_h^2) phi^{n+1} = phi^n/dt + Mob Lap_h((phi^n^3 - phi^n)/eps),
    solved by the transform of the boundary rule; then phi is clamped to [-1, 1]."""
    u = np.array(phi, dtype=np.float64)
    for _ in range(nsteps):
        rhs = u / dt + mobility * lap_bc((u ** 3 - u) / eps, h, bc)
        u = spectral_solve_bc(rhs, (1.0 / dt, 0.0, mobility * eps), h, bc)
    return np.clip(u, -1.0, 1.0)
