"""Python binding of the C ABI in ``include/ccmsav.h`` (ctypes; argument
marshalling only -- every step of the method runs in the CUDA library).

The functions keep the C names.  ``Simulation`` is a small convenience
wrapper that owns one handle and converts numpy arrays.  Loading fails
loudly (``RuntimeError``) when the compiled library is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libccmsav.so")
LIB_BOUNDS_PATH = os.path.join(HERE, "libccmsav_bounds.so")   # index-checked test build

CCMSAV_OK = 0
CCMSAV_EINVAL = -1
CCMSAV_ENOMEM = -2
CCMSAV_ECUDA = -3
CCMSAV_ESTATE = -4
CCMSAV_ENONFINITE = -5
CCMSAV_ETIMEOUT = -6
CCMSAV_FP64 = 0
CCMSAV_FP32_BULK = 1
CCMSAV_TRACK_ENERGY = 1
CCMSAV_BDF1_ALWAYS = 2
CCMSAV_CLASSICAL = 4
CCMSAV_BC_NEUMANN = 0
CCMSAV_BC_DIRICHLET = 1
CCMSAV_BC_PERIODIC = 2
BC_CODES = {"neumann": CCMSAV_BC_NEUMANN, "dirichlet": CCMSAV_BC_DIRICHLET, "periodic": CCMSAV_BC_PERIODIC}

PARAM_FIELDS = ["gamma_surf", "gamma_bend", "gamma_area", "gamma_in", "gamma_out",
                "psi_in", "psi_out", "beta_in", "beta_out", "eps", "M_phi", "M0",
                "theta", "beta", "lam", "dt", "L"]


class ccmsav_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in PARAM_FIELDS]

    @classmethod
    def from_obj(cls, p) -> "ccmsav_params":
        return cls(*[float(getattr(p, n)) for n in PARAM_FIELDS])


class CCMSAVError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {ccmsav_strerror(status)} ({status})")
        self.status = status


_lib = None
_DP = C.POINTER(C.c_double)


def load(path: Optional[str] = None) -> C.CDLL:
    """Load libccmsav.so (built by ``paper_2601_10057_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2601_10057_gb300.build` (nvcc, sm_103a)")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "ccmsav_create": (i, [C.POINTER(vp), C.POINTER(ccmsav_params), i, C.POINTER(i),
                              C.POINTER(ccmsav_params), i, i, vp]),
        "ccmsav_set_state": (i, [vp, i, _DP, _DP]),
        "ccmsav_set_state_device": (i, [vp, i, vp, vp]),
        "ccmsav_set_state_levels": (i, [vp, i, _DP, _DP, _DP, _DP]),
        "ccmsav_step": (i, [vp, i]),
        "ccmsav_sync": (i, [vp]),
        "ccmsav_get_state": (i, [vp, i, _DP, _DP]),
        "ccmsav_get_prev_state": (i, [vp, i, _DP, _DP]),
        "ccmsav_energy": (i, [vp, i, _DP]),
        "ccmsav_mass": (i, [vp, i, _DP]),
        "ccmsav_get_aux": (i, [vp, i, _DP]),
        "ccmsav_get_aux_async": (i, [vp, i, _DP]),
        "ccmsav_set_aux": (i, [vp, i, _DP]),
        "ccmsav_grid_size": (i, [vp, i]),
        "ccmsav_launch_count": (C.c_longlong, [vp]),
        "ccmsav_strerror": (C.c_char_p, [i]),
        "ccmsav_profile": (i, [vp, i]),
        "ccmsav_profile_read": (i, [vp, i, _DP, C.POINTER(C.c_longlong)]),
        "ccmsav_destroy": (None, [vp]),
        "ccmsav_mass_noalloc": (i, [vp, i, i, d, _DP, vp]),
        "ccmsav_set_pcg": (i, [vp, d, i]),
        "ccmsav_autotune": (i, [vp, i, _DP]),
        "ccmsav_bounds_flag": (i, [vp]),
        "ccmsav_set_group_points": (i, [vp, C.c_longlong]),
        "ccmsav_group_points": (C.c_longlong, [vp]),
        "ccmsav_pcg_stats": (i, [vp, i, _DP]),
        "ccmsav_solver_create": (i, [C.POINTER(vp), i, d, i, i, vp]),
        "ccmsav_solver_solve": (i, [vp, _DP, vp, vp]),
        "ccmsav_solver_smooth": (i, [vp, d, d, d, i, vp]),
        "ccmsav_solver_sync": (i, [vp]),
        "ccmsav_solver_launch_count": (C.c_longlong, [vp]),
        "ccmsav_solver_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- C names

def ccmsav_strerror(status: int) -> str:
    return load().ccmsav_strerror(int(status)).decode()


def ccmsav_create(params, N: Sequence[int], precision: int = CCMSAV_FP64, flags: int = 0,
                  stream: Optional[int] = None, per_sim: Optional[Sequence] = None):
    """Returns (status, handle)."""
    lib = load()
    n = len(N)
    Ns = (C.c_int * n)(*[int(x) for x in N])
    h = C.c_void_p()
    p = C.byref(ccmsav_params.from_obj(params)) if params is not None else None
    ps = None
    if per_sim is not None:
        arr = (ccmsav_params * n)(*[ccmsav_params.from_obj(q) for q in per_sim])
        ps = C.cast(arr, C.POINTER(ccmsav_params))
    st = lib.ccmsav_create(C.byref(h), p, n, Ns, ps, int(precision), int(flags),
                           C.c_void_p(stream) if stream else None)
    return st, h


def ccmsav_set_state(h, sim: int, phi, psi) -> int:
    phi, psi = _f64(phi), _f64(psi)
    return load().ccmsav_set_state(h, sim, _ptr(phi), _ptr(psi))


def ccmsav_set_state_device(h, sim: int, phi_ptr: int, psi_ptr: int) -> int:
    return load().ccmsav_set_state_device(h, sim, C.c_void_p(phi_ptr), C.c_void_p(psi_ptr))


def ccmsav_set_state_levels(h, sim: int, phi, psi, phi_prev, psi_prev) -> int:
    a = [_f64(x) for x in (phi, psi, phi_prev, psi_prev)]
    return load().ccmsav_set_state_levels(h, sim, *[_ptr(x) for x in a])


def ccmsav_step(h, nsteps: int) -> int:
    return load().ccmsav_step(h, int(nsteps))


def ccmsav_sync(h) -> int:
    return load().ccmsav_sync(h)


def ccmsav_get_state(h, sim: int, N: int, prev: bool = False):
    phi = np.empty((N, N), np.float64)
    psi = np.empty((N, N), np.float64)
    fn = load().ccmsav_get_prev_state if prev else load().ccmsav_get_state
    st = fn(h, sim, _ptr(phi), _ptr(psi))
    return st, phi, psi


def ccmsav_energy(h, sim: int):
    out = np.zeros(8, np.float64)
    st = load().ccmsav_energy(h, sim, _ptr(out))
    return st, out


def ccmsav_mass(h, sim: int):
    out = np.zeros(1, np.float64)
    st = load().ccmsav_mass(h, sim, _ptr(out))
    return st, float(out[0])


def ccmsav_get_aux(h, sim: int):
    out = np.zeros(12, np.float64)
    st = load().ccmsav_get_aux(h, sim, _ptr(out))
    return st, out


def ccmsav_get_aux_async(h, sim: int, out: np.ndarray) -> int:
    """Queue the copy of the twelve scalars into ``out`` (float64, 12 values,
    C-contiguous; ideally page-locked).  ``out`` must stay alive and is valid
    only after a synchronising call."""
    if out.dtype != np.float64 or out.size < 12 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array of 12 values")
    return load().ccmsav_get_aux_async(h, sim, _ptr(out))


def ccmsav_set_aux(h, sim: int, aux) -> int:
    aux = _f64(aux)
    return load().ccmsav_set_aux(h, sim, _ptr(aux))


def ccmsav_grid_size(h, sim: int) -> int:
    return load().ccmsav_grid_size(h, sim)


def ccmsav_launch_count(h) -> int:
    return int(load().ccmsav_launch_count(h))


def ccmsav_profile(h, enable: bool) -> int:
    return load().ccmsav_profile(h, 1 if enable else 0)


KERNEL_NAMES = ["k_stencil", "k_rowdct_T", "k_coldct_gram", "k_solve", "k_comb_icolT",
                "k_irow", "k_dnorm+k_add_lamsum", "unused"]


def ccmsav_profile_read(h, sim: int = 0):
    """Returns (status, ms[8], nsteps)."""
    ms = np.zeros(8, np.float64)
    n = C.c_longlong(0)
    st = load().ccmsav_profile_read(h, sim, _ptr(ms), C.byref(n))
    return st, ms, int(n.value)


def ccmsav_destroy(h) -> None:
    if h:
        load().ccmsav_destroy(h)


def ccmsav_mass_noalloc(psi_ptr: int, N: int, precision: int, L: float, stream: Optional[int] = None):
    """Mass of a caller-owned device field without library allocation.
    Returns (status, mass)."""
    out = np.zeros(1, np.float64)
    st = load().ccmsav_mass_noalloc(C.c_void_p(psi_ptr), int(N), int(precision), float(L), _ptr(out),
                                    C.c_void_p(stream) if stream else None)
    return st, float(out[0])


def ccmsav_bounds_flag(h) -> int:
    return load().ccmsav_bounds_flag(h)


def ccmsav_autotune(h, steps: int, n_sims: int):
    """Returns (status, report[n_sims, 4]): warp path, carveout, best and
    default ms/step per simulation."""
    rep = np.zeros((n_sims, 4), np.float64)
    st = load().ccmsav_autotune(h, int(steps), _ptr(rep))
    return st, rep


def ccmsav_set_group_points(h, points: int) -> int:
    return load().ccmsav_set_group_points(h, int(points))


def ccmsav_group_points(h) -> int:
    return load().ccmsav_group_points(h)


def ccmsav_set_pcg(h, rtol: float, max_iter: int) -> int:
    return load().ccmsav_set_pcg(h, float(rtol), int(max_iter))


def ccmsav_pcg_stats(h, sim: int = 0):
    """Returns (status, [iterations of the last step, total iterations,
    relative residual of solve 1, of solve 2])."""
    out = np.zeros(4, np.float64)
    st = load().ccmsav_pcg_stats(h, sim, _ptr(out))
    return st, out


def ccmsav_solver_create(N: int, L: float, bc: int, precision: int, stream: Optional[int] = None):
    """Returns (status, solver handle)."""
    h = C.c_void_p()
    st = load().ccmsav_solver_create(C.byref(h), int(N), float(L), int(bc), int(precision),
                                     C.c_void_p(stream) if stream else None)
    return st, h


def ccmsav_solver_solve(s, coef, f_ptr: int, u_ptr: int) -> int:
    c = _f64(coef)
    return load().ccmsav_solver_solve(s, _ptr(c), C.c_void_p(f_ptr), C.c_void_p(u_ptr))


def ccmsav_solver_smooth(s, eps: float, mobility: float, dt: float, nsteps: int, phi_ptr: int) -> int:
    return load().ccmsav_solver_smooth(s, float(eps), float(mobility), float(dt), int(nsteps), C.c_void_p(phi_ptr))


def ccmsav_solver_sync(s) -> int:
    return load().ccmsav_solver_sync(s)


def ccmsav_solver_launch_count(s) -> int:
    return int(load().ccmsav_solver_launch_count(s))


def ccmsav_solver_destroy(s) -> None:
    if s:
        load().ccmsav_solver_destroy(s)


# ---------------------------------------------------------------- wrapper

class Simulation:
    """Owns one handle for one or more simulations; raises on error codes."""

    def __init__(self, params, N, precision: str = "fp64", track_energy: bool = False,
                 stream: Optional[int] = None, per_sim=None, bdf1_always: bool = False,
                 classical: bool = False):
        Ns = [int(N)] if np.isscalar(N) else [int(x) for x in N]
        prec = CCMSAV_FP64 if precision == "fp64" else CCMSAV_FP32_BULK
        flags = ((CCMSAV_TRACK_ENERGY if track_energy else 0) | (CCMSAV_BDF1_ALWAYS if bdf1_always else 0)
                 | (CCMSAV_CLASSICAL if classical else 0))
        st, h = ccmsav_create(params, Ns, prec, flags, stream, per_sim)
        if st != CCMSAV_OK:
            raise CCMSAVError(st, "ccmsav_create")
        self.h, self.N, self.precision = h, Ns, precision

    def _check(self, st, where):
        if st != CCMSAV_OK:
            raise CCMSAVError(st, where)

    def set_state(self, phi, psi, sim: int = 0):
        self._check(ccmsav_set_state(self.h, sim, phi, psi), "ccmsav_set_state")

    def set_levels(self, phi, psi, phi_prev, psi_prev, sim: int = 0):
        self._check(ccmsav_set_state_levels(self.h, sim, phi, psi, phi_prev, psi_prev),
                    "ccmsav_set_state_levels")

    def step(self, n: int = 1):
        self._check(ccmsav_step(self.h, n), "ccmsav_step")

    def sync(self):
        self._check(ccmsav_sync(self.h), "ccmsav_sync")

    def state(self, sim: int = 0, prev: bool = False):
        st, phi, psi = ccmsav_get_state(self.h, sim, self.N[sim], prev)
        self._check(st, "ccmsav_get_state")
        return phi, psi

    def energy(self, sim: int = 0):
        st, out = ccmsav_energy(self.h, sim)
        self._check(st, "ccmsav_energy")
        return out

    def mass(self, sim: int = 0) -> float:
        st, m = ccmsav_mass(self.h, sim)
        self._check(st, "ccmsav_mass")
        return m

    def aux(self, sim: int = 0):
        st, a = ccmsav_get_aux(self.h, sim)
        self._check(st, "ccmsav_get_aux")
        return a

    def aux_async(self, out: np.ndarray, sim: int = 0):
        """Queue the scalars' copy into ``out`` (see ccmsav_get_aux_async)."""
        self._check(ccmsav_get_aux_async(self.h, sim, out), "ccmsav_get_aux_async")

    def set_aux(self, aux, sim: int = 0):
        self._check(ccmsav_set_aux(self.h, sim, aux), "ccmsav_set_aux")

    def launches(self) -> int:
        return ccmsav_launch_count(self.h)

    def autotune(self, steps: int = 12):
        """Pick the fastest line-transform schedule per grid size (ccmsav_autotune)."""
        st, rep = ccmsav_autotune(self.h, steps, len(self.N))
        self._check(st, "ccmsav_autotune")
        return rep

    def set_group_points(self, points: int):
        """Grid points per launch group of the batched step (0: no grouping)."""
        self._check(ccmsav_set_group_points(self.h, points), "ccmsav_set_group_points")

    def group_points(self) -> int:
        return ccmsav_group_points(self.h)

    def set_pcg(self, rtol: float, max_iter: int = 200):
        self._check(ccmsav_set_pcg(self.h, rtol, max_iter), "ccmsav_set_pcg")

    def pcg_stats(self, sim: int = 0):
        st, out = ccmsav_pcg_stats(self.h, sim)
        self._check(st, "ccmsav_pcg_stats")
        return out

    def close(self):
        if self.h:
            ccmsav_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SpectralSolver:
    """Owns one ccmsav_solver handle; fields are torch CUDA tensors of the
    solver's precision (float64 or float32), N x N, contiguous."""

    def __init__(self, N: int, L: float, bc: str = "neumann", precision: str = "fp64",
                 stream: Optional[int] = None):
        prec = CCMSAV_FP64 if precision == "fp64" else CCMSAV_FP32_BULK
        st, h = ccmsav_solver_create(N, L, BC_CODES[bc], prec, stream)
        if st != CCMSAV_OK:
            raise CCMSAVError(st, "ccmsav_solver_create")
        self.h, self.N, self.precision = h, int(N), precision

    def _chk(self, t):
        import torch
        want = torch.float64 if self.precision == "fp64" else torch.float32
        if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.numel() != self.N * self.N:
            raise ValueError(f"expected a contiguous CUDA {want} tensor of {self.N} x {self.N} values")
        return t.data_ptr()

    def solve(self, coef, f, out=None):
        """u = (c0 - c1 Lap_h + c2 Lap_h^2)^{-1} f (asynchronous on the solver's stream)."""
        import torch
        u = torch.empty_like(f) if out is None else out
        st = ccmsav_solver_solve(self.h, coef, self._chk(f), self._chk(u))
        if st != CCMSAV_OK:
            raise CCMSAVError(st, "ccmsav_solver_solve")
        return u

    def smooth(self, phi, eps: float, mobility: float = 0.01, dt: float = 1e-6, nsteps: int = 10):
        """The smoother of Appendix F in place on phi (then clamped to [-1, 1])."""
        st = ccmsav_solver_smooth(self.h, eps, mobility, dt, nsteps, self._chk(phi))
        if st != CCMSAV_OK:
            raise CCMSAVError(st, "ccmsav_solver_smooth")
        return phi

    def sync(self):
        st = ccmsav_solver_sync(self.h)
        if st != CCMSAV_OK:
            raise CCMSAVError(st, "ccmsav_solver_sync")

    def launches(self) -> int:
        return ccmsav_solver_launch_count(self.h)

    def close(self):
        if self.h:
            ccmsav_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
