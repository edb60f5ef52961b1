"""FP64 CPU oracle of the TRT-R lattice Boltzmann step (arXiv 2312.10316), ctypes wrapper.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are the only callers.  The CUDA library never imports, links or calls it,
and this module imports nothing from the CUDA path.

The C source (``trtr_oracle.c``) writes the paper's evolution equation out literally in
physical units with push streaming; see its header for the readings of the points the
paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import sysconfig
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trtr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

Q = 9
_dbl_p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, openmp: bool = True, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle with gcc into a shared object; returns its path."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    cmd = [cc, "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", src, "-o", out + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("tau2_mode", ctypes.c_int), ("magic", ctypes.c_double), ("tau2", ctypes.c_double),
        ("tau1_const", ctypes.c_double),
        ("grad_mode", ctypes.c_int), ("src_mode", ctypes.c_int),
        ("omega", ctypes.c_double), ("xc", ctypes.c_double), ("yc", ctypes.c_double),
        ("sigma0", ctypes.c_double), ("D0", ctypes.c_double), ("D_amp", ctypes.c_double),
        ("bc_mode", ctypes.c_int),
    ]


class PaperParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("kappa", ctypes.c_double), ("dt", ctypes.c_double),
                ("model", ctypes.c_int), ("magic", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load (building first if needed) the oracle shared object."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or build()
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    sig = {
        "oracle_equilibrium": (None, [ctypes.c_double] * 5 + [_dbl_p]),
        "oracle_collide": (None, [ctypes.c_double, ctypes.c_double, _dbl_p] + [ctypes.c_double] * 4 + [_dbl_p]),
        "oracle_aux_G": (None, [ctypes.c_double] * 5 + [_dbl_p, ctypes.c_double, _dbl_p]),
        "oracle_source_F": (None, [ctypes.c_double] * 6 + [_dbl_p]),
        "oracle_tau1": (ctypes.c_double, [ctypes.c_double] * 3),
        "oracle_tau2_magic": (ctypes.c_double, [ctypes.c_double] * 2),
        "oracle_d2q9": (None, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dbl_p]),
        "oracle_create": (vp, [ctypes.POINTER(Params)]),
        "oracle_destroy": (None, [vp]),
        "oracle_set_fields": (None, [vp, _dbl_p, _dbl_p, _dbl_p]),
        "oracle_set_source": (None, [vp, _dbl_p]),
        "oracle_set_source_prev": (None, [vp, _dbl_p]),
        "oracle_set_dirichlet": (None, [vp, _dbl_p]),
        "oracle_pulse_source": (None, [vp, ctypes.c_double, _dbl_p]),
        "oracle_init_equilibrium": (None, [vp, _dbl_p]),
        "oracle_step": (None, [vp, ctypes.c_long]),
        "oracle_step_rows_sample": (None, [vp, ctypes.c_int, ctypes.c_int]),
        "oracle_step_count": (ctypes.c_long, [vp]),
        "oracle_phi": (None, [vp, _dbl_p]),
        "oracle_get_g": (None, [vp, _dbl_p]),
        "oracle_set_g": (None, [vp, _dbl_p, ctypes.c_long]),
        "oracle_mass": (ctypes.c_double, [vp]),
        "oracle_error": (None, [vp, _dbl_p, _dbl_p, _dbl_p]),
        "oracle_num_threads": (ctypes.c_int, []),
        "oracle_node_post": (None, [ctypes.POINTER(Params), _dbl_p, ctypes.c_double, ctypes.c_double, _dbl_p,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, _dbl_p]),
        "oracle_pulse_source_at": (ctypes.c_double, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "oracle_adjoint": (ctypes.c_int, [vp, ctypes.c_long, _dbl_p, _dbl_p, _dbl_p]),
        "oracle_paper_pulse": (ctypes.c_int, [ctypes.POINTER(PaperParams), ctypes.c_double, _dbl_p, _dbl_p]),
        "oracle_paper_slip": (ctypes.c_long, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_long, ctypes.c_double, _dbl_p, _dbl_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dbl_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------------------
# Single-node functions


def equilibrium(dx, dt, phi, ux, uy, lib=None) -> np.ndarray:
    lib = lib or load()
    out = np.zeros(Q)
    lib.oracle_equilibrium(dx, dt, phi, ux, uy, _ptr(out))
    return out


def collide(dx, dt, g, ux, uy, tau1, tau2, lib=None) -> np.ndarray:
    lib = lib or load()
    g = _f64(g)
    out = np.zeros(Q)
    lib.oracle_collide(dx, dt, _ptr(g), ux, uy, tau1, tau2, _ptr(out))
    return out


def aux_G(dx, dt, phi, ux, uy, du, tau1, lib=None) -> np.ndarray:
    """du = [d_x u_x, d_y u_x, d_x u_y, d_y u_y]."""
    lib = lib or load()
    du = _f64(du)
    out = np.zeros(Q)
    lib.oracle_aux_G(dx, dt, phi, ux, uy, _ptr(du), tau1, _ptr(out))
    return out


def source_F(dx, dt, S, ux, uy, tau1, lib=None) -> np.ndarray:
    lib = lib or load()
    out = np.zeros(Q)
    lib.oracle_source_F(dx, dt, S, ux, uy, tau1, _ptr(out))
    return out


def node_post(p: "SimParams", g, ux, uy, du, D, Sn=0.0, Snm1=0.0, lib=None) -> np.ndarray:
    """Right-hand side of the evolution equation at one node (collision + dt G + dt F + dt^2/2 d_t F).
    du = [d_x u_x, d_y u_x, d_x u_y, d_y u_y] in physical units."""
    lib = lib or load()
    cp = p.to_c()
    g = _f64(g)
    du = _f64(du)
    out = np.zeros(Q)
    lib.oracle_node_post(ctypes.byref(cp), _ptr(g), ux, uy, _ptr(du), D, Sn, Snm1, _ptr(out))
    return out


def tau1(D, dx, dt, lib=None) -> float:
    return (lib or load()).oracle_tau1(D, dx, dt)


def tau2_magic(t1, magic, lib=None) -> float:
    return (lib or load()).oracle_tau2_magic(t1, magic)


def d2q9(lib=None):
    lib = lib or load()
    ex = (ctypes.c_int * Q)()
    ey = (ctypes.c_int * Q)()
    w = (ctypes.c_double * Q)()
    lib.oracle_d2q9(ex, ey, w)
    return np.array(ex[:]), np.array(ey[:]), np.array(w[:])


# --------------------------------------------------------------------------------------
# Grid simulation


@dataclass
class SimParams:
    nx: int
    ny: int
    dx: float
    dt: float
    x0: float = -1.0
    y0: float = -1.0
    tau2_mode: int = 0       # 0 magic, 1 fixed
    magic: float = 1.0 / 12.0
    tau2: float = 1.0
    tau1_const: float = 0.0
    grad_mode: int = 1       # 0 periodic central, 1 one-sided at the edges
    src_mode: int = 0        # 0 none, 1 field, 2 manufactured pulse
    omega: float = 0.0
    xc: float = 0.0
    yc: float = 0.0
    sigma0: float = 0.1
    D0: float = 0.0
    D_amp: float = 0.0
    bc_mode: int = 0         # 0 periodic, 1 Dirichlet by non-equilibrium extrapolation

    def to_c(self) -> Params:
        return Params(**{k: getattr(self, k) for k, _ in Params._fields_})


class Sim:
    """Grid state g_i(x, t_n) of the oracle; arrays are [ny][nx] (x fastest) and [9][ny][nx]."""

    def __init__(self, p: SimParams, lib=None):
        self.lib = lib or load()
        self.p = p
        self._cp = p.to_c()
        self.h = self.lib.oracle_create(ctypes.byref(self._cp))
        if not self.h:
            raise ValueError(f"oracle_create rejected {p}")
        self.shape = (p.ny, p.nx)

    def close(self):
        if self.h:
            self.lib.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, a):
        a = _f64(a)
        if a.shape != self.shape:
            raise ValueError(f"field shape {a.shape} != {self.shape}")
        return a

    def set_fields(self, ux, uy, D):
        self._keep = (self._field(ux), self._field(uy), self._field(D))
        self.lib.oracle_set_fields(self.h, *(_ptr(a) for a in self._keep))

    def set_source(self, S):
        S = self._field(S)
        self.lib.oracle_set_source(self.h, _ptr(S))

    def set_source_prev(self, S):
        S = self._field(S)
        self.lib.oracle_set_source_prev(self.h, _ptr(S))

    def set_dirichlet(self, phi_b):
        phi_b = self._field(phi_b)
        self.lib.oracle_set_dirichlet(self.h, _ptr(phi_b))

    def pulse_source(self, t) -> np.ndarray:
        out = np.zeros(self.shape)
        self.lib.oracle_pulse_source(self.h, float(t), _ptr(out))
        return out

    def pulse_source_at(self, x, y, t) -> float:
        return float(self.lib.oracle_pulse_source_at(self.h, float(x), float(y), float(t)))

    def init_equilibrium(self, phi0):
        phi0 = self._field(phi0)
        self.lib.oracle_init_equilibrium(self.h, _ptr(phi0))

    def step(self, n: int = 1):
        self.lib.oracle_step(self.h, int(n))

    def step_rows_sample(self, j0: int, j1: int):
        self.lib.oracle_step_rows_sample(self.h, int(j0), int(j1))

    @property
    def step_count(self) -> int:
        return int(self.lib.oracle_step_count(self.h))

    def phi(self) -> np.ndarray:
        out = np.zeros(self.shape)
        self.lib.oracle_phi(self.h, _ptr(out))
        return out

    def get_g(self) -> np.ndarray:
        out = np.zeros((Q,) + self.shape)
        self.lib.oracle_get_g(self.h, _ptr(out))
        return out

    def set_g(self, g, step: int = 0):
        g = _f64(g)
        if g.shape != (Q,) + self.shape:
            raise ValueError("bad population shape")
        self.lib.oracle_set_g(self.h, _ptr(g), int(step))

    def adjoint(self, nsteps: int, lamN, want_lam0: bool = False):
        """Runs nsteps forward (the state advances) and sweeps back: returns dJ/dD [ny][nx]
        (and dJ/dg^0 [9][ny][nx]) for lamN = dJ/dphi^N."""
        lamN = self._field(lamN)
        grad = np.zeros(self.shape)
        lam0 = np.zeros((Q,) + self.shape) if want_lam0 else None
        rc = self.lib.oracle_adjoint(self.h, int(nsteps), _ptr(lamN), _ptr(grad),
                                     _ptr(lam0) if want_lam0 else None)
        if rc != 0:
            raise RuntimeError("oracle_adjoint: out of memory, or the boundaries are not periodic")
        return (grad, lam0) if want_lam0 else grad

    def mass(self) -> float:
        return float(self.lib.oracle_mass(self.h))

    def error(self, phi_ref):
        phi_ref = self._field(phi_ref)
        rms = ctypes.c_double()
        rel = ctypes.c_double()
        self.lib.oracle_error(self.h, _ptr(phi_ref), ctypes.byref(rms), ctypes.byref(rel))
        return rms.value, rel.value


def num_threads(lib=None) -> int:
    return int((lib or load()).oracle_num_threads())


def paper_pulse(N: int, kappa: float, dt: float, model: int = 0, t_end: float = 1.0, magic: float = 1.0 / 12.0,
                L: float = 4.0 * np.pi, lib=None, want_phi: bool = False):
    """The paper's rotating-pulse benchmark (Sec. 3) to t_end: (RMS error of Eq. (33), blew_up)
    and, with want_phi, phi at t_end ([N + 1][N + 1])."""
    lib = lib or load()
    pp = PaperParams(N, L, kappa, dt, model, magic)
    rms = ctypes.c_double()
    phi = np.zeros((N + 1, N + 1)) if want_phi else None
    rc = lib.oracle_paper_pulse(ctypes.byref(pp), float(t_end), ctypes.byref(rms),
                                _ptr(phi) if want_phi else None)
    if rc < 0:
        raise ValueError("bad benchmark parameters")
    if want_phi:
        return rms.value, bool(rc), phi
    return rms.value, bool(rc)


def paper_slip(ny: int, tau1: float, tau2: float, S: float = 1e-3, phi_w: float = 0.0, max_steps: int = 200000,
               tol: float = 1e-16, lib=None):
    """Steady wall-bounded diffusion (Sec. 3.2): (RMS error against the parabola, phi [ny], steps)."""
    lib = lib or load()
    rms = ctypes.c_double()
    phi = np.zeros(ny)
    n = lib.oracle_paper_slip(int(ny), float(tau1), float(tau2), float(S), float(phi_w), int(max_steps), float(tol),
                              ctypes.byref(rms), _ptr(phi))
    if n < 0:
        raise ValueError("bad slip-check parameters")
    return rms.value, phi, int(n)
