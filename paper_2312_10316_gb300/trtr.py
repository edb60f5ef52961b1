"""Python binding of the C ABI in ``include/trtr.h`` (argument marshalling only).

Every function keeps the C name and forwards to ``libtrtr.so``; all computation runs in the
library's CUDA kernels.  Arrays are numpy float64 (host, ``on_device=0``) or CUDA torch
tensors of dtype float64 (device, ``on_device=1``); torch provides device memory and the
stream handle only.  There is no fallback: if ``libtrtr.so`` is missing or fails to load,
importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields as dc_fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TRTR_BOUNDS_CHECK=1 in the environment loads the bounds-checked debug build instead
BOUNDS_CHECKED = os.environ.get("TRTR_BOUNDS_CHECK", "0") == "1"
LIB_PATH = os.path.join(_HERE, "libtrtr_checked.so" if BOUNDS_CHECKED else "libtrtr.so")

TRTR_OK, TRTR_EINVAL, TRTR_ENOMEM, TRTR_ECUDA, TRTR_EUNSTABLE, TRTR_ETIMEOUT, TRTR_ESTATE, TRTR_EBOUNDS = range(8)
TRTR_F64, TRTR_F32, TRTR_F16_OFS, TRTR_BF16_OFS = range(4)
TRTR_TAU2_MAGIC, TRTR_TAU2_FIXED = range(2)
TRTR_GRAD_PERIODIC, TRTR_GRAD_ONESIDED_EDGE = range(2)
TRTR_SRC_NONE, TRTR_SRC_FIELD, TRTR_SRC_PULSE = range(3)
TRTR_BC_PERIODIC, TRTR_BC_DIRICHLET_NEE = range(2)
TRTR_ROUND_STOCHASTIC, TRTR_ROUND_NEAREST = range(2)

PRECISIONS = {"f64": TRTR_F64, "f32": TRTR_F32, "f16": TRTR_F16_OFS, "bf16": TRTR_BF16_OFS}


class TrtrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class trtr_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("precision", ctypes.c_int), ("phi_ref", ctypes.c_double),
        ("tau2_mode", ctypes.c_int), ("magic", ctypes.c_double), ("tau2", ctypes.c_double),
        ("tau1_const", ctypes.c_double),
        ("grad_mode", ctypes.c_int), ("src_mode", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("bc_mode", ctypes.c_int),
        ("rounding", ctypes.c_int),
    ]


class trtr_instance(ctypes.Structure):
    _fields_ = [("p", trtr_params), ("omega", ctypes.c_double), ("xc", ctypes.c_double), ("yc", ctypes.c_double),
                ("sigma0", ctypes.c_double), ("D0", ctypes.c_double), ("D_amp", ctypes.c_double)]


_dbl_p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_st = ctypes.c_int

_SIGNATURES = {
    "trtr_create": (_st, [ctypes.POINTER(trtr_params), _vp, ctypes.POINTER(_vp)]),
    "trtr_destroy": (_st, [_vp]),
    "trtr_set_fields": (_st, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "trtr_set_source": (_st, [_vp, _vp, ctypes.c_int]),
    "trtr_set_source_prev": (_st, [_vp, _vp, ctypes.c_int]),
    "trtr_set_dirichlet": (_st, [_vp, _vp, ctypes.c_int]),
    "trtr_set_pulse": (_st, [_vp] + [ctypes.c_double] * 6),
    "trtr_init_equilibrium": (_st, [_vp, _vp, ctypes.c_int]),
    "trtr_step": (_st, [_vp, ctypes.c_long]),
    "trtr_moments": (_st, [_vp, _vp, ctypes.c_int]),
    "trtr_mass": (_st, [_vp, _dbl_p]),
    "trtr_error_vs_pulse": (_st, [_vp, _dbl_p, _dbl_p]),
    "trtr_error_vs": (_st, [_vp, _vp, ctypes.c_int, _dbl_p, _dbl_p]),
    "trtr_get_populations": (_st, [_vp, _vp, ctypes.c_int]),
    "trtr_set_populations": (_st, [_vp, _vp, ctypes.c_int, ctypes.c_long]),
    "trtr_sample_populations": (_st, [_vp, ctypes.POINTER(ctypes.c_long), ctypes.c_int, _dbl_p]),
    "trtr_time": (_st, [_vp, ctypes.POINTER(ctypes.c_long), _dbl_p]),
    "trtr_save": (_st, [_vp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
    "trtr_load": (_st, [_vp, _vp, ctypes.c_size_t]),
    "trtr_sync": (_st, [_vp]),
    "trtr_launch_count": (_st, [_vp, ctypes.POINTER(ctypes.c_long)]),
    "trtr_phi_sums_noalloc": (_st, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    "trtr_forward_record": (_st, [_vp, ctypes.c_long, ctypes.c_int]),
    "trtr_adjoint": (_st, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int]),
    "trtr_batch_create": (_st, [ctypes.POINTER(trtr_instance), ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "trtr_batch_destroy": (_st, [_vp]),
    "trtr_batch_config_count": (ctypes.c_int, []),
    "trtr_batch_config_name": (ctypes.c_char_p, [ctypes.c_int]),
    "trtr_batch_tune": (_st, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "trtr_batch_set_config": (_st, [_vp, ctypes.c_int]),
    "trtr_batch_step": (_st, [_vp, ctypes.c_long]),
    "trtr_batch_sync": (_st, [_vp]),
    "trtr_batch_instance": (_st, [_vp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "trtr_batch_info": (_st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int)]),
    "trtr_status_str": (ctypes.c_char_p, [_st]),
    "trtr_last_error": (ctypes.c_char_p, [_vp]),
    "trtr_d2q9": (None, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dbl_p]),
    "trtr_abi_version": (ctypes.c_int, []),
    "trtr_check_timeout_path": (_st, [_vp, ctypes.c_longlong]),
    "trtr_bounds_checked": (ctypes.c_int, []),
    "trtr_bounds_report": (_st, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "trtr_check_bounds_path": (_st, [_vp]),
    "trtr_set_steps_per_launch": (_st, [_vp, ctypes.c_int]),
    "trtr_batch_set_steps_per_launch": (_st, [_vp, ctypes.c_int]),
    "trtr_batch_get_steps_per_launch": (_st, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "trtr_get_steps_per_launch": (_st, [_vp, ctypes.POINTER(ctypes.c_int)]),
}


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2312_10316_gb300.build.build_library"
                          f"({'checked=True' if BOUNDS_CHECKED else ''})")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def symbols() -> list[str]:
    return list(_SIGNATURES)


# --------------------------------------------------------------------------------------
# marshalling helpers


def _arr(a, count: int | None = None):
    """(pointer, on_device, keepalive) for a float64 numpy array or CUDA torch tensor."""
    if a is None:
        return None, 0, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if count is not None and a.size != count:
            raise ValueError(f"expected {count} values, got {a.size}")
        return a.ctypes.data, 0, a
    # torch tensor
    if getattr(a, "is_cuda", False):
        import torch

        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float64 tensors")
        if count is not None and a.numel() != count:
            raise ValueError(f"expected {count} values, got {a.numel()}")
        return a.data_ptr(), 1, a
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return _arr(arr, count)


def _check(ctx, status: int):
    if status != TRTR_OK:
        msg = lib.trtr_last_error(ctx).decode() if ctx else ""
        raise TrtrError(status, f"{lib.trtr_status_str(status).decode()}: {msg}")


# --------------------------------------------------------------------------------------
# the C ABI, one function per entry point


def trtr_create(params: trtr_params, cuda_stream: int | None = None):
    out = _vp()
    s = lib.trtr_create(ctypes.byref(params), cuda_stream, ctypes.byref(out))
    if s != TRTR_OK:
        raise TrtrError(s, f"trtr_create: {lib.trtr_status_str(s).decode()}")
    return out


def trtr_destroy(ctx):
    _check(None, lib.trtr_destroy(ctx))


def trtr_set_fields(ctx, n: int, ux, uy, D=None, S=None):
    pu, du, ku = _arr(ux, n)
    pv, dv, kv = _arr(uy, n)
    pd, dd, kd = _arr(D, n)
    ps, ds, ks = _arr(S, n)
    devs = {d for p, d in ((pu, du), (pv, dv), (pd, dd), (ps, ds)) if p is not None}
    if len(devs) != 1:
        raise ValueError("fields must all be host arrays or all device tensors")
    _check(ctx, lib.trtr_set_fields(ctx, pu, pv, pd, ps, devs.pop()))


def trtr_set_source(ctx, n: int, S):
    p, d, k = _arr(S, n)
    _check(ctx, lib.trtr_set_source(ctx, p, d))


def trtr_set_source_prev(ctx, n: int, S):
    p, d, k = _arr(S, n)
    _check(ctx, lib.trtr_set_source_prev(ctx, p, d))


def trtr_set_dirichlet(ctx, n: int, phi_b):
    p, d, k = _arr(phi_b, n)
    _check(ctx, lib.trtr_set_dirichlet(ctx, p, d))


def trtr_set_pulse(ctx, omega, xc, yc, sigma0, D0, D_amp):
    _check(ctx, lib.trtr_set_pulse(ctx, omega, xc, yc, sigma0, D0, D_amp))


def trtr_init_equilibrium(ctx, n: int, phi0=None):
    p, d, k = _arr(phi0, n)
    _check(ctx, lib.trtr_init_equilibrium(ctx, p, d))


def trtr_step(ctx, n: int):
    _check(ctx, lib.trtr_step(ctx, int(n)))


def trtr_moments(ctx, out):
    p, d, k = _arr(out)
    if d == 0 and p is not None and k is not out:
        raise ValueError("host output must be a contiguous float64 numpy array")
    _check(ctx, lib.trtr_moments(ctx, p, d))
    return out


def trtr_mass(ctx) -> float:
    v = ctypes.c_double()
    _check(ctx, lib.trtr_mass(ctx, ctypes.byref(v)))
    return v.value


def trtr_error_vs_pulse(ctx):
    rms, rel = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib.trtr_error_vs_pulse(ctx, ctypes.byref(rms), ctypes.byref(rel)))
    return rms.value, rel.value


def trtr_error_vs(ctx, n: int, phi_ref):
    p, d, k = _arr(phi_ref, n)
    rms, rel = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib.trtr_error_vs(ctx, p, d, ctypes.byref(rms), ctypes.byref(rel)))
    return rms.value, rel.value


def trtr_get_populations(ctx, out):
    p, d, k = _arr(out)
    if d == 0 and k is not out:
        raise ValueError("host output must be a contiguous float64 numpy array")
    _check(ctx, lib.trtr_get_populations(ctx, p, d))
    return out


def trtr_set_populations(ctx, n9: int, g, step: int = 0):
    p, d, k = _arr(g, n9)
    _check(ctx, lib.trtr_set_populations(ctx, p, d, int(step)))


def trtr_sample_populations(ctx, nodes) -> np.ndarray:
    idx = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
    out = np.zeros((idx.size, 9))
    _check(ctx, lib.trtr_sample_populations(ctx, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), int(idx.size),
                                            out.ctypes.data_as(_dbl_p)))
    return out


def trtr_time(ctx):
    n, t = ctypes.c_long(), ctypes.c_double()
    _check(ctx, lib.trtr_time(ctx, ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def trtr_save(ctx) -> bytes:
    size = ctypes.c_size_t()
    _check(ctx, lib.trtr_save(ctx, None, ctypes.byref(size)))
    buf = ctypes.create_string_buffer(size.value)
    _check(ctx, lib.trtr_save(ctx, buf, ctypes.byref(size)))
    return buf.raw[: size.value]


def trtr_load(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(ctx, lib.trtr_load(ctx, buf, len(blob)))


def trtr_sync(ctx):
    _check(ctx, lib.trtr_sync(ctx))


def trtr_launch_count(ctx) -> int:
    v = ctypes.c_long()
    _check(ctx, lib.trtr_launch_count(ctx, ctypes.byref(v)))
    return v.value


def trtr_phi_sums_noalloc(g, nx: int, ny: int, phi_ref, out, cuda_stream: int | None = None) -> int:
    """FP64 sums of phi over caller-owned device populations with no device allocation:
    g (9*ny*nx float64 CUDA tensor), phi_ref (ny*nx float64 CUDA tensor or None), out (3
    float64 CUDA tensor), each contiguous.

    Arguments the kernels could not read safely (not a CUDA tensor, not float64, not
    contiguous, or too few values) raise ValueError before anything reaches the library.
    Otherwise the library's status code is returned as it is (TRTR_EINVAL for sizes beyond the
    static scratch, TRTR_ECUDA for a failed launch), with no exception."""
    import torch

    def _ok(name, t, count):
        if not getattr(t, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 tensor (got {t.dtype})")
        if t.numel() < count:
            raise ValueError(f"{name} holds {t.numel()} values, needs {count}")

    _ok("g", g, 9 * max(nx, 0) * max(ny, 0))
    _ok("out", out, 3)
    if phi_ref is not None:
        _ok("phi_ref", phi_ref, max(nx, 0) * max(ny, 0))
    return int(lib.trtr_phi_sums_noalloc(g.data_ptr(), int(nx), int(ny),
                                         None if phi_ref is None else phi_ref.data_ptr(), out.data_ptr(), cuda_stream))


def trtr_forward_record(ctx, steps: int, interval: int = 0):
    _check(ctx, lib.trtr_forward_record(ctx, int(steps), int(interval)))


def trtr_adjoint(ctx, n: int, dJ_dphi, grad_out):
    pd, dd, kd = _arr(dJ_dphi, n)
    pg, dg, kg = _arr(grad_out, n)
    if dg == 0 and kg is not grad_out:
        raise ValueError("host output must be a contiguous float64 numpy array")
    _check(ctx, lib.trtr_adjoint(ctx, pd, dd, pg, dg))
    return grad_out


def trtr_status_str(s: int) -> str:
    return lib.trtr_status_str(s).decode()


def trtr_last_error(ctx) -> str:
    return lib.trtr_last_error(ctx).decode()


def trtr_d2q9():
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    lib.trtr_d2q9(ex, ey, w)
    return np.array(ex[:]), np.array(ey[:]), np.array(w[:])


def trtr_check_timeout_path(ctx, cycles: int) -> int:
    """Status of the failure-detection check (TRTR_ETIMEOUT when the timeout path works)."""
    return int(lib.trtr_check_timeout_path(ctx, int(cycles)))


def trtr_abi_version() -> int:
    return int(lib.trtr_abi_version())


def trtr_set_steps_per_launch(ctx, k: int):
    _check(ctx, lib.trtr_set_steps_per_launch(ctx, int(k)))


def trtr_get_steps_per_launch(ctx) -> int:
    k = ctypes.c_int()
    _check(ctx, lib.trtr_get_steps_per_launch(ctx, ctypes.byref(k)))
    return int(k.value)


def trtr_check_bounds_path(ctx) -> int:
    """Status of the bounds-check probe (TRTR_EBOUNDS in the checked build, TRTR_OK otherwise)."""
    return int(lib.trtr_check_bounds_path(ctx))


def trtr_bounds_checked() -> bool:
    return bool(lib.trtr_bounds_checked())


def trtr_bounds_report() -> tuple[int, int, int, int]:
    """(accesses caught, kind of the first, its column or x, its row or y) since the last report;
    the record is cleared.  Zeros in the default build."""
    out = (ctypes.c_ulonglong * 3)()
    _check(None, lib.trtr_bounds_report(out))
    where = int(out[2])
    i, j = where & 0xFFFFFFFF, where >> 32
    signed = lambda v: v - (1 << 32) if v >= 1 << 31 else v  # noqa: E731
    return int(out[0]), int(out[1]), signed(i), signed(j)


# --------------------------------------------------------------------------------------
# convenience object over the same calls


@dataclass
class Params:
    nx: int
    ny: int
    dx: float
    dt: float
    x0: float = -1.0
    y0: float = -1.0
    precision: int = TRTR_F32
    phi_ref: float = 0.0
    tau2_mode: int = TRTR_TAU2_MAGIC
    magic: float = 1.0 / 12.0
    tau2: float = 1.0
    tau1_const: float = 0.0
    grad_mode: int = TRTR_GRAD_ONESIDED_EDGE
    src_mode: int = TRTR_SRC_NONE
    check_every: int = 0
    bc_mode: int = TRTR_BC_PERIODIC
    rounding: int = TRTR_ROUND_STOCHASTIC  # 2-byte storages only

    def to_c(self) -> trtr_params:
        return trtr_params(**{f.name: getattr(self, f.name) for f in dc_fields(self)})


class Solver:
    """Owns one trtr context; methods map 1:1 onto the C calls."""

    def __init__(self, params: Params, stream: int | None = None):
        self.params = params
        self.n = params.nx * params.ny
        self.ctx = trtr_create(params.to_c(), stream)

    def close(self):
        if self.ctx:
            trtr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, ux, uy, D=None, S=None):
        trtr_set_fields(self.ctx, self.n, ux, uy, D, S)

    def set_source(self, S):
        trtr_set_source(self.ctx, self.n, S)

    def set_source_prev(self, S):
        trtr_set_source_prev(self.ctx, self.n, S)

    def set_dirichlet(self, phi_b):
        trtr_set_dirichlet(self.ctx, self.n, phi_b)

    def set_pulse(self, omega, xc, yc, sigma0, D0, D_amp=0.0):
        trtr_set_pulse(self.ctx, omega, xc, yc, sigma0, D0, D_amp)

    def init_equilibrium(self, phi0=None):
        trtr_init_equilibrium(self.ctx, self.n, phi0)

    def step(self, n: int = 1):
        trtr_step(self.ctx, n)

    def set_steps_per_launch(self, k: int):
        trtr_set_steps_per_launch(self.ctx, k)

    @property
    def steps_per_launch(self) -> int:
        return trtr_get_steps_per_launch(self.ctx)

    def moments(self, out=None):
        if out is None:
            out = np.zeros((self.params.ny, self.params.nx))
        return trtr_moments(self.ctx, out)

    def mass(self) -> float:
        return trtr_mass(self.ctx)

    def error_vs_pulse(self):
        return trtr_error_vs_pulse(self.ctx)

    def error_vs(self, phi_ref):
        return trtr_error_vs(self.ctx, self.n, phi_ref)

    def get_populations(self, out=None):
        if out is None:
            out = np.zeros((9, self.params.ny, self.params.nx))
        return trtr_get_populations(self.ctx, out)

    def set_populations(self, g, step: int = 0):
        trtr_set_populations(self.ctx, 9 * self.n, g, step)

    def sample(self, nodes):
        return trtr_sample_populations(self.ctx, nodes)

    def time(self):
        return trtr_time(self.ctx)

    def save(self) -> bytes:
        return trtr_save(self.ctx)

    def load(self, blob: bytes):
        trtr_load(self.ctx, blob)

    def sync(self):
        trtr_sync(self.ctx)

    def forward_record(self, steps: int, interval: int = 0):
        trtr_forward_record(self.ctx, steps, interval)

    def adjoint(self, dJ_dphi, out=None):
        if out is None:
            out = np.zeros((self.params.ny, self.params.nx))
        return trtr_adjoint(self.ctx, self.n, dJ_dphi, out)

    @property
    def launches(self) -> int:
        return trtr_launch_count(self.ctx)


def pulse_solver(pulse, precision: int = TRTR_F32, stream: int | None = None, src_mode: int | None = None,
                 **overrides) -> Solver:
    """A Solver set up for a ``workloads.Pulse`` (fields from the closed form, on the device)."""
    if src_mode is None:
        src_mode = TRTR_SRC_PULSE if pulse.D_amp != 0.0 else TRTR_SRC_NONE
    if pulse.tau2 is not None:
        overrides.setdefault("tau2_mode", TRTR_TAU2_FIXED)
        overrides.setdefault("tau2", pulse.tau2)
    p = Params(nx=pulse.nx, ny=pulse.ny, dx=pulse.dx, dt=pulse.dt, x0=pulse.x0, y0=pulse.y0,
               precision=precision, src_mode=src_mode, grad_mode=TRTR_GRAD_ONESIDED_EDGE, **overrides)
    s = Solver(p, stream)
    s.set_pulse(pulse.omega, pulse.xc, pulse.yc, pulse.sigma0, pulse.D0, pulse.D_amp)
    s.init_equilibrium(None)
    return s


# --------------------------------------------------------------------------------------
# batched instances


def _bcheck(status: int, what: str):
    if status != TRTR_OK:
        raise TrtrError(status, f"{what}: {lib.trtr_status_str(status).decode()}")


def trtr_batch_create(instances, cuda_stream: int | None = None):
    arr = (trtr_instance * len(instances))(*instances)
    out = _vp()
    _bcheck(lib.trtr_batch_create(arr, len(instances), cuda_stream, ctypes.byref(out)), "trtr_batch_create")
    return out


def trtr_batch_destroy(b):
    _bcheck(lib.trtr_batch_destroy(b), "trtr_batch_destroy")


def trtr_batch_config_count() -> int:
    return int(lib.trtr_batch_config_count())


def trtr_batch_config_name(c: int) -> str:
    return lib.trtr_batch_config_name(c).decode()


def trtr_batch_tune(b, trial_steps: int):
    n = trtr_batch_config_count()
    ms = (ctypes.c_float * n)()
    best = ctypes.c_int()
    _bcheck(lib.trtr_batch_tune(b, int(trial_steps), ctypes.byref(best), ms), "trtr_batch_tune")
    return best.value, list(ms)


def trtr_batch_set_config(b, config: int):
    _bcheck(lib.trtr_batch_set_config(b, int(config)), "trtr_batch_set_config")


def trtr_batch_step(b, n: int):
    _bcheck(lib.trtr_batch_step(b, int(n)), "trtr_batch_step")


def trtr_batch_set_steps_per_launch(b, k: int):
    _bcheck(lib.trtr_batch_set_steps_per_launch(b, int(k)), "trtr_batch_set_steps_per_launch")


def trtr_batch_get_steps_per_launch(b) -> int:
    k = ctypes.c_int()
    _bcheck(lib.trtr_batch_get_steps_per_launch(b, ctypes.byref(k)), "trtr_batch_get_steps_per_launch")
    return k.value


def trtr_batch_sync(b):
    _bcheck(lib.trtr_batch_sync(b), "trtr_batch_sync")


def trtr_batch_instance(b, k: int):
    out = _vp()
    _bcheck(lib.trtr_batch_instance(b, int(k), ctypes.byref(out)), "trtr_batch_instance")
    return out


def trtr_batch_info(b):
    c, nodes, step, cfg = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_long(), ctypes.c_int()
    _bcheck(lib.trtr_batch_info(b, ctypes.byref(c), ctypes.byref(nodes), ctypes.byref(step), ctypes.byref(cfg)),
            "trtr_batch_info")
    return {"count": c.value, "nodes": nodes.value, "step": step.value, "config": cfg.value}


def pulse_instance(pulse, precision: int = TRTR_F32, **overrides) -> trtr_instance:
    """A trtr_instance for a workloads.Pulse (source mode PULSE when D varies)."""
    src = TRTR_SRC_PULSE if pulse.D_amp != 0.0 else TRTR_SRC_NONE
    if pulse.tau2 is not None:
        overrides.setdefault("tau2_mode", TRTR_TAU2_FIXED)
        overrides.setdefault("tau2", pulse.tau2)
    p = Params(nx=pulse.nx, ny=pulse.ny, dx=pulse.dx, dt=pulse.dt, x0=pulse.x0, y0=pulse.y0, precision=precision,
               src_mode=src, grad_mode=TRTR_GRAD_ONESIDED_EDGE, **overrides)
    return trtr_instance(p.to_c(), pulse.omega, pulse.xc, pulse.yc, pulse.sigma0, pulse.D0, pulse.D_amp)


class InstanceView(Solver):
    """A Solver-like view of one instance of a batch (the batch owns the context)."""

    def __init__(self, batch: "Batch", k: int, params: Params):
        self.params = params
        self.n = params.nx * params.ny
        self.ctx = trtr_batch_instance(batch.b, k)
        self._batch = batch

    def close(self):
        self.ctx = None  # owned by the batch

    def step(self, n: int = 1):
        raise TrtrError(TRTR_ESTATE, "instances of a batch advance through Batch.step")


class Batch:
    """Owns a trtr_batch; methods map onto the C calls."""

    def __init__(self, instances, stream: int | None = None):
        self.instances = list(instances)
        self.b = trtr_batch_create(self.instances, stream)

    def close(self):
        if self.b:
            trtr_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, trial_steps: int = 10):
        return trtr_batch_tune(self.b, trial_steps)

    def set_config(self, c: int):
        trtr_batch_set_config(self.b, c)

    def set_steps_per_launch(self, k: int):
        trtr_batch_set_steps_per_launch(self.b, k)

    @property
    def steps_per_launch(self) -> int:
        return trtr_batch_get_steps_per_launch(self.b)

    def step(self, n: int = 1):
        trtr_batch_step(self.b, n)

    def sync(self):
        trtr_batch_sync(self.b)

    def info(self):
        return trtr_batch_info(self.b)

    def instance(self, k: int) -> InstanceView:
        ip = self.instances[k].p
        params = Params(**{name: getattr(ip, name) for name, _ in trtr_params._fields_})
        return InstanceView(self, k, params)
