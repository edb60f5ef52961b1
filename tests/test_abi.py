"""The C ABI library without a GPU: it loads, exports every function include/*.h declares,
and its host-only calls and argument validation behave as documented."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2312_10316_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\*?\s+\**(trtr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def T():
    build.build_library()
    from paper_2312_10316_gb300 import trtr

    return trtr


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["trtr_create", "trtr_destroy", "trtr_set_fields", "trtr_set_source", "trtr_set_pulse",
                     "trtr_init_equilibrium", "trtr_step", "trtr_moments", "trtr_mass", "trtr_error_vs_pulse",
                     "trtr_error_vs", "trtr_time", "trtr_save", "trtr_load"]:
        assert required in names


def test_library_exports_every_declared_symbol(T):
    lib = ctypes.CDLL(T.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", T.LIB_PATH], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\s[TW]\s+(trtr_\w+)$", out.stdout, flags=re.M))
        assert set(declared_functions()) <= exported


def test_binding_covers_the_header(T):
    assert set(T.symbols()) == set(declared_functions())


def test_host_only_calls(T):
    assert T.trtr_abi_version() == 3
    # zero-initialised parameters round the 2-byte storages stochastically
    assert T.trtr_params().rounding == T.TRTR_ROUND_STOCHASTIC == 0 and T.Params(1, 1, 1.0, 1.0).rounding == 0
    ex, ey, w = T.trtr_d2q9()
    assert np.isclose(w.sum(), 1.0)
    assert np.array_equal(ex + 0, [0, 1, -1, 0, 0, 1, -1, 1, -1])
    assert np.array_equal(ey + 0, [0, 0, 0, 1, -1, 1, -1, -1, 1])
    # opposite directions sit in adjacent slots (1,2), (3,4), (5,6), (7,8)
    for a in (1, 3, 5, 7):
        assert ex[a] == -ex[a + 1] and ey[a] == -ey[a + 1]
    assert T.trtr_status_str(T.TRTR_EUNSTABLE).startswith("non-finite")
    assert "bounds" in T.trtr_status_str(T.TRTR_EBOUNDS)
    assert T.trtr_last_error(None) == "null context"
    assert T.trtr_bounds_checked() == T.BOUNDS_CHECKED


def test_bounds_checked_build_exports_the_same_boundary(T):
    """The debug build (TRTR_BOUNDS_CHECK=1) is a second library with the same entry points."""
    from paper_2312_10316_gb300.build import build_library

    path = build_library(checked=True)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.trtr_bounds_checked.restype = ctypes.c_int
    assert lib.trtr_bounds_checked() == 1
    assert lib.trtr_bounds_report(None) == T.TRTR_EINVAL
    assert lib.trtr_check_bounds_path(None) == T.TRTR_EINVAL
    assert lib.trtr_set_steps_per_launch(None, 2) == T.TRTR_EINVAL
    assert lib.trtr_get_steps_per_launch(None, None) == T.TRTR_EINVAL


def test_library_and_oracle_share_the_lattice_convention(T):
    import oracle

    oex, oey, ow = oracle.d2q9()
    ex, ey, w = T.trtr_d2q9()
    assert np.array_equal(oex, ex) and np.array_equal(oey, ey) and np.array_equal(ow, w)


BAD = [
    dict(nx=0), dict(ny=-3), dict(dx=0.0), dict(dt=-1.0), dict(dx=float("nan")), dict(precision=7),
    dict(tau2_mode=2), dict(magic=0.0), dict(tau2_mode=1, tau2=0.5), dict(tau1_const=0.4),
    dict(grad_mode=5), dict(src_mode=3), dict(check_every=-1), dict(phi_ref=float("inf")),
    dict(nx=70000, ny=40000), dict(bc_mode=2), dict(bc_mode=1, nx=2), dict(bc_mode=1, ny=1),
    dict(rounding=2), dict(rounding=-1),
]


@pytest.mark.parametrize("bad", BAD, ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_create_rejects_bad_parameters_before_touching_cuda(T, bad):
    base = dict(nx=16, ny=16, dx=0.1, dt=0.01)
    base.update(bad)
    p = T.Params(**base)
    with pytest.raises(T.TrtrError) as e:
        T.trtr_create(p.to_c(), None)
    assert e.value.status == T.TRTR_EINVAL


def test_null_arguments(T):
    lib = T.lib
    assert lib.trtr_create(None, None, None) == T.TRTR_EINVAL
    assert lib.trtr_destroy(None) == T.TRTR_OK
    assert lib.trtr_step(None, 1) == T.TRTR_EINVAL
    assert lib.trtr_sync(None) == T.TRTR_EINVAL
    assert lib.trtr_set_dirichlet(None, None, 0) == T.TRTR_EINVAL
    assert lib.trtr_set_source_prev(None, None, 0) == T.TRTR_EINVAL
    assert lib.trtr_check_timeout_path(None, 1000) == T.TRTR_EINVAL
    assert lib.trtr_bounds_report(None) == T.TRTR_EINVAL
    assert lib.trtr_batch_set_steps_per_launch(None, 2) == T.TRTR_EINVAL
    assert lib.trtr_batch_get_steps_per_launch(None, None) == T.TRTR_EINVAL
    assert lib.trtr_get_steps_per_launch(None, None) == T.TRTR_EINVAL


def test_batch_rejects_bad_instances_before_touching_cuda(T):
    from paper_2312_10316_gb300 import workloads as W

    a = T.pulse_instance(W.Pulse(n=32), T.TRTR_F32)
    b = T.pulse_instance(W.Pulse(n=40), T.TRTR_F16_OFS)
    c = T.pulse_instance(W.Pulse(n=32), T.TRTR_F32)
    c.p.bc_mode = T.TRTR_BC_DIRICHLET_NEE
    d = T.pulse_instance(W.Pulse(n=40), T.TRTR_F16_OFS)
    e = T.pulse_instance(W.Pulse(n=40), T.TRTR_F16_OFS, rounding=T.TRTR_ROUND_NEAREST)
    f = T.pulse_instance(W.Pulse(n=40), T.TRTR_F16_OFS, rounding=5)
    for bad in ([a, b], [T.pulse_instance(W.Pulse(n=32), T.TRTR_F64)], [], [a, c], [d, e], [f]):
        with pytest.raises(T.TrtrError) as e:
            T.trtr_batch_create(bad)
        assert e.value.status == T.TRTR_EINVAL
    assert T.trtr_batch_config_count() == 20
    assert "128x8" in T.trtr_batch_config_name(0) and T.trtr_batch_config_name(99) == "invalid"


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor on a machine without a GPU: the binding's checks read only
    these attributes; reaching the library (data_ptr) fails the test."""

    is_cuda = True

    def __init__(self, dtype, n, contiguous=True):
        self.dtype, self._n, self._c = dtype, n, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def data_ptr(self):
        raise AssertionError("an unchecked argument reached the library")


def test_noalloc_binding_rejects_what_its_kernels_cannot_read(T):
    torch = pytest.importorskip("torch")
    nx, ny = 8, 4
    good_g = _FakeDeviceTensor(torch.float64, 9 * nx * ny)
    good_out = _FakeDeviceTensor(torch.float64, 3)
    cases = [
        (_FakeDeviceTensor(torch.float32, 9 * nx * ny), good_out, None),   # float32 populations
        (good_g, _FakeDeviceTensor(torch.float32, 3), None),               # float32 out
        (good_g, good_out, _FakeDeviceTensor(torch.float32, nx * ny)),     # float32 reference
        (_FakeDeviceTensor(torch.float64, 9 * nx * ny, contiguous=False), good_out, None),
        (_FakeDeviceTensor(torch.float64, 9 * nx * ny - 1), good_out, None),  # too short
        (np.zeros(9 * nx * ny), good_out, None),                           # host array
    ]
    for g, out, ref in cases:
        with pytest.raises(ValueError):
            T.trtr_phi_sums_noalloc(g, nx, ny, ref, out)
