"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative L2 against the oracle): FP64 storage <= 1e-12, FP32 <= 1e-5; the
half-precision offset storage is bounded by its rounding unit (see each test)."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_10316_gb300 import workloads as W

from ._gpu_util import TOL_F32, TOL_F64, assert_elementwise, oracle_for_pulse, random_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402  (loads libtrtr.so)

PREC = {"f64": T.TRTR_F64, "f32": T.TRTR_F32, "f16": T.TRTR_F16_OFS, "bf16": T.TRTR_BF16_OFS}
ONE_STEP_TOL = {"f64": TOL_F64, "f32": TOL_F32, "f16": 2e-3, "bf16": 1.5e-2}


# ------------------------------------------------------------------------ workload 1


def test_pulse64_f64_against_oracle():
    """64^2 rotating pulse, FP64, constant D, S = 0, Courant 0.2, 500 steps."""
    pulse = W.C1_F64_64
    o = oracle_for_pulse(pulse)
    with T.pulse_solver(pulse, precision=T.TRTR_F64) as s:
        m0 = s.mass()
        assert abs(m0 - o.mass()) <= 1e-13 * abs(m0)
        s.step(pulse.steps)
        o.step(pulse.steps)
        phi = s.moments()
        assert rel_l2(phi, o.phi()) <= TOL_F64
        assert rel_l2(s.get_populations(), o.get_g()) <= TOL_F64
        # reductions
        assert abs(s.mass() - o.mass()) <= 1e-13 * abs(m0)
        assert abs(s.mass() - m0) <= 1e-13 * abs(m0)  # conservation with S = 0
        pa = W.phi_analytic(pulse, pulse.steps * pulse.dt)
        rms_o, rel_o = o.error(pa)
        rms_g, rel_g = s.error_vs_pulse()
        assert abs(rms_g - rms_o) <= 1e-10 * rms_o and abs(rel_g - rel_o) <= 1e-10 * rel_o
        rms_f, rel_f = s.error_vs(pa)
        assert abs(rms_f - rms_o) <= 1e-10 * rms_o and abs(rel_f - rel_o) <= 1e-10 * rel_o
        n, t = s.time()
        assert n == pulse.steps and abs(t - pulse.steps * pulse.dt) < 1e-15


# ------------------------------------------------------------- random states, all modes

GRIDS = [(1, 1), (1, 5), (7, 1), (2, 3), (5, 3), (33, 17), (37, 23), (64, 64), (100, 67), (129, 40)]


def _pair(case, nx, ny, prec, src_mode, grad_mode, tau2_mode, tau1_const=0.0, phi_ref=0.0, pulse=None):
    common = dict(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], x0=-0.3, y0=-0.2, tau2_mode=tau2_mode, magic=1 / 12,
                  tau2=1.2, tau1_const=tau1_const, grad_mode=grad_mode, src_mode=src_mode)
    pul = dict(omega=0.0, xc=0.0, yc=0.0, sigma0=0.1, D0=0.0, D_amp=0.0)
    if pulse is not None:
        pul = dict(omega=pulse[0], xc=pulse[1], yc=pulse[2], sigma0=pulse[3], D0=pulse[4], D_amp=pulse[5])
    o = oracle.Sim(oracle.SimParams(**common, **pul))
    s = T.Solver(T.Params(precision=prec, phi_ref=phi_ref, **common))
    return o, s


@pytest.mark.parametrize("nx,ny", GRIDS)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("src_mode", [0, 1, 2])
def test_random_state_steps(nx, ny, prec, src_mode):
    case = random_case(100 + nx * 131 + ny, nx, ny)
    grad_mode = (nx + ny) % 2
    tau2_mode = (nx * ny) % 2
    pulse = (0.0, -0.1, 0.05, 0.2, 5e-3, 0.5) if src_mode == 2 else None
    o, s = _pair(case, nx, ny, PREC[prec], src_mode, grad_mode, tau2_mode, pulse=pulse)
    with s:
        S1 = case["S1"] if src_mode == 1 else None
        o.set_fields(case["ux"], case["uy"], case["D"])
        s.set_fields(case["ux"], case["uy"], case["D"], S1)
        if src_mode == 1:
            o.set_source(S1)
        if src_mode == 2:
            s.set_pulse(*pulse)
            s.set_fields(case["ux"], case["uy"], case["D"])  # random u / D over the pulse's fields
        o.set_g(case["g"], step=5)
        s.set_populations(case["g"], step=5)
        assert rel_l2(s.get_populations(), case["g"]) <= (TOL_F64 if prec == "f64" else 1e-7)
        for k in range(3):
            o.step(1)
            s.step(1)
            gp, og = s.get_populations(), o.get_g()
            assert rel_l2(gp, og) <= ONE_STEP_TOL[prec], (k, prec)
            assert_elementwise(gp, og, ONE_STEP_TOL[prec], f"step {k} {prec}", tile=(64, 8))
            if src_mode == 1:
                Sn = case["S2"] if k % 2 == 0 else case["S1"]
                o.set_source(Sn)
                s.set_source(Sn)
        assert rel_l2(s.moments(), o.phi()) <= ONE_STEP_TOL[prec]
        assert_elementwise(s.moments(), o.phi(), ONE_STEP_TOL[prec], "phi", tile=(64, 8))
        assert abs(s.mass() - o.mass()) <= 10 * ONE_STEP_TOL[prec] * abs(o.mass())


@pytest.mark.parametrize("prec,src_mode", [("f64", 0), ("f64", 1), ("f64", 2), ("f32", 0), ("f32", 1), ("f32", 2),
                                           ("f16", 0), ("f16", 2), ("bf16", 2)])
def test_large_geometry_ragged_grid(prec, src_mode):
    """1101 x 700 nodes: enough tiles for the large-grid step geometry (128 x 16 tiles, or 128 x 8
    for FP64 and the FP32 source fields; at least two per SM on a 152-SM GPU; FP32 without a
    source keeps the small-grid tiles up to about 4096^2, see the sampled 8192^2 check), with a ragged last
    tile column (77 nodes: the FP32 pulse path's bulk row copies leave its last column, the
    2-byte storages' its last five, to the lanes) and a ragged last tile row.  Two steps from
    random populations against the oracle; the 2-byte storages use phi_ref = 1."""
    nx, ny = 1101, 700
    case = random_case(900 + src_mode, nx, ny)
    pulse = (0.0, -0.1, 0.05, 0.2, 5e-3, 0.5) if src_mode == 2 else None
    phi_ref = 1.0 if prec in ("f16", "bf16") else 0.0
    o, s = _pair(case, nx, ny, PREC[prec], src_mode, 1, 0, phi_ref=phi_ref, pulse=pulse)
    with s:
        S1 = case["S1"] if src_mode == 1 else None
        o.set_fields(case["ux"], case["uy"], case["D"])
        s.set_fields(case["ux"], case["uy"], case["D"], S1)
        if src_mode == 1:
            o.set_source(S1)
        if src_mode == 2:
            s.set_pulse(*pulse)
            s.set_fields(case["ux"], case["uy"], case["D"])
        o.set_g(case["g"], step=5)
        s.set_populations(case["g"], step=5)
        tile = (128, 8) if prec == "f64" or src_mode == 1 else (128, 16)
        for k in range(2):
            o.step(1)
            s.step(1)
            gp, og = s.get_populations(), o.get_g()
            assert rel_l2(gp, og) <= ONE_STEP_TOL[prec], (k, prec)
            assert_elementwise(gp, og, ONE_STEP_TOL[prec], f"step {k} {prec}", tile=tile)
            if src_mode == 1:
                o.set_source(case["S2"])
                s.set_source(case["S2"])
        assert rel_l2(s.moments(), o.phi()) <= ONE_STEP_TOL[prec]
        assert_elementwise(s.moments(), o.phi(), ONE_STEP_TOL[prec], "phi", tile=tile)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tau1_const_and_fixed_tau2(prec):
    nx, ny = 45, 38
    case = random_case(7, nx, ny)
    o, s = _pair(case, nx, ny, PREC[prec], 0, 0, 1, tau1_const=0.9)
    with s:
        o.set_fields(case["ux"], case["uy"], case["D"])
        s.set_fields(case["ux"], case["uy"], None)
        o.set_g(case["g"])
        s.set_populations(case["g"])
        o.step(4)
        s.step(4)
        assert rel_l2(s.get_populations(), o.get_g()) <= ONE_STEP_TOL[prec]
        assert_elementwise(s.get_populations(), o.get_g(), ONE_STEP_TOL[prec], prec, tile=(64, 8))


@pytest.mark.parametrize("prec,phi_ref", [("f16", 1.0), ("bf16", 1.0), ("f16", 0.0), ("bf16", 0.0)])
def test_half_offset_storage_one_step(prec, phi_ref):
    """Populations stored as half-precision offsets g - w_i phi_ref, FP32 arithmetic: one
    step stays within a few rounding units of the format (2^-11 f16, 2^-8 bf16)."""
    nx, ny = 70, 41
    case = random_case(11, nx, ny)
    o, s = _pair(case, nx, ny, PREC[prec], 0, 1, 0, phi_ref=phi_ref)
    with s:
        o.set_fields(case["ux"], case["uy"], case["D"])
        s.set_fields(case["ux"], case["uy"], case["D"])
        o.set_g(case["g"])
        s.set_populations(case["g"])
        o.step(1)
        s.step(1)
        err = rel_l2(s.get_populations(), o.get_g())
        unit = 2.0**-11 if prec == "f16" else 2.0**-8
        assert err <= 4 * unit, err
        assert_elementwise(s.get_populations(), o.get_g(), 4 * unit, prec, tile=(64, 8))


# ------------------------------------------------------------------- multi-step, FP32


def test_pulse200_f32_variable_D_multistep():
    """Workload-2 physics (variable D, manufactured source, Courant 0.8, the 1024^2 grid's
    relaxation times: D0 scaled so that tau1 - 1/2 = 0.2766) on a 200^2 grid (ragged against
    the 32 x 16 tiles), 1000 FP32 steps against the FP64 oracle."""
    base = W.Pulse(n=200, courant=0.8)
    D0 = 0.2766 / 3.0 * base.dx**2 / base.dt
    pulse = W.Pulse(n=200, D_amp=0.5, D0=D0, courant=0.8, steps=1000)
    o = oracle_for_pulse(pulse)
    with T.pulse_solver(pulse, precision=T.TRTR_F32) as s:
        s.step(pulse.steps)
        o.step(pulse.steps)
        phi_g, phi_o = s.moments(), o.phi()
        assert rel_l2(phi_g, phi_o) <= TOL_F32
        assert_elementwise(phi_g, phi_o, TOL_F32, "phi after 1000 steps", tile=(32, 16))
        rms_g, _ = s.error_vs_pulse()
        rms_o, _ = o.error(W.phi_analytic(pulse, pulse.steps * pulse.dt))
        # triangle inequality: the two RMS errors differ by at most the RMS of phi_g - phi_o
        assert abs(rms_g - rms_o) <= math.sqrt(np.mean((phi_g - phi_o) ** 2)) * (1 + 1e-9) + 1e-15


# ------------------------------------------------------- full sizes, sampled one step


def _sampled_step_check(pulse, prec, warm_steps, nsamples, tol, seed=0):
    """After `warm_steps` GPU steps, the populations the GPU writes in one more step at
    sampled nodes equal the oracle's single-node update of the GPU's own pre-collision
    state (rotation u: d_y u_x = -omega, d_x u_y = omega exactly on the lattice)."""
    rng = np.random.default_rng(seed)
    n = pulse.nx
    corners = [0, n - 1, (n - 1) * n, n * n - 1, n // 2, (n // 2) * n]
    nodes = np.unique(np.concatenate([rng.integers(0, n * n, size=nsamples), corners]))
    ex, ey, _ = T.trtr_d2q9()
    op = oracle.SimParams(nx=n, ny=n, dx=pulse.dx, dt=pulse.dt, grad_mode=1, src_mode=2, omega=pulse.omega,
                          xc=pulse.xc, yc=pulse.yc, sigma0=pulse.sigma0, D0=pulse.D0, D_amp=pulse.D_amp,
                          tau2_mode=0 if pulse.tau2 is None else 1, tau2=pulse.tau2 or 1.0)
    osim = oracle.Sim(oracle.SimParams(nx=1, ny=1, dx=pulse.dx, dt=pulse.dt, src_mode=2, omega=pulse.omega,
                                       xc=pulse.xc, yc=pulse.yc, sigma0=pulse.sigma0, D0=pulse.D0,
                                       D_amp=pulse.D_amp))
    with T.pulse_solver(pulse, precision=prec) as s:
        s.step(warm_steps)
        g_n = s.sample(nodes)
        step_n, t_n = s.time()
        s.step(1)
        j, i = nodes // n, nodes % n
        pushed = [((j + ey[q]) % n) * n + (i + ex[q]) % n for q in range(9)]
        after = [s.sample(pushed[q])[:, q] for q in range(9)]
    gpu = np.stack(after, axis=1)
    ref = np.zeros_like(gpu)
    du = [0.0, -pulse.omega, pulse.omega, 0.0]
    for k, node in enumerate(nodes):
        x = pulse.x0 + (node % n) * pulse.dx
        y = pulse.y0 + (node // n) * pulse.dx
        D = pulse.D0 * (1 + pulse.D_amp * math.sin(math.pi * x) * math.sin(math.pi * y))
        Sn = osim.pulse_source_at(x, y, t_n)
        Sp = osim.pulse_source_at(x, y, t_n - pulse.dt)  # the closed form at t_n - dt (first step too)
        ref[k] = oracle.node_post(op, g_n[k], -pulse.omega * y, pulse.omega * x, du, D, Sn, Sp)
    err = rel_l2(gpu, ref)
    assert err <= tol, err
    return err


@pytest.mark.parametrize("pulse", [W.C2A_F32_1024, W.C2B_F32_4096], ids=lambda p: p.name)
def test_fullsize_sampled_f32(pulse):
    _sampled_step_check(pulse, T.TRTR_F32, 100, 4000, 2e-6)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_fullsize_sampled_half_8192(prec):
    """The 8192^2 half-precision storage workload in the bench's launch configuration: one step at
    sampled nodes against the oracle's single-node update of the GPU's own (decoded) state; the
    results are rounded to the storage format, so the one-step tolerance of that format."""
    _sampled_step_check(W.C3_HALF_8192, PREC[prec], 20, 2000, ONE_STEP_TOL[prec])


def test_fullsize_sampled_f32_no_source_8192():
    """FP32 without a source takes the large-grid tile geometry only on the largest grids
    (the small tiles measured faster up to 4096^2): 8192^2, constant D, S = 0."""
    _sampled_step_check(W.Pulse(n=8192, courant=0.8, tau2=0.8), T.TRTR_F32, 20, 2000, 2e-6)


def test_fullsize_sampled_f64_8192():
    _sampled_step_check(W.C3_HALF_8192, T.TRTR_F64, 20, 2000, 1e-13)


def test_mass_conserved_f32_1024():
    """S = 0: FP64 sum of phi is conserved up to FP32 rounding of the stored populations."""
    pulse = W.Pulse(n=1024, courant=0.8)
    with T.pulse_solver(pulse, precision=T.TRTR_F32) as s:
        m0 = s.mass()
        s.step(500)
        assert abs(s.mass() - m0) <= 1e-5 * abs(m0)


# ------------------------------------------------------------------- host-side paths


def test_device_tensors_and_stream_match_host_path():
    pulse = W.Pulse(n=96, D_amp=0.5, courant=0.8)
    f = W.fields(pulse)
    stream = torch.cuda.Stream()
    dev = {k: torch.from_numpy(v).cuda() for k, v in f.items()}
    p = T.Params(nx=96, ny=96, dx=pulse.dx, dt=pulse.dt, precision=T.TRTR_F32, src_mode=T.TRTR_SRC_PULSE)
    with T.Solver(p, stream.cuda_stream) as a, T.Solver(p) as b:
        a.set_pulse(pulse.omega, pulse.xc, pulse.yc, pulse.sigma0, pulse.D0, pulse.D_amp)
        b.set_pulse(pulse.omega, pulse.xc, pulse.yc, pulse.sigma0, pulse.D0, pulse.D_amp)
        a.set_fields(dev["ux"], dev["uy"], dev["D"])
        b.set_fields(f["ux"], f["uy"], f["D"])
        a.init_equilibrium(dev["phi0"])
        b.init_equilibrium(f["phi0"])
        a.step(37)
        b.step(37)
        out = torch.empty((96, 96), dtype=torch.float64, device="cuda")
        a.moments(out)
        stream.synchronize()
        assert np.array_equal(out.cpu().numpy(), b.moments())


def test_save_load_roundtrip_is_bitwise():
    pulse = W.Pulse(n=80, D_amp=0.5, courant=0.8)
    with T.pulse_solver(pulse, precision=T.TRTR_F32) as s:
        s.step(10)
        blob = s.save()
        s.step(25)
        ref = s.get_populations().copy()
        s.load(blob)
        assert s.time()[0] == 10
        s.step(25)
        assert np.array_equal(s.get_populations(), ref)


def test_field_source_save_load():
    nx, ny = 40, 24
    case = random_case(3, nx, ny)
    p = T.Params(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], precision=T.TRTR_F64, src_mode=T.TRTR_SRC_FIELD)
    with T.Solver(p) as s:
        s.set_fields(case["ux"], case["uy"], case["D"], case["S1"])
        s.set_populations(case["g"])
        s.step(2)
        s.set_source(case["S2"])
        blob = s.save()
        s.step(3)
        ref = s.get_populations().copy()
        s.load(blob)
        s.step(3)
        assert np.array_equal(s.get_populations(), ref)


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection without a fault: a kernel waits on a barrier that nothing completes,
    gives up after about half a millisecond through the step kernels' bounded-wait path, and
    the host reads TRTR_ETIMEOUT; the flag is cleared as it is reported, and the context then
    steps exactly as a fresh one does."""
    nx, ny = 40, 24
    case = random_case(3, nx, ny)
    p = T.Params(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], precision=T.TRTR_F64)
    results = []
    for check in (True, False):
        with T.Solver(p) as s:
            s.set_fields(case["ux"], case["uy"], case["D"])
            s.set_populations(case["g"])
            if check:
                assert T.trtr_check_timeout_path(s.ctx, 1_000_000) == T.TRTR_ETIMEOUT
                assert "timed out" in T.trtr_last_error(s.ctx)
                assert T.trtr_check_timeout_path(s.ctx, 0) == T.TRTR_EINVAL
                s.sync()  # reported once: nothing pending any more
            s.step(3)
            s.sync()
            results.append(s.get_populations())
    assert np.array_equal(results[0], results[1])


def test_unstable_run_is_reported():
    """Host-side fault injection: a NaN population is detected by the periodic check."""
    nx, ny = 32, 32
    case = random_case(5, nx, ny)
    g = case["g"].copy()
    g[3, 7, 11] = np.nan
    p = T.Params(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], precision=T.TRTR_F32, check_every=2)
    with T.Solver(p) as s:
        s.set_fields(case["ux"], case["uy"], case["D"])
        s.set_populations(g)
        with pytest.raises(T.TrtrError) as e:
            s.step(4)
        assert e.value.status == T.TRTR_EUNSTABLE


def test_call_order_and_argument_errors():
    p = T.Params(nx=16, ny=16, dx=0.1, dt=0.02, precision=T.TRTR_F32)
    with T.Solver(p) as s:
        with pytest.raises(T.TrtrError) as e:
            s.step(1)
        assert e.value.status == T.TRTR_ESTATE
        case = random_case(1, 16, 16)
        s.set_fields(case["ux"], case["uy"], case["D"])
        s.set_populations(case["g"])
        before = s.get_populations().copy()
        s.step(0)
        assert np.array_equal(s.get_populations(), before)
        with pytest.raises(T.TrtrError) as e:
            s.sample([256])
        assert e.value.status == T.TRTR_EINVAL
        with pytest.raises(T.TrtrError) as e:
            s.step(-1)
        assert e.value.status == T.TRTR_EINVAL
        bad = case["D"].copy()
        bad[0, 0] = -1.0
        with pytest.raises(T.TrtrError) as e:
            s.set_fields(case["ux"], case["uy"], bad)
        assert e.value.status == T.TRTR_EINVAL
        # the same check on device-resident D (zero, negative, NaN, infinite), fields unchanged
        dux = torch.from_numpy(case["ux"]).cuda()
        duy = torch.from_numpy(case["uy"]).cuda()
        for v in (0.0, -1e-3, float("nan"), float("inf")):
            dbad = torch.from_numpy(case["D"]).cuda()
            dbad[5, 7] = v
            with pytest.raises(T.TrtrError) as e:
                s.set_fields(dux, duy, dbad)
            assert e.value.status == T.TRTR_EINVAL, v
        s.set_fields(dux, duy, torch.from_numpy(case["D"]).cuda())  # a valid device D passes
        s.step(1)
        with T.Solver(p) as ref:
            ref.set_fields(case["ux"], case["uy"], case["D"])
            ref.set_populations(before)
            ref.step(1)
            assert np.array_equal(s.get_populations(), ref.get_populations())


# ------------------------------------------------------ half-precision storage, many steps


def _half_tol(prec: str, steps: int) -> float:
    """Each step rounds every stored population to the half format (unit roundoff 2^-11 for
    FP16, 2^-8 for BF16, relative to |g - w phi_ref|).  Rounded stochastically (the default),
    the rounding errors are independent and zero-mean, so they accumulate no faster than
    sqrt(n) and the relative L2 error of phi after n steps stays below u * sqrt(n) (measured:
    it barely grows at all; test_gpu_rounding.py and test_gpu_accuracy.py)."""
    u = 2.0**-11 if prec == "f16" else 2.0**-8
    return u * math.sqrt(steps)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_half_offset_storage_multistep_against_oracle(prec):
    """200^2 pulse with the 1024^2 relaxation times, 1000 steps, phi_ref = 0."""
    base = W.Pulse(n=200, courant=0.8)
    D0 = 0.2766 / 3.0 * base.dx**2 / base.dt
    pulse = W.Pulse(n=200, D_amp=0.5, D0=D0, courant=0.8, steps=1000)
    o = oracle_for_pulse(pulse)
    with T.pulse_solver(pulse, precision=PREC[prec]) as s:
        s.step(pulse.steps)
        o.step(pulse.steps)
        err = rel_l2(s.moments(), o.phi())
    assert err <= _half_tol(prec, pulse.steps), err


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_precision_1024_against_oracle(prec):
    """The 1024^2 workload (variable D, manufactured source, Courant 0.8, magic tau2) for 300
    steps: each storage precision against the FP64 oracle at the same size."""
    pulse = W.C2A_F32_1024
    steps = 300
    o = oracle_for_pulse(pulse)
    with T.pulse_solver(pulse, precision=PREC[prec]) as s:
        s.step(steps)
        o.step(steps)
        err = rel_l2(s.moments(), o.phi())
    tol = TOL_F32 if prec == "f32" else _half_tol(prec, steps)
    assert err <= tol, err


@pytest.mark.parametrize("k", [1, 2, 5, 8, 10])  # an FP32 periodic context makes 10 allocations
def test_allocation_failure_is_reported_and_leaves_nothing(k, monkeypatch):
    """Host-side fault injection: TRTR_FAULT_ALLOC=k fails the k-th device allocation of
    trtr_create, which returns TRTR_ENOMEM after freeing what it had allocated; the next
    create succeeds and the free device memory is back where it was."""
    p = T.Params(nx=600, ny=500, dx=0.01, dt=1e-4, precision=T.TRTR_F32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("TRTR_FAULT_ALLOC", str(k))
    for _ in range(3):
        with pytest.raises(T.TrtrError) as e:
            T.Solver(p)
        assert e.value.status == T.TRTR_ENOMEM
    monkeypatch.delenv("TRTR_FAULT_ALLOC")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 8 * 2**20  # no allocation left behind (driver granularity aside)
    with T.Solver(p) as s:
        s.set_fields(np.zeros((500, 600)), np.zeros((500, 600)), np.full((500, 600), 1e-3))
        s.init_equilibrium(np.ones((500, 600)))
        s.step(2)
        assert np.abs(s.moments() - 1.0).max() <= 1e-6
