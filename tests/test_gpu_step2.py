"""The two-step kernel (two time steps of Eq. (14) per launch; FP32 storage, or FP16 / BF16
offset storage on grids of even nx; periodic boundaries, no source or the pulse source).

Its node update is the one-step kernel's, and the 2-byte storages round the intermediate state
exactly as a one-step launch stores it (the same stochastic-rounding bits), so the populations
after any number of steps must equal those of one launch per step bit for bit; the one-step path
is checked against the FP64 oracle elsewhere, and cases here check the two-step path against the
oracle directly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2312_10316_gb300 import workloads as W

from ._gpu_util import TOL_F32, assert_elementwise, oracle_for_pulse, random_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402

GRIDS = [(2, 3), (3, 5), (5, 3), (37, 23), (130, 9), (128, 8), (257, 19), (300, 130)]


def _random_solver(nx, ny, grad_mode, k, precision=T.TRTR_F32, **kw):
    case = random_case(900 + 13 * nx + ny, nx, ny)
    p = T.Params(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], precision=precision, grad_mode=grad_mode,
                 src_mode=T.TRTR_SRC_NONE, **kw)
    s = T.Solver(p)
    s.set_steps_per_launch(k)
    s.set_fields(case["ux"], case["uy"], case["D"])
    s.set_populations(case["g"], step=0)
    return s


def _pulse_solver(nx, ny, grad_mode, k, D_amp=0.5, precision=T.TRTR_F32, **kw):
    pulse = W.Pulse(n=max(nx, ny), D_amp=D_amp, courant=0.4)
    p = T.Params(nx=nx, ny=ny, dx=pulse.dx, dt=pulse.dt, x0=pulse.x0, y0=pulse.y0, precision=precision,
                 grad_mode=grad_mode, src_mode=T.TRTR_SRC_PULSE, **kw)
    s = T.Solver(p)
    s.set_steps_per_launch(k)
    s.set_pulse(pulse.omega, pulse.xc, pulse.yc, pulse.sigma0, pulse.D0, pulse.D_amp)
    s.init_equilibrium(None)
    return s


@pytest.mark.parametrize("nx,ny", GRIDS)
@pytest.mark.parametrize("grad_mode", [T.TRTR_GRAD_PERIODIC, T.TRTR_GRAD_ONESIDED_EDGE])
@pytest.mark.parametrize("kind", ["none", "pulse"])
def test_two_steps_per_launch_equal_one_step_launches_bitwise(nx, ny, grad_mode, kind):
    make = _random_solver if kind == "none" else _pulse_solver
    out = {}
    for k in (1, 2):
        with make(nx, ny, grad_mode, k) as s:
            s.step(5)  # two two-step launches and one single step
            s.step(3)  # the ghost frame's refresh after that single step, a pair, a single step
            out[k] = (s.get_populations(), s.launches)
    assert np.array_equal(out[1][0], out[2][0], equal_nan=True)
    if min(nx, ny) >= 8:
        assert np.isfinite(out[2][0]).all()


HALF = {"f16": T.TRTR_F16_OFS, "bf16": T.TRTR_BF16_OFS}
ROUND = {"sr": T.TRTR_ROUND_STOCHASTIC, "rn": T.TRTR_ROUND_NEAREST}
HALF_GRIDS = [(2, 3), (4, 5), (6, 2), (38, 23), (130, 9), (128, 8), (258, 19), (300, 130)]


@pytest.mark.parametrize("nx,ny", HALF_GRIDS)
@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("rounding", ["sr", "rn"])
@pytest.mark.parametrize("kind", ["none", "pulse"])
def test_two_byte_two_step_launches_equal_one_step_launches_bitwise(nx, ny, prec, rounding, kind):
    """The 2-byte storages: the same bits as one launch per step, for both roundings (the
    stochastic bits of the intermediate state, halo nodes included, are the one-step kernel's)
    and an offset phi_ref away from zero on the random states."""
    make = _random_solver if kind == "none" else _pulse_solver
    kw = dict(precision=HALF[prec], rounding=ROUND[rounding])
    if kind == "none":
        kw["phi_ref"] = 0.75
    out = {}
    for k in (1, 2):
        with make(nx, ny, T.TRTR_GRAD_ONESIDED_EDGE, k, **kw) as s:
            assert s.steps_per_launch == k
            s.step(5)
            s.step(3)
            out[k] = s.get_populations()
    assert np.array_equal(out[1], out[2], equal_nan=True)
    if min(nx, ny) >= 8:
        assert np.isfinite(out[2]).all()


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_two_byte_odd_nx_runs_one_step_per_launch(prec):
    with _random_solver(37, 12, T.TRTR_GRAD_PERIODIC, 2, precision=HALF[prec]) as s:
        assert s.steps_per_launch == 1
        l0 = s.launches
        s.step(4)
        assert s.launches - l0 == 4


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_two_byte_two_step_path_against_the_oracle(prec):
    """200^2 pulse, 8 steps (four two-step launches) against the FP64 oracle, per element."""
    pulse = W.Pulse(n=200, D_amp=0.5, courant=0.4)
    with T.pulse_solver(pulse, precision=HALF[prec]) as s:
        assert s.steps_per_launch == 2
        l0 = s.launches
        s.step(8)
        launches = s.launches - l0
        phi = s.moments()
    o = oracle_for_pulse(pulse)
    o.step(8)
    tol = {"f16": 1e-3, "bf16": 8e-3}[prec]
    assert rel_l2(phi, o.phi()) <= tol
    assert_elementwise(phi, o.phi(), 4 * tol, "phi", tile=(32, 8))
    assert launches == 1 + 4  # field packing, four two-step launches


@pytest.mark.parametrize("precision", [T.TRTR_F32, T.TRTR_F16_OFS])
def test_launch_counts_and_the_stability_check_cadence(precision):
    with _pulse_solver(64, 48, T.TRTR_GRAD_ONESIDED_EDGE, 2, precision=precision) as s:
        l0 = s.launches
        s.step(6)
        assert s.launches - l0 == 1 + 3  # field packing, then three two-step launches
        s.step(6)
        assert s.launches - l0 == 1 + 6
        s.step(1)
        s.step(2)
        assert s.launches - l0 == 1 + 6 + 1 + 2  # a single step, then ghost refresh + a pair
    # check_every = 3: the pair whose middle step is a check point runs as single steps
    ref = None
    for k in (1, 2):
        pulse = W.Pulse(n=64, D_amp=0.5, courant=0.4)
        p = T.Params(nx=64, ny=48, dx=pulse.dx, dt=pulse.dt, x0=pulse.x0, y0=pulse.y0, precision=precision,
                     grad_mode=T.TRTR_GRAD_ONESIDED_EDGE, src_mode=T.TRTR_SRC_PULSE, check_every=3)
        with T.Solver(p) as s:
            s.set_steps_per_launch(k)
            s.set_pulse(pulse.omega, pulse.xc, pulse.yc, pulse.sigma0, pulse.D0, pulse.D_amp)
            s.init_equilibrium(None)
            s.step(7)
            g = s.get_populations()
        ref = g if ref is None else ref
        assert np.array_equal(g, ref)


def test_new_fields_after_steps_are_repacked():
    nx, ny = 96, 40
    res = {}
    for k in (1, 2):
        with _random_solver(nx, ny, T.TRTR_GRAD_ONESIDED_EDGE, k) as s:
            s.step(4)
            case = random_case(77, nx, ny)
            s.set_fields(case["ux"], case["uy"], case["D"])
            s.step(4)
            res[k] = s.get_populations()
    assert np.array_equal(res[1], res[2])


def test_two_step_path_against_the_oracle():
    pulse = W.Pulse(n=200, D_amp=0.5, courant=0.4)
    with T.pulse_solver(pulse, precision=T.TRTR_F32) as s:
        assert s.params.src_mode == T.TRTR_SRC_PULSE
        l0 = s.launches
        s.step(8)
        launches = s.launches - l0
        phi = s.moments()
    o = oracle_for_pulse(pulse)
    o.step(8)
    assert rel_l2(phi, o.phi()) <= TOL_F32
    assert_elementwise(phi, o.phi(), TOL_F32, "phi", tile=(32, 8))
    assert launches == 1 + 4  # field packing, four two-step launches


def _sampled_two_step_check(pulse, warm, nsamples, tol, seed=1, precision=T.TRTR_F32):
    """Full-size check of one two-step launch in the bench's launch configuration: after `warm`
    steps (two per launch), the populations that one more launch writes at sampled nodes equal
    two applications of the oracle's single-node update (Eq. (14)) to the GPU's own state: the
    first to the pre-collision state of the 3 x 3 block around the node, the second to what the
    node then pulls from that block (rotation u: d_y u_x = -omega, d_x u_y = omega exactly on
    the lattice, the one-sided edge differences included)."""
    rng = np.random.default_rng(seed)
    n = pulse.nx
    ex, ey, _ = T.trtr_d2q9()
    edges = [0, 1, n - 2, n - 1]
    centres = [(int(j), int(i)) for j, i in rng.integers(0, n, size=(nsamples, 2))]
    centres += [(j, i) for j in edges for i in edges] + [(j, n // 2) for j in edges] + [(n // 2, i) for i in edges]
    centres = sorted(set(centres))
    block = [((j + dj) % n, (i + di) % n) for (j, i) in centres for dj in (-1, 0, 1) for di in (-1, 0, 1)]
    bnodes = np.array([j * n + i for j, i in block])
    op = oracle.SimParams(nx=n, ny=n, dx=pulse.dx, dt=pulse.dt, grad_mode=1, src_mode=2, omega=pulse.omega,
                          xc=pulse.xc, yc=pulse.yc, sigma0=pulse.sigma0, D0=pulse.D0, D_amp=pulse.D_amp,
                          tau2_mode=0 if pulse.tau2 is None else 1, tau2=pulse.tau2 or 1.0)
    osim = oracle.Sim(oracle.SimParams(nx=1, ny=1, dx=pulse.dx, dt=pulse.dt, src_mode=2, omega=pulse.omega,
                                       xc=pulse.xc, yc=pulse.yc, sigma0=pulse.sigma0, D0=pulse.D0,
                                       D_amp=pulse.D_amp))
    with T.pulse_solver(pulse, precision=precision) as s:
        assert s.steps_per_launch == 2 and warm % 2 == 0
        s.step(warm)
        g_n = s.sample(bnodes)
        step_n, t_n = s.time()
        l0 = s.launches
        s.step(2)
        assert s.launches - l0 == 1  # one launch of the two-step kernel
        after = np.stack([s.sample([((j + ey[q]) % n) * n + (i + ex[q]) % n for (j, i) in centres])[:, q]
                          for q in range(9)], axis=1)
    du = [0.0, -pulse.omega, pulse.omega, 0.0]

    def post(j, i, g, t):
        x, y = pulse.x0 + i * pulse.dx, pulse.y0 + j * pulse.dx
        D = pulse.D0 * (1 + pulse.D_amp * math.sin(math.pi * x) * math.sin(math.pi * y))
        Sn, Sp = osim.pulse_source_at(x, y, t), osim.pulse_source_at(x, y, t - pulse.dt)
        return oracle.node_post(op, g, -pulse.omega * y, pulse.omega * x, du, D, Sn, Sp)

    ref = np.zeros_like(after)
    for c, (j, i) in enumerate(centres):
        p1 = {block[9 * c + k]: post(*block[9 * c + k], g_n[9 * c + k], t_n) for k in range(9)}
        pre2 = np.array([p1[((j - ey[q]) % n, (i - ex[q]) % n)][q] for q in range(9)])
        ref[c] = post(j, i, pre2, t_n + pulse.dt)
    err = rel_l2(after, ref)
    assert err <= tol, err
    assert np.max(np.abs(after - ref)) <= tol * np.max(np.abs(ref))
    return err


@pytest.mark.parametrize("pulse", [W.C2A_F32_1024, W.C2B_F32_4096], ids=lambda p: p.name)
def test_fullsize_sampled_two_step_launch(pulse):
    _sampled_two_step_check(pulse, 100, 1500, 2e-6)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("pulse", [W.C2B_F32_4096, W.C3_HALF_8192], ids=lambda p: p.name)
def test_fullsize_sampled_two_byte_two_step_launch(pulse, prec):
    """The 2-byte storages at the bench's sizes: the GPU rounds the intermediate state and the
    result to the format (stochastically), the oracle does not, so the bound is a few units of
    the format (2^-11 FP16, 2^-8 BF16) of the largest population."""
    unit = {"f16": 2.0**-11, "bf16": 2.0**-8}[prec]
    _sampled_two_step_check(pulse, 100, 1500, 8 * unit, precision=HALF[prec])


@pytest.mark.parametrize("precision", [T.TRTR_F32, T.TRTR_F16_OFS, T.TRTR_BF16_OFS])
def test_save_load_and_recorded_runs_keep_the_two_step_path_exact(precision):
    nx, ny = 70, 33
    res = {}
    for k in (1, 2):
        with _pulse_solver(nx, ny, T.TRTR_GRAD_ONESIDED_EDGE, k, precision=precision) as s:
            s.step(3)
            blob = s.save()
            s.step(2)
            s.load(blob)  # back to step 3, saved after a single step
            s.step(4)
            res[k] = s.get_populations()
    assert np.array_equal(res[1], res[2])


def test_steps_per_launch_is_validated():
    with _random_solver(16, 16, T.TRTR_GRAD_PERIODIC, 2) as s:
        for bad in (0, 3, -1):
            with pytest.raises(T.TrtrError) as e:
                s.set_steps_per_launch(bad)
            assert e.value.status == T.TRTR_EINVAL
