"""Batched instances (one persistent launch per step over a tile work-list spanning every
instance, replayed from a CUDA graph) against single-instance solves and the oracle."""
import math

import numpy as np
import pytest

from paper_2312_10316_gb300 import workloads as W

from ._gpu_util import TOL_F32, assert_elementwise, oracle_for_pulse, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402


def _uneven_pulses(seed=3, sizes=(48, 64, 100, 130, 200, 37), D_amp=0.0):
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        base = W.Pulse(n=n, courant=0.5)
        # relaxation times in the stable range: tau1 - 1/2 in (0.15, 0.6)
        D0 = float(rng.uniform(0.15, 0.6)) / 3.0 * base.dx**2 / base.dt
        out.append(W.Pulse(n=n, omega=float(rng.uniform(0.5, 2.0) * math.pi), sigma0=float(rng.uniform(0.1, 0.15)),
                           D0=D0, D_amp=D_amp, courant=0.5))
    return out


def _single_solution(pulse, precision, steps, **kw):
    with T.pulse_solver(pulse, precision=precision, **kw) as s:
        s.step(steps)
        return s.get_populations().copy()


@pytest.mark.parametrize("precision", [T.TRTR_F32, T.TRTR_F16_OFS])
def test_every_batch_config_is_bitwise_the_single_solve(precision):
    pulses = _uneven_pulses()
    steps = 37  # odd: one direct launch besides the graph replays
    ref = [_single_solution(p, precision, steps) for p in pulses]
    for config in range(T.trtr_batch_config_count()):
        with T.Batch([T.pulse_instance(p, precision) for p in pulses]) as b:
            b.set_config(config)
            b.set_steps_per_launch(1)  # every step through the configured one-step kernel
            b.step(steps)
            b.sync()
            assert b.info()["step"] == steps
            for k, p in enumerate(pulses):
                got = b.instance(k).get_populations()
                assert np.array_equal(got, ref[k]), (T.trtr_batch_config_name(config), k, p.n)


def test_batch_with_pulse_source_against_oracle_and_single():
    pulses = _uneven_pulses(seed=5, sizes=(64, 96, 150), D_amp=0.5)
    steps = 120
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in pulses]) as b:
        b.step(steps)
        b.sync()
        for k, p in enumerate(pulses):
            phi = b.instance(k).moments()
            o = oracle_for_pulse(p)
            o.step(steps)
            assert rel_l2(phi, o.phi()) <= TOL_F32
            assert_elementwise(phi, o.phi(), TOL_F32, f"instance {k}")
            with T.pulse_solver(p, precision=T.TRTR_F32) as s:
                s.step(steps)
                # the time uniforms come from the device clock (double cos/sin) here and
                # from the host in the single solve: equal to within FP32 rounding
                assert rel_l2(phi, s.moments()) <= 1e-6


def test_tune_restores_the_initial_state_and_picks_a_config():
    pulses = _uneven_pulses(seed=9, sizes=(64, 128, 80))
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in pulses]) as b:
        g0 = [b.instance(k).get_populations().copy() for k in range(len(pulses))]
        best, ms = b.tune(4)
        assert 0 <= best < T.trtr_batch_config_count()
        assert len(ms) == T.trtr_batch_config_count() and all(m > 0 for m in ms)
        info = b.info()
        assert info["step"] == 0 and info["config"] == best
        for k in range(len(pulses)):
            assert np.array_equal(b.instance(k).get_populations(), g0[k])
        b.step(10)
        ref = _single_solution(pulses[1], T.TRTR_F32, 10)
        assert np.array_equal(b.instance(1).get_populations(), ref)


def test_tune_at_step_zero_keeps_the_callers_own_state():
    """Instances set by the caller (populations of their own, not the pulse's initial condition)
    come back from the tuner's trial steps unchanged, and then step as single solves do."""
    pulses = _uneven_pulses(seed=11, sizes=(64, 96))
    own = [W.random_populations(40 + k, p.ny, p.nx, base=0.5, amp=0.2) for k, p in enumerate(pulses)]
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in pulses]) as b:
        for k in range(len(pulses)):
            b.instance(k).set_populations(own[k])
        g0 = [b.instance(k).get_populations().copy() for k in range(len(pulses))]
        b.tune(4)
        assert b.info()["step"] == 0
        for k in range(len(pulses)):
            assert np.array_equal(b.instance(k).get_populations(), g0[k]), k
        b.step(9)
        b.sync()
        for k, p in enumerate(pulses):
            with T.pulse_solver(p, precision=T.TRTR_F32) as s:
                s.set_populations(own[k])
                s.step(9)
                assert np.array_equal(b.instance(k).get_populations(), s.get_populations()), k


def test_instances_cannot_be_stepped_alone():
    pulses = _uneven_pulses(sizes=(32, 40))
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in pulses]) as b:
        with pytest.raises(T.TrtrError):
            b.instance(0).step(1)
        ctx = b.instance(0).ctx
        T.lib.trtr_step(ctx, 1)  # through the raw C call: the batch then refuses to step
        with pytest.raises(T.TrtrError) as e:
            b.step(1)
        assert e.value.status == T.TRTR_ESTATE


@pytest.mark.parametrize("steps", [[37], [3, 5, 2, 7, 1, 9]])
@pytest.mark.parametrize("D_amp", [0.0, 0.5])
def test_two_steps_per_launch_batch_is_bitwise_the_single_solve(steps, D_amp):
    """FP32 batches run pairs of steps through the two-step kernel; odd steps, and step counts
    split over several calls, interleave it with the one-step kernel (D_amp > 0: the in-kernel
    pulse source, whose time uniforms both kernels advance)."""
    pulses = _uneven_pulses(D_amp=D_amp)
    total = sum(steps)
    ref = [_single_solution(p, T.TRTR_F32, total) for p in pulses]
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in pulses]) as b:
        for n in steps:
            b.step(n)
        b.sync()
        assert b.info()["step"] == total
        for k, p in enumerate(pulses):
            assert np.array_equal(b.instance(k).get_populations(), ref[k]), (k, p.n)


@pytest.mark.parametrize("precision", [T.TRTR_F16_OFS, T.TRTR_BF16_OFS])
@pytest.mark.parametrize("rounding", [T.TRTR_ROUND_STOCHASTIC, T.TRTR_ROUND_NEAREST])
@pytest.mark.parametrize("D_amp", [0.0, 0.5])
def test_two_byte_two_step_batch_is_bitwise_the_single_solve(precision, rounding, D_amp):
    """2-byte batches of even-sized instances run pairs of steps through the two-step kernel,
    whose intermediate state is rounded with the one-step kernel's bits; step counts split over
    several calls interleave it with the one-step batch kernel."""
    pulses = _uneven_pulses(D_amp=D_amp, sizes=(48, 64, 100, 130, 200, 38))
    steps = [3, 5, 2, 7, 1, 9]
    total = sum(steps)
    ref = [_single_solution(p, precision, total, rounding=rounding) for p in pulses]
    with T.Batch([T.pulse_instance(p, precision, rounding=rounding) for p in pulses]) as b:
        assert b.steps_per_launch == 2
        for n in steps:
            b.step(n)
        b.sync()
        for k, p in enumerate(pulses):
            assert np.array_equal(b.instance(k).get_populations(), ref[k]), (k, p.n)


def test_steps_per_launch_of_batches():
    even = _uneven_pulses(sizes=(48, 64))
    odd = _uneven_pulses(sizes=(48, 37))
    with T.Batch([T.pulse_instance(p, T.TRTR_F16_OFS) for p in even]) as b:
        assert b.steps_per_launch == 2
        b.set_steps_per_launch(1)
        assert b.steps_per_launch == 1
    with T.Batch([T.pulse_instance(p, T.TRTR_F16_OFS) for p in odd]) as b:
        assert b.steps_per_launch == 1  # an instance of odd nx: one step per launch
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in odd]) as b:
        assert b.steps_per_launch == 2


def test_batch_steps_per_launch_is_validated():
    pulses = _uneven_pulses()[:2]
    with T.Batch([T.pulse_instance(p, T.TRTR_F32) for p in pulses]) as b:
        for bad in (0, 3):
            with pytest.raises(T.TrtrError):
                b.set_steps_per_launch(bad)
