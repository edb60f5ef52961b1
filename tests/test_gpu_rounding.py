"""Stochastic rounding of the 2-byte storages (TRTR_ROUND_STOCHASTIC) against nearest rounding
and the FP64 oracle.

The method (Eq. (14) of Sec. 2.2) is stated in exact arithmetic; storing its populations as
FP16 / BF16 offsets rounds every stored value each step.  Rounded to nearest, a smooth field
makes the same rounding error at neighbouring nodes and steps, so the errors add up like a bias
(the error of phi grows linearly with the step count).  Rounded stochastically, each rounding
error has zero mean and is independent of the others, and the diffusion of the method damps
them.  The random bits are a fixed hash of the node, the step and the population, so a run is
reproducible and independent of how its steps are split into calls."""
import numpy as np
import pytest

import oracle
from paper_2312_10316_gb300 import workloads as W

from ._gpu_util import assert_elementwise, oracle_for_pulse, random_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402

PREC = {"f16": T.TRTR_F16_OFS, "bf16": T.TRTR_BF16_OFS}
UNIT = {"f16": 2.0**-11, "bf16": 2.0**-8}  # unit roundoff of the formats


def _random_pair(prec, rounding, nx=70, ny=41, phi_ref=0.0, seed=11):
    case = random_case(seed, nx, ny)
    common = dict(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], x0=-0.3, y0=-0.2, grad_mode=1)
    o = oracle.Sim(oracle.SimParams(**common))
    s = T.Solver(T.Params(precision=PREC[prec], phi_ref=phi_ref, rounding=rounding, **common))
    for x in (o, s):
        x.set_fields(case["ux"], case["uy"], case["D"])
    o.set_g(case["g"])
    s.set_populations(case["g"])
    return o, s


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_runs_are_reproducible_and_independent_of_the_step_split(prec):
    res = []
    for split in ((7,), (3, 4), (1, 1, 5)):
        o, s = _random_pair(prec, T.TRTR_ROUND_STOCHASTIC)
        with s:
            for n in split:
                s.step(n)
            res.append(s.get_populations())
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
    o, s = _random_pair(prec, T.TRTR_ROUND_NEAREST)
    with s:
        s.step(7)
        assert not np.array_equal(s.get_populations(), res[0])  # the rounding mode is in effect


@pytest.mark.parametrize("prec,phi_ref", [("f16", 0.0), ("f16", 1.0), ("bf16", 0.0), ("bf16", 1.0)])
def test_one_step_stays_within_one_unit_of_the_format(prec, phi_ref):
    """A stochastically rounded value is one of the two neighbours of the exact one: within one
    unit of the format (twice the nearest-rounding bound)."""
    o, s = _random_pair(prec, T.TRTR_ROUND_STOCHASTIC, phi_ref=phi_ref)
    with s:
        o.step(1)
        s.step(1)
        gp, og = s.get_populations(), o.get_g()
        assert rel_l2(gp, og) <= 4 * UNIT[prec]
        assert_elementwise(gp, og, 8 * UNIT[prec], prec, tile=(64, 8))


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_rounding_errors_have_zero_mean(prec):
    """Many nodes of the same step: the mean of the stored-minus-exact differences over every
    population is far below one unit (nearest rounding of these smooth values is biased)."""
    pulse = W.Pulse(n=256, courant=0.4)
    errs = {}
    for rounding in (T.TRTR_ROUND_NEAREST, T.TRTR_ROUND_STOCHASTIC):
        with T.pulse_solver(pulse, precision=T.TRTR_F32) as ref, \
                T.pulse_solver(pulse, precision=PREC[prec], rounding=rounding) as s:
            ref.step(40)
            s.set_populations(ref.get_populations(), step=40)  # rounded to the format on the way in
            ref.set_populations(s.get_populations(), step=40)  # the same (exactly representable) state
            ref.step(1)
            s.step(1)
            r = ref.get_populations()
            d = s.get_populations() - r
            big = np.abs(r) > 1e-3  # away from the underflow of the far field
            errs[rounding] = (float(np.mean(d[big] / np.abs(r[big]))), float(np.std(d[big] / np.abs(r[big]))))
    mean_sr, std_sr = errs[T.TRTR_ROUND_STOCHASTIC]
    assert abs(mean_sr) <= 0.02 * UNIT[prec], errs
    assert std_sr <= UNIT[prec], errs


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_stochastic_rounding_error_grows_slower_than_nearest(prec):
    """The 1024^2 workload's relaxation times on a 200^2 grid, 2000 steps, both roundings
    against the FP64 oracle: stochastic rounding ends several times closer."""
    base = W.Pulse(n=200, courant=0.8)
    D0 = 0.2766 / 3.0 * base.dx**2 / base.dt
    pulse = W.Pulse(n=200, D_amp=0.5, D0=D0, courant=0.8, steps=2000)
    o = oracle_for_pulse(pulse)
    o.step(pulse.steps)
    phi_o = o.phi()
    err = {}
    for rounding in (T.TRTR_ROUND_NEAREST, T.TRTR_ROUND_STOCHASTIC):
        with T.pulse_solver(pulse, precision=PREC[prec], rounding=rounding) as s:
            s.step(pulse.steps)
            err[rounding] = rel_l2(s.moments(), phi_o)
    assert err[T.TRTR_ROUND_STOCHASTIC] <= err[T.TRTR_ROUND_NEAREST] / 3, err
