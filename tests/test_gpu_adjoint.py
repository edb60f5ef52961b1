"""The CUDA adjoint (trtr_forward_record / trtr_adjoint) against the oracle's discrete
adjoint, against central finite differences, and through torch.autograd."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_10316_gb300 import workloads as W

from ._gpu_util import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402
from paper_2312_10316_gb300.autograd import PhiOfD, misfit_and_gradient  # noqa: E402


def _setup(n, steps_courant=0.5, seed=4, tau2=None, nx=None, ny=None):
    """Rotating pulse with a seeded smooth D field (tau1 - 1/2 around 0.3)."""
    nx = nx or n
    ny = ny or n
    base = W.Pulse(n=n, courant=steps_courant)
    D0 = 0.3 / 3.0 * base.dx**2 / base.dt
    pulse = W.Pulse(n=n, courant=steps_courant, D0=D0, tau2=tau2)
    D = W.smooth_random_field(seed, n, amp=0.3, mean=D0)[:ny, :nx]
    f = W.fields(pulse)
    return pulse, f["ux"][:ny, :nx], f["uy"][:ny, :nx], D, f["phi0"][:ny, :nx]


def _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, precision, interval=0, nx=None, ny=None, spl=2):
    nx = nx or pulse.nx
    ny = ny or pulse.ny
    over = {} if pulse.tau2 is None else {"tau2_mode": T.TRTR_TAU2_FIXED, "tau2": pulse.tau2}
    p = T.Params(nx=nx, ny=ny, dx=pulse.dx, dt=pulse.dt, precision=precision, **over)
    with T.Solver(p) as s:
        s.set_steps_per_launch(spl)
        s.set_fields(ux, uy, D)
        s.init_equilibrium(phi0)
        s.forward_record(steps, interval)
        phi = s.moments()
        grad = s.adjoint(lamN)
    return phi, grad


def _oracle_grad(pulse, ux, uy, D, phi0, lamN, steps, nx=None, ny=None):
    nx = nx or pulse.nx
    ny = ny or pulse.ny
    sp = oracle.SimParams(nx=nx, ny=ny, dx=pulse.dx, dt=pulse.dt, grad_mode=1,
                          tau2_mode=0 if pulse.tau2 is None else 1, tau2=pulse.tau2 or 1.0)
    o = oracle.Sim(sp)
    o.set_fields(ux, uy, D)
    o.init_equilibrium(phi0)
    grad = o.adjoint(steps, lamN)
    phi = o.phi()
    o.close()
    return phi, grad


@pytest.mark.parametrize("tau2", [None, 0.9])
def test_adjoint_f64_matches_the_oracle_adjoint_64(tau2):
    pulse, ux, uy, D, phi0 = _setup(64, tau2=tau2)
    steps = 120
    lamN = np.random.default_rng(1).uniform(-1, 1, size=(64, 64))
    phi_g, grad_g = _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, T.TRTR_F64)
    phi_o, grad_o = _oracle_grad(pulse, ux, uy, D, phi0, lamN, steps)
    assert rel_l2(phi_g, phi_o) <= 1e-12
    assert rel_l2(grad_g, grad_o) <= 1e-10


def test_adjoint_ragged_grid_and_checkpoint_intervals():
    """37 x 23 grid, 30 steps: the gradient does not depend on the checkpoint spacing
    (recomputed segments are bit-identical) and matches the oracle."""
    pulse, ux, uy, D, phi0 = _setup(40, nx=37, ny=23)
    lamN = np.random.default_rng(2).uniform(-1, 1, size=(23, 37))
    steps = 30
    grads = [_gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, T.TRTR_F64, iv, nx=37, ny=23)[1] for iv in (1, 7, 0, 30)]
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])
    _, grad_o = _oracle_grad(pulse, ux, uy, D, phi0, lamN, steps, nx=37, ny=23)
    assert rel_l2(grads[0], grad_o) <= 1e-10


def test_recorded_run_with_two_steps_per_launch_gives_the_same_gradient():
    """FP32: the recorded forward run takes pairs of steps between checkpoints through the
    two-step kernel; its checkpoints, hence phi and the gradient, are the one-step run's bits."""
    pulse, ux, uy, D, phi0 = _setup(40, nx=37, ny=23)
    lamN = np.random.default_rng(5).uniform(-1, 1, size=(23, 37))
    for steps, iv in ((30, 7), (31, 0), (30, 1), (29, 29), (40, 8)):
        one = _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, T.TRTR_F32, iv, nx=37, ny=23, spl=1)
        two = _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, T.TRTR_F32, iv, nx=37, ny=23, spl=2)
        assert np.array_equal(one[0], two[0]), (steps, iv)
        assert np.array_equal(one[1], two[1]), (steps, iv)


@pytest.mark.parametrize("precision", [T.TRTR_F16_OFS, T.TRTR_BF16_OFS])
def test_two_byte_recorded_run_and_recomputation_with_two_steps_per_launch(precision):
    """2-byte storages on an even-nx grid: the recorded run and the segment recomputation (which
    also stores the intermediate state) take pairs of steps through the two-step kernel; phi and
    the gradient are the one-step run's bits."""
    pulse, ux, uy, D, phi0 = _setup(40, nx=38, ny=23)
    lamN = np.random.default_rng(6).uniform(-1, 1, size=(23, 38))
    for steps, iv in ((30, 7), (31, 0), (40, 8)):
        one = _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, precision, iv, nx=38, ny=23, spl=1)
        two = _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, precision, iv, nx=38, ny=23, spl=2)
        assert np.array_equal(one[0], two[0]), (steps, iv)
        assert np.array_equal(one[1], two[1]), (steps, iv)
        assert np.isfinite(two[1]).all()


def test_adjoint_f32_against_the_oracle_adjoint_64():
    """FP32 forward states and FP32 adjoint arithmetic (FP64 accumulation of dJ/dD)."""
    pulse, ux, uy, D, phi0 = _setup(64)
    steps = 120
    lamN = np.random.default_rng(3).uniform(-1, 1, size=(64, 64))
    _, grad_g = _gpu_grad(pulse, ux, uy, D, phi0, lamN, steps, T.TRTR_F32)
    _, grad_o = _oracle_grad(pulse, ux, uy, D, phi0, lamN, steps)
    assert rel_l2(grad_g, grad_o) <= 1e-4


def test_autograd_function_gives_the_adjoint_gradient():
    pulse, ux, uy, D, phi0 = _setup(48)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    phi_obs = dev(W.phi_analytic(pulse, 0.0) * 0.9)
    p = T.Params(nx=48, ny=48, dx=pulse.dx, dt=pulse.dt, precision=T.TRTR_F64)
    with T.Solver(p) as s:
        J, g = misfit_and_gradient(s, dev(ux), dev(uy), dev(D), dev(phi0), phi_obs, 40)
        lam = (torch.empty(48, 48, dtype=torch.float64, device="cuda"))
        s.set_fields(ux, uy, D)
        s.init_equilibrium(phi0)
        s.forward_record(40)
        s.moments(lam)
        lam -= phi_obs
        ref = s.adjoint(lam.cpu().numpy())
    assert np.allclose(g.cpu().numpy(), ref, rtol=1e-13, atol=0)
    assert float(J) > 0
    # a step along -grad lowers J (first-order check of the sign)
    with T.Solver(p) as s:
        Dn = dev(D) - 1e-3 * float(dev(D).abs().max()) * g / float(g.abs().max())
        J2, _ = misfit_and_gradient(s, dev(ux), dev(uy), Dn, dev(phi0), phi_obs, 40)
    assert float(J2) < float(J)


@pytest.mark.slow
def test_adjoint_512_2000_steps_against_central_differences():
    """The adjoint workload: 512^2 pulse, Courant 0.8, 2000 steps.  phi_obs comes from a
    seeded smooth D field (8 Fourier modes, 30 %, mean 1e-3); J = 1/2 sum (phi - phi_obs)^2 is
    differentiated at D = 1e-3.

    * FP64 path: the adjoint gradient equals central differences of the FP64 forward run
      (h = 1e-3 D) at 16 random nodes to 1e-5 relative (it is exact up to FD truncation).
    * FP32 path: its gradient differs from the FP64 one by the FP32 forward trajectory's
      error, 2.7e-7 of phi after 2000 steps, which enters through the misfit phi - phi_obs,
      itself only 3e-3 of phi here: measured 2.0e-5 relative L2 against the FP64 gradient and
      5.4e-5 per node against the differences, held to 2e-4 and 5e-4.  (Before the FP32 rest
      population closed the mass balance, the trajectory drifted by ~1e-5 and these were ~1e-3
      and ~1e-2.)"""
    pulse = W.C5_ADJ_512
    n, steps = pulse.n, pulse.steps
    f = W.fields(pulse)
    D_true = W.smooth_random_field(5, n, modes=8, kmax=4, amp=0.3, mean=1e-3)
    D = np.full((n, n), 1e-3)

    def forward(Dv, prec):
        p = T.Params(nx=n, ny=n, dx=pulse.dx, dt=pulse.dt, precision=prec)
        with T.Solver(p) as s:
            s.set_fields(f["ux"], f["uy"], Dv)
            s.init_equilibrium(f["phi0"])
            s.step(steps)
            return s.moments()

    phi_obs = forward(D_true, T.TRTR_F64)
    grads = {}
    for prec in (T.TRTR_F64, T.TRTR_F32):
        p = T.Params(nx=n, ny=n, dx=pulse.dx, dt=pulse.dt, precision=prec)
        with T.Solver(p) as s:
            s.set_fields(f["ux"], f["uy"], D)
            s.init_equilibrium(f["phi0"])
            s.forward_record(steps)
            phi = s.moments()
            grads[prec] = s.adjoint(phi - phi_obs)
    g64, g32 = grads[T.TRTR_F64], grads[T.TRTR_F32]
    assert rel_l2(g32, g64) <= 2e-4

    def J(Dv):
        return 0.5 * float(np.sum((forward(Dv, T.TRTR_F64) - phi_obs) ** 2))

    rng = np.random.default_rng(16)
    cand = np.argwhere(np.abs(g64) > 0.05 * np.abs(g64).max())  # where the pulse has passed
    picks = cand[rng.choice(len(cand), size=16, replace=False)]
    e64, e32 = [], []
    for j, i in picks:
        h = 1e-3 * D[j, i]
        Dp, Dm = D.copy(), D.copy()
        Dp[j, i] += h
        Dm[j, i] -= h
        fd = (J(Dp) - J(Dm)) / (2 * h)
        e64.append(abs(g64[j, i] - fd) / abs(fd))
        e32.append(abs(g32[j, i] - fd) / abs(fd))
    assert max(e64) <= 1e-5, e64
    assert max(e32) <= 5e-4, e32
