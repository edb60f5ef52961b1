"""Linear (von Neumann) stability of the TRT-R step for the named pulse workloads.

For frozen coefficients (u, tau1, tau2 at a node) one step maps a Fourier mode through
A(k) = diag(exp(-i k.e_q)) C, with C the node's collision matrix from the moment-space
statement of Eq. (12) (tests/_moments.py).  A workload is used only if max |eig A(k)| <= 1
at every sampled node.  The magic choice Lambda = 1/12 fails this at Courant 0.8 once
tau1 - 1/2 is large (the 4096^2 grid at the box corners); the paper leaves tau2 free, and
the 4096^2 / 8192^2 workloads take tau2 = 0.8.
"""
import math

import numpy as np
import pytest

from paper_2312_10316_gb300 import workloads as W

from . import _moments as MS


def spectral_radius(uh_x, uh_y, tau1, tau2, nk=16):
    """max over a k grid of |eig(diag(exp(-i k.e)) C)| for each node (vectorised)."""
    C = np.stack([MS.collision_matrix(a, b, t1, t2) for a, b, t1, t2 in zip(uh_x, uh_y, tau1, tau2)])
    ks = np.linspace(-np.pi, np.pi, nk, endpoint=False)
    KX, KY = np.meshgrid(ks, ks)
    S = np.exp(-1j * (KX.ravel()[:, None] * MS.EX[None, :] + KY.ravel()[:, None] * MS.EY[None, :]))  # (K, 9)
    A = S[None, :, :, None] * C[:, None, :, :]
    ev = np.linalg.eigvals(A)
    return np.abs(ev).max(axis=(1, 2))


def node_parameters(pulse: W.Pulse, stride_nodes: int = 24, magic=1 / 12, tau2=None):
    n = pulse.n
    idx = np.unique(np.concatenate([np.linspace(0, n - 1, stride_nodes).round().astype(int), [0, 1, n - 2, n - 1]]))
    x = pulse.x0 + pulse.dx * idx
    X, Y = np.meshgrid(x, x, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    c = pulse.dx / pulse.dt
    ux, uy = -pulse.omega * Y / c, pulse.omega * X / c
    D = pulse.D0 * (1 + pulse.D_amp * np.sin(np.pi * X) * np.sin(np.pi * Y))
    tau1 = 0.5 + 3.0 * D * pulse.dt / pulse.dx**2  # kappa = (tau1 - 1/2) cs^2 dt
    t2 = np.full_like(tau1, tau2) if tau2 is not None else 0.5 + magic / (tau1 - 0.5)
    return ux, uy, tau1, t2


@pytest.mark.parametrize("pulse", [W.C2A_F32_1024, W.C2B_F32_4096, W.C3_HALF_8192], ids=lambda p: p.name)
def test_named_large_time_step_workloads_are_stable(pulse):
    ux, uy, t1, t2 = node_parameters(pulse, tau2=pulse.tau2)
    assert np.max(np.hypot(ux, uy)) == pytest.approx(pulse.courant, rel=1e-9)
    rho = spectral_radius(ux, uy, t1, t2)
    assert rho.max() <= 1.0 + 1e-9, rho.max()


def test_magic_tau2_is_unstable_at_4096_courant_08():
    """The reason the 4096^2 workload does not take the magic tau2: at the corner node
    (|u dt/dx| = 0.8, D = D0, tau1 - 1/2 = 1.106) some mode grows every step."""
    p = W.C2B_F32_4096
    c = p.dx / p.dt
    ux, uy = -p.omega * p.y0 / c, p.omega * p.x0 / c
    tau1 = 0.5 + 3.0 * p.D0 * p.dt / p.dx**2
    rho = spectral_radius([ux], [uy], [tau1], [0.5 + (1 / 12) / (tau1 - 0.5)], nk=32)
    assert rho[0] > 1.05
    rho_fixed = spectral_radius([ux], [uy], [tau1], [p.tau2], nk=32)
    assert rho_fixed[0] <= 1.0 + 1e-9


def test_relaxation_times_of_the_workloads():
    """tau1 - 1/2 at D0 for the stated grids (Courant 0.8): 0.2766 (1024^2), 1.106 (4096^2)."""
    for pulse, expect in ((W.C2A_F32_1024, 0.2766), (W.C2B_F32_4096, 1.1063), (W.C1_F64_64, 0.004322)):
        t1m = 3.0 * pulse.D0 * pulse.dt / pulse.dx**2
        assert t1m == pytest.approx(expect, rel=2e-3)
    assert W.C1_F64_64.dt == pytest.approx(1.40674e-3, rel=1e-5)
    assert math.isclose(W.C2B_F32_4096.dt, 8.79215e-5, rel_tol=1e-5)
