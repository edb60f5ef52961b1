"""Independent moment-space statement of the TRT-R step, used only to pin the oracle.

The oracle works in population space (explicit g^eq, g^neq, B^neq, then the rebuild of
Eq. (12)).  Here the same operator is stated in the space of the nine D2Q9 Hermite
moments {1, x, y, H_xx, H_yy, H_xy, H_xxy, H_xyy, H_xxyy} (lattice units, c = 1,
cs^2 = 1/3):

  - the equilibrium's moments are its Hermite coefficients phi, phi u_a, phi u_a u_b,
    phi u_x^2 u_y, phi u_x u_y^2 and 0 for H_xxyy (Eq. (6), orthogonality of the Hermite
    polynomials under the D2Q9 weights);
  - TRT-R relaxes the first-order non-equilibrium moment by (1 - 1/tau1), the second-order
    one by (1 - 1/tau2) and drops everything above (Eq. (12));
  - G adds dt (1 - 1/(2 tau1)) phi (u.grad)u to the first moment only (Eq. (16));
  - F adds S to the zeroth and (1 - 1/(2 tau1)) u S to the first moment (Eq. (3)).

Post-collision populations follow by inverting the 9 x 9 moment matrix.
"""
from __future__ import annotations

import numpy as np

EX = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1], dtype=np.float64)
EY = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1], dtype=np.float64)
CS2 = 1.0 / 3.0


def moment_matrix() -> np.ndarray:
    """Rows: Hermite polynomials evaluated at the nine lattice velocities (c = 1)."""
    hxx = EX * EX - CS2
    hyy = EY * EY - CS2
    return np.stack([
        np.ones(9), EX, EY, hxx, hyy, EX * EY,
        EX * EX * EY - CS2 * EY, EX * EY * EY - CS2 * EX, hxx * hyy,
    ])


M = moment_matrix()
MINV = np.linalg.inv(M)


def relaxation_operator(ux, uy, tau1, tau2, ax=0.0, ay=0.0, dt_g=0.0) -> np.ndarray:
    """9x9 map of pre- to post-collision moments (lattice units).

    (ax, ay) is (u.grad)u in lattice units and dt_g switches the auxiliary term on
    (dt_g = 1 means ``+ dt G`` with dt = 1 in lattice units)."""
    R = np.zeros((9, 9))
    R[0, 0] = 1.0
    k1 = 1.0 - 1.0 / tau1
    k2 = 1.0 - 1.0 / tau2
    kg = dt_g * (1.0 - 1.0 / (2.0 * tau1))
    # first order: phi u + k1 (m - phi u) + kg phi a
    R[1, 1] = k1
    R[1, 0] = (1.0 - k1) * ux + kg * ax
    R[2, 2] = k1
    R[2, 0] = (1.0 - k1) * uy + kg * ay
    # second order: phi u_a u_b + k2 (m - phi u_a u_b)
    for row, val in ((3, ux * ux), (4, uy * uy), (5, ux * uy)):
        R[row, row] = k2
        R[row, 0] = (1.0 - k2) * val
    # third order: equilibrium values
    R[6, 0] = ux * ux * uy
    R[7, 0] = ux * uy * uy
    # fourth order: equilibrium value 0
    return R


def collision_matrix(ux, uy, tau1, tau2, ax=0.0, ay=0.0, dt_g=0.0) -> np.ndarray:
    """Node-local linear map g -> post-collision (+ dt G) in population space."""
    return MINV @ relaxation_operator(ux, uy, tau1, tau2, ax, ay, dt_g) @ M


def source_populations(S_eff, ux, uy, tau1) -> np.ndarray:
    """Populations carrying zeroth moment S_eff and first moment (1 - 1/(2 tau1)) u S_eff."""
    m = np.zeros(9)
    m[0] = S_eff
    m[1] = (1.0 - 1.0 / (2.0 * tau1)) * ux * S_eff
    m[2] = (1.0 - 1.0 / (2.0 * tau1)) * uy * S_eff
    return MINV @ m
