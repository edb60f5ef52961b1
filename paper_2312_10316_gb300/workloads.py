"""Seeded synthetic inputs for the rotating, spreading Gaussian pulse workloads.

This module holds the WORKLOAD only: grids, closed-form fields, the analytic solution,
the manufactured source and seeded random states.  It contains none of the lattice
Boltzmann method's arithmetic (no equilibrium, collision, relaxation-time relation or
streaming), so both the CUDA path and the FP64 oracle can be fed from it.

Pulse (the paper's benchmark family of Sec. 3, a Gaussian carried by a rigid-body
rotation while it diffuses), on the periodic box [-1, 1)^2 with nodes
x_i = -1 + i dx, dx = 2/N:

    u = omega (-y, x)
    phi_a(x, t) = (s0^2 / s^2) exp(-|x - c(t)|^2 / (2 s^2)),  s^2 = s0^2 + 2 D0 t,
    c(t) = R(omega t) (xc, yc)

phi_a solves Eq. (1) with constant kappa = D0 and S = 0 in free space (the rotation is
solenoidal and the Gaussian isotropic).  With the variable diffusivity
D(x) = D0 (1 + a sin(pi x) sin(pi y)) the manufactured source
S = -div((D - D0) grad phi_a) keeps phi_a exact.  The time step follows from the Courant
number Cr = max|u| dt / dx = omega sqrt(2) dt / dx (the corner node has r = sqrt(2)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Pulse:
    """One rotating-pulse problem on an N x N periodic grid."""

    n: int
    omega: float = math.pi
    xc: float = -0.5
    yc: float = 0.0
    sigma0: float = 0.1
    D0: float = 1e-3
    D_amp: float = 0.0
    courant: float = 0.2
    steps: int = 500
    name: str = ""
    tau2: float | None = None  # None: tau2 from the magic parameter 1/12; else fixed tau2

    @property
    def nx(self) -> int:
        return self.n

    @property
    def ny(self) -> int:
        return self.n

    @property
    def x0(self) -> float:
        return -1.0

    @property
    def y0(self) -> float:
        return -1.0

    @property
    def dx(self) -> float:
        return 2.0 / self.n

    @property
    def dt(self) -> float:
        return self.courant * self.dx / (self.omega * math.sqrt(2.0))

    @property
    def manufactured_source(self) -> bool:
        return self.D_amp != 0.0


# The five workloads (sizes and parameters as stated for each).  At Courant 0.8 the magic
# choice Lambda = 1/12 makes the step linearly unstable at the box corners (|u dt/dx| = 0.8)
# once tau1 - 1/2 exceeds ~0.9, which is the case on the 4096^2 and 8192^2 grids; tau2 is the
# paper's free parameter, and tau2 = 0.8 (the magic value of the 1024^2 grid at D0) keeps
# every node of those grids stable.
C1_F64_64 = Pulse(n=64, courant=0.2, steps=500, name="pulse64_f64_constD")
C2A_F32_1024 = Pulse(n=1024, D_amp=0.5, courant=0.8, steps=10_000, name="pulse1024_f32_varD_mms")
C2B_F32_4096 = Pulse(n=4096, D_amp=0.5, courant=0.8, steps=10_000, tau2=0.8, name="pulse4096_f32_varD_mms")
C3_HALF_8192 = Pulse(n=8192, D_amp=0.5, courant=0.8, steps=10_000, tau2=0.8, name="pulse8192_half_varD_mms")
C5_ADJ_512 = Pulse(n=512, courant=0.8, steps=2000, name="pulse512_adjoint")


def coords(p: Pulse) -> tuple[np.ndarray, np.ndarray]:
    """Node coordinates X[j, i] = x0 + i dx, Y[j, i] = y0 + j dx (row-major, x fastest)."""
    x = p.x0 + p.dx * np.arange(p.nx, dtype=np.float64)
    y = p.y0 + p.dx * np.arange(p.ny, dtype=np.float64)
    return np.meshgrid(x, y, indexing="xy")


def velocity(p: Pulse) -> tuple[np.ndarray, np.ndarray]:
    X, Y = coords(p)
    return -p.omega * Y, p.omega * X


def diffusivity(p: Pulse) -> np.ndarray:
    X, Y = coords(p)
    return p.D0 * (1.0 + p.D_amp * np.sin(np.pi * X) * np.sin(np.pi * Y))


def centre(p: Pulse, t: float) -> tuple[float, float]:
    c, s = math.cos(p.omega * t), math.sin(p.omega * t)
    return p.xc * c - p.yc * s, p.xc * s + p.yc * c


def phi_analytic(p: Pulse, t: float, X=None, Y=None) -> np.ndarray:
    if X is None:
        X, Y = coords(p)
    cx, cy = centre(p, t)
    s2 = p.sigma0**2 + 2.0 * p.D0 * t
    return (p.sigma0**2 / s2) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * s2))


def source(p: Pulse, t: float, X=None, Y=None) -> np.ndarray:
    """Manufactured S = -[grad D . grad phi_a + (D - D0) lap phi_a] (zero when D_amp = 0)."""
    if X is None:
        X, Y = coords(p)
    cx, cy = centre(p, t)
    s2 = p.sigma0**2 + 2.0 * p.D0 * t
    rx, ry = X - cx, Y - cy
    r2 = rx * rx + ry * ry
    ph = (p.sigma0**2 / s2) * np.exp(-r2 / (2.0 * s2))
    gx, gy = -rx / s2 * ph, -ry / s2 * ph
    lap = (r2 / s2**2 - 2.0 / s2) * ph
    a = p.D0 * p.D_amp
    dD = a * np.sin(np.pi * X) * np.sin(np.pi * Y)
    dDx = a * np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
    dDy = a * np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
    return -(dDx * gx + dDy * gy + dD * lap)


def fields(p: Pulse) -> dict[str, np.ndarray]:
    ux, uy = velocity(p)
    return {"ux": ux, "uy": uy, "D": diffusivity(p), "phi0": phi_analytic(p, 0.0)}


def disk_mask(p: Pulse, radius: float = 0.9) -> np.ndarray:
    X, Y = coords(p)
    return X * X + Y * Y <= radius * radius


# --------------------------------------------------------------------------------------
# Seeded generic inputs for parity tests (not pulse-shaped)


def random_populations(seed: int, ny: int, nx: int, base: float = 1.0, amp: float = 0.1) -> np.ndarray:
    """[9][ny][nx] positive populations around base * w_i-like magnitudes (uniform noise)."""
    rng = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return w[:, None, None] * base * (1.0 + amp * rng.uniform(-1.0, 1.0, size=(9, ny, nx)))


def random_field(seed: int, ny: int, nx: int, lo: float, hi: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(ny, nx))


def smooth_random_field(seed: int, n: int, modes: int = 8, kmax: int = 4, amp: float = 0.3,
                        mean: float = 1e-3) -> np.ndarray:
    """mean * (1 + amp * m / max|m|), m a sum of `modes` seeded periodic Fourier modes on [-1,1)^2."""
    rng = np.random.default_rng(seed)
    x = -1.0 + (2.0 / n) * np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    m = np.zeros((n, n))
    for _ in range(modes):
        kx, ky = rng.integers(1, kmax + 1, size=2)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        m += np.cos(np.pi * (kx * X + ky * Y) + ph)
    return mean * (1.0 + amp * m / np.max(np.abs(m)))


@dataclass(frozen=True)
class BatchInstance:
    pulse: Pulse
    offset: int  # node offset of this instance in the packed batch


def batch_instances(seed: int = 0, count: int = 256, sizes=(64, 128, 256, 512, 1024),
                    courant: float = 0.2, steps: int = 1000) -> list[BatchInstance]:
    """Seeded uneven batch: square grids drawn from `sizes`, omega in [pi/2, 2 pi],
    sigma0 in [0.05, 0.15], D0 in [1e-4, 1e-2] (constant per instance)."""
    rng = np.random.default_rng(seed)
    out: list[BatchInstance] = []
    off = 0
    for k in range(count):
        n = int(rng.choice(sizes))
        omega = float(rng.uniform(0.5 * math.pi, 2.0 * math.pi))
        sigma0 = float(rng.uniform(0.05, 0.15))
        D0 = float(rng.uniform(1e-4, 1e-2))
        p = Pulse(n=n, omega=omega, sigma0=sigma0, D0=D0, courant=courant, steps=steps, name=f"inst{k}")
        out.append(BatchInstance(p, off))
        off += n * n
    return out


# --- The paper's own benchmark (Sec. 3, Table 2) -------------------------------------------
#
# Rigid rotation u = (-y, x) on [-2 pi, 2 pi]^2 with constant kappa; Table 2 reports t = 1.
# The closed form
#     phi_a(x, y, t) = exp(-(x^2 + 3 y^2 + 2 kappa t)),
#     S(x, y, t) = [6 kappa - 4 x y - 4 kappa (x^2 + 9 y^2)] exp(-(x^2 + 3 y^2 + 2 kappa t)),
# held on the boundary by Dirichlet conditions.  Nodes: N intervals per side, N + 1 nodes
# including both edges, dx = L / N; Table 2's diffusive scaling is (dx)^2 / dt = 0.16 pi^2.


@dataclass(frozen=True)
class PaperPulse:
    N: int                      # intervals per side
    kappa: float
    L: float = 4.0 * math.pi
    dt: float | None = None     # None: Table 2's scaling (dx)^2 / dt = 0.16 pi^2
    t_end: float = 1.0

    @property
    def nx(self) -> int:
        return self.N + 1

    @property
    def ny(self) -> int:
        return self.N + 1

    @property
    def x0(self) -> float:
        return -self.L / 2.0

    @property
    def y0(self) -> float:
        return -self.L / 2.0

    @property
    def dx(self) -> float:
        return self.L / self.N

    @property
    def time_step(self) -> float:
        return self.dt if self.dt is not None else self.dx**2 / (0.16 * math.pi**2)

    @property
    def steps(self) -> int:
        return int(round(self.t_end / self.time_step))


def paper_coords(p: PaperPulse) -> tuple[np.ndarray, np.ndarray]:
    x = p.x0 + np.arange(p.nx) * p.dx
    y = p.y0 + np.arange(p.ny) * p.dx
    return np.meshgrid(x, y, indexing="xy")


def paper_fields(p: PaperPulse) -> dict[str, np.ndarray]:
    X, Y = paper_coords(p)
    return {"ux": -Y, "uy": X.copy(), "D": np.full_like(X, p.kappa), "phi0": paper_phi(p, 0.0)}


def paper_phi(p: PaperPulse, t: float) -> np.ndarray:
    X, Y = paper_coords(p)
    return np.exp(-(X * X + 3.0 * Y * Y + 2.0 * p.kappa * t))


def paper_source(p: PaperPulse, t: float) -> np.ndarray:
    X, Y = paper_coords(p)
    k = p.kappa
    return (6.0 * k - 4.0 * X * Y - 4.0 * k * (X * X + 9.0 * Y * Y)) * np.exp(-(X * X + 3.0 * Y * Y + 2.0 * k * t))
