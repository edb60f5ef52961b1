"""Shared setup of the GPU parity tests: the same seeded inputs go to the CUDA library
(through the C ABI binding) and to the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2312_10316_gb300 import workloads as W

# Relative-L2 tolerances on phi / populations against the FP64 oracle.
TOL_F64 = 1e-12
TOL_F32 = 1e-5


def oracle_for_pulse(pulse: W.Pulse, src_mode: int | None = None) -> oracle.Sim:
    if src_mode is None:
        src_mode = 2 if pulse.D_amp != 0.0 else 0
    sp = oracle.SimParams(nx=pulse.nx, ny=pulse.ny, dx=pulse.dx, dt=pulse.dt, x0=pulse.x0, y0=pulse.y0,
                          src_mode=src_mode, grad_mode=1, omega=pulse.omega, xc=pulse.xc, yc=pulse.yc,
                          sigma0=pulse.sigma0, D0=pulse.D0, D_amp=pulse.D_amp,
                          tau2_mode=0 if pulse.tau2 is None else 1, tau2=pulse.tau2 or 1.0)
    s = oracle.Sim(sp)
    f = W.fields(pulse)
    s.set_fields(f["ux"], f["uy"], f["D"])
    s.init_equilibrium(f["phi0"])
    return s


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def random_case(seed: int, nx: int, ny: int, dx: float = 0.1, dt: float = 0.02):
    """Seeded generic inputs: populations, u with |u dt/dx| <= 0.3, D giving tau1 in
    (0.55, 1.5), and two source fields."""
    rng = np.random.default_rng(seed)
    c = dx / dt
    g = W.random_populations(seed, ny, nx, base=1.0, amp=0.3)
    ux = c * rng.uniform(-0.2, 0.2, size=(ny, nx))
    uy = c * rng.uniform(-0.2, 0.2, size=(ny, nx))
    tau1 = rng.uniform(0.55, 1.5, size=(ny, nx))
    D = (tau1 - 0.5) * (c * c / 3.0) * dt
    S1 = rng.uniform(-1.0, 1.0, size=(ny, nx))
    S2 = rng.uniform(-1.0, 1.0, size=(ny, nx))
    return dict(g=g, ux=ux, uy=uy, D=D, S1=S1, S2=S2, dx=dx, dt=dt)


def regions(nx: int, ny: int, tile=(128, 16), edge: int = 2):
    """Boolean [ny][nx] masks of the node sets that break differently: the nodes within `edge` of
    a grid edge (they pull across the periodic seam from the ghost frame and store ghost copies),
    the last, ragged tile column and tile row of a `tile`-sized tiling, and the rest."""
    j, i = np.mgrid[0:ny, 0:nx]
    near = (i < edge) | (i >= nx - edge) | (j < edge) | (j >= ny - edge)
    tx, ty = tile
    ragged = np.zeros((ny, nx), dtype=bool)
    if nx % tx:
        ragged |= i >= nx - nx % tx
    if ny % ty:
        ragged |= j >= ny - ny % ty
    return {"edge": near, "ragged tile": ragged & ~near, "interior": ~near & ~ragged}


def assert_elementwise(got, ref, tol: float, what: str = "", tile=(128, 16)):
    """Element by element: |got - ref| <= tol * max|ref| on every node of every plane, reported
    separately for the edge nodes, the ragged last tile column/row and the interior (arrays
    [ny][nx] or [planes][ny][nx]).  One wrong node, or a wrong edge row, fails this where a
    relative L2 norm over the whole field could still pass."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = float(np.max(np.abs(ref))) or 1.0
    err = np.abs(got - ref) / scale
    if err.ndim == 2:
        err = err[None]
    ny, nx = err.shape[-2:]
    worst = {}
    for name, mask in regions(nx, ny, tile).items():
        if mask.any():
            worst[name] = float(err[:, mask].max())
    bad = {k: v for k, v in worst.items() if not v <= tol}
    if bad:
        q, jj, ii = np.unravel_index(int(np.nanargmax(err)), err.shape)
        raise AssertionError(f"{what}: per-element error above {tol:g} x max|ref| in {bad}; "
                             f"worst at plane {q}, node ({ii}, {jj}); all regions: {worst}")
    return worst
