"""The spatial decomposition a multi-GPU solve would use, emulated on CPU ranks (gloo).

The domain is split into y-slabs that span the full width, one per rank.  A rank owning
rows [a, b) steps an extended slab of rows [a - 1, b + 1) (one ghost row on each side,
periodic inside the slab) with the FP64 oracle.  The streaming of Eq. (14) moves a node's
post-collision populations to x + e_i, so after a step only the populations with e_y = +1
at row a and those with e_y = -1 at row b - 1 are wrong: they came from the rank's own
ghost rows.  The right values sit in the neighbours' ghost rows (the rank below pushed its
top row's upward populations into its ghost row b, the rank above its bottom row's
downward ones into its ghost row a - 1), so one exchange of three populations per edge
node per side and step makes every owned node equal to the single-domain result.  The
velocity rows that the gradient of the auxiliary term (Eq. (16)) reads across a slab edge
are exchanged once, before the first step.  The ghost populations and ghost sources are
NaN throughout, so any use of ghost state by an owned node would show.  Mass
(the sum of all populations) is reduced over ranks in FP64.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

# Oracle population order: e_3 = (0, 1), e_5 = (1, 1), e_8 = (-1, 1); e_4, e_6, e_7 their opposites.
UP = [3, 5, 8]
DOWN = [4, 6, 7]
TAG_UP, TAG_DOWN, TAG_FIELD = 1, 2, 3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def slab_rows(ny: int, world: int):
    """Row ranges [a, b) of the y-slabs, the first ny % world slabs one row taller."""
    base, extra = divmod(ny, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def global_case(seed: int, nx: int, ny: int, steps: int):
    """Seeded inputs of the whole domain, FP64: populations, u, D, and one source per step."""
    from paper_2312_10316_gb300 import workloads as W

    rng = np.random.default_rng(seed)
    dx, dt = 0.1, 0.02
    c = dx / dt
    g = W.random_populations(seed, ny, nx, base=1.0, amp=0.3)
    ux = c * rng.uniform(-0.2, 0.2, size=(ny, nx))
    uy = c * rng.uniform(-0.2, 0.2, size=(ny, nx))
    tau1 = rng.uniform(0.55, 1.5, size=(ny, nx))
    D = (tau1 - 0.5) * (c * c / 3.0) * dt
    S = [rng.uniform(-1.0, 1.0, size=(ny, nx)) for _ in range(steps + 2)]  # S^{-1}, S^0, ..., S^steps
    return dict(g=g, ux=ux, uy=uy, D=D, S=S, dx=dx, dt=dt)


def _params(nx, ny, case):
    import oracle

    return oracle.SimParams(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], grad_mode=0, src_mode=1)


def _exchange(send_up, send_down, prev, nxt):
    """Sends the top ghost row's upward populations to the next rank and the bottom ghost
    row's downward ones to the previous rank; returns what arrives from the neighbours."""
    recv_up = torch.empty_like(send_up)
    recv_down = torch.empty_like(send_down)
    reqs = [dist.isend(send_up, nxt, tag=TAG_UP), dist.isend(send_down, prev, tag=TAG_DOWN),
            dist.irecv(recv_up, prev, tag=TAG_UP), dist.irecv(recv_down, nxt, tag=TAG_DOWN)]
    for q in reqs:
        q.wait()
    return recv_up, recv_down


def _ghost_fields(own, prev, nxt):
    """The velocity and diffusivity rows just outside the slab, from the neighbours (once)."""
    below = torch.empty_like(own[:, 0])
    above = torch.empty_like(own[:, -1])
    reqs = [dist.isend(own[:, -1].contiguous(), nxt, tag=TAG_FIELD),
            dist.isend(own[:, 0].contiguous(), prev, tag=TAG_FIELD + 1),
            dist.irecv(below, prev, tag=TAG_FIELD), dist.irecv(above, nxt, tag=TAG_FIELD + 1)]
    for q in reqs:
        q.wait()
    return below, above


def run_slab(rank, world, nx, ny, seed, steps, exchange=True):
    """Steps this rank's slab; returns (owned phi, owned populations, mass over all ranks)."""
    import oracle

    case = global_case(seed, nx, ny, steps)
    a, b = slab_rows(ny, world)[rank]
    h = b - a
    prev, nxt = (rank - 1) % world, (rank + 1) % world

    # owned rows of the static fields; the ghost rows come from the neighbours
    own = torch.from_numpy(np.stack([case["ux"][a:b], case["uy"][a:b], case["D"][a:b]]).copy())
    below, above = _ghost_fields(own, prev, nxt)
    fields = torch.cat([below[:, None], own, above[:, None]], dim=1).numpy()

    def ext(field):  # owned rows of a per-node field, NaN in the ghost rows
        out = np.full((h + 2, nx), np.nan)
        out[1:h + 1] = field[a:b]
        return out

    g = np.full((9, h + 2, nx), np.nan)
    g[:, 1:h + 1] = case["g"][:, a:b]
    S = case["S"]
    sim = oracle.Sim(_params(nx, h + 2, case))
    sim.set_fields(fields[0], fields[1], fields[2])
    sim.set_g(g, step=0)
    sim.set_source_prev(ext(S[0]))
    sim.set_source(ext(S[1]))
    for n in range(steps):
        sim.step(1)
        g = sim.get_g()
        if exchange:
            up, down = _exchange(torch.from_numpy(g[UP, h + 1].copy()), torch.from_numpy(g[DOWN, 0].copy()), prev, nxt)
            g[UP, 1] = up.numpy()
            g[DOWN, h] = down.numpy()
        g[:, 0] = np.nan
        g[:, h + 1] = np.nan
        sim.set_g(g, step=n + 1)  # resets S^{n-1}; restored below
        sim.set_source_prev(ext(S[n + 1]))
        sim.set_source(ext(S[n + 2]))
    g = sim.get_g()[:, 1:h + 1]
    sim.close()
    mass = torch.tensor([float(np.sum(g))], dtype=torch.float64)
    dist.all_reduce(mass)
    return g.sum(axis=0), g, float(mass[0])


def _exchange_rows(rows_up, rows_down, prev, nxt, tag):
    """Sends rows_up (this slab's top owned rows) to the next rank and rows_down (its bottom owned
    rows) to the previous one; returns (rows from the previous rank, rows from the next)."""
    from_prev = torch.empty_like(rows_up)
    from_next = torch.empty_like(rows_down)
    reqs = [dist.isend(rows_up, nxt, tag=tag), dist.isend(rows_down, prev, tag=tag + 1),
            dist.irecv(from_prev, prev, tag=tag), dist.irecv(from_next, nxt, tag=tag + 1)]
    for q in reqs:
        q.wait()
    return from_prev, from_next


def run_slab_two(rank, world, nx, ny, seed, steps):
    """Two steps per exchange (the two-step kernel's tile logic across ranks).  A slab of rows
    [a, b) steps an extended slab [a - 3, b + 3) twice between exchanges.  Before each pair the
    two ghost rows next to the slab on each side receive the neighbours' full pre-collision
    state; the third ghost row holds no state (NaN), only the velocity and D rows that the
    second ghost row's gradient of the auxiliary term reads (exchanged once, like the packed
    acceleration field of the two-step kernel).  After two steps the owned rows are exact: an
    owned row's second step reads first-step values of the rows up to one outside the slab,
    and those read the exchanged rows and their exact collisions."""
    import oracle

    case = global_case(seed, nx, ny, steps)
    a, b = slab_rows(ny, world)[rank]
    h = b - a
    assert h >= 3 and steps % 2 == 0
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    own = torch.from_numpy(np.stack([case["ux"][a:b], case["uy"][a:b], case["D"][a:b]]).copy())
    below, above = _exchange_rows(own[:, -3:].contiguous(), own[:, :3].contiguous(), prev, nxt, TAG_FIELD)
    fields = torch.cat([below, own, above], dim=1).numpy()

    def ext(field):  # a per-node field over the extended rows (the sources are local inputs)
        return np.take(field, np.arange(a - 3, b + 3) % ny, axis=0)

    S = case["S"]
    sim = oracle.Sim(_params(nx, h + 6, case))
    sim.set_fields(fields[0], fields[1], fields[2])
    g = np.full((9, h + 6, nx), np.nan)
    g[:, 3:h + 3] = case["g"][:, a:b]
    for n in range(0, steps, 2):
        top, bottom = _exchange_rows(torch.from_numpy(g[:, h + 1:h + 3].copy()),
                                     torch.from_numpy(g[:, 3:5].copy()), prev, nxt, TAG_UP)
        g[:, 1:3] = top.numpy()             # the previous rank's top two owned rows
        g[:, h + 3:h + 5] = bottom.numpy()  # the next rank's bottom two owned rows
        sim.set_g(g, step=n)
        sim.set_source_prev(ext(S[n]))
        sim.set_source(ext(S[n + 1]))
        sim.step(1)
        sim.set_source(ext(S[n + 2]))
        sim.step(1)
        g = sim.get_g()
        g[:, :3] = np.nan
        g[:, h + 3:] = np.nan
    sim.close()
    return g[:, 3:h + 3]


def run_global(nx, ny, seed, steps):
    import oracle

    case = global_case(seed, nx, ny, steps)
    S = case["S"]
    sim = oracle.Sim(_params(nx, ny, case))
    sim.set_fields(case["ux"], case["uy"], case["D"])
    sim.set_g(case["g"], step=0)
    sim.set_source_prev(S[0])
    sim.set_source(S[1])
    for n in range(steps):
        sim.step(1)
        sim.set_source(S[n + 2])
    out = sim.phi(), sim.get_g(), sim.mass()
    sim.close()
    return out


def _worker(rank, world, port, nx, ny, seed, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        phi, g, mass = run_slab(rank, world, nx, ny, seed, steps)
        phi_x, _, _ = run_slab(rank, world, nx, ny, seed, steps, exchange=False)
        thin = min(b - a for a, b in slab_rows(ny, world)) < 3  # too thin for two steps per exchange
        g2 = None if thin else run_slab_two(rank, world, nx, ny, seed, steps - steps % 2)
        q.put((rank, phi, g, mass, phi_x, g2))
    finally:
        dist.destroy_process_group()


def test_slab_rows_cover_the_domain():
    for ny in (1, 5, 29, 64):
        for world in range(1, min(ny, 5) + 1):
            rows = slab_rows(ny, world)
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(r0[1] == r1[0] for r0, r1 in zip(rows, rows[1:]))
            assert max(b - a for a, b in rows) - min(b - a for a, b in rows) <= 1


@pytest.mark.parametrize("world,nx,ny,steps", [(2, 37, 29, 6), (3, 16, 10, 5), (3, 16, 5, 5)])
def test_slabs_equal_the_single_domain_oracle_bitwise(world, nx, ny, steps):
    """One exchange per step (three populations per edge node and side), and one per two steps
    (two full rows per side).  (3, 16, 10) gives slabs of 4, 3 and 3 rows; (3, 16, 5) slabs of 2,
    2 and 1 rows, where a one-row slab receives both halos (one step per exchange only)."""
    seed = 1000 + nx + ny
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nx, ny, seed, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    phi_ref, g_ref, mass_ref = run_global(nx, ny, seed, steps)
    _, g_ref2, _ = run_global(nx, ny, seed, steps - steps % 2)
    rows = slab_rows(ny, world)
    for (rank, phi, g, mass, phi_x, g2), (a, b) in zip(results, rows):
        if g2 is not None:
            assert np.array_equal(g2, g_ref2[:, a:b]), rank
        assert np.array_equal(g, g_ref[:, a:b]), rank
        assert np.array_equal(phi, g_ref[:, a:b].sum(axis=0)), rank
        assert np.allclose(phi, phi_ref[a:b], rtol=0, atol=1e-13)
        assert abs(mass / mass_ref - 1.0) <= 1e-13
        # without the exchange the edge rows take the (NaN) ghost state
        assert np.isnan(phi_x[0]).all() and np.isnan(phi_x[-1]).all()
