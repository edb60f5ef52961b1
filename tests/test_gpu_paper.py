"""The paper's own benchmark (Sec. 3, Table 2) through the CUDA library: Dirichlet boundaries by
non-equilibrium extrapolation (TRTR_BC_DIRICHLET_NEE), the closed-form source fed as a field
with S^{-1} = S(-dt), against the FP64 oracle node by node and against Table 2's printed RMS
errors.  Also the boundary pass on random states of ragged grids in every storage type."""
import numpy as np
import pytest

import oracle
from paper_2312_10316_gb300 import workloads as W

from . import oracle_pins as P
from ._gpu_util import TOL_F32, TOL_F64, assert_elementwise, random_case, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402

PREC = {"f64": T.TRTR_F64, "f32": T.TRTR_F32, "f16": T.TRTR_F16_OFS, "bf16": T.TRTR_BF16_OFS}


def run_paper(pp: W.PaperPulse, precision: int):
    """Runs the benchmark to pp.steps through the library; returns phi [N + 1][N + 1]."""
    f = W.paper_fields(pp)
    p = T.Params(nx=pp.nx, ny=pp.ny, x0=pp.x0, y0=pp.y0, dx=pp.dx, dt=pp.time_step, precision=precision,
                 grad_mode=T.TRTR_GRAD_ONESIDED_EDGE, src_mode=T.TRTR_SRC_FIELD, bc_mode=T.TRTR_BC_DIRICHLET_NEE)
    with T.Solver(p) as s:
        s.set_fields(f["ux"], f["uy"], f["D"], W.paper_source(pp, 0.0))
        s.init_equilibrium(f["phi0"])
        s.set_source_prev(W.paper_source(pp, -pp.time_step))
        for n in range(pp.steps):
            s.set_dirichlet(W.paper_phi(pp, (n + 1) * pp.time_step))
            s.step(1)
            s.set_source(W.paper_source(pp, (n + 1) * pp.time_step))
        return s.moments()


@pytest.mark.parametrize("N", [20, 40, 100])
def test_paper_benchmark_f64_against_oracle_and_table2(N):
    rows = {(r["kappa"], r["N"]): r for r in P.table2_rows()}
    for kappa in (0.005, 0.01, 0.05):
        pp = W.PaperPulse(N=N, kappa=kappa)
        phi = run_paper(pp, T.TRTR_F64)
        rms_o, blew, phi_o = oracle.paper_pulse(N, kappa, pp.time_step, 0, want_phi=True)
        assert not blew
        assert rel_l2(phi, phi_o) <= TOL_F64
        rms = float(np.sqrt(np.mean((phi - W.paper_phi(pp, pp.steps * pp.time_step)) ** 2)))
        assert abs(rms / rms_o - 1.0) <= 1e-9
        if (kappa, N) != (0.005, 40):  # the printed 3.471e-03 is a digit transposition
            assert abs(rms / rows[(kappa, N)]["present"] - 1.0) <= 1e-3, (kappa, N, rms)


def test_paper_benchmark_f32_table2_column():
    """FP32 storage and arithmetic: phi within 1e-5 of the FP64 oracle, and the RMS error of
    Table 2 within 1 % at N = 100."""
    rows = {(r["kappa"], r["N"]): r for r in P.table2_rows()}
    for kappa in (0.005, 0.01, 0.05):
        pp = W.PaperPulse(N=100, kappa=kappa)
        phi = run_paper(pp, T.TRTR_F32)
        _, _, phi_o = oracle.paper_pulse(100, kappa, pp.time_step, 0, want_phi=True)
        assert rel_l2(phi, phi_o) <= TOL_F32
        rms = float(np.sqrt(np.mean((phi - W.paper_phi(pp, pp.steps * pp.time_step)) ** 2)))
        assert abs(rms / rows[(kappa, 100)]["present"] - 1.0) <= 1e-2


BC_GRIDS = [(3, 3), (4, 7), (37, 23), (130, 9), (129, 40)]
BC_TOL = {"f64": TOL_F64, "f32": TOL_F32, "f16": 2e-3, "bf16": 1.5e-2}


@pytest.mark.parametrize("nx,ny", BC_GRIDS)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_dirichlet_random_states(nx, ny, prec):
    """Random populations, velocities, diffusivities, sources and edge values: three steps with
    a new source and new edge values each step, against the oracle's bc_mode 1."""
    case = random_case(500 + 7 * nx + ny, nx, ny)
    rng = np.random.default_rng(nx * 1000 + ny)
    phi_ref = 1.0 if prec in ("f16", "bf16") else 0.0
    common = dict(nx=nx, ny=ny, dx=case["dx"], dt=case["dt"], x0=-0.3, y0=-0.2, grad_mode=1, src_mode=1)
    o = oracle.Sim(oracle.SimParams(bc_mode=1, **common))
    with T.Solver(T.Params(precision=PREC[prec], phi_ref=phi_ref, bc_mode=T.TRTR_BC_DIRICHLET_NEE, **common)) as s:
        o.set_fields(case["ux"], case["uy"], case["D"])
        s.set_fields(case["ux"], case["uy"], case["D"], case["S1"])
        o.set_source(case["S1"])
        o.set_g(case["g"], step=3)
        s.set_populations(case["g"], step=3)
        o.set_source_prev(case["S2"])
        s.set_source_prev(case["S2"])
        for k in range(3):
            phi_b = rng.uniform(0.5, 1.5, size=(ny, nx))
            o.set_dirichlet(phi_b)
            s.set_dirichlet(phi_b if k % 2 else torch.from_numpy(phi_b).cuda())
            o.step(1)
            s.step(1)
            gp, og = s.get_populations(), o.get_g()
            assert rel_l2(gp, og) <= BC_TOL[prec], (k, prec)
            assert_elementwise(gp, og, BC_TOL[prec], f"step {k} {prec}", tile=(64, 8))
            Sn = rng.uniform(-1.0, 1.0, size=(ny, nx))
            o.set_source(Sn)
            s.set_source(Sn)
        phi = s.moments()
        assert rel_l2(phi, o.phi()) <= BC_TOL[prec]
        assert_elementwise(phi, o.phi(), BC_TOL[prec], "phi", tile=(64, 8))
        # the edge nodes hold the imposed values exactly (up to storage rounding)
        edge = np.zeros((ny, nx), dtype=bool)
        edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
        tol = {"f64": 1e-13, "f32": 1e-5, "f16": 5e-3, "bf16": 4e-2}[prec]
        assert np.abs(phi[edge] - phi_b[edge]).max() <= tol


def test_dirichlet_needs_values_and_excludes_the_adjoint():
    case = random_case(3, 16, 16)
    p = T.Params(nx=16, ny=16, dx=case["dx"], dt=case["dt"], precision=T.TRTR_F64, bc_mode=T.TRTR_BC_DIRICHLET_NEE)
    with T.Solver(p) as s:
        s.set_fields(case["ux"], case["uy"], case["D"])
        s.init_equilibrium(np.ones((16, 16)))
        with pytest.raises(T.TrtrError) as e:
            s.step(1)
        assert e.value.status == T.TRTR_ESTATE
        s.set_dirichlet(np.ones((16, 16)))
        with pytest.raises(T.TrtrError) as e:
            s.forward_record(4)
        assert e.value.status == T.TRTR_EINVAL
        # uniform phi, uniform edge values, u = 0 and S = 0 stay a fixed point
        s.set_fields(np.zeros((16, 16)), np.zeros((16, 16)), case["D"])
        s.init_equilibrium(np.ones((16, 16)))
        s.step(5)
        assert np.abs(s.moments() - 1.0).max() <= 1e-14
    with T.Solver(T.Params(nx=16, ny=16, dx=case["dx"], dt=case["dt"], precision=T.TRTR_F64)) as s:
        with pytest.raises(T.TrtrError) as e:
            s.set_dirichlet(np.ones((16, 16)))
        assert e.value.status == T.TRTR_EINVAL
