"""Planted mistakes in a COPY of the oracle must each fail at least one pin.

Each mutant is a one-expression edit of ``oracle/trtr_oracle.c`` of the kind a plausible
slip would make (a dropped term, a wrong sign, a transposed index, a swapped relaxation
time).  The copy is compiled into a temporary shared object and the whole pin set is run
against it; a mutant that passes every pin would mean the pins cannot see that mistake.
"""
import os
import shutil
import subprocess

import pytest

import oracle

from . import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "trtr_oracle.c")

MUTANTS = {
    "G_sign": ("G[i] = WEIGHT[i] * ea / L->cs2 * (1.0 - 1.0 / (2.0 * tau1)) * phi;",
               "G[i] = -WEIGHT[i] * ea / L->cs2 * (1.0 - 1.0 / (2.0 * tau1)) * phi;"),
    "G_dropped": ("post[q] = post[q] + dt * G[q] + dt * Fn[q] + dtF;",
                  "post[q] = post[q] + dt * Fn[q] + dtF;"),
    "G_grad_transposed": ("adv[a] += u[b] * du[a][b];\n    }\n    for (int i = 0; i < Q; ++i) {\n        double ea = 0.0;",
                          "adv[a] += u[b] * du[b][a];\n    }\n    for (int i = 0; i < Q; ++i) {\n        double ea = 0.0;"),
    "G_tau_factor": ("G[i] = WEIGHT[i] * ea / L->cs2 * (1.0 - 1.0 / (2.0 * tau1)) * phi;",
                     "G[i] = WEIGHT[i] * ea / L->cs2 * (1.0 - 1.0 / tau1) * phi;"),
    "F_first_order_dropped": (
        "F[i] = WEIGHT[i] * S + (1.0 - 1.0 / (2.0 * tau1)) * WEIGHT[i] * eu * S / L->cs2;",
        "F[i] = WEIGHT[i] * S;"),
    "dtF_sign": ("const double dtF = (dt * dt / 2.0) * (Fn[q] - Fnm1[q]) / dt;",
                 "const double dtF = (dt * dt / 2.0) * (Fnm1[q] - Fn[q]) / dt;"),
    "tau2_for_tau1": ("(1.0 - 1.0 / tau2) * WEIGHT[i] * r2 / (2.0 * cs4);",
                      "(1.0 - 1.0 / tau1) * WEIGHT[i] * r2 / (2.0 * cs4);"),
    "second_order_reg_dropped": ("+\n                 (1.0 - 1.0 / tau2) * WEIGHT[i] * r2 / (2.0 * cs4);", ";"),
    "third_order_eq_dropped": ("+ t3 / (6.0 * cs6));", ");"),
    "H2_sign": ("L->H2[i][a][b] = L->e[i][a] * L->e[i][b] - L->cs2 * kron(a, b);",
                "L->H2[i][a][b] = L->e[i][a] * L->e[i][b] + L->cs2 * kron(a, b);"),
    "push_direction": ("post);\n            for (int q = 0; q < Q; ++q) {\n                const int it = ((i + EHAT[q][0]) % nx + nx) % nx;",
                       "post);\n            for (int q = 0; q < Q; ++q) {\n                const int it = ((i - EHAT[q][0]) % nx + nx) % nx;"),
    "adjoint_tau2_chain_dropped": ("acc += mu[q] * (d1[q] + dtau2_dtau1 * d2[q]);", "acc += mu[q] * d1[q];"),
    "adjoint_no_transpose_shift": ("mu[q] = lam[q * n + (size_t)jt * nx + it];", "mu[q] = lam[q * n + k];"),
    "adjoint_jacobian_not_transposed": ("acc += jac[(k * Q + q) * Q + c] * mu[q];",
                                        "acc += jac[(k * Q + c) * Q + q] * mu[q];"),
    "adjoint_dkh": ("dkh = 1.0 / (2.0 * tau1 * tau1)", "dkh = 1.0 / (tau1 * tau1)"),
    "weight_swap": ("static const double WEIGHT[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,\n"
                    "                                 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};",
                    "static const double WEIGHT[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0, 1.0 / 9.0,\n"
                    "                                 1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};"),
    "tau1_cs2_missing": ("return 0.5 + kappa / (L->cs2 * dt);", "return 0.5 + kappa / dt;"),
    "grad_one_sided_wrong": ("du[a][0] = (u[(size_t)j * nx + 1] - u[(size_t)j * nx]) / s->p.dx;",
                             "du[a][0] = (u[(size_t)j * nx + 1] - u[(size_t)j * nx]) / (2.0 * s->p.dx);"),
    "source_prev_time": ("Snm1 = pulse_source(s, x, y, t_nm1); /* closed form",
                         "Snm1 = pulse_source(s, x, y, t_n); /* closed form"),
    "nee_interior_phi_exact": ("equilibrium(&Lat, phif, uf, geqf);",
                               "equilibrium(&Lat, paper_phi(xf, yf, pp->kappa, t1), uf, geqf);"),
    "bounce_back_sign": ("else v = -post[(size_t)OPPOSITE[q] * ny + j] + 2.0 * WEIGHT[q] * phi_w;",
                         "else v = post[(size_t)OPPOSITE[q] * ny + j] + 2.0 * WEIGHT[q] * phi_w;"),
    "bgk_relaxation": ("out[i] = geq[i] + (1.0 - 1.0 / tau) * (g[i] - geq[i]);",
                       "out[i] = geq[i] + (1.0 - 0.5 / tau) * (g[i] - geq[i]);"),
    "traditional_G_factor": ("G[q] = WEIGHT[q] * eu / Lat.cs2 * (1.0 - 1.0 / (2.0 * tau1)) * dphidt;",
                             "G[q] = WEIGHT[q] * eu / Lat.cs2 * dphidt;"),
    "paper_source_sign": ("return (6.0 * kappa - 4.0 * x * y - 4.0 * kappa",
                          "return (6.0 * kappa + 4.0 * x * y - 4.0 * kappa"),
    "source_laplacian_sign": ("return -(dDx * gx + dDy * gy + dD * lap);",
                              "return -(dDx * gx + dDy * gy - dD * lap);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    so = str(tmp_path / "mutant.so")
    oracle.build(force=True, src=str(src), out=so)
    lib = oracle.load(so)
    failed = []
    # the cheap pins first; the convergence pin runs on smaller grids here
    for pin in P.ALL_PINS:
        try:
            if pin is P.pin_second_order_convergence:
                pin(lib, sizes=(32, 64, 128))
            else:
                pin(lib)
        except (AssertionError, FloatingPointError, ValueError):
            failed.append(pin.__name__)
            break
    assert failed, f"mutant {name} passed every pin"


def test_anchor_sanity():
    """The unmutated source contains every anchor exactly once."""
    text = open(SRC).read()
    for name, (old, _) in MUTANTS.items():
        assert text.count(old) == 1, name
