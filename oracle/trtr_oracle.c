/*
 * trtr_oracle.c -- plain FP64 CPU oracle of the TRT-R lattice Boltzmann step for the
 * convection-diffusion equation with variable coefficients (Yu, Qin, Yuan, Shu,
 * arXiv 2312.10316).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file: only the tests, the smoke check and the CPU-baseline leg of the benchmark use
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Structure: the evolution equation is written out literally, in the paper's notation
 * and PHYSICAL units (e_i = c*ehat_i, c_s^2 = c^2/3, u in length/time, kappa in
 * length^2/time), with explicit Hermite tensors and explicit tensor contractions:
 *
 *   g_i(x + e_i dt, t + dt) = g_i^eq + (1 - 1/tau1) w_i H_ia B_a^neq / cs^2
 *                           + (1 - 1/tau2) w_i H_iab B_ab^neq / (2 cs^4)
 *                           + dt G_i + dt F_i + dt^2/2 d_t F_i              Eq. (14) [eq_ev]
 *
 * and streaming is done by PUSHING the post-collision value to x + e_i dt, the form the
 * left-hand side of Eq. (14) states.  The stored state is the pre-collision population
 * g_i(x, t_n).
 *
 * Equation numbers count the paper's displayed equations in order; the LaTeX label is
 * given in brackets.  Readings of points the paper leaves open:
 *  - d_beta u_alpha in G_i (Eq. (16) [eq_aux_new]) is a second-order central difference of
 *    the nodal u field; mode 1 uses the one-sided two-point difference on the first and
 *    last column/row instead of wrapping (both are exact for a linear u).
 *  - dt^2/2 d_t F_i is (dt^2/2)(F_i^n - F_i^{n-1})/dt.  A closed-form source (the built-in pulse,
 *    the Sec. 3 benchmark) gives S^{n-1} = S(t_n - dt) at the first step too (Table 2's printed
 *    errors agree with this to their last digit); a source field without a predecessor takes
 *    F^{-1} := F^0 at the first step
 *    after initialisation (u is time-independent within a step, Sec. 2.3).
 *  - phi = sum_i g_i of the pre-collision populations (B_0^neq = 0, Sec. 2.2).
 *  - tau1 from kappa = (tau1 - 1/2) c_s^2 dt (Sec. 2.4), per node from D(x); tau2 from the
 *    magic parameter Lambda = (tau1 - 1/2)(tau2 - 1/2) (Eq. (28)) or given.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared [-fopenmp] trtr_oracle.c -lm
 * (-ffp-contract=off: every product and sum rounds as written).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define PI 3.14159265358979323846

/* D2Q9 (Sec. 2.2): e_0 = (0,0), (+-c,0), (0,+-c), (+-c,+-c); w_0 = 4/9, w_1..4 = 1/9,
 * w_5..8 = 1/36.  Index order (shared convention of this project, not the paper's):
 * 0:(0,0) 1:(1,0) 2:(-1,0) 3:(0,1) 4:(0,-1) 5:(1,1) 6:(-1,-1) 7:(1,-1) 8:(-1,1). */
static const int EHAT[Q][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1},
                               {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
static const double WEIGHT[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPPOSITE[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7}; /* e_OPPOSITE[i] = -e_i */

typedef struct {
    int nx, ny;
    double x0, y0, dx, dt;
    int tau2_mode;      /* 0: magic parameter, 1: fixed tau2 */
    double magic, tau2; /* Lambda (Eq. (28)); fixed tau2 */
    double tau1_const;  /* > 0: tau1 given directly, D ignored */
    int grad_mode;      /* 0: periodic central differences, 1: one-sided at the edges */
    int src_mode;       /* 0: S = 0, 1: given field, 2: manufactured pulse source */
    double omega, xc, yc, sigma0, D0, D_amp; /* pulse parameters (src_mode 2) */
    int bc_mode;        /* 0: periodic, 1: Dirichlet by non-equilibrium extrapolation (Sec. 3) */
} oracle_params;

/* Lattice constants and Hermite tensors in physical units (Sec. 2.2, text after Eq. (10)):
 * H0 = 1, H_a = e_a, H_ab = e_a e_b - cs^2 d_ab,
 * H_abg = e_a e_b e_g - cs^2 (e_a d_bg + e_b d_ga + e_g d_ab). */
typedef struct {
    double c, cs2;
    double e[Q][2];
    double H1[Q][2];
    double H2[Q][2][2];
    double H3[Q][2][2][2];
} oracle_lattice;

static double kron(int a, int b) { return a == b ? 1.0 : 0.0; }

static void lattice_init(oracle_lattice* L, double dx, double dt) {
    L->c = dx / dt;
    L->cs2 = L->c * L->c / 3.0;
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 2; ++a) L->e[i][a] = L->c * (double)EHAT[i][a];
        for (int a = 0; a < 2; ++a) {
            L->H1[i][a] = L->e[i][a];
            for (int b = 0; b < 2; ++b) {
                L->H2[i][a][b] = L->e[i][a] * L->e[i][b] - L->cs2 * kron(a, b);
                for (int g = 0; g < 2; ++g)
                    L->H3[i][a][b][g] = L->e[i][a] * L->e[i][b] * L->e[i][g] -
                                        L->cs2 * (L->e[i][a] * kron(b, g) + L->e[i][b] * kron(g, a) +
                                                  L->e[i][g] * kron(a, b));
            }
        }
    }
}

/* Third-order Hermite equilibrium, Eq. (6):
 * g_i^eq = w_i phi { H0 + H_a u_a / cs^2 + H_ab u_a u_b / (2 cs^4) + H_abg u_a u_b u_g / (6 cs^6) } */
static void equilibrium(const oracle_lattice* L, double phi, const double u[2], double geq[Q]) {
    const double cs2 = L->cs2, cs4 = cs2 * cs2, cs6 = cs4 * cs2;
    for (int i = 0; i < Q; ++i) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int a = 0; a < 2; ++a) {
            t1 += L->H1[i][a] * u[a];
            for (int b = 0; b < 2; ++b) {
                t2 += L->H2[i][a][b] * u[a] * u[b];
                for (int g = 0; g < 2; ++g) t3 += L->H3[i][a][b][g] * u[a] * u[b] * u[g];
            }
        }
        geq[i] = WEIGHT[i] * phi * (1.0 + t1 / cs2 + t2 / (2.0 * cs4) + t3 / (6.0 * cs6));
    }
}

/* TRT-R collision operator, Eq. (12) [eq11], with
 *   g_i^neq = g_i - g_i^eq                     Eq. (5)
 *   B_a^neq  = sum_i H_ia  g_i^neq            Eq. (8)
 *   B_ab^neq = sum_i H_iab (g_i - g_i^eq)     Eq. (13)
 *   phi = sum_i g_i                            (B_0^neq = 0, text after Eq. (10)) */
static void collide_trtr(const oracle_lattice* L, const double g[Q], const double u[2], double tau1,
                         double tau2, double out[Q], double* phi_out) {
    const double cs2 = L->cs2, cs4 = cs2 * cs2;
    double phi = 0.0;
    for (int i = 0; i < Q; ++i) phi += g[i];
    double geq[Q], gneq[Q];
    equilibrium(L, phi, u, geq);
    for (int i = 0; i < Q; ++i) gneq[i] = g[i] - geq[i];
    double B1[2] = {0.0, 0.0};
    double B2[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 2; ++a) {
            B1[a] += L->H1[i][a] * gneq[i];
            for (int b = 0; b < 2; ++b) B2[a][b] += L->H2[i][a][b] * gneq[i];
        }
    for (int i = 0; i < Q; ++i) {
        double r1 = 0.0, r2 = 0.0;
        for (int a = 0; a < 2; ++a) {
            r1 += L->H1[i][a] * B1[a];
            for (int b = 0; b < 2; ++b) r2 += L->H2[i][a][b] * B2[a][b];
        }
        out[i] = geq[i] + (1.0 - 1.0 / tau1) * WEIGHT[i] * r1 / cs2 +
                 (1.0 - 1.0 / tau2) * WEIGHT[i] * r2 / (2.0 * cs4);
    }
    if (phi_out) *phi_out = phi;
}

/* New space-derivative auxiliary term, Eq. (16) [eq_aux_new]:
 *   G_i = w_i e_ia / cs^2 (1 - 1/(2 tau1)) phi u_b d_b u_a,   du[a][b] = d_b u_a */
static void aux_G(const oracle_lattice* L, double phi, const double u[2], const double du[2][2],
                  double tau1, double G[Q]) {
    double adv[2];
    for (int a = 0; a < 2; ++a) {
        adv[a] = 0.0;
        for (int b = 0; b < 2; ++b) adv[a] += u[b] * du[a][b];
    }
    for (int i = 0; i < Q; ++i) {
        double ea = 0.0;
        for (int a = 0; a < 2; ++a) ea += L->e[i][a] * adv[a];
        G[i] = WEIGHT[i] * ea / L->cs2 * (1.0 - 1.0 / (2.0 * tau1)) * phi;
    }
}

/* First-order discrete-velocity source term, Eq. (3) [eq_Fi]:
 *   F_i = w_i S + (1 - 1/(2 tau1)) w_i e_ia u_a S / cs^2 */
static void source_F(const oracle_lattice* L, double S, const double u[2], double tau1, double F[Q]) {
    for (int i = 0; i < Q; ++i) {
        double eu = 0.0;
        for (int a = 0; a < 2; ++a) eu += L->e[i][a] * u[a];
        F[i] = WEIGHT[i] * S + (1.0 - 1.0 / (2.0 * tau1)) * WEIGHT[i] * eu * S / L->cs2;
    }
}

/* kappa = (tau1 - 1/2) cs^2 dt (Sec. 2.4, after Eq. (27)) solved for tau1. */
static double tau1_from_kappa(const oracle_lattice* L, double kappa, double dt) {
    return 0.5 + kappa / (L->cs2 * dt);
}

/* Lambda = (tau1 - 1/2)(tau2 - 1/2), Eq. (28), solved for tau2. */
static double tau2_from_magic(double tau1, double magic) { return 0.5 + magic / (tau1 - 0.5); }

/* ------------------------------------------------------------------------------------ */
/* Single-node entry points (used by the pins on their own).                            */

void oracle_equilibrium(double dx, double dt, double phi, double ux, double uy, double* geq) {
    oracle_lattice L;
    lattice_init(&L, dx, dt);
    const double u[2] = {ux, uy};
    equilibrium(&L, phi, u, geq);
}

void oracle_collide(double dx, double dt, const double* g, double ux, double uy, double tau1, double tau2,
                    double* out) {
    oracle_lattice L;
    lattice_init(&L, dx, dt);
    const double u[2] = {ux, uy};
    collide_trtr(&L, g, u, tau1, tau2, out, NULL);
}

/* du = {d_x u_x, d_y u_x, d_x u_y, d_y u_y} */
void oracle_aux_G(double dx, double dt, double phi, double ux, double uy, const double* du, double tau1,
                  double* G) {
    oracle_lattice L;
    lattice_init(&L, dx, dt);
    const double u[2] = {ux, uy};
    const double d[2][2] = {{du[0], du[1]}, {du[2], du[3]}};
    aux_G(&L, phi, u, d, tau1, G);
}

void oracle_source_F(double dx, double dt, double S, double ux, double uy, double tau1, double* F) {
    oracle_lattice L;
    lattice_init(&L, dx, dt);
    const double u[2] = {ux, uy};
    source_F(&L, S, u, tau1, F);
}

double oracle_tau1(double D, double dx, double dt) {
    oracle_lattice L;
    lattice_init(&L, dx, dt);
    return tau1_from_kappa(&L, D, dt);
}

double oracle_tau2_magic(double tau1, double magic) { return tau2_from_magic(tau1, magic); }

void oracle_d2q9(int* ex, int* ey, double* w) {
    for (int i = 0; i < Q; ++i) {
        ex[i] = EHAT[i][0];
        ey[i] = EHAT[i][1];
        w[i] = WEIGHT[i];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Grid simulation.                                                                     */

typedef struct {
    oracle_params p;
    oracle_lattice L;
    size_t n;                  /* nx * ny */
    double *g, *gnext;         /* [Q][ny][nx] pre-collision populations g_i(x, t_n) */
    double *ux, *uy, *D;       /* physical fields */
    double *S_cur, *S_prev;    /* src_mode 1: S used at this step and at the previous one */
    int S_prev_valid;          /* 0 right after init: F^{-1} := F^0 */
    double* phi_b;             /* bc_mode 1: Dirichlet values; only the edge nodes are read */
    long step;
} oracle_sim;

#define AT(s, q, j, i) ((size_t)(q) * (s)->n + (size_t)(j) * (size_t)(s)->p.nx + (size_t)(i))

oracle_sim* oracle_create(const oracle_params* p) {
    if (p->nx < 1 || p->ny < 1 || !(p->dx > 0.0) || !(p->dt > 0.0)) return NULL;
    if (p->bc_mode == 1 && (p->nx < 3 || p->ny < 3)) return NULL;
    oracle_sim* s = (oracle_sim*)calloc(1, sizeof(oracle_sim));
    if (!s) return NULL;
    s->p = *p;
    lattice_init(&s->L, p->dx, p->dt);
    s->n = (size_t)p->nx * (size_t)p->ny;
    s->g = (double*)calloc(Q * s->n, sizeof(double));
    s->gnext = (double*)calloc(Q * s->n, sizeof(double));
    s->ux = (double*)calloc(s->n, sizeof(double));
    s->uy = (double*)calloc(s->n, sizeof(double));
    s->D = (double*)calloc(s->n, sizeof(double));
    s->S_cur = (double*)calloc(s->n, sizeof(double));
    s->S_prev = (double*)calloc(s->n, sizeof(double));
    s->phi_b = (double*)calloc(s->n, sizeof(double));
    if (!s->g || !s->gnext || !s->ux || !s->uy || !s->D || !s->S_cur || !s->S_prev || !s->phi_b) {
        free(s->g); free(s->gnext); free(s->ux); free(s->uy); free(s->D); free(s->S_cur); free(s->S_prev);
        free(s->phi_b);
        free(s);
        return NULL;
    }
    return s;
}

void oracle_destroy(oracle_sim* s) {
    if (!s) return;
    free(s->g); free(s->gnext); free(s->ux); free(s->uy); free(s->D); free(s->S_cur); free(s->S_prev);
    free(s->phi_b);
    free(s);
}

/* Physical fields u_x, u_y, D (= kappa) on the nodes, row-major [ny][nx]. */
void oracle_set_fields(oracle_sim* s, const double* ux, const double* uy, const double* D) {
    memcpy(s->ux, ux, s->n * sizeof(double));
    memcpy(s->uy, uy, s->n * sizeof(double));
    memcpy(s->D, D, s->n * sizeof(double));
}

/* src_mode 1: S for the next step.  The previous step's S stays as S^{n-1}. */
void oracle_set_source(oracle_sim* s, const double* S) { memcpy(s->S_cur, S, s->n * sizeof(double)); }

/* src_mode 1: S^{n-1} for the next step (a closed-form source known at t_n - dt). */
void oracle_set_source_prev(oracle_sim* s, const double* S) {
    memcpy(s->S_prev, S, s->n * sizeof(double));
    s->S_prev_valid = 1;
}

/* bc_mode 1: the Dirichlet values phi_b(x) imposed after the next step's streaming ([ny][nx];
 * only the edge nodes are read). */
void oracle_set_dirichlet(oracle_sim* s, const double* phi_b) { memcpy(s->phi_b, phi_b, s->n * sizeof(double)); }

static double node_x(const oracle_sim* s, int i) { return s->p.x0 + (double)i * s->p.dx; }
static double node_y(const oracle_sim* s, int j) { return s->p.y0 + (double)j * s->p.dx; }

/* Manufactured source of the rotating, spreading Gaussian pulse with
 * D(x) = D0 (1 + D_amp sin(pi x) sin(pi y)):  phi_a = (s0^2/s^2) exp(-|x - c(t)|^2 / (2 s^2)),
 * s^2 = s0^2 + 2 D0 t, c(t) = R(omega t)(xc, yc), solves the constant-D0 equation (1) with
 * u = omega(-y, x); S = -div((D - D0) grad phi_a) makes it solve the variable-D one. */
static double pulse_source(const oracle_sim* s, double x, double y, double t) {
    const oracle_params* p = &s->p;
    const double cx = p->xc * cos(p->omega * t) - p->yc * sin(p->omega * t);
    const double cy = p->xc * sin(p->omega * t) + p->yc * cos(p->omega * t);
    const double s2 = p->sigma0 * p->sigma0 + 2.0 * p->D0 * t;
    const double rx = x - cx, ry = y - cy, r2 = rx * rx + ry * ry;
    const double phia = p->sigma0 * p->sigma0 / s2 * exp(-r2 / (2.0 * s2));
    const double gx = -rx / s2 * phia, gy = -ry / s2 * phia;       /* grad phi_a */
    const double lap = (r2 / (s2 * s2) - 2.0 / s2) * phia;          /* laplacian phi_a */
    const double dD = p->D0 * p->D_amp * sin(PI * x) * sin(PI * y); /* D - D0 */
    const double dDx = p->D0 * p->D_amp * PI * cos(PI * x) * sin(PI * y);
    const double dDy = p->D0 * p->D_amp * PI * sin(PI * x) * cos(PI * y);
    return -(dDx * gx + dDy * gy + dD * lap);
}

void oracle_pulse_source(const oracle_sim* s, double t, double* out) {
    for (int j = 0; j < s->p.ny; ++j)
        for (int i = 0; i < s->p.nx; ++i)
            out[(size_t)j * s->p.nx + i] = pulse_source(s, node_x(s, i), node_y(s, j), t);
}

/* Initial condition g_i = g_i^eq(phi_0, u) (Sec. 3). */
void oracle_init_equilibrium(oracle_sim* s, const double* phi0) {
    for (int j = 0; j < s->p.ny; ++j)
        for (int i = 0; i < s->p.nx; ++i) {
            const size_t k = (size_t)j * s->p.nx + i;
            const double u[2] = {s->ux[k], s->uy[k]};
            double geq[Q];
            equilibrium(&s->L, phi0[k], u, geq);
            for (int q = 0; q < Q; ++q) s->g[AT(s, q, j, i)] = geq[q];
        }
    s->step = 0;
    s->S_prev_valid = 0;
}

/* d_b u_a at node (i, j): du[a][b]. */
static void grad_u(const oracle_sim* s, int i, int j, double du[2][2]) {
    const int nx = s->p.nx, ny = s->p.ny;
    const double* f[2] = {s->ux, s->uy};
    for (int a = 0; a < 2; ++a) {
        const double* u = f[a];
        /* x derivative */
        if (nx == 1) {
            du[a][0] = 0.0;
        } else if (s->p.grad_mode == 1 && i == 0) {
            du[a][0] = (u[(size_t)j * nx + 1] - u[(size_t)j * nx]) / s->p.dx;
        } else if (s->p.grad_mode == 1 && i == nx - 1) {
            du[a][0] = (u[(size_t)j * nx + i] - u[(size_t)j * nx + i - 1]) / s->p.dx;
        } else {
            const int ip = (i + 1) % nx, im = (i - 1 + nx) % nx;
            du[a][0] = (u[(size_t)j * nx + ip] - u[(size_t)j * nx + im]) / (2.0 * s->p.dx);
        }
        /* y derivative */
        if (ny == 1) {
            du[a][1] = 0.0;
        } else if (s->p.grad_mode == 1 && j == 0) {
            du[a][1] = (u[(size_t)nx + i] - u[i]) / s->p.dx;
        } else if (s->p.grad_mode == 1 && j == ny - 1) {
            du[a][1] = (u[(size_t)j * nx + i] - u[(size_t)(j - 1) * nx + i]) / s->p.dx;
        } else {
            const int jp = (j + 1) % ny, jm = (j - 1 + ny) % ny;
            du[a][1] = (u[(size_t)jp * nx + i] - u[(size_t)jm * nx + i]) / (2.0 * s->p.dx);
        }
    }
}

static void node_taus(const oracle_sim* s, size_t k, double* tau1, double* tau2) {
    *tau1 = s->p.tau1_const > 0.0 ? s->p.tau1_const : tau1_from_kappa(&s->L, s->D[k], s->p.dt);
    *tau2 = s->p.tau2_mode == 1 ? s->p.tau2 : tau2_from_magic(*tau1, s->p.magic);
}

/* Right-hand side of Eq. (14) at one node: TRT-R collision, + dt G_i + dt F_i
 * + dt^2/2 d_t F_i, with d_t F_i = (F_i^n - F_i^{n-1}) / dt. */
static void node_post(const oracle_lattice* L, double dt, const double g[Q], const double u[2],
                      const double du[2][2], double tau1, double tau2, double Sn, double Snm1, double post[Q]) {
    double G[Q], Fn[Q], Fnm1[Q], phi;
    collide_trtr(L, g, u, tau1, tau2, post, &phi);
    aux_G(L, phi, u, du, tau1, G);
    source_F(L, Sn, u, tau1, Fn);
    source_F(L, Snm1, u, tau1, Fnm1);
    for (int q = 0; q < Q; ++q) {
        const double dtF = (dt * dt / 2.0) * (Fn[q] - Fnm1[q]) / dt; /* dt^2/2 d_t F_i */
        post[q] = post[q] + dt * G[q] + dt * Fn[q] + dtF;
    }
}

/* One time step over rows [j0, j1): collide each node, then push the post-collision value
 * to x + e_i dt (periodic), Eq. (14). */
static void step_rows(oracle_sim* s, int j0, int j1, double t_n, double t_nm1) {
    const int nx = s->p.nx, ny = s->p.ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = j0; j < j1; ++j) {
        for (int i = 0; i < nx; ++i) {
            const size_t k = (size_t)j * nx + i;
            double g[Q], post[Q];
            for (int q = 0; q < Q; ++q) g[q] = s->g[AT(s, q, j, i)];
            const double u[2] = {s->ux[k], s->uy[k]};
            double tau1, tau2;
            node_taus(s, k, &tau1, &tau2);
            double du[2][2];
            grad_u(s, i, j, du);

            double Sn = 0.0, Snm1 = 0.0;
            if (s->p.src_mode == 1) {
                Sn = s->S_cur[k];
                Snm1 = s->S_prev_valid ? s->S_prev[k] : Sn;
            } else if (s->p.src_mode == 2) {
                const double x = node_x(s, i), y = node_y(s, j);
                Sn = pulse_source(s, x, y, t_n);
                Snm1 = pulse_source(s, x, y, t_nm1); /* closed form: S(t_{-1}) at the first step too */
            }
            node_post(&s->L, s->p.dt, g, u, du, tau1, tau2, Sn, Snm1, post);
            for (int q = 0; q < Q; ++q) {
                const int it = ((i + EHAT[q][0]) % nx + nx) % nx;
                const int jt = ((j + EHAT[q][1]) % ny + ny) % ny;
                s->gnext[AT(s, q, jt, it)] = post[q];
            }
        }
    }
}

/* Single-node right-hand side of Eq. (14) for sampled checks: g (pre-collision), physical u,
 * du = {d_x u_x, d_y u_x, d_x u_y, d_y u_y}, kappa = D, S^n, S^{n-1}; tau rules from p. */
void oracle_node_post(const oracle_params* p, const double* g, double ux, double uy, const double* du, double D,
                      double Sn, double Snm1, double* post) {
    oracle_lattice L;
    lattice_init(&L, p->dx, p->dt);
    const double u[2] = {ux, uy};
    const double d[2][2] = {{du[0], du[1]}, {du[2], du[3]}};
    const double tau1 = p->tau1_const > 0.0 ? p->tau1_const : tau1_from_kappa(&L, D, p->dt);
    const double tau2 = p->tau2_mode == 1 ? p->tau2 : tau2_from_magic(tau1, p->magic);
    node_post(&L, p->dt, g, u, d, tau1, tau2, Sn, Snm1, post);
}

/* Manufactured pulse source at one point (src_mode 2 closed form). */
double oracle_pulse_source_at(const oracle_sim* s, double x, double y, double t) { return pulse_source(s, x, y, t); }

/* bc_mode 1 (Sec. 3): at every edge node x_b the streamed populations are replaced by
 * g_i(x_b) = g_i^eq(phi_b(x_b), u(x_b)) + g_i(x_f) - g_i^eq(phi(x_f), u(x_f)), x_f the next node
 * inward along the normal (diagonally at corners); every edge node takes all nine. */
static void dirichlet_nee(oracle_sim* s) {
    const int nx = s->p.nx, ny = s->p.ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (i != 0 && i != nx - 1 && j != 0 && j != ny - 1) continue;
            const int fi = i == 0 ? 1 : (i == nx - 1 ? nx - 2 : i);
            const int fj = j == 0 ? 1 : (j == ny - 1 ? ny - 2 : j);
            const size_t kb = (size_t)j * nx + i, kf = (size_t)fj * nx + fi;
            const double ub[2] = {s->ux[kb], s->uy[kb]}, uf[2] = {s->ux[kf], s->uy[kf]};
            double phif = 0.0, geqb[Q], geqf[Q];
            for (int q = 0; q < Q; ++q) phif += s->g[AT(s, q, fj, fi)];
            equilibrium(&s->L, s->phi_b[kb], ub, geqb);
            equilibrium(&s->L, phif, uf, geqf);
            for (int q = 0; q < Q; ++q) s->g[AT(s, q, j, i)] = geqb[q] + s->g[AT(s, q, fj, fi)] - geqf[q];
        }
}

void oracle_step(oracle_sim* s, long nsteps) {
    for (long n = 0; n < nsteps; ++n) {
        const double t_n = (double)s->step * s->p.dt;
        const double t_nm1 = (double)(s->step - 1) * s->p.dt;
        step_rows(s, 0, s->p.ny, t_n, t_nm1);
        double* tmp = s->g;
        s->g = s->gnext;
        s->gnext = tmp;
        if (s->p.bc_mode == 1) dirichlet_nee(s);
        if (s->p.src_mode == 1) {
            memcpy(s->S_prev, s->S_cur, s->n * sizeof(double));
            s->S_prev_valid = 1;
        }
        s->step += 1;
    }
}

/* Timing sample: the collide-and-push work of one step restricted to rows [j0, j1), written
 * into the scratch array only (the state does not advance).  Used by the CPU baseline. */
void oracle_step_rows_sample(oracle_sim* s, int j0, int j1) {
    const double t_n = (double)s->step * s->p.dt;
    step_rows(s, j0, j1, t_n, t_n - s->p.dt);
}

long oracle_step_count(const oracle_sim* s) { return s->step; }

/* phi(x, t_n) = sum_i g_i(x, t_n). */
void oracle_phi(const oracle_sim* s, double* out) {
    for (size_t k = 0; k < s->n; ++k) {
        double phi = 0.0;
        for (int q = 0; q < Q; ++q) phi += s->g[(size_t)q * s->n + k];
        out[k] = phi;
    }
}

void oracle_get_g(const oracle_sim* s, double* out) { memcpy(out, s->g, Q * s->n * sizeof(double)); }

/* Sets the pre-collision state g_i(x, t_n) and the step counter n. */
void oracle_set_g(oracle_sim* s, const double* g, long step) {
    memcpy(s->g, g, Q * s->n * sizeof(double));
    s->step = step;
    s->S_prev_valid = 0;
}

double oracle_mass(const oracle_sim* s) {
    double m = 0.0;
    for (size_t k = 0; k < s->n; ++k)
        for (int q = 0; q < Q; ++q) m += s->g[(size_t)q * s->n + k];
    return m;
}

/* RMS error, Eq. (33) [eq19]: E_r = sqrt(sum |phi - phi_ref|^2 / (Nx Ny)), and the relative
 * L2 error ||phi - phi_ref|| / ||phi_ref||. */
void oracle_error(const oracle_sim* s, const double* phi_ref, double* rms, double* rel_l2) {
    double num = 0.0, den = 0.0;
    for (size_t k = 0; k < s->n; ++k) {
        double phi = 0.0;
        for (int q = 0; q < Q; ++q) phi += s->g[(size_t)q * s->n + k];
        const double d = phi - phi_ref[k];
        num += d * d;
        den += phi_ref[k] * phi_ref[k];
    }
    *rms = sqrt(num / (double)s->n);
    *rel_l2 = den > 0.0 ? sqrt(num / den) : sqrt(num);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Discrete adjoint of the step (for gradients with respect to D).                       */

/* Derivatives of the right-hand side of Eq. (14) at one node with respect to tau1 and tau2
 * (the per-node relaxation times), from Eqs. (12), (16) and (3):
 *   d/dtau1: (1/tau1^2) w_i H_ia B_a^neq / cs^2 + dt dG_i/dtau1 + dt dF_i^n/dtau1
 *            + dt/2 (dF_i^n/dtau1 - dF_i^{n-1}/dtau1),
 *            dG_i/dtau1 = w_i e_ia/cs^2 phi u_b d_b u_a / (2 tau1^2),
 *            dF_i/dtau1 = w_i e_ia u_a S / (cs^2 2 tau1^2);
 *   d/dtau2: (1/tau2^2) w_i H_iab B_ab^neq / (2 cs^4). */
static void node_dpost_dtau(const oracle_lattice* L, double dt, const double g[Q], const double u[2],
                            const double du[2][2], double tau1, double tau2, double Sn, double Snm1, double d1[Q],
                            double d2[Q]) {
    const double cs2 = L->cs2, cs4 = cs2 * cs2;
    double phi = 0.0;
    for (int i = 0; i < Q; ++i) phi += g[i];
    double geq[Q], gneq[Q];
    equilibrium(L, phi, u, geq);
    for (int i = 0; i < Q; ++i) gneq[i] = g[i] - geq[i];
    double B1[2] = {0.0, 0.0};
    double B2[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 2; ++a) {
            B1[a] += L->H1[i][a] * gneq[i];
            for (int b = 0; b < 2; ++b) B2[a][b] += L->H2[i][a][b] * gneq[i];
        }
    double adv[2];
    for (int a = 0; a < 2; ++a) {
        adv[a] = 0.0;
        for (int b = 0; b < 2; ++b) adv[a] += u[b] * du[a][b];
    }
    const double dk1 = 1.0 / (tau1 * tau1), dkh = 1.0 / (2.0 * tau1 * tau1), dk2 = 1.0 / (tau2 * tau2);
    for (int i = 0; i < Q; ++i) {
        double r1 = 0.0, r2 = 0.0, ea = 0.0, eu = 0.0;
        for (int a = 0; a < 2; ++a) {
            r1 += L->H1[i][a] * B1[a];
            ea += L->e[i][a] * adv[a];
            eu += L->e[i][a] * u[a];
            for (int b = 0; b < 2; ++b) r2 += L->H2[i][a][b] * B2[a][b];
        }
        const double dG = WEIGHT[i] * ea / cs2 * dkh * phi;
        const double dFn = WEIGHT[i] * eu * Sn / cs2 * dkh;
        const double dFnm1 = WEIGHT[i] * eu * Snm1 / cs2 * dkh;
        d1[i] = dk1 * WEIGHT[i] * r1 / cs2 + dt * dG + dt * dFn + (dt / 2.0) * (dFn - dFnm1);
        d2[i] = dk2 * WEIGHT[i] * r2 / (2.0 * cs4);
    }
}

static void node_sources(const oracle_sim* s, int i, int j, const double* Scur, const double* Sprev, int prev_valid,
                         long step, double* Sn, double* Snm1) {
    *Sn = 0.0;
    *Snm1 = 0.0;
    const size_t k = (size_t)j * s->p.nx + i;
    if (s->p.src_mode == 1) {
        *Sn = Scur[k];
        *Snm1 = prev_valid ? Sprev[k] : *Sn;
    } else if (s->p.src_mode == 2) {
        const double x = node_x(s, i), y = node_y(s, j);
        *Sn = pulse_source(s, x, y, (double)step * s->p.dt);
        *Snm1 = pulse_source(s, x, y, (double)(step - 1) * s->p.dt);
    }
}

/* Runs `nsteps` steps forward from the current state, keeping every state, then sweeps
 * back: with J any function of the final phi and lamN = dJ/dphi^N ([ny][nx]),
 *   lambda^N_i(x) = lamN(x);
 *   mu_i(x) = lambda^{n+1}_i(x + e_i)          (transpose of the push of Eq. (14))
 *   lambda^n_j(x) = sum_i A_ij(x) mu_i(x)      (A(x): the node map's Jacobian in g)
 *   dJ/dD(x) += sum_i mu_i(x) dpost_i/dD(x, g^n(x))
 * with dpost/dD = dtau1/dD (dpost/dtau1 + dtau2/dtau1 dpost/dtau2), dtau1/dD = 1/(cs^2 dt),
 * dtau2/dtau1 = -Lambda/(tau1 - 1/2)^2 for the magic parameter and 0 for a fixed tau2.
 * A(x) is built column by column from the node map applied to unit vectors minus its value
 * at zero (the map is affine in g).  src_mode 1 keeps one source field for every step.
 * Outputs grad [ny][nx] (dJ/dD) and, if lam0 is not NULL, lam0 [9][ny][nx] = dJ/dg^0.
 * Returns 0, or -1 if memory runs out or the boundaries are not periodic (bc_mode 1). */
int oracle_adjoint(oracle_sim* s, long nsteps, const double* lamN, double* grad, double* lam0) {
    if (s->p.bc_mode != 0) return -1;
    const int nx = s->p.nx, ny = s->p.ny;
    const size_t n = s->n, st = Q * n;
    double* states = (double*)malloc((size_t)(nsteps + 1) * st * sizeof(double));
    double* Sstore = s->p.src_mode == 1 ? (double*)malloc(2 * n * sizeof(double)) : NULL;
    double* jac = (double*)malloc(n * Q * Q * sizeof(double));
    double* lam = (double*)malloc(st * sizeof(double));
    double* lnext = (double*)malloc(st * sizeof(double));
    if (!states || !jac || !lam || !lnext || (s->p.src_mode == 1 && !Sstore)) {
        free(states); free(Sstore); free(jac); free(lam); free(lnext);
        return -1;
    }
    const long step0 = s->step;
    const int prev_valid0 = s->S_prev_valid;
    if (Sstore) {
        memcpy(Sstore, s->S_cur, n * sizeof(double));
        memcpy(Sstore + n, s->S_prev, n * sizeof(double));
    }
    memcpy(states, s->g, st * sizeof(double));
    for (long k = 0; k < nsteps; ++k) {
        oracle_step(s, 1);
        memcpy(states + (size_t)(k + 1) * st, s->g, st * sizeof(double));
    }
    /* node Jacobians (independent of g and of time) */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t k = (size_t)j * nx + i;
            const double u[2] = {s->ux[k], s->uy[k]};
            double du[2][2], tau1, tau2, zero[Q] = {0}, e[Q], p0[Q], pe[Q];
            grad_u(s, i, j, du);
            node_taus(s, k, &tau1, &tau2);
            node_post(&s->L, s->p.dt, zero, u, du, tau1, tau2, 0.0, 0.0, p0);
            for (int c = 0; c < Q; ++c) {
                for (int q = 0; q < Q; ++q) e[q] = q == c ? 1.0 : 0.0;
                node_post(&s->L, s->p.dt, e, u, du, tau1, tau2, 0.0, 0.0, pe);
                for (int q = 0; q < Q; ++q) jac[(k * Q + q) * Q + c] = pe[q] - p0[q];
            }
        }
    for (size_t k = 0; k < n; ++k) {
        grad[k] = 0.0;
        for (int q = 0; q < Q; ++q) lam[q * n + k] = lamN[k];
    }
    const double dtau1_dD = 1.0 / (s->L.cs2 * s->p.dt);
    for (long m = nsteps - 1; m >= 0; --m) {
        const double* gm = states + (size_t)m * st;
        const long stepm = step0 + m;
        const int prev_valid = m == 0 ? prev_valid0 : 1;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t k = (size_t)j * nx + i;
                double mu[Q], g[Q], d1[Q], d2[Q];
                for (int q = 0; q < Q; ++q) {
                    const int it = ((i + EHAT[q][0]) % nx + nx) % nx;
                    const int jt = ((j + EHAT[q][1]) % ny + ny) % ny;
                    mu[q] = lam[q * n + (size_t)jt * nx + it];
                    g[q] = gm[q * n + k];
                }
                for (int c = 0; c < Q; ++c) {
                    double acc = 0.0;
                    for (int q = 0; q < Q; ++q) acc += jac[(k * Q + q) * Q + c] * mu[q];
                    lnext[c * n + k] = acc;
                }
                if (s->p.tau1_const > 0.0) continue; /* D does not enter */
                const double u[2] = {s->ux[k], s->uy[k]};
                double du[2][2], tau1, tau2, Sn, Snm1;
                grad_u(s, i, j, du);
                node_taus(s, k, &tau1, &tau2);
                /* src_mode 1: the field stays S^n; S^{n-1} is the stored one only at the first step */
                node_sources(s, i, j, Sstore, Sstore ? (m == 0 ? Sstore + n : Sstore) : NULL, prev_valid, stepm, &Sn,
                             &Snm1);
                node_dpost_dtau(&s->L, s->p.dt, g, u, du, tau1, tau2, Sn, Snm1, d1, d2);
                const double dtau2_dtau1 = s->p.tau2_mode == 1 ? 0.0 : -s->p.magic / ((tau1 - 0.5) * (tau1 - 0.5));
                double acc = 0.0;
                for (int q = 0; q < Q; ++q) acc += mu[q] * (d1[q] + dtau2_dtau1 * d2[q]);
                grad[k] += dtau1_dD * acc;
            }
        double* t = lam;
        lam = lnext;
        lnext = t;
    }
    if (lam0) memcpy(lam0, lam, st * sizeof(double));
    free(states); free(Sstore); free(jac); free(lam); free(lnext);
    return 0;
}


/* The paper's benchmark (Sec. 3): a rotating Gaussian pulse with a manufactured source on
 * [-L/2, L/2]^2, L = 4 pi, with Dirichlet boundaries by non-equilibrium extrapolation.
 *
 *   u = (-y, x), kappa constant, phi_a = exp(-(x^2 + 3 y^2 + 2 kappa t)),
 *   S = [6 kappa - 4 x y - 4 kappa (x^2 + 9 y^2)] exp(-(x^2 + 3 y^2 + 2 kappa t)),
 *   g = g^eq(phi_0, u) at t = 0; RMS error of Eq. (33) over all nodes at t_end.
 *
 * Models (the columns of Table 2):
 *   0  present: TRT-R (Eq. (12)), G of Eq. (16), F of Eq. (3), dt^2/2 d_t F;
 *   1  TRT-R with the traditional terms: G of Eq. (15)/(34) with d_t(phi u) taken as
 *      (phi^n - phi^{n-1}) u / dt (u is steady; 0 at the first step), F = w S (Eq. (35));
 *   2  BGK (Eq. (4), tau = tau1) with the same traditional terms.
 * All three take d_t F as (F^n - F^{n-1}) / dt with S^{n-1} = S(t_n - dt), the closed form, at
 * the first step too.
 *
 * Readings: nodes x_i = -L/2 + i L/N, i = 0..N (N + 1 per side; both boundaries are nodes and
 * dx = L / N); at a boundary node after streaming, g_i = g_i^eq(phi_a, u) + g_i(x_f) -
 * g_i^eq(phi(x_f), u(x_f)) for every i, x_f the adjacent interior node along the inward normal
 * (the diagonal one at corners); d_beta u_alpha is exact (u is linear); tau2 from Lambda. */

typedef struct {
    int N;          /* intervals per side */
    double L;       /* side length */
    double kappa;   /* diffusivity */
    double dt;      /* time step */
    int model;      /* 0, 1, 2 (above) */
    double magic;   /* Lambda for tau2 */
} oracle_paper_params;

static double paper_phi(double x, double y, double kappa, double t) {
    return exp(-(x * x + 3.0 * y * y + 2.0 * kappa * t));
}

static double paper_source(double x, double y, double kappa, double t) {
    return (6.0 * kappa - 4.0 * x * y - 4.0 * kappa * (x * x + 9.0 * y * y)) * exp(-(x * x + 3.0 * y * y + 2.0 * kappa * t));
}

/* BGK collision, Eq. (4): g^eq + (1 - 1/tau) (g - g^eq). */
static void collide_bgk(const oracle_lattice* L, const double g[Q], const double u[2], double tau, double out[Q],
                        double* phi_out) {
    double phi = 0.0;
    for (int i = 0; i < Q; ++i) phi += g[i];
    double geq[Q];
    equilibrium(L, phi, u, geq);
    for (int i = 0; i < Q; ++i) out[i] = geq[i] + (1.0 - 1.0 / tau) * (g[i] - geq[i]);
    *phi_out = phi;
}

/* Runs the benchmark to t_end (round(t_end / dt) steps).  Writes the RMS error of Eq. (33)
 * at t_end and, if phi_out is not NULL, phi there ([N + 1][N + 1], x fastest); returns 0, 1 if
 * the run blew up (non-finite or |phi| > 1e3), -1 on bad input. */
int oracle_paper_pulse(const oracle_paper_params* pp, double t_end, double* rms_out, double* phi_out) {
    const int N = pp->N, n1 = N + 1;
    if (N < 2 || !(pp->dt > 0.0) || !(pp->L > 0.0)) return -1;
    const double dx = pp->L / N, dt = pp->dt, x0 = -pp->L / 2.0;
    oracle_lattice Lat;
    lattice_init(&Lat, dx, dt);
    const size_t n = (size_t)n1 * n1;
    double* g = (double*)calloc(Q * n, sizeof(double));
    double* gn = (double*)calloc(Q * n, sizeof(double));
    double* phi_prev = (double*)calloc(n, sizeof(double));
    double* phi_cur = (double*)calloc(n, sizeof(double));
    if (!g || !gn || !phi_prev || !phi_cur) {
        free(g); free(gn); free(phi_prev); free(phi_cur);
        return -1;
    }
    const double tau1 = 0.5 + pp->kappa / (Lat.cs2 * dt);
    const double tau2 = 0.5 + pp->magic / (tau1 - 0.5);
    const double du[2][2] = {{0.0, -1.0}, {1.0, 0.0}}; /* d_b u_a for u = (-y, x) */
#define PIDX(q, j, i) ((size_t)(q) * n + (size_t)(j) * n1 + (size_t)(i))
    for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
            const double x = x0 + i * dx, y = x0 + j * dx, u[2] = {-y, x};
            double geq[Q];
            equilibrium(&Lat, paper_phi(x, y, pp->kappa, 0.0), u, geq);
            for (int q = 0; q < Q; ++q) g[PIDX(q, j, i)] = geq[q];
            phi_cur[(size_t)j * n1 + i] = paper_phi(x, y, pp->kappa, 0.0);
            phi_prev[(size_t)j * n1 + i] = phi_cur[(size_t)j * n1 + i];
        }
    const long steps = lround(t_end / dt);
    int blew = 0;
    for (long s = 0; s < steps && !blew; ++s) {
        const double tn = s * dt, tnm1 = (s - 1) * dt;
        memset(gn, 0, Q * n * sizeof(double));
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
                const double x = x0 + i * dx, y = x0 + j * dx, u[2] = {-y, x};
                const size_t k = (size_t)j * n1 + i;
                double gl[Q], post[Q], G[Q], Fn[Q], Fp[Q], phi;
                for (int q = 0; q < Q; ++q) gl[q] = g[PIDX(q, j, i)];
                const double Sn = paper_source(x, y, pp->kappa, tn);
                const double Sp = paper_source(x, y, pp->kappa, tnm1); /* S(-dt) at the first step */
                if (pp->model == 2) collide_bgk(&Lat, gl, u, tau1, post, &phi);
                else collide_trtr(&Lat, gl, u, tau1, tau2, post, &phi);
                phi_cur[k] = phi;
                if (pp->model == 0) {
                    aux_G(&Lat, phi, u, du, tau1, G);
                    source_F(&Lat, Sn, u, tau1, Fn);
                    source_F(&Lat, Sp, u, tau1, Fp);
                } else {
                    /* G_i = w_i e_ia / cs^2 (1 - 1/(2 tau1)) d_t(phi u_a), Eq. (15) */
                    const double dphidt = s > 0 ? (phi - phi_prev[k]) / dt : 0.0;
                    for (int q = 0; q < Q; ++q) {
                        const double eu = Lat.e[q][0] * u[0] + Lat.e[q][1] * u[1];
                        G[q] = WEIGHT[q] * eu / Lat.cs2 * (1.0 - 1.0 / (2.0 * tau1)) * dphidt;
                        Fn[q] = WEIGHT[q] * Sn; /* Eq. (35) */
                        Fp[q] = WEIGHT[q] * Sp;
                    }
                }
                for (int q = 0; q < Q; ++q) {
                    const double v = post[q] + dt * G[q] + dt * Fn[q] + (dt * dt / 2.0) * (Fn[q] - Fp[q]) / dt;
                    const int it = i + EHAT[q][0], jt = j + EHAT[q][1];
                    if (it >= 0 && it < n1 && jt >= 0 && jt < n1) gn[PIDX(q, jt, it)] = v;
                }
            }
        memcpy(phi_prev, phi_cur, n * sizeof(double));
        /* non-equilibrium extrapolation at the boundary nodes */
        const double t1 = (s + 1) * dt;
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
                if (i != 0 && i != N && j != 0 && j != N) continue;
                const int fi = i == 0 ? 1 : (i == N ? N - 1 : i);
                const int fj = j == 0 ? 1 : (j == N ? N - 1 : j);
                const double xb = x0 + i * dx, yb = x0 + j * dx, ub[2] = {-yb, xb};
                const double xf = x0 + fi * dx, yf = x0 + fj * dx, uf[2] = {-yf, xf};
                double phif = 0.0, geqb[Q], geqf[Q];
                for (int q = 0; q < Q; ++q) phif += gn[PIDX(q, fj, fi)];
                equilibrium(&Lat, paper_phi(xb, yb, pp->kappa, t1), ub, geqb);
                equilibrium(&Lat, phif, uf, geqf);
                for (int q = 0; q < Q; ++q) gn[PIDX(q, j, i)] = geqb[q] + gn[PIDX(q, fj, fi)] - geqf[q];
            }
        double* t = g;
        g = gn;
        gn = t;
        for (size_t k = 0; k < n && !blew; ++k) {
            double phi = 0.0;
            for (int q = 0; q < Q; ++q) phi += g[(size_t)q * n + k];
            if (!isfinite(phi) || fabs(phi) > 1e3) blew = 1;
        }
    }
    double num = 0.0;
    const double tf = steps * dt;
    for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
            double phi = 0.0;
            for (int q = 0; q < Q; ++q) phi += g[PIDX(q, j, i)];
            const double d = phi - paper_phi(x0 + i * dx, x0 + j * dx, pp->kappa, tf);
            num += d * d;
            if (phi_out) phi_out[(size_t)j * n1 + i] = phi;
        }
#undef PIDX
    *rms_out = sqrt(num / (double)n);
    free(g); free(gn); free(phi_prev); free(phi_cur);
    return blew;
}

/* The slip check of Sec. 3.2: steady diffusion with a uniform source S between two walls at
 * y = 0 and y = H = ny dx held at phi_w, in lattice units (dx = dt = 1, u = 0), one column
 * periodic in x.  Nodes sit at y_j = j + 1/2 (halfway walls); a population that would stream
 * through a wall returns to its node reversed by the Dirichlet bounce-back rule
 * g_ibar(x_f, t + 1) = -P_i(x_f, t) + 2 w_i phi_w.  The exact solution of kappa phi'' = -S is
 * the parabola phi_w + S/(2 kappa) y (H - y), kappa = (tau1 - 1/2) / 3; Eq. (37) names the
 * tau2 for which the scheme has no slip at the wall.  Steps until max |phi^{n+1} - phi^n| <=
 * tol (or max_steps); writes the RMS error of Eq. (33) against the parabola and, if phi_out
 * is not NULL, the ny values of phi.  Returns the number of steps, or -1 on bad input. */
long oracle_paper_slip(int ny, double tau1, double tau2, double S, double phi_w, long max_steps, double tol,
                       double* rms_out, double* phi_out) {
    if (ny < 2 || !(tau1 > 0.5) || !(tau2 > 0.5) || max_steps < 1) return -1;
    oracle_lattice Lat;
    lattice_init(&Lat, 1.0, 1.0);
    const double kappa = (tau1 - 0.5) * Lat.cs2;
    double* g = (double*)calloc((size_t)Q * ny, sizeof(double));
    double* post = (double*)calloc((size_t)Q * ny, sizeof(double));
    double* phi = (double*)calloc((size_t)ny, sizeof(double));
    if (!g || !post || !phi) {
        free(g); free(post); free(phi);
        return -1;
    }
    const double u[2] = {0.0, 0.0};
    for (int j = 0; j < ny; ++j) {
        double geq[Q];
        equilibrium(&Lat, phi_w, u, geq);
        for (int q = 0; q < Q; ++q) g[(size_t)q * ny + j] = geq[q];
        phi[j] = phi_w;
    }
    long s = 0;
    for (; s < max_steps; ++s) {
        for (int j = 0; j < ny; ++j) {
            double gl[Q], pl[Q], p;
            for (int q = 0; q < Q; ++q) gl[q] = g[(size_t)q * ny + j];
            collide_trtr(&Lat, gl, u, tau1, tau2, pl, &p);
            /* u = 0: G = 0 and F_i = w_i S (Eq. (3)); S is steady, so d_t F = 0 */
            for (int q = 0; q < Q; ++q) post[(size_t)q * ny + j] = pl[q] + WEIGHT[q] * S;
        }
        double change = 0.0;
        for (int j = 0; j < ny; ++j) {
            double p = 0.0;
            for (int q = 0; q < Q; ++q) {
                const int js = j - EHAT[q][1];
                double v;
                if (js >= 0 && js < ny) v = post[(size_t)q * ny + js];
                else v = -post[(size_t)OPPOSITE[q] * ny + j] + 2.0 * WEIGHT[q] * phi_w;
                g[(size_t)q * ny + j] = v;
                p += v;
            }
            change = fmax(change, fabs(p - phi[j]));
            phi[j] = p;
        }
        if (change <= tol) {
            ++s;
            break;
        }
    }
    double num = 0.0;
    const double H = (double)ny;
    for (int j = 0; j < ny; ++j) {
        const double y = j + 0.5, d = phi[j] - (phi_w + S / (2.0 * kappa) * y * (H - y));
        num += d * d;
        if (phi_out) phi_out[j] = phi[j];
    }
    *rms_out = sqrt(num / ny);
    free(g); free(post); free(phi);
    return s;
}
