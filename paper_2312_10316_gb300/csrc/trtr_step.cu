// trtr_step.cu -- the fused TRT-R time step: one kernel per step does pull-streaming,
// the phi moment, the TRT-R regularised relaxation, the auxiliary term G and the source
// term F of the evolution equation (14) of Sec. 2.2, and stores the post-collision values.
//
// Arithmetic, in lattice units (e = ehat integer, cs^2 = 1/3, uhat = u dt/dx):
//   phi = sum g_i                                               (B_0^neq = 0, Sec. 2.2)
//   B_a  = sum e_ia g_i - phi u_a                               Eq. (8)
//   B_ab = sum (e_ia e_ib - d_ab/3) g_i - phi u_a u_b           Eq. (13)
// (the equilibrium's Hermite moments are phi u_a and phi u_a u_b by D2Q9 quadrature).
// The right-hand side of Eq. (14) is a Hermite series with coefficients
//   m0    = phi + s                                  (s = dt S^n + dt/2 (S^n - S^{n-1}))
//   m1_a  = phi u_a + (1 - 1/tau1) B_a + (1 - 1/(2 tau1)) (phi a_a + u_a s)
//   A_ab  = phi u_a u_b + (1 - 1/tau2) B_ab
//   T_xxy = phi u_x^2 u_y,  T_xyy = phi u_x u_y^2        (third-order equilibrium, Eq. (6))
// where a_a = u_b d_b u_a (Eq. (16)) comes from central differences of the staged u tile,
// and the D2Q9 populations are rebuilt pairwise from their even and odd halves.
//
// Layout: one warp covers 32 consecutive x nodes, so every population plane is read and
// written in 128-byte rows; pulls with e_x != 0 are the same rows shifted by one element.
#include "trtr_internal.cuh"

namespace trtr {
namespace {

constexpr int kBX = 32;          // nodes per block along x (one warp)
constexpr int kBY = 8;           // warps per block
constexpr int kRY = 2;           // rows per thread
constexpr int kTY = kBY * kRY;   // tile height

template <typename C>
__device__ __forceinline__ C pulse_source(C x, C y, C cx, C cy, C inv_s2, C amp, C dD, C dDx, C dDy) {
    // S = phi_a / s^2 [grad D . r - (D - D0)(|r|^2 / s^2 - 2)],  r = x - c(t)
    const C rx = x - cx, ry = y - cy;
    const C r2 = rx * rx + ry * ry;
    const C e = amp * exp(C(-0.5) * r2 * inv_s2);
    return e * inv_s2 * ((dDx * rx + dDy * ry) - dD * (r2 * inv_s2 - C(2)));
}

template <typename S, int SRC>
__global__ void __launch_bounds__(kBX * kBY)
    step_kernel(const StepArgs<typename Store<S>::C> a) {
    using C = typename Store<S>::C;
    using ST = Store<S>;
    __shared__ C su[2][kTY + 2][kBX + 2];  // uhat_x, uhat_y with a one-node halo

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kTY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;

    // Stage the u tile.  Halo cells just outside the domain wrap periodically; cells
    // further out are never read by an in-domain node and are clamped to a valid index.
    for (int k = ty * kBX + tx; k < (kTY + 2) * (kBX + 2); k += kBX * kBY) {
        const int r = k / (kBX + 2), c = k - r * (kBX + 2);
        int gi = i0 + c - 1, gj = j0 + r - 1;
        gi = gi < 0 ? gi + nx : gi;
        gi = gi >= nx ? gi - nx : gi;
        gi = gi >= nx ? 0 : gi;
        gj = gj < 0 ? gj + ny : gj;
        gj = gj >= ny ? gj - ny : gj;
        gj = gj >= ny ? 0 : gj;
        const size_t o = (size_t)gj * pitch + gi;
        su[0][r][c] = a.ux[o];
        su[1][r][c] = a.uy[o];
    }
    __syncthreads();

    const int i = i0 + tx;
    if (i >= nx) return;
    const int im = (i == 0) ? nx - 1 : i - 1;
    const int ip = (i == nx - 1) ? 0 : i + 1;
    const C phi_ref = a.phi_ref;
    const C o0 = C(4.0 / 9.0) * phi_ref, o1 = C(1.0 / 9.0) * phi_ref, o5 = C(1.0 / 36.0) * phi_ref;
    const S* P = static_cast<const S*>(a.src);
    S* Pn = static_cast<S*>(a.dst);
    const size_t pl = a.plane;

    // x-direction stencil weights for d_x (uniform except at the domain edges)
    C wxp = C(0.5), wx0 = C(0), wxm = C(-0.5);
    if (nx == 1) {
        wxp = wx0 = wxm = C(0);
    } else if (a.grad_mode == TRTR_GRAD_ONESIDED_EDGE && i == 0) {
        wxp = C(1); wx0 = C(-1); wxm = C(0);
    } else if (a.grad_mode == TRTR_GRAD_ONESIDED_EDGE && i == nx - 1) {
        wxp = C(0); wx0 = C(1); wxm = C(-1);
    }

#pragma unroll
    for (int rr = 0; rr < kRY; ++rr) {
        const int tr = ty + rr * kBY;  // row inside the tile
        const int j = j0 + tr;
        if (j >= ny) break;
        const int jm = (j == 0) ? ny - 1 : j - 1;
        const int jp = (j == ny - 1) ? 0 : j + 1;
        const size_t rm = (size_t)jm * pitch, r0 = (size_t)j * pitch, rp = (size_t)jp * pitch;

        // a1: pull-streaming, g_i(x) = P_i(x - e_i)
        const C g0 = ST::load(P + 0 * pl + r0 + i, o0);
        const C g1 = ST::load(P + 1 * pl + r0 + im, o1);
        const C g2 = ST::load(P + 2 * pl + r0 + ip, o1);
        const C g3 = ST::load(P + 3 * pl + rm + i, o1);
        const C g4 = ST::load(P + 4 * pl + rp + i, o1);
        const C g5 = ST::load(P + 5 * pl + rm + im, o5);
        const C g6 = ST::load(P + 6 * pl + rp + ip, o5);
        const C g7 = ST::load(P + 7 * pl + rp + im, o5);
        const C g8 = ST::load(P + 8 * pl + rm + ip, o5);
        const C Dh = __ldg(a.Dh + r0 + i);

        // coefficients at the node and d_b u_a from the staged tile
        const C ux = su[0][tr + 1][tx + 1];
        const C uy = su[1][tr + 1][tx + 1];
        C wyp = C(0.5), wy0 = C(0), wym = C(-0.5);
        if (ny == 1) {
            wyp = wy0 = wym = C(0);
        } else if (a.grad_mode == TRTR_GRAD_ONESIDED_EDGE && j == 0) {
            wyp = C(1); wy0 = C(-1); wym = C(0);
        } else if (a.grad_mode == TRTR_GRAD_ONESIDED_EDGE && j == ny - 1) {
            wyp = C(0); wy0 = C(1); wym = C(-1);
        }
        const C dxux = wxp * su[0][tr + 1][tx + 2] + wx0 * ux + wxm * su[0][tr + 1][tx];
        const C dxuy = wxp * su[1][tr + 1][tx + 2] + wx0 * uy + wxm * su[1][tr + 1][tx];
        const C dyux = wyp * su[0][tr + 2][tx + 1] + wy0 * ux + wym * su[0][tr][tx + 1];
        const C dyuy = wyp * su[1][tr + 2][tx + 1] + wy0 * uy + wym * su[1][tr][tx + 1];
        const C ax = ux * dxux + uy * dyux;  // (u.grad) u_x
        const C ay = ux * dxuy + uy * dyuy;  // (u.grad) u_y

        // relaxation rates: tau1 - 1/2 = 3 Dh (Sec. 2.4); tau2 from Lambda (Eq. (28))
        const C t1m = C(3) * Dh;
        const C w1 = C(1) / (C(0.5) + t1m);
        const C w2 = a.tau2_fixed ? a.omega2_fixed : t1m / (C(0.5) * t1m + a.magic);
        const C k1 = C(1) - w1, k2 = C(1) - w2, kh = C(1) - C(0.5) * w1;

        // a7: s = dt S^n + dt/2 (S^n - S^{n-1})
        C s = C(0);
        if (SRC == TRTR_SRC_FIELD) {
            const C sn = __ldg(a.S_cur + r0 + i);
            const C sp = __ldg(a.S_prev + r0 + i);
            s = sn + C(0.5) * (sn - sp);
        } else if (SRC == TRTR_SRC_PULSE) {
            const C x = a.x0 + C(i) * a.dx, y = a.y0 + C(j) * a.dx;
            const C sxi = __ldg(a.tab_x + i), cxi = __ldg(a.tab_x + pitch + i);
            const C syj = __ldg(a.tab_y + j), cyj = __ldg(a.tab_y + ny + j);
            const C dD = a.dD_amp * sxi * syj;
            const C dDx = a.dD_amp * C(3.14159265358979323846) * cxi * syj;
            const C dDy = a.dD_amp * C(3.14159265358979323846) * sxi * cyj;
            const C Sn = pulse_source(x, y, a.cx_n, a.cy_n, a.inv_s2_n, a.amp_n, dD, dDx, dDy);
            const C Sp = a.first_step ? Sn : pulse_source(x, y, a.cx_p, a.cy_p, a.inv_s2_p, a.amp_p, dD, dDx, dDy);
            s = a.dt * (Sn + C(0.5) * (Sn - Sp));
        }

        // a2 + a4: moments
        const C phi = ((g0 + g1) + (g2 + g3)) + ((g4 + g5) + (g6 + g7)) + g8;
        const C jx = (g1 - g2) + (g5 - g6) + (g7 - g8);
        const C jy = (g3 - g4) + (g5 - g6) + (g8 - g7);
        const C pdiag = (g5 + g6) + (g7 + g8);
        const C pxx = (g1 + g2) + pdiag;
        const C pyy = (g3 + g4) + pdiag;
        const C pxy = (g5 + g6) - (g7 + g8);

        const C phux = phi * ux, phuy = phi * uy;
        const C euxx = phux * ux, euyy = phuy * uy, euxy = phux * uy;
        const C third = phi * C(1.0 / 3.0);
        // a5 + a6 + a7: post-collision Hermite coefficients
        const C m0 = phi + s;
        const C m1x = phux + k1 * (jx - phux) + kh * (phi * ax + ux * s);
        const C m1y = phuy + k1 * (jy - phuy) + kh * (phi * ay + uy * s);
        const C Axx = euxx + k2 * (pxx - third - euxx);
        const C Ayy = euyy + k2 * (pyy - third - euyy);
        const C Axy = euxy + k2 * (pxy - euxy);
        const C Txxy = euxx * uy;
        const C Txyy = euxy * uy;

        // rebuild, even (E) and odd (O) halves of the opposite pairs
        const C Asum = Axx + Ayy;
        const C h0 = C(4.0 / 9.0) * (m0 - C(1.5) * Asum);
        const C E1 = m0 + C(3) * Axx - C(1.5) * Ayy;
        const C O1 = C(3) * m1x - C(4.5) * Txyy;
        const C E3 = m0 + C(3) * Ayy - C(1.5) * Axx;
        const C O3 = C(3) * m1y - C(4.5) * Txxy;
        const C Ed = m0 + C(3) * Asum;
        const C E5 = Ed + C(9) * Axy;
        const C O5 = C(3) * (m1x + m1y) + C(9) * (Txxy + Txyy);
        const C E7 = Ed - C(9) * Axy;
        const C O7 = C(3) * (m1x - m1y) + C(9) * (Txyy - Txxy);

        // a8: store P_i(x)
        const size_t o = r0 + i;
        ST::store(Pn + 0 * pl + o, h0, o0);
        ST::store(Pn + 1 * pl + o, C(1.0 / 9.0) * (E1 + O1), o1);
        ST::store(Pn + 2 * pl + o, C(1.0 / 9.0) * (E1 - O1), o1);
        ST::store(Pn + 3 * pl + o, C(1.0 / 9.0) * (E3 + O3), o1);
        ST::store(Pn + 4 * pl + o, C(1.0 / 9.0) * (E3 - O3), o1);
        ST::store(Pn + 5 * pl + o, C(1.0 / 36.0) * (E5 + O5), o5);
        ST::store(Pn + 6 * pl + o, C(1.0 / 36.0) * (E5 - O5), o5);
        ST::store(Pn + 7 * pl + o, C(1.0 / 36.0) * (E7 + O7), o5);
        ST::store(Pn + 8 * pl + o, C(1.0 / 36.0) * (E7 - O7), o5);
    }
}

template <typename S, int SRC>
cudaError_t launch_typed(trtr_ctx* ctx) {
    using C = typename Store<S>::C;
    StepArgs<C> a;
    a.src = ctx->pop[ctx->cur];
    a.dst = ctx->pop[ctx->cur ^ 1];
    a.ux = static_cast<const C*>(ctx->ux);
    a.uy = static_cast<const C*>(ctx->uy);
    a.Dh = static_cast<const C*>(ctx->Dh);
    const int sc = ctx->S_cur;
    const int sp = ctx->S_prev >= 0 ? ctx->S_prev : ctx->S_cur;
    a.S_cur = sc >= 0 ? static_cast<const C*>(ctx->S[sc]) : nullptr;
    a.S_prev = sp >= 0 ? static_cast<const C*>(ctx->S[sp]) : nullptr;
    a.tab_x = static_cast<const C*>(ctx->tab_x);
    a.tab_y = static_cast<const C*>(ctx->tab_y);
    a.nx = ctx->p.nx;
    a.ny = ctx->p.ny;
    a.pitch = ctx->pitch;
    a.plane = ctx->plane;
    a.grad_mode = ctx->p.grad_mode;
    a.tau2_fixed = ctx->p.tau2_mode == TRTR_TAU2_FIXED;
    a.magic = C(ctx->p.magic);
    a.omega2_fixed = C(ctx->p.tau2_mode == TRTR_TAU2_FIXED ? 1.0 / ctx->p.tau2 : 0.0);
    a.tau1_const_dh = C(0);
    a.phi_ref = C(ctx->p.phi_ref);
    a.x0 = C(ctx->p.x0);
    a.y0 = C(ctx->p.y0);
    a.dx = C(ctx->p.dx);
    a.dt = C(ctx->p.dt);
    a.first_step = ctx->step == 0;
    if (SRC == TRTR_SRC_PULSE) {
        const PulseTime tn = pulse_at(ctx->pulse, (double)ctx->step * ctx->p.dt);
        const PulseTime tp = pulse_at(ctx->pulse, (double)(ctx->step - 1) * ctx->p.dt);
        a.dD_amp = C(ctx->pulse.D0 * ctx->pulse.D_amp);
        a.cx_n = C(tn.cx); a.cy_n = C(tn.cy); a.inv_s2_n = C(tn.inv_s2); a.amp_n = C(tn.amp);
        a.cx_p = C(tp.cx); a.cy_p = C(tp.cy); a.inv_s2_p = C(tp.inv_s2); a.amp_p = C(tp.amp);
    } else {
        a.dD_amp = C(0);
        a.cx_n = a.cy_n = a.inv_s2_n = a.amp_n = C(0);
        a.cx_p = a.cy_p = a.inv_s2_p = a.amp_p = C(0);
    }
    const dim3 block(kBX, kBY);
    const dim3 grid((ctx->p.nx + kBX - 1) / kBX, (ctx->p.ny + kTY - 1) / kTY);
    step_kernel<S, SRC><<<grid, block, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_src(trtr_ctx* ctx) {
    switch (ctx->p.src_mode) {
        case TRTR_SRC_FIELD: return launch_typed<S, TRTR_SRC_FIELD>(ctx);
        case TRTR_SRC_PULSE: return launch_typed<S, TRTR_SRC_PULSE>(ctx);
        default: return launch_typed<S, TRTR_SRC_NONE>(ctx);
    }
}

}  // namespace

cudaError_t launch_step(trtr_ctx* ctx) {
    switch (ctx->p.precision) {
        case TRTR_F64: return launch_src<double>(ctx);
        case TRTR_F32: return launch_src<float>(ctx);
        case TRTR_F16_OFS: return launch_src<__half>(ctx);
        case TRTR_BF16_OFS: return launch_src<__nv_bfloat16>(ctx);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace trtr
