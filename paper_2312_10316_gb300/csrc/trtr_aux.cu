// trtr_aux.cu -- kernels around the step: coefficient fields (with their ghost cells),
// the pulse closed form, equilibrium initialisation (shifted into the pull layout), the
// phi moment, the FP64 reductions (mass, RMS / relative L2 error of Eq. (33)) and
// population I/O.
#include <math.h>

#include <type_traits>

#include "trtr_internal.cuh"

namespace trtr {

PulseTime pulse_at(const Pulse& p, double t) {
    PulseTime r;
    const double c = cos(p.omega * t), s = sin(p.omega * t);
    r.cx = p.xc * c - p.yc * s;
    r.cy = p.xc * s + p.yc * c;
    const double s2 = p.sigma0 * p.sigma0 + 2.0 * p.D0 * t;
    r.inv_s2 = 1.0 / s2;
    r.amp = p.sigma0 * p.sigma0 / s2;
    return r;
}

PlaneLayout make_layout(int nx, int ny, int elem_bytes, int ghost) {
    PlaneLayout L;
    L.nx = nx;
    L.ny = ny;
    const int line = 128 / elem_bytes;  // elements per 128-byte line
    L.gx = line;
    L.gy = ghost;
    long long pitch = ((long long)nx + 2LL * line + line - 1) / line * line;
    if (pitch < 320) pitch = 320;  // wider than every TMA box (<= 256 elements + origin shift)
    L.pitch = (int)pitch;
    L.rows = ny + 2 * ghost < 16 ? 16 : ny + 2 * ghost;
    L.plane = (size_t)L.rows * (size_t)L.pitch;
    return L;
}

namespace {

__constant__ int c_ex[kQ] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
__constant__ int c_ey[kQ] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
__constant__ double c_w[kQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Value of a field at ghosted position (i, j), i in [-1, nx], j in [-1, ny], from its interior
// values f(i, j): periodic wrap, or the linear extrapolation 2 f(edge) - f(edge -+ 1) (grad
// mode one-sided; a single node repeats itself).  Corners compose the two rules.
template <typename F>
__device__ __forceinline__ double ghosted(const F& f, int i, int j, int nx, int ny, int grad_mode) {
    auto along_x = [&](int jj) -> double {
        if (i >= 0 && i < nx) return f(i, jj);
        if (grad_mode == TRTR_GRAD_PERIODIC || nx == 1) return f(wrap(i, nx), jj);
        return i < 0 ? 2.0 * f(0, jj) - f(1, jj) : 2.0 * f(nx - 1, jj) - f(nx - 2, jj);
    };
    if (j >= 0 && j < ny) return along_x(j);
    if (grad_mode == TRTR_GRAD_PERIODIC || ny == 1) return along_x(wrap(j, ny));
    return j < 0 ? 2.0 * along_x(0) - along_x(1) : 2.0 * along_x(ny - 1) - along_x(ny - 2);
}

// u (with ghosts) and D from caller arrays [ny][nx] in physical units.
template <typename C>
__global__ void convert_fields_kernel(C* uv, C* Dh, const double* sux, const double* suy, const double* sD,
                                      PlaneLayout L, int grad_mode, double u_scale, double d_scale, double dh_const,
                                      int use_const) {
    const int gw = L.nx + 2, gh = L.ny + 2;
    const size_t n = (size_t)gw * gh;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / gw) - 1, i = (int)(k % gw) - 1;
        auto fx = [&](int ii, int jj) { return sux[(size_t)jj * L.nx + ii]; };
        auto fy = [&](int ii, int jj) { return suy[(size_t)jj * L.nx + ii]; };
        uv[L.at(i, j)] = C(ghosted(fx, i, j, L.nx, L.ny, grad_mode) * u_scale);
        uv[L.plane + L.at(i, j)] = C(ghosted(fy, i, j, L.nx, L.ny, grad_mode) * u_scale);
        if (i >= 0 && i < L.nx && j >= 0 && j < L.ny)
            Dh[L.at(i, j)] = C(use_const ? dh_const : sD[(size_t)j * L.nx + i] * d_scale);
    }
}

template <typename C>
__global__ void pulse_fields_kernel(C* uv, C* Dh, C* tab_x, C* tab_y, PlaneLayout L, int grad_mode, double x0,
                                    double y0, double dx, double dt, Pulse pp, double dh_const, int use_const) {
    const int gw = L.nx + 2, gh = L.ny + 2;
    const size_t n = (size_t)gw * gh;
    const double us = dt / dx, ds = dt / (dx * dx);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / gw) - 1, i = (int)(k % gw) - 1;
        auto fx = [&](int ii, int jj) { return -pp.omega * (y0 + jj * dx); };
        auto fy = [&](int ii, int jj) { return pp.omega * (x0 + ii * dx); };
        uv[L.at(i, j)] = C(ghosted(fx, i, j, L.nx, L.ny, grad_mode) * us);
        uv[L.plane + L.at(i, j)] = C(ghosted(fy, i, j, L.nx, L.ny, grad_mode) * us);
        if (i < 0 || i >= L.nx || j < 0 || j >= L.ny) continue;
        const double x = x0 + i * dx, y = y0 + j * dx;
        Dh[L.at(i, j)] = C(use_const ? dh_const : pp.D0 * (1.0 + pp.D_amp * sin(M_PI * x) * sin(M_PI * y)) * ds);
        if (j == 0) {
            tab_x[i] = C(sin(M_PI * x));
            tab_x[L.nx + i] = C(cos(M_PI * x));
        }
        if (i == 0) {
            tab_y[j] = C(sin(M_PI * y));
            tab_y[L.ny + j] = C(cos(M_PI * y));
        }
    }
}

template <typename C>
__global__ void convert_source_kernel(C* dst, const double* S, PlaneLayout L, double dt) {
    const size_t n = (size_t)L.nx * L.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / L.nx), i = (int)(k - (size_t)j * L.nx);
        dst[L.at(i, j)] = C(dt * S[k]);
    }
}

__device__ __forceinline__ double pulse_phi(const PulseTime& pt, double x, double y) {
    const double rx = x - pt.cx, ry = y - pt.cy;
    return pt.amp * exp(-0.5 * (rx * rx + ry * ry) * pt.inv_s2);
}

// Third-order Hermite equilibrium (Eq. (6)) in lattice units, in FP64:
// w_i phi [1 + 3 eu + 4.5 ((eu)^2 - |u|^2/3) + 4.5 ((eu)^3 - eu |u|^2)], eu = e_i . uhat.
template <typename T>
__device__ __forceinline__ T equilibrium(int q, T phi, T u, T v) {
    const T eu = T(c_ex[q]) * u + T(c_ey[q]) * v;
    const T uu = u * u + v * v;
    return T(c_w[q]) * phi *
           (T(1) + T(3) * eu + T(4.5) * (eu * eu - uu / T(3)) + T(4.5) * (eu * eu * eu - eu * uu));
}

// Initial condition g_i(x) = g_i^eq(phi0(x), u(x)) in the pull layout: node x evaluates phi0
// once (FP64) and its nine equilibria in the compute type, and stores g_i(x) where x pulls it,
// P_i(x - e_i), periodic images included (each slot has exactly one writer).
template <typename S, typename C>
__global__ void init_eq_kernel(S* P, const C* uv, const double* phi0, PlaneLayout lp, PlaneLayout lf, double x0,
                               double y0, double dx, PulseTime pt, C phi_ref) {
    const int nx = lp.nx, ny = lp.ny;
    const size_t n = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / nx), i = (int)(k - (size_t)j * nx);
        const C phi = (C)(phi0 ? phi0[k] : pulse_phi(pt, x0 + i * dx, y0 + j * dx));
        const C u = uv[lf.at(i, j)], v = uv[lf.plane + lf.at(i, j)];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int ti = wrap(i - c_ex[q], nx), tj = wrap(j - c_ey[q], ny);
            store_with_ghosts(P + q * lp.plane, lp, ti, tj,
                              Store<S>::encode(equilibrium<C>(q, phi, u, v), (C)(c_w[q]) * phi_ref));
        }
    }
}

// Dirichlet boundary by non-equilibrium extrapolation (Sec. 3) over the buffer P that a step
// has just written.  For edge node b and its inward neighbour f (diagonal at corners):
//   g_i(b) = g_i^eq(phi_b, u_b) + g_i(f) - g_i^eq(phi(f), u_f),  g_i(f) = P_i(f - e_i),
// stored where b pulls it, P_i(b - e_i) (a ghost cell when b - e_i is outside the grid).  A
// slot P_i(y) is pulled by the node y + e_i alone, so the slots written here (pulled by edge
// nodes) and the slots read (pulled by interior nodes f) are disjoint: no thread ordering.
template <typename S, typename C>
__global__ void dirichlet_nee_kernel(S* P, const C* uv, const double* phib, PlaneLayout lp, PlaneLayout lf,
                                     C phi_ref) {
    const int nx = lp.nx, ny = lp.ny, nb = edge_count(nx, ny);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
        int i, j;
        edge_node(k, nx, ny, &i, &j);
        const int fi = i == 0 ? 1 : (i == nx - 1 ? nx - 2 : i);
        const int fj = j == 0 ? 1 : (j == ny - 1 ? ny - 2 : j);
        double gf[kQ], phif = 0.0;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            gf[q] = (double)Store<S>::decode(P[q * lp.plane + lp.at(fi - c_ex[q], fj - c_ey[q])],
                                             (C)(c_w[q]) * phi_ref);
            phif += gf[q];
        }
        const double ub = (double)uv[lf.at(i, j)], vb = (double)uv[lf.plane + lf.at(i, j)];
        const double uf = (double)uv[lf.at(fi, fj)], vf = (double)uv[lf.plane + lf.at(fi, fj)];
        const double phi_b = phib[k];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const double g = equilibrium(q, phi_b, ub, vb) + gf[q] - equilibrium(q, phif, uf, vf);
            P[q * lp.plane + lp.at(i - c_ex[q], j - c_ey[q])] = Store<S>::encode((C)g, (C)(c_w[q]) * phi_ref);
        }
    }
}

__global__ void gather_edges_kernel(double* phib, const double* phi, int nx, int ny) {
    const int nb = edge_count(nx, ny);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
        int i, j;
        edge_node(k, nx, ny, &i, &j);
        phib[k] = phi[(size_t)j * nx + i];
    }
}

// g_i(x, t_n) = P_i(x - e_i), decoded to the compute type.  x - e_i may be a ghost cell: it
// holds the periodic image, or the Dirichlet pass's value (TRTR_BC_DIRICHLET_NEE).
template <typename S, typename C>
__device__ __forceinline__ C pulled(const S* P, int q, int i, int j, const PlaneLayout& L, C phi_ref) {
    return Store<S>::decode(P[q * L.plane + L.at(i - c_ex[q], j - c_ey[q])], (C)(c_w[q]) * phi_ref);
}

template <typename S, typename C>
__device__ __forceinline__ double node_phi(const S* P, int i, int j, const PlaneLayout& L, C phi_ref) {
    double phi = 0.0;
#pragma unroll
    for (int q = 0; q < kQ; ++q) phi += (double)pulled<S, C>(P, q, i, j, L, phi_ref);
    return phi;
}

template <typename S, typename C>
__global__ void moments_kernel(double* out, const S* P, PlaneLayout L, C phi_ref) {
    const size_t n = (size_t)L.nx * L.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / L.nx), i = (int)(k - (size_t)j * L.nx);
        out[k] = node_phi<S, C>(P, i, j, L, phi_ref);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic two-value block sum (fixed tree); result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[kThreads / 32], sb[kThreads / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < kThreads / 32 ? sa[lane] : 0.0;
        b = lane < kThreads / 32 ? sb[lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

// Per-block FP64 partial sums into scratch[2 * block + {0, 1}]:
//  kind 0: sum phi;  1: sum (phi - phi_a)^2, sum phi_a^2;  2: same against phi_ref field;
//  3: number of non-finite populations;  4: number of values of ref that are not finite and > 0.
template <typename S, typename C>
__global__ void reduce_kernel(double* partial, const S* P, PlaneLayout L, C phi_ref, int kind, PulseTime pt,
                              double x0, double y0, double dx, const double* ref) {
    const size_t n = (size_t)L.nx * L.ny;
    double a = 0.0, b = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / L.nx), i = (int)(k - (size_t)j * L.nx);
        if (kind == kReduceBadField) {
            const double v = ref[k];
            a += (v > 0.0 && isfinite(v)) ? 0.0 : 1.0;
            continue;
        }
        if (kind == kReduceNonFinite) {
            for (int q = 0; q < kQ; ++q) {
                const double v = (double)pulled<S, C>(P, q, i, j, L, phi_ref);
                a += isfinite(v) ? 0.0 : 1.0;
            }
            continue;
        }
        const double phi = node_phi<S, C>(P, i, j, L, phi_ref);
        if (kind == kReduceMass) {
            a += phi;
        } else {
            const double r = kind == kReducePulse ? pulse_phi(pt, x0 + i * dx, y0 + j * dx) : ref[k];
            const double d = phi - r;
            a += d * d;
            b += r * r;
        }
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

__global__ void finish_kernel(double* out, const double* partial, int nblocks) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

template <typename S, typename C>
__global__ void get_pop_kernel(double* g, const S* P, PlaneLayout L, C phi_ref) {
    const size_t n = (size_t)L.nx * L.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / L.nx), i = (int)(k - (size_t)j * L.nx);
        for (int q = 0; q < kQ; ++q) g[q * n + k] = (double)pulled<S, C>(P, q, i, j, L, phi_ref);
    }
}

template <typename S, typename C>
__global__ void set_pop_kernel(S* P, const double* g, PlaneLayout L, C phi_ref) {
    const size_t n = (size_t)L.nx * L.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / L.nx), i = (int)(k - (size_t)j * L.nx);
        for (int q = 0; q < kQ; ++q) {
            const int si = wrap(i + c_ex[q], L.nx), sj = wrap(j + c_ey[q], L.ny);
            store_with_ghosts(P + q * L.plane, L, i, j,
                              Store<S>::encode((C)g[q * n + (size_t)sj * L.nx + si], (C)(c_w[q]) * phi_ref));
        }
    }
}

template <typename S, typename C>
__global__ void sample_kernel(double* out, const long* nodes, int count, const S* P, PlaneLayout L, C phi_ref) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * kQ) return;
    const int s = t / kQ, q = t - s * kQ;
    const long k = nodes[s];
    const int j = (int)(k / L.nx), i = (int)(k - (long)j * L.nx);
    out[t] = (double)pulled<S, C>(P, q, i, j, L, phi_ref);
}

int grid_for(const trtr_ctx* ctx, size_t n) {
    const size_t want = (n + kThreads - 1) / kThreads;
    const size_t cap = (size_t)ctx->num_sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

template <typename F>
cudaError_t dispatch(trtr_ctx* ctx, F&& f) {
    switch (ctx->p.precision) {
        case TRTR_F64: f((double*)nullptr, (double*)nullptr); break;
        case TRTR_F32: f((float*)nullptr, (float*)nullptr); break;
        case TRTR_F16_OFS: f((__half*)nullptr, (float*)nullptr); break;
        case TRTR_BF16_OFS: f((__nv_bfloat16*)nullptr, (float*)nullptr); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_convert_fields(trtr_ctx* ctx, const double* ux, const double* uy, const double* D) {
    const size_t n = (size_t)(ctx->p.nx + 2) * (ctx->p.ny + 2);
    const double us = ctx->p.dt / ctx->p.dx, ds = ctx->p.dt / (ctx->p.dx * ctx->p.dx);
    const int use_const = ctx->p.tau1_const > 0.0;
    const double dh = use_const ? (ctx->p.tau1_const - 0.5) / 3.0 : 0.0;
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using C = std::remove_pointer_t<decltype(cp)>;
        (void)sp;
        convert_fields_kernel<C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(
            (C*)ctx->uv, (C*)ctx->Dh, ux, uy, D, ctx->lf, ctx->p.grad_mode, us, ds, dh, use_const);
    });
}

cudaError_t launch_pulse_fields(trtr_ctx* ctx) {
    const size_t n = (size_t)(ctx->p.nx + 2) * (ctx->p.ny + 2);
    const int use_const = ctx->p.tau1_const > 0.0;
    const double dh = use_const ? (ctx->p.tau1_const - 0.5) / 3.0 : 0.0;
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using C = std::remove_pointer_t<decltype(cp)>;
        (void)sp;
        pulse_fields_kernel<C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(
            (C*)ctx->uv, (C*)ctx->Dh, (C*)ctx->tab_x, (C*)ctx->tab_y, ctx->lf, ctx->p.grad_mode, ctx->p.x0, ctx->p.y0,
            ctx->p.dx, ctx->p.dt, ctx->pulse, dh, use_const);
    });
}

cudaError_t launch_convert_source(trtr_ctx* ctx, const double* S, int buffer) {
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using C = std::remove_pointer_t<decltype(cp)>;
        (void)sp;
        convert_source_kernel<C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(
            (C*)ctx->S + (size_t)buffer * ctx->lf.plane, S, ctx->lf, ctx->p.dt);
    });
}

cudaError_t launch_init_equilibrium(trtr_ctx* ctx, const double* phi0) {
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    const PulseTime pt = pulse_at(ctx->pulse, 0.0);
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        init_eq_kernel<S, C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(
            (S*)ctx->pop[ctx->cur], (const C*)ctx->uv, phi0, ctx->lp, ctx->lf, ctx->p.x0, ctx->p.y0, ctx->p.dx, pt,
            (C)ctx->p.phi_ref);
    });
}

cudaError_t launch_moments(trtr_ctx* ctx, double* phi_out) {
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        moments_kernel<S, C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(phi_out, (const S*)ctx->pop[ctx->cur],
                                                                             ctx->lp, (C)ctx->p.phi_ref);
    });
}

cudaError_t launch_reduce(trtr_ctx* ctx, int kind, const double* ref) {
    const PulseTime pt = pulse_at(ctx->pulse, (double)ctx->step * ctx->p.dt);
    ctx->launches += 2;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        reduce_kernel<S, C><<<ctx->red_blocks, kThreads, 0, ctx->stream>>>(
            ctx->scratch, (const S*)ctx->pop[ctx->cur], ctx->lp, (C)ctx->p.phi_ref, kind, pt, ctx->p.x0, ctx->p.y0,
            ctx->p.dx, ref);
        finish_kernel<<<1, kThreads, 0, ctx->stream>>>(ctx->dres, ctx->scratch, ctx->red_blocks);
    });
}

cudaError_t launch_get_populations(trtr_ctx* ctx, double* g) {
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        get_pop_kernel<S, C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>(g, (const S*)ctx->pop[ctx->cur], ctx->lp,
                                                                             (C)ctx->p.phi_ref);
    });
}

cudaError_t launch_set_populations(trtr_ctx* ctx, const double* g) {
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        set_pop_kernel<S, C><<<grid_for(ctx, n), kThreads, 0, ctx->stream>>>((S*)ctx->pop[ctx->cur], g, ctx->lp,
                                                                             (C)ctx->p.phi_ref);
    });
}

cudaError_t launch_sample(trtr_ctx* ctx, const long* nodes, int count, double* out) {
    ctx->launches += 1;
    const int total = count * kQ;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        sample_kernel<S, C><<<(total + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
            out, nodes, count, (const S*)ctx->pop[ctx->cur], ctx->lp, (C)ctx->p.phi_ref);
    });
}

cudaError_t launch_gather_edges(trtr_ctx* ctx, const double* phi_b) {
    const int nb = edge_count(ctx->p.nx, ctx->p.ny);
    ctx->launches += 1;
    gather_edges_kernel<<<(nb + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(ctx->phib, phi_b, ctx->p.nx,
                                                                                      ctx->p.ny);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet(trtr_ctx* ctx, void* P) {
    const int nb = edge_count(ctx->p.nx, ctx->p.ny);
    ctx->launches += 1;
    return dispatch(ctx, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        dirichlet_nee_kernel<S, C><<<(nb + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
            (S*)P, (const C*)ctx->uv, ctx->phib, ctx->lp, ctx->lf, (C)ctx->p.phi_ref);
    });
}

TRTR_BOUNDS_TAKE(aux)

}  // namespace trtr
