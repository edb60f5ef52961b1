// trtr_adjoint.cu -- discrete adjoint of the TRT-R step (Eq. (14)) for gradients of a
// function J of the final phi with respect to the diffusivity field D(x).
//
// Forward (trtr_forward_record): n steps of the ordinary step kernel, keeping a copy of
// the state every k steps (k = ceil(sqrt(n)) by default).  Backward (trtr_adjoint): for
// each segment, last to first, the state at the segment start is copied into a pool and
// the segment's states are recomputed by the step kernel; then one backward kernel per
// step runs from the segment's end to its start.  Total work: two forward sweeps and one
// backward sweep; memory: about 2 sqrt(n) states.
//
// Notation (lattice units, S = 0).  The stored array holds P_i(x) = post_i(g(x)) with
// g_i(x) = P_i(x - e_i); Q_i(x) = dJ/dP_i(x).  Per node the step is
//   raw moments (phi, j, Pi) of g  ->  Hermite coefficients c  ->  post = R c,
//   c0 = phi, c1 = (1-k1) phi u + kh phi a + k1 j, c2 = (1-k2) phi (u u - 1/3 I) + k2 Pi,
//   c3 = phi (u_x^2 u_y, u_x u_y^2),  post_i = w_i [c0 + 3 e.c1 + 4.5 H2_i:c2 + 13.5 H3_i.c3],
// with k1 = 1 - 1/tau1, kh = 1 - 1/(2 tau1), k2 = 1 - 1/tau2.  Hence, with mu = Q^{n+1}(x):
//   r = R^T mu  (r0 = sum w mu, r1 = 3 sum w mu e, r2 = 4.5 sum w mu H2, r3 = 13.5 sum w mu H3),
//   lambda^n_i(x) = dJ/dg^n_i(x) = [moments^T  relax^T  r]_i,   Q^n_i(x - e_i) = lambda^n_i(x),
//   dJ/dD(x) += dtau1/dD [ r1 . dc1/dtau1 + dtau2/dtau1  r2 : dc2/dtau2 ],
//   dc1/dtau1 = (j - phi u)/tau1^2 + phi a/(2 tau1^2),   dc2/dtau2 = (Pi - phi/3 I - phi u u)/tau2^2,
//   dtau1/dD = 3 dt/dx^2,  dtau2/dtau1 = -Lambda/(tau1 - 1/2)^2 (magic) or 0 (fixed tau2).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include "trtr_internal.cuh"
#include "trtr_trace.h"

struct trtr_adjoint_state {
    long n0, steps;
    int interval, nseg;
    size_t state_bytes;
    std::vector<void*> ckpt;
    std::vector<void*> pool;
    std::vector<CUtensorMap> pool_maps;
    std::vector<CUtensorMap> pool_maps2;  // the two-step kernel's maps of the pool (FP32)
    bool two;                             // the recomputation takes pairs of steps per launch
    void* Q[2];
    double* grad;
    trtr::PlaneLayout lq;
};

namespace trtr {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <typename C>
__global__ void adj_init_kernel(C* Q, const double* dJ, PlaneLayout lq) {
    // Q_i(x) = dJ/dP_i(x) = dJ/dg^N_i(x + e_i) = dJ/dphi(x + e_i)
    const size_t n = (size_t)lq.nx * lq.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / lq.nx), i = (int)(k - (size_t)j * lq.nx);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int si = wrapi(i + lattice_ex(q), lq.nx), sj = wrapi(j + lattice_ey(q), lq.ny);
            Q[q * lq.plane + lq.at(i, j)] = C(dJ[(size_t)sj * lq.nx + si]);
        }
    }
}

template <typename C>
__device__ __forceinline__ C wq(int q) {
    return q == 0 ? C(4.0 / 9.0) : (q < 5 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}

template <typename S, typename C>
__global__ void __launch_bounds__(kThreads)
    adj_step_kernel(const S* __restrict__ P, const C* __restrict__ Qin, C* __restrict__ Qout, double* grad,
                    const typename Store<S>::C* __restrict__ uv, const typename Store<S>::C* __restrict__ Dh,
                    PlaneLayout lp, PlaneLayout lf,
                    PlaneLayout lq, C phi_ref, int tau2_fixed, C magic, C w2_fixed, double dtau1_dD, int d_enters) {
    // programmatic dependent launch (as the step kernel): let the next launch be set up, then
    // wait for the kernels before this one
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const size_t n = (size_t)lp.nx * lp.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / lp.nx), i = (int)(k - (size_t)j * lp.nx);
        C g[kQ], wm[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            // pull (the ghost cells hold the periodic images)
            g[q] = C(Store<S>::decode(P[q * lp.plane + lp.at(i - lattice_ex(q), j - lattice_ey(q))],
                                      wq<typename Store<S>::C>(q) * (typename Store<S>::C)phi_ref));
            wm[q] = wq<C>(q) * Qin[q * lq.plane + lq.at(i, j)];
        }
        const size_t o = lf.at(i, j);
        const C ux = C(uv[o]), uy = C(uv[lf.plane + o]);
        const C dxux = C(0.5) * (C(uv[o + 1]) - C(uv[o - 1]));
        const C dxuy = C(0.5) * (C(uv[lf.plane + o + 1]) - C(uv[lf.plane + o - 1]));
        const C dyux = C(0.5) * (C(uv[o + lf.pitch]) - C(uv[o - lf.pitch]));
        const C dyuy = C(0.5) * (C(uv[lf.plane + o + lf.pitch]) - C(uv[lf.plane + o - lf.pitch]));
        const C ax = ux * dxux + uy * dyux, ay = ux * dxuy + uy * dyuy;
        const C t1m = C(3) * C(Dh[o]);
        const C w1 = C(1) / (C(0.5) + t1m);
        const C w2 = tau2_fixed ? w2_fixed : t1m / (C(0.5) * t1m + magic);
        const C k1 = C(1) - w1, k2 = C(1) - w2, kh = C(1) - C(0.5) * w1;

        // raw moments of g
        const C phi = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
        const C jx = g[1] - g[2] + g[5] - g[6] + g[7] - g[8];
        const C jy = g[3] - g[4] + g[5] - g[6] - g[7] + g[8];
        const C pd = g[5] + g[6] + g[7] + g[8];
        const C pxx = g[1] + g[2] + pd, pyy = g[3] + g[4] + pd, pxy = g[5] + g[6] - g[7] - g[8];

        // r = R^T mu
        const C r0 = wm[0] + wm[1] + wm[2] + wm[3] + wm[4] + wm[5] + wm[6] + wm[7] + wm[8];
        const C sx = wm[1] - wm[2] + wm[5] - wm[6] + wm[7] - wm[8];
        const C sy = wm[3] - wm[4] + wm[5] - wm[6] - wm[7] + wm[8];
        const C wd = wm[5] + wm[6] + wm[7] + wm[8];
        const C sxx = wm[1] + wm[2] + wd, syy = wm[3] + wm[4] + wd, sxy = wm[5] + wm[6] - wm[7] - wm[8];
        const C sxxy = wm[5] - wm[6] - wm[7] + wm[8], sxyy = wm[5] - wm[6] + wm[7] - wm[8];
        const C r1x = C(3) * sx, r1y = C(3) * sy;
        const C rxx = C(4.5) * (sxx - r0 / C(3)), ryy = C(4.5) * (syy - r0 / C(3)), rxy = C(9) * sxy;
        const C r3a = C(13.5) * (sxxy - sy / C(3)), r3b = C(13.5) * (sxyy - sx / C(3));

        // relax^T r  ->  adjoints of the raw moments
        const C nphi = r0 + r1x * ((C(1) - k1) * ux + kh * ax) + r1y * ((C(1) - k1) * uy + kh * ay) +
                       rxx * ((C(1) - k2) * ux * ux - k2 / C(3)) + ryy * ((C(1) - k2) * uy * uy - k2 / C(3)) +
                       rxy * (C(1) - k2) * ux * uy + r3a * ux * ux * uy + r3b * ux * uy * uy;
        const C njx = k1 * r1x, njy = k1 * r1y, nxx = k2 * rxx, nyy = k2 * ryy, nxy = k2 * rxy;

        // moments^T -> lambda, stored pushed back: Q^n_q(x - e_q) = lambda_q(x)
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int ex = lattice_ex(q), ey = lattice_ey(q);
            const C lam = nphi + njx * C(ex) + njy * C(ey) + nxx * C(ex * ex) + nyy * C(ey * ey) + nxy * C(ex * ey);
            const int ti = wrapi(i - ex, lp.nx), tj = wrapi(j - ey, lp.ny);
            Qout[q * lq.plane + lq.at(ti, tj)] = lam;
        }

        if (d_enters) {
            const C w1s = w1 * w1, w2s = w2 * w2;
            const C dc1x = w1s * (jx - phi * ux) + C(0.5) * w1s * phi * ax;
            const C dc1y = w1s * (jy - phi * uy) + C(0.5) * w1s * phi * ay;
            const C dcxx = w2s * (pxx - phi / C(3) - phi * ux * ux);
            const C dcyy = w2s * (pyy - phi / C(3) - phi * uy * uy);
            const C dcxy = w2s * (pxy - phi * ux * uy);
            const C dtau2_dtau1 = tau2_fixed ? C(0) : -magic / (t1m * t1m);
            const double contrib = (double)(r1x * dc1x + r1y * dc1y) +
                                   (double)dtau2_dtau1 * (double)(rxx * dcxx + ryy * dcyy + rxy * dcxy);
            grad[k] += dtau1_dD * contrib;
        }
    }
}

int grid_for(const trtr_ctx* ctx) {
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    const size_t want = (n + kThreads - 1) / kThreads, cap = (size_t)ctx->num_sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

// Arithmetic type of the adjoint sweep (lambda recursion and gradient terms).
#ifndef TRTR_ADJ_F64
#define TRTR_ADJ_F64 0
#endif
using AdjF = std::conditional_t<TRTR_ADJ_F64 != 0, double, float>;

template <typename F>
cudaError_t dispatch(trtr_ctx* ctx, F&& f) {
    switch (ctx->p.precision) {
        case TRTR_F64: f((double*)nullptr, (double*)nullptr); break;
        case TRTR_F32: f((float*)nullptr, (AdjF*)nullptr); break;
        case TRTR_F16_OFS: f((__half*)nullptr, (AdjF*)nullptr); break;
        case TRTR_BF16_OFS: f((__nv_bfloat16*)nullptr, (AdjF*)nullptr); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int adj_csize(const trtr_ctx* ctx) { return ctx->p.precision == TRTR_F64 ? 8 : (int)sizeof(AdjF); }

}  // namespace

void free_adjoint(trtr_ctx* ctx) {
    trtr_adjoint_state* a = ctx->adj;
    if (!a) return;
    cudaStreamSynchronize(ctx->stream);
    for (void* p : a->ckpt) cudaFree(p);
    for (void* p : a->pool) cudaFree(p);
    if (a->Q[0]) cudaFree(a->Q[0]);
    if (a->Q[1]) cudaFree(a->Q[1]);
    if (a->grad) cudaFree(a->grad);
    cudaGetLastError();
    delete a;
    ctx->adj = nullptr;
}

TRTR_BOUNDS_TAKE(adjoint)

}  // namespace trtr

namespace {

trtr_status adj_fail(trtr_ctx* ctx, trtr_status s, const char* msg) {
    snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
    return s;
}

}  // namespace

extern "C" {

trtr_status trtr_forward_record(trtr_ctx* ctx, long steps, int interval) {
    trtr::TraceRange trace("trtr_forward_record");
    if (!ctx) return TRTR_EINVAL;
    if (steps < 1 || interval < 0) return adj_fail(ctx, TRTR_EINVAL, "steps >= 1 and interval >= 0 required");
    if (!ctx->initialized) return adj_fail(ctx, TRTR_ESTATE, "populations not initialised");
    if (ctx->p.src_mode != TRTR_SRC_NONE) return adj_fail(ctx, TRTR_EINVAL, "the adjoint supports S = 0 only");
    if (ctx->p.bc_mode != TRTR_BC_PERIODIC)
        return adj_fail(ctx, TRTR_EINVAL, "the adjoint supports periodic boundaries only");
    trtr::free_adjoint(ctx);
    trtr_adjoint_state* a = new (std::nothrow) trtr_adjoint_state();
    if (!a) return TRTR_ENOMEM;
    ctx->adj = a;
    a->n0 = ctx->step;
    a->steps = steps;
    a->interval = interval > 0 ? interval : (int)ceil(sqrt((double)steps));
    if (a->interval > steps) a->interval = (int)steps;
    a->nseg = (int)((steps + a->interval - 1) / a->interval);
    a->state_bytes = trtr::kQ * ctx->lp.plane * ctx->esize;
    a->lq = trtr::make_layout(ctx->p.nx, ctx->p.ny, trtr::adj_csize(ctx), 1);
    const size_t qbytes = trtr::kQ * a->lq.plane * trtr::adj_csize(ctx);
    bool ok = cudaMalloc(&a->Q[0], qbytes) == cudaSuccess && cudaMalloc(&a->Q[1], qbytes) == cudaSuccess &&
              cudaMalloc(&a->grad, (size_t)ctx->p.nx * ctx->p.ny * sizeof(double)) == cudaSuccess;
    for (int s = 0; ok && s < a->nseg; ++s) {
        void* p = nullptr;
        ok = cudaMalloc(&p, a->state_bytes) == cudaSuccess;
        if (ok) a->ckpt.push_back(p);
    }
    a->two = trtr::two_step_applies(ctx);
    for (int s = 0; ok && s < a->interval; ++s) {
        void* p = nullptr;
        ok = cudaMalloc(&p, a->state_bytes) == cudaSuccess;
        if (ok) {
            a->pool.push_back(p);
            CUtensorMap m;
            ok = trtr::encode_pop_map(ctx, p, &m) == cudaSuccess;
            a->pool_maps.push_back(m);
            if (ok && a->two) {
                ok = trtr::encode_pop_map2(ctx, p, &m) == cudaSuccess;
                a->pool_maps2.push_back(m);
            }
        }
    }
    if (!ok) {
        cudaGetLastError();
        trtr::free_adjoint(ctx);
        return adj_fail(ctx, TRTR_ENOMEM, "cannot allocate the checkpoints of the adjoint");
    }
    // the recorded run keeps only the checkpoint states, so pairs of steps between two
    // checkpoints may run as one launch of the two-step kernel (the same states bit for bit)
    const bool two = trtr::two_step_applies(ctx);
    for (long k = 0; k < steps;) {
        if (k % a->interval == 0 &&
            cudaMemcpyAsync(a->ckpt[k / a->interval], ctx->pop[ctx->cur], a->state_bytes, cudaMemcpyDeviceToDevice,
                            ctx->stream) != cudaSuccess)
            return adj_fail(ctx, TRTR_ECUDA, "checkpoint copy failed");
        const long to_checkpoint = a->interval - k % a->interval;
        if (two && to_checkpoint >= 2 && steps - k >= 2) {
            if (!ctx->fld2_ready) {
                if (trtr::launch_pack_fields2(ctx) != cudaSuccess) return adj_fail(ctx, TRTR_ECUDA, "field packing failed");
                ctx->fld2_ready = true;
            }
            if (!ctx->ghost2_ready && trtr::launch_refresh_ghosts2(ctx) != cudaSuccess)
                return adj_fail(ctx, TRTR_ECUDA, "ghost refresh failed");
            if (trtr::launch_step2(ctx) != cudaSuccess) return adj_fail(ctx, TRTR_ECUDA, "step launch failed");
            ctx->launches += 1;
            ctx->cur ^= 1;
            ctx->ghost2_ready = true;
            ctx->step += 2;
            k += 2;
        } else {
            if (trtr::launch_step(ctx) != cudaSuccess) return adj_fail(ctx, TRTR_ECUDA, "step launch failed");
            ctx->launches += 1;
            ctx->cur ^= 1;
            ctx->ghost2_ready = false;
            ctx->step += 1;
            k += 1;
        }
    }
    return TRTR_OK;
}

trtr_status trtr_adjoint(trtr_ctx* ctx, const double* dJ_dphi, int on_device, double* grad_D, int grad_on_device) {
    trtr::TraceRange trace("trtr_adjoint");
    if (!ctx) return TRTR_EINVAL;
    if (!dJ_dphi || !grad_D) return adj_fail(ctx, TRTR_EINVAL, "dJ_dphi and grad_D are required");
    trtr_adjoint_state* a = ctx->adj;
    if (!a || ctx->step != a->n0 + a->steps)
        return adj_fail(ctx, TRTR_ESTATE, "no recorded forward run ending at the current step");
    const size_t n = (size_t)ctx->p.nx * ctx->p.ny;
    cudaStream_t st = ctx->stream;
    const double* dJ = dJ_dphi;
    double* stage = nullptr;
    if (!on_device) {
        if (cudaMalloc(&stage, n * sizeof(double)) != cudaSuccess) return TRTR_ENOMEM;
        if (cudaMemcpyAsync(stage, dJ_dphi, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaFree(stage);
            return TRTR_ECUDA;
        }
        dJ = stage;
    }
    const double dtau1_dD = 3.0 * ctx->p.dt / (ctx->p.dx * ctx->p.dx);
    const int d_enters = !(ctx->p.tau1_const > 0.0);
    const int grid = trtr::grid_for(ctx);
    cudaError_t e = cudaMemsetAsync(a->grad, 0, n * sizeof(double), st);
    if (e == cudaSuccess)
        e = trtr::dispatch(ctx, [&](auto* sp, auto* cp) {
            using C = std::remove_pointer_t<decltype(cp)>;
            (void)sp;
            trtr::adj_init_kernel<C><<<grid, trtr::kThreads, 0, st>>>((C*)a->Q[0], dJ, a->lq);
        });
    int qc = 0;
    for (int seg = a->nseg - 1; seg >= 0 && e == cudaSuccess; --seg) {
        const long s0 = (long)seg * a->interval;
        const long len = a->steps - s0 < a->interval ? a->steps - s0 : a->interval;
        e = cudaMemcpyAsync(a->pool[0], a->ckpt[seg], a->state_bytes, cudaMemcpyDeviceToDevice, st);
        // recompute the segment's states: pairs through the two-step kernel, which stores the
        // intermediate state as well (FP32; the checkpoint may carry only the one-wide ghost
        // frame, so its outer ring is refreshed first), a last odd step by the one-step kernel
        const bool pairs = a->two && len >= 3;
        if (pairs && e == cudaSuccess) e = trtr::launch_refresh_ghosts2_buffer(ctx, a->pool[0]);
        long recompute_launches = 0;
        for (long k = 0; k + 1 < len && e == cudaSuccess; ++recompute_launches) {
            if (pairs && k + 2 < len) {
                e = trtr::launch_step2_from(ctx, &a->pool_maps2[k], a->pool[k + 2], a->pool[k + 1], a->n0 + s0 + k);
                k += 2;
            } else {
                e = trtr::launch_step_from(ctx, &a->pool_maps[k], a->pool[k + 1], a->n0 + s0 + k);
                k += 1;
            }
        }
        for (long k = len - 1; k >= 0 && e == cudaSuccess; --k) {
            cudaError_t le = cudaSuccess;
            e = trtr::dispatch(ctx, [&](auto* sp, auto* cp) {
                using S = std::remove_pointer_t<decltype(sp)>;
                using C = std::remove_pointer_t<decltype(cp)>;
                using F = typename trtr::Store<S>::C;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(grid);
                cfg.blockDim = dim3(trtr::kThreads);
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                attr[0].val.programmaticStreamSerializationAllowed = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                le = cudaLaunchKernelEx(&cfg, trtr::adj_step_kernel<S, C>, (const S*)a->pool[k], (const C*)a->Q[qc],
                                   (C*)a->Q[qc ^ 1], a->grad, (const F*)ctx->uv, (const F*)ctx->Dh, ctx->lp, ctx->lf,
                                   a->lq, (C)ctx->p.phi_ref, (int)(ctx->p.tau2_mode == TRTR_TAU2_FIXED),
                                   (C)ctx->p.magic,
                                   (C)(ctx->p.tau2_mode == TRTR_TAU2_FIXED ? 1.0 / ctx->p.tau2 : 0.0), dtau1_dD,
                                   d_enters);
            });
            if (e == cudaSuccess) e = le;
            qc ^= 1;
        }
        ctx->launches += recompute_launches + len;  // the recomputation and the adjoint steps
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad_D, a->grad, n * sizeof(double),
                            grad_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (stage) cudaFree(stage);
    if (e != cudaSuccess || es != cudaSuccess) {
        cudaGetLastError();
        return adj_fail(ctx, TRTR_ECUDA, cudaGetErrorString(e != cudaSuccess ? e : es));
    }
    return TRTR_OK;
}

}  // extern "C"
