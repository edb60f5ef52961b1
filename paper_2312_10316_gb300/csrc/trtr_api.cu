// trtr_api.cu -- the C ABI declared in include/trtr.h: validation, device memory of a
// context, ping-pong bookkeeping and the host side of every call.  All compute runs in the
// kernels of trtr_step.cu and trtr_aux.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "trtr_internal.cuh"
#include "trtr_trace.h"

namespace trtr {
cudaError_t bounds_take_all(cudaStream_t s, unsigned long long* out) {
    out[0] = out[1] = out[2] = 0ull;
    cudaError_t (*units[])(cudaStream_t, unsigned long long*) = {bounds_take_step, bounds_take_aux, bounds_take_batch,
                                                                  bounds_take_adjoint, bounds_take_step2};
    for (auto take : units) {
        unsigned long long u[3];
        const cudaError_t e = take(s, u);
        if (e != cudaSuccess) return e;
        if (u[0] != 0ull && out[0] == 0ull) {
            out[1] = u[1];
            out[2] = u[2];
        }
        out[0] += u[0];
    }
    return cudaSuccess;
}
}  // namespace trtr

namespace {

constexpr int kAbiVersion = 3;
constexpr uint64_t kSaveMagic = 0x3152545254ULL;  // "TRTR1"

struct SaveHeader {
    uint64_t magic;
    int32_t nx, ny, precision, src_mode;
    int64_t step;
    int32_t S_cur, S_prev;
    uint64_t pop_bytes, src_bytes;
};

trtr_status fail(trtr_ctx* ctx, trtr_status s, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

trtr_status cuda_fail(trtr_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, TRTR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define TRTR_CUDA(ctx, call, where)                     \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

size_t storage_size(int precision) {
    switch (precision) {
        case TRTR_F64: return 8;
        case TRTR_F32: return 4;
        case TRTR_F16_OFS:
        case TRTR_BF16_OFS: return 2;
        default: return 0;
    }
}

size_t n_nodes(const trtr_ctx* ctx) { return (size_t)ctx->p.nx * (size_t)ctx->p.ny; }

// Device staging buffer of at least `doubles` doubles.
trtr_status ensure_tmp(trtr_ctx* ctx, size_t doubles) {
    if (ctx->dtmp_len >= doubles) return TRTR_OK;
    if (ctx->dtmp) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->dtmp);
        ctx->dtmp = nullptr;
        ctx->dtmp_len = 0;
    }
    if (cudaMalloc(&ctx->dtmp, doubles * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TRTR_ENOMEM, "cannot allocate %zu bytes of staging memory", doubles * sizeof(double));
    }
    ctx->dtmp_len = doubles;
    return TRTR_OK;
}

// Stages `count` doubles of caller input on the device into slot `slot` of the staging
// buffer; returns the device pointer to read.  The caller must have sized the buffer for
// every slot of the call with ensure_tmp first: growing it frees the old buffer, which
// would invalidate pointers to slots staged earlier in the same call.
trtr_status stage_in(trtr_ctx* ctx, const double* src, size_t count, int on_device, size_t slot,
                     const double** dev) {
    if (on_device) {
        *dev = src;
        return TRTR_OK;
    }
    if (ctx->dtmp_len < (slot + 1) * count)
        return fail(ctx, TRTR_ESTATE, "internal: staging buffer not sized for slot %zu", slot);
    double* d = ctx->dtmp + slot * count;
    TRTR_CUDA(ctx, cudaMemcpyAsync(d, src, count * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
              "host-to-device copy");
    *dev = d;
    return TRTR_OK;
}

trtr_status check_launch(trtr_ctx* ctx, cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    return TRTR_OK;
}

// Synchronises the context's stream and reports a step kernel whose bounded wait gave up.  The
// flag is cleared once reported, so the context stays usable.
trtr_status sync_and_check(trtr_ctx* ctx, const char* where) {
    int* hflag = reinterpret_cast<int*>(ctx->hres + 3);
    TRTR_CUDA(ctx, cudaMemcpyAsync(hflag, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), where);
    TRTR_CUDA(ctx, cudaStreamSynchronize(ctx->stream), where);
    if (*hflag != 0) {
        TRTR_CUDA(ctx, cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->stream), where);
        return fail(ctx, TRTR_ETIMEOUT, "%s: a kernel timed out waiting for its loads", where);
    }
#if TRTR_BOUNDS_CHECK
    unsigned long long log[3];
    TRTR_CUDA(ctx, trtr::bounds_take_all(ctx->stream, log), where);
    if (log[0] != 0ull)
        return fail(ctx, TRTR_EBOUNDS, "%s: %llu out-of-bounds accesses; the first of kind %llu at (%d, %d)", where,
                    log[0], log[1], (int)(unsigned)(log[2] & 0xffffffffull), (int)(unsigned)(log[2] >> 32));
#endif
    return TRTR_OK;
}

trtr_status reduce(trtr_ctx* ctx, int kind, const double* ref_dev, double out[2]) {
    trtr::TraceRange trace("trtr reduce");
    trtr_status s = check_launch(ctx, trtr::launch_reduce(ctx, kind, ref_dev), "reduction launch");
    if (s != TRTR_OK) return s;
    TRTR_CUDA(ctx, cudaMemcpyAsync(ctx->hres, ctx->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
              "reduction result copy");
    s = sync_and_check(ctx, "reduction");
    if (s != TRTR_OK) return s;
    out[0] = ctx->hres[0];
    out[1] = ctx->hres[1];
    return TRTR_OK;
}

bool ready(trtr_ctx* ctx, trtr_status* s) {
    if (!ctx->initialized) {
        *s = fail(ctx, TRTR_ESTATE, "populations not initialised (call trtr_init_equilibrium or trtr_set_populations)");
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

int trtr_abi_version(void) { return kAbiVersion; }

int trtr_bounds_checked(void) { return TRTR_BOUNDS_CHECK; }

trtr_status trtr_bounds_report(unsigned long long out[3]) {
    if (!out) return TRTR_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return TRTR_ECUDA;
    return trtr::bounds_take_all(0, out) == cudaSuccess ? TRTR_OK : TRTR_ECUDA;
}

const char* trtr_status_str(trtr_status s) {
    switch (s) {
        case TRTR_OK: return "ok";
        case TRTR_EINVAL: return "invalid argument";
        case TRTR_ENOMEM: return "out of device memory";
        case TRTR_ECUDA: return "CUDA error";
        case TRTR_EUNSTABLE: return "non-finite populations (unstable run)";
        case TRTR_ETIMEOUT: return "timed out";
        case TRTR_ESTATE: return "call out of order";
        case TRTR_EBOUNDS: return "out-of-bounds access caught (bounds-checked build)";
        default: return "unknown status";
    }
}

const char* trtr_last_error(const trtr_ctx* ctx) { return ctx ? ctx->err : "null context"; }

void trtr_d2q9(int* ex, int* ey, double* w) {
    static const int EX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    static const int EY[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    for (int i = 0; i < 9; ++i) {
        if (ex) ex[i] = EX[i];
        if (ey) ey[i] = EY[i];
        if (w) w[i] = W[i];
    }
}

trtr_status trtr_create(const trtr_params* p, void* cuda_stream, trtr_ctx** out) {
    if (!out) return TRTR_EINVAL;
    *out = nullptr;
    if (!p) return TRTR_EINVAL;
    if (p->nx < 1 || p->ny < 1) return TRTR_EINVAL;
    if (!(p->dx > 0.0) || !(p->dt > 0.0) || !isfinite(p->dx) || !isfinite(p->dt)) return TRTR_EINVAL;
    if (!isfinite(p->x0) || !isfinite(p->y0)) return TRTR_EINVAL;
    const size_t es = storage_size(p->precision);
    if (es == 0) return TRTR_EINVAL;
    if (p->tau2_mode != TRTR_TAU2_MAGIC && p->tau2_mode != TRTR_TAU2_FIXED) return TRTR_EINVAL;
    if (p->tau2_mode == TRTR_TAU2_MAGIC && !(p->magic > 0.0 && isfinite(p->magic))) return TRTR_EINVAL;
    if (p->tau2_mode == TRTR_TAU2_FIXED && !(p->tau2 > 0.5 && isfinite(p->tau2))) return TRTR_EINVAL;
    if (p->tau1_const != 0.0 && !(p->tau1_const > 0.5 && isfinite(p->tau1_const))) return TRTR_EINVAL;
    if (p->grad_mode != TRTR_GRAD_PERIODIC && p->grad_mode != TRTR_GRAD_ONESIDED_EDGE) return TRTR_EINVAL;
    if (p->src_mode < TRTR_SRC_NONE || p->src_mode > TRTR_SRC_PULSE) return TRTR_EINVAL;
    if (p->check_every < 0 || !isfinite(p->phi_ref)) return TRTR_EINVAL;
    if (p->bc_mode != TRTR_BC_PERIODIC && p->bc_mode != TRTR_BC_DIRICHLET_NEE) return TRTR_EINVAL;
    if (p->rounding != TRTR_ROUND_NEAREST && p->rounding != TRTR_ROUND_STOCHASTIC) return TRTR_EINVAL;
    if (p->bc_mode == TRTR_BC_DIRICHLET_NEE && (p->nx < 3 || p->ny < 3)) return TRTR_EINVAL;
    const trtr::PlaneLayout lp = trtr::make_layout(p->nx, p->ny, (int)es, trtr::kGhostP);
    const trtr::PlaneLayout lf = trtr::make_layout(p->nx, p->ny, p->precision == TRTR_F64 ? 8 : 4, trtr::kGhostF);
    if ((long long)trtr::kQ * (long long)lp.plane >= (1LL << 31) || 2LL * (long long)lf.plane >= (1LL << 31))
        return TRTR_EINVAL;

    trtr_ctx* ctx = new (std::nothrow) trtr_ctx();
    if (!ctx) return TRTR_ENOMEM;
    memset(static_cast<void*>(ctx), 0, sizeof(*ctx));
    ctx->p = *p;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->esize = (int)es;
    ctx->csize = p->precision == TRTR_F64 ? 8 : 4;
    ctx->lp = lp;
    ctx->lf = lf;
    ctx->S_cur = ctx->S_prev = -1;
    ctx->steps_per_launch = 2;
    // the two-step kernel's packed fields (FP32 or 2-byte storage, periodic, no field source; the
    // 2-byte kernel rounds the one-step kernel's node pairs, so nx is even there)
    const bool two_step_storage =
        p->precision == TRTR_F32 ||
        ((p->precision == TRTR_F16_OFS || p->precision == TRTR_BF16_OFS) && p->nx % 2 == 0);
    const bool two_step = two_step_storage && p->bc_mode == TRTR_BC_PERIODIC && p->src_mode != TRTR_SRC_FIELD &&
                          p->nx >= 2 && p->ny >= 2;
    ctx->lt = trtr::make_layout(p->nx, p->ny, 4, trtr::kGhostP);

    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return TRTR_ECUDA;
    }
    ctx->red_blocks = ctx->num_sms * 4;

    const size_t pop_bytes = trtr::kQ * lp.plane * es;
    const size_t fld_bytes = lf.plane * ctx->csize;
    struct {
        void** ptr;
        size_t bytes;
        bool zero;
    } allocs[] = {
        {&ctx->pop[0], pop_bytes, true},
        {&ctx->pop[1], pop_bytes, true},
        {&ctx->uv, 2 * fld_bytes, true},
        {&ctx->Dh, fld_bytes, true},
        {&ctx->S, p->src_mode == TRTR_SRC_FIELD ? 2 * fld_bytes : 0, true},
        {&ctx->tab_x, 2 * (size_t)p->nx * ctx->csize, true},
        {&ctx->tab_y, 2 * (size_t)p->ny * ctx->csize, true},
        {(void**)&ctx->scratch, 2 * (size_t)ctx->red_blocks * sizeof(double), false},
        {(void**)&ctx->dres, 4 * sizeof(double), false},
        {(void**)&ctx->dflag, 4 * sizeof(int), true},  // the timeout flag, then the tile counters
        {(void**)&ctx->phib,
         p->bc_mode == TRTR_BC_DIRICHLET_NEE ? (size_t)trtr::edge_count(p->nx, p->ny) * sizeof(double) : 0, true},
        {&ctx->fld2, two_step ? 5 * ctx->lt.plane * sizeof(float) : 0, true},
    };
    // fault injection for tests: TRTR_FAULT_ALLOC=k makes the k-th device allocation here fail
    const char* fault = getenv("TRTR_FAULT_ALLOC");
    const int fail_at = fault ? atoi(fault) : 0;
    int nalloc = 0;
    for (auto& a : allocs) {
        if (a.bytes == 0) continue;
        if (++nalloc == fail_at || cudaMalloc(a.ptr, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            trtr_destroy(ctx);
            return TRTR_ENOMEM;
        }
        // defined contents everywhere, padding and ghost cells included
        if (a.zero && cudaMemsetAsync(*a.ptr, 0, a.bytes, ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            trtr_destroy(ctx);
            return TRTR_ECUDA;
        }
    }
    if (cudaMallocHost((void**)&ctx->hres, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        trtr_destroy(ctx);
        return TRTR_ENOMEM;
    }
    if (trtr::encode_maps(ctx) != cudaSuccess || trtr::encode_maps2(ctx) != cudaSuccess) {
        cudaGetLastError();
        trtr_destroy(ctx);
        return TRTR_ECUDA;
    }
    *out = ctx;
    return TRTR_OK;
}

trtr_status trtr_destroy(trtr_ctx* ctx) {
    if (!ctx) return TRTR_OK;
    cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();
    trtr::free_adjoint(ctx);
    void* ptrs[] = {ctx->pop[0], ctx->pop[1],  ctx->uv,   ctx->Dh,    ctx->S,    ctx->tab_x,
                    ctx->tab_y,  ctx->scratch, ctx->dres, ctx->dflag, ctx->dtmp, ctx->phib, ctx->fld2};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (ctx->hres) cudaFreeHost(ctx->hres);
    cudaGetLastError();
    delete ctx;
    return TRTR_OK;
}

static trtr_status set_source_impl(trtr_ctx* ctx, const double* S, int on_device) {
    const size_t n = n_nodes(ctx);
    // The buffer that will hold S^n: not the one kept as S^{n-1}.
    int dst;
    if (ctx->S_cur < 0) dst = 0;
    else if (ctx->S_prev == ctx->S_cur || ctx->S_prev < 0) dst = ctx->S_cur ^ 1;
    else dst = ctx->S_cur;
    const double* dev = nullptr;
    trtr_status s = on_device ? TRTR_OK : ensure_tmp(ctx, n);
    if (s == TRTR_OK) s = stage_in(ctx, S, n, on_device, 0, &dev);
    if (s != TRTR_OK) return s;
    s = check_launch(ctx, trtr::launch_convert_source(ctx, dev, dst), "source conversion");
    if (s != TRTR_OK) return s;
    ctx->S_cur = dst;
    return TRTR_OK;
}

trtr_status trtr_set_source_prev(trtr_ctx* ctx, const double* S, int on_device) {
    if (!ctx) return TRTR_EINVAL;
    if (!S) return fail(ctx, TRTR_EINVAL, "S is NULL");
    if (ctx->p.src_mode != TRTR_SRC_FIELD) return fail(ctx, TRTR_EINVAL, "src_mode is not FIELD");
    if (ctx->S_cur < 0) return fail(ctx, TRTR_ESTATE, "set the current source (trtr_set_source) first");
    const size_t n = n_nodes(ctx);
    const int dst = ctx->S_cur ^ 1;
    const double* dev = nullptr;
    trtr_status s = on_device ? TRTR_OK : ensure_tmp(ctx, n);
    if (s == TRTR_OK) s = stage_in(ctx, S, n, on_device, 0, &dev);
    if (s != TRTR_OK) return s;
    s = check_launch(ctx, trtr::launch_convert_source(ctx, dev, dst), "source conversion");
    if (s != TRTR_OK) return s;
    ctx->S_prev = dst;
    return TRTR_OK;
}

trtr_status trtr_set_dirichlet(trtr_ctx* ctx, const double* phi_b, int on_device) {
    if (!ctx) return TRTR_EINVAL;
    if (!phi_b) return fail(ctx, TRTR_EINVAL, "phi_b is NULL");
    if (ctx->p.bc_mode != TRTR_BC_DIRICHLET_NEE) return fail(ctx, TRTR_EINVAL, "bc_mode is not DIRICHLET_NEE");
    const int nx = ctx->p.nx, ny = ctx->p.ny, nb = trtr::edge_count(nx, ny);
    if (on_device) {
        trtr_status s = check_launch(ctx, trtr::launch_gather_edges(ctx, phi_b), "edge gather");
        if (s != TRTR_OK) return s;
    } else {
        // gathered on the host; the copy is ordered after the kernels already on the stream
        double* edge = (double*)malloc((size_t)nb * sizeof(double));
        if (!edge) return fail(ctx, TRTR_ENOMEM, "host memory");
        for (int k = 0; k < nb; ++k) {
            int i, j;
            trtr::edge_node(k, nx, ny, &i, &j);
            edge[k] = phi_b[(size_t)j * nx + i];
        }
        cudaError_t e = cudaMemcpyAsync(ctx->phib, edge, (size_t)nb * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        free(edge);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "edge values copy");
    }
    ctx->dirichlet_set = true;
    return TRTR_OK;
}

trtr_status trtr_set_fields(trtr_ctx* ctx, const double* ux, const double* uy, const double* D, const double* S,
                            int on_device) {
    if (!ctx) return TRTR_EINVAL;
    if (!ux || !uy) return fail(ctx, TRTR_EINVAL, "ux and uy are required");
    if (!D && !(ctx->p.tau1_const > 0.0)) return fail(ctx, TRTR_EINVAL, "D is required unless tau1_const > 0");
    if (S && ctx->p.src_mode != TRTR_SRC_FIELD) return fail(ctx, TRTR_EINVAL, "S given but src_mode is not FIELD");
    const size_t n = n_nodes(ctx);
    const double *dux, *duy, *dD = nullptr;
    trtr_status s = on_device ? TRTR_OK : ensure_tmp(ctx, 3 * n);
    if (s == TRTR_OK) s = stage_in(ctx, ux, n, on_device, 0, &dux);
    if (s == TRTR_OK) s = stage_in(ctx, uy, n, on_device, 1, &duy);
    if (s == TRTR_OK && D) s = stage_in(ctx, D, n, on_device, 2, &dD);
    if (s != TRTR_OK) return s;
    if (D && !(ctx->p.tau1_const > 0.0)) {  // D > 0 and finite everywhere, checked on the device copy
        double r[2];
        s = reduce(ctx, trtr::kReduceBadField, dD, r);
        if (s != TRTR_OK) return s;
        if (r[0] > 0.0)
            return fail(ctx, TRTR_EINVAL, "D must be > 0 and finite at every node (%.0f nodes are not)", r[0]);
    }
    s = check_launch(ctx, trtr::launch_convert_fields(ctx, dux, duy, dD), "field conversion");
    if (s != TRTR_OK) return s;
    ctx->fields_set = true;
    ctx->fld2_ready = false;
    if (S) {
        ctx->S_cur = ctx->S_prev = -1;
        // staging slot 0 is reused; the copy into it is ordered after the conversion above
        s = set_source_impl(ctx, S, on_device);
        if (s != TRTR_OK) return s;
    }
    return TRTR_OK;
}

trtr_status trtr_set_source(trtr_ctx* ctx, const double* S, int on_device) {
    if (!ctx) return TRTR_EINVAL;
    if (!S) return fail(ctx, TRTR_EINVAL, "S is NULL");
    if (ctx->p.src_mode != TRTR_SRC_FIELD) return fail(ctx, TRTR_ESTATE, "src_mode is not TRTR_SRC_FIELD");
    return set_source_impl(ctx, S, on_device);
}

trtr_status trtr_set_pulse(trtr_ctx* ctx, double omega, double xc, double yc, double sigma0, double D0,
                           double D_amp) {
    if (!ctx) return TRTR_EINVAL;
    if (!(sigma0 > 0.0) || !(D0 >= 0.0) || !isfinite(omega) || !isfinite(xc) || !isfinite(yc) || !isfinite(D0) ||
        !isfinite(D_amp) || !isfinite(sigma0))
        return fail(ctx, TRTR_EINVAL, "bad pulse parameters");
    if (!(ctx->p.tau1_const > 0.0) && !(D0 * (1.0 - fabs(D_amp)) > 0.0))
        return fail(ctx, TRTR_EINVAL, "D0 (1 - |D_amp|) must be > 0 when tau1 comes from D");
    ctx->pulse = trtr::Pulse{omega, xc, yc, sigma0, D0, D_amp};
    trtr_status s = check_launch(ctx, trtr::launch_pulse_fields(ctx), "pulse fields");
    if (s != TRTR_OK) return s;
    ctx->pulse_set = true;
    ctx->fields_set = true;
    ctx->fld2_ready = false;
    return TRTR_OK;
}

trtr_status trtr_init_equilibrium(trtr_ctx* ctx, const double* phi0, int on_device) {
    if (!ctx) return TRTR_EINVAL;
    if (!ctx->fields_set) return fail(ctx, TRTR_ESTATE, "fields not set");
    if (!phi0 && !ctx->pulse_set) return fail(ctx, TRTR_ESTATE, "phi0 is NULL and no pulse is set");
    if (ctx->p.src_mode == TRTR_SRC_PULSE && !ctx->pulse_set)
        return fail(ctx, TRTR_ESTATE, "src_mode PULSE needs trtr_set_pulse");
    const double* dev = nullptr;
    if (phi0) {
        trtr_status s = on_device ? TRTR_OK : ensure_tmp(ctx, n_nodes(ctx));
        if (s == TRTR_OK) s = stage_in(ctx, phi0, n_nodes(ctx), on_device, 0, &dev);
        if (s != TRTR_OK) return s;
    }
    trtr_status s = check_launch(ctx, trtr::launch_init_equilibrium(ctx, dev), "init");
    if (s != TRTR_OK) return s;
    ctx->ghost2_ready = true;  // written with the whole ghost frame
    ctx->step = 0;
    ctx->initialized = true;
    ctx->S_prev = -1;
    return TRTR_OK;
}

trtr_status trtr_step(trtr_ctx* ctx, long n) {
    trtr::TraceRange trace("trtr_step");
    if (!ctx) return TRTR_EINVAL;
    if (n < 0) return fail(ctx, TRTR_EINVAL, "negative step count");
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    if (ctx->p.src_mode == TRTR_SRC_FIELD && ctx->S_cur < 0)
        return fail(ctx, TRTR_ESTATE, "src_mode FIELD needs a source (trtr_set_source)");
    if (ctx->p.src_mode == TRTR_SRC_PULSE && !ctx->pulse_set)
        return fail(ctx, TRTR_ESTATE, "src_mode PULSE needs trtr_set_pulse");
    const bool nee = ctx->p.bc_mode == TRTR_BC_DIRICHLET_NEE;
    if (nee && !ctx->dirichlet_set)
        return fail(ctx, TRTR_ESTATE, "bc_mode DIRICHLET_NEE needs boundary values (trtr_set_dirichlet)");
    const bool two = trtr::two_step_applies(ctx);
    const long every = ctx->p.check_every;
    for (long k = 0; k < n;) {
        // two steps per launch where the kernel applies, unless the step between them is one
        // that the stability check looks at
        if (two && n - k >= 2 && !(every > 0 && (ctx->step + 1) % every == 0)) {
            if (!ctx->fld2_ready) {
                cudaError_t e = trtr::launch_pack_fields2(ctx);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "field packing launch");
                ctx->fld2_ready = true;
            }
            if (!ctx->ghost2_ready) {  // after one-step launches: complete the two-wide frame
                cudaError_t e = trtr::launch_refresh_ghosts2(ctx);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "ghost refresh launch");
            }
            cudaError_t e = trtr::launch_step2(ctx);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "two-step launch");
            ctx->launches += 1;
            ctx->ghost2_ready = true;
            ctx->cur ^= 1;
            ctx->step += 2;
            k += 2;
        } else {
            cudaError_t e = trtr::launch_step(ctx);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
            ctx->launches += 1;
            ctx->ghost2_ready = false;  // the one-step kernel writes the one-wide frame
            if (nee) {
                e = trtr::launch_dirichlet(ctx, ctx->pop[ctx->cur ^ 1]);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "boundary launch");
            }
            ctx->cur ^= 1;
            ctx->step += 1;
            k += 1;
        }
        if (ctx->p.src_mode == TRTR_SRC_FIELD) ctx->S_prev = ctx->S_cur;
        if (ctx->p.check_every > 0 && (ctx->step % ctx->p.check_every) == 0) {
            double r[2];
            s = reduce(ctx, trtr::kReduceNonFinite, nullptr, r);
            if (s != TRTR_OK) return s;
            if (r[0] != 0.0)
                return fail(ctx, TRTR_EUNSTABLE, "%.0f non-finite populations after step %ld", r[0], ctx->step);
        }
    }
    return TRTR_OK;
}

trtr_status trtr_moments(trtr_ctx* ctx, double* phi_out, int on_device) {
    trtr::TraceRange trace("trtr_moments");
    if (!ctx) return TRTR_EINVAL;
    if (!phi_out) return fail(ctx, TRTR_EINVAL, "phi_out is NULL");
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    const size_t n = n_nodes(ctx);
    double* dev = phi_out;
    if (!on_device) {
        s = ensure_tmp(ctx, n);
        if (s != TRTR_OK) return s;
        dev = ctx->dtmp;
    }
    s = check_launch(ctx, trtr::launch_moments(ctx, dev), "moments");
    if (s != TRTR_OK) return s;
    if (!on_device)
        TRTR_CUDA(ctx, cudaMemcpyAsync(phi_out, dev, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                  "device-to-host copy");
    return sync_and_check(ctx, "moments");
}

trtr_status trtr_mass(trtr_ctx* ctx, double* sum_phi) {
    if (!ctx) return TRTR_EINVAL;
    if (!sum_phi) return fail(ctx, TRTR_EINVAL, "sum_phi is NULL");
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    double r[2];
    s = reduce(ctx, trtr::kReduceMass, nullptr, r);
    if (s == TRTR_OK) *sum_phi = r[0];
    return s;
}

static void finish_error(const trtr_ctx* ctx, const double r[2], double* rms, double* rel) {
    if (rms) *rms = sqrt(r[0] / (double)n_nodes(ctx));
    if (rel) *rel = r[1] > 0.0 ? sqrt(r[0] / r[1]) : sqrt(r[0]);
}

trtr_status trtr_error_vs_pulse(trtr_ctx* ctx, double* rms, double* rel_l2) {
    if (!ctx) return TRTR_EINVAL;
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    if (!ctx->pulse_set) return fail(ctx, TRTR_ESTATE, "no pulse set");
    double r[2];
    s = reduce(ctx, trtr::kReducePulse, nullptr, r);
    if (s == TRTR_OK) finish_error(ctx, r, rms, rel_l2);
    return s;
}

trtr_status trtr_error_vs(trtr_ctx* ctx, const double* phi_ref, int on_device, double* rms, double* rel_l2) {
    if (!ctx) return TRTR_EINVAL;
    if (!phi_ref) return fail(ctx, TRTR_EINVAL, "phi_ref is NULL");
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    const double* dev = nullptr;
    s = on_device ? TRTR_OK : ensure_tmp(ctx, n_nodes(ctx));
    if (s == TRTR_OK) s = stage_in(ctx, phi_ref, n_nodes(ctx), on_device, 0, &dev);
    if (s != TRTR_OK) return s;
    double r[2];
    s = reduce(ctx, trtr::kReduceField, dev, r);
    if (s == TRTR_OK) finish_error(ctx, r, rms, rel_l2);
    return s;
}

trtr_status trtr_get_populations(trtr_ctx* ctx, double* g_out, int on_device) {
    if (!ctx) return TRTR_EINVAL;
    if (!g_out) return fail(ctx, TRTR_EINVAL, "g_out is NULL");
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    const size_t n = trtr::kQ * n_nodes(ctx);
    double* dev = g_out;
    if (!on_device) {
        s = ensure_tmp(ctx, n);
        if (s != TRTR_OK) return s;
        dev = ctx->dtmp;
    }
    s = check_launch(ctx, trtr::launch_get_populations(ctx, dev), "get populations");
    if (s != TRTR_OK) return s;
    if (!on_device)
        TRTR_CUDA(ctx, cudaMemcpyAsync(g_out, dev, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                  "device-to-host copy");
    return sync_and_check(ctx, "get populations");
}

trtr_status trtr_set_populations(trtr_ctx* ctx, const double* g, int on_device, long step) {
    if (!ctx) return TRTR_EINVAL;
    if (!g || step < 0) return fail(ctx, TRTR_EINVAL, "g is NULL or step < 0");
    if (!ctx->fields_set) return fail(ctx, TRTR_ESTATE, "fields not set");
    const double* dev = nullptr;
    trtr_status s = on_device ? TRTR_OK : ensure_tmp(ctx, trtr::kQ * n_nodes(ctx));
    if (s == TRTR_OK) s = stage_in(ctx, g, trtr::kQ * n_nodes(ctx), on_device, 0, &dev);
    if (s != TRTR_OK) return s;
    s = check_launch(ctx, trtr::launch_set_populations(ctx, dev), "set populations");
    if (s == TRTR_OK) ctx->ghost2_ready = true;
    if (s != TRTR_OK) return s;
    ctx->step = step;
    ctx->initialized = true;
    ctx->S_prev = -1;
    return TRTR_OK;
}

trtr_status trtr_sample_populations(trtr_ctx* ctx, const long* nodes, int count, double* out) {
    if (!ctx) return TRTR_EINVAL;
    if (count < 0 || (count > 0 && (!nodes || !out))) return fail(ctx, TRTR_EINVAL, "bad sample arguments");
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    if (count == 0) return TRTR_OK;
    const long n = (long)n_nodes(ctx);
    for (int k = 0; k < count; ++k)
        if (nodes[k] < 0 || nodes[k] >= n) return fail(ctx, TRTR_EINVAL, "node index %ld out of range", nodes[k]);
    // staging: count longs (rounded up to doubles) followed by 9 * count doubles
    const size_t idx_d = ((size_t)count * sizeof(long) + sizeof(double) - 1) / sizeof(double);
    TRTR_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "staging");
    s = ensure_tmp(ctx, idx_d + (size_t)count * trtr::kQ);
    if (s != TRTR_OK) return s;
    long* dnodes = (long*)ctx->dtmp;
    double* dout = ctx->dtmp + idx_d;
    TRTR_CUDA(ctx, cudaMemcpyAsync(dnodes, nodes, count * sizeof(long), cudaMemcpyHostToDevice, ctx->stream),
              "host-to-device copy");
    s = check_launch(ctx, trtr::launch_sample(ctx, dnodes, count, dout), "sample");
    if (s != TRTR_OK) return s;
    TRTR_CUDA(ctx, cudaMemcpyAsync(out, dout, (size_t)count * trtr::kQ * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream),
              "device-to-host copy");
    return sync_and_check(ctx, "sample");
}

trtr_status trtr_time(const trtr_ctx* ctx, long* step, double* t) {
    if (!ctx) return TRTR_EINVAL;
    if (step) *step = ctx->step;
    if (t) *t = (double)ctx->step * ctx->p.dt;
    return TRTR_OK;
}

trtr_status trtr_save(trtr_ctx* ctx, void* host_buf, size_t* bytes) {
    if (!ctx || !bytes) return TRTR_EINVAL;
    trtr_status s;
    if (!ready(ctx, &s)) return s;
    const size_t pop_bytes = trtr::kQ * ctx->lp.plane * ctx->esize;
    const size_t src_bytes = ctx->p.src_mode == TRTR_SRC_FIELD ? 2 * ctx->lf.plane * ctx->csize : 0;
    const size_t need = sizeof(SaveHeader) + pop_bytes + src_bytes;
    if (!host_buf) {
        *bytes = need;
        return TRTR_OK;
    }
    if (*bytes < need) return fail(ctx, TRTR_EINVAL, "buffer too small (%zu < %zu)", *bytes, need);
    SaveHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kSaveMagic;
    h.nx = ctx->p.nx;
    h.ny = ctx->p.ny;
    h.precision = ctx->p.precision;
    h.src_mode = ctx->p.src_mode;
    h.step = ctx->step;
    h.S_cur = ctx->S_cur;
    h.S_prev = ctx->S_prev;
    h.pop_bytes = pop_bytes;
    h.src_bytes = src_bytes;
    char* b = (char*)host_buf;
    memcpy(b, &h, sizeof(h));
    TRTR_CUDA(ctx, cudaMemcpyAsync(b + sizeof(h), ctx->pop[ctx->cur], pop_bytes, cudaMemcpyDeviceToHost, ctx->stream),
              "save copy");
    if (src_bytes)
        TRTR_CUDA(ctx, cudaMemcpyAsync(b + sizeof(h) + pop_bytes, ctx->S, src_bytes, cudaMemcpyDeviceToHost, ctx->stream),
                  "save copy");
    s = sync_and_check(ctx, "save");
    if (s != TRTR_OK) return s;
    *bytes = need;
    return TRTR_OK;
}

trtr_status trtr_load(trtr_ctx* ctx, const void* host_buf, size_t bytes) {
    if (!ctx || !host_buf) return TRTR_EINVAL;
    if (bytes < sizeof(SaveHeader)) return fail(ctx, TRTR_EINVAL, "checkpoint too small");
    SaveHeader h;
    memcpy(&h, host_buf, sizeof(h));
    const size_t pop_bytes = trtr::kQ * ctx->lp.plane * ctx->esize;
    const size_t src_bytes = ctx->p.src_mode == TRTR_SRC_FIELD ? 2 * ctx->lf.plane * ctx->csize : 0;
    if (h.magic != kSaveMagic || h.nx != ctx->p.nx || h.ny != ctx->p.ny || h.precision != ctx->p.precision ||
        h.src_mode != ctx->p.src_mode || h.pop_bytes != pop_bytes || h.src_bytes != src_bytes ||
        bytes < sizeof(h) + pop_bytes + src_bytes || h.step < 0 || h.S_cur < -1 || h.S_cur > 1 || h.S_prev < -1 ||
        h.S_prev > 1)
        return fail(ctx, TRTR_EINVAL, "checkpoint does not match this context");
    const char* b = (const char*)host_buf;
    TRTR_CUDA(ctx, cudaMemcpyAsync(ctx->pop[ctx->cur], b + sizeof(h), pop_bytes, cudaMemcpyHostToDevice, ctx->stream),
              "load copy");
    if (src_bytes) {
        TRTR_CUDA(ctx, cudaMemcpyAsync(ctx->S, b + sizeof(h) + pop_bytes, src_bytes, cudaMemcpyHostToDevice, ctx->stream),
                  "load copy");
        ctx->S_cur = h.S_cur;
        ctx->S_prev = h.S_prev;
    }
    TRTR_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "load");
    ctx->step = h.step;
    ctx->ghost2_ready = false;  // the saved frame may be the one-step kernels' one-wide one
    ctx->initialized = true;
    return TRTR_OK;
}

trtr_status trtr_sync(trtr_ctx* ctx) {
    if (!ctx) return TRTR_EINVAL;
    trtr_status s = sync_and_check(ctx, "sync");
    if (s != TRTR_OK) return s;
    TRTR_CUDA(ctx, cudaGetLastError(), "sync");
    return TRTR_OK;
}

trtr_status trtr_check_timeout_path(trtr_ctx* ctx, long long cycles) {
    if (!ctx) return TRTR_EINVAL;
    if (cycles < 1 || cycles > (1LL << 31)) return fail(ctx, TRTR_EINVAL, "cycles must be in 1 .. 2^31");
    trtr_status s = check_launch(ctx, trtr::launch_wait_timeout(ctx, cycles), "timeout check");
    if (s != TRTR_OK) return s;
    return sync_and_check(ctx, "timeout check");
}

trtr_status trtr_check_bounds_path(trtr_ctx* ctx) {
    if (!ctx) return TRTR_EINVAL;
    trtr_status s = check_launch(ctx, trtr::launch_bounds_probe(ctx), "bounds check");
    if (s != TRTR_OK) return s;
    return sync_and_check(ctx, "bounds check");
}

trtr_status trtr_set_steps_per_launch(trtr_ctx* ctx, int k) {
    if (!ctx) return TRTR_EINVAL;
    if (k != 1 && k != 2) return fail(ctx, TRTR_EINVAL, "steps per launch must be 1 or 2");
    ctx->steps_per_launch = k;
    return TRTR_OK;
}

trtr_status trtr_get_steps_per_launch(const trtr_ctx* ctx, int* k) {
    if (!ctx || !k) return TRTR_EINVAL;
    *k = trtr::two_step_applies(ctx) ? 2 : 1;
    return TRTR_OK;
}

trtr_status trtr_launch_count(const trtr_ctx* ctx, long* launches) {
    if (!ctx || !launches) return TRTR_EINVAL;
    *launches = ctx->launches;
    return TRTR_OK;
}

}  // extern "C"
