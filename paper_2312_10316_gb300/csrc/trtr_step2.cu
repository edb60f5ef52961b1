// trtr_step2.cu -- two time steps of the evolution equation (14) per launch (temporal blocking
// of the fused TRT-R step), for FP32 storage or FP16 / BF16 offset storage (FP32 arithmetic),
// periodic boundaries and no source or the manufactured pulse source.  The node update is the
// one-step kernel's (collide_node, the same source and acceleration arithmetic, the same
// rounding of the stored 2-byte values), so two steps here give the bits of two one-step
// launches; what changes is the data movement: the populations are read and written once per
// two steps.
//
// Tile: BX x BY output nodes (i0.., j0..).  One TMA box of depth 9 brings P (the previous
// step's post-collision values) over columns [i0 - HX, i0 + BX + HX) (HX = 16 bytes of columns:
// 4 FP32, 8 2-byte values) and rows [j0 - 2, j0 + BY + 2), one box of depth 5 the packed fields
// (uhat, a = uhat . grad uhat, Dh) over the columns [i0 - 4, i0 + BX + 4) and the rows
// [j0 - 1, j0 + BY + 1).  The population planes keep a two-wide ghost frame of periodic copies,
// so the two-node halo is a plain tile read at the edges too.
//   Step 1 runs on the halo region R1 = columns [i0 - 2, i0 + BX + 2) x rows [j0 - 1, j0 + BY + 1)
//   (its outermost columns are computed and not used).  Node (r, c) of R1 pulls
//   g_q = P_q(x - e_q) from the stage at (row r + 1 - ey_q, column c + HX - 2 - ex_q); that slot
//   is pulled by this node alone, so the node writes its post-collision value P1_q back into
//   the same slot (in place, no second buffer; 2-byte storages round it to the storage format
//   as a one-step launch would store it).
//   Step 2 runs on the output nodes: node (r2, c2) = R1 node (r2 + 1, c2 + 2) pulls
//   P1_q(x - e_q) from (row r2 + 2 - 2 ey_q, column c2 + HX - 2 ex_q) and stores P2 to global
//   memory with its ghost copies (nodes within two of an edge).
// Geometry (Geom2For): narrow tiles (32 columns; 8 rows with the pulse source, 16 without) and
// several CTAs per SM with two stages each, so that while one CTA waits at the barrier between
// its two steps the others compute (the kernel is latency-bound, not HBM-bound).
// R1 nodes outside the grid are periodic images: their populations come from the ghost frame,
// their fields from the packed fields' ghost frame (copies of the wrapped node, the acceleration
// included, whatever the gradient mode), their source from the wrapped node's coordinates and
// their rounding bits from the wrapped node pair, so they compute exactly what the wrapped node
// computes.
#include "trtr_step2_core.cuh"

namespace trtr {
namespace {

using namespace core;

template <typename S, int SRC, class G, bool P1, bool SR>
__global__ void __launch_bounds__(G::kThreads, G::kCtas)
    step2_kernel(const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap mf, const Step2Args args) {
    constexpr int STAGES = G::kStages, NT = G::kThreads;
    using T = typename G::T;
    const StepArgs<float>& a = args.a;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * T::Stage);

    const int tid = threadIdx.x;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const int ntx = (nx + T::X - 1) / T::X, nty = (ny + T::Y - 1) / T::Y;
    const int ntiles = ntx * nty;
#ifndef TRTR_STEP2_ORDER
#define TRTR_STEP2_ORDER 0
#endif
    // tile order: 0 interleaved (tile = CTA + k grid), 1 a contiguous row-major run per CTA
    const int chunk = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
    const int first = TRTR_STEP2_ORDER ? (int)blockIdx.x * chunk : (int)blockIdx.x;
    const int stride = TRTR_STEP2_ORDER ? 1 : (int)gridDim.x;
    const int my_tiles = TRTR_STEP2_ORDER ? (first < ntiles ? min(chunk, ntiles - first) : 0)
                                          : (first < ntiles ? (ntiles - 1 - first) / stride + 1 : 0);
    // The tile of each stage.  TRTR_STEP2_DYN = G > 0: thread 0 takes runs of G consecutive tiles
    // of the row-major order from the context's counter whenever it needs the next tile, so that
    // faster CTAs take more and the launch ends evenly; 0: tile k of this CTA is first + k stride,
    // walked without a division per tile.  s_org[s] holds the origin of the tile loaded into
    // stage s (x = -1: none left), written by thread 0 before the loads are issued and read by
    // every thread STAGES - 1 barriers later.
#ifndef TRTR_STEP2_DYN
#define TRTR_STEP2_DYN 4  // measured on GB300 (4096^2 / 8192^2 pulse): static 97.0 / 95.2 GLUPS, runs
                          // of 1: 108.9 / 113.5, 2: 112.2 / 117.7, 4: 112.4 / 120.7, 8: 109.4 / 119.3
#endif
    constexpr int kRun = TRTR_STEP2_DYN;
    const bool dyn = kRun > 0 && (a.sched & kSchedDynamic);
    const bool rev = (a.sched & kSchedReverse) != 0;  // tile (a, b) stands for (ntx-1-a, nty-1-b)
    __shared__ int2 s_org[STAGES];
    TileCursor ahead;  // thread 0: the next tile to load
    int run_left = 0;  // thread 0 (dynamic): tiles left in the current run
    bool more = true;  // thread 0 (dynamic): the counter has tiles left
    int taken = 0;     // thread 0 (static): tiles of this CTA loaded so far
    auto take = [&]() -> int2 {
        if (dyn) {
            if (run_left == 0) {
                if (!more) return make_int2(-1, 0);
                const unsigned t = atomicAdd(a.tile_ctr, (unsigned)kRun);
                if (t >= (unsigned)ntiles) {
                    more = false;
                    return make_int2(-1, 0);
                }
                ahead.init((int)t, 1, ntx);
                run_left = min(kRun, ntiles - (int)t);
            } else {
                ahead.next();
            }
            --run_left;
        } else {
            if (taken == my_tiles) return make_int2(-1, 0);
            if (taken++ > 0) ahead.next();
        }
        return rev ? make_int2((ntx - 1 - ahead.a) * T::X, (nty - 1 - ahead.b) * T::Y)
                   : make_int2(ahead.a * T::X, ahead.b * T::Y);
    };
    auto finish = [&]() {  // the last CTA of the launch sets the counter back to zero
        if (dyn && tid == 0) {
            __threadfence();
            if (atomicAdd(a.tile_ctr + 1, 1u) == gridDim.x - 1) {
                atomicExch(a.tile_ctr, 0u);
                atomicExch(a.tile_ctr + 1, 0u);
            }
        }
    };
    auto issue = [&](int s) {
        const int2 o = take();
        s_org[s] = o;
        if (o.x >= 0) {
            mbar_expect_tx(&full[s], T::TX);
            step2_issue<T>(smem + s * T::Stage, &full[s], &mp, &mf, o.x, o.y, a.lp.gx, a.lf.gx);
        }
    };

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0) {
        if (!dyn) ahead.init(first, stride, ntx);
        for (int s = 0; s < STAGES; ++s) issue(s);
    }
    __syncthreads();

    for (int k = 0;; ++k) {
        const int s = k % STAGES;
        const int2 o = s_org[s];
        if (o.x < 0) break;
        const int i0 = o.x, j0 = o.y;
        const bool ok = mbar_wait_bounded(&full[s], (k / STAGES) & 1);
        if (!ok) s_abort = 1;
        S* sp = reinterpret_cast<S*>(smem + s * T::Stage);
        const float* sf = reinterpret_cast<const float*>(smem + s * T::Stage + T::FldOff);
        if (ok) step2_first<S, SRC, T, NT, SR>(sp, sf, i0, j0, a, a.tf, tid, a.rkey);
        __syncthreads();  // P1 complete (and s_abort visible)
        if (ok && !s_abort)
            step2_second<S, SRC, T, NT, P1, SR>(sp, sf, i0, j0, a, args.tf2, tid, static_cast<S*>(args.dst1), args.rkey2);
        __syncthreads();  // stage s fully read
        if (s_abort) {
            if (tid == 0) {
                atomicExch(a.flag, 1);
                for (int kk = k + 1; kk < k + STAGES; ++kk)
                    if (s_org[kk % STAGES].x >= 0) mbar_wait_bounded(&full[kk % STAGES], (kk / STAGES) & 1);
            }
            finish();
            return;
        }
        if (tid == 0) issue(s);
        if constexpr (STAGES == 1) __syncthreads();  // s_org[0] is read again at once
    }
    finish();
}

// Packed fields of the two-step kernel at every node of the two-wide ghost frame, from the
// one-step kernel's field planes (one-wide ghosts by gradient mode) at the wrapped node, with
// the one-step kernel's roundings: a_a = uhat_x d_x uhat_a + uhat_y d_y uhat_a, central
// differences 0.5 (u(+1) - u(-1)).
__global__ void pack_fields2_kernel(float* f2, const float* uv, const float* Dh, PlaneLayout lt, PlaneLayout lf) {
    const int gw = lt.nx + 2 * kGhostP, gh = lt.ny + 2 * kGhostP;
    const size_t n = (size_t)gw * gh;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / gw) - kGhostP, i = (int)(k % gw) - kGhostP;
        const int wi = wrap_clamp(i, lt.nx), wj = wrap_clamp(j, lt.ny);
        const size_t o = lf.at(wi, wj);
        const float* u = uv;
        const float* v = uv + lf.plane;
        const float ux = u[o], uy = v[o];
        const float dxux = __fmul_rn(0.5f, __fsub_rn(u[o + 1], u[o - 1]));
        const float dxuy = __fmul_rn(0.5f, __fsub_rn(v[o + 1], v[o - 1]));
        const float dyux = __fmul_rn(0.5f, __fsub_rn(u[o + lf.pitch], u[o - lf.pitch]));
        const float dyuy = __fmul_rn(0.5f, __fsub_rn(v[o + lf.pitch], v[o - lf.pitch]));
        const size_t t = lt.at(i, j);
        f2[t] = ux;
        f2[lt.plane + t] = uy;
        f2[2 * lt.plane + t] = __fmaf_rn(ux, dxux, __fmul_rn(uy, dyux));
        f2[3 * lt.plane + t] = __fmaf_rn(ux, dxuy, __fmul_rn(uy, dyuy));
        f2[4 * lt.plane + t] = Dh[o];
    }
}

// The ghost cells at distance 2 of every plane (the outer ring of the two-wide frame) from the
// interior node they repeat.  The distance-1 ring already holds its images: every step
// kernel writes it.  Reads touch the interior only, writes the ring only.
template <typename E>
__global__ void refresh_ghosts2_kernel(E* P, PlaneLayout L) {
    const int gw = L.nx + 2 * kGhostP, gh = L.ny + 2 * kGhostP;
    const int n = 2 * gw + 2 * (gh - 2);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kQ * n; k += gridDim.x * blockDim.x) {
        const int q = k / n, t = k - q * n;
        int i, j;
        if (t < 2 * gw) {  // rows -2 and ny + 1, i in [-2, nx + 1]
            i = t % gw - kGhostP;
            j = t < gw ? -kGhostP : L.ny + kGhostP - 1;
        } else {  // columns -2 and nx + 1, j in [-1, ny]
            const int u = t - 2 * gw;
            j = u % (gh - 2) - kGhostP + 1;
            i = u < gh - 2 ? -kGhostP : L.nx + kGhostP - 1;
        }
        E* plane = P + (size_t)q * L.plane;
        plane[L.at_g<kGhostP>(i, j)] = plane[L.at_g<kGhostP>(wrap_clamp(i, L.nx), wrap_clamp(j, L.ny))];
    }
}

#ifndef TRTR_STEP2_PDL
#define TRTR_STEP2_PDL 1  // 0: never launch with programmatic dependent launch (sweeps)
#endif

// One launch: two steps from the buffer described by src_map into dst (dst1: the intermediate
// state too, or null), as steps `step` and `step + 1` (the pulse source's time levels).
template <typename S, int SRC, class G, bool P1, bool SR>
cudaError_t launch2_typed(trtr_ctx* ctx, const CUtensorMap& src_map, void* dst, void* dst1, long step) {
    auto kernel = step2_kernel<S, SRC, G, P1, SR>;
    const size_t smem = (size_t)G::kStages * G::T::Stage + 128 + G::kStages * sizeof(uint64_t);
    static int configured_device = -1;
    static int ctas_per_sm = 1;
    if (configured_device != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, kernel, G::kThreads, smem);
        if (e != cudaSuccess) return e;
        if (ctas_per_sm < 1) return cudaErrorInvalidConfiguration;
        configured_device = ctx->device;
    }
    Step2Args args;
    StepArgs<float>& a = args.a;
    memset(static_cast<void*>(&args), 0, sizeof(args));
    a.dst = dst;
    args.dst1 = dst1;
    a.tab_x = static_cast<const float*>(ctx->tab_x);
    a.tab_y = static_cast<const float*>(ctx->tab_y);
    a.flag = ctx->dflag;
    a.tile_ctr = reinterpret_cast<unsigned*>(ctx->dflag + 2);
    a.lp = ctx->lp;
    a.lf = ctx->lt;
    a.tau2_fixed = ctx->p.tau2_mode == TRTR_TAU2_FIXED;
    a.magic = (float)ctx->p.magic;
    a.omega2_fixed = (float)(ctx->p.tau2_mode == TRTR_TAU2_FIXED ? 1.0 / ctx->p.tau2 : 0.0);
    a.phi_ref = (float)ctx->p.phi_ref;
    a.x0 = (float)ctx->p.x0;
    a.y0 = (float)ctx->p.y0;
    a.dx = (float)ctx->p.dx;
    a.dt = (float)ctx->p.dt;
    a.rkey = sr_step_key(step);
    args.rkey2 = sr_step_key(step + 1);
    if (SRC == TRTR_SRC_PULSE) {
        a.dD_amp = (float)(ctx->pulse.D0 * ctx->pulse.D_amp);
        a.tf = pulse_time_fields<float>(ctx->pulse, ctx->p.dt, step);
        args.tf2 = pulse_time_fields<float>(ctx->pulse, ctx->p.dt, step + 1);
    }
    const long ntiles = (long)((ctx->lp.nx + G::T::X - 1) / G::T::X) * ((ctx->lp.ny + G::T::Y - 1) / G::T::Y);
    const long cap = (long)ctx->num_sms * ctas_per_sm;
    const long grid = ntiles < cap ? ntiles : cap;
    a.sched = (ntiles > kDynMinTilesPerCta * grid ? kSchedDynamic : 0) | (ctx->sweeps++ & 1u ? kSchedReverse : 0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(G::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = TRTR_STEP2_PDL && ntiles <= kPdlMaxTilesPerCta * grid;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, src_map, ctx->maps2[2], args);
}

}  // namespace

bool two_step_applies(const trtr_ctx* ctx) {
    return ctx->fld2 != nullptr && ctx->steps_per_launch == 2 && ctx->p.bc_mode == TRTR_BC_PERIODIC &&
           (ctx->p.src_mode == TRTR_SRC_NONE || ctx->p.src_mode == TRTR_SRC_PULSE);
}

template <typename S, class G>
cudaError_t encode_pop2_typed(trtr_ctx* ctx, void* buffer, CUtensorMap* out) {
    using T = typename G::T;
    return encode(out, tma_type<S>(), (int)sizeof(S), buffer, ctx->lp, kQ, T::W, T::PR, kQ) ? cudaSuccess
                                                                                          : cudaErrorInvalidValue;
}

template <typename S, class G>
cudaError_t encode2_typed(trtr_ctx* ctx) {
    using T = typename G::T;
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        ok = ok && encode(&ctx->maps2[b], tma_type<S>(), (int)sizeof(S), ctx->pop[b], ctx->lp, kQ, T::W, T::PR, kQ);
    ok = ok && encode(&ctx->maps2[2], tma_type<float>(), 4, ctx->fld2, ctx->lt, kT2NF, T::WF, T::FR, kT2NF);
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}

// Calls f((S*)nullptr, Geom2Of<SRC, sizeof(S)>-typed tag, SRC) for the context's storage and
// source mode (FP32, FP16 or BF16 populations; no source or the pulse source).
template <typename S, class F>
cudaError_t by_source(const trtr_ctx* ctx, F&& f) {
    return ctx->p.src_mode == TRTR_SRC_PULSE
               ? f((S*)nullptr, (Geom2Of<TRTR_SRC_PULSE, (int)sizeof(S)>*)nullptr, std::integral_constant<int, TRTR_SRC_PULSE>())
               : f((S*)nullptr, (Geom2Of<TRTR_SRC_NONE, (int)sizeof(S)>*)nullptr, std::integral_constant<int, TRTR_SRC_NONE>());
}
template <class F>
cudaError_t by_storage(const trtr_ctx* ctx, F&& f) {
    switch (ctx->p.precision) {
        case TRTR_F32: return by_source<float>(ctx, f);
        case TRTR_F16_OFS: return by_source<__half>(ctx, f);
        case TRTR_BF16_OFS: return by_source<__nv_bfloat16>(ctx, f);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t encode_maps2(trtr_ctx* ctx) {
    if (!ctx->fld2) return cudaSuccess;
    return by_storage(ctx, [&](auto* sp, auto* gp, auto) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using G = std::remove_pointer_t<decltype(gp)>;
        return encode2_typed<S, G>(ctx);
    });
}

cudaError_t launch_pack_fields2(trtr_ctx* ctx) {
    const size_t n = (size_t)(ctx->p.nx + 2 * kGhostP) * (ctx->p.ny + 2 * kGhostP);
    const size_t want = (n + 255) / 256, cap = (size_t)ctx->num_sms * 8;
    ctx->launches += 1;
    pack_fields2_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, ctx->stream>>>(
        static_cast<float*>(ctx->fld2), static_cast<const float*>(ctx->uv), static_cast<const float*>(ctx->Dh),
        ctx->lt, ctx->lf);
    return cudaGetLastError();
}

cudaError_t launch_refresh_ghosts2_buffer(trtr_ctx* ctx, void* P) {
    const int n = 2 * (ctx->p.nx + 2 * kGhostP) + 2 * (ctx->p.ny + 2 * kGhostP - 2);
    const int want = (kQ * n + 255) / 256, cap = ctx->num_sms * 4;
    ctx->launches += 1;
    if (ctx->esize == 4)
        refresh_ghosts2_kernel<<<want < cap ? want : cap, 256, 0, ctx->stream>>>(static_cast<float*>(P), ctx->lp);
    else if (ctx->esize == 2)
        refresh_ghosts2_kernel<<<want < cap ? want : cap, 256, 0, ctx->stream>>>(static_cast<unsigned short*>(P), ctx->lp);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_refresh_ghosts2(trtr_ctx* ctx) { return launch_refresh_ghosts2_buffer(ctx, ctx->pop[ctx->cur]); }

cudaError_t encode_pop_map2(trtr_ctx* ctx, void* buffer, CUtensorMap* out) {
    return by_storage(ctx, [&](auto* sp, auto* gp, auto) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using G = std::remove_pointer_t<decltype(gp)>;
        return encode_pop2_typed<S, G>(ctx, buffer, out);
    });
}

cudaError_t launch_step2_from(trtr_ctx* ctx, const CUtensorMap* src_map, void* dst, void* dst1, long step) {
    const bool sr = ctx->esize == 2 && ctx->p.rounding == TRTR_ROUND_STOCHASTIC;
    return by_storage(ctx, [&](auto* sp, auto* gp, auto src) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using G = std::remove_pointer_t<decltype(gp)>;
        constexpr int SRC = decltype(src)::value;
        if constexpr (sizeof(S) == 2) {
            if (sr)
                return dst1 ? launch2_typed<S, SRC, G, true, true>(ctx, *src_map, dst, dst1, step)
                            : launch2_typed<S, SRC, G, false, true>(ctx, *src_map, dst, dst1, step);
        }
        return dst1 ? launch2_typed<S, SRC, G, true, false>(ctx, *src_map, dst, dst1, step)
                    : launch2_typed<S, SRC, G, false, false>(ctx, *src_map, dst, dst1, step);
    });
}

cudaError_t launch_step2(trtr_ctx* ctx) {
    return launch_step2_from(ctx, &ctx->maps2[ctx->cur], ctx->pop[ctx->cur ^ 1], nullptr, ctx->step);
}

TRTR_BOUNDS_TAKE(step2)

}  // namespace trtr
