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
// and the nine populations are rebuilt pairwise from their even and odd halves.
//
// Data movement (sm_103a): a persistent kernel walks 128 x BY-node tiles with the CTAs per SM
// and stages of Geom below.  For each tile one thread issues TMA loads (cp.async.bulk.tensor)
// of the nine shifted population tiles, the u tile with its one-node halo and the D tile into
// a shared-memory stage and arms an mbarrier with the expected byte count; the stages form a
// ring so the loads of the next tiles are in flight while the current one is computed.
// The pull shift of plane i is a tile origin moved by -e_i; TMA needs 16-byte aligned x
// origins, so the planes with e_x = +1 start one 16-byte chunk early and are read from
// shared memory with a column offset.  Ghost cells of the layout make the periodic wrap a
// plain tile read.  Results leave one warp = one 128-node row at a time: coalesced lane stores,
// or (FP32 pulse) one bulk copy per plane of the row staged in shared memory; edge nodes also
// store their ghost copies.  Every mbarrier wait is bounded: on timeout the kernel raises the
// context's flag and returns.
#include "trtr_step_core.cuh"

namespace trtr {
namespace {

using namespace core;

constexpr int kBX = 128;  // nodes per tile along x

// Pipeline geometry per storage type and source mode.  A CTA owns STAGES tile buffers of
// BY x 128 nodes: while its warps work on one, the TMA loads of the next STAGES - 1 are in
// flight.  WPR warps share a tile row (a lane takes 128 / (64 WPR) node pairs); CTAS CTAs per SM
// set the register budget (65536 / (threads x CTAS) per thread).  ORDER is the order in which
// the persistent CTAs take the tiles: 0 = interleaved row-major (tile = CTA + k * grid, so the
// CTAs sweep the grid together and neighbouring tiles' halos are fetched at the same time),
// 1 = contiguous column-major chunk per CTA, 2 = contiguous row-major chunk per CTA.  TST = 1:
// results leave through bulk copies of whole tile rows from shared memory (one warp per row),
// 0: lane stores.  Chosen by sweeps on GB300 (4096^2 FP32 and 8192^2 FP16 steps in each source
// mode): one CTA of 16 warps per SM on 128 x 16 tiles, two stages for FP32 and three for the
// 2-byte storages (as many as fit), bulk row stores for the FP32 pulse; the FP32 source-field
// mode, whose stages carry two more planes, runs two CTAs per SM on 128 x 8 tiles so that each
// still has two stages.  The TRTR_STEP_* macros override the geometry of the storages of
// TRTR_STEP_SIZE bytes in source mode TRTR_STEP_SRC (sweeps).
//
// SMALL_BELOW: grids with fewer than this many of these tiles per SM take the small-grid
// geometry (SmallPipe below) instead; measured per storage and source mode.
template <typename S, int SRC>
struct Geom {  // FP64
    static constexpr int BY = 8, WPR = 1, CTAS = 2, STAGES = 2, ORDER = 2, TST = 0, SMALL_BELOW = 2;
    static constexpr bool UNROLL = false;  // UNROLL: the pair loop of the row interleaves both pairs
};
template <int SRC>
struct Geom<float, SRC> {  // pulse source
    static constexpr int BY = 16, WPR = 1, CTAS = 1, STAGES = 2, ORDER = 0, TST = 1, SMALL_BELOW = 2;
    static constexpr bool UNROLL = false;
};
template <>
struct Geom<float, TRTR_SRC_NONE> {  // the small tiles win up to 4096^2 here (not at 8192^2)
    static constexpr int BY = 16, WPR = 1, CTAS = 1, STAGES = 2, ORDER = 2, TST = 0, SMALL_BELOW = 100;
    static constexpr bool UNROLL = false;
};
template <>
struct Geom<float, TRTR_SRC_FIELD> {
    static constexpr int BY = 8, WPR = 1, CTAS = 2, STAGES = 2, ORDER = 0, TST = 0, SMALL_BELOW = 2;
    static constexpr bool UNROLL = false;
};
template <int SRC>
struct Geom<__half, SRC> {
    static constexpr int BY = 16, WPR = 1, CTAS = 1, STAGES = 3, ORDER = 0, TST = 0, SMALL_BELOW = 2;
    // both pairs at once: +5 % without a source; with the pulse source +5.5 % at 4096^2 once the
    // source's weights went into its exponent and the offsets were rounded stochastically
    static constexpr bool UNROLL = SRC != TRTR_SRC_FIELD;
};
template <int SRC>
struct Geom<__nv_bfloat16, SRC> : Geom<__half, SRC> {};

#ifdef TRTR_STEP_ROWS
#ifndef TRTR_STEP_SRC
#define TRTR_STEP_SRC -1
#endif
#ifndef TRTR_STEP_TMA_STORE
#define TRTR_STEP_TMA_STORE 0
#endif
#ifndef TRTR_STEP_UNROLL
#define TRTR_STEP_UNROLL 0
#endif
template <typename S, int SRC>
struct Sweep {
    static constexpr bool on = sizeof(S) == TRTR_STEP_SIZE && (TRTR_STEP_SRC < 0 || SRC == TRTR_STEP_SRC);
    static constexpr int BY = on ? TRTR_STEP_ROWS : Geom<S, SRC>::BY;
    static constexpr int WPR = on ? TRTR_STEP_WARPS_PER_ROW : Geom<S, SRC>::WPR;
    static constexpr int CTAS = on ? TRTR_STEP_CTAS_PER_SM : Geom<S, SRC>::CTAS;
    static constexpr int STAGES = on ? TRTR_STEP_STAGES : Geom<S, SRC>::STAGES;
    static constexpr int ORDER = on ? TRTR_STEP_ORDER : Geom<S, SRC>::ORDER;
    static constexpr int TST = on ? TRTR_STEP_TMA_STORE : Geom<S, SRC>::TST;
    static constexpr bool UNROLL = on ? TRTR_STEP_UNROLL != 0 : Geom<S, SRC>::UNROLL;
};
#else
template <typename S, int SRC>
using Sweep = Geom<S, SRC>;
#endif

// DYN: the CTAs take their tiles from a device counter (in the interleaved order) instead of a
// fixed share, so that CTAs that run faster take more tiles and the launch ends evenly.  Measured
// on GB300 (4096^2 pulse): FP32 one step per launch 70.0 -> 76.0 GLUPS, FP16 101.0 -> 103.8;
// 8192^2 FP16 112.2 -> 114.3.  TRTR_STEP_DYN=0 restores the fixed shares (sweeps).
#ifndef TRTR_STEP_DYN
#define TRTR_STEP_DYN 1
#endif

template <typename S, int SRC>
struct Pipe {
    static constexpr bool DYN = TRTR_STEP_DYN != 0;
    static constexpr int BX = kBX;
    static constexpr int BY = Sweep<S, SRC>::BY, WPR = Sweep<S, SRC>::WPR, CTAS = Sweep<S, SRC>::CTAS,
                         STAGES = Sweep<S, SRC>::STAGES, ORDER = Sweep<S, SRC>::ORDER;
    static constexpr bool TST = Sweep<S, SRC>::TST != 0 && WPR == 1;
    static constexpr int THREADS = 32 * BY * WPR;
    static constexpr int PAIRS = BX / 64 / WPR;  // node pairs per lane (FP64: 2 PAIRS nodes)
    static constexpr int UNR = Sweep<S, SRC>::UNROLL ? PAIRS : 1;
    static_assert(BY >= 1 && CTAS >= 1 && STAGES >= 1 && THREADS <= 1024, "pipeline geometry");
    static_assert((WPR == 1 || WPR == 2) && PAIRS >= 1, "warps per row");
};

// Small grids: with the geometry above a grid of a few hundred nodes per side has fewer tiles
// than SMs, and each step is one tile's load-compute-store latency.  64 x 8 tiles, two
// 256-thread CTAs per SM, one node pair per lane, spread such a grid over the whole GPU.
// Chosen when the geometry above would give fewer than Geom::SMALL_BELOW tiles per SM
// (TRTR_SMALL_TILES_PER_SM overrides that for every storage and mode: sweeps).
template <typename S, int SRC>
struct SmallPipe {
    static constexpr bool DYN = false;
    static constexpr int BX = 64, BY = 8, WPR = 1, CTAS = 2, STAGES = 2, ORDER = 0;
    static constexpr bool TST = false;
    static constexpr int THREADS = 32 * BY * WPR;
    static constexpr int PAIRS = BX / 64 / WPR;
    static constexpr int UNR = 1;
};

#ifndef TRTR_STEP_PDL
#define TRTR_STEP_PDL 1  // 0: never launch the step with programmatic dependent launch (sweeps)
#endif

template <typename S, int SRC, int STAGES, class G, bool SR>
__global__ void __launch_bounds__(G::THREADS, G::CTAS)
    step_kernel(const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap mu,
                const __grid_constant__ CUtensorMap md, const __grid_constant__ CUtensorMap ms,
                const StepArgs<typename Store<S>::C> a) {
    constexpr int kBX = G::BX, kBY = G::BY, kWPR = G::WPR, kPairsPerLane = G::PAIRS;
    constexpr bool kTST = G::TST;
    using T = Tile<S, SRC, kBX, kBY>;
    constexpr bool kPairs = !std::is_same<S, double>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    // stages on a 128-byte boundary (TMA destination alignment), barriers after them
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * T::STAGE);

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int r = w / kWPR;                // tile row of this warp
    const int c0 = (w % kWPR) * 64 * kPairsPerLane;  // its first column in the row
    const int nx = a.lp.nx, ny = a.lp.ny;
    const int ntx = (nx + kBX - 1) / kBX, nty = (ny + kBY - 1) / kBY;
    const int ntiles = ntx * nty;
    constexpr int kOrder = G::ORDER;
    const int chunk = (ntiles + gridDim.x - 1) / gridDim.x;
    const int first = kOrder == 0 ? blockIdx.x : blockIdx.x * chunk;
    const int stride = kOrder == 0 ? gridDim.x : 1;
    const int my_tiles = kOrder == 0 ? (first < ntiles ? (ntiles - 1 - first) / stride + 1 : 0)
                                     : (first < ntiles ? min(chunk, ntiles - first) : 0);

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // Programmatic dependent launch: the next launch on the stream may be set up from here on,
    // and nothing written by earlier kernels is read before they have completed (both no-ops
    // when the launch does not allow it).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // The tile of each stage: G::DYN hands out the tiles of the interleaved order from the
    // context's counter (thread 0 takes the next one whenever it refills a stage; -1: none left);
    // otherwise tile k of this CTA is first + k stride.  A reversed launch takes tile
    // ntiles - 1 - t in place of t.  s_tile[s] is written by thread 0 before
    // the loads into stage s are issued and read by every thread STAGES - 1 barriers later.
    __shared__ int s_tile[STAGES];
    __shared__ int s_more;
    const bool dyn = G::DYN && (a.sched & kSchedDynamic);
    const bool rev = (a.sched & kSchedReverse) != 0;
    auto take = [&](int k) -> int {  // thread 0: the tile that the CTA's k-th stage fill loads
        int t = -1;
        if (dyn) {
            if (s_more) {
                const unsigned c = atomicAdd(a.tile_ctr, 1u);
                if (c < (unsigned)ntiles)
                    t = (int)c;
                else
                    s_more = 0;
            }
        } else if (k < my_tiles) {
            t = first + k * stride;
        }
        return t >= 0 && rev ? ntiles - 1 - t : t;
    };
    // tile t's origin (a division per tile measured 2 % faster here than the two-step kernel's
    // TileCursor, which wins there)
    auto tile_x0 = [&](int t) { return (kOrder == 1 ? t / nty : t % ntx) * kBX; };
    auto tile_y0 = [&](int t) { return (kOrder == 1 ? t % nty : t / ntx) * kBY; };
    // the end of the CTA's work: the last CTA of the launch sets the counter back to zero
    auto finish = [&]() {
        if (dyn && tid == 0) {
            __threadfence();
            if (atomicAdd(a.tile_ctr + 1, 1u) == gridDim.x - 1) {
                atomicExch(a.tile_ctr, 0u);
                atomicExch(a.tile_ctr + 1, 0u);
            }
        }
    };
    if (tid == 0) {
        s_more = 1;
        for (int k = 0; k < STAGES; ++k) {
            const int t = take(k);
            s_tile[k] = t;
            if (t >= 0) issue_tile<S, SRC, kBX, kBY>(smem + k * T::STAGE, &full[k], &mp, &mu, &md, &ms, tile_x0(t),
                                                     tile_y0(t), a);
        }
    }
    __syncthreads();

    for (int k = 0;; ++k) {
        const int s = k % STAGES;
        const int t = s_tile[s];
        if (t < 0) break;
        const int i0 = tile_x0(t), j0 = tile_y0(t);
        const int j = j0 + r;

        // per-column / per-row pulse tables, loaded before the wait so their latency hides
        F2 sx[kPairsPerLane], cx[kPairsPerLane];
        float sy = 0.f, cy = 0.f;
        if (kPairs && SRC == TRTR_SRC_PULSE) {
#pragma unroll
            for (int m = 0; m < kPairsPerLane; ++m) {
                const int i = i0 + c0 + 64 * m + 2 * lane;
                const float* tx = reinterpret_cast<const float*>(a.tab_x);
                const float s0 = i < nx ? __ldg(tx + i) : 0.f, s1 = i + 1 < nx ? __ldg(tx + i + 1) : 0.f;
                const float c0 = i < nx ? __ldg(tx + nx + i) : 0.f, c1 = i + 1 < nx ? __ldg(tx + nx + i + 1) : 0.f;
                sx[m] = F2(s0, s1);
                cx[m] = F2(c0, c1);
            }
            if (j < ny) {
                const float* ty = reinterpret_cast<const float*>(a.tab_y);
                sy = __ldg(ty + j);
                cy = __ldg(ty + ny + j);
            }
        }

        const bool ok = mbar_wait_bounded(&full[s], (k / STAGES) & 1);
        if (!ok) s_abort = 1;
        if (ok && j < ny) {
            const unsigned char* st = smem + s * T::STAGE;
            if constexpr (kPairs)
                tile_row_pairs<S, SRC, kBX, kBY, kPairsPerLane, kTST, G::UNR, SR>(st, r, lane, i0, j, a, sx, cx, sy,
                                                                                  cy, c0);
            else
                tile_row_f64<SRC, kBX, kBY, 2 * kPairsPerLane, kTST>(st, r, lane, i0, j, a, c0);
        }
        __syncthreads();  // stage s fully read (and s_abort visible)
        if (s_abort) {
            if (tid == 0) {
                atomicExch(a.flag, 1);
                // let the loads already issued into this CTA's shared memory land (bounded)
                for (int kk = k + 1; kk < k + STAGES; ++kk)
                    if (s_tile[kk % STAGES] >= 0) mbar_wait_bounded(&full[kk % STAGES], (kk / STAGES) & 1);
            }
            if (kTST && lane == 0) bulk_wait_all();
            finish();
            return;
        }
        if (tid == 0) {
            const int tn = take(k + STAGES);
            s_tile[s] = tn;
            if (tn >= 0)
                issue_tile<S, SRC, kBX, kBY>(smem + s * T::STAGE, &full[s], &mp, &mu, &md, &ms, tile_x0(tn),
                                             tile_y0(tn), a);
        }
        if constexpr (STAGES == 1) __syncthreads();  // s_tile[0] is read again at once
    }
    if (kTST && lane == 0) bulk_wait_all();  // this warp's row copies have completed
    finish();
}

// The failure path of the step kernels' bounded waits, on its own: a barrier that nothing ever
// completes (no copy is issued), waited on for `cycles`, then the context's timeout flag.
__global__ void wait_timeout_kernel(int* flag, long long cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait_bounded(&bar, 0, cycles)) atomicExch(flag, 1);
    }
}

// The recording path of the bounds-checked build, on its own: one thread puts four bad
// arguments to the checks -- a plane index one column past the ghost frame, a TMA x coordinate
// of 12 bytes, a TMA destination 16 bytes off a 128-byte boundary, and a bulk row copy past the
// row end -- and performs no access with any of them (the clamped plane index is compared, not
// used).  The checked build records the four; the default build records nothing.
__global__ void bounds_probe_kernel(PlaneLayout L) {
    __shared__ __align__(128) unsigned char buf[256];
    if (threadIdx.x != 0) return;
    const size_t k = L.at(L.nx + L.gy, 0);
    const bool clamped = k == L.at(L.nx + L.gy - 1, 0);
    const bool t1 = tma_ok(buf, 3, 0, 4);
    const bool t2 = tma_ok(buf + 16, 0, 0, 4);
    const bool b1 = bulk_ok(static_cast<const float*>(nullptr), buf, L.nx - 4, 0, 8, L);
    if (clamped && t1 && t2 && b1) buf[0] = 0;  // keeps the checks (no global access)
}

// Stages per CTA: G::STAGES, or fewer while they do not fit in the 227 KB a CTA may use.
template <typename S, int SRC, class G>
constexpr int stages_for() {
    constexpr int kStage = Tile<S, SRC, G::BX, G::BY>::STAGE;
    static_assert(kStage + 256 <= 227 * 1024, "one tile stage must fit in shared memory");
    int s = G::STAGES;
    while (s > 1 && s * kStage + 256 > 227 * 1024) --s;
    return s;
}

// ------------------------------------------------------------------------------ host side

template <typename S, int SRC, class G>
cudaError_t encode_typed(trtr_ctx* ctx) {
    using C = typename Store<S>::C;
    constexpr int kBX = G::BX, kBY = G::BY;
    // The box shapes do not depend on the source mode (TX bytes do).
    using T = Tile<S, TRTR_SRC_NONE, kBX, kBY>;
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        ok = ok && encode(&ctx->maps[kMapPop0 + b], tma_type<S>(), sizeof(S), ctx->pop[b], ctx->lp, kQ, T::PW, kBY, 1);
    ok = ok && encode(&ctx->maps[kMapU], tma_type<C>(), sizeof(C), ctx->uv, ctx->lf, 2, T::UW, T::UH, 2);
    ok = ok && encode(&ctx->maps[kMapD], tma_type<C>(), sizeof(C), ctx->Dh, ctx->lf, 1, kBX, kBY, 1);
    if (ctx->S) ok = ok && encode(&ctx->maps[kMapS], tma_type<C>(), sizeof(C), ctx->S, ctx->lf, 2, kBX, kBY, 1);
    else ctx->maps[kMapS] = ctx->maps[kMapD];
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}

// One step from the population buffer described by src_map into dst, as step `step` (its
// source terms and first-step rule).  SR: stochastic rounding of the 2-byte storages.
template <typename S, int SRC, class G, bool SR = false>
cudaError_t launch_typed(trtr_ctx* ctx, const CUtensorMap& src_map, void* dst, long step) {
    using C = typename Store<S>::C;
    constexpr int kBX = G::BX, kBY = G::BY, kThreads = G::THREADS;
    using T = Tile<S, SRC, kBX, kBY>;
    constexpr int kStages = stages_for<S, SRC, G>();
    auto kernel = step_kernel<S, SRC, kStages, G, SR>;
    const size_t smem = (size_t)kStages * T::STAGE + 128 + kStages * sizeof(uint64_t);
    static int configured_device = -1;
    static int ctas_per_sm = 1;
    if (configured_device != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, kernel, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (ctas_per_sm < 1) return cudaErrorInvalidConfiguration;
        configured_device = ctx->device;
    }
    StepArgs<C> a;
    a.dst = dst;
    a.tab_x = static_cast<const C*>(ctx->tab_x);
    a.tab_y = static_cast<const C*>(ctx->tab_y);
    a.flag = ctx->dflag;
    a.tile_ctr = reinterpret_cast<unsigned*>(ctx->dflag + 2);
    a.lp = ctx->lp;
    a.lf = ctx->lf;
    a.s_cur = ctx->S_cur < 0 ? 0 : ctx->S_cur;
    a.s_prev = ctx->S_prev >= 0 ? ctx->S_prev : a.s_cur;
    a.tau2_fixed = ctx->p.tau2_mode == TRTR_TAU2_FIXED;
    a.magic = C(ctx->p.magic);
    a.omega2_fixed = C(ctx->p.tau2_mode == TRTR_TAU2_FIXED ? 1.0 / ctx->p.tau2 : 0.0);
    a.phi_ref = C(ctx->p.phi_ref);
    a.x0 = C(ctx->p.x0);
    a.y0 = C(ctx->p.y0);
    a.dx = C(ctx->p.dx);
    a.dt = C(ctx->p.dt);
    a.rkey = sr_step_key(step);
    if (SRC == TRTR_SRC_PULSE) {
        a.dD_amp = C(ctx->pulse.D0 * ctx->pulse.D_amp);
        a.tf = pulse_time_fields<C>(ctx->pulse, ctx->p.dt, step);
    } else {
        a.dD_amp = C(0);
        a.tf.cx_n = a.tf.cy_n = a.tf.inv_s2_n = a.tf.a_n = C(0);
        a.tf.cx_p = a.tf.cy_p = a.tf.inv_s2_p = a.tf.a_p = C(0);
    }
    const long ntiles = (long)((ctx->lp.nx + kBX - 1) / kBX) * ((ctx->lp.ny + kBY - 1) / kBY);
    const long cap = (long)ctx->num_sms * ctas_per_sm;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    a.sched = (ntiles > kDynMinTilesPerCta * grid ? kSchedDynamic : 0) | (ctx->sweeps++ & 1u ? kSchedReverse : 0);
    // launched with programmatic stream serialisation: the launch overlaps the tail of the
    // kernel before it, whose results the kernel waits for (griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = TRTR_STEP_PDL && ntiles <= kPdlMaxTilesPerCta * grid;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, src_map, ctx->maps[kMapU], ctx->maps[kMapD], ctx->maps[kMapS], a);
}

template <typename S, int SRC>
cudaError_t launch_geom(trtr_ctx* ctx, const CUtensorMap& src_map, void* dst, long step) {
    if constexpr (sizeof(S) == 2) {
        if (ctx->p.rounding == TRTR_ROUND_STOCHASTIC)
            return ctx->small_tiles ? launch_typed<S, SRC, SmallPipe<S, SRC>, true>(ctx, src_map, dst, step)
                                    : launch_typed<S, SRC, Pipe<S, SRC>, true>(ctx, src_map, dst, step);
    }
    return ctx->small_tiles ? launch_typed<S, SRC, SmallPipe<S, SRC>>(ctx, src_map, dst, step)
                            : launch_typed<S, SRC, Pipe<S, SRC>>(ctx, src_map, dst, step);
}

template <typename S>
cudaError_t launch_src(trtr_ctx* ctx, const CUtensorMap& src_map, void* dst, long step) {
    switch (ctx->p.src_mode) {
        case TRTR_SRC_FIELD: return launch_geom<S, TRTR_SRC_FIELD>(ctx, src_map, dst, step);
        case TRTR_SRC_PULSE: return launch_geom<S, TRTR_SRC_PULSE>(ctx, src_map, dst, step);
        default: return launch_geom<S, TRTR_SRC_NONE>(ctx, src_map, dst, step);
    }
}

template <typename S, class G>
cudaError_t encode_pop_geom(trtr_ctx* ctx, void* buffer, CUtensorMap* out) {
    using T = Tile<S, TRTR_SRC_NONE, G::BX, G::BY>;
    return encode(out, tma_type<S>(), sizeof(S), buffer, ctx->lp, kQ, T::PW, G::BY, 1) ? cudaSuccess
                                                                                      : cudaErrorInvalidValue;
}

// population maps of the source-free kernel (the adjoint's recomputation)
template <typename S>
cudaError_t encode_pop_typed(trtr_ctx* ctx, void* buffer, CUtensorMap* out) {
    return ctx->small_tiles ? encode_pop_geom<S, SmallPipe<S, TRTR_SRC_NONE>>(ctx, buffer, out)
                            : encode_pop_geom<S, Pipe<S, TRTR_SRC_NONE>>(ctx, buffer, out);
}

template <typename S, int SRC>
cudaError_t encode_geom(trtr_ctx* ctx) {
    // the small-grid geometry when the large one leaves most SMs without a second tile
    using G = Pipe<S, SRC>;
    const long tiles = (long)((ctx->lp.nx + G::BX - 1) / G::BX) * ((ctx->lp.ny + G::BY - 1) / G::BY);
#ifdef TRTR_SMALL_TILES_PER_SM
    constexpr long kBelow = TRTR_SMALL_TILES_PER_SM;
#else
    constexpr long kBelow = Geom<S, SRC>::SMALL_BELOW;
#endif
    ctx->small_tiles = tiles < kBelow * ctx->num_sms;
    return ctx->small_tiles ? encode_typed<S, SRC, SmallPipe<S, SRC>>(ctx) : encode_typed<S, SRC, G>(ctx);
}

}  // namespace

template <typename S>
cudaError_t encode_src(trtr_ctx* ctx) {
    switch (ctx->p.src_mode) {
        case TRTR_SRC_FIELD: return encode_geom<S, TRTR_SRC_FIELD>(ctx);
        case TRTR_SRC_PULSE: return encode_geom<S, TRTR_SRC_PULSE>(ctx);
        default: return encode_geom<S, TRTR_SRC_NONE>(ctx);
    }
}

// Encodes the context's TMA descriptors and picks its tile geometry (ctx->small_tiles).
cudaError_t encode_maps(trtr_ctx* ctx) {
    switch (ctx->p.precision) {
        case TRTR_F64: return encode_src<double>(ctx);
        case TRTR_F32: return encode_src<float>(ctx);
        case TRTR_F16_OFS: return encode_src<__half>(ctx);
        case TRTR_BF16_OFS: return encode_src<__nv_bfloat16>(ctx);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wait_timeout(trtr_ctx* ctx, long long cycles) {
    ctx->launches += 1;
    wait_timeout_kernel<<<1, 32, 0, ctx->stream>>>(ctx->dflag, cycles);
    return cudaGetLastError();
}

cudaError_t launch_bounds_probe(trtr_ctx* ctx) {
    ctx->launches += 1;
    bounds_probe_kernel<<<1, 32, 0, ctx->stream>>>(ctx->lp);
    return cudaGetLastError();
}

cudaError_t launch_step_from(trtr_ctx* ctx, const CUtensorMap* src_map, void* dst, long step) {
    switch (ctx->p.precision) {
        case TRTR_F64: return launch_src<double>(ctx, *src_map, dst, step);
        case TRTR_F32: return launch_src<float>(ctx, *src_map, dst, step);
        case TRTR_F16_OFS: return launch_src<__half>(ctx, *src_map, dst, step);
        case TRTR_BF16_OFS: return launch_src<__nv_bfloat16>(ctx, *src_map, dst, step);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(trtr_ctx* ctx) {
    return launch_step_from(ctx, &ctx->maps[kMapPop0 + ctx->cur], ctx->pop[ctx->cur ^ 1], ctx->step);
}

cudaError_t encode_pop_map(trtr_ctx* ctx, void* buffer, CUtensorMap* out) {
    switch (ctx->p.precision) {
        case TRTR_F64: return encode_pop_typed<double>(ctx, buffer, out);
        case TRTR_F32: return encode_pop_typed<float>(ctx, buffer, out);
        case TRTR_F16_OFS: return encode_pop_typed<__half>(ctx, buffer, out);
        case TRTR_BF16_OFS: return encode_pop_typed<__nv_bfloat16>(ctx, buffer, out);
        default: return cudaErrorInvalidValue;
    }
}

TRTR_BOUNDS_TAKE(step)

}  // namespace trtr
