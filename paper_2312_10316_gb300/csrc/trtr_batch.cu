// trtr_batch.cu -- many independent pulse problems of uneven sizes advanced together.
//
// Every instance is an ordinary context (its own ghosted planes, fields and reductions).
// A persistent kernel launch walks a work-list of (instance, tile) pairs spanning all
// instances, one time step per launch (batch_kernel) or, for FP32 instances, two
// (batch2_kernel, the two-step kernel's tile code).  Per tile the producer thread issues the
// instance's TMA loads, then copies the instance's step arguments from a device descriptor
// into a shared-memory slot of the stage and gives the stage's mbarrier its second arrival,
// so the consumers read the arguments after their acquire-wait.  The arithmetic per node is
// the single-grid step's (Eq. (14)); only the work distribution differs.
//
// Time-dependent uniforms (the pulse source at t_n and t_{n-1}, and for two-step launches at
// t_{n+1}) live in device tables that the last CTA to finish a launch advances, together
// with a device step clock, so two-launch CUDA graphs can be replayed with no host
// involvement.
//
// The autotuner (trtr_batch_tune) times every tile shape x schedule and keeps the fastest.
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "trtr_step2_core.cuh"
#include "trtr_trace.h"

namespace trtr {
namespace {

using namespace core;

struct BatchClock {
    long long n;        // step of the instances
    unsigned int done;  // CTAs of the running launch that have finished
    unsigned int next;  // next work-list entry of a dynamically scheduled launch
};

template <typename C>
struct alignas(64) InstanceDesc {
    CUtensorMap mp[2];    // populations, source buffer 0 / 1
    CUtensorMap mu;       // uhat_x, uhat_y
    CUtensorMap md;       // Dh
    StepArgs<C> base[2];  // step arguments by source-buffer parity (dst differs); time part unused
    Pulse pulse;
    double dt;
};
// Two-step launches (FP32 or 2-byte instances): the two-step kernel's maps and arguments per instance.
struct alignas(64) InstanceDesc2 {
    CUtensorMap mp[2];        // populations, source buffer 0 / 1, the two-step tile's box
    CUtensorMap mf;           // packed fields
    StepArgs<float> base[2];  // by source-buffer parity; time part unused
    Pulse pulse;
    double dt;
};
// Pulse uniforms of a two-step launch from step n: steps n and n + 1.
struct alignas(16) TimeFields2 {
    TimeFields<float> t1, t2;
};
static_assert(sizeof(StepArgs<float>) % 16 == 0 && sizeof(TimeFields<float>) % 16 == 0, "16-byte chunks");
static_assert(offsetof(InstanceDesc2, base) % 16 == 0, "16-byte aligned arguments");
static_assert(offsetof(InstanceDesc<float>, base) % 16 == 0, "16-byte aligned arguments");

struct Geometry {
    int bx, by;
};
// 8-row tiles: two 256-thread CTAs per SM; 4-row: four 128-thread CTAs; 16-row: one 512-thread CTA
// (the single-grid step's geometry).
constexpr Geometry kGeoms[] = {{128, 8}, {64, 8}, {128, 4}, {128, 16}, {64, 16}};
constexpr int kNumGeoms = 5;
// 0 interleaved, 1 chunked, 2 chunked with the largest instances first, 3 dynamic (the CTAs take
// the entries of the instance-by-instance work-list from a counter)
constexpr int kNumSchedules = 4;
constexpr int kNumConfigs = kNumGeoms * kNumSchedules;
constexpr int kDefaultConfig = 3 * kNumSchedules + 3;  // 128 x 16 tiles, dynamic
#ifndef TRTR_BATCH2_RUN
#define TRTR_BATCH2_RUN 4
#endif
constexpr int kBatch2Run = TRTR_BATCH2_RUN;  // work-list entries per take of the two-step batch kernel
// kernel mode of a schedule: 0 chunked, 1 interleaved, 2 dynamic
constexpr int schedule_mode(int schedule) { return schedule == 0 ? 1 : (schedule == 3 ? 2 : 0); }

// Pulse source uniforms of step n (t_n = n dt and t_{n-1}), in double, stored as float.
__host__ __device__ inline TimeFields<float> time_fields(const Pulse& p, double dt, long long n) {
    return pulse_time_fields<float>(p, dt, n);
}

// Asynchronous copy of `bytes` (a multiple of 16) from global to shared memory.
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc, int bytes) {
    for (int o = 0; o < bytes; o += 16)
        asm volatile(
            "{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %1;\n\t"
            "cp.async.cg.shared.global [%0], [g], 16;\n\t}" ::"r"(smem_addr(static_cast<char*>(sdst) + o)),
            "l"(static_cast<const char*>(gsrc) + o)
            : "memory");
}

template <int BY>
constexpr int min_blocks() {
    return BY >= 16 ? 1 : (BY == 8 ? 2 : 4);  // keeps the register budget at 128 per thread
}

template <typename S, int SRC, int BX, int BY, int STAGES>
__global__ void __launch_bounds__(32 * BY, min_blocks<BY>())
    batch_kernel(const InstanceDesc<typename Store<S>::C>* __restrict__ desc, const int4* __restrict__ tiles,
                 int ntiles, TimeFields<float>* tu, TimeFields2* tu2, BatchClock* clk, int count, int parity,
                 int mode, int sr) {
    using C = typename Store<S>::C;
    using T = Tile<S, SRC, BX, BY>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(16) StepArgs<C> sargs[STAGES];
    __shared__ int4 s_t[STAGES];  // the work-list entry loaded into each stage (x = -1: none)
    __shared__ int s_abort, s_last, s_more;
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * T::STAGE);
    const int tid = threadIdx.x, lane = tid & 31, r = tid >> 5;

    // mode 0: a contiguous chunk of the work-list per CTA; 1: entries CTA + k grid; 2: thread 0
    // takes the next entry from the batch's counter whenever it refills a stage (faster CTAs take
    // more; the last CTA of the launch resets the counter)
    const int chunk = (ntiles + gridDim.x - 1) / gridDim.x;
    const int first = mode == 1 ? blockIdx.x : blockIdx.x * chunk;
    const int stride = mode == 1 ? gridDim.x : 1;
    const int my_tiles = mode == 1 ? (first < ntiles ? (ntiles - 1 - first) / stride + 1 : 0)
                                   : (first < ntiles ? min(chunk, ntiles - first) : 0);
    auto take = [&](int k) -> int {  // thread 0: the work-list index of the CTA's k-th stage fill
        if (mode == 2) {
            if (!s_more) return -1;
            const unsigned i = atomicAdd(&clk->next, 1u);
            if (i < (unsigned)ntiles) return (int)i;
            s_more = 0;
            return -1;
        }
        return k < my_tiles ? first + k * stride : -1;
    };

    // A stage's barrier completes after two arrivals and the TMA bytes: the producer's
    // arrival with the byte count goes out right before the tile loads; the second arrives
    // when its asynchronous copies of the instance's arguments into the stage's shared slot
    // land (cp.async.mbarrier.arrive), so the producer never waits on global memory.
    auto issue = [&](int k, int s) {
        const int idx = take(k);
        if (idx < 0) {
            s_t[s] = make_int4(-1, 0, 0, 0);
            return;
        }
        const int4 t = tiles[idx];  // (instance, i0, j0, gx_p | gx_f << 16)
        s_t[s] = t;
        const InstanceDesc<C>* d = desc + t.x;
        const int gxp = t.w & 0xffff, gxf = t.w >> 16;
        unsigned char* stage = smem + s * T::STAGE;
        uint64_t* bar = &full[s];
        mbar_expect_tx(bar, T::TX);
        constexpr int kPe = (int)sizeof(S), kFe = (int)sizeof(C);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int x = t.y + gxp - (lattice_ex(q) == 1 ? T::A : 0), y = t.z + kGhostP - lattice_ey(q);
            if (tma_ok(stage + q * T::POP_PLANE, x, y, kPe)) tma_load_3d(stage + q * T::POP_PLANE, &d->mp[parity], bar, x, y, q);
        }
        if (tma_ok(stage + T::POP, t.y + gxf - T::AC, t.z + kGhostF - 1, kFe))
            tma_load_3d(stage + T::POP, &d->mu, bar, t.y + gxf - T::AC, t.z + kGhostF - 1, 0);
        if (tma_ok(stage + T::POP + T::U, t.y + gxf, t.z + kGhostF, kFe))
            tma_load_2d(stage + T::POP + T::U, &d->md, bar, t.y + gxf, t.z + kGhostF);
        constexpr int kStatic = (int)(sizeof(StepArgs<C>) - sizeof(TimeFields<C>));
        cp_async_16(&sargs[s], &d->base[parity], kStatic);
        if (SRC == TRTR_SRC_PULSE) cp_async_16(&sargs[s].tf, &tu[t.x], (int)sizeof(TimeFields<C>));
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
    };

    if (tid == 0) {
        s_abort = 0;
        s_more = 1;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < STAGES; ++k) issue(k, k);
    // stochastic rounding of the 2-byte storages: the key of this step (the clock is advanced
    // only after every CTA of the launch has finished its tiles)
    const uint32_t rkey = sr ? sr_step_key((long)*reinterpret_cast<volatile long long*>(&clk->n)) : 0u;
    __syncthreads();  // s_t of the first stages

    for (int k = 0;; ++k) {
        const int s = k % STAGES;
        const int4 t = s_t[s];
        if (t.x < 0) break;
        const int i0 = t.y, j0 = t.z, j = j0 + r;

        F2 sx[BX / 64 > 0 ? BX / 64 : 1], cx[BX / 64 > 0 ? BX / 64 : 1];
        float sy = 0.f, cy = 0.f;
        if (SRC == TRTR_SRC_PULSE) {  // per-column tables, fetched before the wait
            const StepArgs<C>& g = desc[t.x].base[0];
            const int nx = g.lp.nx, ny = g.lp.ny;
            const float* tx = reinterpret_cast<const float*>(g.tab_x);
#pragma unroll
            for (int m = 0; m < BX / 64; ++m) {
                const int i = i0 + 64 * m + 2 * lane;
                const float s0 = i < nx ? __ldg(tx + i) : 0.f, s1 = i + 1 < nx ? __ldg(tx + i + 1) : 0.f;
                const float c0 = i < nx ? __ldg(tx + nx + i) : 0.f, c1 = i + 1 < nx ? __ldg(tx + nx + i + 1) : 0.f;
                sx[m] = F2(s0, s1);
                cx[m] = F2(c0, c1);
            }
            if (j < ny) {
                const float* ty = reinterpret_cast<const float*>(g.tab_y);
                sy = __ldg(ty + j);
                cy = __ldg(ty + ny + j);
            }
        }

        const bool ok = mbar_wait_bounded(&full[s], (k / STAGES) & 1);
        if (!ok) s_abort = 1;
        if (ok && j < sargs[s].lp.ny) {
            // a private copy: the row's global stores cannot alias it, so its fields are read once
            StepArgs<C> args = sargs[s];
            if constexpr (sizeof(S) == 2) {
                if (sr) {
                    args.rkey = rkey;
                    tile_row_pairs<S, SRC, BX, BY, BX / 64, false, 1, true>(smem + s * T::STAGE, r, lane, i0, j, args,
                                                                          sx, cx, sy, cy);
                } else {
                    tile_row_pairs<S, SRC, BX, BY>(smem + s * T::STAGE, r, lane, i0, j, args, sx, cx, sy, cy);
                }
            } else {
                tile_row_pairs<S, SRC, BX, BY>(smem + s * T::STAGE, r, lane, i0, j, args, sx, cx, sy, cy);
            }
        }
        __syncthreads();
        if (s_abort) {
            if (tid == 0) {
                atomicExch(desc[t.x].base[0].flag, 1);
                for (int kk = k + 1; kk < k + STAGES; ++kk)
                    if (s_t[kk % STAGES].x >= 0) mbar_wait_bounded(&full[kk % STAGES], (kk / STAGES) & 1);
                // the counters go back to zero when the last CTA is out (the step's results are void)
                __threadfence();
                if (atomicAdd(&clk->done, 1u) == gridDim.x - 1) {
                    atomicExch(&clk->next, 0u);
                    atomicExch(&clk->done, 0u);
                }
            }
            return;
        }
        if (tid == 0) issue(k + STAGES, s);
        if constexpr (STAGES == 1) __syncthreads();  // s_t[0] is read again at once
    }

    // The last CTA to finish advances the step clock and every instance's time uniforms.
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&clk->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const long long n1 = clk->n + 1;
        if (SRC == TRTR_SRC_PULSE)
            for (int k = tid; k < count; k += blockDim.x) {
                tu[k] = time_fields(desc[k].pulse, desc[k].dt, n1);
                if (tu2) tu2[k] = TimeFields2{tu[k], time_fields(desc[k].pulse, desc[k].dt, n1 + 1)};
            }
        __syncthreads();
        if (tid == 0) {
            clk->n = n1;
            clk->next = 0;
            clk->done = 0;
            __threadfence();
        }
    }
}

// Two time steps per launch over the work-list of two-step tiles (FP32 or 2-byte instances):
// per tile the producer issues the instance's two TMA boxes and copies its arguments and the
// time uniforms of both steps into the stage's slot (the barrier's second arrival), then the
// block runs the two-step kernel's two steps on the staged tile (SR: the 2-byte values rounded
// stochastically with both steps' keys, from the clock).  The last CTA advances the clock by two
// steps and both time tables.
template <typename S, int SRC, class G, bool SR>
__global__ void __launch_bounds__(G::kThreads, G::kCtas)
    batch2_kernel(const InstanceDesc2* __restrict__ desc, const int4* __restrict__ tiles, int ntiles,
                  TimeFields<float>* tu, TimeFields2* tu2, BatchClock* clk, int count, int parity) {
    constexpr int STAGES = G::kStages, NT = G::kThreads;
    using T = typename G::T;
    const long long n0 = *reinterpret_cast<volatile long long*>(&clk->n);
    const uint32_t rkey1 = SR ? sr_step_key((long)n0) : 0u, rkey2 = SR ? sr_step_key((long)n0 + 1) : 0u;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(16) StepArgs<float> sargs[STAGES];
    __shared__ __align__(16) TimeFields<float> stf2[STAGES];
    __shared__ int s_abort, s_last;
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * T::Stage);
    const int tid = threadIdx.x;
    // thread 0 takes runs of kBatch2Run consecutive work-list entries from the batch's counter
    // whenever it refills a stage (faster CTAs take more; the last CTA resets the counter)
    __shared__ int4 s_t[STAGES];  // the entry loaded into each stage (x = -1: none)
    int run_at = 0, run_left = 0;  // thread 0
    bool more = true;              // thread 0
    auto take = [&]() -> int {
        if (run_left == 0) {
            if (!more) return -1;
            const unsigned i = atomicAdd(&clk->next, (unsigned)kBatch2Run);
            if (i >= (unsigned)ntiles) {
                more = false;
                return -1;
            }
            run_at = (int)i;
            run_left = min(kBatch2Run, ntiles - (int)i);
        }
        --run_left;
        return run_at++;
    };

    auto issue = [&](int s) {
        const int idx = take();
        if (idx < 0) {
            s_t[s] = make_int4(-1, 0, 0, 0);
            return;
        }
        const int4 t = tiles[idx];  // (instance, i0, j0, gx_p | gx_f << 16)
        s_t[s] = t;
        const InstanceDesc2* d = desc + t.x;
        uint64_t* bar = &full[s];
        mbar_expect_tx(bar, T::TX);
        step2_issue<T>(smem + s * T::Stage, bar, &d->mp[parity], &d->mf, t.y, t.z, t.w & 0xffff, t.w >> 16);
        constexpr int kStatic = (int)(sizeof(StepArgs<float>) - sizeof(TimeFields<float>));
        cp_async_16(&sargs[s], &d->base[parity], kStatic);
        if (SRC == TRTR_SRC_PULSE) {
            cp_async_16(&sargs[s].tf, &tu2[t.x].t1, (int)sizeof(TimeFields<float>));
            cp_async_16(&stf2[s], &tu2[t.x].t2, (int)sizeof(TimeFields<float>));
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
    };

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < STAGES; ++s) issue(s);
    __syncthreads();  // s_t of the first stages

    for (int k = 0;; ++k) {
        const int s = k % STAGES;
        const int4 t = s_t[s];
        if (t.x < 0) break;
        const bool ok = mbar_wait_bounded(&full[s], (k / STAGES) & 1);
        if (!ok) s_abort = 1;
        S* sp = reinterpret_cast<S*>(smem + s * T::Stage);
        const float* sf = reinterpret_cast<const float*>(smem + s * T::Stage + T::FldOff);
        if (ok) step2_first<S, SRC, T, NT, SR>(sp, sf, t.y, t.z, sargs[s], sargs[s].tf, tid, rkey1);
        __syncthreads();  // step 1 complete (and s_abort visible)
        if (ok && !s_abort)
            step2_second<S, SRC, T, NT, false, SR>(sp, sf, t.y, t.z, sargs[s], stf2[s], tid, nullptr, rkey2);
        __syncthreads();  // stage s and its argument slot fully read
        if (s_abort) {
            if (tid == 0) {
                atomicExch(desc[t.x].base[0].flag, 1);
                for (int kk = k + 1; kk < k + STAGES; ++kk)
                    if (s_t[kk % STAGES].x >= 0) mbar_wait_bounded(&full[kk % STAGES], (kk / STAGES) & 1);
                __threadfence();
                if (atomicAdd(&clk->done, 1u) == gridDim.x - 1) {
                    atomicExch(&clk->next, 0u);
                    atomicExch(&clk->done, 0u);
                }
            }
            return;
        }
        if (tid == 0) issue(s);
        if constexpr (STAGES == 1) __syncthreads();  // s_t[0] is read again at once
    }

    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&clk->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const long long n2 = clk->n + 2;
        if (SRC == TRTR_SRC_PULSE)
            for (int k = tid; k < count; k += blockDim.x) {
                tu[k] = time_fields(desc[k].pulse, desc[k].dt, n2);
                tu2[k] = TimeFields2{tu[k], time_fields(desc[k].pulse, desc[k].dt, n2 + 1)};
            }
        __syncthreads();
        if (tid == 0) {
            clk->n = n2;
            clk->next = 0;
            clk->done = 0;
            __threadfence();
        }
    }
}

}  // namespace
}  // namespace trtr

using trtr::BatchClock;
using trtr::TimeFields2;
using TimeUniforms = trtr::TimeFields<float>;

struct trtr_batch {
    int count;
    trtr_ctx** ctx;
    cudaStream_t stream;
    bool own_stream;
    int precision;
    int src;
    void* d_desc;
    int4* d_tiles;
    int ntiles;
    TimeUniforms* d_tu;  // per-instance pulse uniforms of the current step
    // two steps per launch (FP32 instances): descriptors, work-list and time table of the
    // two-step kernel, its graph, and whether pairs of steps use it
    void* d_desc2;
    int4* d_tiles2;
    int ntiles2;
    TimeFields2* d_tu2;
    int grid2;
    bool two_step;
    int steps_per_launch;
    cudaGraphExec_t graph2;
    bool graph2_valid;
    BatchClock* d_clk;
    int* d_flag;
    int* h_flag;
    int config;
    int grid;
    cudaGraphExec_t graph;
    bool graph_valid;
    long step;
    int parity;
    long long nodes;
    bool sr;  // 2-byte instances rounded stochastically (TRTR_ROUND_STOCHASTIC)
    std::vector<trtr::Pulse> pulses;
};

namespace trtr {
namespace {

template <typename S, int SRC, int BX, int BY>
struct BatchLaunch {
    using C = typename Store<S>::C;
    using T = Tile<S, SRC, BX, BY>;
    // two stages, or (one CTA per SM: 16-row tiles) as many as fit, up to three
    static constexpr int kMaxStages = BY >= 16 ? 3 : 2;
    static constexpr int stages() {
        int s = kMaxStages;
        while (s > 1 && s * T::STAGE + 256 > 227 * 1024) --s;
        return s;
    }
    static constexpr int kStages = stages();
    static size_t smem() { return (size_t)kStages * T::STAGE + 128 + kStages * sizeof(uint64_t); }
    static cudaError_t configure(int device, int num_sms, int* grid_cap) {
        auto kernel = batch_kernel<S, SRC, BX, BY, kStages>;
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * BY, smem());
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        *grid_cap = num_sms * per_sm;
        (void)device;
        return cudaSuccess;
    }
    static cudaError_t launch(trtr_batch* b, int parity, int mode) {
        auto kernel = batch_kernel<S, SRC, BX, BY, kStages>;
        kernel<<<b->grid, 32 * BY, smem(), b->stream>>>(static_cast<const InstanceDesc<C>*>(b->d_desc), b->d_tiles,
                                                         b->ntiles, b->d_tu, b->d_tu2, b->d_clk, b->count, parity,
                                                         mode, b->sr ? 1 : 0);
        return cudaGetLastError();
    }
    static bool encode_desc(trtr_batch* b, InstanceDesc<C>* h) {
        for (int k = 0; k < b->count; ++k) {
            const trtr_ctx* c = b->ctx[k];
            InstanceDesc<C>& d = h[k];
            bool ok = true;
            for (int p = 0; p < 2; ++p)
                ok = ok && encode(&d.mp[p], tma_type<S>(), sizeof(S), c->pop[p], c->lp, kQ, T::PW, BY, 1);
            ok = ok && encode(&d.mu, tma_type<C>(), sizeof(C), c->uv, c->lf, 2, T::UW, T::UH, 2);
            ok = ok && encode(&d.md, tma_type<C>(), sizeof(C), c->Dh, c->lf, 1, BX, BY, 1);
            if (!ok) return false;
            StepArgs<C>& a = d.base[0];
            memset(static_cast<void*>(&a), 0, sizeof(a));
            a.tab_x = static_cast<const C*>(c->tab_x);
            a.tab_y = static_cast<const C*>(c->tab_y);
            a.flag = b->d_flag;
            a.lp = c->lp;
            a.lf = c->lf;
            a.tau2_fixed = c->p.tau2_mode == TRTR_TAU2_FIXED;
            a.magic = C(c->p.magic);
            a.omega2_fixed = C(c->p.tau2_mode == TRTR_TAU2_FIXED ? 1.0 / c->p.tau2 : 0.0);
            a.phi_ref = C(c->p.phi_ref);
            a.x0 = C(c->p.x0);
            a.y0 = C(c->p.y0);
            a.dx = C(c->p.dx);
            a.dt = C(c->p.dt);
            a.dD_amp = C(c->pulse.D0 * c->pulse.D_amp);
            d.base[1] = a;
            d.base[0].dst = c->pop[1];  // source buffer 0 -> write buffer 1
            d.base[1].dst = c->pop[0];
            d.pulse = c->pulse;
            d.dt = c->p.dt;
        }
        return true;
    }
};

// Calls f with the BatchLaunch of tile geometry `geom`.
template <typename S, int SRC, typename F>
cudaError_t with_geom(int geom, F&& f) {
    switch (geom) {
        case 0: return f(BatchLaunch<S, SRC, 128, 8>());
        case 1: return f(BatchLaunch<S, SRC, 64, 8>());
        case 2: return f(BatchLaunch<S, SRC, 128, 4>());
        case 3: return f(BatchLaunch<S, SRC, 128, 16>());
        case 4: return f(BatchLaunch<S, SRC, 64, 16>());
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, int SRC>
cudaError_t dispatch_geom(trtr_batch* b, int geom, int what, int parity, int mode, bool* enc_ok) {
    // what: 0 configure, 1 launch, 2 encode descriptors (built host-side, then copied)
    using C = typename Store<S>::C;
    return with_geom<S, SRC>(geom, [&](auto L) -> cudaError_t {
        using Launch = decltype(L);
        if (what == 0) return Launch::configure(b->ctx[0]->device, b->ctx[0]->num_sms, &b->grid);
        if (what == 1) return Launch::launch(b, parity, mode);
        std::vector<InstanceDesc<C>> h(b->count);
        *enc_ok = Launch::encode_desc(b, h.data());
        if (!*enc_ok) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemcpyAsync(b->d_desc, h.data(), sizeof(InstanceDesc<C>) * b->count,
                                        cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(b->stream);  // h goes out of scope
    });
}

cudaError_t dispatch(trtr_batch* b, int geom, int what, int parity = 0, int mode = 0) {
    bool enc_ok = true;
    const bool pulse = b->src == TRTR_SRC_PULSE;
    switch (b->precision) {
        case TRTR_F32:
            return pulse ? dispatch_geom<float, TRTR_SRC_PULSE>(b, geom, what, parity, mode, &enc_ok)
                         : dispatch_geom<float, TRTR_SRC_NONE>(b, geom, what, parity, mode, &enc_ok);
        case TRTR_F16_OFS:
            return pulse ? dispatch_geom<__half, TRTR_SRC_PULSE>(b, geom, what, parity, mode, &enc_ok)
                         : dispatch_geom<__half, TRTR_SRC_NONE>(b, geom, what, parity, mode, &enc_ok);
        case TRTR_BF16_OFS:
            return pulse ? dispatch_geom<__nv_bfloat16, TRTR_SRC_PULSE>(b, geom, what, parity, mode, &enc_ok)
                         : dispatch_geom<__nv_bfloat16, TRTR_SRC_NONE>(b, geom, what, parity, mode, &enc_ok);
        default:
            return cudaErrorInvalidValue;
    }
}

// Geometry of the two-step batch kernel: 32 x 8 tiles in 128-thread CTAs for every storage and
// source mode, where the single grid takes 32 x 16 (FP32 without a source) or 64 x 16 (2-byte):
// the batch's many small instances favour small tiles.  Measured on the 256 uneven instances
// (GLUPS): FP32 32 x 16 in two 256-thread CTAs 102.6, 32 x 8 in three or four CTAs 110.4; FP16
// 64 x 16 110.6, 64 x 8 in three CTAs 96.1, 32 x 16 in two 256-thread CTAs 124.1, 32 x 12 in
// three 117.1, 32 x 8 in three or four 125.9 (three stages 108.8).  The
// TRTR_BATCH2_{STAGES,CTAS,THREADS,BX,BY} macros set it for both storages (sweeps).
template <int SRC, int ES>
struct BatchGeom2 {
    using type = Geom2<2, ES == 2 ? 4 : 3, 128, 32, 8, ES>;
};
#ifdef TRTR_BATCH2_BX
template <int SRC, int ES>
using BatchGeom2Of = Geom2<TRTR_BATCH2_STAGES, TRTR_BATCH2_CTAS, TRTR_BATCH2_THREADS, TRTR_BATCH2_BX, TRTR_BATCH2_BY, ES>;
#else
template <int SRC, int ES>
using BatchGeom2Of = typename BatchGeom2<SRC, ES>::type;
#endif

// The two-step kernel over the batch (storage S, the batch geometry of the storage and source
// mode, SR: stochastic rounding of 2-byte instances).
template <typename S, int SRC, bool SR>
struct Batch2Launch {
    using G = BatchGeom2Of<SRC, (int)sizeof(S)>;
    using T = typename G::T;
    static size_t smem() { return (size_t)G::kStages * T::Stage + 128 + G::kStages * sizeof(uint64_t); }
    static cudaError_t configure(trtr_batch* b) {
        auto kernel = batch2_kernel<S, SRC, G, SR>;
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, G::kThreads, smem());
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        b->grid2 = b->ctx[0]->num_sms * per_sm;
        return cudaSuccess;
    }
    static cudaError_t launch(trtr_batch* b, int parity) {
        batch2_kernel<S, SRC, G, SR><<<b->grid2, G::kThreads, smem(), b->stream>>>(
            static_cast<const InstanceDesc2*>(b->d_desc2), b->d_tiles2, b->ntiles2, b->d_tu, b->d_tu2, b->d_clk,
            b->count, parity);
        return cudaGetLastError();
    }
    static bool encode_desc(trtr_batch* b, InstanceDesc2* h) {
        for (int k = 0; k < b->count; ++k) {
            const trtr_ctx* c = b->ctx[k];
            InstanceDesc2& d = h[k];
            bool ok = true;
            for (int p = 0; p < 2; ++p)
                ok = ok && encode(&d.mp[p], tma_type<S>(), (int)sizeof(S), c->pop[p], c->lp, kQ, T::W, T::PR, kQ);
            ok = ok && encode(&d.mf, tma_type<float>(), 4, c->fld2, c->lt, kT2NF, T::WF, T::FR, kT2NF);
            if (!ok) return false;
            StepArgs<float>& a = d.base[0];
            memset(static_cast<void*>(&a), 0, sizeof(a));
            a.tab_x = static_cast<const float*>(c->tab_x);
            a.tab_y = static_cast<const float*>(c->tab_y);
            a.flag = b->d_flag;
            a.lp = c->lp;
            a.lf = c->lt;
            a.tau2_fixed = c->p.tau2_mode == TRTR_TAU2_FIXED;
            a.magic = (float)c->p.magic;
            a.omega2_fixed = (float)(c->p.tau2_mode == TRTR_TAU2_FIXED ? 1.0 / c->p.tau2 : 0.0);
            a.phi_ref = (float)c->p.phi_ref;
            a.x0 = (float)c->p.x0;
            a.y0 = (float)c->p.y0;
            a.dx = (float)c->p.dx;
            a.dt = (float)c->p.dt;
            a.dD_amp = (float)(c->pulse.D0 * c->pulse.D_amp);
            d.base[1] = a;
            d.base[0].dst = c->pop[1];
            d.base[1].dst = c->pop[0];
            d.pulse = c->pulse;
            d.dt = c->p.dt;
        }
        return true;
    }
    // descriptors and the work-list of two-step tiles (taken by the CTAs in runs, from a counter)
    static trtr_status setup(trtr_batch* b) {
        if (configure(b) != cudaSuccess) return TRTR_ECUDA;
        std::vector<InstanceDesc2> h(b->count);
        if (!encode_desc(b, h.data())) return TRTR_ECUDA;
        std::vector<int4> t;
        for (int k = 0; k < b->count; ++k) {
            const int nx = b->ctx[k]->p.nx, ny = b->ctx[k]->p.ny;
            for (int j0 = 0; j0 < ny; j0 += T::Y)
                for (int i0 = 0; i0 < nx; i0 += T::X)
                    t.push_back(make_int4(k, i0, j0, b->ctx[k]->lp.gx | (b->ctx[k]->lt.gx << 16)));
        }
        if (cudaMalloc(&b->d_tiles2, t.size() * sizeof(int4)) != cudaSuccess) return TRTR_ENOMEM;
        if (cudaMemcpyAsync(b->d_desc2, h.data(), sizeof(InstanceDesc2) * b->count, cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess ||
            cudaMemcpyAsync(b->d_tiles2, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            return TRTR_ECUDA;
        b->ntiles2 = (int)t.size();
        if (b->grid2 > b->ntiles2) b->grid2 = b->ntiles2;
        return TRTR_OK;
    }
};

// Calls f with a Batch2Launch<S, SRC, SR> of the batch's storage, source mode and rounding.
template <class F>
auto with_batch2(const trtr_batch* b, F&& f) {
    auto by_src = [&](auto* sp, auto sr) {
        using S = std::remove_pointer_t<decltype(sp)>;
        constexpr bool SR = decltype(sr)::value;
        return b->src == TRTR_SRC_PULSE ? f(Batch2Launch<S, TRTR_SRC_PULSE, SR>()) : f(Batch2Launch<S, TRTR_SRC_NONE, SR>());
    };
    using TrueT = std::integral_constant<bool, true>;
    using FalseT = std::integral_constant<bool, false>;
    if (b->precision == TRTR_F16_OFS) return b->sr ? by_src((__half*)nullptr, TrueT()) : by_src((__half*)nullptr, FalseT());
    if (b->precision == TRTR_BF16_OFS)
        return b->sr ? by_src((__nv_bfloat16*)nullptr, TrueT()) : by_src((__nv_bfloat16*)nullptr, FalseT());
    return by_src((float*)nullptr, FalseT());
}

cudaError_t launch_two(trtr_batch* b, int parity) {
    return with_batch2(b, [&](auto l) { return decltype(l)::launch(b, parity); });
}

trtr_status setup_two_step(trtr_batch* b) {
    return with_batch2(b, [&](auto l) { return decltype(l)::setup(b); });
}

size_t desc_size(int precision) {
    return precision == TRTR_F64 ? sizeof(InstanceDesc<double>) : sizeof(InstanceDesc<float>);
}

// Work-list of (instance, i0, j0) for a tile shape and schedule.
std::vector<int4> make_tiles(const trtr_batch* b, int geom, int schedule) {
    const int bx = kGeoms[geom].bx, by = kGeoms[geom].by;
    std::vector<int> order(b->count);
    for (int k = 0; k < b->count; ++k) order[k] = k;
    if (schedule == 2)
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            return (long long)b->ctx[a]->p.nx * b->ctx[a]->p.ny > (long long)b->ctx[c]->p.nx * b->ctx[c]->p.ny;
        });
    std::vector<int4> t;
    for (int k : order) {
        const int nx = b->ctx[k]->p.nx, ny = b->ctx[k]->p.ny;
        const int gx = b->ctx[k]->lp.gx | (b->ctx[k]->lf.gx << 16);
        for (int j0 = 0; j0 < ny; j0 += by)
            for (int i0 = 0; i0 < nx; i0 += bx) t.push_back(make_int4(k, i0, j0, gx));
    }
    return t;
}

trtr_status apply_config(trtr_batch* b, int config) {
    const int geom = config / kNumSchedules, schedule = config % kNumSchedules;
    if (b->graph_valid) {
        cudaGraphExecDestroy(b->graph);
        b->graph_valid = false;
    }
    if (dispatch(b, geom, 0) != cudaSuccess) return TRTR_ECUDA;
    if (dispatch(b, geom, 2) != cudaSuccess) return TRTR_ECUDA;
    std::vector<int4> t = make_tiles(b, geom, schedule);
    if (b->d_tiles) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
    }
    if (cudaMalloc(&b->d_tiles, t.size() * sizeof(int4)) != cudaSuccess) return TRTR_ENOMEM;
    if (cudaMemcpy(b->d_tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return TRTR_ECUDA;
    b->ntiles = (int)t.size();
    if (b->grid > b->ntiles) b->grid = b->ntiles;
    b->config = config;
    return TRTR_OK;
}

cudaError_t launch_one(trtr_batch* b, int parity) {
    const int geom = b->config / kNumSchedules, schedule = b->config % kNumSchedules;
    return dispatch(b, geom, 1, parity, schedule_mode(schedule));
}

// Two-step graph: parity 0 then parity 1.
trtr_status build_graph(trtr_batch* b) {
    if (b->graph_valid) return TRTR_OK;
    cudaGraph_t g;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TRTR_ECUDA;
    cudaError_t e0 = launch_one(b, 0);
    cudaError_t e1 = launch_one(b, 1);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e0 != cudaSuccess || e1 != cudaSuccess || e != cudaSuccess) {
        cudaGetLastError();
        return TRTR_ECUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return TRTR_ECUDA;
    b->graph_valid = true;
    return TRTR_OK;
}

trtr_status reset_clock(trtr_batch* b) {
    std::vector<TimeUniforms> u(b->count);
    std::vector<TimeFields2> u2(b->count);
    for (int k = 0; k < b->count; ++k) {
        u[k] = time_fields(b->pulses[k], b->ctx[k]->p.dt, b->step);
        u2[k] = TimeFields2{u[k], time_fields(b->pulses[k], b->ctx[k]->p.dt, b->step + 1)};
    }
    if (b->d_tu2 && cudaMemcpyAsync(b->d_tu2, u2.data(), u2.size() * sizeof(TimeFields2), cudaMemcpyHostToDevice,
                                    b->stream) != cudaSuccess)
        return TRTR_ECUDA;
    BatchClock c;
    c.n = b->step;
    c.done = 0;
    c.next = 0;
    if (cudaMemcpyAsync(b->d_tu, u.data(), u.size() * sizeof(TimeUniforms), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_clk, &c, sizeof(c), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return TRTR_ECUDA;
    return TRTR_OK;
}

// Two-launch graph of the two-step kernel: parity 0 then parity 1 (four steps).
trtr_status build_graph2(trtr_batch* b) {
    if (b->graph2_valid) return TRTR_OK;
    cudaGraph_t g;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TRTR_ECUDA;
    cudaError_t e0 = launch_two(b, 0);
    cudaError_t e1 = launch_two(b, 1);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e0 != cudaSuccess || e1 != cudaSuccess || e != cudaSuccess) {
        cudaGetLastError();
        return TRTR_ECUDA;
    }
    e = cudaGraphInstantiate(&b->graph2, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return TRTR_ECUDA;
    b->graph2_valid = true;
    return TRTR_OK;
}

// n steps: pairs through the two-step kernel where it applies (steps_per_launch 2), the rest
// (an odd step, or all with steps_per_launch 1) through the one-step kernel of the configured
// geometry.  Both kernels advance the device clock and both time tables, so they interleave.
trtr_status advance(trtr_batch* b, long n, int steps_per_launch) {
    for (int k = 0; k < b->count; ++k)
        if (b->ctx[k]->step != b->step || b->ctx[k]->cur != b->parity) return TRTR_ESTATE;
    long left = n;
    int par = b->parity;
    bool last_two = false;
    if (b->two_step && steps_per_launch == 2 && left >= 2) {
        for (int k = 0; k < b->count; ++k) {
            trtr_ctx* c = b->ctx[k];  // instances share the batch's stream
            if (!c->fld2_ready) {
                if (launch_pack_fields2(c) != cudaSuccess) return TRTR_ECUDA;
                c->fld2_ready = true;
            }
            if (!c->ghost2_ready && launch_refresh_ghosts2(c) != cudaSuccess) return TRTR_ECUDA;
        }
        long pairs = left / 2;
        left -= 2 * pairs;
        if (par == 1) {
            if (launch_two(b, 1) != cudaSuccess) return TRTR_ECUDA;
            par = 0;
            --pairs;
        }
        if (pairs >= 2) {
            trtr_status s = build_graph2(b);
            if (s != TRTR_OK) return s;
            for (; pairs >= 2; pairs -= 2)
                if (cudaGraphLaunch(b->graph2, b->stream) != cudaSuccess) return TRTR_ECUDA;
        }
        if (pairs == 1) {
            if (launch_two(b, 0) != cudaSuccess) return TRTR_ECUDA;
            par = 1;
        }
        last_two = true;
    }
    if (left > 0) last_two = false;  // one-step launches follow: the one-wide ghost frame
    if (left > 0 && par == 1) {  // bring the ping-pong to parity 0 for the graph
        if (launch_one(b, 1) != cudaSuccess) return TRTR_ECUDA;
        par = 0;
        --left;
    }
    if (left >= 2) {
        trtr_status s = build_graph(b);
        if (s != TRTR_OK) return s;
        for (; left >= 2; left -= 2)
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return TRTR_ECUDA;
    }
    if (left == 1) {
        if (launch_one(b, 0) != cudaSuccess) return TRTR_ECUDA;
        par = 1;
    }
    b->step += n;
    b->parity = par;
    for (int k = 0; k < b->count; ++k) {
        b->ctx[k]->step = b->step;
        b->ctx[k]->cur = b->parity;
        if (n > 0) b->ctx[k]->ghost2_ready = last_two;
        b->ctx[k]->launches += n;
    }
    return TRTR_OK;
}

}  // namespace
TRTR_BOUNDS_TAKE(batch)

}  // namespace trtr

extern "C" {

trtr_status trtr_batch_create(const trtr_instance* inst, int count, void* cuda_stream, trtr_batch** out) {
    if (!out) return TRTR_EINVAL;
    *out = nullptr;
    if (!inst || count < 1) return TRTR_EINVAL;
    const int prec = inst[0].p.precision;
    if (prec != TRTR_F32 && prec != TRTR_F16_OFS && prec != TRTR_BF16_OFS) return TRTR_EINVAL;
    int src = TRTR_SRC_NONE;
    for (int k = 0; k < count; ++k) {
        if (inst[k].p.precision != prec) return TRTR_EINVAL;
        if (inst[k].p.src_mode == TRTR_SRC_FIELD || inst[k].p.bc_mode != TRTR_BC_PERIODIC) return TRTR_EINVAL;
        if (inst[k].p.rounding != inst[0].p.rounding ||
            (inst[k].p.rounding != TRTR_ROUND_STOCHASTIC && inst[k].p.rounding != TRTR_ROUND_NEAREST))
            return TRTR_EINVAL;
        if (inst[k].p.src_mode == TRTR_SRC_PULSE) src = TRTR_SRC_PULSE;
    }
    trtr_batch* b = new (std::nothrow) trtr_batch();
    if (!b) return TRTR_ENOMEM;
    b->count = count;
    b->precision = prec;
    b->sr = prec != TRTR_F32 && inst[0].p.rounding == TRTR_ROUND_STOCHASTIC;
    b->src = src;
    b->config = trtr::kDefaultConfig;
    b->ctx = static_cast<trtr_ctx**>(calloc(count, sizeof(trtr_ctx*)));
    if (!b->ctx) {
        delete b;
        return TRTR_ENOMEM;
    }
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!b->stream) {  // graphs cannot be captured on the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            free(b->ctx);
            delete b;
            return TRTR_ECUDA;
        }
        b->own_stream = true;
    }
    trtr_status s = TRTR_OK;
    for (int k = 0; k < count && s == TRTR_OK; ++k) {
        const trtr_instance& in = inst[k];
        s = trtr_create(&in.p, b->stream, &b->ctx[k]);
        if (s == TRTR_OK) s = trtr_set_pulse(b->ctx[k], in.omega, in.xc, in.yc, in.sigma0, in.D0, in.D_amp);
        if (s == TRTR_OK) s = trtr_init_equilibrium(b->ctx[k], nullptr, 0);
        if (s == TRTR_OK) {
            b->nodes += (long long)in.p.nx * in.p.ny;
            b->pulses.push_back(b->ctx[k]->pulse);
        }
    }
    if (s == TRTR_OK &&
        (cudaMalloc(&b->d_desc, trtr::desc_size(prec) * count) != cudaSuccess ||
         cudaMalloc(&b->d_tu, sizeof(TimeUniforms) * count) != cudaSuccess ||
         cudaMalloc(&b->d_clk, sizeof(BatchClock)) != cudaSuccess || cudaMalloc(&b->d_flag, sizeof(int)) != cudaSuccess ||
         cudaMallocHost(&b->h_flag, sizeof(int)) != cudaSuccess ||
         cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream) != cudaSuccess)) {
        cudaGetLastError();
        s = TRTR_ENOMEM;
    }
    if (s == TRTR_OK) s = trtr::apply_config(b, b->config);
    // two steps per launch where every instance has the two-step kernel's packed fields
    b->steps_per_launch = 2;
    b->two_step = s == TRTR_OK;  // where every instance has the two-step fields (FP32, or 2-byte with even nx)
    for (int k = 0; k < count && b->two_step; ++k) b->two_step = b->ctx[k]->fld2 != nullptr;
    if (s == TRTR_OK && b->two_step &&
        (cudaMalloc(&b->d_desc2, sizeof(trtr::InstanceDesc2) * count) != cudaSuccess ||
         cudaMalloc(&b->d_tu2, sizeof(TimeFields2) * count) != cudaSuccess)) {
        cudaGetLastError();
        s = TRTR_ENOMEM;
    }
    if (s == TRTR_OK && b->two_step) s = trtr::setup_two_step(b);
    if (s == TRTR_OK) s = trtr::reset_clock(b);
    if (s != TRTR_OK) {
        trtr_batch_destroy(b);
        return s;
    }
    *out = b;
    return TRTR_OK;
}

trtr_status trtr_batch_destroy(trtr_batch* b) {
    if (!b) return TRTR_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph_valid) cudaGraphExecDestroy(b->graph);
    if (b->graph2_valid) cudaGraphExecDestroy(b->graph2);
    for (int k = 0; k < b->count; ++k)
        if (b->ctx && b->ctx[k]) trtr_destroy(b->ctx[k]);
    void* ptrs[] = {b->d_desc, b->d_tiles, b->d_tu, b->d_clk, b->d_flag, b->d_desc2, b->d_tiles2, b->d_tu2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->h_flag) cudaFreeHost(b->h_flag);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    free(b->ctx);
    delete b;
    return TRTR_OK;
}

int trtr_batch_config_count(void) { return trtr::kNumConfigs; }

const char* trtr_batch_config_name(int config) {
    static const char* names[trtr::kNumConfigs] = {
        "tile 128x8, interleaved",  "tile 128x8, chunked",  "tile 128x8, chunked largest-first",  "tile 128x8, dynamic",
        "tile 64x8, interleaved",   "tile 64x8, chunked",   "tile 64x8, chunked largest-first",   "tile 64x8, dynamic",
        "tile 128x4, interleaved",  "tile 128x4, chunked",  "tile 128x4, chunked largest-first",  "tile 128x4, dynamic",
        "tile 128x16, interleaved", "tile 128x16, chunked", "tile 128x16, chunked largest-first", "tile 128x16, dynamic",
        "tile 64x16, interleaved",  "tile 64x16, chunked",  "tile 64x16, chunked largest-first",  "tile 64x16, dynamic"};
    return config >= 0 && config < trtr::kNumConfigs ? names[config] : "invalid";
}

trtr_status trtr_batch_set_config(trtr_batch* b, int config) {
    if (!b || config < 0 || config >= trtr::kNumConfigs) return TRTR_EINVAL;
    return trtr::apply_config(b, config);
}

trtr_status trtr_batch_set_steps_per_launch(trtr_batch* b, int k) {
    if (!b || (k != 1 && k != 2)) return TRTR_EINVAL;
    b->steps_per_launch = k;
    return TRTR_OK;
}

trtr_status trtr_batch_get_steps_per_launch(const trtr_batch* b, int* k) {
    if (!b || !k) return TRTR_EINVAL;
    *k = b->two_step && b->steps_per_launch == 2 ? 2 : 1;
    return TRTR_OK;
}

trtr_status trtr_batch_step(trtr_batch* b, long n) {
    trtr::TraceRange trace("trtr_batch_step");
    if (!b || n < 0) return TRTR_EINVAL;
    return trtr::advance(b, n, b->steps_per_launch);
}

trtr_status trtr_batch_sync(trtr_batch* b) {
    if (!b) return TRTR_EINVAL;
    if (cudaMemcpyAsync(b->h_flag, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return TRTR_ECUDA;
    }
#if TRTR_BOUNDS_CHECK
    if (*b->h_flag == 0) {
        unsigned long long log[3];
        if (trtr::bounds_take_all(b->stream, log) != cudaSuccess) {
            cudaGetLastError();
            return TRTR_ECUDA;
        }
        return log[0] != 0ull ? TRTR_EBOUNDS : TRTR_OK;
    }
#endif
    if (*b->h_flag == 0) return TRTR_OK;
    // reported once: cleared for the following steps
    if (cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream) != cudaSuccess) {
        cudaGetLastError();
        return TRTR_ECUDA;
    }
    return TRTR_ETIMEOUT;
}

trtr_status trtr_batch_tune(trtr_batch* b, int trial_steps, int* config_out, float* ms_out) {
    if (!b || trial_steps < 2) return TRTR_EINVAL;
    const bool restart = b->step == 0;
    // At step 0 the trials run from the caller's state, whatever set it (the pulse, phi0 or
    // populations): every instance's current buffer, ghost frame included, is kept in one
    // temporary device copy and put back afterwards.
    std::vector<size_t> off(b->count + 1, 0);
    std::vector<int> cur0(b->count);
    std::vector<char> ghost0(b->count);
    unsigned char* keep = nullptr;
    if (restart) {
        for (int k = 0; k < b->count; ++k) {
            const trtr_ctx* c = b->ctx[k];
            off[k + 1] = off[k] + (size_t)trtr::kQ * c->lp.plane * (size_t)c->esize;
            cur0[k] = c->cur;
            ghost0[k] = c->ghost2_ready;
        }
        if (cudaMalloc(&keep, off[b->count]) != cudaSuccess) {
            cudaGetLastError();
            return TRTR_ENOMEM;
        }
        for (int k = 0; k < b->count; ++k)
            if (cudaMemcpyAsync(keep + off[k], b->ctx[k]->pop[cur0[k]], off[k + 1] - off[k], cudaMemcpyDeviceToDevice,
                                b->stream) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(keep);
                return TRTR_ECUDA;
            }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (keep) cudaFree(keep);
        return TRTR_ECUDA;
    }
    int best = b->config;
    float best_ms = 1e30f;
    trtr_status s = TRTR_OK;
    for (int c = 0; c < trtr::kNumConfigs && s == TRTR_OK; ++c) {
        s = trtr::apply_config(b, c);
        if (s != TRTR_OK) break;
        s = trtr::advance(b, 2, 1);  // warm-up (graph capture, caches); the one-step configs
        if (s != TRTR_OK) break;
        cudaEventRecord(e0, b->stream);
        s = trtr::advance(b, trial_steps - trial_steps % 2, 1);
        cudaEventRecord(e1, b->stream);
        if (s != TRTR_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            s = TRTR_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)(trial_steps - trial_steps % 2);
        if (ms_out) ms_out[c] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == TRTR_OK) s = trtr::apply_config(b, best);
    if (restart) {  // trials started from the state at step 0: put it back
        for (int k = 0; k < b->count && s == TRTR_OK; ++k) {
            trtr_ctx* c = b->ctx[k];
            if (cudaMemcpyAsync(c->pop[cur0[k]], keep + off[k], off[k + 1] - off[k], cudaMemcpyDeviceToDevice,
                                b->stream) != cudaSuccess) {
                cudaGetLastError();
                s = TRTR_ECUDA;
                break;
            }
            c->cur = cur0[k];
            c->ghost2_ready = ghost0[k] != 0;
            c->step = 0;
        }
        if (s == TRTR_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) {
            cudaGetLastError();
            s = TRTR_ECUDA;
        }
        cudaFree(keep);
        if (s == TRTR_OK) {
            b->step = 0;
            b->parity = cur0.empty() ? 0 : cur0[0];
            s = trtr::reset_clock(b);
        }
    }
    if (s == TRTR_OK && config_out) *config_out = best;
    return s;
}

trtr_status trtr_batch_instance(trtr_batch* b, int k, trtr_ctx** ctx) {
    if (!b || !ctx || k < 0 || k >= b->count) return TRTR_EINVAL;
    *ctx = b->ctx[k];
    return TRTR_OK;
}

trtr_status trtr_batch_info(const trtr_batch* b, int* count, long long* nodes, long* step, int* config) {
    if (!b) return TRTR_EINVAL;
    if (count) *count = b->count;
    if (nodes) *nodes = b->nodes;
    if (step) *step = b->step;
    if (config) *config = b->config;
    return TRTR_OK;
}

}  // extern "C"
