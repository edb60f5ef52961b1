// trtr_step2.cu -- two time steps of the evolution equation (14) per launch (temporal blocking
// of the fused TRT-R step), for FP32 storage, periodic boundaries and no source or the
// manufactured pulse source.  The node update is the one-step kernel's (collide_node, the
// same source and acceleration arithmetic), so two steps here give the bits of two one-step
// launches; what changes is the data movement: the populations are read and written once per
// two steps.
//
// Tile: BX x BY output nodes (i0.., j0..).  One TMA box of depth 9 brings P (the previous
// step's post-collision values) over columns [i0 - 4, i0 + BX + 4) and rows [j0 - 2, j0 + BY + 2),
// one box of depth 5 the packed fields (uhat, a = uhat . grad uhat, Dh) over the rows
// [j0 - 1, j0 + BY + 1).  The population planes keep a two-wide ghost frame of periodic copies,
// so the two-node halo is a plain tile read at the edges too.
//   Step 1 runs on the halo region R1 = columns [i0 - 2, i0 + BX + 2) x rows [j0 - 1, j0 + BY + 1)
//   (its outermost columns are computed and not used).  Node (r, c) of R1 pulls
//   g_q = P_q(x - e_q) from the stage at (row r + 1 - ey_q, column c + 2 - ex_q); that slot is
//   pulled by this node alone, so the node writes its post-collision value P1_q back into the
//   same slot (in place, no second buffer).
//   Step 2 runs on the output nodes: node (r2, c2) = R1 node (r2 + 1, c2 + 2) pulls
//   P1_q(x - e_q) from (row r2 + 2 - 2 ey_q, column c2 + 4 - 2 ex_q) and stores P2 to global
//   memory with its ghost copies (nodes within two of an edge).
// Geometry (Geom2For): narrow tiles (32 columns; 8 rows with the pulse source, 16 without) and
// several CTAs per SM with two stages each, so that while one CTA waits at the barrier between
// its two steps the others compute (the kernel is latency-bound, not HBM-bound).
// R1 nodes outside the grid are periodic images: their populations come from the ghost frame,
// their fields from the packed fields' ghost frame (copies of the wrapped node, the acceleration
// included, whatever the gradient mode), and their source from the wrapped node's coordinates,
// so they compute exactly what the wrapped node computes.
#include "trtr_step_core.cuh"

namespace trtr {
namespace {

using namespace core;

constexpr int kT2NF = 5;  // packed fields: uhat_x, uhat_y, a_x, a_y, Dh

// Stage of one BX x BY output tile: the population box (9 planes) and the field box (5 planes).
template <int BX, int BY>
struct Tile2 {
    static constexpr int X = BX, Y = BY;
    static constexpr int W = BX + 8;                     // staged columns [i0 - 4, i0 + BX + 4)
    static constexpr int PR = BY + 4;                    // staged population rows
    static constexpr int FR = BY + 2;                    // staged field rows
    static constexpr int R1 = (BY + 2) * (BX + 4) / 2;  // node pairs of step 1
    static constexpr int R2 = BY * BX / 2;               // node pairs of step 2
    static constexpr int PopPlane = PR * W;              // floats
    static constexpr int FldPlane = FR * W;
    static constexpr int PopBytes = kQ * PopPlane * 4;
    static constexpr int FldBytes = kT2NF * FldPlane * 4;
    static constexpr int TX = PopBytes + FldBytes;       // bytes per tile (boxes include any fill)
    static constexpr int Stage = (TX + 127) / 128 * 128;
    static_assert(BX % 4 == 0, "tile origins on 16-byte boundaries");
    static_assert(PopBytes % 128 == 0, "the field box must start on a 128-byte boundary");
    static_assert(W <= 256 && PR <= 256, "TMA box dimensions are at most 256");
};

template <int STAGES, int CTAS, int THREADS, int BX, int BY>
struct Geom2 {
    static constexpr int kStages = STAGES, kCtas = CTAS, kThreads = THREADS;
    using T = Tile2<BX, BY>;
    static_assert(STAGES * T::Stage + 256 <= 227 * 1024, "the stages must fit in shared memory");
};
// Geometry per source mode (stages, CTAs per SM, threads, tile width, tile height), from the
// sweeps of rebuilds with -DTRTR_STEP2_STAGES=S -DTRTR_STEP2_CTAS=C -DTRTR_STEP2_THREADS=T
// -DTRTR_STEP2_BX=X -DTRTR_STEP2_BY=Y (all five; they set it for both modes): a few
// independent CTAs per SM hide each one's barrier between the two steps, the pulse source's
// arithmetic favours more of them.
template <int SRC>
struct Geom2For {  // in-kernel pulse source
    using type = Geom2<2, 3, 128, 32, 8>;
};
template <>
struct Geom2For<TRTR_SRC_NONE> {
    using type = Geom2<2, 2, 256, 32, 16>;
};
#ifdef TRTR_STEP2_BX
template <int SRC>
using Geom2Of = Geom2<TRTR_STEP2_STAGES, TRTR_STEP2_CTAS, TRTR_STEP2_THREADS, TRTR_STEP2_BX, TRTR_STEP2_BY>;
#else
template <int SRC>
using Geom2Of = typename Geom2For<SRC>::type;
#endif

struct alignas(16) Step2Args {
    StepArgs<float> a;  // tf: the pulse uniforms of the first step
    TimeFields<float> tf2;  // of the second step
};

// Wrapped index of a node of the halo region (v in [-2, n + 1] with n >= 2 maps onto its
// periodic image); indices of the unused nodes past that are clamped into the tables.
__device__ __forceinline__ int wrap_clamp(int v, int n) {
    v = v < 0 ? v + n : (v >= n ? v - n : v);
    return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// Source term s = dt S^n + dt/2 (S^n - S^{n-1}) of the pair (xi0, xi1) in row yj: the one-step
// kernel's expressions, node coordinates from the wrapped indices.
template <int SRC>
__device__ __forceinline__ F2 pair_source(const StepArgs<float>& a, const TimeFields<float>& tf, int xi0, int xi1,
                                          int yj) {
    if (SRC != TRTR_SRC_PULSE) return F2(0.f);
    const int nx = a.lp.nx, ny = a.lp.ny;
    const float* tx = reinterpret_cast<const float*>(a.tab_x);
    const float* ty = reinterpret_cast<const float*>(a.tab_y);
    const F2 sxm(__ldg(tx + xi0), __ldg(tx + xi1));
    const F2 cxm(__ldg(tx + nx + xi0), __ldg(tx + nx + xi1));
    const float sy = __ldg(ty + yj), cy = __ldg(ty + ny + yj);
    const F2 x = vfma(F2((float)xi0, (float)xi1), F2(a.dx), F2(a.x0));
    const F2 y(a.y0 + (float)yj * a.dx);
    const F2 dD = F2(a.dD_amp * sy) * sxm;
    const F2 dDx = F2(a.dD_amp * 3.14159265358979323846f * sy) * cxm;
    const F2 dDy = F2(a.dD_amp * 3.14159265358979323846f * cy) * sxm;
    const F2 Sn = pulse_source(x, y, F2(tf.cx_n), F2(tf.cy_n), F2(tf.inv_s2_n), F2(tf.amp_n), dD, dDx, dDy);
    const F2 Sp = pulse_source(x, y, F2(tf.cx_p), F2(tf.cy_p), F2(tf.inv_s2_p), F2(tf.amp_p), dD, dDx, dDy);
    return F2(a.dt) * vfma(F2(1.5f), Sn, F2(-0.5f) * Sp);
}

template <int SRC, class G>
__global__ void __launch_bounds__(G::kThreads, G::kCtas)
    step2_kernel(const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap mf, const Step2Args args) {
    constexpr int STAGES = G::kStages, kT2Threads = G::kThreads;
    using T = typename G::T;
    constexpr int kT2X = T::X, kT2Y = T::Y, kT2W = T::W, kT2R1 = T::R1, kT2R2 = T::R2;
    constexpr int kT2PopPlane = T::PopPlane, kT2FldPlane = T::FldPlane, kT2PopBytes = T::PopBytes;
    constexpr int kT2TX = T::TX, kT2Stage = T::Stage;
    const StepArgs<float>& a = args.a;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * kT2Stage);

    const int tid = threadIdx.x;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const int ntx = (nx + kT2X - 1) / kT2X, nty = (ny + kT2Y - 1) / kT2Y;
    const int ntiles = ntx * nty;
    const int first = blockIdx.x, stride = gridDim.x;
    const int my_tiles = first < ntiles ? (ntiles - 1 - first) / stride + 1 : 0;
    auto tile_x0 = [&](int k) { return ((first + k * stride) % ntx) * kT2X; };
    auto tile_y0 = [&](int k) { return ((first + k * stride) / ntx) * kT2Y; };
    auto issue = [&](int k, int s) {
        unsigned char* stage = smem + s * kT2Stage;
        const int x = tile_x0(k) + a.lp.gx - 4, y0 = tile_y0(k);
        mbar_expect_tx(&full[s], kT2TX);
        if (tma_ok(stage, x, y0 + kGhostP - 2, 4)) tma_load_3d(stage, &mp, &full[s], x, y0 + kGhostP - 2, 0);
        if (tma_ok(stage + kT2PopBytes, x, y0 + kGhostP - 1, 4))
            tma_load_3d(stage + kT2PopBytes, &mf, &full[s], x, y0 + kGhostP - 1, 0);
    };

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0)
        for (int k = 0; k < STAGES && k < my_tiles; ++k) issue(k, k);

    float* dst = static_cast<float*>(a.dst);
    const size_t pl = a.lp.plane;
    const F2 magic(a.magic), w2f(a.omega2_fixed);

    for (int k = 0; k < my_tiles; ++k) {
        const int s = k % STAGES;
        const int i0 = tile_x0(k), j0 = tile_y0(k);
        const bool ok = mbar_wait_bounded(&full[s], (k / STAGES) & 1);
        if (!ok) s_abort = 1;
        float* sp = reinterpret_cast<float*>(smem + s * kT2Stage);
        const float* sf = reinterpret_cast<const float*>(smem + s * kT2Stage + kT2PopBytes);
        if (ok) {
            // step 1 over the halo region, in place
            for (int p = tid; p < kT2R1; p += kT2Threads) {
                const int r = p / ((kT2X + 4) / 2), c = 2 * (p - r * ((kT2X + 4) / 2));
                F2 g[kQ];
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const float* src = sp + q * kT2PopPlane + (r + 1 - lattice_ey(q)) * kT2W + c + 2 - lattice_ex(q);
                    if (lattice_ex(q) == 0)
                        g[q] = F2(*reinterpret_cast<const float2*>(src));
                    else
                        g[q] = F2(src[0], src[1]);
                }
                const float* f = sf + r * kT2W + c + 2;
                const F2 ux(*reinterpret_cast<const float2*>(f));
                const F2 uy(*reinterpret_cast<const float2*>(f + kT2FldPlane));
                const F2 ax(*reinterpret_cast<const float2*>(f + 2 * kT2FldPlane));
                const F2 ay(*reinterpret_cast<const float2*>(f + 3 * kT2FldPlane));
                const F2 Dh(*reinterpret_cast<const float2*>(f + 4 * kT2FldPlane));
                const int x = i0 - 2 + c, y = j0 - 1 + r;
                const F2 src = pair_source<SRC>(a, a.tf, wrap_clamp(x, nx), wrap_clamp(x + 1, nx), wrap_clamp(y, ny));
                F2 out[kQ];
                collide_node<F2>(g, ux, uy, ax, ay, Dh, src, magic, w2f, a.tau2_fixed, out);
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    float* d = sp + q * kT2PopPlane + (r + 1 - lattice_ey(q)) * kT2W + c + 2 - lattice_ex(q);
                    if (lattice_ex(q) == 0) {
                        *reinterpret_cast<float2*>(d) = out[q].v;
                    } else {
                        d[0] = out[q].v.x;
                        d[1] = out[q].v.y;
                    }
                }
            }
        }
        __syncthreads();  // P1 complete (and s_abort visible)
        if (ok && !s_abort) {
            // step 2 on the output nodes
            for (int p = tid; p < kT2R2; p += kT2Threads) {
                const int r2 = p / (kT2X / 2), c2 = 2 * (p - r2 * (kT2X / 2));
                const int i = i0 + c2, j = j0 + r2;
                if (i >= nx || j >= ny) continue;
                F2 g[kQ];
#pragma unroll
                for (int q = 0; q < kQ; ++q)
                    g[q] = F2(*reinterpret_cast<const float2*>(sp + q * kT2PopPlane +
                                                              (r2 + 2 - 2 * lattice_ey(q)) * kT2W + c2 + 4 -
                                                              2 * lattice_ex(q)));
                const float* f = sf + (r2 + 1) * kT2W + c2 + 4;
                const F2 ux(*reinterpret_cast<const float2*>(f));
                const F2 uy(*reinterpret_cast<const float2*>(f + kT2FldPlane));
                const F2 ax(*reinterpret_cast<const float2*>(f + 2 * kT2FldPlane));
                const F2 ay(*reinterpret_cast<const float2*>(f + 3 * kT2FldPlane));
                const F2 Dh(*reinterpret_cast<const float2*>(f + 4 * kT2FldPlane));
                const F2 src = pair_source<SRC>(a, args.tf2, i, i + 1 < nx ? i + 1 : nx - 1, j);
                F2 out[kQ];
                collide_node<F2>(g, ux, uy, ax, ay, Dh, src, magic, w2f, a.tau2_fixed, out);
                const bool edge = j < kGhostP || j >= ny - kGhostP || i < kGhostP || i + 1 >= nx - kGhostP;
                if (!edge) {
                    float* d0 = dst + a.lp.at_g<kGhostP>(i, j);
#if TRTR_BOUNDS_CHECK
                    if ((reinterpret_cast<uintptr_t>(d0) & 7u) != 0u) {
                        TRTR_BOUNDS_FAULT(kBoundsPair, i, j);
                        continue;
                    }
#endif
#pragma unroll
                    for (int q = 0; q < kQ; ++q) *reinterpret_cast<float2*>(d0 + q * pl) = out[q].v;
                } else {
#pragma unroll
                    for (int q = 0; q < kQ; ++q) {
                        store_with_ghosts<kGhostP, kGhostP>(dst + q * pl, a.lp, i, j, out[q].v.x);
                        if (i + 1 < nx) store_with_ghosts<kGhostP, kGhostP>(dst + q * pl, a.lp, i + 1, j, out[q].v.y);
                    }
                }
            }
        }
        __syncthreads();  // stage s fully read
        if (s_abort) {
            if (tid == 0) {
                atomicExch(a.flag, 1);
                for (int kk = k + 1; kk < my_tiles && kk < k + STAGES; ++kk)
                    mbar_wait_bounded(&full[kk % STAGES], (kk / STAGES) & 1);
            }
            return;
        }
        if (tid == 0 && k + STAGES < my_tiles) issue(k + STAGES, s);
    }
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
__global__ void refresh_ghosts2_kernel(float* P, PlaneLayout L) {
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
        float* plane = P + (size_t)q * L.plane;
        plane[L.at_g<kGhostP>(i, j)] = plane[L.at_g<kGhostP>(wrap_clamp(i, L.nx), wrap_clamp(j, L.ny))];
    }
}

template <int SRC, class G>
cudaError_t launch2_typed(trtr_ctx* ctx) {
    auto kernel = step2_kernel<SRC, G>;
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
    a.dst = ctx->pop[ctx->cur ^ 1];
    a.tab_x = static_cast<const float*>(ctx->tab_x);
    a.tab_y = static_cast<const float*>(ctx->tab_y);
    a.flag = ctx->dflag;
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
    if (SRC == TRTR_SRC_PULSE) {
        const long n = ctx->step;
        const PulseTime t0 = pulse_at(ctx->pulse, (double)(n - 1) * ctx->p.dt);
        const PulseTime t1 = pulse_at(ctx->pulse, (double)n * ctx->p.dt);
        const PulseTime t2 = pulse_at(ctx->pulse, (double)(n + 1) * ctx->p.dt);
        a.dD_amp = (float)(ctx->pulse.D0 * ctx->pulse.D_amp);
        auto put = [](TimeFields<float>& tf, const PulseTime& tn, const PulseTime& tp) {
            tf.cx_n = (float)tn.cx; tf.cy_n = (float)tn.cy; tf.inv_s2_n = (float)tn.inv_s2; tf.amp_n = (float)tn.amp;
            tf.cx_p = (float)tp.cx; tf.cy_p = (float)tp.cy; tf.inv_s2_p = (float)tp.inv_s2; tf.amp_p = (float)tp.amp;
        };
        put(a.tf, t1, t0);
        put(args.tf2, t2, t1);
    }
    const long ntiles = (long)((ctx->lp.nx + G::T::X - 1) / G::T::X) * ((ctx->lp.ny + G::T::Y - 1) / G::T::Y);
    const long cap = (long)ctx->num_sms * ctas_per_sm;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntiles < cap ? ntiles : cap));
    cfg.blockDim = dim3(G::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, ctx->maps2[ctx->cur], ctx->maps2[2], args);
}

}  // namespace

bool two_step_applies(const trtr_ctx* ctx) {
    return ctx->fld2 != nullptr && ctx->steps_per_launch == 2 && ctx->p.bc_mode == TRTR_BC_PERIODIC &&
           (ctx->p.src_mode == TRTR_SRC_NONE || ctx->p.src_mode == TRTR_SRC_PULSE);
}

template <class G>
cudaError_t encode2_typed(trtr_ctx* ctx) {
    using T = typename G::T;
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        ok = ok && encode(&ctx->maps2[b], tma_type<float>(), 4, ctx->pop[b], ctx->lp, kQ, T::W, T::PR, kQ);
    ok = ok && encode(&ctx->maps2[2], tma_type<float>(), 4, ctx->fld2, ctx->lt, kT2NF, T::W, T::FR, kT2NF);
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_maps2(trtr_ctx* ctx) {
    if (!ctx->fld2) return cudaSuccess;
    return ctx->p.src_mode == TRTR_SRC_PULSE ? encode2_typed<Geom2Of<TRTR_SRC_PULSE>>(ctx)
                                             : encode2_typed<Geom2Of<TRTR_SRC_NONE>>(ctx);
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

cudaError_t launch_refresh_ghosts2(trtr_ctx* ctx) {
    const int n = 2 * (ctx->p.nx + 2 * kGhostP) + 2 * (ctx->p.ny + 2 * kGhostP - 2);
    const int want = (kQ * n + 255) / 256, cap = ctx->num_sms * 4;
    ctx->launches += 1;
    refresh_ghosts2_kernel<<<want < cap ? want : cap, 256, 0, ctx->stream>>>(static_cast<float*>(ctx->pop[ctx->cur]),
                                                                            ctx->lp);
    return cudaGetLastError();
}

cudaError_t launch_step2(trtr_ctx* ctx) {
    return ctx->p.src_mode == TRTR_SRC_PULSE ? launch2_typed<TRTR_SRC_PULSE, Geom2Of<TRTR_SRC_PULSE>>(ctx)
                                             : launch2_typed<TRTR_SRC_NONE, Geom2Of<TRTR_SRC_NONE>>(ctx);
}

TRTR_BOUNDS_TAKE(step2)

}  // namespace trtr
