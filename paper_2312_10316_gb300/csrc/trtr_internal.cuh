// trtr_internal.cuh -- context layout, storage traits and kernel launchers of the TRT-R
// library (not part of the public ABI).
//
// Device layout (all buffers owned by the context).  Every plane is "ghosted": the interior
// node (i, j) sits at row j + gy and column gx + i of a [rows][pitch] plane, where gx is one
// 128-byte line of columns, so interior rows start on a 128-byte boundary, and the gy columns
// before / after the interior and the gy rows above / below it hold ghost copies (gy = 2 for
// the populations, 1 for the fields of the one-step kernel):
//
//   populations  2 x [9][rows][pitch] in the storage type: the post-collision values P_i(x)
//                of the previous step; the pre-collision population is the pull
//                g_i(x, t_n) = P_i(x - e_i).  The ghost cells repeat the opposite edge
//                (periodic), so the pull never wraps and TMA tiles never need to.
//   fields       uv = [2][rows][pitch] (uhat_x, uhat_y) and Dh = [rows][pitch] in the compute
//                type, lattice units: uhat = u dt/dx, Dh = D dt/dx^2 (tau1 = 1/2 + 3 Dh).  The
//                u ghosts hold the periodic wrap (TRTR_GRAD_PERIODIC) or the linear
//                extrapolation 2u(edge) - u(edge -+ 1) (TRTR_GRAD_ONESIDED_EDGE), for which the
//                central difference at the edge node equals the one-sided difference.
//   source       [2][rows][pitch] dt*S in the compute type (TRTR_SRC_FIELD only)
//   pulse tab    [2][nx] sin(pi x_i), cos(pi x_i) and [2][ny] sin(pi y_j), cos(pi y_j)
//   edge values  [2 nx + 2 (ny - 2)] FP64 Dirichlet values of the edge nodes
//                (TRTR_BC_DIRICHLET_NEE), in the order of edge_node()
//   scratch      FP64 partial sums of the reductions, one pair per reduction block
//   flag         device int set by a kernel whose bounded wait gave up
// rows >= ny + 2 gy and pitch >= nx + 2 gx are padded so that every TMA box fits inside the
// allocation.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "trtr.h"

namespace trtr {

constexpr int kQ = 9;

struct Pulse {
    double omega, xc, yc, sigma0, D0, D_amp;
};

// Per-time uniforms of the pulse source / closed form, computed on the host in double.
struct PulseTime {
    double cx, cy;    // centre c(t)
    double inv_s2;    // 1 / s^2(t)
    double amp;       // s0^2 / s^2(t)
};

// ---- bounds-checked builds (TRTR_BOUNDS_CHECK=1) ----------------------------------------
// The debug build checks the kernels' memory accesses against the layout: every plane index
// (PlaneLayout::at), the pair stores, the bulk row copies and the TMA load coordinates.  An
// access out of bounds is recorded in this translation unit's log and then skipped, or kept
// inside the ghost frame; it never traps, so the context stays usable and the host reports
// TRTR_EBOUNDS at the next synchronisation.  The default build compiles none of it.
#ifndef TRTR_BOUNDS_CHECK
#define TRTR_BOUNDS_CHECK 0
#endif

enum BoundsKind {
    kBoundsPlane = 1,  // a plane index outside the interior and its ghost frame
    kBoundsPair = 2,   // a two-node store past the row or not aligned to the pair
    kBoundsBulk = 3,   // a bulk row copy outside the interior row, or not 16-byte aligned
    kBoundsTma = 4,    // a TMA load whose x coordinate or destination breaks the alignment rules
    kBoundsTile = 5,   // a tile column or row outside the tile
};

#if TRTR_BOUNDS_CHECK
// [0] number of accesses caught, [1] kind of the first, [2] its (j << 32 | i); one log per
// translation unit (read and cleared by bounds_take_<unit>()).
static __device__ unsigned long long bounds_log[3];
__device__ __forceinline__ void bounds_fault(int kind, int i, int j) {
    if (atomicAdd(&bounds_log[0], 1ull) == 0ull) {
        bounds_log[1] = (unsigned long long)kind;
        bounds_log[2] = ((unsigned long long)(unsigned)j << 32) | (unsigned)i;
    }
}
#define TRTR_BOUNDS_FAULT(kind, i, j) ::trtr::bounds_fault((kind), (i), (j))
#else
#define TRTR_BOUNDS_FAULT(kind, i, j) ((void)0)
#endif

// Host side of a translation unit's log: copies {count, kind, where} to `out` and clears it
// (zeros in the default build).
#if TRTR_BOUNDS_CHECK
#define TRTR_BOUNDS_TAKE(unit)                                                                       \
    cudaError_t bounds_take_##unit(cudaStream_t s, unsigned long long* out) {                        \
        static const unsigned long long zero[3] = {0ull, 0ull, 0ull};                                \
        cudaError_t e = cudaMemcpyFromSymbolAsync(out, bounds_log, sizeof(zero), 0,                  \
                                                  cudaMemcpyDeviceToHost, s);                        \
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);                                          \
        if (e == cudaSuccess && out[0] != 0ull)                                                      \
            e = cudaMemcpyToSymbolAsync(bounds_log, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s); \
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);                                          \
        return e;                                                                                    \
    }
#else
#define TRTR_BOUNDS_TAKE(unit)                                                \
    cudaError_t bounds_take_##unit(cudaStream_t, unsigned long long* out) {   \
        out[0] = out[1] = out[2] = 0ull;                                      \
        return cudaSuccess;                                                   \
    }
#endif
cudaError_t bounds_take_step(cudaStream_t s, unsigned long long* out);
cudaError_t bounds_take_aux(cudaStream_t s, unsigned long long* out);
cudaError_t bounds_take_batch(cudaStream_t s, unsigned long long* out);
cudaError_t bounds_take_adjoint(cudaStream_t s, unsigned long long* out);
cudaError_t bounds_take_step2(cudaStream_t s, unsigned long long* out);
// All units: the summed count, and the kind and place of the first unit's first access.
cudaError_t bounds_take_all(cudaStream_t s, unsigned long long* out);

// Ghost frame widths: the population planes keep two ghost columns and rows on each side (the
// two-step kernel pulls twice across an edge); the field planes of the one-step kernel one.
constexpr int kGhostP = 2;
constexpr int kGhostF = 1;

struct PlaneLayout {
    int nx, ny;
    int gx;        // column of interior x = 0 (128 bytes of columns)
    int gy;        // row of interior y = 0 = width of the ghost frame
    int pitch;     // elements per row
    int rows;      // rows per plane (>= ny + 2 gy)
    size_t plane;  // rows * pitch
    __host__ __device__ __forceinline__ size_t at(int i, int j) const { return at_w(i, j, gy); }
    // the same for a layout whose ghost width G is known at compile time (G == gy)
    template <int G>
    __host__ __device__ __forceinline__ size_t at_g(int i, int j) const {
        return at_w(i, j, G);
    }
    __host__ __device__ __forceinline__ size_t at_w(int i, int j, int g) const {
#if TRTR_BOUNDS_CHECK && defined(__CUDA_ARCH__)
        if (g != gy || i < -g || i >= nx + g || j < -g || j >= ny + g) {  // outside the interior and its ghost frame
            TRTR_BOUNDS_FAULT(kBoundsPlane, i, j);
            g = gy;
            i = i < -g ? -g : (i >= nx + g ? nx + g - 1 : i);
            j = j < -g ? -g : (j >= ny + g ? ny + g - 1 : j);
        }
#endif
        return (size_t)(j + g) * (size_t)pitch + (size_t)(i + gx);
    }
};

PlaneLayout make_layout(int nx, int ny, int elem_bytes, int ghost);

// Storage traits: how a population is kept in memory and turned into the compute type.
template <typename S>
struct Store;

template <>
struct Store<double> {
    using C = double;
    static __device__ __forceinline__ double decode(double v, double) { return v; }
    static __device__ __forceinline__ double encode(double v, double) { return v; }
};

template <>
struct Store<float> {
    using C = float;
    static __device__ __forceinline__ float decode(float v, float) { return v; }
    static __device__ __forceinline__ float encode(float v, float) { return v; }
};

// Half-precision offset storage: h = g - w_i phi_ref.
template <>
struct Store<__half> {
    using C = float;
    static __device__ __forceinline__ float decode(__half v, float off) { return __half2float(v) + off; }
    static __device__ __forceinline__ __half encode(float v, float off) { return __float2half_rn(v - off); }
};

template <>
struct Store<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float decode(__nv_bfloat16 v, float off) { return __bfloat162float(v) + off; }
    static __device__ __forceinline__ __nv_bfloat16 encode(float v, float off) { return __float2bfloat16_rn(v - off); }
};

// Time-dependent uniforms of the pulse source (centre, 1/s^2, amplitude term at t_n and
// t_{n-1}); pulse_time_fields fills them.
template <typename C>
struct alignas(16) TimeFields {
    C cx_n, cy_n, inv_s2_n, a_n;     // at t_n
    C cx_p, cy_p, inv_s2_p, a_p;     // at t_{n-1} (t = -dt at the first step: the closed form)
};

// The uniforms of step n (t_n = n dt, t_{n-1} = t_n - dt), computed in double.  The amplitude
// term: FP64 kernels a = s0^2 / s^2; FP32-computing kernels a_n = log2(1.5 dt s0^2 / s_n^4) and
// a_p = log2(0.5 dt s0^2 / s_p^4), the step's weights of S^n and S^{n-1} in
// dt S^n + dt/2 (S^n - S^{n-1}) and the 1/s^2 of S folded into the exponent (pulse_source_dt).
template <typename C>
__host__ __device__ inline TimeFields<C> pulse_time_fields(const Pulse& p, double dt, long long n) {
    TimeFields<C> u;
    const double tn = (double)n * dt, tp = (double)(n - 1) * dt;
    const double cn = cos(p.omega * tn), sn = sin(p.omega * tn);
    const double cp = cos(p.omega * tp), sp = sin(p.omega * tp);
    const double s2n = p.sigma0 * p.sigma0 + 2.0 * p.D0 * tn, s2p = p.sigma0 * p.sigma0 + 2.0 * p.D0 * tp;
    u.cx_n = (C)(p.xc * cn - p.yc * sn);
    u.cy_n = (C)(p.xc * sn + p.yc * cn);
    u.inv_s2_n = (C)(1.0 / s2n);
    u.cx_p = (C)(p.xc * cp - p.yc * sp);
    u.cy_p = (C)(p.xc * sp + p.yc * cp);
    u.inv_s2_p = (C)(1.0 / s2p);
    if (sizeof(C) == 8) {
        u.a_n = (C)(p.sigma0 * p.sigma0 / s2n);
        u.a_p = (C)(p.sigma0 * p.sigma0 / s2p);
    } else {
        u.a_n = (C)log2(1.5 * dt * p.sigma0 * p.sigma0 / (s2n * s2n));
        u.a_p = (C)log2(0.5 * dt * p.sigma0 * p.sigma0 / (s2p * s2p));
    }
    return u;
}

// Tile schedule bits of a step launch.  kSchedDynamic: the CTAs take their tiles from tile_ctr
// (long launches; kDynMinTilesPerCta).  kSchedReverse: the launch walks the tile order from the
// last tile to the first.  Consecutive launches on a context alternate the direction, so each
// starts on the tiles that the launch before it wrote last, whose lines are still in L2.
constexpr int kSchedDynamic = 1, kSchedReverse = 2;

// Uniform arguments of the fused step kernel (one launch per time step).  The static part
// precedes tf and is a whole number of 16-byte chunks, so the batched kernel can copy the
// two parts into shared memory with asynchronous 16-byte copies.
template <typename C>
struct alignas(16) StepArgs {
    void* dst;              // P written by this step (plain stores, with ghosts)
    const C* tab_x;         // [2][nx]: sin(pi x_i), cos(pi x_i)
    const C* tab_y;         // [2][ny]: sin(pi y_j), cos(pi y_j)
    int* flag;              // set when a bounded wait gives up
    unsigned* tile_ctr;     // [next tile, CTAs done] of kernels that hand out tiles dynamically (zero between launches)
    PlaneLayout lp;         // populations
    PlaneLayout lf;         // fields
    int s_cur, s_prev;      // source buffer indices (TRTR_SRC_FIELD)
    int tau2_fixed;
    C magic;                // Lambda
    C omega2_fixed;         // 1 / tau2 (TRTR_TAU2_FIXED)
    C phi_ref;
    // pulse source (TRTR_SRC_PULSE), physical units
    C x0, y0, dx, dt;
    C dD_amp;               // D0 * D_amp
    uint32_t rkey;          // stochastic rounding of the 2-byte storages: the step's key (sr_step_key)
    int sched;              // kSchedDynamic | kSchedReverse (below)
    TimeFields<C> tf;       // pulse source uniforms of this step (a separate 16-byte block)
};

// Random bits of the stochastic rounding (TRTR_ROUND_STOCHASTIC): Wellons' "lowbias32"
// integer hash (two multiply / xor-shift rounds, published with its measured avalanche bias).
// The step's key hashes the step number; a node pair's key hashes its first node's index with
// the step key, and population q of the pair takes that key rotated by 7 q bits.  The bits
// depend on nothing but (node, step, q), so a run is the same however its steps are launched.
__host__ __device__ __forceinline__ uint32_t sr_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
__host__ __device__ __forceinline__ uint32_t sr_step_key(long step) {
    return sr_hash((uint32_t)step * 0x9E3779B9U + (uint32_t)((unsigned long long)step >> 32) + 0x632BE5ABU);
}

// Programmatic dependent launch of the step kernels: only for launches of a few tiles per CTA,
// where the launch latency it hides is a large part of the step.  On long launches it costs time
// (measured on GB300 without events between the launches: the two-step kernel at 4096^2 0.360
// against 0.346 ms, at 8192^2 1.97 against 1.41 ms; the one-step FP16 kernel at 8192^2 0.634
// against 0.612 ms), and a launch that records an event after it does not overlap anyway.
constexpr long kPdlMaxTilesPerCta = 8;
// Tiles handed out from a counter: only for launches of more than this many tiles per CTA.  On
// short launches the CTAs' few sequential atomic round trips cost more than the balancing gains
// (the 512^2 adjoint's forward steps: 11 -> 18 us per two-step launch).
constexpr long kDynMinTilesPerCta = 8;

enum MapId { kMapPop0 = 0, kMapPop1 = 1, kMapU = 2, kMapD = 3, kMapS = 4, kNumMaps = 5 };

}  // namespace trtr

struct trtr_adjoint_state;  // checkpoints and adjoint buffers (trtr_adjoint.cu)

struct trtr_ctx {
    CUtensorMap maps[trtr::kNumMaps];  // TMA descriptors (64-byte aligned type)
    trtr_params p;
    cudaStream_t stream;
    int device;
    int num_sms;
    int esize;        // bytes per stored population
    int csize;        // bytes per compute value (fields)
    trtr::PlaneLayout lp;  // population planes
    trtr::PlaneLayout lf;  // field planes
    void* pop[2];
    int cur;          // index of the buffer holding P for the current step
    void* uv;         // [2][rows][pitch] uhat_x, uhat_y
    void* Dh;
    void* S;          // [2][rows][pitch] (TRTR_SRC_FIELD)
    int S_cur;        // buffer holding S^n (-1: none set)
    int S_prev;       // buffer holding S^{n-1} (-1: use S^n)
    void* tab_x;
    void* tab_y;
    double* scratch;  // reduction partials
    int red_blocks;
    double* dres;     // device result of the reductions (4 doubles)
    double* hres;     // pinned host copy
    int* dflag;       // device timeout flag; dflag[2], dflag[3]: tile counters of the step kernels
    double* dtmp;     // device staging for double I/O
    size_t dtmp_len;  // in doubles
    double* phib;     // Dirichlet values of the edge nodes (TRTR_BC_DIRICHLET_NEE)
    bool fields_set, pulse_set, initialized, maps_ready, dirichlet_set;
    bool small_tiles;  // step kernel geometry for small grids (chosen by encode_maps)
    // two-step kernel (FP32 storage, periodic boundaries, no source or the pulse source)
    CUtensorMap maps2[3];   // populations (buffers 0, 1) and packed fields, its tile boxes
    void* fld2;             // [5][rows][pitch] float: uhat_x, uhat_y, a_x, a_y, Dh, two-wide periodic ghosts
    trtr::PlaneLayout lt;   // layout of fld2
    bool fld2_ready;        // fld2 holds the current fields
    bool ghost2_ready;      // the current population buffer's whole two-wide ghost frame is up to date
    int steps_per_launch;   // 2: trtr_step uses the two-step kernel where it applies; 1: never
    trtr::Pulse pulse;
    long step;
    long launches;
    unsigned sweeps;        // step launches so far: the parity sets their tile direction (kSchedReverse)
    trtr_adjoint_state* adj;  // recorded forward run (trtr_forward_record), or NULL
    char err[512];
};

namespace trtr {

// Launchers (defined in trtr_step.cu and trtr_aux.cu).  All enqueue on ctx->stream and
// return the cudaGetLastError() of the launch.
cudaError_t encode_maps(trtr_ctx* ctx);
cudaError_t launch_step(trtr_ctx* ctx);
// one step from an arbitrary population buffer (its map from encode_pop_map) into dst, as step `step`
cudaError_t launch_step_from(trtr_ctx* ctx, const CUtensorMap* src_map, void* dst, long step);
cudaError_t encode_pop_map(trtr_ctx* ctx, void* buffer, CUtensorMap* out);
// The two-step kernel: whether it applies to the context, its maps (at creation), the packed
// fields (after each change of u or D), and one launch advancing the state by two steps.
bool two_step_applies(const trtr_ctx* ctx);
cudaError_t encode_maps2(trtr_ctx* ctx);
cudaError_t launch_pack_fields2(trtr_ctx* ctx);
cudaError_t launch_step2(trtr_ctx* ctx);
// the distance-2 ghost cells of the current population buffer (or of buffer P) from its
// interior (periodic)
cudaError_t launch_refresh_ghosts2(trtr_ctx* ctx);
cudaError_t launch_refresh_ghosts2_buffer(trtr_ctx* ctx, void* P);
// the two-step kernel from an arbitrary population buffer (its map from encode_pop_map2) into
// dst, as steps `step` and `step + 1`; dst1 (or null) receives the intermediate state
cudaError_t encode_pop_map2(trtr_ctx* ctx, void* buffer, CUtensorMap* out);
cudaError_t launch_step2_from(trtr_ctx* ctx, const CUtensorMap* src_map, void* dst, void* dst1, long step);
// one block whose bounded wait on a barrier that nothing completes gives up after `cycles`
cudaError_t launch_wait_timeout(trtr_ctx* ctx, long long cycles);
// one thread that gives the bounds checks four bad arguments and accesses nothing with them
cudaError_t launch_bounds_probe(trtr_ctx* ctx);
void free_adjoint(trtr_ctx* ctx);
cudaError_t launch_convert_fields(trtr_ctx* ctx, const double* ux, const double* uy, const double* D);
cudaError_t launch_pulse_fields(trtr_ctx* ctx);
cudaError_t launch_convert_source(trtr_ctx* ctx, const double* S, int buffer);
cudaError_t launch_init_equilibrium(trtr_ctx* ctx, const double* phi0 /* device or NULL = pulse */);
cudaError_t launch_moments(trtr_ctx* ctx, double* phi_out_dev);
cudaError_t launch_reduce(trtr_ctx* ctx, int kind, const double* phi_ref_dev);
cudaError_t launch_get_populations(trtr_ctx* ctx, double* g_dev);
cudaError_t launch_set_populations(trtr_ctx* ctx, const double* g_dev);
cudaError_t launch_sample(trtr_ctx* ctx, const long* nodes_dev, int count, double* out_dev);
// TRTR_BC_DIRICHLET_NEE: edge values from a device [ny][nx] array, and the boundary pass over
// the population buffer P that a step has just written
cudaError_t launch_gather_edges(trtr_ctx* ctx, const double* phi_b_dev);
cudaError_t launch_dirichlet(trtr_ctx* ctx, void* P);

// kReduceBadField: the number of values of the device array `ref` (one per node) that are not
// finite and positive (the check of a device-resident D).
enum ReduceKind { kReduceMass = 0, kReducePulse = 1, kReduceField = 2, kReduceNonFinite = 3, kReduceBadField = 4 };

PulseTime pulse_at(const Pulse& p, double t);

// Edge nodes of an nx x ny grid (nx, ny >= 3), k in [0, 2 nx + 2 (ny - 2)): the bottom row,
// the top row, then the left and right columns without their corners.
__host__ __device__ inline int edge_count(int nx, int ny) { return 2 * nx + 2 * (ny - 2); }
__host__ __device__ inline void edge_node(int k, int nx, int ny, int* i, int* j) {
    if (k < nx) { *i = k; *j = 0; }
    else if (k < 2 * nx) { *i = k - nx; *j = ny - 1; }
    else if (k < 2 * nx + ny - 2) { *i = 0; *j = 1 + (k - 2 * nx); }
    else { *i = nx - 1; *j = 1 + (k - 2 * nx - (ny - 2)); }
}

// D2Q9 in the library's order: 0:(0,0) 1:(1,0) 2:(-1,0) 3:(0,1) 4:(0,-1) 5:(1,1) 6:(-1,-1)
// 7:(1,-1) 8:(-1,1).
__host__ __device__ constexpr int lattice_ex(int q) { return q == 1 || q == 5 || q == 7 ? 1 : (q == 2 || q == 6 || q == 8 ? -1 : 0); }
__host__ __device__ constexpr int lattice_ey(int q) { return q == 3 || q == 5 || q == 8 ? 1 : (q == 4 || q == 6 || q == 7 ? -1 : 0); }

// Stores one population value at every ghost cell that repeats interior node (i, j): the
// periodic images within W of the edges (W = 0: the layout's whole frame, L.gy wide), placed
// by a layout whose ghost width is GY (GY = 0: L.gy, read at run time; the step kernels know
// it at compile time).  The one-step kernels write the W = 1 frame that they read; the
// two-step kernel writes and reads the whole W = 2 frame (refresh_ghosts2 completes a frame
// left by one-step launches).
template <int W = 0, int GY = 0, typename T>
__device__ __forceinline__ void store_ghosts(T* plane, const PlaneLayout& L, int i, int j, T v) {
    const int w = W > 0 ? W : L.gy, g = GY > 0 ? GY : L.gy;
    const bool xl = i < w, xr = i >= L.nx - w, yl = j < w, yr = j >= L.ny - w;
    if (!(xl || xr || yl || yr)) return;
    if (xl) plane[L.at_w(i + L.nx, j, g)] = v;
    if (xr) plane[L.at_w(i - L.nx, j, g)] = v;
    if (yl) plane[L.at_w(i, j + L.ny, g)] = v;
    if (yr) plane[L.at_w(i, j - L.ny, g)] = v;
    if (xl && yl) plane[L.at_w(i + L.nx, j + L.ny, g)] = v;
    if (xl && yr) plane[L.at_w(i + L.nx, j - L.ny, g)] = v;
    if (xr && yl) plane[L.at_w(i - L.nx, j + L.ny, g)] = v;
    if (xr && yr) plane[L.at_w(i - L.nx, j - L.ny, g)] = v;
}

// Stores one population value at interior node (i, j) and at its ghost cells.
template <int W = 0, int GY = 0, typename T>
__device__ __forceinline__ void store_with_ghosts(T* plane, const PlaneLayout& L, int i, int j, T v) {
    plane[L.at_w(i, j, GY > 0 ? GY : L.gy)] = v;
    store_ghosts<W, GY>(plane, L, i, j, v);
}

}  // namespace trtr
