// trtr_step2_core.cuh -- the tile of the two-step kernel (two time steps of Eq. (14) per
// launch), shared by the single-grid kernel (trtr_step2.cu) and the batched one
// (trtr_batch.cu): the tile geometry, its TMA boxes, and the two steps over a staged tile.
// Not part of the public ABI.
#pragma once

#include "trtr_step_core.cuh"

namespace trtr {
namespace core {

constexpr int kT2NF = 5;  // packed fields: uhat_x, uhat_y, a_x, a_y, Dh

// Stage of one BX x BY output tile: the population box (9 planes of ES-byte values) and the
// field box (5 planes of floats).  Both boxes start on a 16-byte column boundary left of the
// two-node halo: HX = 16 / ES population columns, 4 field columns.
template <int BX, int BY, int ES = 4>
struct Tile2 {
    static constexpr int X = BX, Y = BY;
    static constexpr int HX = 16 / ES;                   // staged population columns [i0 - HX, i0 + BX + HX)
    static constexpr int W = BX + 2 * HX;
    static constexpr int WF = BX + 8;                    // staged field columns [i0 - 4, i0 + BX + 4)
    static constexpr int PR = BY + 4;                    // staged population rows
    static constexpr int FR = BY + 2;                    // staged field rows
    static constexpr int R1 = (BY + 2) * (BX + 4) / 2;  // node pairs of step 1
    static constexpr int R2 = BY * BX / 2;               // node pairs of step 2
    static constexpr int PopPlane = PR * W;              // values
    static constexpr int FldPlane = FR * WF;             // floats
    static constexpr int PopBytes = kQ * PopPlane * ES;
    static constexpr int FldOff = (PopBytes + 127) / 128 * 128;  // the field box, 128-byte aligned
    static constexpr int FldBytes = kT2NF * FldPlane * 4;
    static constexpr int TX = PopBytes + FldBytes;       // bytes per tile (boxes include any fill)
    static constexpr int Stage = (FldOff + FldBytes + 127) / 128 * 128;
    static_assert(ES == 4 || ES == 2, "FP32 or 2-byte populations");
    static_assert((BX * ES) % 16 == 0 && BX % 4 == 0, "tile origins on 16-byte boundaries");
    static_assert(W <= 256 && WF <= 256 && PR <= 256, "TMA box dimensions are at most 256");
};

template <int STAGES, int CTAS, int THREADS, int BX, int BY, int ES = 4>
struct Geom2 {
    static constexpr int kStages = STAGES, kCtas = CTAS, kThreads = THREADS;
    using T = Tile2<BX, BY, ES>;
    static_assert(STAGES * T::Stage + 256 <= 227 * 1024, "the stages must fit in shared memory");
};
// Geometry per source mode and population size (stages, CTAs per SM, threads, tile width, tile
// height), from the sweeps of rebuilds with -DTRTR_STEP2_STAGES=S -DTRTR_STEP2_CTAS=C
// -DTRTR_STEP2_THREADS=T -DTRTR_STEP2_BX=X -DTRTR_STEP2_BY=Y (all five; they set it for both
// modes of the FP32 kernel; TRTR_STEP2H_* the same for the 2-byte one): a few independent CTAs
// per SM hide each one's barrier between the two steps, the pulse source's arithmetic favours
// more of them.
// FP32: 32 x 8 tiles in three 128-thread CTAs (GB300, GLUPS at 4096^2 / 8192^2 with the pulse:
// 114.1 / 121.8; without a source 131.6 / 141.0, against 123.2 / 131.4 for 32 x 16 tiles in two
// 256-thread CTAs); wider or taller tiles leave fewer CTAs or one stage (64 x 8 in two
// 256-thread CTAs 108.6 / 115.5, 64 x 16 in one 512-thread CTA 100.2 / 106.6, 60 x 6 104.1 /
// 111.7), and 28-column tiles, whose step-1 pairs fill the block evenly, measured slower
// (28 x 14: 102.2 / 108.7).
template <int SRC, int ES>
struct Geom2For {
    using type = Geom2<2, 3, 128, 32, 8, ES>;
};
// 2-byte storages: half the stage bytes, so wider tiles with less step-1 halo work fit two CTAs
// per SM.  Measured (GB300, FP16 pulse, GLUPS at 4096^2 / 8192^2): 32 x 8 in 3 (4) 128-thread
// CTAs 111.0 / 117.2 (112.2 / 118.4), 64 x 8 in 3 128-thread CTAs 114.9 / 123.5, 64 x 12 in 2
// 256-thread CTAs 115.8 / 125.1, 64 x 16 in 2 256-thread CTAs 120.3 / 131.5, 64 x 32 or 128 x 16
// in one 512-thread CTA 114.5 / 126.5 and 111.4 / 124.5.
template <int SRC>
struct Geom2For<SRC, 2> {
    using type = Geom2<2, 2, 256, 64, 16, 2>;
};
#if defined(TRTR_STEP2_BX) || defined(TRTR_STEP2H_BX)
template <int SRC, int ES>
struct Geom2Sweep {
    using type = typename Geom2For<SRC, ES>::type;
};
#endif
#ifdef TRTR_STEP2_BX
template <int SRC>
struct Geom2Sweep<SRC, 4> {
    using type = Geom2<TRTR_STEP2_STAGES, TRTR_STEP2_CTAS, TRTR_STEP2_THREADS, TRTR_STEP2_BX, TRTR_STEP2_BY, 4>;
};
#endif
#ifdef TRTR_STEP2H_BX
template <int SRC>
struct Geom2Sweep<SRC, 2> {
    using type = Geom2<TRTR_STEP2H_STAGES, TRTR_STEP2H_CTAS, TRTR_STEP2H_THREADS, TRTR_STEP2H_BX, TRTR_STEP2H_BY, 2>;
};
#endif
#if defined(TRTR_STEP2_BX) || defined(TRTR_STEP2H_BX)
template <int SRC, int ES = 4>
using Geom2Of = typename Geom2Sweep<SRC, ES>::type;
#else
template <int SRC, int ES = 4>
using Geom2Of = typename Geom2For<SRC, ES>::type;
#endif

struct alignas(16) Step2Args {
    StepArgs<float> a;  // tf, rkey: the pulse uniforms and rounding key of the first step
    TimeFields<float> tf2;  // of the second step
    void* dst1;             // if not null: also store the first step's state here (one-wide ghosts)
    uint32_t rkey2;         // the second step's rounding key (stochastic rounding of 2-byte storages)
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
    return pulse_source_dt(x, y, tf, dD, dDx, dDy);
}

// The TMA loads of one tile into `stage` (its barrier armed by the caller): the population box of
// depth 9 from column i0 - HX (gxp: the population layout's column of x = 0) and row j0 - 2, and
// the packed-field box of depth 5 from column i0 - 4 (gxf: the field layout's) and row j0 - 1;
// both x origins are 16-byte aligned.
// TRTR_STEP2_L2HINT = 1 (the default): the tile loads ask L2 to keep their lines (the
// neighbouring tiles read the halo again) and the result stores to evict theirs first; measured
// on the 4096^2 pulse: DRAM reads -2.3 %, launch -0.7 %.
#ifndef TRTR_STEP2_L2HINT
#define TRTR_STEP2_L2HINT 1
#endif
template <class T>
__device__ __forceinline__ void step2_issue(unsigned char* stage, uint64_t* bar, const CUtensorMap* mp,
                                            const CUtensorMap* mf, int i0, int j0, int gxp, int gxf) {
    constexpr int kES = 16 / T::HX;
    const int xp = i0 + gxp - T::HX, xf = i0 + gxf - 4;
#if TRTR_STEP2_L2HINT
    const uint64_t keep = l2_evict_last();
    if (tma_ok(stage, xp, j0 + kGhostP - 2, kES)) tma_load_3d_hint(stage, mp, bar, xp, j0 + kGhostP - 2, 0, keep);
    if (tma_ok(stage + T::FldOff, xf, j0 + kGhostP - 1, 4))
        tma_load_3d_hint(stage + T::FldOff, mf, bar, xf, j0 + kGhostP - 1, 0, keep);
#else
    if (tma_ok(stage, xp, j0 + kGhostP - 2, kES)) tma_load_3d(stage, mp, bar, xp, j0 + kGhostP - 2, 0);
    if (tma_ok(stage + T::FldOff, xf, j0 + kGhostP - 1, 4))
        tma_load_3d(stage + T::FldOff, mf, bar, xf, j0 + kGhostP - 1, 0);
#endif
}

// A node pair of a staged population plane (S values; aligned: the pair starts on an even
// column), read as offsets or written from a stored pair.
template <typename S>
__device__ __forceinline__ F2 stage_ld2(const S* v, bool aligned) {
    using P = Pair<S>;
    return aligned ? P::raw(*reinterpret_cast<const typename P::type*>(v)) : P::raw(v[0], v[1]);
}
template <typename S, typename S2>
__device__ __forceinline__ void stage_st2(S* d, S2 v, bool aligned) {
    if (aligned) {
        *reinterpret_cast<S2*>(d) = v;
    } else {
        d[0] = reinterpret_cast<const S*>(&v)[0];
        d[1] = reinterpret_cast<const S*>(&v)[1];
    }
}

// The stored form of population q of a node pair: FP32 as it is; 2-byte offsets rounded to
// nearest, or stochastically (SR) with the bits of the pair's key rk, as the one-step kernel
// stores them.
template <typename S, bool SR>
__device__ __forceinline__ typename Pair<S>::type encode2(F2 v, uint32_t rk, int q) {
    if constexpr (SR)
        return Pair<S>::encode_sr(v, sr_bits(rk, q));
    else
        return Pair<S>::encode_raw(v);
}

// Step 1 over the tile's halo region R1, in place in the stage (thread tid of NT).  2-byte
// storages: the step-1 values are rounded to the storage format with the first step's key rkey1, as
// a one-step launch stores them (halo nodes with the key of the wrapped node; nx is even, so
// the wrapped pairs are the one-step kernel's pairs).
template <typename S, int SRC, class T, int NT, bool SR = false>
__device__ __forceinline__ void step2_first(S* sp, const float* sf, int i0, int j0, const StepArgs<float>& a,
                                            const TimeFields<float>& tf, int tid, uint32_t rkey1 = 0u) {
    constexpr int kT2W = T::W, kT2WF = T::WF, kT2PopPlane = T::PopPlane, kT2FldPlane = T::FldPlane;
    constexpr bool kOfs = sizeof(S) == 2;  // offsets folded into the moments, as in the one-step kernel
    constexpr int kC = T::HX - 2;          // stage column of R1 column 0
    // Node pairs (c, c + 1) of a halo row.  R1SHIFT = 1: c odd, the columns 1 .. X + 2 that step
    // 2 reads (the planes with e_x != 0 then sit on even offsets); 0: c even from 0, including
    // the two outermost columns (the planes with e_x = 0 and the fields on even offsets).
#ifndef TRTR_STEP2_R1SHIFT
#define TRTR_STEP2_R1SHIFT 0
#endif
    constexpr int kShift = TRTR_STEP2_R1SHIFT;
    static_assert(!kOfs || kShift == 0, "2-byte storages round the one-step kernel's pairs");
    constexpr int kRowPairs = (T::X + 4 - 2 * kShift) / 2;
    constexpr int kPairs = (T::Y + 2) * kRowPairs;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const F2 magic(a.magic), w2f(a.omega2_fixed);
    auto ld2 = [](const float* v, bool aligned) {
        return aligned ? F2(*reinterpret_cast<const float2*>(v)) : F2(v[0], v[1]);
    };
    for (int p = tid; p < kPairs; p += NT) {
        const int r = p / kRowPairs, c = 2 * (p - r * kRowPairs) + kShift;
        F2 g[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const S* src = sp + q * kT2PopPlane + (r + 1 - lattice_ey(q)) * kT2W + c + kC - lattice_ex(q);
            g[q] = stage_ld2(src, (lattice_ex(q) != 0) == (kShift == 1));
        }
        const float* f = sf + r * kT2WF + c + 2;
        const bool fa = kShift == 0;
        const F2 ux = ld2(f, fa);
        const F2 uy = ld2(f + kT2FldPlane, fa);
        const F2 ax = ld2(f + 2 * kT2FldPlane, fa);
        const F2 ay = ld2(f + 3 * kT2FldPlane, fa);
        const F2 Dh = ld2(f + 4 * kT2FldPlane, fa);
        const int x = i0 - 2 + c, y = j0 - 1 + r;
        const int wx = wrap_clamp(x, nx), wy = wrap_clamp(y, ny);
        const F2 src = pair_source<SRC>(a, tf, wx, wrap_clamp(x + 1, nx), wy);
        F2 out[kQ];
        collide_node<F2, kOfs>(g, ux, uy, ax, ay, Dh, src, magic, w2f, a.tau2_fixed, out, F2(a.phi_ref));
        const uint32_t rk = SR ? sr_pair_key(wx, wy, nx, rkey1) : 0u;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            S* d = sp + q * kT2PopPlane + (r + 1 - lattice_ey(q)) * kT2W + c + kC - lattice_ex(q);
            stage_st2(d, encode2<S, SR>(out[q], rk, q), (lattice_ex(q) != 0) == (kShift == 1));
        }
    }
}

// Step 2 on the tile's output nodes from the step-1 values in the stage, stored to a.dst with
// the ghost copies of nodes within two of an edge.  P1: the step-1 state of the output nodes is
// stored to dst1 too, with the one-wide ghost frame that one-step kernels read.
template <typename S, int SRC, class T, int NT, bool P1 = false, bool SR = false>
__device__ __forceinline__ void step2_second(const S* sp, const float* sf, int i0, int j0,
                                             const StepArgs<float>& a, const TimeFields<float>& tf2, int tid,
                                             S* dst1 = nullptr, uint32_t rkey2 = 0u) {
    constexpr int kT2X = T::X, kT2W = T::W, kT2WF = T::WF, kT2R2 = T::R2, kT2PopPlane = T::PopPlane,
                  kT2FldPlane = T::FldPlane;
    constexpr bool kOfs = sizeof(S) == 2;
    using S2 = typename Pair<S>::type;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const F2 magic(a.magic), w2f(a.omega2_fixed);
    S* dst = static_cast<S*>(a.dst);
    const size_t pl = a.lp.plane;
    for (int p = tid; p < kT2R2; p += NT) {
        const int r2 = p / (kT2X / 2), c2 = 2 * (p - r2 * (kT2X / 2));
        const int i = i0 + c2, j = j0 + r2;
        if (i >= nx || j >= ny) continue;
        if constexpr (P1) {  // the step-1 value of node (r2, c2) = R1 node (r2 + 1, c2 + 2), plane by plane
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const S* v = sp + q * kT2PopPlane + (r2 + 2 - lattice_ey(q)) * kT2W + c2 + T::HX - lattice_ex(q);
                store_with_ghosts<1, kGhostP>(dst1 + q * pl, a.lp, i, j, v[0]);
                if (i + 1 < nx) store_with_ghosts<1, kGhostP>(dst1 + q * pl, a.lp, i + 1, j, v[1]);
            }
        }
        F2 g[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            g[q] = stage_ld2(sp + q * kT2PopPlane + (r2 + 2 - 2 * lattice_ey(q)) * kT2W + c2 + T::HX - 2 * lattice_ex(q),
                             true);
        const float* f = sf + (r2 + 1) * kT2WF + c2 + 4;
        const F2 ux(*reinterpret_cast<const float2*>(f));
        const F2 uy(*reinterpret_cast<const float2*>(f + kT2FldPlane));
        const F2 ax(*reinterpret_cast<const float2*>(f + 2 * kT2FldPlane));
        const F2 ay(*reinterpret_cast<const float2*>(f + 3 * kT2FldPlane));
        const F2 Dh(*reinterpret_cast<const float2*>(f + 4 * kT2FldPlane));
        const F2 src = pair_source<SRC>(a, tf2, i, i + 1 < nx ? i + 1 : nx - 1, j);
        F2 out[kQ];
        collide_node<F2, kOfs>(g, ux, uy, ax, ay, Dh, src, magic, w2f, a.tau2_fixed, out, F2(a.phi_ref));
        const uint32_t rk = SR ? sr_pair_key(i, j, nx, rkey2) : 0u;
        const bool edge = j < kGhostP || j >= ny - kGhostP || i < kGhostP || i + 1 >= nx - kGhostP;
        if (!edge) {
            S* d0 = dst + a.lp.at_g<kGhostP>(i, j);
#if TRTR_BOUNDS_CHECK
            if ((reinterpret_cast<uintptr_t>(d0) % sizeof(S2)) != 0u) {
                TRTR_BOUNDS_FAULT(kBoundsPair, i, j);
                continue;
            }
#endif
#if TRTR_STEP2_L2HINT
            const uint64_t leave = l2_evict_first();
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                if constexpr (sizeof(S) == 4)
                    st_global_f2_hint(reinterpret_cast<float*>(d0 + q * pl), out[q].v, leave);
                else
                    st_global_b32_hint(reinterpret_cast<S2*>(d0 + q * pl), encode2<S, SR>(out[q], rk, q), leave);
            }
#else
#pragma unroll
            for (int q = 0; q < kQ; ++q) *reinterpret_cast<S2*>(d0 + q * pl) = encode2<S, SR>(out[q], rk, q);
#endif
        } else {
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const S2 v = encode2<S, SR>(out[q], rk, q);
                store_with_ghosts<kGhostP, kGhostP>(dst + q * pl, a.lp, i, j, reinterpret_cast<const S*>(&v)[0]);
                if (i + 1 < nx)
                    store_with_ghosts<kGhostP, kGhostP>(dst + q * pl, a.lp, i + 1, j, reinterpret_cast<const S*>(&v)[1]);
            }
        }
    }
}

}  // namespace core
}  // namespace trtr
