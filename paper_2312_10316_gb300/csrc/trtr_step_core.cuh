// trtr_step_core.cuh -- device machinery of the fused TRT-R step shared by the single-grid
// kernel (trtr_step.cu) and the batched kernel (trtr_batch.cu): TMA / mbarrier helpers,
// packed FP32 pair arithmetic, the moment-space node update of Eq. (14), and the routines
// that compute one tile row from a shared-memory stage.  Tile geometry is BX x BY nodes
// (one warp per tile row).  Internal to the library.
#pragma once

#include <cudaTypedefs.h>

#include <string.h>

#include <type_traits>

#include "trtr_internal.cuh"

namespace trtr {
namespace core {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

template <typename S, int SRC, int BX, int BY>
struct Tile {
    using C = typename Store<S>::C;
    static constexpr int A = 16 / (int)sizeof(S);    // TMA x quantum of the populations
    static constexpr int PW = BX + A;                // population tile width
    static constexpr int AC = 16 / (int)sizeof(C);   // TMA x quantum of the fields
    static constexpr int UW = BX + 2 * AC;           // u tile width (halo rounded to AC)
    static constexpr int UH = BY + 2;
    static constexpr uint32_t pad128(uint32_t b) { return (b + 127) / 128 * 128; }
    // shared-memory tiles start on 128-byte boundaries (TMA destinations)
    static constexpr uint32_t POP_PLANE = pad128(BY * PW * sizeof(S));
    static constexpr int PLANE_ELEMS = POP_PLANE / sizeof(S);
    static constexpr uint32_t POP = kQ * POP_PLANE;
    static constexpr uint32_t U = pad128(2 * UH * UW * sizeof(C));
    static constexpr uint32_t D = pad128(BY * BX * sizeof(C));
    static constexpr uint32_t S_TILE = pad128(BY * BX * sizeof(C));
    static constexpr uint32_t SRCB = SRC == TRTR_SRC_FIELD ? 2 * S_TILE : 0;
    // bytes the TMA delivers per stage (the boxes, without the padding)
    static constexpr uint32_t TX = kQ * BY * PW * sizeof(S) + 2 * UH * UW * sizeof(C) + BY * BX * sizeof(C) +
                                   (SRC == TRTR_SRC_FIELD ? 2 * BY * BX * sizeof(C) : 0);
    static constexpr uint32_t STAGE = POP + U + D + SRCB;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase `parity` of `bar` to complete, for at most `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kWaitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
        "%5}], [%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// L2 eviction priorities (createpolicy): loads whose tiles neighbouring CTAs read again (the
// halo) can ask to stay, stores that nothing in the launch reads again to leave first.
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
        "{%3, %4, %5}], [%2], %6;" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void st_global_f2_hint(float* p, float2 v, uint64_t policy) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(policy)
                 : "memory");
}
// the same for a pair of 2-byte values (one 32-bit word)
template <typename S2>
__device__ __forceinline__ void st_global_b32_hint(S2* p, S2 v, uint64_t policy) {
    static_assert(sizeof(S2) == 4, "a 32-bit pair");
    uint32_t w;
    memcpy(&w, &v, sizeof(w));
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(w), "l"(policy) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16) from shared to global memory, both addresses 16-byte
// aligned; the async proxy reads the source, completion is tracked per thread in bulk
// async-groups.
__device__ __forceinline__ void bulk_store(void* gdst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's bulk stores have been read (may be overwritten)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the async proxy (bulk stores)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Checked builds (TRTR_BOUNDS_CHECK): a tiled TMA load's x coordinate times the element size is
// a multiple of 16 bytes and its shared-memory destination is 128-byte aligned; a load that
// breaks either is recorded and not issued (its barrier then times out, which is reported).
__device__ __forceinline__ bool tma_ok(const void* dst, int x, int y, int elem) {
#if TRTR_BOUNDS_CHECK
    if ((x * elem) % 16 != 0 || (smem_addr(dst) & 127u) != 0u) {
        TRTR_BOUNDS_FAULT(kBoundsTma, x, y);
        return false;
    }
#endif
    return true;
}

// Checked builds: a bulk copy of nb interior columns of row j from column i0 stays inside the
// interior row and has 16-byte aligned addresses and size; otherwise it is recorded and skipped.
template <typename S>
__device__ __forceinline__ bool bulk_ok(const S* gdst, const void* src, int i0, int j, int nb, const PlaneLayout& L) {
#if TRTR_BOUNDS_CHECK
    const unsigned bytes = (unsigned)nb * (unsigned)sizeof(S);
    if (i0 < 0 || i0 + nb > L.nx || j < 0 || j >= L.ny || (reinterpret_cast<uintptr_t>(gdst) & 15u) != 0u ||
        (smem_addr(src) & 15u) != 0u || (bytes & 15u) != 0u) {
        TRTR_BOUNDS_FAULT(kBoundsBulk, i0, j);
        return false;
    }
#endif
    return true;
}

// Walks the linear tile indices t, t + stride, t + 2 stride, ... of a persistent CTA as
// (t mod m, t div m) without a division per tile: one division at the start, then an add and a
// carry per step (m: tiles per row of the order's rows).
struct TileCursor {
    int a, b, da, db, m;
    __device__ __forceinline__ void init(int t, int stride, int m_) {
        m = m_;
        a = t % m;
        b = t / m;
        da = stride % m;
        db = stride / m;
    }
    __device__ __forceinline__ void next() {
        a += da;
        b += db;
        if (a >= m) {
            a -= m;
            ++b;
        }
    }
};

// ---- arithmetic types --------------------------------------------------------------------
// FP32-computing storages work on pairs of adjacent nodes with the packed FP32 instructions
// of sm_100-family SMs (two lanes of FP32 per FADD2 / FMUL2 / FFMA2); FP64 works per node.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 vdiv(F2 a, F2 b) { return F2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)); }
__device__ __forceinline__ double vdiv(double a, double b) { return a / b; }
__device__ __forceinline__ F2 vexp(F2 a) { return F2(__expf(a.v.x), __expf(a.v.y)); }
__device__ __forceinline__ double vexp(double a) { return exp(a); }

template <class V>
struct ScalarOf;
template <>
struct ScalarOf<F2> {
    using type = float;
};
template <>
struct ScalarOf<double> {
    using type = double;
};

// Manufactured pulse source at (x, y) for the time level (cx, cy, inv_s2, amp):
//   S = phi_a / s^2 [grad D . r - (D - D0)(|r|^2 / s^2 - 2)],  r = x - c(t).
template <class V>
__device__ __forceinline__ V pulse_source(V x, V y, V cx, V cy, V inv_s2, V amp, V dD, V dDx, V dDy) {
    using T = typename ScalarOf<V>::type;
    const V rx = x - cx, ry = y - cy;
    const V r2 = vfma(rx, rx, ry * ry);
    const V e = amp * vexp(r2 * (V(T(-0.5)) * inv_s2));
    const V br = vfma(dD, vfma(r2, V(T(0)) - inv_s2, V(T(2))), vfma(dDx, rx, dDy * ry));
    return (e * inv_s2) * br;
}

// 2^a (the hardware's base-2 exponential; results below the normal range flush to zero).
__device__ __forceinline__ float ex2(float a) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// One time level of the source term, w S(x, t) with the level's weight w folded into lg (see
// pulse_time_fields): by exp(z) = 2^(z log2 e),
//   w S = 2^(lg - |r|^2 log2(e) / (2 s^2)) [grad D . r + (D - D0)(2 - |r|^2 / s^2)].
__device__ __forceinline__ F2 pulse_level(F2 x, F2 y, float cx, float cy, float inv_s2, float lg, F2 dD, F2 dDx,
                                          F2 dDy) {
    const F2 rx = x - F2(cx), ry = y - F2(cy);
    const F2 r2 = vfma(rx, rx, ry * ry);
    const F2 z = vfma(r2, F2(-0.72134752044448170368f * inv_s2), F2(lg));  // -log2(e) / 2 = -0.7213...
    const F2 br = vfma(dD, vfma(r2, F2(-inv_s2), F2(2.f)), vfma(dDx, rx, dDy * ry));
    return F2(ex2(z.v.x), ex2(z.v.y)) * br;
}

// s = dt S^n + dt/2 (S^n - S^{n-1}) = 1.5 dt S^n - 0.5 dt S^{n-1} of the manufactured source
// (a7, Eqs. (3) and (14)) for the FP32-computing kernels.
__device__ __forceinline__ F2 pulse_source_dt(F2 x, F2 y, const TimeFields<float>& tf, F2 dD, F2 dDx, F2 dDy) {
    return pulse_level(x, y, tf.cx_n, tf.cy_n, tf.inv_s2_n, tf.a_n, dD, dDx, dDy) -
           pulse_level(x, y, tf.cx_p, tf.cy_p, tf.inv_s2_p, tf.a_p, dD, dDx, dDy);
}

// The node update of Eq. (14) in moment space; g: pre-collision populations, out: P_i(x).
//
// OFS: g and out are the offsets h_i = g_i - w_i phi_ref of the 2-byte storages.  The offset
// folds into the moments: sum w_i = 1 gives phi = sum h_i + phi_ref; sum w_i e_i = 0 leaves the
// first moments alone; sum w_i (e_ia e_ib - d_ab/3) = 0 leaves B_ab alone when its trace part
// uses sum h_i / 3; and the rebuild is linear in m0 with weight w_i, so rebuilding from
// sum h_i + s (in place of phi + s) gives the offsets of the results.
template <typename V, bool OFS = false>
__device__ __forceinline__ void collide_node(const V g[kQ], V ux, V uy, V ax, V ay, V Dh, V s, V magic, V w2_fixed,
                                             bool tau2_fixed, V out[kQ], V phi_ref = V(0.f)) {
    using T = typename ScalarOf<V>::type;
    // relaxation rates: tau1 - 1/2 = 3 Dh (Sec. 2.4); tau2 from Lambda (Eq. (28)) or fixed
    const V t1m = V(T(3)) * Dh;
    const V w1 = vdiv(V(T(1)), V(T(0.5)) + t1m);
    const V w2 = tau2_fixed ? w2_fixed : vdiv(t1m, vfma(V(T(0.5)), t1m, magic));
    const V k1 = V(T(1)) - w1, k2 = V(T(1)) - w2;
    const V kh = vfma(V(T(-0.5)), w1, V(T(1)));

    // a2 + a4: moments (pair sums and differences of opposite directions)
    const V p12 = g[1] + g[2], p34 = g[3] + g[4], p56 = g[5] + g[6], p78 = g[7] + g[8];
    const V d12 = g[1] - g[2], d34 = g[3] - g[4], d56 = g[5] - g[6], d78 = g[7] - g[8];
    const V pdiag = p56 + p78;
    const V phis = (g[0] + p12) + (p34 + pdiag);  // sum of the inputs (phi, or phi - phi_ref)
    V phi = phis;
    if constexpr (OFS) phi = phis + phi_ref;
    const V jx = d12 + (d56 + d78);
    const V jy = d34 + (d56 - d78);
    const V pxx = p12 + pdiag;
    const V pyy = p34 + pdiag;
    const V pxy = p56 - p78;

    // a5 + a6 + a7: post-collision Hermite coefficients
    const V phux = phi * ux, phuy = phi * uy;
    const V euxx = phux * ux, euyy = phuy * uy, euxy = phux * uy;
    const V m0 = phis + s;  // (OFS: its rebuild gives offsets)
    const V m1x = vfma(kh, vfma(phi, ax, ux * s), vfma(k1, jx - phux, phux));
    const V m1y = vfma(kh, vfma(phi, ay, uy * s), vfma(k1, jy - phuy, phuy));
    const V third = phis * V(T(1.0 / 3.0));  // pairs with the input sums pxx, pyy
    const V Axx = vfma(k2, (pxx - third) - euxx, euxx);
    const V Ayy = vfma(k2, (pyy - third) - euyy, euyy);
    const V Axy = vfma(k2, pxy - euxy, euxy);
    const V Txxy = euxx * uy, Txyy = euxy * uy;

    // rebuild from even (E) and odd (O) halves of the opposite pairs, weights folded in:
    //   f_i = w_i [m0 + 3 e.m1 + 4.5 H2:A + 13.5 (H_xxy T_xxy + H_xyy T_xyy)]
    const V Asum = Axx + Ayy;
    const V m9 = m0 * V(T(1.0 / 9.0));
    const V E1 = vfma(V(T(-1.0 / 6.0)), Ayy, vfma(V(T(1.0 / 3.0)), Axx, m9));
    const V E3 = vfma(V(T(-1.0 / 6.0)), Axx, vfma(V(T(1.0 / 3.0)), Ayy, m9));
    const V O1 = vfma(V(T(-0.5)), Txyy, m1x * V(T(1.0 / 3.0)));
    const V O3 = vfma(V(T(-0.5)), Txxy, m1y * V(T(1.0 / 3.0)));
    const V Ed = vfma(V(T(1.0 / 12.0)), Asum, m0 * V(T(1.0 / 36.0)));
    const V E5 = vfma(V(T(0.25)), Axy, Ed);
    const V E7 = vfma(V(T(-0.25)), Axy, Ed);
    const V O5 = vfma(V(T(0.25)), Txxy + Txyy, (m1x + m1y) * V(T(1.0 / 12.0)));
    const V O7 = vfma(V(T(0.25)), Txyy - Txxy, (m1x - m1y) * V(T(1.0 / 12.0)));
    out[1] = E1 + O1;
    out[2] = E1 - O1;
    out[3] = E3 + O3;
    out[4] = E3 - O3;
    out[5] = E5 + O5;
    out[6] = E5 - O5;
    out[7] = E7 + O7;
    out[8] = E7 - O7;
    if constexpr (OFS) {
        out[0] = vfma(V(T(-2.0 / 3.0)), Asum, m0 * V(T(4.0 / 9.0)));
    } else {
        // The nine rebuilt values sum to m0 (the collision keeps phi + s, Sec. 2.2); the other
        // eight are the pairs E +- O, so the rest population is m0 - 2 (E1 + E3 + E5 + E7), which
        // equals w_0 m0 - (2/3)(A_xx + A_yy).  Formed the latter way the sum drifts: the rounded
        // weights 4/9, 1/9, 1/36 add up to 1 + 7.5e-9 in FP32, which multiplied the mass by that
        // every step.  Subtracting the four terms from m0 one at a time leaves a drift of a few
        // 1e-11 per step (summing the eight stored values first: 3e-10).
        out[0] = vfma(V(T(-2)), E1, vfma(V(T(-2)), E3, vfma(V(T(-2)), E5, vfma(V(T(-2)), E7, m0))));
    }
}

template <typename C>
__device__ __forceinline__ C weight(int q) {
    return q == 0 ? C(4.0 / 9.0) : (q < 5 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}

// Columns of a tile row (of `valid` interior columns, at most 128) that one bulk copy writes: a
// whole number of 16-byte chunks.
template <typename S>
__device__ __forceinline__ int bulk_cols(int valid) {
    constexpr int kChunk = 16 / (int)sizeof(S);
    const int v = valid < 128 ? valid : 128;
    return v / kChunk * kChunk;
}

// Shared-memory column offset of plane q's tile (see the TMA origin in issue_tile).
template <int A>
__device__ __forceinline__ constexpr int plane_offset(int q) {
    return lattice_ex(q) == 1 ? A - 1 : (lattice_ex(q) == -1 ? 1 : 0);
}

// Pair (2-element) storage vectors and their conversion to / from packed FP32.
// Random bits of the stochastic rounding of node pair (i, i + 1) of row j (i even): the pair's
// key, and the 32 bits of its population q.
__device__ __forceinline__ uint32_t sr_pair_key(int i, int j, int nx, uint32_t rkey) {
    return sr_hash(((uint32_t)j * (uint32_t)nx + (uint32_t)i) ^ rkey);
}
#ifndef TRTR_SR_WORDS
#define TRTR_SR_WORDS 9
#endif
__device__ __forceinline__ uint32_t sr_bits(uint32_t rk, int q) {
    // 9 words (the key rotated by 7 q), or 3 or 1 words shared by groups of populations (sweeps)
    if (TRTR_SR_WORDS == 9) return __funnelshift_l(rk, rk, 7 * q);
    if (TRTR_SR_WORDS == 3) return q < 3 ? rk : (q < 6 ? rk * 0x85EBCA6Bu : rk * 0xC2B2AE35u);
    return rk;
}

template <typename S>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
    static __device__ __forceinline__ F2 decode(float2 v, float) { return F2(v); }
    static __device__ __forceinline__ F2 decode(float a, float b, float) { return F2(a, b); }
    static __device__ __forceinline__ float2 encode(F2 v, float) { return v.v; }
    static __device__ __forceinline__ F2 raw(float2 v) { return F2(v); }
    static __device__ __forceinline__ F2 raw(float a, float b) { return F2(a, b); }
    static __device__ __forceinline__ float2 encode_raw(F2 v) { return v.v; }
    static __device__ __forceinline__ float2 encode_sr(F2 v, uint32_t) { return v.v; }
};
template <>
struct Pair<__half> {
    using type = __half2;
    static __device__ __forceinline__ F2 decode(__half2 v, float off) {
        const float2 f = __half22float2(v);
        return F2(f.x + off, f.y + off);
    }
    static __device__ __forceinline__ F2 decode(__half a, __half b, float off) {
        return F2(__half2float(a) + off, __half2float(b) + off);
    }
    static __device__ __forceinline__ __half2 encode(F2 v, float off) {
        return __floats2half2_rn(v.v.x - off, v.v.y - off);
    }
    // the stored offsets themselves (their w_i phi_ref is folded into the moments)
    static __device__ __forceinline__ F2 raw(__half2 v) { return F2(__half22float2(v)); }
    static __device__ __forceinline__ F2 raw(__half a, __half b) { return F2(__half2float(a), __half2float(b)); }
    static __device__ __forceinline__ __half2 encode_raw(F2 v) { return __floats2half2_rn(v.v.x, v.v.y); }
    // stochastic rounding of both offsets, 32 random bits (the first node in the low half)
    static __device__ __forceinline__ __half2 encode_sr(F2 v, uint32_t rbits) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(rbits));
        __half2 h;
        memcpy(&h, &d, sizeof(h));
        return h;
    }
};
template <>
struct Pair<__nv_bfloat16> {
    using type = __nv_bfloat162;
    static __device__ __forceinline__ F2 decode(__nv_bfloat162 v, float off) {
        const float2 f = __bfloat1622float2(v);
        return F2(f.x + off, f.y + off);
    }
    static __device__ __forceinline__ F2 decode(__nv_bfloat16 a, __nv_bfloat16 b, float off) {
        return F2(__bfloat162float(a) + off, __bfloat162float(b) + off);
    }
    static __device__ __forceinline__ __nv_bfloat162 encode(F2 v, float off) {
        return __floats2bfloat162_rn(v.v.x - off, v.v.y - off);
    }
    static __device__ __forceinline__ F2 raw(__nv_bfloat162 v) { return F2(__bfloat1622float2(v)); }
    static __device__ __forceinline__ F2 raw(__nv_bfloat16 a, __nv_bfloat16 b) {
        return F2(__bfloat162float(a), __bfloat162float(b));
    }
    static __device__ __forceinline__ __nv_bfloat162 encode_raw(F2 v) { return __floats2bfloat162_rn(v.v.x, v.v.y); }
    static __device__ __forceinline__ __nv_bfloat162 encode_sr(F2 v, uint32_t rbits) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(rbits));
        __nv_bfloat162 h;
        memcpy(&h, &d, sizeof(h));
        return h;
    }
};

template <typename S, int SRC, int BX, int BY>
__device__ __forceinline__ void issue_tile(unsigned char* stage, uint64_t* bar, const CUtensorMap* mp,
                                           const CUtensorMap* mu, const CUtensorMap* md, const CUtensorMap* ms,
                                           int i0, int j0, const StepArgs<typename Store<S>::C>& a) {
    using T = Tile<S, SRC, BX, BY>;
    mbar_expect_tx(bar, T::TX);
    constexpr int kPe = (int)sizeof(S), kFe = (int)sizeof(typename Store<S>::C);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const int x = i0 + a.lp.gx - (lattice_ex(q) == 1 ? T::A : 0);
        const int y = j0 + kGhostP - lattice_ey(q);
        if (tma_ok(stage + q * T::POP_PLANE, x, y, kPe)) tma_load_3d(stage + q * T::POP_PLANE, mp, bar, x, y, q);
    }
    const int yf = j0 + kGhostF;  // field row of the tile's first row
    if (tma_ok(stage + T::POP, i0 + a.lf.gx - T::AC, yf - 1, kFe))
        tma_load_3d(stage + T::POP, mu, bar, i0 + a.lf.gx - T::AC, yf - 1, 0);
    if (tma_ok(stage + T::POP + T::U, i0 + a.lf.gx, yf, kFe))
        tma_load_2d(stage + T::POP + T::U, md, bar, i0 + a.lf.gx, yf);
    if (SRC == TRTR_SRC_FIELD) {
        unsigned char* s = stage + T::POP + T::U + T::D;
        if (tma_ok(s, i0 + a.lf.gx, yf, kFe)) tma_load_3d(s, ms, bar, i0 + a.lf.gx, yf, a.s_cur);
        if (tma_ok(s + T::S_TILE, i0 + a.lf.gx, yf, kFe))
            tma_load_3d(s + T::S_TILE, ms, bar, i0 + a.lf.gx, yf, a.s_prev);
    }
}

// One tile row r of the FP32-computing storages, or NM * 64 columns of it from column c0: lane
// handles the node pairs (i0 + c0 + 64 m + 2 lane, + 1), m = 0 .. NM - 1.
//
// Stores: TST = false writes every value to global memory from the lanes.  TST = true (one warp
// per whole row) writes the row's nine result rows into shared memory over the row's own input
// rows (only this warp reads them; the results of pair m cover columns 64 m .. 64 m + 63, which
// no later pair reads), and lane 0 then copies each plane's row to global memory with one bulk
// copy of the row's first `bulk_cols(nx - i0)` columns (16-byte multiples: the row starts are
// 16-byte aligned in both memories).  The lanes store the few columns past those, and the ghost
// copies of edge nodes, directly.
// UNR: the unroll factor of the pair loop (1: one pair at a time; NM: all pairs interleaved).
// SR: the 2-byte storages round stochastically (TRTR_ROUND_STOCHASTIC), with the random bits of
// sr_hash keyed by the node pair and a.rkey.
template <typename S, int SRC, int BX, int BY, int NM = BX / 64, bool TST = false, int UNR = 1, bool SR = false>
__device__ __forceinline__ void tile_row_pairs(const unsigned char* st, int r, int lane, int i0, int j,
                                               const StepArgs<float>& a, const F2* sx, const F2* cx, float sy,
                                               float cy, int c0 = 0) {
    static_assert(!TST || NM == BX / 64, "bulk row stores need one warp per tile row");
    using T = Tile<S, SRC, BX, BY>;
    using P = Pair<S>;
    using S2 = typename P::type;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const S* sp = reinterpret_cast<const S*>(st) + r * T::PW;
    const float* su = reinterpret_cast<const float*>(st + T::POP) + (r + 1) * T::UW + T::AC;
    const float* sv = su + T::UH * T::UW;
    const float* sd = reinterpret_cast<const float*>(st + T::POP + T::U) + r * BX;
    const float* ss = reinterpret_cast<const float*>(st + T::POP + T::U + T::D) + r * BX;
    const float phi_ref = a.phi_ref;
    constexpr bool kOfs = sizeof(S) == 2;  // offset storages: h_i = g_i - w_i phi_ref, folded into the moments
    S* dst = static_cast<S*>(a.dst);
    const size_t pl = a.lp.plane;
    const F2 magic(a.magic), w2f(a.omega2_fixed);
#pragma unroll (UNR)
    for (int m = 0; m < NM; ++m) {
        const int c = c0 + 64 * m + 2 * lane;  // column of the pair inside the tile
        const int i = i0 + c;
        if (!TST && i >= nx) break;  // (TST: pairs past nx are computed; their columns are not stored)
        // a1: pull-streaming from the shifted tiles
        F2 g[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const S* pq = sp + q * T::PLANE_ELEMS + c + plane_offset<T::A>(q);
            if (plane_offset<T::A>(q) % 2 == 0)
                g[q] = P::raw(*reinterpret_cast<const S2*>(pq));
            else
                g[q] = P::raw(pq[0], pq[1]);
        }
        // u, its central differences (ghosts make edges one-sided or periodic), D
        const float2 uc = *reinterpret_cast<const float2*>(su + c);
        const float2 vc = *reinterpret_cast<const float2*>(sv + c);
        const F2 ux(uc), uy(vc);
        const F2 dxux = F2(0.5f) * (F2(uc.y, su[c + 2]) - F2(su[c - 1], uc.x));
        const F2 dxuy = F2(0.5f) * (F2(vc.y, sv[c + 2]) - F2(sv[c - 1], vc.x));
        const F2 dyux = F2(0.5f) * (F2(*reinterpret_cast<const float2*>(su + c + T::UW)) -
                                    F2(*reinterpret_cast<const float2*>(su + c - T::UW)));
        const F2 dyuy = F2(0.5f) * (F2(*reinterpret_cast<const float2*>(sv + c + T::UW)) -
                                    F2(*reinterpret_cast<const float2*>(sv + c - T::UW)));
        const F2 ax = vfma(ux, dxux, uy * dyux);  // (u.grad) u_x
        const F2 ay = vfma(ux, dxuy, uy * dyuy);  // (u.grad) u_y
        const F2 Dh(*reinterpret_cast<const float2*>(sd + c));

        // a7: s = dt S^n + dt/2 (S^n - S^{n-1})
        F2 src(0.f);
        if (SRC == TRTR_SRC_FIELD) {
            const F2 sn(*reinterpret_cast<const float2*>(ss + c));
            const F2 sp_(*reinterpret_cast<const float2*>(ss + T::S_TILE / sizeof(float) + c));
            src = vfma(F2(1.5f), sn, F2(-0.5f) * sp_);
        } else if (SRC == TRTR_SRC_PULSE) {
            const F2 x = vfma(F2((float)i, (float)(i + 1)), F2(a.dx), F2(a.x0));
            const F2 y(a.y0 + (float)j * a.dx);
            F2 sxm = sx[0], cxm = cx[0];  // compile-time indices only (no local-memory arrays)
#pragma unroll
            for (int mm = 1; mm < NM; ++mm)
                if (m == mm) {
                    sxm = sx[mm];
                    cxm = cx[mm];
                }
            const F2 dD = F2(a.dD_amp * sy) * sxm;
            const F2 dDx = F2(a.dD_amp * 3.14159265358979323846f * sy) * cxm;
            const F2 dDy = F2(a.dD_amp * 3.14159265358979323846f * cy) * sxm;
            src = pulse_source_dt(x, y, a.tf, dD, dDx, dDy);
        }

        F2 out[kQ];
        // 2-byte storages: g and out stay offsets (the offset is folded into the moments)
        collide_node<F2, kOfs>(g, ux, uy, ax, ay, Dh, src, magic, w2f, a.tau2_fixed, out, F2(phi_ref));
        const uint32_t rk = SR ? sr_pair_key(i, j, nx, a.rkey) : 0u;
        auto enc = [&](int q) -> S2 {
            if constexpr (SR)
                return P::encode_sr(out[q], sr_bits(rk, q));
            else
                return P::encode_raw(out[q]);
        };

        // a8: store P_i(x); edge nodes also write their periodic ghost copies (the one-wide frame
        // that the one-step kernel reads)
        const bool edge = j == 0 || j == ny - 1 || i == 0 || i + 1 >= nx - 1;
        if constexpr (TST) {
            __syncwarp();  // every lane has read its inputs of pair m
            S* srow = const_cast<S*>(sp);
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                *reinterpret_cast<S2*>(srow + q * T::PLANE_ELEMS + c) = enc(q);
            const int nb = bulk_cols<S>(nx - i0);
            if ((edge || c + 1 >= nb) && i < nx) {  // ghost copies, and the columns past the bulk copy
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const S2 v = enc(q);
                    const S v0 = reinterpret_cast<const S*>(&v)[0], v1 = reinterpret_cast<const S*>(&v)[1];
                    if (c >= nb) dst[q * pl + a.lp.at_g<kGhostP>(i, j)] = v0;
                    if (c + 1 >= nb && i + 1 < nx) dst[q * pl + a.lp.at_g<kGhostP>(i + 1, j)] = v1;
                    store_ghosts<1, kGhostP>(dst + q * pl, a.lp, i, j, v0);
                    if (i + 1 < nx) store_ghosts<1, kGhostP>(dst + q * pl, a.lp, i + 1, j, v1);
                }
            }
        } else if (!edge) {
            S* d0 = dst + a.lp.at_g<kGhostP>(i, j);
#if TRTR_BOUNDS_CHECK
            if (i + 1 >= nx || (reinterpret_cast<uintptr_t>(d0) % sizeof(S2)) != 0u) {
                TRTR_BOUNDS_FAULT(kBoundsPair, i, j);
                continue;
            }
#endif
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                *reinterpret_cast<S2*>(d0 + q * pl) = enc(q);
        } else {
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const S2 v = enc(q);
                store_with_ghosts<1, kGhostP>(dst + q * pl, a.lp, i, j, reinterpret_cast<const S*>(&v)[0]);
                if (i + 1 < nx) store_with_ghosts<1, kGhostP>(dst + q * pl, a.lp, i + 1, j, reinterpret_cast<const S*>(&v)[1]);
            }
        }
    }
    if constexpr (TST) {
        fence_proxy_async_smem();  // the result rows, for the bulk copies
        __syncwarp();
        const int nb = bulk_cols<S>(nx - i0);
        if (lane == 0 && nb > 0) {
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                if (bulk_ok(dst + q * pl + a.lp.at_g<kGhostP>(i0, j), sp + q * T::PLANE_ELEMS, i0, j, nb, a.lp))
                    bulk_store(dst + q * pl + a.lp.at_g<kGhostP>(i0, j), sp + q * T::PLANE_ELEMS, (uint32_t)(nb * sizeof(S)));
            bulk_commit();
            bulk_wait_read();  // the stage may be refilled after the CTA barrier
        }
    }
}

// One tile row of the FP64 path, or NMF * 32 columns of it from column c0: lane handles nodes
// i0 + c0 + 32 m + lane, m = 0 .. NMF - 1.  TST: bulk row stores as in tile_row_pairs.
template <int SRC, int BX, int BY, int NMF = BX / 32, bool TST = false>
__device__ __forceinline__ void tile_row_f64(const unsigned char* st, int r, int lane, int i0, int j,
                                             const StepArgs<double>& a, int c0 = 0) {
    static_assert(!TST || NMF == BX / 32, "bulk row stores need one warp per tile row");
    using T = Tile<double, SRC, BX, BY>;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const double* sp = reinterpret_cast<const double*>(st) + r * T::PW;
    const double* su = reinterpret_cast<const double*>(st + T::POP) + (r + 1) * T::UW + T::AC;
    const double* sv = su + T::UH * T::UW;
    const double* sd = reinterpret_cast<const double*>(st + T::POP + T::U) + r * BX;
    const double* ss = reinterpret_cast<const double*>(st + T::POP + T::U + T::D) + r * BX;
    double* dst = static_cast<double*>(a.dst);
    const size_t pl = a.lp.plane;
    double sy = 0.0, cy = 0.0;
    if (SRC == TRTR_SRC_PULSE) {
        sy = __ldg(a.tab_y + j);
        cy = __ldg(a.tab_y + ny + j);
    }
#pragma unroll 1
    for (int m = 0; m < NMF; ++m) {
        const int c = c0 + 32 * m + lane;
        const int i = i0 + c;
        if (!TST && i >= nx) break;
        double g[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) g[q] = sp[q * T::PLANE_ELEMS + c + plane_offset<T::A>(q)];
        const double ux = su[c], uy = sv[c];
        const double dxux = 0.5 * (su[c + 1] - su[c - 1]);
        const double dxuy = 0.5 * (sv[c + 1] - sv[c - 1]);
        const double dyux = 0.5 * (su[c + T::UW] - su[c - T::UW]);
        const double dyuy = 0.5 * (sv[c + T::UW] - sv[c - T::UW]);
        const double ax = fma(ux, dxux, uy * dyux);
        const double ay = fma(ux, dxuy, uy * dyuy);
        double src = 0.0;
        if (SRC == TRTR_SRC_FIELD) {
            src = fma(1.5, ss[c], -0.5 * ss[T::S_TILE / sizeof(double) + c]);
        } else if (SRC == TRTR_SRC_PULSE) {
            const double x = a.x0 + (double)i * a.dx, y = a.y0 + (double)j * a.dx;
            const double sx = __ldg(a.tab_x + i), cx = __ldg(a.tab_x + nx + i);
            const double dD = a.dD_amp * sx * sy;
            const double dDx = a.dD_amp * 3.14159265358979323846 * cx * sy;
            const double dDy = a.dD_amp * 3.14159265358979323846 * sx * cy;
            const double Sn = pulse_source(x, y, a.tf.cx_n, a.tf.cy_n, a.tf.inv_s2_n, a.tf.a_n, dD, dDx, dDy);
            const double Sp = pulse_source(x, y, a.tf.cx_p, a.tf.cy_p, a.tf.inv_s2_p, a.tf.a_p, dD, dDx, dDy);
            src = a.dt * fma(1.5, Sn, -0.5 * Sp);
        }
        double out[kQ];
        collide_node<double>(g, ux, uy, ax, ay, sd[c], src, a.magic, a.omega2_fixed, a.tau2_fixed, out);
        if constexpr (TST) {
            __syncwarp();  // every lane has read its inputs of node m
            double* srow = const_cast<double*>(sp);
#pragma unroll
            for (int q = 0; q < kQ; ++q) srow[q * T::PLANE_ELEMS + c] = out[q];
            if (i < nx) {
                const bool tail = c >= bulk_cols<double>(nx - i0);
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    if (tail) dst[q * pl + a.lp.at_g<kGhostP>(i, j)] = out[q];
                    store_ghosts<1, kGhostP>(dst + q * pl, a.lp, i, j, out[q]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < kQ; ++q) store_with_ghosts<1, kGhostP>(dst + q * pl, a.lp, i, j, out[q]);
        }
    }
    if constexpr (TST) {
        fence_proxy_async_smem();
        __syncwarp();
        const int nb = bulk_cols<double>(nx - i0);
        if (lane == 0 && nb > 0) {
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                if (bulk_ok(dst + q * pl + a.lp.at_g<kGhostP>(i0, j), sp + q * T::PLANE_ELEMS, i0, j, nb, a.lp))
                    bulk_store(dst + q * pl + a.lp.at_g<kGhostP>(i0, j), sp + q * T::PLANE_ELEMS,
                               (uint32_t)(nb * sizeof(double)));
            bulk_commit();
            bulk_wait_read();
        }
    }
}


// ---- host side: TMA descriptors --------------------------------------------------------

// L2 fill granularity of the TMA loads: 0 none, 1 64 B, 2 128 B, 3 256 B.
#ifndef TRTR_L2_PROMOTION
#define TRTR_L2_PROMOTION 0
#endif

template <typename S>
CUtensorMapDataType tma_type();
template <>
inline CUtensorMapDataType tma_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <>
inline CUtensorMapDataType tma_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <>
inline CUtensorMapDataType tma_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <>
inline CUtensorMapDataType tma_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

inline PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

constexpr CUtensorMapL2promotion kPromotion =
    TRTR_L2_PROMOTION == 1   ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
    : TRTR_L2_PROMOTION == 2 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
    : TRTR_L2_PROMOTION == 3 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                             : CU_TENSOR_MAP_L2_PROMOTION_NONE;

inline bool encode(CUtensorMap* m, CUtensorMapDataType t, int elem, void* base, const PlaneLayout& L, int depth, int bw,
            int bh, int bd) {
    auto fn = get_encoder();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)depth};
    const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * elem, (cuuint64_t)L.plane * elem};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bd};
    const cuuint32_t es[3] = {1, 1, 1};
    const cuuint32_t rank = depth > 1 ? 3 : 2;
    return fn(m, t, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              kPromotion, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


}  // namespace core
}  // namespace trtr
