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
// Data movement (sm_103a): a persistent kernel, two CTAs per SM, walks 128 x 8-node
// tiles.  For each tile one thread issues TMA loads (cp.async.bulk.tensor) of the nine
// shifted population tiles, the u tile with its one-node halo and the D tile into a
// shared-memory stage and arms an mbarrier with the expected byte count; the stages form a
// ring so the loads of the next tiles are in flight while the current one is computed.
// The pull shift of plane i is a tile origin moved by -e_i; TMA needs 16-byte aligned x
// origins, so the planes with e_x = +1 start one 16-byte chunk early and are read from
// shared memory with a column offset.  Ghost cells of the layout make the periodic wrap a
// plain tile read.  Results go to global memory with coalesced stores (one warp = one
// 128-node row), ghost copies included.  Every mbarrier wait is bounded: on timeout the
// kernel raises the context's flag and returns.
#include <cudaTypedefs.h>

#include <type_traits>

#include "trtr_internal.cuh"

namespace trtr {
namespace {

constexpr int kBX = 128;            // nodes per tile along x (4 per lane)
constexpr int kBY = 8;              // tile rows = warps per CTA
constexpr int kThreads = 32 * kBY;
constexpr int kMinBlocks = 2;  // two CTAs per SM: at most 128 registers per thread

// Tile order across the persistent CTAs: 0 = interleaved row-major (tile = CTA + k * grid,
// so the CTAs sweep the grid together row band by row band and neighbouring tiles are
// fetched at the same time), 1 = contiguous column-major chunk per CTA, 2 = contiguous
// row-major chunk per CTA (x-neighbour tiles follow each other in one CTA, so the 16-byte
// x over-fetch of the shifted planes is still in L2).  Measured on GB300: 4-byte and 8-byte
// storage run fastest with 2, 2-byte storage with 0.
#ifndef TRTR_TILE_ORDER_WIDE
#define TRTR_TILE_ORDER_WIDE 2
#endif
#ifndef TRTR_TILE_ORDER_HALF
#define TRTR_TILE_ORDER_HALF 0
#endif
// L2 fill granularity of the TMA loads: 0 none, 1 64 B, 2 128 B, 3 256 B.
#ifndef TRTR_L2_PROMOTION
#define TRTR_L2_PROMOTION 0
#endif
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

template <typename S, int SRC>
struct Tile {
    using C = typename Store<S>::C;
    static constexpr int A = 16 / (int)sizeof(S);    // TMA x quantum of the populations
    static constexpr int PW = kBX + A;               // population tile width
    static constexpr int AC = 16 / (int)sizeof(C);   // TMA x quantum of the fields
    static constexpr int UW = kBX + 2 * AC;          // u tile width (halo rounded to AC)
    static constexpr int UH = kBY + 2;
    static constexpr uint32_t POP_PLANE = kBY * PW * sizeof(S);
    static constexpr uint32_t POP = kQ * POP_PLANE;
    static constexpr uint32_t U = 2 * UH * UW * sizeof(C);
    static constexpr uint32_t D = kBY * kBX * sizeof(C);
    static constexpr uint32_t SRCB = SRC == TRTR_SRC_FIELD ? 2 * kBY * kBX * sizeof(C) : 0;
    static constexpr uint32_t TX = POP + U + D + SRCB;            // bytes the TMA delivers
    static constexpr uint32_t STAGE = (TX + 127) / 128 * 128;
    static_assert(POP_PLANE % 128 == 0 && U % 128 == 0 && D % 128 == 0, "128-byte aligned tiles");
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

// Waits for the phase `parity` of `bar` to complete, for at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
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

// The node update of Eq. (14) in moment space; g: pre-collision populations, out: P_i(x).
template <class V>
__device__ __forceinline__ void collide_node(const V g[kQ], V ux, V uy, V ax, V ay, V Dh, V s, V magic, V w2_fixed,
                                             bool tau2_fixed, V out[kQ]) {
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
    const V phi = (g[0] + p12) + (p34 + pdiag);
    const V jx = d12 + (d56 + d78);
    const V jy = d34 + (d56 - d78);
    const V pxx = p12 + pdiag;
    const V pyy = p34 + pdiag;
    const V pxy = p56 - p78;

    // a5 + a6 + a7: post-collision Hermite coefficients
    const V phux = phi * ux, phuy = phi * uy;
    const V euxx = phux * ux, euyy = phuy * uy, euxy = phux * uy;
    const V m0 = phi + s;
    const V m1x = vfma(kh, vfma(phi, ax, ux * s), vfma(k1, jx - phux, phux));
    const V m1y = vfma(kh, vfma(phi, ay, uy * s), vfma(k1, jy - phuy, phuy));
    const V third = phi * V(T(1.0 / 3.0));
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
    out[0] = vfma(V(T(-2.0 / 3.0)), Asum, m0 * V(T(4.0 / 9.0)));
    out[1] = E1 + O1;
    out[2] = E1 - O1;
    out[3] = E3 + O3;
    out[4] = E3 - O3;
    out[5] = E5 + O5;
    out[6] = E5 - O5;
    out[7] = E7 + O7;
    out[8] = E7 - O7;
}

template <typename C>
__device__ __forceinline__ C weight(int q) {
    return q == 0 ? C(4.0 / 9.0) : (q < 5 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}

// Shared-memory column offset of plane q's tile (see the TMA origin in issue_tile).
template <int A>
__device__ __forceinline__ constexpr int plane_offset(int q) {
    return lattice_ex(q) == 1 ? A - 1 : (lattice_ex(q) == -1 ? 1 : 0);
}

// Pair (2-element) storage vectors and their conversion to / from packed FP32.
template <typename S>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
    static __device__ __forceinline__ F2 decode(float2 v, float) { return F2(v); }
    static __device__ __forceinline__ F2 decode(float a, float b, float) { return F2(a, b); }
    static __device__ __forceinline__ float2 encode(F2 v, float) { return v.v; }
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
};

template <typename S, int SRC>
__device__ __forceinline__ void issue_tile(unsigned char* stage, uint64_t* bar, const CUtensorMap* mp,
                                           const CUtensorMap* mu, const CUtensorMap* md, const CUtensorMap* ms,
                                           int i0, int j0, const StepArgs<typename Store<S>::C>& a) {
    using T = Tile<S, SRC>;
    mbar_expect_tx(bar, T::TX);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const int x = i0 + a.lp.gx - (lattice_ex(q) == 1 ? T::A : 0);
        const int y = j0 + 1 - lattice_ey(q);
        tma_load_3d(stage + q * T::POP_PLANE, mp, bar, x, y, q);
    }
    tma_load_3d(stage + T::POP, mu, bar, i0 + a.lf.gx - T::AC, j0, 0);
    tma_load_2d(stage + T::POP + T::U, md, bar, i0 + a.lf.gx, j0 + 1);
    if (SRC == TRTR_SRC_FIELD) {
        unsigned char* s = stage + T::POP + T::U + T::D;
        tma_load_3d(s, ms, bar, i0 + a.lf.gx, j0 + 1, a.s_cur);
        tma_load_3d(s + kBY * kBX * sizeof(typename Store<S>::C), ms, bar, i0 + a.lf.gx, j0 + 1, a.s_prev);
    }
}

// One tile row (warp r) of the FP32-computing storages: lane handles the node pairs
// (i0 + 64 m + 2 lane, + 1), m = 0, 1.
template <typename S, int SRC>
__device__ __forceinline__ void tile_row_pairs(const unsigned char* st, int r, int lane, int i0, int j,
                                               const StepArgs<float>& a, const F2 sx[2], const F2 cx[2], float sy,
                                               float cy) {
    using T = Tile<S, SRC>;
    using P = Pair<S>;
    using S2 = typename P::type;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const S* sp = reinterpret_cast<const S*>(st) + r * T::PW;
    const float* su = reinterpret_cast<const float*>(st + T::POP) + (r + 1) * T::UW + T::AC;
    const float* sv = su + T::UH * T::UW;
    const float* sd = reinterpret_cast<const float*>(st + T::POP + T::U) + r * kBX;
    const float* ss = reinterpret_cast<const float*>(st + T::POP + T::U + T::D) + r * kBX;
    const float phi_ref = a.phi_ref;
    S* dst = static_cast<S*>(a.dst);
    const size_t pl = a.lp.plane;
    const F2 magic(a.magic), w2f(a.omega2_fixed);
#pragma unroll 1
    for (int m = 0; m < kBX / 64; ++m) {
        const int c = 64 * m + 2 * lane;  // column of the pair inside the tile
        const int i = i0 + c;
        if (i >= nx) break;
        // a1: pull-streaming from the shifted tiles
        F2 g[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const S* pq = sp + q * (kBY * T::PW) + c + plane_offset<T::A>(q);
            const float off = weight<float>(q) * phi_ref;
            if (plane_offset<T::A>(q) % 2 == 0)
                g[q] = P::decode(*reinterpret_cast<const S2*>(pq), off);
            else
                g[q] = P::decode(pq[0], pq[1], off);
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
            const F2 sp_(*reinterpret_cast<const float2*>(ss + kBY * kBX + c));
            src = vfma(F2(1.5f), sn, F2(-0.5f) * sp_);
        } else if (SRC == TRTR_SRC_PULSE) {
            const F2 x = vfma(F2((float)i, (float)(i + 1)), F2(a.dx), F2(a.x0));
            const F2 y(a.y0 + (float)j * a.dx);
            const F2 sxm = m == 0 ? sx[0] : sx[1], cxm = m == 0 ? cx[0] : cx[1];
            const F2 dD = F2(a.dD_amp * sy) * sxm;
            const F2 dDx = F2(a.dD_amp * 3.14159265358979323846f * sy) * cxm;
            const F2 dDy = F2(a.dD_amp * 3.14159265358979323846f * cy) * sxm;
            const F2 Sn = pulse_source(x, y, F2(a.cx_n), F2(a.cy_n), F2(a.inv_s2_n), F2(a.amp_n), dD, dDx, dDy);
            const F2 Sp = a.first_step
                              ? Sn
                              : pulse_source(x, y, F2(a.cx_p), F2(a.cy_p), F2(a.inv_s2_p), F2(a.amp_p), dD, dDx, dDy);
            src = F2(a.dt) * vfma(F2(1.5f), Sn, F2(-0.5f) * Sp);
        }

        F2 out[kQ];
        collide_node<F2>(g, ux, uy, ax, ay, Dh, src, magic, w2f, a.tau2_fixed, out);

        // a8: store P_i(x); edge nodes also write their periodic ghost copies
        const bool edge = j == 0 || j == ny - 1 || i == 0 || i + 1 >= nx - 1;
        if (!edge) {
            S* d0 = dst + a.lp.at(i, j);
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                *reinterpret_cast<S2*>(d0 + q * pl) = P::encode(out[q], weight<float>(q) * phi_ref);
        } else {
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const float off = weight<float>(q) * phi_ref;
                store_with_ghosts(dst + q * pl, a.lp, i, j, Store<S>::encode(out[q].v.x, off));
                if (i + 1 < nx) store_with_ghosts(dst + q * pl, a.lp, i + 1, j, Store<S>::encode(out[q].v.y, off));
            }
        }
    }
}

// One tile row of the FP64 path: lane handles nodes i0 + 32 m + lane, m = 0..3.
template <int SRC>
__device__ __forceinline__ void tile_row_f64(const unsigned char* st, int r, int lane, int i0, int j,
                                             const StepArgs<double>& a) {
    using T = Tile<double, SRC>;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const double* sp = reinterpret_cast<const double*>(st) + r * T::PW;
    const double* su = reinterpret_cast<const double*>(st + T::POP) + (r + 1) * T::UW + T::AC;
    const double* sv = su + T::UH * T::UW;
    const double* sd = reinterpret_cast<const double*>(st + T::POP + T::U) + r * kBX;
    const double* ss = reinterpret_cast<const double*>(st + T::POP + T::U + T::D) + r * kBX;
    double* dst = static_cast<double*>(a.dst);
    const size_t pl = a.lp.plane;
    double sy = 0.0, cy = 0.0;
    if (SRC == TRTR_SRC_PULSE) {
        sy = __ldg(a.tab_y + j);
        cy = __ldg(a.tab_y + ny + j);
    }
#pragma unroll 1
    for (int m = 0; m < kBX / 32; ++m) {
        const int c = 32 * m + lane;
        const int i = i0 + c;
        if (i >= nx) break;
        double g[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) g[q] = sp[q * (kBY * T::PW) + c + plane_offset<T::A>(q)];
        const double ux = su[c], uy = sv[c];
        const double dxux = 0.5 * (su[c + 1] - su[c - 1]);
        const double dxuy = 0.5 * (sv[c + 1] - sv[c - 1]);
        const double dyux = 0.5 * (su[c + T::UW] - su[c - T::UW]);
        const double dyuy = 0.5 * (sv[c + T::UW] - sv[c - T::UW]);
        const double ax = fma(ux, dxux, uy * dyux);
        const double ay = fma(ux, dxuy, uy * dyuy);
        double src = 0.0;
        if (SRC == TRTR_SRC_FIELD) {
            src = fma(1.5, ss[c], -0.5 * ss[kBY * kBX + c]);
        } else if (SRC == TRTR_SRC_PULSE) {
            const double x = a.x0 + (double)i * a.dx, y = a.y0 + (double)j * a.dx;
            const double sx = __ldg(a.tab_x + i), cx = __ldg(a.tab_x + nx + i);
            const double dD = a.dD_amp * sx * sy;
            const double dDx = a.dD_amp * 3.14159265358979323846 * cx * sy;
            const double dDy = a.dD_amp * 3.14159265358979323846 * sx * cy;
            const double Sn = pulse_source(x, y, a.cx_n, a.cy_n, a.inv_s2_n, a.amp_n, dD, dDx, dDy);
            const double Sp =
                a.first_step ? Sn : pulse_source(x, y, a.cx_p, a.cy_p, a.inv_s2_p, a.amp_p, dD, dDx, dDy);
            src = a.dt * fma(1.5, Sn, -0.5 * Sp);
        }
        double out[kQ];
        collide_node<double>(g, ux, uy, ax, ay, sd[c], src, a.magic, a.omega2_fixed, a.tau2_fixed, out);
#pragma unroll
        for (int q = 0; q < kQ; ++q) store_with_ghosts(dst + q * pl, a.lp, i, j, out[q]);
    }
}

template <typename S, int SRC, int STAGES>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    step_kernel(const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap mu,
                const __grid_constant__ CUtensorMap md, const __grid_constant__ CUtensorMap ms,
                const StepArgs<typename Store<S>::C> a) {
    using T = Tile<S, SRC>;
    constexpr bool kPairs = !std::is_same<S, double>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_abort;
    // stages on a 128-byte boundary (TMA destination alignment), barriers after them
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                           ~static_cast<uintptr_t>(127));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * T::STAGE);

    const int tid = threadIdx.x, lane = tid & 31, r = tid >> 5;
    const int nx = a.lp.nx, ny = a.lp.ny;
    const int ntx = (nx + kBX - 1) / kBX, nty = (ny + kBY - 1) / kBY;
    const int ntiles = ntx * nty;
    constexpr int kOrder = sizeof(S) == 2 ? TRTR_TILE_ORDER_HALF : TRTR_TILE_ORDER_WIDE;
    const int chunk = (ntiles + gridDim.x - 1) / gridDim.x;
    const int first = kOrder == 0 ? blockIdx.x : blockIdx.x * chunk;
    const int stride = kOrder == 0 ? gridDim.x : 1;
    const int my_tiles = kOrder == 0 ? (first < ntiles ? (ntiles - 1 - first) / stride + 1 : 0)
                                     : (first < ntiles ? min(chunk, ntiles - first) : 0);
    auto tile_x0 = [&](int k) {
        const int t = first + k * stride;
        return (kOrder == 1 ? t / nty : t % ntx) * kBX;
    };
    auto tile_y0 = [&](int k) {
        const int t = first + k * stride;
        return (kOrder == 1 ? t % nty : t / ntx) * kBY;
    };

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < STAGES && k < my_tiles; ++k)
            issue_tile<S, SRC>(smem + k * T::STAGE, &full[k], &mp, &mu, &md, &ms, tile_x0(k), tile_y0(k), a);
    }

    for (int k = 0; k < my_tiles; ++k) {
        const int s = k % STAGES;
        const int i0 = tile_x0(k), j0 = tile_y0(k);
        const int j = j0 + r;

        // per-column / per-row pulse tables, loaded before the wait so their latency hides
        F2 sx[2], cx[2];
        float sy = 0.f, cy = 0.f;
        if (kPairs && SRC == TRTR_SRC_PULSE) {
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int i = i0 + 64 * m + 2 * lane;
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
                tile_row_pairs<S, SRC>(st, r, lane, i0, j, a, sx, cx, sy, cy);
            else
                tile_row_f64<SRC>(st, r, lane, i0, j, a);
        }
        __syncthreads();  // stage s fully read (and s_abort visible)
        if (s_abort) {
            if (tid == 0) {
                atomicExch(a.flag, 1);
                // let the loads already issued into this CTA's shared memory land (bounded)
                for (int kk = k + 1; kk < my_tiles && kk < k + STAGES; ++kk)
                    mbar_wait_bounded(&full[kk % STAGES], (kk / STAGES) & 1);
            }
            return;
        }
        if (tid == 0 && k + STAGES < my_tiles)
            issue_tile<S, SRC>(smem + s * T::STAGE, &full[s], &mp, &mu, &md, &ms, tile_x0(k + STAGES),
                               tile_y0(k + STAGES), a);
    }
}

// Stages per CTA: two when they fit in the 227 KB a CTA may use, else one.
template <typename S, int SRC>
constexpr int stages_for() {
    return 2 * Tile<S, SRC>::STAGE + 256 <= 227 * 1024 ? 2 : 1;
}

// ------------------------------------------------------------------------------ host side

template <typename S>
CUtensorMapDataType tma_type();
template <>
CUtensorMapDataType tma_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <>
CUtensorMapDataType tma_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <>
CUtensorMapDataType tma_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <>
CUtensorMapDataType tma_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
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

bool encode(CUtensorMap* m, CUtensorMapDataType t, int elem, void* base, const PlaneLayout& L, int depth, int bw,
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

template <typename S>
cudaError_t encode_typed(trtr_ctx* ctx) {
    using C = typename Store<S>::C;
    // The box shapes do not depend on the source mode (TX bytes do).
    using T = Tile<S, TRTR_SRC_NONE>;
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        ok = ok && encode(&ctx->maps[kMapPop0 + b], tma_type<S>(), sizeof(S), ctx->pop[b], ctx->lp, kQ, T::PW, kBY, 1);
    ok = ok && encode(&ctx->maps[kMapU], tma_type<C>(), sizeof(C), ctx->uv, ctx->lf, 2, T::UW, T::UH, 2);
    ok = ok && encode(&ctx->maps[kMapD], tma_type<C>(), sizeof(C), ctx->Dh, ctx->lf, 1, kBX, kBY, 1);
    if (ctx->S) ok = ok && encode(&ctx->maps[kMapS], tma_type<C>(), sizeof(C), ctx->S, ctx->lf, 2, kBX, kBY, 1);
    else ctx->maps[kMapS] = ctx->maps[kMapD];
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename S, int SRC>
cudaError_t launch_typed(trtr_ctx* ctx) {
    using C = typename Store<S>::C;
    using T = Tile<S, SRC>;
    constexpr int kStages = stages_for<S, SRC>();
    auto kernel = step_kernel<S, SRC, kStages>;
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
    a.dst = ctx->pop[ctx->cur ^ 1];
    a.tab_x = static_cast<const C*>(ctx->tab_x);
    a.tab_y = static_cast<const C*>(ctx->tab_y);
    a.flag = ctx->dflag;
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
    a.first_step = ctx->step == 0;
    if (SRC == TRTR_SRC_PULSE) {
        const PulseTime tn = pulse_at(ctx->pulse, (double)ctx->step * ctx->p.dt);
        const PulseTime tp = pulse_at(ctx->pulse, (double)(ctx->step - 1) * ctx->p.dt);
        a.dD_amp = C(ctx->pulse.D0 * ctx->pulse.D_amp);
        a.cx_n = C(tn.cx); a.cy_n = C(tn.cy); a.inv_s2_n = C(tn.inv_s2); a.amp_n = C(tn.amp);
        a.cx_p = C(tp.cx); a.cy_p = C(tp.cy); a.inv_s2_p = C(tp.inv_s2); a.amp_p = C(tp.amp);
    } else {
        a.dD_amp = C(0);
        a.cx_n = a.cy_n = a.inv_s2_n = a.amp_n = C(0);
        a.cx_p = a.cy_p = a.inv_s2_p = a.amp_p = C(0);
    }
    const long ntiles = (long)((ctx->lp.nx + kBX - 1) / kBX) * ((ctx->lp.ny + kBY - 1) / kBY);
    const long cap = (long)ctx->num_sms * ctas_per_sm;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    kernel<<<grid, kThreads, smem, ctx->stream>>>(ctx->maps[kMapPop0 + ctx->cur], ctx->maps[kMapU], ctx->maps[kMapD],
                                                  ctx->maps[kMapS], a);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_src(trtr_ctx* ctx) {
    switch (ctx->p.src_mode) {
        case TRTR_SRC_FIELD: return launch_typed<S, TRTR_SRC_FIELD>(ctx);
        case TRTR_SRC_PULSE: return launch_typed<S, TRTR_SRC_PULSE>(ctx);
        default: return launch_typed<S, TRTR_SRC_NONE>(ctx);
    }
}

}  // namespace

cudaError_t encode_maps(trtr_ctx* ctx) {
    switch (ctx->p.precision) {
        case TRTR_F64: return encode_typed<double>(ctx);
        case TRTR_F32: return encode_typed<float>(ctx);
        case TRTR_F16_OFS: return encode_typed<__half>(ctx);
        case TRTR_BF16_OFS: return encode_typed<__nv_bfloat16>(ctx);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(trtr_ctx* ctx) {
    switch (ctx->p.precision) {
        case TRTR_F64: return launch_src<double>(ctx);
        case TRTR_F32: return launch_src<float>(ctx);
        case TRTR_F16_OFS: return launch_src<__half>(ctx);
        case TRTR_BF16_OFS: return launch_src<__nv_bfloat16>(ctx);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace trtr
