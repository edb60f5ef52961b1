// trtr_internal.cuh -- context layout, storage traits and kernel launchers of the TRT-R
// library (not part of the public ABI).
//
// Device layout (all buffers owned by the context):
//   populations  2 x [9][ny][pitch]   stored post-collision values P_i(x) of the previous
//                                     step; the pre-collision population is the pull
//                                     g_i(x, t_n) = P_i(x - e_i) (periodic)
//   fields       ux, uy, Dh [ny][pitch] in the compute type, lattice units:
//                uhat = u dt/dx, Dh = D dt/dx^2  (tau1 = 1/2 + 3 Dh)
//   source       2 x [ny][pitch] dt*S (TRTR_SRC_FIELD only)
//   pulse tab    sin(pi x_i), cos(pi x_i) [pitch] and sin(pi y_j), cos(pi y_j) [ny]
//   scratch      FP64 partial sums of the reductions, one pair per reduction block
// pitch = nx rounded up to 32 elements so that every row starts on a 128-byte boundary.
#pragma once

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

// Storage traits: how a population is kept in memory and turned into the compute type.
template <typename S>
struct Store;

template <>
struct Store<double> {
    using C = double;
    static __device__ __forceinline__ double load(const double* p, double) { return __ldg(p); }
    static __device__ __forceinline__ void store(double* p, double v, double) { *p = v; }
};

template <>
struct Store<float> {
    using C = float;
    static __device__ __forceinline__ float load(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, float v, float) { *p = v; }
};

// Half-precision offset storage: h = g - w_i phi_ref.
template <>
struct Store<__half> {
    using C = float;
    static __device__ __forceinline__ float load(const __half* p, float off) {
        return __half2float(__ldg(p)) + off;
    }
    static __device__ __forceinline__ void store(__half* p, float v, float off) { *p = __float2half_rn(v - off); }
};

template <>
struct Store<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p, float off) {
        return __bfloat162float(__ldg(p)) + off;
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v, float off) {
        *p = __float2bfloat16_rn(v - off);
    }
};

// Arguments of the fused step kernel (one launch per time step).
template <typename C>
struct StepArgs {
    const void* src;        // P of the previous step
    void* dst;              // P written by this step
    const C* ux;
    const C* uy;
    const C* Dh;
    const C* S_cur;         // dt * S^n       (TRTR_SRC_FIELD)
    const C* S_prev;        // dt * S^{n-1}
    const C* tab_x;         // [2][pitch]: sin(pi x_i), cos(pi x_i)
    const C* tab_y;         // [2][ny]   : sin(pi y_j), cos(pi y_j)
    int nx, ny, pitch;
    size_t plane;           // ny * pitch
    int grad_mode;
    int tau2_fixed;
    C magic;                // Lambda
    C omega2_fixed;         // 1 / tau2 (TRTR_TAU2_FIXED)
    C tau1_const_dh;        // unused by the kernel (Dh holds it)
    C phi_ref;
    // pulse source (TRTR_SRC_PULSE), physical units
    C x0, y0, dx, dt;
    C dD_amp;               // D0 * D_amp
    C cx_n, cy_n, inv_s2_n, amp_n;     // at t_n
    C cx_p, cy_p, inv_s2_p, amp_p;     // at t_{n-1} (== t_n at the first step)
    int first_step;         // F^{-1} := F^0
};

}  // namespace trtr

struct trtr_ctx {
    trtr_params p;
    cudaStream_t stream;
    int device;
    int num_sms;
    int esize;        // bytes per stored population
    int csize;        // bytes per compute value (fields)
    int pitch;        // elements per row
    size_t plane;     // ny * pitch
    void* pop[2];
    int cur;          // index of the buffer holding P for the current step
    void* ux;
    void* uy;
    void* Dh;
    void* S[2];       // TRTR_SRC_FIELD buffers (dt * S)
    int S_cur;        // buffer holding S^n (-1: none set)
    int S_prev;       // buffer holding S^{n-1} (-1: use S^n)
    void* tab_x;
    void* tab_y;
    double* scratch;  // reduction partials
    int red_blocks;
    double* dres;     // device result of the reductions (4 doubles)
    double* hres;     // pinned host copy
    double* dtmp;     // device staging for double I/O
    size_t dtmp_len;  // in doubles
    bool fields_set, pulse_set, initialized;
    trtr::Pulse pulse;
    long step;
    long launches;
    char err[512];
};

namespace trtr {

// Launchers (defined in trtr_step.cu and trtr_aux.cu).  All enqueue on ctx->stream and
// return the cudaGetLastError() of the launch.
cudaError_t launch_step(trtr_ctx* ctx);
cudaError_t launch_convert_fields(trtr_ctx* ctx, const double* ux, const double* uy, const double* D);
cudaError_t launch_pulse_fields(trtr_ctx* ctx);
cudaError_t launch_convert_source(trtr_ctx* ctx, const double* S, void* dst);
cudaError_t launch_init_equilibrium(trtr_ctx* ctx, const double* phi0 /* device or NULL = pulse */);
cudaError_t launch_moments(trtr_ctx* ctx, double* phi_out_dev);
cudaError_t launch_reduce(trtr_ctx* ctx, int kind, const double* phi_ref_dev);
cudaError_t launch_get_populations(trtr_ctx* ctx, double* g_dev);
cudaError_t launch_set_populations(trtr_ctx* ctx, const double* g_dev);
cudaError_t launch_sample(trtr_ctx* ctx, const long* nodes_dev, int count, double* out_dev);

enum ReduceKind { kReduceMass = 0, kReducePulse = 1, kReduceField = 2, kReduceNonFinite = 3 };

PulseTime pulse_at(const Pulse& p, double t);

}  // namespace trtr
