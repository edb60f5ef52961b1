// trtr_noalloc.cu -- trtr_phi_sums_noalloc: the phi reductions over caller-owned
// populations without any device allocation.
//
// For callers that cannot allocate device memory.  The per-row partial sums live in a
// file-scope static __device__ array of TRTR_NOALLOC_MAX_ROWS triples (384 KiB), which
// every device that loads this library keeps until the process exits.  Host code never
// dereferences the array's name (on the host it is only a stand-in, not a device address):
// the first call on each device, with that device current, resolves the device address
// with cudaGetSymbolAddress and passes it to the kernels.
#include <mutex>

#include "trtr_internal.cuh"

namespace {

constexpr int kMaxRows = TRTR_NOALLOC_MAX_ROWS;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 256;

// One (sum phi, sum (phi - ref)^2, sum ref^2) triple per grid row.  Shared by every call on
// a device; each call writes rows [0, ny) before reading them, so nothing needs clearing.
static __device__ __align__(256) double g_row_partials[3 * kMaxRows];

std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum of three values; the result is valid in thread 0.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
    __shared__ double s[3][kThreads / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][w] = a;
        s[1][w] = b;
        s[2][w] = c;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < kThreads / 32 ? s[0][lane] : 0.0;
        b = lane < kThreads / 32 ? s[1][lane] : 0.0;
        c = lane < kThreads / 32 ? s[2][lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
    }
    __syncthreads();  // s is reused by the next row of the same block
}

// Row j: phi(i, j) = sum_q g[q][j][i]; partial sums of phi, (phi - ref)^2 and ref^2.
__global__ void __launch_bounds__(kThreads)
    row_sums_kernel(double* partials, const double* g, const double* ref, int nx, int ny) {
    const size_t n = (size_t)nx * (size_t)ny;
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = threadIdx.x; i < nx; i += kThreads) {
            const size_t k = (size_t)j * nx + i;
            double phi = 0.0;
#pragma unroll
            for (int q = 0; q < trtr::kQ; ++q) phi += g[q * n + k];
            a += phi;
            if (ref) {
                const double d = phi - ref[k];
                b += d * d;
                c += ref[k] * ref[k];
            }
        }
        block_sum3(a, b, c);
        if (threadIdx.x == 0) {
            partials[3 * j] = a;
            partials[3 * j + 1] = b;
            partials[3 * j + 2] = c;
        }
    }
}

__global__ void __launch_bounds__(kThreads) rows_finish_kernel(double* out, const double* partials, int ny) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < ny; j += kThreads) {
        a += partials[3 * j];
        b += partials[3 * j + 1];
        c += partials[3 * j + 2];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
}

// Device address of g_row_partials on the current device, looked up once per device and kept
// for the life of the process.  A cudaDeviceReset of that device (or any other end of its
// primary context) frees the static array and leaves the kept address stale.
cudaError_t partials_address(double** addr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *addr = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" trtr_status trtr_phi_sums_noalloc(const double* g, int nx, int ny, const double* phi_ref, double* out,
                                             void* cuda_stream) {
    if (!g || !out || nx < 1 || ny < 1) return TRTR_EINVAL;
    if (ny > kMaxRows) return TRTR_EINVAL;
    // An error left pending by earlier work of the caller is not this call's to take: report
    // it without clearing it and enqueue nothing.
    if (cudaPeekAtLastError() != cudaSuccess) return TRTR_ECUDA;
    double* partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) {
        cudaGetLastError();  // the lookup's own error (none was pending before it)
        return TRTR_ECUDA;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const int blocks = ny < 4096 ? ny : 4096;
    row_sums_kernel<<<blocks, kThreads, 0, stream>>>(partials, g, phi_ref, nx, ny);
    rows_finish_kernel<<<1, kThreads, 0, stream>>>(out, partials, ny);
    if (cudaGetLastError() != cudaSuccess) return TRTR_ECUDA;  // a launch error of this call
    return TRTR_OK;
}
