// Allocation-free FP64 norms (lbps_norms_noalloc in include/lbps.h).
//
// Some callers cannot call cudaMalloc or cudaFree on their own:
//   - a serving loop that admits work against a fixed device-memory budget
//     and keeps all memory in its own pool (for example PyTorch's caching
//     allocator), where an allocation behind its back breaks the accounting
//     or fails once the pool holds the free memory;
//   - latency-sensitive loops where cudaFree (which waits for the device) or
//     a first-time allocation would stall the stream.
// lbps_norms needs a lattice, whose device block carries the reduction
// scratch.  This entry point reduces arrays the caller already holds and
// takes its scratch from a fixed array in this file instead, so it allocates
// nothing.  The paper has no counterpart; it is a service routine.
#include <cmath>

#include "lbps.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPointsPerThread = 16;
constexpr size_t kPointsPerBlock = (size_t)kThreads * kPointsPerThread;

// The shared scratch: one slot of 4 partial sums per block of the first pass,
// then the 4 results.  2 MiB + 32 B, held by every device that loads the
// library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[(LBPS_NOALLOC_MAX_BLOCKS + 1) * 4];

// max that keeps a NaN (fmax drops it)
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

__global__ void __launch_bounds__(kThreads) noalloc_partial_kernel(const double* __restrict__ x,
                                                                   const double* __restrict__ ref, size_t n,
                                                                   double* scratch) {
    __shared__ double sh[4][kThreads];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, mx = 0.0;
    size_t base = (size_t)blockIdx.x * kPointsPerBlock;
    for (int q = 0; q < kPointsPerThread; ++q) {
        size_t d = base + (size_t)q * kThreads + threadIdx.x;
        if (d < n) {
            double v = x[d];
            double r = ref ? ref[d] : 0.0;
            double e = v - r;
            s0 += e * e;
            s1 += r * r;
            s2 += v;
            mx = nan_max(mx, fabs(v));
        }
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    sh[3][threadIdx.x] = mx;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] = nan_max(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) scratch[(size_t)blockIdx.x * 4 + q] = sh[q][0];
}

// Reduces the nblk partial slots written by this call's first pass (every
// slot it reads was just overwritten, so the scratch needs no clearing) into
// the result slot after the last partial slot.
__global__ void __launch_bounds__(kThreads) noalloc_final_kernel(double* scratch, int nblk) {
    __shared__ double sh[4][kThreads];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += kThreads) {
        s[0] += scratch[(size_t)b * 4];
        s[1] += scratch[(size_t)b * 4 + 1];
        s[2] += scratch[(size_t)b * 4 + 2];
        s[3] = nan_max(s[3], scratch[(size_t)b * 4 + 3]);
    }
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] = nan_max(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) scratch[(size_t)LBPS_NOALLOC_MAX_BLOCKS * 4 + q] = sh[q][0];
}

// Device address of the scratch on the current device, looked up on every
// call (a lookup allocates nothing, and a cached address would go stale if
// the module were reloaded after a device reset).  The host-side name of the
// array is not a device address and is never passed to a kernel.
int scratch_for_current_device(double** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return LBPS_ERR_CUDA;
    }
    *out = static_cast<double*>(p);
    return LBPS_OK;
}

}  // namespace

extern "C" int lbps_norms_noalloc(const double* d_x, const double* d_ref, size_t n, void* cuda_stream,
                                  double out[4]) {
    if (!d_x || !out || n == 0) return LBPS_ERR_INVALID;
    if (n > LBPS_NOALLOC_MAX_POINTS) return LBPS_ERR_INVALID;  // more blocks than scratch slots
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    // the call ends with a copy into pageable host memory and a wait for the
    // stream, neither of which a capturing stream allows
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return LBPS_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return LBPS_ERR_INVALID;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != LBPS_OK) return rc;
    cudaGetLastError();  // an error left by earlier, unrelated work is not this call's
    int nblk = (int)((n + kPointsPerBlock - 1) / kPointsPerBlock);
    noalloc_partial_kernel<<<nblk, kThreads, 0, st>>>(d_x, d_ref, n, scratch);
    noalloc_final_kernel<<<1, kThreads, 0, st>>>(scratch, nblk);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, scratch + (size_t)LBPS_NOALLOC_MAX_BLOCKS * 4, 4 * sizeof(double),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LBPS_OK : LBPS_ERR_CUDA;
}
