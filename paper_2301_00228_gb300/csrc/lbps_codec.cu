// The 16-bit storage formats' value codec on caller-owned device arrays
// (lbps_codec16 in include/lbps.h).  The kernels below call the same
// conversion routines the time step stores and loads the pair sums with
// (bits2f, f2bits_store, bfp13_encode, bfp13_decode in lbps_device.cuh), so
// a caller can inspect stored codes, and a test can check every code of a
// format against the format's definition.  The paper has no counterpart; it
// is a service routine.
#include "lbps.h"
#include "lbps_device.cuh"

namespace {

constexpr int kThreads = 256;

template <typename H>
__global__ void __launch_bounds__(kThreads) encode_kernel(const float* __restrict__ x, uint16_t* __restrict__ code,
                                                          int64_t n, unsigned key0, bool sr) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        // the key a point at plane offset i has for its slot 0 (PopNeq16::key_of)
        code[i] = (uint16_t)lbps::f2bits_store<H>(x[i], (unsigned)i * 4u + key0, sr);
}

template <typename H>
__global__ void __launch_bounds__(kThreads) decode_kernel(const uint16_t* __restrict__ code, float* __restrict__ x,
                                                          int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        x[i] = lbps::bits2f<H>(code[i]);
}

// BFP13: value pairs (x[2i], x[2i+1]) <-> the 32-bit word at code[2i]
__global__ void __launch_bounds__(kThreads) bfp13_encode_kernel(const float2* __restrict__ x,
                                                                unsigned* __restrict__ word, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const float2 v = x[i];
        word[i] = lbps::bfp13_encode(v.x, v.y);
    }
}

__global__ void __launch_bounds__(kThreads) bfp13_decode_kernel(const unsigned* __restrict__ word,
                                                                float2* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        float2 v;
        lbps::bfp13_decode(word[i], v.x, v.y);
        x[i] = v;
    }
}

unsigned grid_for(int64_t n) {
    const int64_t want = (n + kThreads - 1) / kThreads;
    return (unsigned)(want < 152 * 16 ? want : 152 * 16);
}

template <typename H>
cudaError_t run(int32_t encode, float* x, uint16_t* code, int64_t n, unsigned key0, bool sr, cudaStream_t st) {
    const unsigned blocks = grid_for(n);
    if (encode)
        encode_kernel<H><<<blocks, kThreads, 0, st>>>(x, code, n, key0, sr);
    else
        decode_kernel<H><<<blocks, kThreads, 0, st>>>(code, x, n);
    return cudaGetLastError();
}

}  // namespace

extern "C" int lbps_codec16(int32_t storage, int32_t encode, float* d_x, uint16_t* d_code, int64_t n,
                            uint32_t key0, int32_t stochastic, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!d_x || !d_code)) || (encode != 0 && encode != 1) ||
        (stochastic != 0 && stochastic != 1))
        return LBPS_ERR_INVALID;
    if (storage != LBPS_STORAGE_BF16 && storage != LBPS_STORAGE_F16 && storage != LBPS_STORAGE_BFP13)
        return LBPS_ERR_INVALID;
    if (storage == LBPS_STORAGE_BFP13 &&
        (n % 2 != 0 || reinterpret_cast<uintptr_t>(d_x) % 8 != 0 || reinterpret_cast<uintptr_t>(d_code) % 4 != 0))
        return LBPS_ERR_INVALID;
    if (n == 0) return LBPS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bool sr = stochastic != 0;
    cudaError_t e;
    if (storage == LBPS_STORAGE_BF16) {
        e = run<__nv_bfloat16>(encode, d_x, d_code, n, key0, sr, st);
    } else if (storage == LBPS_STORAGE_F16) {
        e = run<__half>(encode, d_x, d_code, n, key0, sr, st);
    } else {
        const int64_t pairs = n / 2;
        float2* x2 = reinterpret_cast<float2*>(d_x);
        unsigned* w = reinterpret_cast<unsigned*>(d_code);
        if (encode)
            bfp13_encode_kernel<<<grid_for(pairs), kThreads, 0, st>>>(x2, w, pairs);
        else
            bfp13_decode_kernel<<<grid_for(pairs), kThreads, 0, st>>>(w, x2, pairs);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? LBPS_OK : LBPS_ERR_CUDA;
}
