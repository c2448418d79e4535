// Shared device helpers for the tFFR CUDA path: the spreading kernel, modular
// indexing and the padded shared-memory layout used by the FFT passes.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tffr {

constexpr int kFftThreads = 512;        // threads of every FFT-pass CTA
constexpr int kFftNMax = 8192;          // largest oversampled side (M <= 4096)
constexpr int kColGroup = 16;           // x-modes per 128-byte line of the intermediate

// Padded shared-memory index: one spare float2 every 16 keeps the strided
// butterfly stores of the early Stockham stages off the same banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

__device__ __forceinline__ int wrapmod(int c, int n) {  // n is a power of two
    return c & (n - 1);
}

// Exponential-of-semicircle spreading kernel of width w (fine-grid cells):
//   phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)) for |z| < w/2, 0 otherwise.
__device__ __forceinline__ float es_kernel(float z, float beta, float two_over_w) {
    const float x = z * two_over_w;
    const float t = 1.0f - x * x;
    return t > 0.0f ? expf(beta * (sqrtf(t) - 1.0f)) : 0.0f;
}

// Sample-value loads for each storage type, returned as FP32 complex.
template <typename VT> struct ValueIO;
template <> struct ValueIO<float2> {
    static __device__ __forceinline__ float2 load(const void* p, int64_t i) {
        return __ldg(reinterpret_cast<const float2*>(p) + i);
    }
    static __device__ __forceinline__ void store(void* p, int64_t i, float2 v) {
        reinterpret_cast<float2*>(p)[i] = v;
    }
};
template <> struct ValueIO<double2> {
    static __device__ __forceinline__ float2 load(const void* p, int64_t i) {
        const double2 d = __ldg(reinterpret_cast<const double2*>(p) + i);
        return make_float2((float)d.x, (float)d.y);
    }
    static __device__ __forceinline__ void store(void* p, int64_t i, float2 v) {
        reinterpret_cast<double2*>(p)[i] = make_double2((double)v.x, (double)v.y);
    }
};
template <> struct ValueIO<__half2> {
    static __device__ __forceinline__ float2 load(const void* p, int64_t i) {
        return __half22float2(reinterpret_cast<const __half2*>(p)[i]);
    }
    static __device__ __forceinline__ void store(void* p, int64_t i, float2 v) {
        reinterpret_cast<float2*>(p)[i] = v;   // forward output stays complex64
    }
};
template <> struct ValueIO<__nv_bfloat162> {
    static __device__ __forceinline__ float2 load(const void* p, int64_t i) {
        return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(p)[i]);
    }
    static __device__ __forceinline__ void store(void* p, int64_t i, float2 v) {
        reinterpret_cast<float2*>(p)[i] = v;   // forward output stays complex64
    }
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ void atomic_add_f2_shared(float2* p, float2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

}  // namespace tffr
