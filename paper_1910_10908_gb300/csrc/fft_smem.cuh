// Block-wide complex FFT of a power-of-two length n <= 8192 held in padded
// shared memory (Stockham autosort, radix-8 stages plus one radix-2 or radix-4
// stage), computed by kFftThreads threads:
//
//     X[k] = sum_{j<n} x[j] exp(sgn * 2 pi i j k / n),   sgn = +1 or -1.
//
// Each stage reads every butterfly's inputs into registers, synchronises and
// writes the outputs back in place.  Twiddles come from tw[m] = exp(+2 pi i m / n),
// a table built in FP64 on the host (conjugated for sgn = -1).
#pragma once

#include "common.cuh"

namespace tffr {

template <int R> struct SmallDft;

template <> struct SmallDft<2> {
    static __device__ __forceinline__ void run(float2 (&v)[2], float) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

// multiply by sgn * i
__device__ __forceinline__ float2 mul_si(float2 z, float sgn) { return make_float2(-sgn * z.y, sgn * z.x); }

template <> struct SmallDft<4> {
    static __device__ __forceinline__ void run(float2 (&v)[4], float sgn) {
        const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const float2 c = cadd(v[1], v[3]), d = mul_si(csub(v[1], v[3]), sgn);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};

template <> struct SmallDft<8> {
    static __device__ __forceinline__ void run(float2 (&v)[8], float sgn) {
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        SmallDft<4>::run(e, sgn);
        SmallDft<4>::run(o, sgn);
        const float h = 0.70710678118654752440f;
        // w^k o[k], w = exp(sgn * 2 pi i / 8)
        const float2 o1 = make_float2(h * (o[1].x - sgn * o[1].y), h * (o[1].y + sgn * o[1].x));
        const float2 o2 = mul_si(o[2], sgn);
        const float2 o3 = make_float2(h * (-o[3].x - sgn * o[3].y), h * (-o[3].y + sgn * o[3].x));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <int R, int LOGR>
__device__ __forceinline__ void fft_stage(float2* buf, int n, int logn, int logNs,
                                          const float2* __restrict__ tw, float sgn) {
    constexpr int BPT = (kFftNMax / R) / kFftThreads;
    const int nb = n >> LOGR;
    const int Ns = 1 << logNs;
    const int tshift = logn - logNs - LOGR;       // twiddle stride n / (Ns R)
    const int tid = threadIdx.x;
    float2 v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = tid + b * kFftThreads;
        if (j < nb) {
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = buf[pad16(j + r * nb)];
            if (k != 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 t = __ldg(&tw[(r * k) << tshift]);
                    t.y *= sgn;
                    v[b][r] = cmul(v[b][r], t);
                }
            }
            SmallDft<R>::run(v[b], sgn);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = tid + b * kFftThreads;
        if (j < nb) {
            const int k = j & (Ns - 1);
            const int dst = ((j - k) << LOGR) + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[pad16(dst + r * Ns)] = v[b][r];
        }
    }
    __syncthreads();
}

// In-place FFT of buf[pad16(0..n-1)]; n = 2^logn, 2 <= n <= kFftNMax.
__device__ __forceinline__ void fft_smem(float2* buf, int n, int logn, const float2* __restrict__ tw,
                                         float sgn) {
    __syncthreads();
    int logNs = 0;
    const int rem = logn % 3;
    if (rem == 1) {
        fft_stage<2, 1>(buf, n, logn, 0, tw, sgn);
        logNs = 1;
    } else if (rem == 2) {
        fft_stage<4, 2>(buf, n, logn, 0, tw, sgn);
        logNs = 2;
    }
    while (logNs < logn) {
        fft_stage<8, 3>(buf, n, logn, logNs, tw, sgn);
        logNs += 3;
    }
}

}  // namespace tffr
