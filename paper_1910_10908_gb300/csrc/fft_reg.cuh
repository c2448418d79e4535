// Block-wide complex FFT of one line of n = 2^logn points (32 <= n <= 8192),
//
//     X[k] = sum_{j<n} x[j] exp(sgn * 2 pi i j k / n),   sgn = +1 or -1,
//
// computed by T = n / V threads that each hold V points in registers
// (Stockham autosort; stages of radix V, then one smaller radix for the rest).
// Between stages the line goes through padded shared memory (one spare slot
// per V points, which keeps the strided stores of the first stage on distinct
// banks).  Inner DFTs of radix 2..32 are unrolled with constant roots of
// unity; the inter-stage twiddles exp(2 pi i m / n) come from a two-level
// table (exp(2 pi i 64 h / n) * exp(2 pi i l / n), m = 64 h + l) staged in
// shared memory, both levels built in FP64 on the host.
#pragma once

#include "common.cuh"

namespace tffr {

// cos and sin of 2 pi m / 32
__device__ __forceinline__ float w32c(int m) {
    constexpr float c[32] = {
        1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f, 7.071067812e-01f,
        5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f, 0.0f, -1.950903220e-01f, -3.826834324e-01f,
        -5.555702330e-01f, -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
        -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f, -7.071067812e-01f,
        -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f, 0.0f, 1.950903220e-01f, 3.826834324e-01f,
        5.555702330e-01f, 7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f};
    return c[m & 31];
}
__device__ __forceinline__ float w32s(int m) { return w32c(m - 8); }   // sin x = cos(x - pi/2)

// z * exp(sgn * 2 pi i m / 32) for a compile-time m
template <int M>
__device__ __forceinline__ float2 rot32(float2 z, float sgn) {
    constexpr int m = M & 31;
    if (m == 0) return z;
    if (m == 8) return make_float2(-sgn * z.y, sgn * z.x);
    if (m == 16) return make_float2(-z.x, -z.y);
    if (m == 24) return make_float2(sgn * z.y, -sgn * z.x);
    const float c = w32c(m), s = sgn * w32s(m);
    return make_float2(z.x * c - z.y * s, z.x * s + z.y * c);
}

template <int R> struct Dft;

template <> struct Dft<1> {
    static __device__ __forceinline__ void run(float2*, float) {}
};

template <> struct Dft<2> {
    static __device__ __forceinline__ void run(float2* v, float) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <> struct Dft<4> {
    static __device__ __forceinline__ void run(float2* v, float sgn) {
        const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const float2 c = cadd(v[1], v[3]);
        const float2 d = rot32<8>(csub(v[1], v[3]), sgn);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};

// radix 2 x radix R/2 split: X[k] = E[k] + w^k O[k], X[k + R/2] = E[k] - w^k O[k]
template <int R>
__device__ __forceinline__ void dft_split2(float2* v, float sgn) {
    constexpr int H = R / 2;
    float2 e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    Dft<H>::run(e, sgn);
    Dft<H>::run(o, sgn);
#pragma unroll
    for (int k = 0; k < H; ++k) {
        float2 t;
        if (R == 8) {
            t = (k == 0) ? o[k] : (k == 1) ? rot32<4>(o[k], sgn) : (k == 2) ? rot32<8>(o[k], sgn) : rot32<12>(o[k], sgn);
        } else if (R == 16) {
            switch (k) {
                case 0: t = o[0]; break;
                case 1: t = rot32<2>(o[1], sgn); break;
                case 2: t = rot32<4>(o[2], sgn); break;
                case 3: t = rot32<6>(o[3], sgn); break;
                case 4: t = rot32<8>(o[4], sgn); break;
                case 5: t = rot32<10>(o[5], sgn); break;
                case 6: t = rot32<12>(o[6], sgn); break;
                default: t = rot32<14>(o[7], sgn); break;
            }
        } else {
            switch (k) {
                case 0: t = o[0]; break;
                case 1: t = rot32<1>(o[1], sgn); break;
                case 2: t = rot32<2>(o[2], sgn); break;
                case 3: t = rot32<3>(o[3], sgn); break;
                case 4: t = rot32<4>(o[4], sgn); break;
                case 5: t = rot32<5>(o[5], sgn); break;
                case 6: t = rot32<6>(o[6], sgn); break;
                case 7: t = rot32<7>(o[7], sgn); break;
                case 8: t = rot32<8>(o[8], sgn); break;
                case 9: t = rot32<9>(o[9], sgn); break;
                case 10: t = rot32<10>(o[10], sgn); break;
                case 11: t = rot32<11>(o[11], sgn); break;
                case 12: t = rot32<12>(o[12], sgn); break;
                case 13: t = rot32<13>(o[13], sgn); break;
                case 14: t = rot32<14>(o[14], sgn); break;
                default: t = rot32<15>(o[15], sgn); break;
            }
        }
        v[k] = cadd(e[k], t);
        v[k + H] = csub(e[k], t);
    }
}

template <> struct Dft<8> {
    static __device__ __forceinline__ void run(float2* v, float sgn) { dft_split2<8>(v, sgn); }
};
template <> struct Dft<16> {
    static __device__ __forceinline__ void run(float2* v, float sgn) { dft_split2<16>(v, sgn); }
};
template <> struct Dft<32> {
    static __device__ __forceinline__ void run(float2* v, float sgn) { dft_split2<32>(v, sgn); }
};

// Stage plan: radix V stages first, then one stage of radix 2^(logn mod log2 V).
struct LineFft {
    int n, logn;
    const float2* twh;      // shared: exp(2 pi i 64 h / n), h < max(1, n/64)
    const float2* twl;      // shared: exp(2 pi i l / n), l < min(64, n)
    float sgn;
};

__device__ __forceinline__ float2 twiddle(const LineFft& L, int m) {
    return cmul(L.twh[m >> 6], L.twl[m & 63]);
}

template <int V>
__device__ __forceinline__ int fft_pad(int i) {
    constexpr int S = (V >= 32) ? 5 : (V >= 16) ? 4 : (V >= 8) ? 3 : (V >= 4) ? 2 : 1;
    return i + (i >> S);
}

template <int V>
__host__ __device__ constexpr int fft_pad_len(int n) {
    return n + n / (V >= 32 ? 32 : V >= 16 ? 16 : V >= 8 ? 8 : V >= 4 ? 4 : 2) + 1;
}

// Registers v hold the stage input in the pattern v[b*R + r] = x[j_b + r n/R],
// j_b = tid + b T (T = n / V threads, B = V / R butterflies each).  Apply the
// stage's twiddles and DFTs in place.
template <int V, int R, int LOGR>
__device__ __forceinline__ void stage_compute(float2 (&v)[V], const LineFft& L, int logNs) {
    constexpr int B = V / R;
    const int T = L.n / V;
    const int Ns = 1 << logNs;
    const int tshift = L.logn - logNs - LOGR;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = threadIdx.x + b * T;
        const int k = j & (Ns - 1);
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 t = twiddle(L, (r * k) << tshift);
                t.y *= L.sgn;
                v[b * R + r] = cmul(v[b * R + r], t);
            }
        }
        Dft<R>::run(&v[b * R], L.sgn);
    }
}

template <int V, int R>
__device__ __forceinline__ void stage_load(float2 (&v)[V], const float2* buf, int n) {
    constexpr int B = V / R;
    const int T = n / V;
    const int stride = n / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = buf[fft_pad<V>(threadIdx.x + b * T + r * stride)];
}

template <int V, int R, int LOGR>
__device__ __forceinline__ void stage_store(const float2 (&v)[V], float2* buf, int n, int logNs) {
    constexpr int B = V / R;
    const int T = n / V;
    const int Ns = 1 << logNs;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = threadIdx.x + b * T;
        const int k = j & (Ns - 1);
        const int base = ((j - k) << LOGR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[fft_pad<V>(base + r * Ns)] = v[b * R + r];
    }
}

// One full radix-R stage in shared memory: load, sync, compute, store, sync.
template <int V, int R, int LOGR>
__device__ __forceinline__ void stage_smem(float2* buf, const LineFft& L, int logNs) {
    float2 v[V];
    stage_load<V, R>(v, buf, L.n);
    __syncthreads();
    stage_compute<V, R, LOGR>(v, L, logNs);
    stage_store<V, R, LOGR>(v, buf, L.n, logNs);
    __syncthreads();
}

template <int V> struct LogOf;
template <> struct LogOf<2> { static constexpr int v = 1; };
template <> struct LogOf<4> { static constexpr int v = 2; };
template <> struct LogOf<8> { static constexpr int v = 3; };
template <> struct LogOf<16> { static constexpr int v = 4; };
template <> struct LogOf<32> { static constexpr int v = 5; };

// Remainder stage of radix 2^rem < V, dispatched at run time.
template <int V>
__device__ __forceinline__ void stage_rem_smem(float2* buf, const LineFft& L, int logNs, int rem) {
    switch (rem) {
        case 1: stage_smem<V, 2, 1>(buf, L, logNs); break;
        case 2: if constexpr (V >= 4) stage_smem<V, 4, 2>(buf, L, logNs); break;
        case 3: if constexpr (V >= 8) stage_smem<V, 8, 3>(buf, L, logNs); break;
        case 4: if constexpr (V >= 16) stage_smem<V, 16, 4>(buf, L, logNs); break;
        default: break;
    }
}

// Whole FFT in shared memory (buf indexed with fft_pad<V>); the caller has
// synchronised after filling buf, and buf holds the result, in natural order,
// after the call (which ends with a barrier).
template <int V>
__device__ __forceinline__ void fft_line_smem(float2* buf, const LineFft& L) {
    constexpr int LV = LogOf<V>::v;
    int logNs = 0;
    while (logNs + LV <= L.logn) {
        stage_smem<V, V, LV>(buf, L, logNs);
        logNs += LV;
    }
    if (logNs < L.logn) stage_rem_smem<V>(buf, L, logNs, L.logn - logNs);
}

// Load the two-level twiddle table of an n-point line into shared memory.
__device__ __forceinline__ void load_twiddles(float2* s_twh, float2* s_twl, const float2* __restrict__ twh,
                                              const float2* __restrict__ twl, int n) {
    const int nh = n >= 64 ? n / 64 : 1;
    const int nl = n >= 64 ? 64 : n;
    for (int i = threadIdx.x; i < nh; i += blockDim.x) s_twh[i] = twh[i];
    for (int i = threadIdx.x; i < nl; i += blockDim.x) s_twl[i] = twl[i];
}

}  // namespace tffr
