// Shared device helpers for the tFFR CUDA path: the spreading kernel, modular
// indexing and the padded shared-memory layout used by the FFT passes.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tffr {

constexpr int kFftNMax = 8192;          // largest oversampled side (M <= 4096)

__device__ __forceinline__ int wrapmod(int c, int n) {  // n is a power of two
    return c & (n - 1);
}

// floor(2v) and 2v - floor(2v) from the FP64 bit pattern, with integer
// operations only (FP64 arithmetic runs at a small fraction of the FP32 rate
// on this GPU).  The fraction is rounded to FP32 (it may round up to 1.0f,
// which places the sample on the next cell edge: the taps stay consistent).
// Returns false for |v| >= 2^28, infinities and NaN.
struct FineCoord {
    int cell;
    float frac;
    bool ok;
};
static __device__ __noinline__ FineCoord fine_coord_general(double v);

__device__ __forceinline__ bool fine_coord(double v, int& cell, float& frac) {
    // Fast path for 1 <= |2v| < 2^21 with 32-bit integer operations: the
    // significand is mh * 2^32 + lo (mh has 21 bits) and |2v| = m 2^-sh.
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int sh = 1074 - ((hi >> 20) & 0x7ff);
    if (sh >= 32 && sh <= 52) {
        const unsigned mh = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
        const int s = sh - 32;                                   // 0..20
        const unsigned I = mh >> s;
        const unsigned fh = mh & ((1u << s) - 1u);
        const float f = fmaf(__uint2float_rn(lo), __int_as_float((127 - sh) << 23),
                             __uint2float_rn(fh) * __int_as_float((127 - s) << 23));
        if (hi >= 0) {
            cell = (int)I;
            frac = f;
        } else if (f == 0.0f) {
            cell = -(int)I;
            frac = 0.0f;
        } else {
            cell = -(int)I - 1;
            frac = 1.0f - f;
        }
        return true;
    }
    const FineCoord g = fine_coord_general(v);
    cell = g.cell;
    frac = g.frac;
    return g.ok;
}

// floor(2v) alone (same rules as fine_coord, no offset).
__device__ __forceinline__ bool fine_cell(double v, int& cell) {
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int sh = 1074 - ((hi >> 20) & 0x7ff);
    if (sh >= 32 && sh <= 52) {
        const unsigned mh = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
        const int s = sh - 32;
        const unsigned I = mh >> s;
        const bool whole = ((mh & ((1u << s) - 1u)) | lo) == 0u;
        cell = (hi >= 0) ? (int)I : (whole ? -(int)I : -(int)I - 1);
        return true;
    }
    const FineCoord g = fine_coord_general(v);
    cell = g.cell;
    return g.ok;
}

// |v| < 2^28 and finite: the range fine_coord accepts.
__device__ __forceinline__ bool coord_in_range(double v) {
    return ((__double2hiint(v) >> 20) & 0x7ff) <= 1050;
}

// Any magnitude (see fine_coord): 64-bit integer operations.
static __device__ __noinline__ FineCoord fine_coord_general(double v) {
    int cell;
    float frac;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ffu);
    cell = 0;
    frac = 0.0f;
    if (e > 1050) return FineCoord{0, 0.0f, false};   // |v| >= 2^28 (also inf, NaN)
    if (e == 0) return FineCoord{0, 0.0f, true};      // zero or subnormal
    const bool neg = (b >> 63) != 0ull;
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = 1074 - e;                    // |2v| = m * 2^-sh, sh >= 24
    const unsigned long long I = (sh >= 64) ? 0ull : (m >> sh);
    const unsigned long long F = (sh >= 64) ? m : (m & ((1ull << sh) - 1ull));
    const float scale = (sh <= 126) ? __int_as_float((127 - sh) << 23) : 0.0f;
    if (!neg) {
        cell = (int)I;
        frac = __ull2float_rn(F) * scale;
    } else if (F == 0ull) {
        cell = -(int)I;
    } else {
        cell = -(int)I - 1;
        frac = (sh >= 64) ? 1.0f - __ull2float_rn(F) * scale : __ull2float_rn((1ull << sh) - F) * scale;
    }
    return FineCoord{cell, frac, true};
}

// floor(2v) and the fraction 2v - floor(2v) as a 32-bit fixed-point number
// (the fraction's leading 32 bits, truncated), without branches: the fast
// form covers 2^-11 <= |2v| < 2^21 with 32-bit integer operations and returns
// false for other magnitudes (cell and F are then meaningless), which
// fixed_coord_general covers (and returns false for a non-finite v or
// |v| >= 2^28).
static __device__ __noinline__ bool fixed_coord_general(double v, int& cell, unsigned& F);

__device__ __forceinline__ bool fixed_coord_fast(double v, int& cell, unsigned& F) {
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int sft = 1042 - ((hi >> 20) & 0x7ff);      // |2v| = (mh 2^32 + lo) 2^-(32 + sft)
    const unsigned mh = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
    const unsigned I = mh >> (sft & 31);
    const unsigned Fp = __funnelshift_r(lo, mh, (unsigned)sft);
    // negative v: 1 - fraction, the bits below the 32 kept ones borrowing one unit
    const unsigned tail = __funnelshift_lc(0u, lo, (unsigned)(32 - sft));
    const bool neg = hi < 0;
    cell = neg ? ((Fp | tail) ? ~(int)I : -(int)I) : (int)I;
    F = neg ? (tail ? ~Fp : 0u - Fp) : Fp;
    return (unsigned)sft <= 31u;
}

static __device__ __noinline__ bool fixed_coord_general(double v, int& cell, unsigned& F) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ffu);
    cell = 0;
    F = 0u;
    if (e > 1050) return false;                        // |v| >= 2^28 (also inf, NaN)
    if (e == 0) return true;                           // zero or subnormal
    const bool neg = (b >> 63) != 0ull;
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = 1074 - e;                           // |2v| = m 2^-sh, sh >= 24
    unsigned long long I, X;                           // integer part; fraction, sh bits (sh < 64)
    if (sh < 64) {
        I = m >> sh;
        X = m & ((1ull << sh) - 1ull);
    } else {
        I = 0ull;
        X = m;
    }
    if (neg && X != 0ull) {
        cell = -(int)I - 1;
        if (sh < 64) {
            X = (1ull << sh) - X;
        } else {
            // 1 - m 2^-sh, leading 32 bits: the complement of m's leading
            // bits, borrowing one unit when bits below them are set
            const int r = sh - 32;
            const unsigned long long top = (r < 64) ? (m >> r) : 0ull;
            const bool below = (r >= 64) || ((m & ((1ull << r) - 1ull)) != 0ull);
            F = below ? ~(unsigned)top : 0u - (unsigned)top;
            return true;
        }
    } else {
        cell = neg ? -(int)I : (int)I;
        if (sh >= 64) {
            const int r = sh - 32;
            F = (r < 64) ? (unsigned)(m >> r) : 0u;
            return true;
        }
    }
    F = (sh >= 32) ? (unsigned)(X >> (sh - 32)) : (unsigned)(X << (32 - sh));
    return true;
}

// Spreading-kernel taps as polynomials in t = 2f - 1 (f the fine-cell offset
// in [0, 1]): tap s (fine cell floor(u) - (w/2 - 1) + s) has weight
// P_s(t) = sum_k c[s][k] t^k, fitted at plan time in FP64 to the ES kernel
// phi(s - (w/2 - 1) - f).  phi is even, so P_{w-1-s}(t) = P_s(-t).  The fit
// stops at the kernel's own floor, the jump e^{-beta} at the edge of its
// support (1e-6 at w = 6): degree 7 for w <= 6 reaches it (1.6e-6 against
// 1.5e-6 at degree 10), w = 8 needs degree 8 (1.6e-8).  Coefficients past the
// fitted degree are zero.
constexpr int kTapCoefs = 11;                   // storage (degree <= 10)
__host__ __device__ constexpr int tap_coefs(int w) { return w <= 6 ? 8 : 9; }
struct TapPoly {
    float c[8][kTapCoefs];
};

__device__ __forceinline__ float tap_eval(const TapPoly& P, int s, float t) {
    float a = P.c[s][kTapCoefs - 1];
#pragma unroll
    for (int k = kTapCoefs - 2; k >= 0; --k) a = fmaf(a, t, P.c[s][k]);
    return a;
}

// All W taps; mirrored pairs share the even and odd parts in t^2.
template <int W>
__device__ __forceinline__ void taps_all_t(const TapPoly& P, float t, float (&wt)[W]) {
    constexpr int NC = tap_coefs(W);
    constexpr int TOP_E = (NC - 1) & ~1, TOP_O = ((NC - 2) | 1);        // highest even / odd power
    const float t2 = t * t;
#pragma unroll
    for (int s = 0; s < W / 2; ++s) {
        float e = P.c[s][TOP_E];
#pragma unroll
        for (int k = TOP_E - 2; k >= 0; k -= 2) e = fmaf(e, t2, P.c[s][k]);
        float o = P.c[s][TOP_O];
#pragma unroll
        for (int k = TOP_O - 2; k >= 1; k -= 2) o = fmaf(o, t2, P.c[s][k]);
        wt[s] = fmaf(t, o, e);
        wt[W - 1 - s] = fmaf(-t, o, e);
    }
}

template <int W>
__device__ __forceinline__ void taps_all(const TapPoly& P, float f, float (&wt)[W]) {
    taps_all_t<W>(P, 2.0f * f - 1.0f, wt);
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
// Complex add and subtract as one paired FP32 instruction each (add / sub
// .rn.f32x2 on the register pair): the same IEEE rounding per component, half
// the issue slots of two scalar operations.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    float2 r;
    asm("{ .reg .b64 x, y, z; mov.b64 x, {%2, %3}; mov.b64 y, {%4, %5}; add.rn.f32x2 z, x, y; mov.b64 {%0, %1}, z; }"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    float2 r;
    asm("{ .reg .b64 x, y, z; mov.b64 x, {%2, %3}; mov.b64 y, {%4, %5}; sub.rn.f32x2 z, x, y; mov.b64 {%0, %1}, z; }"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// p points into shared memory: two reductions (no value returned).
__device__ __forceinline__ void atomic_add_f2_shared(float2* p, float2 v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v.x) : "memory");
    asm volatile("red.shared.add.f32 [%0+4], %1;" ::"r"(a), "f"(v.y) : "memory");
}

// cp.async of one element (4, 8 or 16 bytes) from global into shared memory.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace tffr
