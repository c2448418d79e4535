// Block-wide complex FFT of one line of N = 2^LOGN points (32 <= N <= 8192),
//
//     X[k] = sum_{j<N} x[j] exp(sgn * 2 pi i j k / N),   sgn = +1 or -1,
//
// computed by T = N / V threads that each hold V points in registers
// (Stockham autosort: stages of radix V, then one smaller radix for the
// rest).  Between stages the line goes through padded shared memory (one
// spare slot per V points keeps the strided stores of the first stage on
// distinct banks).  The line length is a template parameter, so every index,
// stride and twiddle shift is a compile-time constant.  Inner DFTs of radix
// 2..32 are unrolled with constant roots of unity; the inter-stage twiddles
// exp(2 pi i m / N) come from a two-level table (exp(2 pi i 64 h / N) *
// exp(2 pi i l / N), m = 64 h + l) or, for the stages whose twiddles are
// 1024-th roots of unity, from a direct table; all tables are built in FP64 on
// the host and staged in shared memory.
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

// z * exp(SGN * 2 pi i m / 32) for a compile-time m
template <int M, int SGN>
__device__ __forceinline__ float2 rot32(float2 z) {
    constexpr int m = M & 31;
    if (m == 0) return z;
    if (m == 8) return SGN > 0 ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
    if (m == 16) return make_float2(-z.x, -z.y);
    if (m == 24) return SGN > 0 ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
    const float c = w32c(m), s = (SGN > 0) ? w32s(m) : -w32s(m);
    return make_float2(z.x * c - z.y * s, z.x * s + z.y * c);
}

template <int R> struct Dft;

template <> struct Dft<1> {
    template <int SGN>
    static __device__ __forceinline__ void run(float2*) {}
};

template <> struct Dft<2> {
    template <int SGN>
    static __device__ __forceinline__ void run(float2* v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <> struct Dft<4> {
    template <int SGN>
    static __device__ __forceinline__ void run(float2* v) {
        const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const float2 c = cadd(v[1], v[3]);
        const float2 d = rot32<8, SGN>(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};

template <int R, int K, int SGN>
struct Combine {
    static __device__ __forceinline__ void run(float2* v, const float2* e, const float2* o) {
        const float2 t = rot32<(32 / R) * K, SGN>(o[K]);     // w^K O[K], w = exp(SGN 2 pi i / R)
        v[K] = cadd(e[K], t);
        v[K + R / 2] = csub(e[K], t);
        Combine<R, K + 1, SGN>::run(v, e, o);
    }
};
template <int R, int SGN>
struct Combine<R, R / 2, SGN> {
    static __device__ __forceinline__ void run(float2*, const float2*, const float2*) {}
};

// radix 2 x radix R/2 split: X[k] = E[k] + w^k O[k], X[k + R/2] = E[k] - w^k O[k]
template <int R, int SGN>
__device__ __forceinline__ void dft_split2(float2* v) {
    constexpr int H = R / 2;
    float2 e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    Dft<H>::template run<SGN>(e);
    Dft<H>::template run<SGN>(o);
    Combine<R, 0, SGN>::run(v, e, o);
}

template <> struct Dft<8> {
    template <int SGN>
    static __device__ __forceinline__ void run(float2* v) { dft_split2<8, SGN>(v); }
};
template <> struct Dft<16> {
    template <int SGN>
    static __device__ __forceinline__ void run(float2* v) { dft_split2<16, SGN>(v); }
};
template <> struct Dft<32> {
    template <int SGN>
    static __device__ __forceinline__ void run(float2* v) { dft_split2<32, SGN>(v); }
};

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// z * exp(SGN * 2 pi i m / 32), m known once the caller's loops are unrolled.
template <int SGN>
__device__ __forceinline__ float2 rot32_folded(float2 z, int m) {
    m &= 31;
    if (m == 0) return z;
    if (m == 8) return SGN > 0 ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
    if (m == 16) return make_float2(-z.x, -z.y);
    if (m == 24) return SGN > 0 ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
    const float c = w32c(m), s = (SGN > 0) ? w32s(m) : -w32s(m);
    return make_float2(z.x * c - z.y * s, z.x * s + z.y * c);
}

// The first radix-V stage (which has no twiddles) of a line whose points
// x[tid + u T] are zero for u >= U: the V-point DFT of (x_0, .., x_{U-1}, 0, ..)
// splits by output residue b = k mod (V / U) into U-point DFTs,
//     X[(V/U) q + b] = sum_{u<U} (x_u W_V^{u b}) W_U^{u q},
// with constant twiddles W_V^{u b}.  v[u] holds x_u on entry (u < U) and
// X[k] in v[k] on return, as the full radix-V stage leaves it.
template <int V, int U, int SGN>
__device__ __forceinline__ void dft_first_sparse(float2 (&v)[V]) {
    constexpr int G = V / U;
    float2 x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = v[u];
#pragma unroll
    for (int b = 0; b < G; ++b) {
        float2 y[U];
#pragma unroll
        for (int u = 0; u < U; ++u) y[u] = rot32_folded<SGN>(x[u], (32 / V) * u * b);
        Dft<U>::template run<SGN>(y);
#pragma unroll
        for (int q = 0; q < U; ++q) v[G * q + b] = y[q];
    }
}

// Values per thread for an N-point line.
__host__ __device__ constexpr int line_v(int n) {
    return n >= 8192 ? 32 : n >= 512 ? 16 : n >= 256 ? 8 : n >= 128 ? 4 : 2;
}

template <int LOGN>
struct Line {
    static constexpr int N = 1 << LOGN;
    static constexpr int V = line_v(N);
    static constexpr int LV = ilog2c(V);
    static constexpr int T = N / V;                       // threads
    static constexpr int NFULL = LOGN / LV;               // radix-V stages
    static constexpr int REM = LOGN - NFULL * LV;         // log2 of the last radix (0: none)
    static constexpr int PADLEN = N + N / V + 1;          // padded shared line
    static constexpr int NH = N >= 64 ? N / 64 : 1;       // twiddle table levels
    static constexpr int NL = N >= 64 ? 64 : N;
    static constexpr int NT = N >= 1024 ? 1024 : N;       // direct table of the NT-th roots of unity
    static constexpr int NT2 = V == 16 ? 256 : 0;         // transposed 16 x 16 roots (see load_twiddles)
    static constexpr int SMEM_ELEMS = PADLEN + 128 + 64 + 1024 + NT2;
    __device__ __forceinline__ static int pad(int i) { return i + (i >> LV); }
};

struct Twiddles {
    const float2* h;        // shared: exp(2 pi i 64 h / N)
    const float2* l;        // shared: exp(2 pi i l / N)
    const float2* t;        // shared: exp(2 pi i m / NT), NT = min(N, 1024)
    const float2* t2;       // shared (16 values a thread): exp(2 pi i r k / 256) at 16 r + k
    __device__ __forceinline__ float2 operator()(int m) const { return cmul(h[m >> 6], l[m & 63]); }
};

template <int SGN>
__device__ __forceinline__ float2 conj_if(float2 w) {
    return SGN > 0 ? w : make_float2(w.x, -w.y);
}

// Registers v hold the stage input as v[b*R + r] = x[j_b + r N/R], j_b = tid + b T
// (B = V / R butterflies per thread).  Apply twiddles W_{NS R}^{SGN r k}
// (k = j_b mod NS) and the radix-R DFTs in place.  When NS R divides 1024 the
// twiddles come straight from the table of 1024-th roots; otherwise
// w = W_{NS R}^k comes from the two-level table and w^r from a product tree
// (w^{2i} = (w^i)^2, w^{2i+1} = w^{2i} w: at most five products deep).
template <int LOGN, int R, int LOGNS, int SGN>
__device__ __forceinline__ void stage_compute(float2 (&v)[Line<LOGN>::V], const Twiddles& tw) {
    using L = Line<LOGN>;
    constexpr int B = L::V / R;
    constexpr int NS = 1 << LOGNS;
    constexpr int LOGR = ilog2c(R);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if constexpr (NS > 1) {
            const int k = (threadIdx.x + b * L::T) & (NS - 1);
            if constexpr (NS * R <= L::NT) {
                if constexpr (L::V == 32) {
                    // the transposed table (load_twiddles): entry r 32 + k = W_1024^(r k)
                    static_assert(NS == 32 && R == 32, "the transposed direct table serves NS = R = 32 only");
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        v[b * R + r] = cmul(v[b * R + r], conj_if<SGN>(tw.t[r * 32 + k]));
                } else if constexpr (L::V == 16 && NS == 16 && R == 16) {
                    // the transposed 16 x 16 table (load_twiddles): entry r 16 + k = W_256^(r k)
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        v[b * R + r] = cmul(v[b * R + r], conj_if<SGN>(tw.t2[r * 16 + k]));
                } else {
                    constexpr int TS = ilog2c(L::NT) - LOGNS - LOGR;     // W_{NS R} = W_NT^(2^TS)
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        v[b * R + r] = cmul(v[b * R + r], conj_if<SGN>(tw.t[(r * k) << TS]));
                }
            } else {
                constexpr int TSHIFT = LOGN - LOGNS - LOGR;
                float2 p[R];
                p[1] = conj_if<SGN>(tw(k << TSHIFT));
#pragma unroll
                for (int r = 2; r < R; ++r) p[r] = (r & 1) ? cmul(p[r - 1], p[1]) : cmul(p[r / 2], p[r / 2]);
#pragma unroll
                for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], p[r]);
            }
        }
        Dft<R>::template run<SGN>(&v[b * R]);
    }
}

template <int LOGN, int R>
__device__ __forceinline__ void stage_load(float2 (&v)[Line<LOGN>::V], const float2* buf) {
    using L = Line<LOGN>;
    constexpr int B = L::V / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = buf[L::pad(threadIdx.x + b * L::T + r * (L::N / R))];
}

template <int LOGN, int R, int LOGNS>
__device__ __forceinline__ void stage_store(const float2 (&v)[Line<LOGN>::V], float2* buf) {
    using L = Line<LOGN>;
    constexpr int B = L::V / R;
    constexpr int NS = 1 << LOGNS;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = threadIdx.x + b * L::T;
        const int k = j & (NS - 1);
        const int base = ((j - k) * R) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[L::pad(base + r * NS)] = v[b * R + r];
    }
}

// One full stage in shared memory: load, sync, compute, store, sync.
template <int LOGN, int R, int LOGNS, int SGN>
__device__ __forceinline__ void stage_smem(float2* buf, const Twiddles& tw) {
    float2 v[Line<LOGN>::V];
    stage_load<LOGN, R>(v, buf);
    __syncthreads();
    stage_compute<LOGN, R, LOGNS, SGN>(v, tw);
    stage_store<LOGN, R, LOGNS>(v, buf);
    __syncthreads();
}

// Stages S..NFULL-1 of radix V (S counts from 0), as a compile-time recursion.
template <int LOGN, int S, int STOP, int SGN>
struct FullStages {
    static __device__ __forceinline__ void run(float2* buf, const Twiddles& tw) {
        using L = Line<LOGN>;
        stage_smem<LOGN, L::V, S * L::LV, SGN>(buf, tw);
        FullStages<LOGN, S + 1, STOP, SGN>::run(buf, tw);
    }
};
template <int LOGN, int STOP, int SGN>
struct FullStages<LOGN, STOP, STOP, SGN> {
    static __device__ __forceinline__ void run(float2*, const Twiddles&) {}
};

// Whole FFT in shared memory (indexed with Line<LOGN>::pad); the caller has
// synchronised after filling buf; the result is in buf, in natural order,
// after the call (which ends with a barrier).
template <int LOGN, int SGN>
__device__ __forceinline__ void fft_line_smem(float2* buf, const Twiddles& tw) {
    using L = Line<LOGN>;
    FullStages<LOGN, 0, L::NFULL, SGN>::run(buf, tw);
    if constexpr (L::REM > 0) stage_smem<LOGN, (1 << L::REM), L::NFULL * L::LV, SGN>(buf, tw);
}

// As fft_line_smem, but the last stage hands each output to epi(index, value)
// from registers instead of storing it (no barrier after; the stage's loads
// are complete, so the epilogue may write buf).
template <int LOGN, int SGN, typename Epi>
__device__ __forceinline__ void fft_line_epilogue(float2* buf, const Twiddles& tw, Epi& epi) {
    using L = Line<LOGN>;
    constexpr int NSMEM = L::REM ? L::NFULL : L::NFULL - 1;
    constexpr int R = L::REM ? (1 << L::REM) : L::V;
    constexpr int LOGNS = NSMEM * L::LV;
    FullStages<LOGN, 0, NSMEM, SGN>::run(buf, tw);
    float2 v[L::V];
    stage_load<LOGN, R>(v, buf);
    __syncthreads();
    stage_compute<LOGN, R, LOGNS, SGN>(v, tw);
    constexpr int B = L::V / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) epi(threadIdx.x + b * L::T + r * (L::N / R), v[b * R + r]);
}

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// As fft_line_epilogue_regs (below) for a first-stage input with x[tid + u T]
// = 0 for u >= U (U a power of two below V): the first stage takes the sparse
// form.
template <int LOGN, int U, int SGN, typename Epi>
__device__ __forceinline__ void fft_line_epilogue_regs_sparse(float2 (&v)[Line<LOGN>::V], float2* buf,
                                                              const Twiddles& tw, Epi& epi) {
    using L = Line<LOGN>;
    constexpr int NSMEM = L::REM ? L::NFULL : L::NFULL - 1;
    constexpr int R = L::REM ? (1 << L::REM) : L::V;
    constexpr int LOGNS = NSMEM * L::LV;
    static_assert(NSMEM >= 1, "the first stage must not be the last");
    static_assert(U < L::V, "sparse first stage");
    dft_first_sparse<L::V, U, SGN>(v);
    stage_store<LOGN, L::V, 0>(v, buf);
    __syncthreads();
    FullStages<LOGN, 1, NSMEM, SGN>::run(buf, tw);
    stage_load<LOGN, R>(v, buf);
    __syncthreads();
    stage_compute<LOGN, R, LOGNS, SGN>(v, tw);
    constexpr int B = L::V / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) epi(threadIdx.x + b * L::T + r * (L::N / R), v[b * R + r]);
}

// As fft_line_epilogue, but the first stage's input arrives in registers,
// v[r] = x[tid + r T] (the layout the first stage loads); buf is free to be
// overwritten when this is called.  pre() runs after the last stage's
// arithmetic, before the first epilogue call.
template <int LOGN, int SGN, typename Epi, typename Pre = NoHook>
__device__ __forceinline__ void fft_line_epilogue_regs(float2 (&v)[Line<LOGN>::V], float2* buf, const Twiddles& tw,
                                                       Epi& epi, const Pre& pre = Pre()) {
    using L = Line<LOGN>;
    constexpr int NSMEM = L::REM ? L::NFULL : L::NFULL - 1;
    constexpr int R = L::REM ? (1 << L::REM) : L::V;
    constexpr int LOGNS = NSMEM * L::LV;
    static_assert(NSMEM >= 1, "the first stage must not be the last");
    stage_compute<LOGN, L::V, 0, SGN>(v, tw);
    stage_store<LOGN, L::V, 0>(v, buf);
    __syncthreads();
    FullStages<LOGN, 1, NSMEM, SGN>::run(buf, tw);
    stage_load<LOGN, R>(v, buf);
    __syncthreads();
    stage_compute<LOGN, R, LOGNS, SGN>(v, tw);
    pre();
    constexpr int B = L::V / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) epi(threadIdx.x + b * L::T + r * (L::N / R), v[b * R + r]);
}

// As fft_line_smem, with the first stage's input in registers, v[r] =
// x[tid + r T] (the layout the first stage loads); buf is free to be
// overwritten when this is called.  The result is in buf, natural order.
template <int LOGN, int SGN>
__device__ __forceinline__ void fft_line_regs(float2 (&v)[Line<LOGN>::V], float2* buf, const Twiddles& tw) {
    using L = Line<LOGN>;
    static_assert(L::NFULL >= 1, "needs a radix-V first stage");
    stage_compute<LOGN, L::V, 0, SGN>(v, tw);
    stage_store<LOGN, L::V, 0>(v, buf);
    __syncthreads();
    FullStages<LOGN, 1, L::NFULL, SGN>::run(buf, tw);
    if constexpr (L::REM > 0) stage_smem<LOGN, (1 << L::REM), L::NFULL * L::LV, SGN>(buf, tw);
}

// Load the twiddle tables of an N-point line into shared memory: the two
// levels for any exponent and the direct table of the NT-th roots.  With 32
// values a thread (the 8192-point line) the direct table serves one stage
// only, the radix-32 stage with NS = 32, whose thread k needs W_1024^(r k) for
// r < 32: it is stored transposed, entry r 32 + k, so that a warp's 32 lanes
// (k = 0 .. 31) read 32 consecutive words (no bank conflict; in natural order
// lane k reads word r k, up to 32-way conflicts for even r).
template <int LOGN>
__device__ __forceinline__ Twiddles load_twiddles(float2* s_twh, float2* s_twl, float2* s_tt,
                                                  const float2* __restrict__ twh, const float2* __restrict__ twl,
                                                  const float2* __restrict__ tt) {
    using L = Line<LOGN>;
    for (int i = threadIdx.x; i < L::NH; i += L::T) s_twh[i] = twh[i];
    for (int i = threadIdx.x; i < L::NL; i += L::T) s_twl[i] = twl[i];
    if constexpr (L::V == 32) {
        static_assert(L::NT == 1024, "the transposed direct table holds 32 x 32 roots");
        for (int i = threadIdx.x; i < L::NT; i += L::T) s_tt[i] = tt[(i >> 5) * (i & 31)];
    } else {
        for (int i = threadIdx.x; i < L::NT; i += L::T) s_tt[i] = tt[i];
    }
    // 16 values a thread: the radix-16 stage with NS = 16 (thread k needs
    // W_256^(r k), r < 16) reads a transposed copy after the direct table, so
    // that a half-warp's lanes read 16 consecutive words (in the direct table,
    // at stride r NT / 256 words, every r conflicts at least 2-way)
    float2* s_tt2 = s_tt + 1024;
    if constexpr (L::NT2 > 0) {
        static_assert(L::NT >= 256, "W_256 from the direct table");
        for (int i = threadIdx.x; i < L::NT2; i += L::T) s_tt2[i] = tt[(i >> 4) * (i & 15) * (L::NT / 256)];
    }
    return Twiddles{s_twh, s_twl, s_tt, s_tt2};
}

}  // namespace tffr
