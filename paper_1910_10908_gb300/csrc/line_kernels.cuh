// The two FFT passes of the adjoint and of the forward twin, with the azimuth
// taps, the mode pruning and the deapodisation fused in.
//
// Adjoint (type 1): grid b = spread of D_n v_n; B = FFT_{+}(b) over the
// 2M_y x 2M_x fine grid; image f[jy][jx] = B[ky mod 2My][kx mod 2Mx] /
// (phi_hat(kx / 2Mx) phi_hat(ky / 2My)), k = j - M/2 (Eq. (Anu): spread,
// inverse FFT, divide by the window transform; Algorithm 1's final IFFT).
//
//   pass 1 (one CTA per fine row r): build row r in shared memory from the
//     pulse-row buffers R (azimuth taps) or from bucketed samples, FFT along
//     x, keep the M_x wanted modes, multiply by 1/phi_hat(kx), store row r of
//     the intermediate T ([2M_y][M_x] complex64, row-major).
//   pass 2 (clusters of 4 CTAs, one wanted x mode each): the cluster reads
//     32-byte row chunks of T (4 columns) and scatters them to its CTAs
//     through distributed shared memory; each CTA FFTs its column along y,
//     keeps the M_y wanted modes and multiplies by 1/phi_hat(ky); the cluster
//     gathers the results back and stores 32-byte chunks of 4 image columns.
//
// The forward runs the transposed steps in reverse order with FFT sign -1.
// Every kernel is a template on log2 of its line length.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "fft_reg.cuh"
#include "types.cuh"

namespace tffr {

namespace cg = cooperative_groups;

constexpr int kColCluster = 4;
constexpr int kTapChunk = 64;                          // tap entries staged per round

// Cluster barrier without memory ordering (the caller needs none).
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
// Arrive with release semantics: this thread's earlier shared-memory accesses
// are ordered before the peers' accesses that follow their wait.
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}

__device__ __forceinline__ void atomic_add_f2_global(float2* p, float2 v) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
    atomicAdd(p, v);
#else
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
#endif
}

__device__ __forceinline__ bool row_has_taps(const int* bucket_start, int r, int ny, int w) {
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        if (bucket_start[b + 1] > bucket_start[b]) return true;
    }
    return false;
}

template <int LOGN>
struct LineSmem {
    float2* buf;
    float2* twh;
    float2* twl;
    float2* tt;
    __device__ __forceinline__ explicit LineSmem(float2* base) {
        buf = base;
        twh = base + Line<LOGN>::PADLEN;
        twl = twh + 128;
        tt = twl + 64;
    }
};

template <int LOGN>
__host__ __device__ constexpr size_t line_smem_bytes() {
    return (size_t)Line<LOGN>::SMEM_ELEMS * sizeof(float2);
}
// Pass-1 epilogue: keep the M_x = N/2 wanted x modes, deapodise, store row r of T.
template <int LOGN>
struct RowOut {
    int r;
    const float* deap_x;
    float2* T;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        constexpr int N = 1 << LOGN, MX = N / 2, HALF = MX / 2;
        int jx;
        if (o < HALF) jx = o + HALF;
        else if (o >= N - HALF) jx = o - (N - HALF);
        else return;
        T[(size_t)r * MX + jx] = cscale(v, __ldg(&deap_x[jx]));
    }
};

// Pass 1 of the adjoint, pulse rows: fine row r = sum over the pulse rows p
// whose azimuth taps reach r of phi_y(r - v_p) R_p (shifted to its x cells).
template <int LOGN>
__global__ void __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_adj_rows(RowsView rv, const float2* __restrict__ R, int ny, int w, TapPoly tp, FftTables tab,
           const float* __restrict__ deap_x, float2* __restrict__ T) {
    using L = Line<LOGN>;
    constexpr int NX = L::N, MX = NX / 2;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    const int e0 = rv.tap_start[r], e1 = rv.tap_start[r + 1];
    if (e0 == e1) {
        for (int jx = tid; jx < MX; jx += L::T) T[(size_t)r * MX + jx] = make_float2(0.f, 0.f);
        return;
    }
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    for (int i = tid; i < L::PADLEN; i += L::T) S.buf[i] = make_float2(0.f, 0.f);
    __shared__ TapEntry s_tap[kTapChunk];
    for (int base = e0; base < e1; base += kTapChunk) {
        const int cnt = min(kTapChunk, e1 - base);
        __syncthreads();                               // zeroing done / previous chunk consumed
        for (int i = tid; i < cnt; i += L::T) s_tap[i] = rv.taps[base + i];   // T may be < chunk
        __syncthreads();
        for (int e = 0; e < cnt; ++e) {
            const TapEntry te = s_tap[e];
            const float2* Rp = R + te.off;
            for (int i = tid; i < te.len; i += L::T)
                atomic_add_f2_shared(&S.buf[L::pad(wrapmod(te.clo + i, NX))], cscale(__ldg(&Rp[i]), te.wy));
        }
    }
    __syncthreads();
    RowOut<LOGN> epi{r, deap_x, T};
    fft_line_epilogue<LOGN, +1>(S.buf, tw, epi);
}

// Pass 1 of the adjoint, general points: the samples of the w buckets whose
// taps reach fine row r (values already weighted, sorted by bucket) are
// spread straight into the shared row.
template <int LOGN>
__global__ void __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_adj_rows_general(GeneralView gv, const float2* __restrict__ sval, int ny, int w, TapPoly tp, FftTables tab,
                   const float* __restrict__ deap_x, float2* __restrict__ T) {
    using L = Line<LOGN>;
    constexpr int NX = L::N, MX = NX / 2;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (!row_has_taps(gv.bucket_start, r, ny, w)) {
        for (int jx = tid; jx < MX; jx += L::T) T[(size_t)r * MX + jx] = make_float2(0.f, 0.f);
        return;
    }
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    for (int i = tid; i < L::PADLEN; i += L::T) S.buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        for (int q = gv.bucket_start[b] + tid; q < gv.bucket_start[b + 1]; q += L::T) {
            const float2 v0 = sval[q];
            if (v0.x == 0.0f && v0.y == 0.0f) continue;
            const float2 v = cscale(v0, tap_eval(tp, t, 2.0f * gv.sfy[q] - 1.0f));
            const int c0 = gv.slx[q] - (h - 1);
            const float tx = 2.0f * gv.sfx[q] - 1.0f;
            for (int s = 0; s < w; ++s)
                atomic_add_f2_shared(&S.buf[L::pad(wrapmod(c0 + s, NX))], cscale(v, tap_eval(tp, s, tx)));
        }
    }
    __syncthreads();
    RowOut<LOGN> epi{r, deap_x, T};
    fft_line_epilogue<LOGN, +1>(S.buf, tw, epi);
}

// Pass-2 epilogue: keep the M_y = N/2 wanted y modes, deapodise, park them in
// the CTA's own line buffer for the cluster gather.
template <int LOGN>
struct ColPark {
    const float* deap_y;
    float2* buf;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        constexpr int N = 1 << LOGN, HALF = N / 4;
        int jy;
        if (o < HALF) jy = o + HALF;
        else if (o >= N - HALF) jy = o - (N - HALF);
        else return;
        buf[Line<LOGN>::pad(jy)] = cscale(v, __ldg(&deap_y[jy]));
    }
};

template <int LOGN>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_adj_cols(const float2* __restrict__ T, int Mx, FftTables tab, const float* __restrict__ deap_y,
           float2* __restrict__ img) {
    using L = Line<LOGN>;
    constexpr int NY = L::N, MY = NY / 2, V = L::V;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;           // first of the cluster's 4 columns
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    // element i = tid + u T of the scatter/gather belongs to column i % 4 =
    // tid % 4 (T is a multiple of 4), so each thread talks to one peer only
    static_assert(L::T % kColCluster == 0, "line threads must be a multiple of the cluster size");
    float2* const peer = cluster.map_shared_rank(S.buf, tid % kColCluster);
    // scatter: this CTA reads rows [rank NY/4, (rank+1) NY/4) of the 4 columns,
    // exactly V elements per thread; the global loads overlap the barrier that
    // makes sure every CTA of the cluster runs before its memory is written
    constexpr int ROWS = NY / kColCluster;
    {
        cluster_arrive_relaxed();                      // existence only: the sync below orders the data
        float2 tmp[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int i = tid + u * L::T;
            tmp[u] = __ldg(&T[(size_t)(rank * ROWS + i / kColCluster) * Mx + jx0 + i % kColCluster]);
        }
        cluster_wait();
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int i = tid + u * L::T;
            peer[L::pad(rank * ROWS + i / kColCluster)] = tmp[u];
        }
    }
    cluster.sync();
    ColPark<LOGN> epi{deap_y, S.buf};
    fft_line_epilogue<LOGN, +1>(S.buf, tw, epi);
    cluster.sync();
    // gather: this CTA stores image rows [rank MY/4, (rank+1) MY/4) of the 4 columns
    constexpr int OROWS = MY / kColCluster;
    {
        float2 tmp[V / 2];
#pragma unroll
        for (int u = 0; u < V / 2; ++u) {
            const int i = tid + u * L::T;
            tmp[u] = peer[L::pad(rank * OROWS + i / kColCluster)];
        }
#pragma unroll
        for (int u = 0; u < V / 2; ++u) {
            const int i = tid + u * L::T;
            img[(size_t)(rank * OROWS + i / kColCluster) * Mx + jx0 + i % kColCluster] = tmp[u];
        }
    }
    // the stores above consumed every remote load, so peers may leave once all
    // threads got here; no memory ordering is needed
    cluster_arrive_relaxed();
    cluster_wait();
}

template <int LOGN>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_fwd_cols(const float2* __restrict__ img, int Mx, FftTables tab, const float* __restrict__ deap_y,
           const float* __restrict__ deap_x, float2* __restrict__ T) {
    using L = Line<LOGN>;
    constexpr int NY = L::N, MY = NY / 2, V = L::V;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    // the scatter below fills modes [-MY/2, MY/2); zero the rest of this CTA's line
    for (int i = MY / 2 + tid; i < NY - MY / 2; i += L::T) S.buf[L::pad(i)] = make_float2(0.f, 0.f);
    // element i = tid + u T of the scatter/gather belongs to column i % 4 =
    // tid % 4 (T is a multiple of 4), so each thread talks to one peer only
    static_assert(L::T % kColCluster == 0, "line threads must be a multiple of the cluster size");
    float2* const peer = cluster.map_shared_rank(S.buf, tid % kColCluster);
    constexpr int IROWS = MY / kColCluster;
    {
        cluster_arrive_relaxed();                      // every CTA runs before its memory is written
        float2 tmp[V / 2];
#pragma unroll
        for (int u = 0; u < V / 2; ++u) {
            const int i = tid + u * L::T;
            tmp[u] = __ldg(&img[(size_t)(rank * IROWS + i / kColCluster) * Mx + jx0 + i % kColCluster]);
        }
        cluster_wait();
#pragma unroll
        for (int u = 0; u < V / 2; ++u) {
            const int i = tid + u * L::T;
            const int jy = rank * IROWS + i / kColCluster;
            const int k = i % kColCluster;
            const float d = __ldg(&deap_y[jy]) * __ldg(&deap_x[jx0 + k]);
            peer[L::pad(wrapmod(jy - MY / 2, NY))] = cscale(tmp[u], d);
        }
    }
    cluster.sync();
    fft_line_smem<LOGN, -1>(S.buf, tw);
    cluster.sync();
    constexpr int ROWS = NY / kColCluster;
    {
        float2 tmp[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int i = tid + u * L::T;
            tmp[u] = peer[L::pad(rank * ROWS + i / kColCluster)];
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int i = tid + u * L::T;
            T[(size_t)(rank * ROWS + i / kColCluster) * Mx + jx0 + i % kColCluster] = tmp[u];
        }
    }
    cluster_arrive_relaxed();                          // every remote load was consumed above
    cluster_wait();
}

template <int LOGN, bool ROWS>
__global__ void __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_fwd_rows(RowsView rv, GeneralView gv, const float2* __restrict__ T, int ny, int w, TapPoly tp, FftTables tab,
           float2* __restrict__ R, float2* __restrict__ acc) {
    using L = Line<LOGN>;
    constexpr int NX = L::N, MX = NX / 2;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (ROWS) {
        if (rv.tap_start[r] == rv.tap_start[r + 1]) return;
    } else if (!row_has_taps(gv.bucket_start, r, ny, w)) {
        return;
    }
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    for (int i = tid; i < L::PADLEN; i += L::T) S.buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int jx = tid; jx < MX; jx += L::T) S.buf[L::pad(wrapmod(jx - MX / 2, NX))] = T[(size_t)r * MX + jx];
    __syncthreads();
    fft_line_smem<LOGN, -1>(S.buf, tw);
    if (ROWS) {
        __shared__ TapEntry s_tap[kTapChunk];
        const int e0 = rv.tap_start[r], e1 = rv.tap_start[r + 1];
        for (int base = e0; base < e1; base += kTapChunk) {
            const int cnt = min(kTapChunk, e1 - base);
            __syncthreads();
            for (int i = tid; i < cnt; i += L::T) s_tap[i] = rv.taps[base + i];   // T may be < chunk
            __syncthreads();
            for (int e = 0; e < cnt; ++e) {
                const TapEntry te = s_tap[e];
                float2* Rp = R + te.off;
                for (int i = tid; i < te.len; i += L::T)
                    atomic_add_f2_global(&Rp[i], cscale(S.buf[L::pad(wrapmod(te.clo + i, NX))], te.wy));
            }
        }
        return;
    }
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        const int q0 = gv.bucket_start[b], q1 = gv.bucket_start[b + 1];
        {
            for (int q = q0 + tid; q < q1; q += L::T) {
                const float wy = tap_eval(tp, t, 2.0f * gv.sfy[q] - 1.0f);
                const int c0 = gv.slx[q] - (h - 1);
                const float tx = 2.0f * gv.sfx[q] - 1.0f;
                float2 a = make_float2(0.f, 0.f);
                for (int s = 0; s < w; ++s) {
                    const float wt = tap_eval(tp, s, tx);
                    const float2 g = S.buf[L::pad(wrapmod(c0 + s, NX))];
                    a.x = fmaf(wt, g.x, a.x);
                    a.y = fmaf(wt, g.y, a.y);
                }
                atomic_add_f2_global(&acc[q], cscale(a, wy));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Pulse-row order of the two passes (rows layout with at most M_y pulse rows).
// The FFT along x is linear, so it can run on the P pulse-row buffers before
// the azimuth taps instead of on the 2 M_y fine rows after them:
//   F_p = prune(FFT_x(R_p)) / phi_hat(kx)                       ([P][M_x])
//   fine row r of the column line = sum_p phi_y(r - v_p) F_p[kx]
// The taps then become a 1-D spread along y inside the column pass, the x
// FFTs drop from 2 M_y to P lines and the intermediate from 2 M_y M_x to
// P M_x entries.  The forward twin runs the transposed steps.
// row_wy holds the w azimuth taps of each pulse row (stride 8 floats).
// ---------------------------------------------------------------------------

// Column passes in pulse-row order: the line's shared memory, then a column
// of F (up to N / 2 = M_y places) starting on a 128-byte boundary, so that
// the 16 places of each 128 bytes fall in one shared-memory wavefront.  In the
// adjoint the same area later receives the cluster's output rows: 4 columns
// of N / 8 rows, each column padded by kRecvPad entries so that a column
// starts a quarter bank cycle (32 bytes) after the previous one: the 16 lanes
// of a half-warp reading 4 rows x 4 columns then touch 16 different banks.
template <int LOGN>
constexpr int kPulseColOff = (Line<LOGN>::SMEM_ELEMS + 15) & ~15;
constexpr int kRecvPad = 4;

template <int LOGN>
__host__ __device__ constexpr size_t line_smem_pulse_cols() {
    return (size_t)(kPulseColOff<LOGN> + Line<LOGN>::N / 2 + 4 * kRecvPad) * sizeof(float2);
}

// F in the adjoint's pulse-row order, by blocks of four columns: entry q
// (place in fine-y order) of column jx at F[((jx / 4) ldq + q) 4 + jx % 4],
// ldq = P rounded up to 4.  The x pass stores the four columns of a block as
// one 32-byte piece; the four CTAs of a column cluster read their block as
// one contiguous run.
__host__ __device__ __forceinline__ int pulse_ldq(int P) { return (P + 3) & ~3; }

// Pass-1 epilogue of the adjoint in pulse-row order: keep the M_x = N/2
// wanted x modes, deapodise (and, for a shifted line, undo the shift with the
// thread's phase factor), store them as entry q of every column of F.
template <int LOGN, bool RAMP = false>
struct QuadOut {
    int q, ldq;
    const float* deap_x;
    float2* F;
    float2 ramp;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        constexpr int N = 1 << LOGN, MX = N / 2, HALF = MX / 2;
        int jx;
        if (o < HALF) jx = o + HALF;
        else if (o >= N - HALF) jx = o - (N - HALF);
        else return;
        if constexpr (RAMP) v = cmul(v, ramp);
        F[(((size_t)(jx >> 2) * ldq + q) << 2) + (jx & 3)] = cscale(v, __ldg(&deap_x[jx]));
    }
};

template <int LOGN>
__global__ void __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_adj_rows_pulse(RowsView rv, const float2* __restrict__ R, FftTables tab, const float* __restrict__ deap_x,
                 float2* __restrict__ F) {
    using L = Line<LOGN>;
    constexpr int NX = L::N;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    const int q = blockIdx.x;                          // place in fine-y order
    const int p = rv.rank_row[q];
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    const int len = rv.row_len[p], clo = rv.row_clo[p];
    const float2* Rp = R + rv.row_off[p];
    // line cell j holds R_p[(j - clo) mod NX] when that is below len, else 0;
    // read straight into the first FFT stage's registers (cell tid + u T)
    float2 v[L::V];
#pragma unroll
    for (int u = 0; u < L::V; ++u) {
        const int o = wrapmod(tid + u * L::T - clo, NX);
        v[u] = (o < len) ? __ldg(&Rp[o]) : make_float2(0.f, 0.f);
    }
    __syncthreads();                                   // twiddles in place
    QuadOut<LOGN> epi{q, pulse_ldq(rv.P), deap_x, F, make_float2(1.f, 0.f)};
    fft_line_epilogue_regs<LOGN, +1>(v, S.buf, tw, epi);
}

constexpr int kPulseBatch = 8;                         // pulse rows whose taps are loaded together

// The w azimuth taps of pulse row p, two 16-byte loads.
__device__ __forceinline__ void load_row_taps(const float* __restrict__ row_wy, int p, float (&wy)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(row_wy + (size_t)p * 8));
    const float4 b = __ldg(reinterpret_cast<const float4*>(row_wy + (size_t)p * 8 + 4));
    wy[0] = a.x; wy[1] = a.y; wy[2] = a.z; wy[3] = a.w;
    wy[4] = b.x; wy[5] = b.y; wy[6] = b.z; wy[7] = b.w;
}

// Pass-2 epilogue of the adjoint in pulse-row order: keep the M_y = N/2 wanted
// y modes, deapodise, and store each into the receive area of the cluster CTA
// that writes its image row (row jy goes to CTA jy / (N/8), column slot =
// this CTA's rank).
template <int LOGN>
struct ColPush {
    const float* deap_y;
    float2* dst0;
    float2* dst1;
    float2* dst2;
    float2* dst3;
    int rank;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        constexpr int N = 1 << LOGN, HALF = N / 4, OROWS = N / 8;
        int jy;
        if (o < HALF) jy = o + HALF;
        else if (o >= N - HALF) jy = o - (N - HALF);
        else return;
        const int c = jy / OROWS;
        float2* d = c == 0 ? dst0 : c == 1 ? dst1 : c == 2 ? dst2 : dst3;
        d[rank * (OROWS + kRecvPad) + (jy % OROWS)] = cscale(v, __ldg(&deap_y[jy]));
    }
};

// Waits at a cluster barrier whose arrive came earlier (see k_adj_cols_pulse).
struct ClusterWait {
    __device__ __forceinline__ void operator()() const { cluster_wait(); }
};

// Places after the last of an F column that keep copies of the first ones, so
// that a fine row's run of places (modulo P) is read without a wrap test.
constexpr int kPlaceCopies = 8;

// Azimuth taps of fine row r: sum over slots k < 4 K4 of ell_w[k / 4][r].k
// times fcol[ell_first[r] + k] (slots past the row's count weigh 0).
template <int K4>
__device__ __forceinline__ float2 gather_taps(const float2* fcol, int q, const float4 (&wt)[K4]) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < K4; ++h) {
        const float g[4] = {wt[h].x, wt[h].y, wt[h].z, wt[h].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = fcol[q + 4 * h + k];
            acc.x = fmaf(g[k], f.x, acc.x);
            acc.y = fmaf(g[k], f.y, acc.y);
        }
    }
    return acc;
}

template <int LOGN, int K4>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_adj_cols_pulse(const float2* __restrict__ F, int P, int Mx, FftTables tab, const int* __restrict__ ell_first,
                 const float4* __restrict__ ell_w, const float* __restrict__ deap_y, float2* __restrict__ img,
                 int ahead) {
    using L = Line<LOGN>;
    constexpr int NY = L::N, MY = NY / 2, V = L::V;
    constexpr int OROWS = MY / kColCluster;            // image rows each CTA of the cluster writes
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    float2* fcol = smem + kPulseColOff<LOGN>;         // this CTA's column of F, then its receive area
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;
    const int tid = threadIdx.x;
    static_assert(L::T % kColCluster == 0, "line threads must be a multiple of the cluster size");
    // Barrier phases: (A) every CTA runs before its memory is written; (B) the F
    // columns are complete; (C) every CTA has read its F column (its area may
    // receive output rows); (D) every output row has arrived.  C's arrive comes
    // right after the gather and its wait just before the last FFT stage's
    // stores, so the FFT hides it.
    cluster_arrive_relaxed();                          // (A)
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    // The cluster's block of four columns of F is one contiguous run; CTA rank
    // reads the quarter of places [p0, p0 + PQ), each place's 32-byte piece by
    // one thread (two 16-byte loads), and sends column c of it to the fcol of
    // CTA c: a warp's store then carries 32 neighbouring places to one CTA.
    // Places 0 .. 7 also go to P .. P + 7 (modulo P), so that a fine row's run
    // of places is read without a wrap test.
    constexpr int KP = (V / 8) > 0 ? V / 8 : 1;        // places per thread: PQ <= N / 8 = KP T
    const int ldq = pulse_ldq(P), PQ = ldq / kColCluster;
    const int p0 = rank * PQ, nq = max(0, min(P, p0 + PQ) - p0);
    const float4* const Fq = reinterpret_cast<const float4*>(F + ((size_t)(jx0 / kColCluster) * ldq + p0) * kColCluster);
    // the same quarter of the block one wave of clusters ahead (`ahead` blocks
    // later) into L2, so that its CTA's loads find it there
    if (tid == 0 && nq > 0 && jx0 / kColCluster + ahead < Mx / kColCluster) {
        const float2* nxt = F + ((size_t)(jx0 / kColCluster + ahead) * ldq + p0) * kColCluster;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nxt), "r"((unsigned)nq * 32u) : "memory");
    }
    float4 lo[KP], hi[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int j = tid + k * L::T;
        if (j < nq) {
            lo[k] = __ldg(&Fq[2 * j]);
            hi[k] = __ldg(&Fq[2 * j + 1]);
        }
    }
    cluster_wait();                                    // (A), behind the loads
    float2* const peer0 = cluster.map_shared_rank(fcol, 0);
    float2* const peer1 = cluster.map_shared_rank(fcol, 1);
    float2* const peer2 = cluster.map_shared_rank(fcol, 2);
    float2* const peer3 = cluster.map_shared_rank(fcol, 3);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int j = tid + k * L::T;
        if (j < nq) {
            const int q = p0 + j;
            peer0[q] = make_float2(lo[k].x, lo[k].y);
            peer1[q] = make_float2(lo[k].z, lo[k].w);
            peer2[q] = make_float2(hi[k].x, hi[k].y);
            peer3[q] = make_float2(hi[k].z, hi[k].w);
            for (int r = q; r < kPlaceCopies; r += P) {
                peer0[P + r] = make_float2(lo[k].x, lo[k].y);
                peer1[P + r] = make_float2(lo[k].z, lo[k].w);
                peer2[P + r] = make_float2(hi[k].x, hi[k].y);
                peer3[P + r] = make_float2(hi[k].z, hi[k].w);
            }
        }
    }
    cluster_arrive_release();                          // (B)
    cluster_wait();
    // azimuth taps, gathered: fine row r sums its run of places in fine-y
    // order (first place ell_first[r], one weight per slot; a warp's lanes
    // read neighbouring words of fcol), straight into the registers of the
    // first FFT stage (row tid + u T)
    float2 v[V];
    constexpr int UB = V >= 8 ? 8 : V;
#pragma unroll
    for (int u0 = 0; u0 < V; u0 += UB) {
        int q[UB];
        float4 wt[UB][K4];
#pragma unroll
        for (int j = 0; j < UB; ++j) {
            const int r = tid + (u0 + j) * L::T;
            q[j] = __ldg(&ell_first[r]);
#pragma unroll
            for (int h = 0; h < K4; ++h) wt[j][h] = __ldg(&ell_w[h * NY + r]);
        }
#pragma unroll
        for (int j = 0; j < UB; ++j) v[u0 + j] = gather_taps<K4>(fcol, q[j], wt[j]);
    }
    cluster_arrive_release();                          // (C): this CTA's fcol reads are done
    ColPush<LOGN> epi{deap_y,
                      cluster.map_shared_rank(fcol, 0), cluster.map_shared_rank(fcol, 1),
                      cluster.map_shared_rank(fcol, 2), cluster.map_shared_rank(fcol, 3), rank};
    fft_line_epilogue_regs<LOGN, +1>(v, S.buf, tw, epi, ClusterWait{});   // (C) waited before the stores
    cluster_arrive_release();                          // (D)
    cluster_wait();
    // this CTA's image rows [rank OROWS, (rank + 1) OROWS) of the 4 columns, from
    // its receive area (column c at c (OROWS + kRecvPad)), as 32-byte row chunks
#pragma unroll
    for (int u = 0; u < V / 2; ++u) {
        const int i = tid + u * L::T;
        const int r = i / kColCluster, c = i % kColCluster;
        img[(size_t)(rank * OROWS + r) * Mx + jx0 + c] = fcol[c * (OROWS + kRecvPad) + r];
    }
}

template <int LOGN>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_fwd_cols_pulse(const float2* __restrict__ img, int Mx, FftTables tab, const float* __restrict__ deap_y,
                 const float* __restrict__ deap_x, const int* __restrict__ q_ly, const float* __restrict__ q_wy,
                 int w, int P, float2* __restrict__ F) {
    using L = Line<LOGN>;
    constexpr int NY = L::N, MY = NY / 2, V = L::V;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    float2* fcol = smem + kPulseColOff<LOGN>;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    for (int i = MY / 2 + tid; i < NY - MY / 2; i += L::T) S.buf[L::pad(i)] = make_float2(0.f, 0.f);
    static_assert(L::T % kColCluster == 0, "line threads must be a multiple of the cluster size");
    // The cluster's 4 image columns: CTA rank reads rows [rank IROWS, (rank + 1)
    // IROWS), each row's 32-byte piece (all 4 columns) by one thread, and sends
    // column c of it, deapodised and zero-padded into the line, to CTA c: a
    // warp's store carries 32 neighbouring rows to one CTA.
    constexpr int IROWS = MY / kColCluster;
    constexpr int KR = (IROWS + L::T - 1) / L::T;      // rows per thread
    float2* peer[kColCluster];
#pragma unroll
    for (int c = 0; c < kColCluster; ++c) peer[c] = cluster.map_shared_rank(S.buf, c);
    {
        cluster_arrive_relaxed();                      // every CTA runs before its memory is written
        float4 lo[KR], hi[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int j = tid + k * L::T;
            if (j < IROWS) {
                const float4* src = reinterpret_cast<const float4*>(img + (size_t)(rank * IROWS + j) * Mx + jx0);
                lo[k] = __ldg(src);
                hi[k] = __ldg(src + 1);
            }
        }
        float dx[kColCluster];
#pragma unroll
        for (int c = 0; c < kColCluster; ++c) dx[c] = __ldg(&deap_x[jx0 + c]);
        cluster_wait();
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int j = tid + k * L::T;
            if (j < IROWS) {
                const int jy = rank * IROWS + j;
                const float dy = __ldg(&deap_y[jy]);
                const int o = L::pad(wrapmod(jy - MY / 2, NY));
                peer[0][o] = cscale(make_float2(lo[k].x, lo[k].y), dy * dx[0]);
                peer[1][o] = cscale(make_float2(lo[k].z, lo[k].w), dy * dx[1]);
                peer[2][o] = cscale(make_float2(hi[k].x, hi[k].y), dy * dx[2]);
                peer[3][o] = cscale(make_float2(hi[k].z, hi[k].w), dy * dx[3]);
            }
        }
    }
    cluster.sync();
    fft_line_smem<LOGN, -1>(S.buf, tw);
    // transposed azimuth taps, per place q in fine-y order (a warp's lanes
    // read neighbouring cells of the line):
    // F_q = sum_s phi_y(s - (w/2 - 1) - fy_q) line[ly_q - (w/2 - 1) + s],
    // pushed to the CTA that writes place q's row of F: CTA q / PQ keeps the
    // cluster's 4 columns of its places in fcol, column c at c (PQ + kRecvPad)
    const int PQ = (P + kColCluster - 1) / kColCluster;
    float2* dst[kColCluster];
#pragma unroll
    for (int c = 0; c < kColCluster; ++c) dst[c] = cluster.map_shared_rank(fcol, c) + rank * (PQ + kRecvPad);
    const int h = w / 2;
    for (int base = 0; base < P; base += kPulseBatch * L::T) {
        int c0[kPulseBatch];
        float wy[kPulseBatch][8];
#pragma unroll
        for (int b = 0; b < kPulseBatch; ++b) {
            const int q = min(base + tid + b * L::T, P - 1);
            c0[b] = __ldg(&q_ly[q]) - (h - 1);
            load_row_taps(q_wy, q, wy[b]);
        }
#pragma unroll
        for (int b = 0; b < kPulseBatch; ++b) {
            const int p = base + tid + b * L::T;
            if (p >= P) break;
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                if (s < w) {
                    const float2 g = S.buf[L::pad(wrapmod(c0[b] + s, NY))];
                    a.x = fmaf(wy[b][s], g.x, a.x);
                    a.y = fmaf(wy[b][s], g.y, a.y);
                }
            }
            const int o = p / PQ;
            float2* d = o == 0 ? dst[0] : o == 1 ? dst[1] : o == 2 ? dst[2] : dst[3];
            d[p - o * PQ] = a;
        }
    }
    cluster.sync();
    // this CTA's places [p0, p0 + PQ) of the 4 columns, from fcol, as 32-byte row pieces of F
    const int p0 = min(P, rank * PQ), nel = (min(P, p0 + PQ) - p0) * kColCluster;
    for (int i = tid; i < nel; i += L::T) {
        const int r = i / kColCluster, c = i % kColCluster;
        F[(size_t)(p0 + r) * Mx + jx0 + c] = fcol[c * (PQ + kRecvPad) + r];
    }
}

// Forward x-pass epilogue: line cell o goes to the row buffer at
// (o - clo) mod N when that is below len.
template <int LOGN>
struct RowCells {
    int clo, len;
    float2* Rp;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        const int i = wrapmod(o - clo, 1 << LOGN);
        if (i < len) Rp[i] = v;
    }
};

template <int LOGN>
__global__ void __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_fwd_rows_pulse(RowsView rv, const float2* __restrict__ F, FftTables tab, float2* __restrict__ R) {
    using L = Line<LOGN>;
    constexpr int NX = L::N, MX = NX / 2;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    const int q = blockIdx.x;                          // place in fine-y order: row q of F
    const int p = rv.rank_row[q];
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    // line position j holds mode j (j < MX/2) or j - NX (j >= NX - MX/2), i.e.
    // F column j + MX/2 or j - (NX - MX/2); the middle is zero.  Loaded straight
    // into the first FFT stage's registers (position tid + u T).
    float2 v[L::V];
    const float2* Fp = F + (size_t)q * MX;
#pragma unroll
    for (int u = 0; u < L::V; ++u) {
        const int j = tid + u * L::T;
        v[u] = (j < MX / 2) ? __ldg(&Fp[j + MX / 2])
             : (j >= NX - MX / 2) ? __ldg(&Fp[j - (NX - MX / 2)]) : make_float2(0.f, 0.f);
    }
    __syncthreads();                                   // twiddles in place
    // the last stage hands each line cell to the epilogue, which stores the
    // cells of the row buffer (cell clo + i at R_p[i], i < len) and drops the rest
    RowCells<LOGN> epi{rv.row_clo[p], rv.row_len[p], R + rv.row_off[p]};
    fft_line_epilogue_regs<LOGN, -1>(v, S.buf, tw, epi);
}

// ---------------------------------------------------------------------------
// Normal operator E^H D E by its Toeplitz embedding.  On the image grid
// (E^H D E f)[j] = sum_j' k(j - j') f[j'] with k(m) = sum_n D_n exp(2 pi i
// lam_n . m / M), m in (-M, M)^2: a convolution, computed on the 2M x 2M grid
// as crop(IFFT2(Khat . FFT2(pad(f)))) with Khat = FFT2 of k arranged
// circularly (built once).  Lines here are full 2M-point transforms.
// ---------------------------------------------------------------------------

// One row per CTA: in[r][0..n_in) (zero beyond) -> FFT_{SGN} -> out[r][0..n_out).
template <int LOGN, int SGN>
__global__ void __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_fft_rows(const float2* __restrict__ in, int ld_in, int n_in, FftTables tab, float2* __restrict__ out, int ld_out,
           int n_out) {
    using L = Line<LOGN>;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    const float2* row = in + (size_t)r * ld_in;
    float2 v[L::V];
#pragma unroll
    for (int u = 0; u < L::V; ++u) {
        const int j = tid + u * L::T;
        v[u] = (j < n_in) ? __ldg(&row[j]) : make_float2(0.f, 0.f);
    }
    __syncthreads();                                   // twiddles in place
    fft_line_regs<LOGN, SGN>(v, S.buf, tw);
    float2* o = out + (size_t)r * ld_out;
    for (int k = tid; k < n_out; k += L::T) o[k] = S.buf[L::pad(k)];
}

// Clusters of 4 CTAs, one column each, over a row-major array with ld columns:
// column rows [0, n_in) (zero beyond) -> FFT_-.  With khat (column-major,
// khat[col][ky]): times khat, then FFT_+ and rows [0, n_out) out (row-major,
// ld columns).  Without: times (-1)^(ky + col) scale (the circular arrangement
// of k and the inverse's normalisation), stored column-major: out[col][ky].
template <int LOGN>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(Line<LOGN>::T, (Line<LOGN>::T >= 256 ? 2 : 4))
k_fft_cols_conv(const float2* __restrict__ in, int n_in, int ld, FftTables tab, const float2* __restrict__ khat,
                float scale, float2* __restrict__ out, int n_out) {
    using L = Line<LOGN>;
    constexpr int NY = L::N;
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;
    const int col = jx0 + rank;
    const int tid = threadIdx.x;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, tab.twh, tab.twl, tab.tt);
    for (int i = n_in + tid; i < NY; i += L::T) S.buf[L::pad(i)] = make_float2(0.f, 0.f);
    static_assert(L::T % kColCluster == 0, "line threads must be a multiple of the cluster size");
    float2* const peer = cluster.map_shared_rank(S.buf, tid % kColCluster);
    // scatter: this CTA reads rows [r0, r1) of the 4 columns (32-byte chunks)
    const int RQ = (n_in + kColCluster - 1) / kColCluster;
    const int r0 = min(n_in, rank * RQ), nel = (min(n_in, r0 + RQ) - r0) * kColCluster;
    cluster_arrive_relaxed();                          // every CTA runs before its memory is written
    cluster_wait();
    for (int base = 0; base < nel; base += L::V * L::T) {
        float2 tmp[L::V];
#pragma unroll
        for (int u = 0; u < L::V; ++u) {
            const int i = base + tid + u * L::T;
            tmp[u] = (i < nel) ? __ldg(&in[(size_t)(r0 + i / kColCluster) * ld + jx0 + i % kColCluster])
                               : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < L::V; ++u) {
            const int i = base + tid + u * L::T;
            if (i < nel) peer[L::pad(r0 + i / kColCluster)] = tmp[u];
        }
    }
    cluster.sync();
    fft_line_smem<LOGN, -1>(S.buf, tw);
    if (!khat) {
        float2* o = out + (size_t)col * NY;
        for (int k = tid; k < NY; k += L::T) o[k] = cscale(S.buf[L::pad(k)], ((k + col) & 1) ? -scale : scale);
        cluster_arrive_relaxed();                      // no remote access after the scatter barrier
        cluster_wait();
        return;
    }
    {
        const float2* kc = khat + (size_t)col * NY;
        for (int k = tid; k < NY; k += L::T) S.buf[L::pad(k)] = cmul(S.buf[L::pad(k)], __ldg(&kc[k]));
        __syncthreads();
        fft_line_smem<LOGN, +1>(S.buf, tw);
    }
    cluster.sync();
    // gather: this CTA stores rows [o0, o1) of the 4 columns
    const int OQ = (n_out + kColCluster - 1) / kColCluster;
    const int o0 = min(n_out, rank * OQ), nout = (min(n_out, o0 + OQ) - o0) * kColCluster;
    for (int base = 0; base < nout; base += L::V * L::T) {
        float2 tmp[L::V];
#pragma unroll
        for (int u = 0; u < L::V; ++u) {
            const int i = base + tid + u * L::T;
            tmp[u] = (i < nout) ? peer[L::pad(o0 + i / kColCluster)] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < L::V; ++u) {
            const int i = base + tid + u * L::T;
            if (i < nout) out[(size_t)(o0 + i / kColCluster) * ld + jx0 + i % kColCluster] = tmp[u];
        }
    }
    cluster_arrive_relaxed();                          // every remote load was consumed above
    cluster_wait();
}

}  // namespace tffr
