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
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "fft_reg.cuh"
#include "kernels_spread.cuh"

namespace tffr {

namespace cg = cooperative_groups;

constexpr int kColCluster = 4;

struct GeneralView {
    const int* bucket_start;   // [ny + 1] samples grouped by floor(2 lam_y) mod ny
    const int* perm;           // [N] sorted position -> sample index
    const int* slx;            // [N] fine x cell, sorted order
    const float* sfx;          // [N] fine x offset, sorted order
    const float* sfy;          // [N] fine y offset, sorted order
    const float* sD;           // [N] weights, sorted order
};

struct FftTables {
    const float2* twh;         // exp(2 pi i 64 h / n)
    const float2* twl;         // exp(2 pi i l / n)
};

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

// Values per thread for an n-point line, and the matching block size n / V.
__host__ __device__ constexpr int line_v(int n) {
    return n >= 8192 ? 32 : n >= 512 ? 16 : n >= 256 ? 8 : n >= 128 ? 4 : 2;
}

// Shared memory of one line kernel: the padded line plus the twiddle tables.
template <int V>
__host__ __device__ constexpr size_t line_smem_bytes(int n) {
    return (size_t)(fft_pad_len<V>(n) + 128 + 64) * sizeof(float2);
}

template <int V>
struct LineSmem {
    float2* buf;
    float2* twh;
    float2* twl;
    __device__ __forceinline__ LineSmem(float2* base, int n) {
        buf = base;
        twh = base + fft_pad_len<V>(n);
        twl = twh + 128;
    }
};

// The last stage of the FFT computed into registers, each output handed to
// epi(output index, value).  Ends with no barrier; buf may be rewritten by
// the epilogue (the stage's loads are complete).
template <int V, int R, int LOGR, typename Epi>
__device__ __forceinline__ void last_stage(float2* buf, const LineFft& L, int logNs, Epi& epi) {
    float2 v[V];
    stage_load<V, R>(v, buf, L.n);
    __syncthreads();
    stage_compute<V, R, LOGR>(v, L, logNs);
    constexpr int B = V / R;
    const int T = L.n / V;
    const int stride = L.n / R;
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) epi(threadIdx.x + b * T + r * stride, v[b * R + r]);
}

template <int V, typename Epi>
__device__ __forceinline__ void fft_line_epilogue(float2* buf, const LineFft& L, Epi& epi) {
    constexpr int LV = LogOf<V>::v;
    const int nfull = L.logn / LV;
    const int rem = L.logn - nfull * LV;
    const int nsmem = rem ? nfull : nfull - 1;
    int logNs = 0;
    for (int s = 0; s < nsmem; ++s) {
        stage_smem<V, V, LV>(buf, L, logNs);
        logNs += LV;
    }
    switch (rem) {
        case 0: last_stage<V, V, LV>(buf, L, logNs, epi); break;
        case 1: last_stage<V, 2, 1>(buf, L, logNs, epi); break;
        case 2: if constexpr (V >= 4) last_stage<V, 4, 2>(buf, L, logNs, epi); break;
        case 3: if constexpr (V >= 8) last_stage<V, 8, 3>(buf, L, logNs, epi); break;
        default: if constexpr (V >= 16) last_stage<V, 16, 4>(buf, L, logNs, epi); break;
    }
}

// Pass-1 epilogue: keep the M_x wanted x modes, deapodise, store row r of T.
struct RowOut {
    int n, Mx, r;
    const float* deap_x;
    float2* T;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        const int half = Mx >> 1;
        int jx;
        if (o < half) jx = o + half;
        else if (o >= n - half) jx = o - (n - half);
        else return;
        T[(size_t)r * Mx + jx] = cscale(v, __ldg(&deap_x[jx]));
    }
};

// Pass 1 of the adjoint, pulse rows: fine row r = sum over the pulse rows p
// whose azimuth taps reach r of phi_y(r - v_p) R_p (shifted to its x cells).
template <int V>
__global__ void __launch_bounds__(256, 2)
k_adj_rows(RowsView rv, const float2* __restrict__ R, int nx, int lognx, int ny, int Mx, int w, TapPoly tp,
           FftTables tab, const float* __restrict__ deap_x, float2* __restrict__ T) {
    extern __shared__ float2 smem[];
    LineSmem<V> S(smem, nx);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (!row_has_taps(rv.bucket_start, r, ny, w)) {
        for (int jx = tid; jx < Mx; jx += blockDim.x) T[(size_t)r * Mx + jx] = make_float2(0.f, 0.f);
        return;
    }
    load_twiddles(S.twh, S.twl, tab.twh, tab.twl, nx);
    const int nsm = fft_pad_len<V>(nx);
    for (int i = tid; i < nsm; i += blockDim.x) S.buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        for (int q = rv.bucket_start[b]; q < rv.bucket_start[b + 1]; ++q) {
            const int p = rv.bucket_rows[q];
            const float wy = tap_eval(tp, t, 2.0f * rv.row_fy[p] - 1.0f);
            const int clo = rv.row_clo[p], len = rv.row_len[p];
            const float2* Rp = R + rv.row_off[p];
            for (int i = tid; i < len; i += blockDim.x) {
                const int c = wrapmod(clo + i, nx);
                atomic_add_f2_shared(&S.buf[fft_pad<V>(c)], cscale(Rp[i], wy));
            }
        }
    }
    __syncthreads();
    const LineFft L{nx, lognx, S.twh, S.twl, +1.0f};
    RowOut epi{nx, Mx, r, deap_x, T};
    fft_line_epilogue<V>(S.buf, L, epi);
}

// Pass 1 of the adjoint, general points: the samples of the w buckets whose
// taps reach fine row r (values already weighted, sorted by bucket) are
// spread straight into the shared row.
template <int V>
__global__ void __launch_bounds__(256, 2)
k_adj_rows_general(GeneralView gv, const float2* __restrict__ sval, int nx, int lognx, int ny, int Mx, int w,
                   TapPoly tp, FftTables tab, const float* __restrict__ deap_x, float2* __restrict__ T) {
    extern __shared__ float2 smem[];
    LineSmem<V> S(smem, nx);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (!row_has_taps(gv.bucket_start, r, ny, w)) {
        for (int jx = tid; jx < Mx; jx += blockDim.x) T[(size_t)r * Mx + jx] = make_float2(0.f, 0.f);
        return;
    }
    load_twiddles(S.twh, S.twl, tab.twh, tab.twl, nx);
    const int nsm = fft_pad_len<V>(nx);
    for (int i = tid; i < nsm; i += blockDim.x) S.buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        for (int q = gv.bucket_start[b] + tid; q < gv.bucket_start[b + 1]; q += blockDim.x) {
            const float2 v0 = sval[q];
            if (v0.x == 0.0f && v0.y == 0.0f) continue;
            const float2 v = cscale(v0, tap_eval(tp, t, 2.0f * gv.sfy[q] - 1.0f));
            const int c0 = gv.slx[q] - (h - 1);
            const float tx = 2.0f * gv.sfx[q] - 1.0f;
            for (int s = 0; s < w; ++s)
                atomic_add_f2_shared(&S.buf[fft_pad<V>(wrapmod(c0 + s, nx))], cscale(v, tap_eval(tp, s, tx)));
        }
    }
    __syncthreads();
    const LineFft L{nx, lognx, S.twh, S.twl, +1.0f};
    RowOut epi{nx, Mx, r, deap_x, T};
    fft_line_epilogue<V>(S.buf, L, epi);
}

// Pass-2 epilogue: keep the M_y wanted y modes, deapodise, park them in the
// CTA's own line buffer for the cluster gather.
template <int V>
struct ColPark {
    int n, My;
    const float* deap_y;
    float2* buf;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        const int half = My >> 1;
        int jy;
        if (o < half) jy = o + half;
        else if (o >= n - half) jy = o - (n - half);
        else return;
        buf[fft_pad<V>(jy)] = cscale(v, __ldg(&deap_y[jy]));
    }
};

template <int V>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(256, 2)
k_adj_cols(const float2* __restrict__ T, int ny, int logny, int My, int Mx, FftTables tab,
           const float* __restrict__ deap_y, float2* __restrict__ img) {
    extern __shared__ float2 smem[];
    LineSmem<V> S(smem, ny);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;           // first of the cluster's 4 columns
    const int tid = threadIdx.x;
    load_twiddles(S.twh, S.twl, tab.twh, tab.twl, ny);
    float2* peer[kColCluster];
#pragma unroll
    for (int k = 0; k < kColCluster; ++k) peer[k] = cluster.map_shared_rank(S.buf, k);
    // scatter: this CTA reads rows [rank ny/4, (rank+1) ny/4) of the 4 columns
    const int rows = ny / kColCluster;
    for (int i = tid; i < rows * kColCluster; i += blockDim.x) {
        const int rr = rank * rows + i / kColCluster;
        const int k = i % kColCluster;
        peer[k][fft_pad<V>(rr)] = T[(size_t)rr * Mx + jx0 + k];
    }
    cluster.sync();
    const LineFft L{ny, logny, S.twh, S.twl, +1.0f};
    ColPark<V> epi{ny, My, deap_y, S.buf};
    fft_line_epilogue<V>(S.buf, L, epi);
    cluster.sync();
    // gather: this CTA stores image rows [rank My/4, (rank+1) My/4) of the 4 columns
    const int orows = My / kColCluster;
    for (int i = tid; i < orows * kColCluster; i += blockDim.x) {
        const int jy = rank * orows + i / kColCluster;
        const int k = i % kColCluster;
        img[(size_t)jy * Mx + jx0 + k] = peer[k][fft_pad<V>(jy)];
    }
    cluster.sync();                                    // peers may still read this CTA's buffer
}

template <int V>
__global__ void __cluster_dims__(kColCluster, 1, 1) __launch_bounds__(256, 2)
k_fwd_cols(const float2* __restrict__ img, int ny, int logny, int My, int Mx, FftTables tab,
           const float* __restrict__ deap_y, const float* __restrict__ deap_x, float2* __restrict__ T) {
    extern __shared__ float2 smem[];
    LineSmem<V> S(smem, ny);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int jx0 = (int)blockIdx.x - rank;
    const int tid = threadIdx.x;
    load_twiddles(S.twh, S.twl, tab.twh, tab.twl, ny);
    const int nsm = fft_pad_len<V>(ny);
    for (int i = tid; i < nsm; i += blockDim.x) S.buf[i] = make_float2(0.f, 0.f);
    float2* peer[kColCluster];
#pragma unroll
    for (int k = 0; k < kColCluster; ++k) peer[k] = cluster.map_shared_rank(S.buf, k);
    cluster.sync();                                    // every buffer zeroed before the scatter
    const int irows = My / kColCluster;
    const int half = My >> 1;
    for (int i = tid; i < irows * kColCluster; i += blockDim.x) {
        const int jy = rank * irows + i / kColCluster;
        const int k = i % kColCluster;
        const float d = __ldg(&deap_y[jy]) * __ldg(&deap_x[jx0 + k]);
        peer[k][fft_pad<V>(wrapmod(jy - half, ny))] = cscale(img[(size_t)jy * Mx + jx0 + k], d);
    }
    cluster.sync();
    const LineFft L{ny, logny, S.twh, S.twl, -1.0f};
    fft_line_smem<V>(S.buf, L);
    cluster.sync();
    const int rows = ny / kColCluster;
    for (int i = tid; i < rows * kColCluster; i += blockDim.x) {
        const int rr = rank * rows + i / kColCluster;
        const int k = i % kColCluster;
        T[(size_t)rr * Mx + jx0 + k] = peer[k][fft_pad<V>(rr)];
    }
    cluster.sync();
}

template <int V, bool ROWS>
__global__ void __launch_bounds__(256, 2)
k_fwd_rows(RowsView rv, GeneralView gv, const float2* __restrict__ T, int nx, int lognx, int ny, int Mx, int w,
           TapPoly tp, FftTables tab, float2* __restrict__ R, float2* __restrict__ acc) {
    extern __shared__ float2 smem[];
    LineSmem<V> S(smem, nx);
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    const int* bstart = ROWS ? rv.bucket_start : gv.bucket_start;
    if (!row_has_taps(bstart, r, ny, w)) return;
    load_twiddles(S.twh, S.twl, tab.twh, tab.twl, nx);
    const int nsm = fft_pad_len<V>(nx);
    for (int i = tid; i < nsm; i += blockDim.x) S.buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int half = Mx >> 1;
    for (int jx = tid; jx < Mx; jx += blockDim.x)
        S.buf[fft_pad<V>(wrapmod(jx - half, nx))] = T[(size_t)r * Mx + jx];
    __syncthreads();
    const LineFft L{nx, lognx, S.twh, S.twl, -1.0f};
    fft_line_smem<V>(S.buf, L);
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        const int q0 = bstart[b], q1 = bstart[b + 1];
        if (ROWS) {
            for (int q = q0; q < q1; ++q) {
                const int p = rv.bucket_rows[q];
                const float wy = tap_eval(tp, t, 2.0f * rv.row_fy[p] - 1.0f);
                const int clo = rv.row_clo[p], len = rv.row_len[p];
                float2* Rp = R + rv.row_off[p];
                for (int i = tid; i < len; i += blockDim.x) {
                    const int c = wrapmod(clo + i, nx);
                    atomic_add_f2_global(&Rp[i], cscale(S.buf[fft_pad<V>(c)], wy));
                }
            }
        } else {
            for (int q = q0 + tid; q < q1; q += blockDim.x) {
                const float wy = tap_eval(tp, t, 2.0f * gv.sfy[q] - 1.0f);
                const int c0 = gv.slx[q] - (h - 1);
                const float tx = 2.0f * gv.sfx[q] - 1.0f;
                float2 a = make_float2(0.f, 0.f);
                for (int s = 0; s < w; ++s) {
                    const float wt = tap_eval(tp, s, tx);
                    const float2 g = S.buf[fft_pad<V>(wrapmod(c0 + s, nx))];
                    a.x = fmaf(wt, g.x, a.x);
                    a.y = fmaf(wt, g.y, a.y);
                }
                atomic_add_f2_global(&acc[q], cscale(a, wy));
            }
        }
    }
}

// General points: values in bucket order, weighted and converted to FP32.
template <typename VT>
__global__ void k_gather_values(int64_t N, const int* __restrict__ perm, const void* __restrict__ values,
                                const float* __restrict__ sD, float2* __restrict__ sval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        sval[q] = cscale(ValueIO<VT>::load(values, perm[q]), sD[q]);
}

}  // namespace tffr
