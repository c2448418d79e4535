// Range-axis (x) spreading of whole pulse rows, and its transpose (the
// type-2 interpolation along x).  Every sample of a pulse row shares one
// azimuth wavenumber, so the row is first spread in 1-D onto the fine x grid
// (Algorithm 1 corrects each azimuth slice on its own); the azimuth taps are
// applied later, inside the first FFT pass.
#pragma once

#include <climits>

#include "common.cuh"
#include "kernels_points.cuh"
#include "types.cuh"

namespace tffr {


constexpr int kSpreadThreads = 256;
constexpr int kSpreadPerThread = 8;                      // samples per thread per staged tile
constexpr int kSpreadTile = kSpreadThreads * kSpreadPerThread;
// staged lam_x and values of one tile, one pad slot per 64 samples
constexpr int kSpreadStageElems = kSpreadTile + kSpreadTile / 64 + 1;
constexpr int kSpreadStageBytes = kSpreadStageElems * (int)(sizeof(double) + sizeof(float2));

// Samples whose weight needs the FP64 decision (1/G within the guard band of
// tau, a grid edge or a truncation breakpoint; rare) are not spread inline:
// k_spread_rows lists them and k_spread_deferred adds them afterwards.  The
// FP64 closed form then stays out of the hot kernel (and its registers).
struct DeferList {
    int* count;                     // [0] listed samples, [1] finished blocks of k_spread_deferred;
                                    // both zero before the spread, and left zero by k_spread_deferred
    int2* item;                     // [cap] (sample, pulse row)
    int cap;                        // N: every sample is listed at most once per adjoint
};

// Adjoint, step 1: R_p[c] = sum_{n in row p} D_n v_n phi(c - u_n) over the W
// taps of each sample.  Samples are staged tile by tile with coalesced loads;
// each thread then walks a contiguous run of samples (which move slowly along
// x) and keeps the W cells under its current footprint in registers, flushing
// a cell into the shared row (atomic add) only when the footprint moves past
// it.  D_n is evaluated inline from lam_x (tFFR mode) or read (user mode).
template <typename VT, int W>
__global__ void __launch_bounds__(kSpreadThreads, 4)
k_spread_rows(RowsView rv, int64_t N, int nx, int Mx, int My, const double* __restrict__ lam_x,
              const void* __restrict__ values, WeightArgs wa, TapPoly tp, DeferList defer, float2* __restrict__ R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s_lam = reinterpret_cast<double*>(smem_raw);
    float2* s_val = reinterpret_cast<float2*>(s_lam + kSpreadStageElems);
    float2* s_row = s_val + kSpreadStageElems;
    constexpr int H = W / 2;
    const int p = blockIdx.x;
    const int len = rv.row_len[p];
    const int clo = rv.row_clo[p];
    const bool periodic = (len == nx) && (clo == 0);
    const int64_t s0 = rv.row_start[p];
    const int64_t s1 = rv.row_end[p];
    const int L = (int)(s1 - s0);
    const int tid = threadIdx.x;
    for (int i = tid; i < len; i += kSpreadThreads) s_row[i] = make_float2(0.f, 0.f);

    // azimuth factor of the separable weight variant: one value per row
    float gy = 1.0f;
    bool gy_exact = false;
    if (wa.mode == 0 && wa.separable) gy = g_fitted(rv.row_ly[p], rv.row_fy[p], My, wa, gy_exact);

    // Thread (warp wid, lane) walks run number wid + 8 * lane of the tile: the
    // lanes of a warp are 8 runs apart, so their footprints (and the shared
    // adds of their flushes) rarely overlap.
    const int run = (tid >> 5) + (kSpreadThreads / 32) * (tid & 31);
    for (int t0 = 0; t0 < L; t0 += kSpreadTile) {
        const int cnt = min(kSpreadTile, L - t0);
        const int chunk = (cnt + kSpreadThreads - 1) / kSpreadThreads;
        __syncthreads();                                   // previous tile fully consumed
        for (int i = tid; i < cnt; i += kSpreadThreads) {
            const int k = i + (i >> 6);                    // pad: strided reads below stay off one bank
            s_lam[k] = lam_x[s0 + t0 + i];
            s_val[k] = ValueIO<VT>::load(values, s0 + t0 + i);
        }
        __syncthreads();
        const int i0 = run * chunk;
        const int i1 = min(cnt, i0 + chunk);
        float2 acc[W];
#pragma unroll
        for (int s = 0; s < W; ++s) acc[s] = make_float2(0.f, 0.f);
        int wbase = INT_MIN;                               // first fine cell held in acc
        for (int i = i0; i < i1; ++i) {
            const int k = i + (i >> 6);
            const double lam = s_lam[k];
            int cell;
            float f;
            fine_coord(lam, cell, f);
            float d;
            if (wa.mode == 1) {
                d = 1.0f;
            } else if (wa.mode == 2) {
                d = wa.user_D[s0 + t0 + i];
            } else {
                bool exact = gy_exact;
                float G = g_fitted(cell, f, Mx, wa, exact) * gy;
                d = (G != 0.0f) ? __frcp_rn(G) : 0.0f;
                if (exact || !(fabsf(d - wa.tau) > wa.guard * fabsf(wa.tau))) {
                    const int slot = atomicAdd(defer.count, 1);
                    if (slot < defer.cap) defer.item[slot] = make_int2((int)(s0 + t0 + i), p);
                    continue;
                }
                if (d < wa.tau) d = 0.0f;
            }
            if (d == 0.0f) continue;
            const float2 v = cscale(s_val[k], d);
            float wt[W];
            taps_all<W>(tp, f, wt);
            const int c0 = cell - (H - 1);
            if (c0 != wbase) {
                if (wbase != INT_MIN && c0 > wbase && c0 - wbase < W) {
                    // slide the footprint right, flushing the cells it leaves
                    do {
                        const int idx = periodic ? wrapmod(wbase, nx) : (wbase - clo);
                        atomic_add_f2_shared(&s_row[idx], acc[0]);
#pragma unroll
                        for (int s = 0; s < W - 1; ++s) acc[s] = acc[s + 1];
                        acc[W - 1] = make_float2(0.f, 0.f);
                        ++wbase;
                    } while (wbase < c0);
                } else {
                    if (wbase != INT_MIN) {
#pragma unroll
                        for (int s = 0; s < W; ++s) {
                            const int idx = periodic ? wrapmod(wbase + s, nx) : (wbase + s - clo);
                            atomic_add_f2_shared(&s_row[idx], acc[s]);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < W; ++s) acc[s] = make_float2(0.f, 0.f);
                    wbase = c0;
                }
            }
#pragma unroll
            for (int s = 0; s < W; ++s) {
                acc[s].x = fmaf(wt[s], v.x, acc[s].x);
                acc[s].y = fmaf(wt[s], v.y, acc[s].y);
            }
        }
        if (wbase != INT_MIN) {
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const int idx = periodic ? wrapmod(wbase + s, nx) : (wbase + s - clo);
                atomic_add_f2_shared(&s_row[idx], acc[s]);
            }
        }
    }
    __syncthreads();
    float2* out = R + rv.row_off[p];
    for (int i = tid; i < len; i += kSpreadThreads) out[i] = s_row[i];
}

// The deferred samples of k_spread_rows: D_n decided in FP64, then added into
// their pulse-row buffers with global atomics (after k_spread_rows stored them).
template <typename VT, int W>
__global__ void __launch_bounds__(256)
k_spread_deferred(RowsView rv, int nx, int Mx, int My, const double* __restrict__ lam_x,
                  const void* __restrict__ values, WeightArgs wa, TapPoly tp, DeferList defer,
                  float2* __restrict__ R) {
    constexpr int H = W / 2;
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = *(volatile int*)defer.count;
    __syncthreads();
    const int count = min(s_count, defer.cap);
    // the last block to have read the count puts both counters back to zero
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&defer.count[1], 1) == (int)gridDim.x - 1) {
            defer.count[0] = 0;
            defer.count[1] = 0;
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int2 e = defer.item[i];
        const int n = e.x, p = e.y;
        const double lam = lam_x[n];
        int cell;
        float f;
        fine_coord(lam, cell, f);
        const float d = weight_exact(lam, rv.row_lam_y[p], Mx, My, wa);
        if (d == 0.0f) continue;
        const float2 v = cscale(ValueIO<VT>::load(values, n), d);
        float wt[W];
        taps_all<W>(tp, f, wt);
        const int len = rv.row_len[p], clo = rv.row_clo[p];
        const bool periodic = (len == nx) && (clo == 0);
        float2* out = R + rv.row_off[p];
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const int c = cell - (H - 1) + s;
            atomicAdd(&out[periodic ? wrapmod(c, nx) : (c - clo)], cscale(v, wt[s]));
        }
    }
}

// Forward, last step: y_n = D_n sum_s phi(c_s - u_n) R_p[c_s] (or without D_n).
template <typename VT, int W>
__global__ void __launch_bounds__(kSpreadThreads, 4)
k_interp_rows(RowsView rv, int64_t N, int nx, int Mx, int My, const double* __restrict__ lam_x,
              const float2* __restrict__ R, WeightArgs wa, TapPoly tp, int apply_weights, void* __restrict__ out) {
    constexpr int H = W / 2;
    const int p = blockIdx.x;
    const int len = rv.row_len[p];
    const int clo = rv.row_clo[p];
    const bool periodic = (len == nx) && (clo == 0);
    const int64_t s0 = rv.row_start[p];
    const int64_t s1 = rv.row_end[p];
    const float2* Rp = R + rv.row_off[p];
    float gy = 1.0f;
    bool gy_exact = false;
    const double lam_y_row = rv.row_lam_y[p];
    if (apply_weights && wa.mode == 0 && wa.separable) gy = g_fitted(rv.row_ly[p], rv.row_fy[p], My, wa, gy_exact);
    // y_n for one sample of this row
    auto interp = [&](int64_t n, double lam) -> float2 {
        int cell;
        float f;
        fine_coord(lam, cell, f);
        float wt[W];
        taps_all<W>(tp, f, wt);
        const int c0 = cell - (H - 1);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const int c = c0 + s;
            const float2 r = Rp[periodic ? wrapmod(c, nx) : (c - clo)];
            acc.x = fmaf(wt[s], r.x, acc.x);
            acc.y = fmaf(wt[s], r.y, acc.y);
        }
        float d = 1.0f;
        if (apply_weights) {
            if (wa.mode == 2) {
                d = wa.user_D[n];
            } else if (wa.mode == 0) {
                bool exact = gy_exact;
                float G = g_fitted(cell, f, Mx, wa, exact) * gy;
                d = (G != 0.0f) ? __frcp_rn(G) : 0.0f;
                if (exact || !(fabsf(d - wa.tau) > wa.guard * fabsf(wa.tau)))
                    d = weight_exact(lam, lam_y_row, Mx, My, wa);
                else if (d < wa.tau)
                    d = 0.0f;
            }
        }
        return cscale(acc, d);
    };
    // two samples per thread and iteration (two independent chains of loads);
    // the next iteration's coordinates are loaded before this iteration's work
    const int64_t step = blockDim.x;
    int64_t n = s0 + threadIdx.x;
    double lam0 = (n < s1) ? lam_x[n] : 0.0;
    double lam1 = (n + step < s1) ? lam_x[n + step] : 0.0;
    for (; n < s1; n += 2 * step) {
        const int64_t n1 = n + step;
        const bool two = n1 < s1;
        const int64_t m = n + 2 * step;
        const double next0 = (m < s1) ? lam_x[m] : 0.0;
        const double next1 = (m + step < s1) ? lam_x[m + step] : 0.0;
        const float2 y0 = interp(n, lam0);
        const float2 y1 = interp(two ? n1 : n, two ? lam1 : lam0);
        ValueIO<VT>::store(out, n, y0);
        if (two) ValueIO<VT>::store(out, n1, y1);
        lam0 = next0;
        lam1 = next1;
    }
}

// General points: values in bucket order, weighted and converted to FP32.
template <typename VT>
__global__ void k_gather_values(int64_t N, const int* __restrict__ perm, const void* __restrict__ values,
                                const float* __restrict__ sD, float2* __restrict__ sval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        sval[q] = cscale(ValueIO<VT>::load(values, perm[q]), sD[q]);
}

// Forward, general points: y_{perm[q]} = D * acc[q].
template <typename VT>
__global__ void k_unpermute_output(int64_t N, const int* __restrict__ perm, const float2* __restrict__ acc,
                                   const float* __restrict__ sD, int apply_weights, void* __restrict__ out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const float d = apply_weights ? sD[q] : 1.0f;
        ValueIO<VT>::store(out, perm[q], cscale(acc[q], d));
    }
}

}  // namespace tffr
