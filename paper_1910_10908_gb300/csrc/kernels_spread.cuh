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
constexpr int kSpreadRun = 8;                            // consecutive samples per thread per tile
constexpr int kSpreadTile = kSpreadThreads * kSpreadRun;

// Samples whose weight needs the FP64 decision (1/G within the guard band of
// tau, a grid edge or a truncation breakpoint; rare) are not spread inline:
// the runs list them in their pulse row's own region of the list (one slot
// per sample of the row), and the block that spreads the row adds them after
// its runs, before it stores the row (spread_deferred_row), with D_n from
// the FP64 closed form.  The closed form then stays out of the runs (and their
// registers), and no other launch or global atomic is needed.
struct RowDefer {
    int* count;                     // shared memory: samples of the row listed so far, zero before its runs
    int* item;                      // the whole list; the row's region starts at the run's n0 in MODE 0
};

// One thread's run of up to kSpreadRun consecutive samples of a pulse row
// (samples move slowly along x: a run usually spans under two fine cells).
// The run accumulates into W + 1 register cells from its first sample's first
// tap cell `base`: a sample whose first tap cell is base + dlt, dlt in {0, 1},
// adds tap s into cell s + dlt (a select, no branch); a sample further right
// flushes the window into the shared row and starts a new one (rare).  D_n:
// MODE 0 the tFFR weight (the direct FP32 fit of 1/G times the row's azimuth
// factor), 1 unit, 2 the caller's array.  In MODE 0 a sample whose weight
// needs the FP64 decision (near tau, off the fit's first piece or on a
// truncation breakpoint, near a grid edge for rows not inside the grid's
// interior, or with |2 lam| outside the fast coordinate split) is listed for
// the block's deferred samples and adds nothing here.  The per-sample path has two
// branches, both rarely taken: the listing and the window flush.
// Sample i of the run comes from src.lam(i), src.val(i) (the caller's arrays
// or a staged copy in shared memory).  n0: in MODE 2 the index of the row's
// first sample in user_D; in MODE 0 the first slot of the row's region of the
// deferred list (a row of L samples owns L slots).
template <typename VT, int W, int MODE, typename Src>
__device__ __forceinline__ void spread_run(int64_t n0, int i0, int i1, int nx, int clo, int len, bool periodic,
                                           int Mx, bool edges, float dy, bool dy_exact, const Src& src,
                                           const WeightArgs& wa, const TapPoly& tp, const RowDefer& defer,
                                           float2* s_row, const float* __restrict__ user_D) {
    constexpr int H = W / 2;
    constexpr int kNoBase = -(1 << 30);                // below every cell (|cell| < 2^29), no overflow
    float2 acc[W + 1];
#pragma unroll
    for (int s = 0; s <= W; ++s) acc[s] = make_float2(0.f, 0.f);
    int base = kNoBase;
    // cells base .. base + W - 1 lie inside the row buffer (every sample's taps
    // do); cell base + W only when some sample used it, so it is checked
    auto flush = [&]() {
#pragma unroll
        for (int s = 0; s <= W; ++s) {
            const int c = base + s;
            const int idx = periodic ? wrapmod(c, nx) : (c - clo);
            if (s < W || idx < len) atomic_add_f2_shared(&s_row[idx], acc[s]);
            acc[s] = make_float2(0.f, 0.f);
        }
    };
    // grid-edge test as one unsigned compare: image cell j0 = floor(lam) needs
    // the FP64 decision unless e_lo <= j0 < e_lo + e_span (rows inside the
    // interior: never)
    int e_lo = -(1 << 30);
    unsigned e_span = 1u << 31;
    if (MODE == 0 && edges) {
        e_lo = wa.reach - Mx / 2;
        e_span = (unsigned)max(0, (Mx - Mx / 2 - wa.reach) - e_lo);
    }
    const float tau_band = wa.guard * fabsf(wa.tau);
    int prev = clo + (H - 1);                          // a cell whose taps lie in the row
    for (int i = i0; i < i1; ++i) {
        const int64_t n = n0 + i;
        const double lam = src.lam(i);
        const float2 v0 = src.val(i);
        int cell;
        unsigned F;
        const bool fast = fixed_coord_fast(lam, cell, F);
        float d;
        if constexpr (MODE == 0) {
            // a sample without the fast split is deferred: it keeps the previous
            // cell (its window stays put) and adds nothing here
            cell = fast ? cell : prev;
            bool exact = dy_exact | ((unsigned)((cell >> 1) - e_lo) >= e_span);
            d = d_fixed0(cell, F, wa, exact) * dy;
            if (!fast | exact | !(fabsf(d - wa.tau) > tau_band)) {
                const int slot = atomicAdd(defer.count, 1);
                defer.item[n0 + slot] = i;
                d = 0.0f;
            }
            d = (d >= wa.tau) ? d : 0.0f;
        } else {
            if (!fast) fixed_coord_general(lam, cell, F);
            d = (MODE == 1) ? 1.0f : __ldg(&user_D[n]);
        }
        prev = cell;
        const float t = fmaf(__uint2float_rn(F), 0x1p-31f, -1.0f);   // 2 f - 1
        const float2 v = cscale(v0, d);
        float wt[W];
        taps_all_t<W>(tp, t, wt);
        const int c0 = cell - (H - 1);
        int dlt = c0 - base;
        if ((unsigned)dlt > 1u) {                      // first sample of the run, or a jump: new window
            if (base != kNoBase) flush();
            base = c0;
            dlt = 0;
        }
        const bool one = dlt != 0;
        acc[0].x = fmaf(one ? 0.0f : wt[0], v.x, acc[0].x);
        acc[0].y = fmaf(one ? 0.0f : wt[0], v.y, acc[0].y);
#pragma unroll
        for (int s = 1; s < W; ++s) {
            const float w_s = one ? wt[s - 1] : wt[s];
            acc[s].x = fmaf(w_s, v.x, acc[s].x);
            acc[s].y = fmaf(w_s, v.y, acc[s].y);
        }
        acc[W].x = fmaf(one ? wt[W - 1] : 0.0f, v.x, acc[W].x);
        acc[W].y = fmaf(one ? wt[W - 1] : 0.0f, v.y, acc[W].y);
    }
    if (base != kNoBase) flush();
}

// A staged value (the caller's bytes in shared memory) as FP32 complex.
__device__ __forceinline__ float2 to_f2(const float2& v) { return v; }
__device__ __forceinline__ float2 to_f2(const double2& v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 to_f2(const __half2& v) { return __half22float2(v); }
__device__ __forceinline__ float2 to_f2(const __nv_bfloat162& v) { return __bfloat1622float2(v); }

// The row's listed samples, after every run of the block and before the row
// is stored: D_n from the FP64 closed form (the definition the fitted weight
// approximates), then added into the shared row.  item: the row's region of
// the list (indices of samples within the row); lam_row, val_row: the row's
// coordinates and values in global memory; lam_y: its azimuth coordinate
// (separable weights).  Not inlined, and without the fitted-weight path: the
// runs' registers stay those of the runs.
template <typename VT, int W>
__device__ __noinline__ void spread_deferred_row(int count, const int* __restrict__ item,
                                                 const double* __restrict__ lam_row, const VT* __restrict__ val_row,
                                                 double lam_y, int Mx, int My, int nx, int clo, bool periodic,
                                                 const WeightArgs& wa, const TapPoly& tp, float2* s_row) {
    constexpr int H = W / 2;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        const int i = item[k];
        const double lam = lam_row[i];
        const float d = weight_exact(lam, lam_y, Mx, My, wa);
        if (d == 0.0f) continue;
        int cell;
        float f;
        fine_coord(lam, cell, f);
        const float2 v = cscale(to_f2(val_row[i]), d);
        float wt[W];
        taps_all<W>(tp, f, wt);
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const int c = cell - (H - 1) + s;
            atomic_add_f2_shared(&s_row[periodic ? wrapmod(c, nx) : (c - clo)], cscale(v, wt[s]));
        }
    }
}

// A tile of samples staged in shared memory, element i at i + i / kSpreadPadEvery
// (the runs a warp's lanes read at once then fall on different banks).
constexpr int kSpreadPadEvery = 8 * kSpreadRun;
__host__ __device__ constexpr int spread_pad(int i) { return i + i / kSpreadPadEvery; }
constexpr int kSpreadStageElems = (spread_pad(kSpreadTile - 1) + 2) & ~1;   // even: the values start 16-byte aligned

template <typename VT>
struct StagedSamples {
    const double* s_lam;
    const VT* s_val;
    int t0;                                            // the tile's first sample (run indices are row-relative)
    __device__ __forceinline__ double lam(int i) const { return s_lam[spread_pad(i - t0)]; }
    __device__ __forceinline__ float2 val(int i) const { return to_f2(s_val[spread_pad(i - t0)]); }
};

// Adjoint, step 1: R_p[c] = sum_{n in row p} D_n v_n phi(c - u_n) over the W
// taps of each sample.  Each tile of kSpreadTile samples is staged in shared
// memory by asynchronous copies (coalesced, every load in flight at once);
// thread (warp wid, lane) then walks run wid + 8 lane of the tile: the lanes of
// a warp are 8 runs apart, so their footprints (and the shared adds of their
// flushes) rarely overlap.
template <typename VT, int W>
__global__ void __launch_bounds__(kSpreadThreads, 4)
k_spread_rows(RowsView rv, int64_t N, int nx, int Mx, int My, const double* __restrict__ lam_x,
              const void* __restrict__ values, WeightArgs wa, TapPoly tp, int* __restrict__ defer_item,
              float2* __restrict__ R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s_lam = reinterpret_cast<double*>(smem_raw);
    VT* s_val = reinterpret_cast<VT*>(s_lam + kSpreadStageElems);
    float2* s_row = reinterpret_cast<float2*>(s_val + kSpreadStageElems);
    constexpr int H = W / 2;
    const int p = blockIdx.x;
    const int len = rv.row_len[p];
    const int clo = rv.row_clo[p];
    const bool periodic = (len == nx) && (clo == 0);
    const int64_t s0 = rv.row_start[p];
    const int L = (int)(rv.row_end[p] - s0);
    const int tid = threadIdx.x;
    __shared__ int s_ndef;
    if (tid == 0) s_ndef = 0;
    for (int i = tid; i < len; i += kSpreadThreads) s_row[i] = make_float2(0.f, 0.f);
    // row-wide weight facts: the azimuth factor of the separable variant, and
    // whether every sample of the row is at least q + 1 image cells inside the
    // grid's edges (then no sample needs the per-sample edge test)
    float dy = 1.0f;
    bool dy_exact = false;
    bool edges = true;
    if (wa.mode == 0) {
        if (wa.separable) {
            const float gy = g_fitted(rv.row_ly[p], rv.row_fy[p], My, wa, dy_exact);
            dy = (gy != 0.0f) ? __frcp_rn(gy) : 0.0f;
        }
        const int mn = clo + (H - 1), mx = clo + len - H - 1;    // fine cells of the row's samples
        edges = periodic || (mn >> 1) - wa.reach < -(Mx / 2) || (mx >> 1) + wa.reach >= Mx - Mx / 2;
    }
    __syncthreads();
    const int run = (tid >> 5) + (kSpreadThreads / 32) * (tid & 31);
    const double* __restrict__ g_lam = lam_x + s0;
    const VT* __restrict__ g_val = reinterpret_cast<const VT*>(values) + s0;
    for (int t0 = 0; t0 < L; t0 += kSpreadTile) {
        const int cnt = min(kSpreadTile, L - t0);
        __syncthreads();                                   // the previous tile is consumed
        for (int e = tid; e < cnt; e += kSpreadThreads) {
            cp_async_elem<8>(&s_lam[spread_pad(e)], &g_lam[t0 + e]);
            cp_async_elem<(int)sizeof(VT)>(&s_val[spread_pad(e)], &g_val[t0 + e]);
        }
        cp_async_wait_all();
        __syncthreads();
        // a short tile spreads its samples over every thread: runs of
        // ceil(cnt / threads) samples (at most kSpreadRun)
        const int rl = min(kSpreadRun, (cnt + kSpreadThreads - 1) / kSpreadThreads);
        const int i0 = t0 + run * rl;
        const int i1 = min(t0 + cnt, i0 + rl);
        if (i0 >= i1) continue;
        const StagedSamples<VT> src{s_lam, s_val, t0};
        const RowDefer rd{&s_ndef, defer_item};
        if (wa.mode == 0)
            spread_run<VT, W, 0>(s0, i0, i1, nx, clo, len, periodic, Mx, edges, dy, dy_exact, src, wa, tp, rd,
                                 s_row, wa.user_D);
        else if (wa.mode == 1)
            spread_run<VT, W, 1>(s0, i0, i1, nx, clo, len, periodic, Mx, edges, dy, dy_exact, src, wa, tp, rd,
                                 s_row, wa.user_D);
        else
            spread_run<VT, W, 2>(s0, i0, i1, nx, clo, len, periodic, Mx, edges, dy, dy_exact, src, wa, tp, rd,
                                 s_row, wa.user_D);
    }
    __syncthreads();
    const int ndef = s_ndef;
    if (ndef > 0) {
        spread_deferred_row<VT, W>(ndef, defer_item + s0, g_lam, g_val, rv.row_lam_y[p], Mx, My, nx, clo, periodic,
                                   wa, tp, s_row);
        __syncthreads();
    }
    float2* out = R + rv.row_off[p];
    for (int i = tid; i < len; i += kSpreadThreads) out[i] = s_row[i];
}

// The interpolation's listed samples (after the block's loop): y_n from the
// exact fine cell, its taps and D_n by the FP64 closed form.  Not inlined: the
// loop's registers stay those of the loop.
template <typename VT, int W>
__device__ __noinline__ void interp_listed_row(int count, const int* __restrict__ item,
                                               const double* __restrict__ lam_row, const float2* __restrict__ Rp,
                                               int nx, int clo, bool periodic, double lam_y, int Mx, int My,
                                               const WeightArgs& wa, const TapPoly& tp, void* __restrict__ out,
                                               int64_t s0) {
    constexpr int H = W / 2;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        const int i = item[k];
        const double lam = lam_row[i];
        int cell;
        float f;
        fine_coord(lam, cell, f);
        float wt[W];
        taps_all<W>(tp, f, wt);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const int c = cell - (H - 1) + s;
            const float2 r = Rp[periodic ? wrapmod(c, nx) : (c - clo)];
            acc.x = fmaf(wt[s], r.x, acc.x);
            acc.y = fmaf(wt[s], r.y, acc.y);
        }
        ValueIO<VT>::store(out, s0 + i, cscale(acc, weight_exact(lam, lam_y, Mx, My, wa)));
    }
}

// Forward, last step: y_n = D_n sum_s phi(c_s - u_n) R_p[c_s] (or without D_n).
// GRAD: the gradient of a real loss with respect to real weights D instead,
// grad[n] = Re(conj(a_n) y_n) with a_n the unweighted sum and y_n read from y_in
// (in the value type VT).  The sample's fine cell and offset come from the
// branch-free fixed-point split; in tFFR mode D_n is the direct fit of 1/G
// (times the row's azimuth factor), and a sample that needs the FP64 decision
// (or lacks the fast split) is listed in its row's region of defer_item and
// recomputed after the loop (interp_listed_row), as in the spread.
template <typename VT, int W, bool GRAD = false>
__global__ void __launch_bounds__(kSpreadThreads, 4)
k_interp_rows(RowsView rv, int64_t N, int nx, int Mx, int My, const double* __restrict__ lam_x,
              const float2* __restrict__ R, WeightArgs wa, TapPoly tp, int apply_weights,
              int* __restrict__ defer_item, void* __restrict__ out, const void* __restrict__ y_in = nullptr) {
    constexpr int H = W / 2;
    const int p = blockIdx.x;
    const int len = rv.row_len[p];
    const int clo = rv.row_clo[p];
    const bool periodic = (len == nx) && (clo == 0);
    const int64_t s0 = rv.row_start[p];
    const int64_t s1 = rv.row_end[p];
    const float2* Rp = R + rv.row_off[p];
    __shared__ int s_ndef;
    if (threadIdx.x == 0) s_ndef = 0;
    __syncthreads();
    const bool fit = !GRAD && apply_weights && wa.mode == 0;
    // row-wide facts of the fitted weight: the azimuth factor (separable
    // variant) and the grid-edge test as one unsigned compare (rows inside
    // the grid's interior: never)
    float dy = 1.0f;
    bool dy_exact = false;
    int e_lo = -(1 << 30);
    unsigned e_span = 1u << 31;
    if (fit) {
        if (wa.separable) {
            const float gy = g_fitted(rv.row_ly[p], rv.row_fy[p], My, wa, dy_exact);
            dy = (gy != 0.0f) ? __frcp_rn(gy) : 0.0f;
        }
        const int mn = clo + (H - 1), mx = clo + len - H - 1;
        if (periodic || (mn >> 1) - wa.reach < -(Mx / 2) || (mx >> 1) + wa.reach >= Mx - Mx / 2) {
            e_lo = wa.reach - Mx / 2;
            e_span = (unsigned)max(0, (Mx - Mx / 2 - wa.reach) - e_lo);
        }
    }
    const float tau_band = wa.guard * fabsf(wa.tau);
    const int safe = clo + (H - 1);                    // a cell whose taps lie in the row
    // y for sample n; listed: the sample is recomputed after the loop
    auto interp = [&](int64_t n, double lam, bool& listed) -> float2 {
        int cell;
        unsigned F;
        const bool fast = fixed_coord_fast(lam, cell, F);
        float d = 1.0f;
        listed = false;
        if (fit) {
            cell = fast ? cell : safe;
            bool exact = dy_exact | ((unsigned)((cell >> 1) - e_lo) >= e_span);
            d = d_fixed0(cell, F, wa, exact) * dy;
            listed = !fast | exact | !(fabsf(d - wa.tau) > tau_band);
            d = (d >= wa.tau) ? d : 0.0f;
        } else {
            if (!fast) fixed_coord_general(lam, cell, F);
            if (!GRAD && apply_weights && wa.mode == 2) d = wa.user_D[n];
        }
        const float t = fmaf(__uint2float_rn(F), 0x1p-31f, -1.0f);   // 2 f - 1
        float wt[W];
        taps_all_t<W>(tp, t, wt);
        const int c0 = cell - (H - 1);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < W; ++s) {
            const int c = c0 + s;
            const float2 r = Rp[periodic ? wrapmod(c, nx) : (c - clo)];
            acc.x = fmaf(wt[s], r.x, acc.x);
            acc.y = fmaf(wt[s], r.y, acc.y);
        }
        return cscale(acc, d);
    };
    auto list = [&](int64_t n) {
        const int slot = atomicAdd(&s_ndef, 1);
        defer_item[s0 + slot] = (int)(n - s0);
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
        bool l0, l1;
        const float2 y0 = interp(n, lam0, l0);
        const float2 y1 = interp(two ? n1 : n, two ? lam1 : lam0, l1);
        if constexpr (GRAD) {
            float* g = reinterpret_cast<float*>(out);
            const float2 v0 = ValueIO<VT>::load(y_in, n);
            g[n] = fmaf(y0.x, v0.x, y0.y * v0.y);
            if (two) {
                const float2 v1 = ValueIO<VT>::load(y_in, n1);
                g[n1] = fmaf(y1.x, v1.x, y1.y * v1.y);
            }
        } else {
            ValueIO<VT>::store(out, n, y0);
            if (two) ValueIO<VT>::store(out, n1, y1);
            if (l0) list(n);
            if (two && l1) list(n1);
        }
        lam0 = next0;
        lam1 = next1;
    }
    if (fit) {
        __syncthreads();                               // every listing and first store is done
        const int nd = s_ndef;
        if (nd > 0)
            interp_listed_row<VT, W>(nd, defer_item + s0, lam_x + s0, Rp, nx, clo, periodic, rv.row_lam_y[p], Mx,
                                     My, wa, tp, out, s0);
    }
}

// General points: values in bucket order, weighted (sD; NULL: unweighted) and converted to FP32.
template <typename VT>
__global__ void k_gather_values(int64_t N, const int* __restrict__ perm, const void* __restrict__ values,
                                const float* __restrict__ sD, float2* __restrict__ sval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        sval[q] = cscale(ValueIO<VT>::load(values, perm[q]), sD ? sD[q] : 1.0f);
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

// Gradient with respect to the weights, general points: grad[perm[q]] =
// Re(conj(acc[q]) y_{perm[q]}), acc the unweighted forward sum in bucket order.
template <typename VT>
__global__ void k_unpermute_grad(int64_t N, const int* __restrict__ perm, const float2* __restrict__ acc,
                                 const void* __restrict__ y_in, float* __restrict__ grad) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const int n = perm[q];
        const float2 a = acc[q], y = ValueIO<VT>::load(y_in, n);
        grad[n] = fmaf(a.x, y.x, a.y * y.y);
    }
}

}  // namespace tffr
