// Range-axis (x) spreading of whole pulse rows, and its transpose (the
// type-2 interpolation along x).  Every sample of a pulse row shares one
// azimuth wavenumber, so the row is first spread in 1-D onto the fine x grid
// (Algorithm 1 corrects each azimuth slice on its own); the azimuth taps are
// applied later, inside the first FFT pass.
#pragma once

#include "common.cuh"

namespace tffr {

struct RowsView {
    int P;                          // pulse rows
    const int* row_start;           // [P] first sample of the row (rows are contiguous runs)
    const int* row_clo;             // [P] first fine x cell of the row buffer
    const int* row_len;             // [P] cells in the row buffer (nx: periodic row)
    const int* row_ly;              // [P] fine y cell floor(2 lam_y)
    const float* row_fy;            // [P] fine y offset in [0, 1]
    const int64_t* row_off;         // [P] offset of the row buffer in R (cells)
    const int* bucket_start;        // [ny + 1] rows grouped by row_ly mod ny
    const int* bucket_rows;         // [P]
};

constexpr int kSpreadThreads = 256;

// Adjoint, step 1: R_p[c] = sum_{n in row p} D_n v_n phi(c - u_n) over the w
// taps of each sample, accumulated in shared memory, then stored contiguously.
template <typename VT>
__global__ void __launch_bounds__(kSpreadThreads)
k_spread_rows(RowsView rv, int64_t N, int nx, int w, float beta, const void* __restrict__ values,
              const float* __restrict__ D, const int* __restrict__ lx, const float* __restrict__ fx,
              float2* __restrict__ R) {
    extern __shared__ float2 s_row[];
    const int p = blockIdx.x;
    const int len = rv.row_len[p];
    const int clo = rv.row_clo[p];
    const bool periodic = (len == nx) && (clo == 0);
    const int64_t s0 = rv.row_start[p];
    const int64_t s1 = (p + 1 < rv.P) ? rv.row_start[p + 1] : N;
    for (int i = threadIdx.x; i < len; i += blockDim.x) s_row[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int L = (int)(s1 - s0);
    const int chunk = (L + blockDim.x - 1) / blockDim.x;
    const int h = w / 2;
    const float two_over_w = 2.0f / (float)w;
    // Thread t walks samples [t*chunk, (t+1)*chunk): lanes of a warp sit far
    // apart along the row, so their shared-memory adds rarely collide.
    for (int k = 0; k < chunk; ++k) {
        const int i = threadIdx.x * chunk + k;
        if (i >= L) break;
        const int64_t n = s0 + i;
        const float d = D[n];
        if (d == 0.0f) continue;
        const float2 v = cscale(ValueIO<VT>::load(values, n), d);
        const int c0 = lx[n] - (h - 1);
        const float f = fx[n];
        for (int s = 0; s < w; ++s) {
            const float wt = es_kernel((float)(s - (h - 1)) - f, beta, two_over_w);
            const int c = c0 + s;
            const int idx = periodic ? wrapmod(c, nx) : (c - clo);
            atomic_add_f2_shared(&s_row[idx], cscale(v, wt));
        }
    }
    __syncthreads();
    float2* out = R + rv.row_off[p];
    for (int i = threadIdx.x; i < len; i += blockDim.x) out[i] = s_row[i];
}

// Forward, last step: y_n = D_n sum_s phi(c_s - u_n) R_p[c_s] (or without D_n).
template <typename VT>
__global__ void __launch_bounds__(kSpreadThreads)
k_interp_rows(RowsView rv, int64_t N, int nx, int w, float beta, const float2* __restrict__ R,
              const float* __restrict__ D, int apply_weights, const int* __restrict__ lx,
              const float* __restrict__ fx, void* __restrict__ out) {
    const int p = blockIdx.x;
    const int len = rv.row_len[p];
    const int clo = rv.row_clo[p];
    const bool periodic = (len == nx) && (clo == 0);
    const int64_t s0 = rv.row_start[p];
    const int64_t s1 = (p + 1 < rv.P) ? rv.row_start[p + 1] : N;
    const float2* Rp = R + rv.row_off[p];
    const int h = w / 2;
    const float two_over_w = 2.0f / (float)w;
    for (int64_t n = s0 + threadIdx.x; n < s1; n += blockDim.x) {
        const int c0 = lx[n] - (h - 1);
        const float f = fx[n];
        float2 acc = make_float2(0.f, 0.f);
        for (int s = 0; s < w; ++s) {
            const float wt = es_kernel((float)(s - (h - 1)) - f, beta, two_over_w);
            const int c = c0 + s;
            const int idx = periodic ? wrapmod(c, nx) : (c - clo);
            const float2 r = Rp[idx];
            acc.x += wt * r.x;
            acc.y += wt * r.y;
        }
        const float d = apply_weights ? D[n] : 1.0f;
        ValueIO<VT>::store(out, n, cscale(acc, d));
    }
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
