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
//     x, keep the M_x wanted modes, multiply by 1/phi_hat(kx), store into the
//     intermediate T.
//   pass 2 (one CTA per wanted x mode): FFT along y, keep the M_y wanted modes,
//     multiply by 1/phi_hat(ky), store the image column.
//
// The forward runs the transposed steps in reverse order with FFT sign -1.
//
// Layout of T: [Mx/16][ny][16] complex64, i.e. T(r, jx) at
// ((jx / 16) * ny + r) * 16 + jx % 16.  Pass 1 stores 128-byte lines (16 x
// modes of one row); the 16 column CTAs of a line group read the same lines.
#pragma once

#include "common.cuh"
#include "fft_smem.cuh"
#include "kernels_spread.cuh"

namespace tffr {

struct GeneralView {
    const int* bucket_start;   // [ny + 1] samples grouped by floor(2 lam_y) mod ny
    const int* perm;           // [N] sorted position -> sample index
    const int* slx;            // [N] fine x cell, sorted order
    const float* sfx;          // [N] fine x offset, sorted order
    const float* sfy;          // [N] fine y offset, sorted order
    const float* sD;           // [N] weights, sorted order
};

__device__ __forceinline__ size_t t_index(int jx, int r, int ny) {
    return ((size_t)(jx >> 4) * (size_t)ny + (size_t)r) * kColGroup + (size_t)(jx & (kColGroup - 1));
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

// Shared tail of the adjoint row pass: FFT along x, keep the Mx wanted modes,
// deapodise, store row r of T.
__device__ __forceinline__ void adj_row_finish(float2* sm, int r, int nx, int lognx, int ny, int Mx,
                                               const float2* __restrict__ twx, const float* __restrict__ deap_x,
                                               float2* __restrict__ T) {
    fft_smem(sm, nx, lognx, twx, +1.0f);
    const int half = Mx >> 1;
    for (int jx = threadIdx.x; jx < Mx; jx += kFftThreads) {
        const float2 v = sm[pad16(wrapmod(jx - half, nx))];
        T[t_index(jx, r, ny)] = cscale(v, deap_x[jx]);
    }
}

// Pass 1 of the adjoint, pulse rows: fine row r = sum over the pulse rows p
// whose azimuth taps reach r of phi_y(r - v_p) R_p (shifted to its x cells).
__global__ void __launch_bounds__(kFftThreads)
k_adj_rows(RowsView rv, const float2* __restrict__ R, int nx, int lognx, int ny, int Mx, int w, TapPoly tp,
           const float2* __restrict__ twx, const float* __restrict__ deap_x, float2* __restrict__ T) {
    extern __shared__ float2 sm[];
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (!row_has_taps(rv.bucket_start, r, ny, w)) {
        for (int jx = tid; jx < Mx; jx += kFftThreads) T[t_index(jx, r, ny)] = make_float2(0.f, 0.f);
        return;
    }
    const int nsm = nx + (nx >> 4);
    for (int i = tid; i < nsm; i += kFftThreads) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        for (int q = rv.bucket_start[b]; q < rv.bucket_start[b + 1]; ++q) {
            const int p = rv.bucket_rows[q];
            const float wy = tap_eval(tp, t, 2.0f * rv.row_fy[p] - 1.0f);
            const int clo = rv.row_clo[p], len = rv.row_len[p];
            const float2* Rp = R + rv.row_off[p];
            for (int i = tid; i < len; i += kFftThreads) {
                const int c = wrapmod(clo + i, nx);
                atomic_add_f2_shared(&sm[pad16(c)], cscale(Rp[i], wy));
            }
        }
    }
    adj_row_finish(sm, r, nx, lognx, ny, Mx, twx, deap_x, T);
}

// Pass 1 of the adjoint, general points: the samples of the w buckets whose
// taps reach fine row r are spread straight into the shared row.
template <typename VT>
__global__ void __launch_bounds__(kFftThreads)
k_adj_rows_general(GeneralView gv, const void* __restrict__ values, int nx, int lognx, int ny, int Mx, int w,
                   TapPoly tp, const float2* __restrict__ twx, const float* __restrict__ deap_x,
                   float2* __restrict__ T) {
    extern __shared__ float2 sm[];
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (!row_has_taps(gv.bucket_start, r, ny, w)) {
        for (int jx = tid; jx < Mx; jx += kFftThreads) T[t_index(jx, r, ny)] = make_float2(0.f, 0.f);
        return;
    }
    const int nsm = nx + (nx >> 4);
    for (int i = tid; i < nsm; i += kFftThreads) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int h = w / 2;
    for (int t = 0; t < w; ++t) {
        const int b = wrapmod(r + h - 1 - t, ny);
        for (int q = gv.bucket_start[b] + tid; q < gv.bucket_start[b + 1]; q += kFftThreads) {
            const float d = gv.sD[q];
            if (d == 0.0f) continue;
            const float wy = tap_eval(tp, t, 2.0f * gv.sfy[q] - 1.0f);
            const float2 v = cscale(ValueIO<VT>::load(values, gv.perm[q]), d * wy);
            const int c0 = gv.slx[q] - (h - 1);
            const float tx = 2.0f * gv.sfx[q] - 1.0f;
            for (int s = 0; s < w; ++s)
                atomic_add_f2_shared(&sm[pad16(wrapmod(c0 + s, nx))], cscale(v, tap_eval(tp, s, tx)));
        }
    }
    adj_row_finish(sm, r, nx, lognx, ny, Mx, twx, deap_x, T);
}

__global__ void __launch_bounds__(kFftThreads)
k_adj_cols(const float2* __restrict__ T, int ny, int logny, int My, int Mx, const float2* __restrict__ twy,
           const float* __restrict__ deap_y, float2* __restrict__ img) {
    extern __shared__ float2 sm[];
    const int jx = blockIdx.x;
    const int tid = threadIdx.x;
    const float2* col = T + t_index(jx, 0, ny);
    for (int r = tid; r < ny; r += kFftThreads) sm[pad16(r)] = col[(size_t)r * kColGroup];
    fft_smem(sm, ny, logny, twy, +1.0f);
    const int half = My >> 1;
    for (int jy = tid; jy < My; jy += kFftThreads) {
        const float2 v = sm[pad16(wrapmod(jy - half, ny))];
        img[(size_t)jy * Mx + jx] = cscale(v, deap_y[jy]);
    }
}

__global__ void __launch_bounds__(kFftThreads)
k_fwd_cols(const float2* __restrict__ img, int ny, int logny, int My, int Mx, const float2* __restrict__ twy,
           const float* __restrict__ deap_y, const float* __restrict__ deap_x, float2* __restrict__ T) {
    extern __shared__ float2 sm[];
    const int jx = blockIdx.x;
    const int tid = threadIdx.x;
    const int nsm = ny + (ny >> 4);
    for (int i = tid; i < nsm; i += kFftThreads) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const float dx = deap_x[jx];
    const int half = My >> 1;
    for (int jy = tid; jy < My; jy += kFftThreads)
        sm[pad16(wrapmod(jy - half, ny))] = cscale(img[(size_t)jy * Mx + jx], deap_y[jy] * dx);
    fft_smem(sm, ny, logny, twy, -1.0f);
    float2* col = T + t_index(jx, 0, ny);
    for (int r = tid; r < ny; r += kFftThreads) col[(size_t)r * kColGroup] = sm[pad16(r)];
}

template <bool ROWS>
__global__ void __launch_bounds__(kFftThreads)
k_fwd_rows(RowsView rv, GeneralView gv, const float2* __restrict__ T, int nx, int lognx, int ny, int Mx, int w,
           TapPoly tp, const float2* __restrict__ twx, float2* __restrict__ R, float2* __restrict__ acc) {
    extern __shared__ float2 sm[];
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    const int* bstart = ROWS ? rv.bucket_start : gv.bucket_start;
    if (!row_has_taps(bstart, r, ny, w)) return;
    const int nsm = nx + (nx >> 4);
    for (int i = tid; i < nsm; i += kFftThreads) sm[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int half = Mx >> 1;
    for (int jx = tid; jx < Mx; jx += kFftThreads) sm[pad16(wrapmod(jx - half, nx))] = T[t_index(jx, r, ny)];
    fft_smem(sm, nx, lognx, twx, -1.0f);
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
                for (int i = tid; i < len; i += kFftThreads) {
                    const int c = wrapmod(clo + i, nx);
                    atomic_add_f2_global(&Rp[i], cscale(sm[pad16(c)], wy));
                }
            }
        } else {
            for (int q = q0 + tid; q < q1; q += kFftThreads) {
                const float wy = tap_eval(tp, t, 2.0f * gv.sfy[q] - 1.0f);
                const int c0 = gv.slx[q] - (h - 1);
                const float tx = 2.0f * gv.sfx[q] - 1.0f;
                float2 a = make_float2(0.f, 0.f);
                for (int s = 0; s < w; ++s) {
                    const float wt = tap_eval(tp, s, tx);
                    const float2 g = sm[pad16(wrapmod(c0 + s, nx))];
                    a.x = fmaf(wt, g.x, a.x);
                    a.y = fmaf(wt, g.y, a.y);
                }
                atomic_add_f2_global(&acc[q], cscale(a, wy));
            }
        }
    }
}

}  // namespace tffr
