// Point preparation (coordinate -> fine-grid cell + offset, pulse-row
// detection, bucketing by grid row) and the tFFR frame weights.
#pragma once

#include "common.cuh"

namespace tffr {

// ---------------------------------------------------------------------------
// Coordinates.  u = sigma * lam (sigma = 2) in fine-grid cells, unwrapped;
// cell = floor(u) (int32), offset = u - cell in [0, 1] (FP32).  The reduction
// runs in FP64: at 8192 cells an FP32 coordinate keeps only ~1e-3 of a cell.
// A run start marks a sample whose lam_y differs (bitwise) from the previous
// sample's: runs of equal lam_y are pulse rows (azimuth is uniform, Sec. II.A).
// ---------------------------------------------------------------------------
__global__ void k_prep_points(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y,
                              double* __restrict__ keep_x, double* __restrict__ keep_y,
                              int* __restrict__ lx, float* __restrict__ fx, int* __restrict__ ly,
                              float* __restrict__ fy, uint8_t* __restrict__ run_start, int* __restrict__ err) {
    const double lim = 268435456.0;   // |lam| < 2^28 keeps 2 lam in int32
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const double a = lam_x[n], b = lam_y[n];
        keep_x[n] = a;
        keep_y[n] = b;
        int cx = 0, cy = 0;
        float ox = 0.f, oy = 0.f;
        if (!(fabs(a) < lim) || !(fabs(b) < lim)) {   // also catches NaN
            atomicOr(err, 1);
        } else {
            const double u = 2.0 * a, v = 2.0 * b;
            const double fu = floor(u), fv = floor(v);
            cx = (int)fu;
            cy = (int)fv;
            ox = (float)(u - fu);
            oy = (float)(v - fv);
        }
        lx[n] = cx;
        fx[n] = ox;
        ly[n] = cy;
        fy[n] = oy;
        uint8_t s = 1;
        if (n > 0) s = (__double_as_longlong(b) != __double_as_longlong(lam_y[n - 1])) ? 1 : 0;
        run_start[n] = s;
    }
}

// ---------------------------------------------------------------------------
// Order-preserving compaction of run starts (three-pass block scan).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int x, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int before = (wid > 0 ? s_warp[wid - 1] : 0) + v - x;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_count_flags(int64_t N, const uint8_t* __restrict__ flag, int* __restrict__ tile_count) {
    __shared__ int s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int c = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t n = base + (int64_t)threadIdx.x * kScanItems + i;
        if (n < N) c += flag[n];
    }
    int total;
    block_exclusive_scan(c, s_warp, &total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

// Exclusive scan of tile counts in place (single block, any length); writes the sum to *sum.
__global__ void k_scan_tile_counts(int ntiles, int* __restrict__ counts, int* __restrict__ sum) {
    __shared__ int s_warp[32];
    int carry = 0;
    for (int base = 0; base < ntiles; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int x = (i < ntiles) ? counts[i] : 0;
        int total;
        const int ex = block_exclusive_scan(x, s_warp, &total);
        if (i < ntiles) counts[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *sum = carry;
}

__global__ void k_emit_run_starts(int64_t N, const uint8_t* __restrict__ flag, const int* __restrict__ tile_off,
                                  int* __restrict__ row_start) {
    __shared__ int s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int c = 0;
    uint8_t f[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t n = base + (int64_t)threadIdx.x * kScanItems + i;
        f[i] = (n < N) ? flag[n] : 0;
        c += f[i];
    }
    int total;
    int pos = tile_off[blockIdx.x] + block_exclusive_scan(c, s_warp, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (f[i]) row_start[pos++] = (int)(base + (int64_t)threadIdx.x * kScanItems + i);
    }
}

// ---------------------------------------------------------------------------
// Per pulse row: extent of its x footprint and its y cell/offset.
// row_clo: first fine cell of the 1-D row buffer; row_len: cells in it.
// A row whose footprint spans >= nx cells uses the whole periodic row
// (row_clo = 0, row_len = nx, indices reduced modulo nx).
// ---------------------------------------------------------------------------
__global__ void k_row_info(int P, int64_t N, int nx, int w, const int* __restrict__ row_start,
                           const int* __restrict__ lx, const int* __restrict__ ly, const float* __restrict__ fy,
                           int* __restrict__ row_clo, int* __restrict__ row_len, int* __restrict__ row_ly,
                           float* __restrict__ row_fy) {
    __shared__ int s_min[32], s_max[32];
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        const int64_t s = row_start[p];
        const int64_t e = (p + 1 < P) ? row_start[p + 1] : N;
        int mn = 0x7fffffff, mx = -0x7fffffff;
        for (int64_t n = s + threadIdx.x; n < e; n += blockDim.x) {
            const int c = lx[n];
            mn = min(mn, c);
            mx = max(mx, c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            s_min[wid] = mn;
            s_max[wid] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
                mn = min(mn, s_min[i]);
                mx = max(mx, s_max[i]);
            }
            const int h = w / 2;
            const long long span = (long long)mx - (long long)mn + w;
            if (span >= nx) {
                row_clo[p] = 0;
                row_len[p] = nx;
            } else {
                row_clo[p] = mn - (h - 1);
                row_len[p] = (int)span;
            }
            row_ly[p] = ly[s];
            row_fy[p] = fy[s];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Bucketing by fine-grid row (general points): histogram, then scatter.
// ---------------------------------------------------------------------------
__global__ void k_bucket_hist(int64_t N, int ny, const int* __restrict__ ly, int* __restrict__ hist) {
    extern __shared__ int s_hist[];
    for (int i = threadIdx.x; i < ny; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&s_hist[wrapmod(ly[n], ny)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < ny; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

__global__ void k_bucket_scatter(int64_t N, int ny, const int* __restrict__ ly, const int* __restrict__ bucket_start,
                                 int* __restrict__ cursor, int* __restrict__ perm) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int b = wrapmod(ly[n], ny);
        const int pos = bucket_start[b] + atomicAdd(&cursor[b], 1);
        perm[pos] = (int)n;
    }
}

__global__ void k_gather_sorted(int64_t N, const int* __restrict__ perm, const int* __restrict__ lx,
                                const float* __restrict__ fx, const float* __restrict__ fy, int* __restrict__ slx,
                                float* __restrict__ sfx, float* __restrict__ sfy) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const int n = perm[q];
        slx[q] = lx[n];
        sfx[q] = fx[n];
        sfy[q] = fy[n];
    }
}

// ---------------------------------------------------------------------------
// tFFR weights (Algorithm 1, Sec. III.B-C), FP64:
//   w_hat(xi)  = 2 [a + e^{-a/2}(-a cos(pi xi) + 2 pi xi sin(pi xi))] / (a^2 + 4 pi^2 xi^2)
//   psi(eta)   = 2 [-a + e^{a/2}(a cos(pi eta) + 2 pi eta sin(pi eta))] / (a^2 + 4 pi^2 eta^2)
//   G(lam)     = sum over grid points l in [-M/2, M/2) with |lam - l| < q of psi(lam - l) w_hat(l - lam)
//   D          = R_tau(1/G)  (0 when G = 0; kept when 1/G >= tau)
// These are the transforms of the window w(t) = exp(-a|t|) and of 1/w on the
// centred domain t in [-1/2, 1/2] (Eq. (Psi); the window of Sec. IV).
// ---------------------------------------------------------------------------
struct WeightParams {
    int mode;          // 0 tFFR, 1 unit, 2 user
    int separable;     // 0 range only, 1 product of range and azimuth factors
    double a, q, tau;
    double e_minus, e_plus;   // exp(-a/2), exp(+a/2)
    const float* user_D;
};

__device__ __forceinline__ double window_hat(double xi, const WeightParams& p) {
    double s, c;
    sincospi(xi, &s, &c);
    const double two_pi = 6.283185307179586476925286766559;
    const double num = p.a + p.e_minus * (-p.a * c + two_pi * xi * s);
    return 2.0 * num / (p.a * p.a + two_pi * two_pi * xi * xi);
}

__device__ __forceinline__ double inv_window_hat(double eta, const WeightParams& p) {
    double s, c;
    sincospi(eta, &s, &c);
    const double two_pi = 6.283185307179586476925286766559;
    const double num = -p.a + p.e_plus * (p.a * c + two_pi * eta * s);
    return 2.0 * num / (p.a * p.a + two_pi * two_pi * eta * eta);
}

__device__ double diag_psi_w(double lam, int M, const WeightParams& p) {
    const double base = floor(lam);
    const int reach = (int)ceil(p.q) + 1;
    const double lo = -(double)(M / 2), hi = (double)(M - M / 2);
    double G = 0.0;
    for (int off = -reach; off <= reach; ++off) {
        const double l = base + off;
        if (l < lo || l >= hi) continue;
        const double eta = lam - l;
        if (!(fabs(eta) < p.q)) continue;
        G += inv_window_hat(eta, p) * window_hat(-eta, p);
    }
    return G;
}

__global__ void k_weights(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y, int Mx,
                          int My, WeightParams p, float* __restrict__ D, unsigned long long* __restrict__ kept) {
    int c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        double d;
        if (p.mode == 1) {
            d = 1.0;
        } else if (p.mode == 2) {
            d = (double)p.user_D[n];
        } else {
            double G = diag_psi_w(lam_x[n], Mx, p);
            if (p.separable) G *= diag_psi_w(lam_y[n], My, p);
            d = (G != 0.0) ? 1.0 / G : 0.0;
            if (!(d >= p.tau)) d = 0.0;
        }
        D[n] = (float)d;
        c += (d != 0.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(kept, (unsigned long long)c);
}

__global__ void k_gather_weights(int64_t N, const int* __restrict__ perm, const float* __restrict__ D,
                                 float* __restrict__ sD) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        sD[q] = D[perm[q]];
}

}  // namespace tffr
