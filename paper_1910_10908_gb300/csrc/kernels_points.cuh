// Point preparation (pulse-row detection, bucketing by fine row) and the tFFR
// frame weights.
#pragma once

#include "common.cuh"
#include "types.cuh"

namespace tffr {

// ---------------------------------------------------------------------------
// tFFR weights (Algorithm 1, Sec. III.B-C).  For a sample at frequency lam
// (grid units) on an axis with an M-point Fourier grid l in [-M/2, M/2):
//   w_hat(xi) = 2 [a + e^{-a/2}(-a cos(pi xi) + 2 pi xi sin(pi xi))] / (a^2 + 4 pi^2 xi^2)
//   psi(eta)  = 2 [-a + e^{a/2}(a cos(pi eta) + 2 pi eta sin(pi eta))] / (a^2 + 4 pi^2 eta^2)
//   G(lam)    = sum_{l on the grid, |lam - l| < q} psi(lam - l) w_hat(l - lam)
//   D         = R_tau(1 / G)      (0 when G = 0; kept when 1/G >= tau)
// These are the transforms of the window w(t) = exp(-a|t|) and of 1/w on the
// centred domain t in [-1/2, 1/2] (Eq. (Psi); the window of Sec. IV).
//
// Away from the grid edges G depends only on the offset delta = lam - floor(lam)
// and is symmetric about delta = 1/2, so the plan fits it once (FP64, on the
// host) as polynomials in v = |delta - 1/2| and evaluates those in FP32 here.
// Samples near the grid edges, on a breakpoint of the truncation, or with
// 1/G within a guard band of tau take the closed form in FP64, so the
// threshold decision is always made in FP64.
// ---------------------------------------------------------------------------
constexpr int kGCoefs = 16;
constexpr int kG0Coefs = 12;       // piece 0 (the whole range for integer q): fixed length
constexpr int kD0Coefs = 10;       // 1/G on piece 0, fitted directly (1.5e-8 at a = 0.01, q = 3)

struct WeightArgs {
    int mode;              // 0 tFFR, 1 unit, 2 user (per-sample array)
    int separable;         // 0 range only, 1 product of range and azimuth factors
    float tau, guard;      // threshold and relative guard band for the FP64 re-check
    double tau_d;
    // fitted G: piece 0 on v in [0, vb] as a polynomial in s = 2 (v/vb)^2 - 1;
    // piece 1 on v in [vb, 1/2] as a polynomial in s = (2v - vb - 1/2)/(1/2 - vb)
    float vb, inv_vb;
    int n0, n1;
    float c0[kGCoefs], c1[kGCoefs];
    float d0[kD0Coefs];    // 1/G on piece 0, same variable s (the spread's fast path)
    // closed-form parameters
    double a, q, e_minus, e_plus;
    int reach;             // ceil(q) + 1
    const float* user_D;
};

__host__ __device__ inline double wt_sinpi(double x);
__host__ __device__ inline double wt_cospi(double x);

#ifdef __CUDA_ARCH__
__device__ inline double wt_sinpi(double x) { return sinpi(x); }
__device__ inline double wt_cospi(double x) { return cospi(x); }
#else
inline double wt_sinpi(double x) {
    const double r = x - 2.0 * std::floor(0.5 * x);       // [0, 2)
    return std::sin(3.14159265358979323846 * r);
}
inline double wt_cospi(double x) {
    const double r = x - 2.0 * std::floor(0.5 * x);
    return std::cos(3.14159265358979323846 * r);
}
#endif

__host__ __device__ inline double window_hat(double xi, double a, double e_minus) {
    const double two_pi = 6.283185307179586476925286766559;
    const double num = a + e_minus * (-a * wt_cospi(xi) + two_pi * xi * wt_sinpi(xi));
    return 2.0 * num / (a * a + two_pi * two_pi * xi * xi);
}

__host__ __device__ inline double inv_window_hat(double eta, double a, double e_plus) {
    const double two_pi = 6.283185307179586476925286766559;
    const double num = -a + e_plus * (a * wt_cospi(eta) + two_pi * eta * wt_sinpi(eta));
    return 2.0 * num / (a * a + two_pi * two_pi * eta * eta);
}

// G(lam) with the grid truncation; M <= 0 means an unbounded grid.
__host__ __device__ inline double diag_psi_w(double lam, int M, double a, double q, double e_minus,
                                             double e_plus, int reach) {
    const double base = floor(lam);
    double G = 0.0;
    for (int off = -reach; off <= reach; ++off) {
        const double l = base + off;
        if (M > 0 && (l < -(double)(M / 2) || l >= (double)(M - M / 2))) continue;
        const double eta = lam - l;
        if (!(fabs(eta) < q)) continue;
        G += inv_window_hat(eta, a, e_plus) * window_hat(-eta, a, e_minus);
    }
    return G;
}

__device__ __forceinline__ float horner(const float* c, int n, float s) {
    float a = c[n - 1];
    for (int k = n - 2; k >= 0; --k) a = fmaf(a, s, c[k]);
    return a;
}

// FP32 G from the fine cell (floor(2 lam)) and offset; sets exact = true when the
// closed form must decide instead (grid edge or truncation breakpoint).
__device__ __forceinline__ float g_fitted(int cell, float f, int M, const WeightArgs& A, bool& exact) {
    const int j0 = cell >> 1;                                    // floor(lam)
    if (j0 - A.reach < -(M / 2) || j0 + A.reach >= M - M / 2) exact = true;
    const float delta = 0.5f * ((float)(cell & 1) + f);          // lam - floor(lam), exact in FP32
    const float v = fabsf(delta - 0.5f);
    if (v == A.vb || v == 0.5f) exact = true;                    // on a breakpoint of the truncation
    if (v < A.vb) {
        const float r = v * A.inv_vb;
        const float s = fmaf(2.0f * r, r, -1.0f);
        float g = A.c0[kG0Coefs - 1];
#pragma unroll
        for (int k = kG0Coefs - 2; k >= 0; --k) g = fmaf(g, s, A.c0[k]);
        return g;
    }
    return horner(A.c1, A.n1, (2.0f * v - A.vb - 0.5f) / (0.5f - A.vb));
}

// 1/G (before the threshold) by its direct fit on piece 0, from the fine
// cell and the fixed-point offset F (fixed_coord_fast): lam - floor(lam) is
// the 0.32 fixed-point number (cell & 1, F) >> 1.  No branch: a sample outside
// piece 0 (v >= vb, which includes the truncation breakpoints) sets exact, and
// its value is not used.
__device__ __forceinline__ float d_fixed0(int cell, unsigned F, const WeightArgs& A, bool& exact) {
    const unsigned D = __funnelshift_r(F, (unsigned)cell, 1);
    const float v = fabsf(fmaf(__uint2float_rn(D), 0x1p-32f, -0.5f));   // |lam - floor(lam) - 1/2|
    exact |= !(v < A.vb);
    const float r = v * A.inv_vb;
    const float s = fmaf(2.0f * r, r, -1.0f);
    float d = A.d0[kD0Coefs - 1];
#pragma unroll
    for (int k = kD0Coefs - 2; k >= 0; --k) d = fmaf(d, s, A.d0[k]);
    return d;
}

static __device__ __noinline__ float weight_exact_args(double lam_x, double lam_y, int Mx, int My, double a, double q,
                                                double e_minus, double e_plus, int reach, double tau, int separable) {
    double G = diag_psi_w(lam_x, Mx, a, q, e_minus, e_plus, reach);
    if (separable) G *= diag_psi_w(lam_y, My, a, q, e_minus, e_plus, reach);
    double d = (G != 0.0) ? 1.0 / G : 0.0;
    if (!(d >= tau)) d = 0.0;
    return (float)d;
}

// D_n by the closed form in FP64 (the FP64 decision path).
__device__ __forceinline__ float weight_exact(double lam_x, double lam_y, int Mx, int My, const WeightArgs& A) {
    return weight_exact_args(lam_x, lam_y, Mx, My, A.a, A.q, A.e_minus, A.e_plus, A.reach, A.tau_d, A.separable);
}

// D_n in tFFR mode from the x cell/offset (and the y ones in separable mode).
__device__ __forceinline__ float weight_tffr(double lam_x, int cx, float fx, double lam_y, int cy, float fy, int Mx,
                                             int My, const WeightArgs& A) {
    bool exact = false;
    float G = g_fitted(cx, fx, Mx, A, exact);
    if (A.separable) G *= g_fitted(cy, fy, My, A, exact);
    const float d = (G != 0.0f) ? __frcp_rn(G) : 0.0f;
    if (!exact && fabsf(d - A.tau) > A.guard * fabsf(A.tau)) return (d >= A.tau) ? d : 0.0f;
    return weight_exact(lam_x, lam_y, Mx, My, A);
}

// ---------------------------------------------------------------------------
// Pulse rows: runs of samples with bit-equal lam_y (azimuth is uniform,
// Sec. II.A).  One pass over both coordinate arrays finds the run starts,
// checks every coordinate and takes each run's extent of fine x cells.
// Tiles number their runs from one atomic counter (row ids follow sample
// order inside a tile, not across tiles: nothing downstream needs more), so
// no tile waits on another; k_row_finish then hands each tile's leading
// samples to the row they continue and closes each tile's last row.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;                     // single-block scans below

// Exclusive scan of one int per thread across the block; *total = block sum.
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

constexpr int kRowScanWarps = 8;
constexpr int kRowScanK = 8;                           // samples per lane
constexpr int kRowScanTile = kRowScanWarps * 32 * kRowScanK;
constexpr int kIntMax = 0x7fffffff, kIntMin = -0x7fffffff - 1;

struct RowScanArgs {
    int* row_start;                                    // [cap] first sample of each row
    int* row_end;                                      // [cap] one past its last sample
    int* row_min;                                      // [cap] smallest fine x cell, kIntMax at entry
    int* row_max;                                      // [cap] largest fine x cell, kIntMin at entry
    int cap;
    int4* tile;                                        // [tiles] first row id (-1: none), last row id, first row start
    int2* head;                                        // [tiles] cell extent of the samples before the first start
    int* flags;                                        // [0] error bits, [1] rows, [3] overflow
    // zeroed by the scan for the kernels after it (no separate memset launches)
    int* zero_i;                                       // [n_zero_i] the per-fine-row and per-cell counters
    int n_zero_i;
    float4* zero_w;                                    // [n_zero_w] the fine-row tap weights
    int n_zero_w;
};

// Error bits: 1 bad lam_y, 2 bad lam_x.  Local run index -1 marks the samples
// of a tile that continue a row started in an earlier tile.
static __global__ void __launch_bounds__(kRowScanWarps * 32, 4)
k_scan_rows(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y, RowScanArgs a) {
    __shared__ int s_cnt[kRowScanWarps];
    __shared__ int s_base, s_first, s_hmin, s_hmax;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    const int64_t wbase = (int64_t)tile * kRowScanTile + (int64_t)wid * (32 * kRowScanK);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_zero_i; i += gridDim.x * blockDim.x) a.zero_i[i] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_zero_w; i += gridDim.x * blockDim.x)
        a.zero_w[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) {
        s_first = -1;
        s_hmin = kIntMax;
        s_hmax = kIntMin;
    }
    unsigned ball[kRowScanK];
    int cx[kRowScanK];
    bool bad_x = false, bad_y = false;
    int cnt = 0;
    // 32-bit offsets from the warp's first sample; rem = samples left from there
    const int64_t left = N - wbase;
    const int rem = left <= 0 ? 0 : (left >= 32 * kRowScanK ? 32 * kRowScanK : (int)left);
    const double* __restrict__ wy = lam_y + wbase;
    const double* __restrict__ wx = lam_x + wbase;
    long long prev = (wbase > 0 && rem > 0) ? __double_as_longlong(__ldg(wy - 1)) : 0;
#pragma unroll
    for (int h = 0; h < kRowScanK; h += 8) {
        long long yb[8];
        double xv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int o = (h + k) * 32 + lane;
            yb[k] = (o < rem) ? __double_as_longlong(__ldg(wy + o)) : 0;
            xv[k] = (o < rem) ? __ldg(wx + o) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int o = (h + k) * 32 + lane;
            long long up = __shfl_up_sync(FULL, yb[k], 1);
            if (lane == 0) up = prev;
            prev = __shfl_sync(FULL, yb[k], 31);
            const bool in = o < rem;
            ball[h + k] = __ballot_sync(FULL, in && ((wbase == 0 && o == 0) || yb[k] != up));
            cnt += __popc(ball[h + k]);
            int c = 0;
            if (in) {
                bad_y |= !coord_in_range(__longlong_as_double(yb[k]));
                bad_x |= !fine_cell(xv[k], c);
            }
            cx[h + k] = c;
        }
    }
    if (bad_y) atomicOr(&a.flags[0], 1);
    if (bad_x) atomicOr(&a.flags[0], 2);
    if (lane == 0) s_cnt[wid] = cnt;
    __syncthreads();
    int woff = 0, agg = 0;
#pragma unroll
    for (int i = 0; i < kRowScanWarps; ++i) {
        const int t = s_cnt[i];
        woff += (i < wid) ? t : 0;
        agg += t;
    }
    if (threadIdx.x == 0) s_base = agg ? atomicAdd(&a.flags[1], agg) : 0;
    __syncthreads();
    const int base = s_base;
    // emit the starts, close the rows that end inside the tile, and fold each
    // lane's cells into the extent of its row (a lane's run index only grows)
    const unsigned le = FULL >> (31 - lane);
    constexpr int kNone = -2;
    int pre = woff;
    int cur = kNone, mn = kIntMax, mx = kIntMin;
    bool over = false;
    auto flush = [&](int local, int lo, int hi) {
        if (local < 0) {
            atomicMin(&s_hmin, lo);
            atomicMax(&s_hmax, hi);
        } else if (base + local < a.cap) {
            atomicMin(&a.row_min[base + local], lo);
            atomicMax(&a.row_max[base + local], hi);
        } else {
            over = true;
        }
    };
    const int nbase = (int)wbase;                      // N < 2^31
    unsigned starts = 0;
#pragma unroll
    for (int k = 0; k < kRowScanK; ++k) starts |= ball[k];
    if (starts == 0) {
        // no run starts among the warp's samples (the common case): all of
        // them continue run woff - 1, whose extent takes the warp's min / max
#pragma unroll
        for (int k = 0; k < kRowScanK; ++k)
            if (k * 32 + lane < rem) {
                mn = min(mn, cx[k]);
                mx = max(mx, cx[k]);
            }
        const int m0 = __reduce_min_sync(FULL, mn), m1 = __reduce_max_sync(FULL, mx);
        if (lane == 0 && rem > 0) flush(woff - 1, m0, m1);
    } else {
#pragma unroll
        for (int k = 0; k < kRowScanK; ++k) {
            const int o = k * 32 + lane;
            const int n = nbase + o;
            const int local = pre + __popc(ball[k] & le) - 1;
            if (o < rem) {
                if ((ball[k] >> lane) & 1u) {
                    const int p = base + local;
                    if (p < a.cap) a.row_start[p] = n;
                    else over = true;
                    if (local > 0) {
                        if (p - 1 < a.cap) a.row_end[p - 1] = n;
                    } else {
                        s_first = n;
                    }
                }
                if (local != cur) {
                    if (cur != kNone) flush(cur, mn, mx);
                    cur = local;
                    mn = mx = cx[k];
                } else {
                    mn = min(mn, cx[k]);
                    mx = max(mx, cx[k]);
                }
            }
            pre += __popc(ball[k]);
        }
        if (__all_sync(FULL, cur == __shfl_sync(FULL, cur, 0))) {
            const int m0 = __reduce_min_sync(FULL, mn), m1 = __reduce_max_sync(FULL, mx);
            if (lane == 0 && cur != kNone) flush(cur, m0, m1);
        } else if (cur != kNone) {
            flush(cur, mn, mx);
        }
    }
    if (over) atomicOr(&a.flags[3], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.tile[tile] = make_int4(agg ? base : -1, base + agg - 1, s_first, 0);
        a.head[tile] = make_int2(s_hmin, s_hmax);
    }
}

static __global__ void k_fill_int(int n, int v, int* __restrict__ a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}

// Per pulse row: the end of a row that is the last one started in its tile
// (the first start of the next tile that has one, or N), folding in the
// leading samples of the tiles up to there; the x footprint from the cell
// extent (the row buffer's first fine cell row_clo and its length row_len; a
// footprint of >= nx cells takes the whole periodic row, row_clo = 0,
// row_len = nx); the row's y cell, its w azimuth taps row_wy[p][s] =
// phi(s - (w/2 - 1) - fy) (stride 8) and the count of pulse rows reaching
// each fine row (tap_count, zeroed), and how many rows have each fine y cell
// (ly_count, zeroed).  Puts the extent arrays back to their identities for
// the next scan.  The walk over tiles is O(tiles) in total.
static __global__ void k_row_finish(const int* __restrict__ runs, int cap, int64_t N, int ntiles,
                             const int4* __restrict__ tile, const int2* __restrict__ head, int nx, int ny, int w,
                             TapPoly tp, const double* __restrict__ lam_y, const int* __restrict__ row_start,
                             int* __restrict__ row_end, int* __restrict__ row_min, int* __restrict__ row_max,
                             int* __restrict__ row_clo, int* __restrict__ row_len, int* __restrict__ row_ly,
                             float* __restrict__ row_fy, double* __restrict__ row_lam_y, float* __restrict__ row_wy,
                             int* __restrict__ tap_count, int* __restrict__ ly_count) {
    const int P = min(*runs, cap);
    const int h = w / 2;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        int mn = row_min[p], mx = row_max[p];
        row_min[p] = kIntMax;
        row_max[p] = kIntMin;
        const int s0 = row_start[p];
        const int t = s0 / kRowScanTile;
        const double ly = lam_y[s0];                   // issued with the tile's load below
        if (tile[t].y == p) {
            int t2 = t + 1;
            int e = (int)N;
            for (; t2 < ntiles; ++t2) {
                const int2 hd = head[t2];
                mn = min(mn, hd.x);
                mx = max(mx, hd.y);
                const int4 ti = tile[t2];
                if (ti.x >= 0) {
                    e = ti.z;
                    break;
                }
            }
            row_end[p] = e;
        }
        const long long span = (long long)mx - (long long)mn + w;
        if (span >= nx) {
            row_clo[p] = 0;
            row_len[p] = nx;
        } else {
            row_clo[p] = mn - (h - 1);
            row_len[p] = (int)span;
        }
        int cy;
        float fy;
        fine_coord(ly, cy, fy);
        row_ly[p] = cy;
        row_fy[p] = fy;
        row_lam_y[p] = ly;
        const float tt = 2.0f * fy - 1.0f;
#pragma unroll
        for (int s = 0; s < 8; ++s) row_wy[(size_t)p * 8 + s] = (s < w) ? tap_eval(tp, s, tt) : 0.0f;
        for (int s = 0; s < w; ++s) atomicAdd(&tap_count[wrapmod(cy - (h - 1) + s, ny)], 1);
        atomicAdd(&ly_count[wrapmod(cy, ny)], 1);
    }
}

constexpr int kScanItems = 8;                          // consecutive items per thread in a block pass
constexpr int kScanPass = kScanThreads * kScanItems;
__host__ __device__ constexpr int scan_pad(int i) { return i + (i >> 5); }
constexpr int kScanStage = scan_pad(kScanPass);        // ints of the shared staging of one pass

// Exclusive scan of in[0..n) into out[0..n) by one block, kScanPass items a
// pass.  A pass stages its items in shared memory with coalesced loads; each
// thread scans kScanItems consecutive items (one spare word per 32 keeps a
// warp's reads on distinct banks); the pass-relative results go back through
// shared memory and leave with coalesced stores.  out may be in (a pass reads
// all its items before writing any).  Starts from carry and returns the carry
// after the last item (to every thread); folds the items into mx.  The sum of
// one pass must fit an int.
template <typename OutT>
__device__ long long block_scan_items(const int* in, OutT* out, int n, long long carry, int* s_warp, int* s_items,
                                      int& mx) {
    for (int base = 0; base < n; base += kScanPass) {
        const int cnt = min(kScanPass, n - base);
        __syncthreads();                               // the previous pass's stores have read s_items
        for (int i = threadIdx.x; i < kScanPass; i += kScanThreads) s_items[scan_pad(i)] = (i < cnt) ? in[base + i] : 0;
        __syncthreads();
        const int i0 = (int)threadIdx.x * kScanItems;
        int x[kScanItems];
        int sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            x[k] = s_items[scan_pad(i0 + k)];
            mx = max(mx, x[k]);
            sum += x[k];
        }
        int tot;
        int ex = block_exclusive_scan(sum, s_warp, &tot);   // ends with a barrier: every x[] is read
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            s_items[scan_pad(i0 + k)] = ex;
            ex += x[k];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kScanThreads) out[base + i] = (OutT)(carry + s_items[scan_pad(i)]);
        carry += tot;
    }
    return carry;
}

// Three blocks, after k_row_finish, one independent scan each.  Block 0: row
// buffer offsets (exclusive scan of row_len over the P rows), their total
// and the longest row (atomic max into *max_len, zero before).  Block 1: the
// exclusive scan of the per-fine-row tap counts into tap_start[0..ny] and the
// largest count (atomic max into *max_count, zero before), after which
// tap_count is zeroed again (the per-fine-row cursor of k_ell_fill).  Block
// 2: ly_count[0..ny) replaced in place by its exclusive scan, the first place
// in fine-y order of the rows of each fine y cell.
static __global__ void __launch_bounds__(kScanThreads)
k_row_scans(const int* __restrict__ runs, int cap, const int* __restrict__ row_len, int64_t* __restrict__ row_off,
            long long* __restrict__ total, int ny, int* tap_count, int* __restrict__ tap_start,
            int* __restrict__ max_len, int* __restrict__ max_count, int* ly_count) {
    __shared__ int s_warp[32];
    __shared__ int s_items[kScanStage];
    int mx = 0;
    if (blockIdx.x == 0) {
        const int P = min(*runs, cap);
        const long long cells = block_scan_items(row_len, row_off, P, 0, s_warp, s_items, mx);
        if (threadIdx.x == 0) *total = cells;
    } else if (blockIdx.x == 1) {
        const long long taps = block_scan_items(tap_count, tap_start, ny, 0, s_warp, s_items, mx);
        if (threadIdx.x == 0) tap_start[ny] = (int)taps;
        for (int i = threadIdx.x; i < ny; i += kScanThreads) tap_count[i] = 0;   // every read is behind a barrier
    } else {
        block_scan_items(ly_count, ly_count, ny, 0, s_warp, s_items, mx);
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(blockIdx.x == 0 ? max_len : max_count, mx);
}

// Azimuth taps as a table of fixed width per fine row (pulse-row order of
// the FFT passes).  Each pulse row p first takes its place q in fine-y order,
// q = ly_first[c] + (its arrival among the rows of its fine y cell c), and
// rank_row[q] = p: the x pass puts row p at place q of F; the row's y cell
// and taps are copied to place q (q_ly, q_wy) for the forward twin.
//
// Row p reaches the fine rows c - h + 1 .. c + h (h = w / 2, modulo ny), so
// fine row r receives the rows whose cell lies in the cyclic window
// [r - h, r + h - 1]: in fine-y order a run of consecutive places (modulo P)
// starting at first[r] = ly_first[(r - h) mod ny] (an empty cell's ly_first is
// the next row's place; P stands for 0).  The table therefore stores first[r]
// and the weight of each place of the run by its slot k = q - first[r]
// (modulo P): slots 0-3 in the float4 w[r], slots 4-7 in w[ny + r]; slots
// past the row's count stay 0.  A gather reads F at first[r] + k, so the
// reader keeps copies of the first 8 places after the last.  cell_cursor
// (arrivals per fine y cell): zeroed.
static __global__ void k_ell_fill(const int* __restrict__ runs, int cap, int ny, int w, const int* __restrict__ row_ly,
                           const float* __restrict__ row_wy, const int* __restrict__ ly_first,
                           int* __restrict__ rank_row, int* __restrict__ q_ly, float4* __restrict__ q_wy,
                           int* __restrict__ cell_cursor, int* __restrict__ first, float* __restrict__ wt) {
    const int P = min(*runs, cap);
    const int h = w / 2;
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < ny; r += stride) first[r] = ly_first[wrapmod(r - h, ny)];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
        const int ly = row_ly[p];
        const int c = wrapmod(ly, ny);
        const int q = ly_first[c] + atomicAdd(&cell_cursor[c], 1);
        rank_row[q] = p;
        q_ly[q] = ly;
        q_wy[2 * q] = reinterpret_cast<const float4*>(row_wy)[2 * p];
        q_wy[2 * q + 1] = reinterpret_cast<const float4*>(row_wy)[2 * p + 1];
        for (int t = 0; t < w; ++t) {
            const int r = wrapmod(c - (h - 1) + t, ny);
            int k = q - ly_first[wrapmod(r - h, ny)];
            if (k < 0) k += P;
            if (k < kEllMax) wt[((size_t)(k >> 2) * ny + r) * 4 + (k & 3)] = row_wy[(size_t)p * 8 + t];
        }
    }
}

static __global__ void k_tap_fill(const int* __restrict__ runs, int cap, int ny, int w, TapPoly tp, const int* __restrict__ row_ly,
                           const float* __restrict__ row_fy, const int* __restrict__ row_clo,
                           const int* __restrict__ row_len, const int64_t* __restrict__ row_off,
                           const int* __restrict__ start, int* __restrict__ cursor, TapEntry* __restrict__ taps) {
    const int P = min(*runs, cap);
    const int h = w / 2;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const float s = 2.0f * row_fy[p] - 1.0f;
        for (int t = 0; t < w; ++t) {
            const int r = wrapmod(row_ly[p] - (h - 1) + t, ny);
            TapEntry e;
            e.off = row_off[p];
            e.clo = row_clo[p];
            e.len = row_len[p];
            e.wy = tap_eval(tp, t, s);
            e.p = p;
            taps[start[r] + atomicAdd(&cursor[r], 1)] = e;
        }
    }
}

// ---------------------------------------------------------------------------
// General points: fine cells of both axes (err bit 1 on a bad coordinate),
// then bucketing by fine row (histogram, scatter) and a sorted copy.
// ---------------------------------------------------------------------------
static __global__ void k_prep_general(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y,
                               int* __restrict__ lx, float* __restrict__ fx, int* __restrict__ ly,
                               float* __restrict__ fy, int* __restrict__ err) {
    bool bad = false;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        int cx, cy;
        float ox, oy;
        bad |= !fine_coord(lam_x[n], cx, ox);
        bad |= !fine_coord(lam_y[n], cy, oy);
        lx[n] = cx;
        fx[n] = ox;
        ly[n] = cy;
        fy[n] = oy;
    }
    if (bad) atomicOr(err, 1);
}

static __global__ void k_bucket_hist(int64_t N, int ny, const int* __restrict__ ly, int* __restrict__ hist) {
    extern __shared__ int s_hist[];
    for (int i = threadIdx.x; i < ny; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&s_hist[wrapmod(ly[n], ny)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < ny; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

static __global__ void k_bucket_scatter(int64_t N, int ny, const int* __restrict__ ly, const int* __restrict__ bucket_start,
                                 int* __restrict__ cursor, int* __restrict__ perm) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int b = wrapmod(ly[n], ny);
        const int pos = bucket_start[b] + atomicAdd(&cursor[b], 1);
        perm[pos] = (int)n;
    }
}

static __global__ void k_gather_sorted(int64_t N, const int* __restrict__ perm, const int* __restrict__ lx,
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
// D_n for every sample in the caller's order (D_out, n_kept, general points).
// ---------------------------------------------------------------------------
static __global__ void k_weights(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y, int Mx,
                          int My, WeightArgs A, float* __restrict__ D, unsigned long long* __restrict__ kept) {
    int c = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float d;
        if (A.mode == 1) {
            d = 1.0f;
        } else if (A.mode == 2) {
            d = A.user_D[n];
        } else {
            const double x = lam_x[n];
            const double y = A.separable ? lam_y[n] : 0.0;
            int cx = 0, cy = 0;
            float ox = 0.f, oy = 0.f;
            fine_coord(x, cx, ox);
            if (A.separable) fine_coord(y, cy, oy);
            d = weight_tffr(x, cx, ox, y, cy, oy, Mx, My, A);
        }
        D[n] = d;
        c += (d != 0.0f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(kept, (unsigned long long)c);
}

static __global__ void k_gather_weights(int64_t N, const int* __restrict__ perm, const float* __restrict__ D,
                                 float* __restrict__ sD) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        sD[q] = D[perm[q]];
}

}  // namespace tffr
