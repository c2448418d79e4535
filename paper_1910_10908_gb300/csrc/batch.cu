// Adjoint of a batch of pulse-row patches (sub-apertures of uneven size):
// one spread launch over every pulse row of every patch, then one persistent
// FFT launch per image side.
//
// The spread launch (k_batch_spread) is the range spread of the single-image
// path with the patches' rows as one grid: block b looks up its patch and
// pulse row, stages the row's samples in shared memory and writes the row
// buffer R_p; the samples whose weight needs the FP64 decision are added by
// the same block after its runs, before it stores the row.
//
// The persistent FFT launch of a class (k_batch_fft) loops over work items
// claimed from one device counter:
//   row items (pulse-row order of the passes, one per pulse row): the x FFT
//     of R_p, the M kept modes into the patch's intermediate F (column-major:
//     F[jx ldq + q]);
//   fine-row items (fine-row order, one per fine row): the azimuth taps of the
//     row buffers, then the x FFT into T (column-major: T[jx n + r]);
//   column items (one per image column): wait until the patch's row (or
//     fine-row) items are done, gather the azimuth taps from the column of F
//     (or read the column of T), FFT along y, deapodise, store the column.
// Items are claimed in that order, so a column item only ever waits for items
// that running blocks have already claimed, and the wait ends; it is still
// bounded (wait_ns of device time), and a wait that runs out raises an error
// bit and an abort flag that ends every later wait at once.

#include <algorithm>

#include "batch_launch.h"
#include "kernels_spread.cuh"
#include "line_kernels.cuh"

namespace tffr {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The largest k < n with first[k] <= x (first is non-decreasing, first[0] = 0).
__device__ __forceinline__ int find_patch(const int* __restrict__ first, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&first[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Spread of every pulse row of every patch
// ---------------------------------------------------------------------------
// The batch spread's own block shape: its rows are short (a few hundred to
// 2048 samples), so 128 threads a row keep runs near kSpreadRun samples and let
// more rows (blocks) share an SM to hide each row's setup latency.  The staging
// pads every 32 elements: a warp's lanes walk runs 4 apart (32 samples).
constexpr int kBatchThreads = 128;
constexpr int kBatchTile = kBatchThreads * kSpreadRun;
constexpr int kBatchPadEvery = (kBatchThreads / 32) * kSpreadRun;
__host__ __device__ constexpr int batch_pad(int i) { return i + i / kBatchPadEvery; }
constexpr int kBatchStageElems = (batch_pad(kBatchTile - 1) + 2) & ~1;   // even: the values start 16-byte aligned

struct BatchStaged {
    const double* s_lam;
    const float2* s_val;
    int t0;
    __device__ __forceinline__ double lam(int i) const { return s_lam[batch_pad(i - t0)]; }
    __device__ __forceinline__ float2 val(int i) const { return s_val[batch_pad(i - t0)]; }
};

template <int W>
__global__ void __launch_bounds__(kBatchThreads, 8)
k_batch_spread(BatchSpreadArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* s_lam = reinterpret_cast<double*>(smem_raw);
    float2* s_val = reinterpret_cast<float2*>(s_lam + kBatchStageElems);
    float2* s_row = s_val + kBatchStageElems;
    constexpr int H = W / 2;
    const int tid = threadIdx.x;
    const BatchRow row = a.rows[blockIdx.x];
    const int tag = row.tag;                               // also the deferred list's row field
    const int M = row.M, n = row.n, len = row.len, clo = row.clo, L = row.L;
    const int64_t s0 = row.s0;
    const bool periodic = (len == n) && (clo == 0);
    const WeightArgs& wa = a.wa;
    __shared__ int s_ndef;
    if (tid == 0) s_ndef = 0;
    for (int i = tid; i < len; i += kBatchThreads) s_row[i] = make_float2(0.f, 0.f);
    float dy = 1.0f;
    bool dy_exact = false, edges = true;
    if (wa.mode == 0) {
        if (wa.separable) {
            const BatchPatch* __restrict__ bp = a.patches + (tag >> 16);
            const int p = tag & 0xffff;
            const float gy = g_fitted(__ldg(&bp->row_ly[p]), __ldg(&bp->row_fy[p]), M, wa, dy_exact);
            dy = (gy != 0.0f) ? __frcp_rn(gy) : 0.0f;
        }
        const int mn = clo + (H - 1), mx = clo + len - H - 1;
        edges = periodic || (mn >> 1) - wa.reach < -(M / 2) || (mx >> 1) + wa.reach >= M - M / 2;
    }
    const int run = (tid >> 5) + (kBatchThreads / 32) * (tid & 31);
    const double* __restrict__ g_lam = row.lam;
    const float2* __restrict__ g_val = row.val;
    const float* user_D = wa.mode == 2 ? a.patches[tag >> 16].user_D : nullptr;
    for (int t0 = 0; t0 < L; t0 += kBatchTile) {
        const int cnt = min(kBatchTile, L - t0);
        __syncthreads();                                   // row zeroed / previous tile consumed
        for (int e = tid; e < cnt; e += kBatchThreads) {
            cp_async_elem<8>(&s_lam[batch_pad(e)], &g_lam[t0 + e]);
            cp_async_elem<8>(&s_val[batch_pad(e)], &g_val[t0 + e]);
        }
        cp_async_wait_all();
        __syncthreads();
        // a short tile spreads its samples over every thread: runs of
        // ceil(cnt / threads) samples (at most kSpreadRun)
        const int rl = min(kSpreadRun, (cnt + kBatchThreads - 1) / kBatchThreads);
        const int i0 = t0 + run * rl;
        const int i1 = min(t0 + cnt, i0 + rl);
        if (i0 >= i1) continue;
        const BatchStaged src{s_lam, s_val, t0};
        const RowDefer rd{&s_ndef, a.defer_item};
        // n0: the row's first slot in the batch's list (tFFR weights), or its
        // first sample in the patch's user_D (user weights)
        if (wa.mode == 0)
            spread_run<float2, W, 0>(row.d0, i0, i1, n, clo, len, periodic, M, edges, dy, dy_exact, src, wa, a.tp, rd,
                                     s_row, user_D);
        else if (wa.mode == 1)
            spread_run<float2, W, 1>(s0, i0, i1, n, clo, len, periodic, M, edges, dy, dy_exact, src, wa, a.tp, rd,
                                     s_row, user_D);
        else
            spread_run<float2, W, 2>(s0, i0, i1, n, clo, len, periodic, M, edges, dy, dy_exact, src, wa, a.tp, rd,
                                     s_row, user_D);
    }
    __syncthreads();
    const int ndef = s_ndef;
    if (ndef > 0) {
        const BatchPatch* __restrict__ bp = a.patches + (tag >> 16);
        const int p = tag & 0xffff;
        spread_deferred_row<float2, W>(ndef, a.defer_item + row.d0, g_lam, g_val, bp->row_lam_y[p], M, M, n, clo,
                                       periodic, wa, a.tp, s_row);
        __syncthreads();
    }
    for (int i = tid; i < len; i += kBatchThreads) row.out[i] = s_row[i];
}

// Each block's pulse row of the spread launch, from the row tags and the
// patches' row arrays.
static __global__ void k_batch_rows(BatchSpreadArgs a, int rows) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const int tag = a.row_tag[r];
        const BatchPatch* bp = a.patches + (tag >> 16);
        const int p = tag & 0xffff;
        BatchRow row;
        const int64_t s0 = bp->row_start[p];
        row.lam = bp->lam_x + s0;
        row.val = bp->values + s0;
        row.out = bp->R + bp->row_off[p];
        row.s0 = (int)s0;
        row.L = (int)(bp->row_end[p] - s0);
        row.clo = bp->row_clo[p];
        row.len = bp->row_len[p];
        row.tag = tag;
        row.M = bp->M;
        row.n = bp->n;
        row.d0 = bp->defer_off + (int)s0;
        a.rows[r] = row;
    }
}

// ---------------------------------------------------------------------------
// Persistent FFT items of one class
// ---------------------------------------------------------------------------

// Column epilogue: keep the M = N/2 wanted y modes, deapodise, store column jx.
template <int LOGN>
struct ColStore {
    const float* deap_y;
    float2* img;
    int jx;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        constexpr int N = 1 << LOGN, M = N / 2, HALF = N / 4;
        int jy;
        if (o < HALF) jy = o + HALF;
        else if (o >= N - HALF) jy = o - (N - HALF);
        else return;
        img[(size_t)jy * M + jx] = cscale(v, __ldg(&deap_y[jy]));
    }
};

// Row epilogue into a column-major intermediate: keep the M = N/2 wanted x
// modes, deapodise (and undo a shift with the thread's phase factor), store
// entry `row` of column jx at X[jx ld + row].  The column items then read
// their column contiguously; the scattered stores are the row items' (stores
// do not stall the issuing thread).
template <int LOGN, bool RAMP>
struct RowOutCM {
    int row, ld;
    const float* deap_x;
    float2* X;
    float2 ramp;
    __device__ __forceinline__ void operator()(int o, float2 v) const {
        constexpr int N = 1 << LOGN, HALF = N / 4;
        int jx;
        if (o < HALF) jx = o + HALF;
        else if (o >= N - HALF) jx = o - (N - HALF);
        else return;
        if constexpr (RAMP) v = cmul(v, ramp);
        X[(size_t)jx * ld + row] = cscale(v, __ldg(&deap_x[jx]));
    }
};

// x FFT of a row buffer Rp[0, len) (line cell j = Rp[(j - clo) mod N]),
// shifted by a multiple of T so that a short row touches only the first U of
// each thread's V first-stage points (the shift s = j0 T is undone by the
// phase factor W_V^{j0 k}, k = tid mod V for every output of the thread).
template <int LOGN, int U>
__device__ __forceinline__ void row_fft_sparse(const float2* __restrict__ Rp, int off, int len, int j0, float2* buf,
                                               const Twiddles& tw, RowOutCM<LOGN, true>& epi) {
    using L = Line<LOGN>;
    const int tid = threadIdx.x;
    float2 v[L::V];
#pragma unroll
    for (int u = 0; u < L::V; ++u) {
        const int i = tid + u * L::T - off;
        v[u] = (u < U && i >= 0 && i < len) ? __ldg(&Rp[i]) : make_float2(0.f, 0.f);
    }
    epi.ramp = tw.t[((j0 * tid) & (L::V - 1)) * (L::NT / L::V)];
    fft_line_epilogue_regs_sparse<LOGN, U, +1>(v, buf, tw, epi);
}

// Thread 0 waits until *cnt reaches target (bounded; see the file comment);
// returns, to every thread of the block, whether it did.
__device__ __forceinline__ bool wait_count(const BatchClassArgs& a, const int* cnt, int target, int* s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire(cnt) < target) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire(cnt) < target) {
                if (*(volatile int*)&a.err[1]) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > a.wait_ns) {
                    atomicOr(&a.err[0], 1);
                    atomicExch(&a.err[1], 1);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Every thread's global stores of the item before the count (release).
__device__ __forceinline__ void publish(const BatchClassArgs& a, int* cnt) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && !a.hold) atomicAdd(cnt, 1);
}

// Row item (pulse-row order): x FFT of the row buffer of place q.
template <int LOGN>
__device__ void batch_row(const BatchClassArgs& a, int item, float2* buf, const Twiddles& tw) {
    using L = Line<LOGN>;
    constexpr int N = L::N;
    const int tid = threadIdx.x;
    const int k = find_patch(a.row_first, a.npatch, item);
    const BatchPatch* __restrict__ bp = a.patches + k;
    const int q = item - __ldg(&a.row_first[k]);
    const int p = __ldg(&bp->rank_row[q]);
    const int len = __ldg(&bp->row_len[p]), clo = __ldg(&bp->row_clo[p]);
    const float2* Rp = bp->R + __ldg(&bp->row_off[p]);
    float2* F = bp->F;
    const int ldq = __ldg(&bp->ldq);
    const float* deap_x = bp->deap_x;
    const int c = wrapmod(clo, N);
    const int j0 = c / L::T, off = c - j0 * L::T;
    const int U = (off + len + L::T - 1) / L::T;
    bool done = false;
    if constexpr (L::V >= 8) {
        if (U <= L::V / 4) {
            RowOutCM<LOGN, true> epi{q, ldq, deap_x, F, make_float2(1.f, 0.f)};
            if (U <= 1) row_fft_sparse<LOGN, 1>(Rp, off, len, j0, buf, tw, epi);
            else if (U <= 2) row_fft_sparse<LOGN, 2>(Rp, off, len, j0, buf, tw, epi);
            else if constexpr (L::V >= 16) row_fft_sparse<LOGN, 4>(Rp, off, len, j0, buf, tw, epi);
            done = true;
        }
    }
    if (!done) {
        float2 v[L::V];
#pragma unroll
        for (int u = 0; u < L::V; ++u) {
            const int o = wrapmod(tid + u * L::T - clo, N);
            v[u] = (o < len) ? __ldg(&Rp[o]) : make_float2(0.f, 0.f);
        }
        RowOutCM<LOGN, false> epi{q, ldq, deap_x, F, make_float2(1.f, 0.f)};
        fft_line_epilogue_regs<LOGN, +1>(v, buf, tw, epi);
    }
    publish(a, &a.done[k]);
}

// Fine-row item (fine-row order): fine row r of the patch = sum of its azimuth
// taps times the pulse-row buffers, then the x FFT, the M kept modes into T.
template <int LOGN>
__device__ void batch_fine(const BatchClassArgs& a, int item, float2* buf, const Twiddles& tw) {
    using L = Line<LOGN>;
    constexpr int N = L::N;
    const int tid = threadIdx.x;
    const int k = find_patch(a.fine_first, a.npatch, item);
    const BatchPatch* __restrict__ bp = a.patches + k;
    const int r = item - __ldg(&a.fine_first[k]);
    for (int i = tid; i < L::PADLEN; i += L::T) buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const float2* R = bp->R;
    const int e0 = __ldg(&bp->tap_start[r]), e1 = __ldg(&bp->tap_start[r + 1]);
    for (int e = e0; e < e1; ++e) {
        const TapEntry te = bp->taps[e];
        const float2* Rp = R + te.off;
        for (int i = tid; i < te.len; i += L::T)
            atomic_add_f2_shared(&buf[L::pad(wrapmod(te.clo + i, N))], cscale(__ldg(&Rp[i]), te.wy));
    }
    __syncthreads();
    RowOutCM<LOGN, false> epi{r, N, bp->deap_x, bp->F, make_float2(1.f, 0.f)};
    fft_line_epilogue<LOGN, +1>(buf, tw, epi);
    publish(a, &a.fine_done[k]);
}

// Column item: wait for the patch's rows, then the y pass of column jx.
template <int LOGN>
__device__ void batch_col(const BatchClassArgs& a, int item, float2* buf, const Twiddles& tw, int* s_ok) {
    using L = Line<LOGN>;
    constexpr int N = L::N, V = L::V;
    const int tid = threadIdx.x;
    const int k = find_patch(a.col_first, a.npatch, item);
    const BatchPatch* __restrict__ bp = a.patches + k;
    const int jx = item - __ldg(&a.col_first[k]);
    const int P = __ldg(&bp->P);
    ColStore<LOGN> epi{bp->deap_y, bp->image, jx};
    if (!__ldg(&bp->pulse)) {
        // fine-row order: column jx of T straight into the first stage's registers
        if (!wait_count(a, &a.fine_done[k], N, s_ok)) return;
        const float2* Tc = bp->F + (size_t)jx * N;
        float2 v[V];
#pragma unroll
        for (int u = 0; u < V; ++u) v[u] = __ldcg(&Tc[tid + u * L::T]);
        fft_line_epilogue_regs<LOGN, +1>(v, buf, tw, epi);
        return;
    }
    if (!wait_count(a, &a.done[k], P, s_ok)) return;   // the block's threads leave together
    // column jx of F into shared memory (read through L2: written in this launch)
    float2* fcol = buf + N / 2;
    const int ldq = __ldg(&bp->ldq);
    const float2* Fc = bp->F + (size_t)jx * ldq;
    for (int qq = tid; qq < P; qq += L::T) fcol[qq] = __ldcg(&Fc[qq]);
    if (tid < kPlaceCopies) fcol[P + tid] = __ldcg(&Fc[tid % P]);   // the run of a fine row wraps modulo P
    __syncthreads();
    // azimuth taps gathered from the fine-row table (first place, then one
    // weight per slot)
    const int* first = bp->ell_first;
    const float4* wt = bp->ell_w;
    const int K = __ldg(&bp->K);
    float2 v[V];
    if (K <= 4) {
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int r = tid + u * L::T;
            const float4 w4[1] = {__ldg(&wt[r])};
            v[u] = gather_taps<1>(fcol, __ldg(&first[r]), w4);
        }
    } else {
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int r = tid + u * L::T;
            const float4 w4[2] = {__ldg(&wt[r]), __ldg(&wt[N + r])};
            v[u] = gather_taps<2>(fcol, __ldg(&first[r]), w4);
        }
    }
    __syncthreads();                                   // fcol read before the first stage overwrites buf
    fft_line_epilogue_regs<LOGN, +1>(v, buf, tw, epi);
}

// 96 registers a thread (Line<LOGN>::T threads, 65536 / (96 T) blocks an SM),
// as the single-image x pass of these line lengths.
template <int LOGN>
__global__ void __launch_bounds__(Line<LOGN>::T, 65536 / (96 * Line<LOGN>::T))
k_batch_fft(BatchClassArgs a) {
    extern __shared__ float2 smem[];
    LineSmem<LOGN> S(smem);
    __shared__ int s_item, s_ok;
    const Twiddles tw = load_twiddles<LOGN>(S.twh, S.twl, S.tt, a.tab.twh, a.tab.twl, a.tab.tt);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();                               // read by every thread before the next claim
        if (item >= a.total) break;
        if (item < a.rows_total) batch_row<LOGN>(a, item, S.buf, tw);
        else if (item < a.rows_total + a.fine_total) batch_fine<LOGN>(a, item - a.rows_total, S.buf, tw);
        else batch_col<LOGN>(a, item - a.rows_total - a.fine_total, S.buf, tw, &s_ok);
    }
}

template <int LOGN>
int occupancy_one() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_fft<LOGN>, Line<LOGN>::T,
                                                      line_smem_bytes<LOGN>()) != cudaSuccess)
        return 0;
    return b;
}

}  // namespace

bool batch_class_supported(int logn, int w) { return logn >= 9 && logn <= 11 && w >= 2 && w <= 8 && !(w & 1); }

size_t batch_spread_smem(int max_len) {
    return (size_t)kBatchStageElems * (sizeof(double) + sizeof(float2)) + (size_t)max_len * sizeof(float2);
}

cudaError_t batch_set_attributes() {
    const int spread_max = (int)batch_spread_smem(kFftNMax);
    cudaError_t e = cudaFuncSetAttribute(k_batch_spread<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, spread_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_spread<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, spread_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_spread<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, spread_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_spread<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, spread_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_fft<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_smem_bytes<9>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_fft<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)line_smem_bytes<10>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_fft<11>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)line_smem_bytes<11>());
    return e;
}

int batch_max_blocks_per_sm(int logn) {
    switch (logn) {
        case 9: return occupancy_one<9>();
        case 10: return occupancy_one<10>();
        case 11: return occupancy_one<11>();
        default: return 0;
    }
}

void launch_batch_spread(int w, int rows, int max_len, cudaStream_t s, const BatchSpreadArgs& a) {
    const size_t smem = batch_spread_smem(max_len);
    switch (w) {
        case 2: k_batch_spread<2><<<rows, kBatchThreads, smem, s>>>(a); break;
        case 4: k_batch_spread<4><<<rows, kBatchThreads, smem, s>>>(a); break;
        case 6: k_batch_spread<6><<<rows, kBatchThreads, smem, s>>>(a); break;
        default: k_batch_spread<8><<<rows, kBatchThreads, smem, s>>>(a); break;
    }
}

void launch_batch_rows(int rows, cudaStream_t s, const BatchSpreadArgs& a) {
    k_batch_rows<<<std::max(1, std::min((rows + 255) / 256, 152 * 4)), 256, 0, s>>>(a, rows);
}

void launch_batch_fft(int logn, int grid, cudaStream_t s, const BatchClassArgs& a) {
    switch (logn) {
        case 9: k_batch_fft<9><<<grid, Line<9>::T, line_smem_bytes<9>(), s>>>(a); break;
        case 10: k_batch_fft<10><<<grid, Line<10>::T, line_smem_bytes<10>(), s>>>(a); break;
        default: k_batch_fft<11><<<grid, Line<11>::T, line_smem_bytes<11>(), s>>>(a); break;
    }
}

}  // namespace tffr
