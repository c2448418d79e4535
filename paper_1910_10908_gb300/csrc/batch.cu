// Persistent adjoint of a batch of pulse-row patches (sub-apertures of uneven
// size), one launch per image-size class.
//
// Every block loops over work items claimed from one device counter:
//   row items (one per pulse row of every patch): the row is spread into
//     shared memory (the range spread of the single-image path, with the FP64
//     weight decisions taken inline); in the pulse-row order of the passes it
//     is transformed along x right there (the x pass, with its sparse first
//     stage), the M kept modes going to the patch's intermediate F; in the
//     fine-row order it is stored to the patch's row buffers R;
//   fine-row items (fine-row order only, one per fine row): wait for the
//     patch's row items, add the azimuth taps of the row buffers, transform
//     along x into the intermediate T;
//   column items (one per image column of every patch): wait for the patch's
//     row (or fine-row) items, gather the column's azimuth taps from F (or read
//     the column of T), transform along y, deapodise and store the column of
//     the image.
// Items are claimed in that order, so a wait is only ever on items that
// running blocks have already claimed, and it ends; it is still bounded
// (wait_ns of device time), and a wait that runs out raises an error bit and
// an abort flag that ends every later wait at once.

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

// x FFT of a row held in buf[0, len) (line cell j = buf[(j - clo) mod N]),
// shifted by a multiple of T so that a short row touches only the first U of
// each thread's V first-stage points (see k_adj_rows_pulse).
template <int LOGN, int U>
__device__ __forceinline__ void row_fft_sparse(float2* buf, int off, int len, int j0, const Twiddles& tw,
                                               QuadOut<LOGN, true>& epi) {
    using L = Line<LOGN>;
    const int tid = threadIdx.x;
    float2 v[L::V];
#pragma unroll
    for (int u = 0; u < L::V; ++u) {
        const int i = tid + u * L::T - off;
        v[u] = (u < U && i >= 0 && i < len) ? buf[i] : make_float2(0.f, 0.f);
    }
    epi.ramp = tw.t[((j0 * tid) & (L::V - 1)) * (L::NT / L::V)];
    __syncthreads();                                   // buf read before the first stage overwrites it
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

template <int LOGN, int W>
__device__ void batch_row(const BatchClassArgs& a, int item, float2* buf, const Twiddles& tw) {
    using L = Line<LOGN>;
    constexpr int N = L::N, M = N / 2, H = W / 2;
    const int tid = threadIdx.x;
    const int k = find_patch(a.row_first, a.npatch, item);
    const BatchPatch* __restrict__ bp = a.patches + k;
    const int q = item - __ldg(&a.row_first[k]);
    const bool pulse = __ldg(&bp->pulse) != 0;
    const int p = pulse ? __ldg(&bp->rank_row[q]) : q;      // fine-row order: pulse row q
    const int len = __ldg(&bp->row_len[p]), clo = __ldg(&bp->row_clo[p]);
    const bool periodic = (len == N) && (clo == 0);
    const int64_t s0 = __ldg(&bp->row_start[p]);
    const int Lr = (int)(__ldg(&bp->row_end[p]) - s0);
    const double* lam_x = bp->lam_x;
    const float2* values = bp->values;
    const WeightArgs& wa = a.wa;
    const float* user_D = bp->user_D;
    for (int i = tid; i < len; i += L::T) buf[i] = make_float2(0.f, 0.f);
    float dy = 1.0f;
    bool dy_exact = false, edges = true;
    const double lam_y_row = __ldg(&bp->row_lam_y[p]);
    if (wa.mode == 0) {
        if (wa.separable) {
            const float gy = g_fitted(__ldg(&bp->row_ly[p]), __ldg(&bp->row_fy[p]), M, wa, dy_exact);
            dy = (gy != 0.0f) ? __frcp_rn(gy) : 0.0f;
        }
        const int mn = clo + (H - 1), mx = clo + len - H - 1;
        edges = periodic || (mn >> 1) - wa.reach < -(M / 2) || (mx >> 1) + wa.reach >= M - M / 2;
    }
    __syncthreads();
    // range spread (runs of a.run consecutive samples per thread and tile; the
    // lanes of a warp are T / 32 runs apart)
    const int run = L::T >= 32 ? (tid >> 5) + (L::T / 32) * (tid & 31) : tid;
    const int tile = L::T * a.run;
    const DeferList none{nullptr, nullptr, 0};
    const GlobalSamples<float2> src{lam_x, values, s0};
    for (int t0 = 0; t0 < Lr; t0 += tile) {
        const int i0 = t0 + run * a.run;
        const int i1 = min(Lr, i0 + a.run);
        if (i0 >= i1) continue;
        if (wa.mode == 0)
            spread_run<float2, W, 0, true>(s0, i0, i1, p, N, clo, len, periodic, M, edges, dy, dy_exact, src, wa,
                                           a.tp, none, buf, user_D, lam_y_row, M);
        else if (wa.mode == 1)
            spread_run<float2, W, 1, true>(s0, i0, i1, p, N, clo, len, periodic, M, edges, dy, dy_exact, src, wa,
                                           a.tp, none, buf, user_D, lam_y_row, M);
        else
            spread_run<float2, W, 2, true>(s0, i0, i1, p, N, clo, len, periodic, M, edges, dy, dy_exact, src, wa,
                                           a.tp, none, buf, user_D, lam_y_row, M);
    }
    __syncthreads();
    if (!pulse) {
        // fine-row order: the row buffer goes to R for the fine-row items
        float2* out = bp->R + __ldg(&bp->row_off[p]);
        for (int i = tid; i < len; i += L::T) out[i] = buf[i];
        publish(a, &a.done[k]);
        return;
    }
    // x FFT of the row, M kept modes into F (entry q of every column)
    const int c = wrapmod(clo, N);
    const int j0 = c / L::T, off = c - j0 * L::T;
    const int U = (off + len + L::T - 1) / L::T;
    float2* F = bp->F;
    const int ldq = __ldg(&bp->ldq);
    const float* deap_x = bp->deap_x;
    bool done = false;
    if constexpr (L::V >= 8) {
        if (U <= L::V / 4) {
            QuadOut<LOGN, true> epi{q, ldq, deap_x, F, make_float2(1.f, 0.f)};
            if (U <= 1) row_fft_sparse<LOGN, 1>(buf, off, len, j0, tw, epi);
            else if (U <= 2) row_fft_sparse<LOGN, 2>(buf, off, len, j0, tw, epi);
            else if constexpr (L::V >= 16) row_fft_sparse<LOGN, 4>(buf, off, len, j0, tw, epi);
            done = true;
        }
    }
    if (!done) {
        float2 v[L::V];
#pragma unroll
        for (int u = 0; u < L::V; ++u) {
            const int o = wrapmod(tid + u * L::T - clo, N);
            v[u] = (o < len) ? buf[o] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        QuadOut<LOGN> epi{q, ldq, deap_x, F, make_float2(1.f, 0.f)};
        fft_line_epilogue_regs<LOGN, +1>(v, buf, tw, epi);
    }
    publish(a, &a.done[k]);
}

// Fine-row item (fine-row order): fine row r of the patch = sum of its azimuth
// taps times the pulse-row buffers (written in this launch: read through L2),
// then the x FFT, the M kept modes into row r of T.
template <int LOGN>
__device__ void batch_fine(const BatchClassArgs& a, int item, float2* buf, const Twiddles& tw, int* s_ok) {
    using L = Line<LOGN>;
    constexpr int N = L::N;
    const int tid = threadIdx.x;
    const int k = find_patch(a.fine_first, a.npatch, item);
    const BatchPatch* __restrict__ bp = a.patches + k;
    const int r = item - __ldg(&a.fine_first[k]);
    for (int i = tid; i < L::PADLEN; i += L::T) buf[i] = make_float2(0.f, 0.f);
    if (!wait_count(a, &a.done[k], __ldg(&bp->P), s_ok)) return;      // (also orders the zeroing)
    const float2* R = bp->R;
    const int e0 = __ldg(&bp->tap_start[r]), e1 = __ldg(&bp->tap_start[r + 1]);
    for (int e = e0; e < e1; ++e) {
        const TapEntry te = bp->taps[e];
        const float2* Rp = R + te.off;
        for (int i = tid; i < te.len; i += L::T)
            atomic_add_f2_shared(&buf[L::pad(wrapmod(te.clo + i, N))], cscale(__ldcg(&Rp[i]), te.wy));
    }
    __syncthreads();
    RowOut<LOGN> epi{r, bp->deap_x, bp->F};
    fft_line_epilogue<LOGN, +1>(buf, tw, epi);
    publish(a, &a.fine_done[k]);
}

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
        // fine-row order: column jx of T [N][M] straight into the first stage's registers
        if (!wait_count(a, &a.fine_done[k], N, s_ok)) return;
        const float2* Tc = bp->F + jx;
        float2 v[V];
#pragma unroll
        for (int u = 0; u < V; ++u) v[u] = __ldcg(&Tc[(size_t)(tid + u * L::T) * (N / 2)]);
        fft_line_epilogue_regs<LOGN, +1>(v, buf, tw, epi);
        return;
    }
    if (!wait_count(a, &a.done[k], P, s_ok)) return;   // the block's threads leave together
    // column jx of F into shared memory (read through L2: written in this launch)
    float2* fcol = buf + N / 2;
    const int ldq = __ldg(&bp->ldq);
    const float2* Fb = bp->F + (size_t)(jx >> 2) * ldq * 4 + (jx & 3);
    for (int qq = tid; qq < P; qq += L::T) fcol[qq] = __ldcg(&Fb[(size_t)qq * 4]);
    __syncthreads();
    // azimuth taps gathered from the fine-row table (K slots per fine row)
    const int2* ell = bp->ell;
    const int K = __ldg(&bp->K);
    float2 v[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const int r = tid + u * L::T;
        float2 acc = make_float2(0.f, 0.f);
        for (int s = 0; s < K; ++s) {
            const int2 e = __ldg(&ell[(size_t)s * N + r]);
            const float2 f = fcol[e.x];
            const float g = __int_as_float(e.y);
            acc.x = fmaf(g, f.x, acc.x);
            acc.y = fmaf(g, f.y, acc.y);
        }
        v[u] = acc;
    }
    __syncthreads();                                   // fcol read before the first stage overwrites buf
    fft_line_epilogue_regs<LOGN, +1>(v, buf, tw, epi);
}

// 128 registers a thread: Line<LOGN>::T threads, 65536 / (128 T) blocks an SM.
template <int LOGN, int W>
__global__ void __launch_bounds__(Line<LOGN>::T, 65536 / (128 * Line<LOGN>::T))
k_batch_adjoint(BatchClassArgs a) {
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
        if (item < a.rows_total) batch_row<LOGN, W>(a, item, S.buf, tw);
        else if (item < a.rows_total + a.fine_total) batch_fine<LOGN>(a, item - a.rows_total, S.buf, tw, &s_ok);
        else batch_col<LOGN>(a, item - a.rows_total - a.fine_total, S.buf, tw, &s_ok);
    }
}

template <int LOGN, int W>
cudaError_t attr_one() {
    return cudaFuncSetAttribute(k_batch_adjoint<LOGN, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)line_smem_bytes<LOGN>());
}

template <int LOGN, int W>
int occupancy_one() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_adjoint<LOGN, W>, Line<LOGN>::T,
                                                      line_smem_bytes<LOGN>()) != cudaSuccess)
        return 0;
    return b;
}

}  // namespace

// Image sides 256, 512 and 1024 (lines of 512, 1024, 2048 fine cells),
// spreading widths 6 and 8.
#define TFFR_BATCH_SWITCH(logn, w, CALL)                       \
    switch ((logn) * 16 + (w)) {                               \
        case 9 * 16 + 6: CALL(9, 6); break;                    \
        case 9 * 16 + 8: CALL(9, 8); break;                    \
        case 10 * 16 + 6: CALL(10, 6); break;                  \
        case 10 * 16 + 8: CALL(10, 8); break;                  \
        case 11 * 16 + 6: CALL(11, 6); break;                  \
        case 11 * 16 + 8: CALL(11, 8); break;                  \
        default: break;                                        \
    }

bool batch_class_supported(int logn, int w) { return logn >= 9 && logn <= 11 && (w == 6 || w == 8); }

int batch_threads(int logn) { return (1 << logn) / line_v(1 << logn); }

size_t batch_smem(int logn) {
    switch (logn) {
        case 9: return line_smem_bytes<9>();
        case 10: return line_smem_bytes<10>();
        default: return line_smem_bytes<11>();
    }
}

cudaError_t batch_set_attributes() {
    cudaError_t e = cudaSuccess;
#define A(LG, W) if (e == cudaSuccess) e = attr_one<LG, W>()
    A(9, 6); A(9, 8); A(10, 6); A(10, 8); A(11, 6); A(11, 8);
#undef A
    return e;
}

int batch_max_blocks_per_sm(int logn, int w) {
    int b = 0;
#define O(LG, W) b = occupancy_one<LG, W>()
    TFFR_BATCH_SWITCH(logn, w, O)
#undef O
    return b;
}

void launch_batch_class(int logn, int w, int grid, cudaStream_t s, const BatchClassArgs& a) {
#define L(LG, W) k_batch_adjoint<LG, W><<<grid, Line<LG>::T, line_smem_bytes<LG>(), s>>>(a)
    TFFR_BATCH_SWITCH(logn, w, L)
#undef L
}

}  // namespace tffr
