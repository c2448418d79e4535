// Host side of the C ABI declared in include/tffr.h: plan set-up (FP64
// tables and polynomial fits), point preparation, weights, and the launch
// sequences of the adjoint and forward transforms.  All device work is in
// the .cuh kernels.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/tffr.h"
#include "batch_launch.h"
#include "common.cuh"
#include "line_launch.h"
#include "kernels_points.cuh"
#include "kernels_spread.cuh"

using namespace tffr;

// Device buffer with a capacity; grown (never shrunk) on demand.
template <typename T>
struct DevBuf {
    T* ptr = nullptr;
    int64_t cap = 0;
};

// Event pairs recorded around one stage's kernels.
struct StageProf {
    std::vector<cudaEvent_t> ev;
    int64_t n = 0;
};
constexpr int64_t kProfMaxPerStage = 4096;

struct tffr_plan_s {
    int Mx = 0, My = 0, nx = 0, ny = 0, lognx = 0, logny = 0, w = 6;
    double beta = 0.0;
    int values = TFFR_VALUES_C64;
    int layout_hint = TFFR_POINTS_AUTO;
    int order_hint = TFFR_ORDER_AUTO;
    cudaStream_t stream = nullptr;
    std::string last_error;
    size_t device_bytes = 0;
    TapPoly taps;                          // spreading-kernel taps, fitted at plan time
    WeightArgs wargs;                      // weight evaluation, set by tffr_weights
    WeightArgs fit_cache;                  // last fitted G pieces, reused while (a, q) stay the same
    bool fit_valid = false;

    // plan-time tables and the intermediate of the FFT passes
    DevBuf<float2> twh_x, twl_x, twh_y, twl_y, tt_x, tt_y, T;
    DevBuf<float> deap_x, deap_y;
    DevBuf<int> d_small;                   // [0] error bits, [1] rows, [2] longest row, [3] row overflow,
                                           // [4] most pulse rows reaching one fine row,
                                           // [8..9] total row-buffer cells (int64)
    DevBuf<int> defer;                     // [N] samples for the FP64 weight decision: the region of each
                                           // pulse row (its samples' slots) lists samples of the row
    int* h_small = nullptr;                // pinned read-back of d_small[0..9]
    cudaEvent_t readback = nullptr;        // recorded after that read-back
    DevBuf<unsigned long long> d_kept;

    // points (the caller's coordinate arrays are used in place)
    int64_t N = 0;
    const double* lam_x = nullptr;
    const double* lam_y = nullptr;
    bool have_points = false, have_weights = false;
    bool normal_ready = false;             // Khat of the Toeplitz normal operator built for these points/weights
    DevBuf<float2> khat, nwork1, nwork2;   // Khat column-major [2Mx][2My]; two [My][2Mx] work arrays
    DevBuf<float2> cg_r, cg_p, cg_Ap;      // conjugate gradients: residual, direction, N direction ([My][Mx])
    DevBuf<float2> cg_y;                   // [N] samples E p (CG without the Toeplitz operator)
    DevBuf<double> cg_s;                   // [2 iters + 1] |r_k|^2 (k = 0..iters), then Re <p_k, N p_k>
    int layout = 0;
    int64_t n_kept = -1;
    DevBuf<float> D;                       // per-sample weights when materialised
    DevBuf<int4> tile_info;                // pulse-row scan: per tile first / last row id, first start
    DevBuf<int2> tile_head;                // pulse-row scan: cell extent of each tile's leading samples

    // pulse rows
    int P = 0;
    int64_t R_cells = 0;
    int max_len = 0;
    int row_cap = 0;                       // capacity of the per-row arrays
    bool pulse_order = false;              // FFT passes in pulse-row order (F in T's memory)
    DevBuf<float> row_wy;                  // [cap][8] azimuth taps of each pulse row
    DevBuf<int> ell_first;                 // [ny] first place in fine-y order of each fine row's taps
    DevBuf<float4> ell_w;                  // [2][ny] tap weights of slots 0-3 and 4-7 (pulse-row order)
    int ell_k = 0;                         // slots in use: the most pulse rows a fine row receives
    DevBuf<int> row_start, row_end, row_clo, row_len, row_ly, row_min, row_max, bucket_start;
    DevBuf<float> row_fy;
    DevBuf<double> row_lam_y;
    DevBuf<int64_t> row_off;
    DevBuf<float2> R;
    DevBuf<int> tap_start;                 // [ny + 1] taps of each fine row
    DevBuf<int> rank_row;                  // [cap] pulse row at each place in fine-y order
    DevBuf<int> q_ly;                      // [cap] y cell of the pulse row at each place
    DevBuf<float> q_wy;                    // [cap][8] its azimuth taps
    DevBuf<TapEntry> tap_list;             // [P * w]

    // general points
    DevBuf<int> lx, ly, perm, slx, cursor;
    DevBuf<float> fx, fy, sfx, sfy, sD;
    DevBuf<float2> acc;

    // launch count and optional per-stage event timing
    int64_t launches = 0;
    bool prof_on = false;
    StageProf prof[TFFR_NUM_STAGES];
};

namespace {

int fail(tffr_plan_s* p, int status, const std::string& msg) {
    if (p) p->last_error = msg;
    return status;
}

int cuda_fail(tffr_plan_s* p, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
    return fail(p, e == cudaErrorMemoryAllocation ? TFFR_ERR_OOM : TFFR_ERR_CUDA, m);
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(p, e_, #call); \
    } while (0)

#define CK_LAUNCH(where)                                       \
    do {                                                       \
        ++p->launches;                                         \
        cudaError_t e_ = cudaGetLastError();                   \
        if (e_ != cudaSuccess) return cuda_fail(p, e_, where); \
    } while (0)

int stage_mark(tffr_plan_s* p, int stage, bool end) {
    if (!p->prof_on) return TFFR_OK;
    StageProf& sp = p->prof[stage];
    if (sp.n >= kProfMaxPerStage) return TFFR_OK;
    const size_t idx = (size_t)(2 * sp.n + (end ? 1 : 0));
    while (sp.ev.size() <= idx) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        sp.ev.push_back(e);
    }
    CK(cudaEventRecord(sp.ev[idx], p->stream));
    if (end) ++sp.n;
    return TFFR_OK;
}

#define STAGE_BEGIN(st)                          \
    do {                                         \
        int s_ = stage_mark(p, (st), false);     \
        if (s_ != TFFR_OK) return s_;            \
    } while (0)
#define STAGE_END(st)                            \
    do {                                         \
        int s_ = stage_mark(p, (st), true);      \
        if (s_ != TFFR_OK) return s_;            \
    } while (0)

template <typename T>
cudaError_t grow(tffr_plan_s* p, DevBuf<T>& b, int64_t want) {
    if (b.ptr && want <= b.cap) return cudaSuccess;
    if (b.ptr) {
        cudaFree(b.ptr);
        p->device_bytes -= (size_t)b.cap * sizeof(T);
        b.ptr = nullptr;
        b.cap = 0;
    }
    const int64_t n = std::max<int64_t>(want, 1);
    cudaError_t e = cudaMalloc((void**)&b.ptr, (size_t)n * sizeof(T));
    if (e == cudaSuccess) {
        b.cap = n;
        p->device_bytes += (size_t)n * sizeof(T);
    }
    return e;
}

template <typename T>
void release(DevBuf<T>& b) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// ---------------------------------------------------------------------------
// FP64 host numerics: quadrature, Chebyshev fits
// ---------------------------------------------------------------------------

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wts) {
    x.assign(n, 0.0);
    wts.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        wts[i] = wts[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

double es_phi(double z, int w, double beta) {
    const double x = 2.0 * z / w;
    const double t = 1.0 - x * x;
    return t > 0 ? std::exp(beta * (std::sqrt(t) - 1.0)) : 0.0;
}

// phi_hat(xi) = int_{-w/2}^{w/2} phi(z) exp(2 pi i xi z) dz for the ES kernel (real, even).
std::vector<double> es_transform(const std::vector<double>& xi, int w, double beta) {
    std::vector<double> gx, gw;
    const int nq = 160;
    gauss_legendre(nq, gx, gw);
    const double hw = 0.5 * w, two_pi = 6.283185307179586476925286766559;
    std::vector<double> z(nq), phi(nq), wz(nq);
    for (int i = 0; i < nq; ++i) {
        z[i] = 0.5 * hw * (gx[i] + 1.0);       // [0, w/2]
        wz[i] = 0.5 * hw * gw[i];
        phi[i] = es_phi(z[i], w, beta);
    }
    std::vector<double> out(xi.size());
    for (size_t k = 0; k < xi.size(); ++k) {
        double acc = 0.0;
        for (int i = 0; i < nq; ++i) acc += wz[i] * phi[i] * std::cos(two_pi * xi[k] * z[i]);
        out[k] = 2.0 * acc;
    }
    return out;
}

// Chebyshev interpolant of f on [-1, 1] at n nodes, returned as power-basis
// coefficients a_0..a_{n-1} of the variable s in [-1, 1].
template <typename F>
std::vector<double> cheb_fit_power(F f, int n) {
    const double pi = 3.14159265358979323846;
    std::vector<double> fv(n), c(n, 0.0);
    for (int k = 0; k < n; ++k) fv[k] = f(std::cos(pi * (k + 0.5) / n));
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += fv[k] * std::cos(pi * j * (k + 0.5) / n);
        c[j] = (j == 0 ? 1.0 : 2.0) * s / n;
    }
    // T_j in the power basis, by T_{j+1} = 2 s T_j - T_{j-1}
    std::vector<double> a(n, 0.0), tprev(n, 0.0), tcur(n, 0.0), tnext(n, 0.0);
    tprev[0] = 1.0;
    if (n > 1) tcur[1] = 1.0;
    for (int i = 0; i < n; ++i) a[i] += c[0] * tprev[i];
    if (n > 1)
        for (int i = 0; i < n; ++i) a[i] += c[1] * tcur[i];
    for (int j = 2; j < n; ++j) {
        for (int i = 0; i < n; ++i) tnext[i] = (i > 0 ? 2.0 * tcur[i - 1] : 0.0) - tprev[i];
        for (int i = 0; i < n; ++i) a[i] += c[j] * tnext[i];
        tprev.swap(tcur);
        tcur.swap(tnext);
    }
    return a;
}

template <typename F>
double power_fit_error(const std::vector<double>& a, F f) {
    double err = 0.0;
    for (int i = 0; i <= 2000; ++i) {
        const double s = -1.0 + 2.0 * i / 2000.0;
        double v = 0.0;
        for (int k = (int)a.size() - 1; k >= 0; --k) v = v * s + a[k];
        err = std::max(err, std::fabs(v - f(s)));
    }
    return err;
}

// Taps P_s(t), t = 2f - 1, for s < w/2; the mirrored taps are P_s(-t).
void fit_taps(tffr_plan_s* p) {
    std::memset(&p->taps, 0, sizeof(p->taps));
    const int w = p->w, h = w / 2;
    const int nc = tap_coefs(w);
    for (int s = 0; s < h; ++s) {
        auto f = [&](double t) { return es_phi((double)(s - (h - 1)) - 0.5 * (t + 1.0), w, p->beta); };
        const std::vector<double> a = cheb_fit_power(f, nc);
        for (int k = 0; k < nc; ++k) {
            p->taps.c[s][k] = (float)a[k];
            p->taps.c[w - 1 - s][k] = (float)((k & 1) ? -a[k] : a[k]);
        }
    }
}

// Polynomial pieces of G(delta) (unbounded grid) in v = |delta - 1/2|; see WeightArgs.
void fit_weights(WeightArgs& A) {
    const double fq = A.q - std::floor(A.q);
    A.vb = (float)std::fabs(fq - 0.5);
    const double vb = A.vb;
    auto G = [&](double v) { return diag_psi_w(0.5 + v, 0, A.a, A.q, A.e_minus, A.e_plus, A.reach); };
    A.n0 = A.n1 = 1;
    A.c0[0] = A.c1[0] = 0.0f;
    A.inv_vb = vb > 0.0 ? (float)(1.0 / vb) : 0.0f;
    if (vb > 0.0) {
        // G is even in v about delta = 1/2, hence smooth in s = 2 (v/vb)^2 - 1
        auto f0 = [&](double s) { return G(vb * std::sqrt(std::max(0.0, 0.5 * (s + 1.0)))); };
        std::vector<double> a = cheb_fit_power(f0, kG0Coefs);
        A.n0 = kG0Coefs;
        for (int k = 0; k < kG0Coefs; ++k) A.c0[k] = (float)a[k];
        // and 1/G itself on the same piece (G >= 0.93 there for the paper's a, q)
        auto r0 = [&](double s) {
            const double g = f0(s);
            return g != 0.0 ? 1.0 / g : 0.0;
        };
        std::vector<double> b = cheb_fit_power(r0, kD0Coefs);
        for (int k = 0; k < kD0Coefs; ++k) A.d0[k] = (float)b[k];
    }
    if (vb < 0.5) {
        auto f1 = [&](double s) { return G(vb + (0.5 - vb) * 0.5 * (s + 1.0)); };
        for (int n = 8; n <= kGCoefs; ++n) {
            std::vector<double> a = cheb_fit_power(f1, n);
            A.n1 = n;
            for (int k = 0; k < n; ++k) A.c1[k] = (float)a[k];
            if (power_fit_error(a, f1) < 1e-10) break;
        }
    }
}

// The fitted part of the weight evaluation (everything fit_weights sets).
void copy_fit(WeightArgs& dst, const WeightArgs& src) {
    dst.vb = src.vb;
    dst.inv_vb = src.inv_vb;
    dst.n0 = src.n0;
    dst.n1 = src.n1;
    std::memcpy(dst.c0, src.c0, sizeof(dst.c0));
    std::memcpy(dst.c1, src.c1, sizeof(dst.c1));
    std::memcpy(dst.d0, src.d0, sizeof(dst.d0));
}

int upload_tables(tffr_plan_s* p) {
    // two-level twiddles of an n-point line: exp(2 pi i 64 h / n) and exp(2 pi i l / n)
    auto level = [](int n, int count, int step) {
        std::vector<float2> t(count);
        const double two_pi = 6.283185307179586476925286766559;
        for (int m = 0; m < count; ++m) {
            const double a = two_pi * (double)((int64_t)m * step % n) / (double)n;
            t[m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        return t;
    };
    auto deapod = [&](int M, int n) {
        std::vector<double> xi(M);
        for (int j = 0; j < M; ++j) xi[j] = (double)(j - M / 2) / (double)n;
        std::vector<double> ph = es_transform(xi, p->w, p->beta);
        std::vector<float> d(M);
        for (int j = 0; j < M; ++j) d[j] = (float)(1.0 / ph[j]);
        return d;
    };
    const int nhx = std::max(1, p->nx / 64), nlx = std::min(64, p->nx);
    const int nhy = std::max(1, p->ny / 64), nly = std::min(64, p->ny);
    std::vector<float2> hx = level(p->nx, nhx, 64), lx = level(p->nx, nlx, 1);
    std::vector<float2> hy = level(p->ny, nhy, 64), ly = level(p->ny, nly, 1);
    const int ntx = std::min(1024, p->nx), nty = std::min(1024, p->ny);
    std::vector<float2> ttx = level(ntx, ntx, 1), tty = level(nty, nty, 1);
    CK(grow(p, p->tt_x, ntx));
    CK(grow(p, p->tt_y, nty));
    CK(cudaMemcpyAsync(p->tt_x.ptr, ttx.data(), ttx.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->tt_y.ptr, tty.data(), tty.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    std::vector<float> dx = deapod(p->Mx, p->nx), dy = deapod(p->My, p->ny);
    CK(grow(p, p->twh_x, nhx));
    CK(grow(p, p->twl_x, nlx));
    CK(grow(p, p->twh_y, nhy));
    CK(grow(p, p->twl_y, nly));
    CK(grow(p, p->deap_x, p->Mx));
    CK(grow(p, p->deap_y, p->My));
    CK(cudaMemcpyAsync(p->twh_x.ptr, hx.data(), hx.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->twl_x.ptr, lx.data(), lx.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->twh_y.ptr, hy.data(), hy.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->twl_y.ptr, ly.data(), ly.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->deap_x.ptr, dx.data(), dx.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->deap_y.ptr, dy.data(), dy.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));   // the host vectors end with this scope
    return TFFR_OK;
}

// staged tile (lam_x and the widest value type) and the longest (periodic) row
constexpr int kSpreadSmemMax = kSpreadStageElems * (int)(sizeof(double) + sizeof(double2)) +
                               kFftNMax * (int)sizeof(float2);

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename VT>
cudaError_t spread_attrs() {
    cudaError_t e = smem_attr(k_spread_rows<VT, 2>, kSpreadSmemMax);
    if (e == cudaSuccess) e = smem_attr(k_spread_rows<VT, 4>, kSpreadSmemMax);
    if (e == cudaSuccess) e = smem_attr(k_spread_rows<VT, 6>, kSpreadSmemMax);
    if (e == cudaSuccess) e = smem_attr(k_spread_rows<VT, 8>, kSpreadSmemMax);
    return e;
}

int set_kernel_attributes(tffr_plan_s* p) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    static bool done[64] = {false};
    if (dev < 64 && done[dev]) return TFFR_OK;
    CK(line_set_attributes());
    CK(batch_set_attributes());
    CK(spread_attrs<float2>());
    CK(spread_attrs<double2>());
    CK(spread_attrs<__half2>());
    CK(spread_attrs<__nv_bfloat162>());
    if (dev < 64) done[dev] = true;
    return TFFR_OK;
}

int grid_for(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

RowsView rows_view(const tffr_plan_s* p) {
    RowsView v;
    v.P = p->P;
    v.row_start = p->row_start.ptr;
    v.row_end = p->row_end.ptr;
    v.row_clo = p->row_clo.ptr;
    v.row_len = p->row_len.ptr;
    v.row_ly = p->row_ly.ptr;
    v.row_fy = p->row_fy.ptr;
    v.row_lam_y = p->row_lam_y.ptr;
    v.row_off = p->row_off.ptr;
    v.rank_row = p->rank_row.ptr;
    v.tap_start = p->tap_start.ptr;
    v.taps = p->tap_list.ptr;
    return v;
}

GeneralView general_view(const tffr_plan_s* p) {
    GeneralView v;
    v.bucket_start = p->bucket_start.ptr;
    v.perm = p->perm.ptr;
    v.slx = p->slx.ptr;
    v.sfx = p->sfx.ptr;
    v.sfy = p->sfy.ptr;
    v.sD = p->sD.ptr;
    return v;
}

// Per-row arrays for up to cap pulse rows; the extent arrays start at their
// identities (the scan folds cells in with atomic min / max).
int reserve_rows(tffr_plan_s* p, int cap) {
    if (cap <= p->row_cap) return TFFR_OK;
    const int w = p->w;
    p->row_cap = 0;
    CK(grow(p, p->row_start, cap));
    CK(grow(p, p->row_end, cap));
    CK(grow(p, p->row_min, cap));
    CK(grow(p, p->row_max, cap));
    CK(grow(p, p->row_clo, cap));
    CK(grow(p, p->row_len, cap));
    CK(grow(p, p->row_ly, cap));
    CK(grow(p, p->row_fy, cap));
    CK(grow(p, p->row_lam_y, cap));
    CK(grow(p, p->row_off, cap));
    CK(grow(p, p->rank_row, cap));
    CK(grow(p, p->q_ly, cap));
    CK(grow(p, p->q_wy, (int64_t)cap * 8));
    CK(grow(p, p->row_wy, (int64_t)cap * 8));
    CK(grow(p, p->tap_list, (int64_t)cap * w));
    k_fill_int<<<grid_for(cap, 256), 256, 0, p->stream>>>(cap, kIntMax, p->row_min.ptr);
    CK_LAUNCH("k_fill_int");
    k_fill_int<<<grid_for(cap, 256), 256, 0, p->stream>>>(cap, kIntMin, p->row_max.ptr);
    CK_LAUNCH("k_fill_int");
    p->row_cap = cap;
    return TFFR_OK;
}

// Pulse rows (runs of bit-equal lam_y) with their buffers and azimuth tap
// lists, and one read-back (error bits, runs, longest row, total cells).  On
// return *P_out holds the number of runs; the row structures are complete
// only when the function returns OK and *P_out <= p->row_cap.
int scan_rows(tffr_plan_s* p, int* P_out) {
    const int64_t N = p->N;
    const int64_t ntiles = (N + kRowScanTile - 1) / kRowScanTile;
    const int ny = p->ny, w = p->w, cap = p->row_cap;
    const int prow = std::min(std::max(1, (cap + 255) / 256), 152 * 8);
    CK(grow(p, p->tile_info, ntiles));
    CK(grow(p, p->tile_head, ntiles));
    CK(grow(p, p->tap_start, ny + 1));
    CK(grow(p, p->cursor, 3 * ny + 1));
    // cursor[0..ny]: tap counts per fine row, then the table's fill cursor;
    // cursor[ny + 1..2 ny]: pulse rows per fine y cell, then their first places
    // in fine-y order; cursor[2 ny + 1..3 ny]: arrivals per fine y cell
    int* const ly_first = p->cursor.ptr + ny + 1;
    CK(grow(p, p->ell_first, ny));
    CK(grow(p, p->ell_w, (int64_t)(kEllMax / 4) * ny));
    CK(cudaMemsetAsync(p->d_small.ptr, 0, 5 * sizeof(int), p->stream));
    RowScanArgs a;
    a.row_start = p->row_start.ptr;
    a.row_end = p->row_end.ptr;
    a.row_min = p->row_min.ptr;
    a.row_max = p->row_max.ptr;
    a.cap = cap;
    a.tile = p->tile_info.ptr;
    a.head = p->tile_head.ptr;
    a.flags = p->d_small.ptr;
    a.zero_i = p->cursor.ptr;                          // every counter of cursor[], zero for k_row_finish
    a.n_zero_i = 3 * ny + 1;
    a.zero_w = p->ell_w.ptr;                           // the tap weights, zero for k_ell_fill
    a.n_zero_w = (kEllMax / 4) * ny;
    k_scan_rows<<<(unsigned)ntiles, kRowScanWarps * 32, 0, p->stream>>>(N, p->lam_x, p->lam_y, a);
    CK_LAUNCH("k_scan_rows");
    const int* runs = p->d_small.ptr + 1;
    k_row_finish<<<prow, 256, 0, p->stream>>>(runs, cap, N, (int)ntiles, p->tile_info.ptr, p->tile_head.ptr, p->nx,
                                              ny, w, p->taps, p->lam_y, p->row_start.ptr, p->row_end.ptr,
                                              p->row_min.ptr, p->row_max.ptr, p->row_clo.ptr, p->row_len.ptr,
                                              p->row_ly.ptr, p->row_fy.ptr, p->row_lam_y.ptr, p->row_wy.ptr,
                                              p->cursor.ptr, ly_first);
    CK_LAUNCH("k_row_finish");
    // row buffer offsets, longest row (-> d_small[2]) and the per-fine-row tap
    // counts with the largest (-> d_small[4], which picks the pass order)
    long long* d_total = reinterpret_cast<long long*>(p->d_small.ptr + 8);
    k_row_scans<<<3, kScanThreads, 0, p->stream>>>(runs, cap, p->row_len.ptr, p->row_off.ptr, d_total, ny,
                                                    p->cursor.ptr, p->tap_start.ptr, p->d_small.ptr + 2,
                                                    p->d_small.ptr + 4, ly_first);
    CK_LAUNCH("k_row_scans");
    // one read-back: d_small[0..4] and the total cells in d_small[8..9].  The
    // fine-row tap table of the pulse-row order is filled after it on the
    // stream while the host waits for the read-back alone (unused in the
    // fine-row order).
    CK(cudaMemcpyAsync(p->h_small, p->d_small.ptr, 10 * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaEventRecord(p->readback, p->stream));
    k_ell_fill<<<prow, 256, 0, p->stream>>>(runs, cap, ny, w, p->row_ly.ptr, p->row_wy.ptr, ly_first,
                                            p->rank_row.ptr, p->q_ly.ptr, reinterpret_cast<float4*>(p->q_wy.ptr),
                                            ly_first + ny, p->ell_first.ptr,
                                            reinterpret_cast<float*>(p->ell_w.ptr));
    CK_LAUNCH("k_ell_fill");
    CK(cudaEventSynchronize(p->readback));
    int hs[5];
    long long tot;
    std::memcpy(hs, p->h_small, sizeof(hs));
    std::memcpy(&tot, p->h_small + 8, sizeof(tot));
    if (hs[0] & 1) return fail(p, TFFR_ERR_INVALID_ARG, "non-finite lam_y or |lam_y| >= 2^28");
    if (hs[0] & 2) return fail(p, TFFR_ERR_INVALID_ARG, "non-finite lam_x or |lam_x| >= 2^28");
    *P_out = hs[1];
    if (hs[1] > cap || hs[3]) return TFFR_OK;          // caller grows the row arrays and scans again
    p->P = hs[1];
    p->max_len = hs[2];
    p->R_cells = tot;
    CK(grow(p, p->R, tot));
    // the fine-row order needs the azimuth tap lists of every fine row (built
    // after the read-back, ordered on the stream like everything else)
    p->pulse_order = p->order_hint == TFFR_ORDER_AUTO && p->P >= 1 && p->P <= p->My && hs[4] <= kEllMax;
    if (p->pulse_order) {
        p->ell_k = hs[4];                              // the table itself was filled before the read-back
    } else {
        CK(cudaMemsetAsync(p->cursor.ptr, 0, (size_t)(ny + 1) * sizeof(int), p->stream));
        k_tap_fill<<<prow, 256, 0, p->stream>>>(runs, cap, ny, w, p->taps, p->row_ly.ptr, p->row_fy.ptr,
                                                p->row_clo.ptr, p->row_len.ptr, p->row_off.ptr, p->tap_start.ptr,
                                                p->cursor.ptr, p->tap_list.ptr);
        CK_LAUNCH("k_tap_fill");
    }
    return TFFR_OK;
}

int build_general(tffr_plan_s* p) {
    const int64_t N = p->N;
    p->P = 0;
    CK(grow(p, p->bucket_start, p->ny + 1));
    CK(grow(p, p->cursor, p->ny + 1));
    CK(grow(p, p->lx, N));
    CK(grow(p, p->ly, N));
    CK(grow(p, p->fx, N));
    CK(grow(p, p->fy, N));
    CK(grow(p, p->perm, N));
    CK(grow(p, p->slx, N));
    CK(grow(p, p->sfx, N));
    CK(grow(p, p->sfy, N));
    CK(grow(p, p->sD, N));
    CK(grow(p, p->acc, N));
    CK(cudaMemsetAsync(p->d_small.ptr, 0, sizeof(int), p->stream));
    k_prep_general<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->lam_x, p->lam_y, p->lx.ptr, p->fx.ptr, p->ly.ptr,
                                                           p->fy.ptr, p->d_small.ptr);
    CK_LAUNCH("k_prep_general");
    CK(cudaMemsetAsync(p->cursor.ptr, 0, (size_t)(p->ny + 1) * sizeof(int), p->stream));
    k_bucket_hist<<<grid_for(N, 256), 256, p->ny * sizeof(int), p->stream>>>(N, p->ny, p->ly.ptr, p->cursor.ptr);
    CK_LAUNCH("k_bucket_hist");
    std::vector<int> cnt(p->ny);
    int err = 0;
    CK(cudaMemcpyAsync(cnt.data(), p->cursor.ptr, (size_t)p->ny * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(&err, p->d_small.ptr, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (err) return fail(p, TFFR_ERR_INVALID_ARG, "non-finite coordinate or |lam| >= 2^28");
    std::vector<int> bstart(p->ny + 1, 0);
    for (int b = 0; b < p->ny; ++b) bstart[b + 1] = bstart[b] + cnt[b];
    CK(cudaMemcpyAsync(p->bucket_start.ptr, bstart.data(), (size_t)(p->ny + 1) * sizeof(int),
                       cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemsetAsync(p->cursor.ptr, 0, (size_t)(p->ny + 1) * sizeof(int), p->stream));
    k_bucket_scatter<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->ny, p->ly.ptr, p->bucket_start.ptr,
                                                               p->cursor.ptr, p->perm.ptr);
    CK_LAUNCH("k_bucket_scatter");
    k_gather_sorted<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->perm.ptr, p->lx.ptr, p->fx.ptr, p->fy.ptr,
                                                              p->slx.ptr, p->sfx.ptr, p->sfy.ptr);
    CK_LAUNCH("k_gather_sorted");
    CK(cudaStreamSynchronize(p->stream));
    return TFFR_OK;
}

FftTables tables_x(const tffr_plan_s* p) { return FftTables{p->twh_x.ptr, p->twl_x.ptr, p->tt_x.ptr}; }
FftTables tables_y(const tffr_plan_s* p) { return FftTables{p->twh_y.ptr, p->twl_y.ptr, p->tt_y.ptr}; }

// The plan's weights, or unit weights (the unweighted adjoint E^H y).
WeightArgs spread_weights(const tffr_plan_s* p, bool weighted) {
    if (weighted) return p->wargs;
    WeightArgs u;
    std::memset(&u, 0, sizeof(u));
    u.mode = TFFR_WEIGHTS_UNIT;
    return u;
}

template <typename VT, int W>
void launch_spread(tffr_plan_s* p, const RowsView& rv, const void* values, bool weighted) {
    const size_t smem = (size_t)kSpreadStageElems * (sizeof(double) + sizeof(VT)) + (size_t)p->max_len * sizeof(float2);
    const WeightArgs wa = spread_weights(p, weighted);
    k_spread_rows<VT, W><<<p->P, kSpreadThreads, smem, p->stream>>>(rv, p->N, p->nx, p->Mx, p->My, p->lam_x, values,
                                                                     wa, p->taps, p->defer.ptr, p->R.ptr);
}

template <typename VT>
int adjoint_impl(tffr_plan_s* p, const void* values, float2* image, bool weighted = true) {
    const int ny = p->ny;
    if (p->layout == TFFR_POINTS_ROWS) {
        const RowsView rv = rows_view(p);
        STAGE_BEGIN(TFFR_STAGE_SPREAD);
        switch (p->w) {
            case 2: launch_spread<VT, 2>(p, rv, values, weighted); break;
            case 4: launch_spread<VT, 4>(p, rv, values, weighted); break;
            case 6: launch_spread<VT, 6>(p, rv, values, weighted); break;
            default: launch_spread<VT, 8>(p, rv, values, weighted); break;
        }
        CK_LAUNCH("k_spread_rows");
        STAGE_END(TFFR_STAGE_SPREAD);
        STAGE_BEGIN(TFFR_STAGE_ROW_FFT);
        if (p->pulse_order) {
            launch_adj_rows_pulse(p->lognx, p->P, p->stream, rv, p->R.ptr, tables_x(p), p->deap_x.ptr, p->T.ptr);
            CK_LAUNCH("k_adj_rows_pulse");
            STAGE_END(TFFR_STAGE_ROW_FFT);
            STAGE_BEGIN(TFFR_STAGE_COL_FFT);
            launch_adj_cols_pulse(p->logny, p->Mx, p->P, p->stream, p->T.ptr, tables_y(p), p->ell_first.ptr, p->ell_w.ptr, p->ell_k,
                                  p->deap_y.ptr, image);
            CK_LAUNCH("k_adj_cols_pulse");
            STAGE_END(TFFR_STAGE_COL_FFT);
            return TFFR_OK;
        }
        launch_adj_rows(p->lognx, ny, p->stream, rv, p->R.ptr, p->w, p->taps, tables_x(p), p->deap_x.ptr, p->T.ptr);
        CK_LAUNCH("k_adj_rows");
        STAGE_END(TFFR_STAGE_ROW_FFT);
    } else {
        STAGE_BEGIN(TFFR_STAGE_ROW_FFT);
        k_gather_values<VT><<<grid_for(p->N, 256), 256, 0, p->stream>>>(p->N, p->perm.ptr, values,
                                                                         weighted ? p->sD.ptr : nullptr, p->acc.ptr);
        CK_LAUNCH("k_gather_values");
        const GeneralView gv = general_view(p);
        launch_adj_rows_general(p->lognx, ny, p->stream, gv, p->acc.ptr, p->w, p->taps, tables_x(p), p->deap_x.ptr,
                                p->T.ptr);
        CK_LAUNCH("k_adj_rows_general");
        STAGE_END(TFFR_STAGE_ROW_FFT);
    }
    STAGE_BEGIN(TFFR_STAGE_COL_FFT);
    launch_adj_cols(p->logny, p->Mx, p->stream, p->T.ptr, tables_y(p), p->deap_y.ptr, image);
    CK_LAUNCH("k_adj_cols");
    STAGE_END(TFFR_STAGE_COL_FFT);
    return TFFR_OK;
}

template <typename VT, int W>
void launch_interp(tffr_plan_s* p, const RowsView& rv, void* values, int apply_weights, const void* y_in) {
    if (y_in)
        k_interp_rows<VT, W, true><<<p->P, kSpreadThreads, 0, p->stream>>>(
            rv, p->N, p->nx, p->Mx, p->My, p->lam_x, p->R.ptr, p->wargs, p->taps, 0, p->defer.ptr, values, y_in);
    else
        k_interp_rows<VT, W><<<p->P, kSpreadThreads, 0, p->stream>>>(rv, p->N, p->nx, p->Mx, p->My, p->lam_x,
                                                                      p->R.ptr, p->wargs, p->taps, apply_weights,
                                                                      p->defer.ptr, values);
}

// values = (D) E image; with y_in, values (float[N]) = Re(conj(E image) y) instead:
// the gradient of a real loss with respect to real weights, for grad_image = its
// gradient with respect to the image (y_in in the value type VT).
template <typename VT>
int forward_impl(tffr_plan_s* p, const float2* image, void* values, int apply_weights, const void* y_in = nullptr) {
    const int ny = p->ny;
    const bool pulse = p->layout == TFFR_POINTS_ROWS && p->pulse_order;
    const RowsView rv = rows_view(p);
    const GeneralView gv = general_view(p);
    STAGE_BEGIN(TFFR_STAGE_FWD_COL_FFT);
    if (pulse) {
        launch_fwd_cols_pulse(p->logny, p->Mx, p->P, p->stream, image, tables_y(p), p->deap_y.ptr, p->deap_x.ptr,
                              p->q_ly.ptr, p->q_wy.ptr, p->w, p->T.ptr);
        CK_LAUNCH("k_fwd_cols_pulse");
    } else {
        launch_fwd_cols(p->logny, p->Mx, p->stream, image, tables_y(p), p->deap_y.ptr, p->deap_x.ptr, p->T.ptr);
        CK_LAUNCH("k_fwd_cols");
    }
    STAGE_END(TFFR_STAGE_FWD_COL_FFT);
    STAGE_BEGIN(TFFR_STAGE_FWD_ROW_FFT);
    if (p->layout == TFFR_POINTS_ROWS) {
        if (pulse) {
            launch_fwd_rows_pulse(p->lognx, p->P, p->stream, rv, p->T.ptr, tables_x(p), p->R.ptr);
            CK_LAUNCH("k_fwd_rows_pulse");
        } else {
            CK(cudaMemsetAsync(p->R.ptr, 0, (size_t)p->R_cells * sizeof(float2), p->stream));
            launch_fwd_rows(p->lognx, ny, true, p->stream, rv, gv, p->T.ptr, p->w, p->taps, tables_x(p), p->R.ptr,
                            p->acc.ptr);
            CK_LAUNCH("k_fwd_rows");
        }
        STAGE_END(TFFR_STAGE_FWD_ROW_FFT);
        STAGE_BEGIN(TFFR_STAGE_INTERP);
        switch (p->w) {
            case 2: launch_interp<VT, 2>(p, rv, values, apply_weights, y_in); break;
            case 4: launch_interp<VT, 4>(p, rv, values, apply_weights, y_in); break;
            case 6: launch_interp<VT, 6>(p, rv, values, apply_weights, y_in); break;
            default: launch_interp<VT, 8>(p, rv, values, apply_weights, y_in); break;
        }
        CK_LAUNCH("k_interp_rows");
        STAGE_END(TFFR_STAGE_INTERP);
    } else {
        CK(cudaMemsetAsync(p->acc.ptr, 0, (size_t)p->N * sizeof(float2), p->stream));
        launch_fwd_rows(p->lognx, ny, false, p->stream, rv, gv, p->T.ptr, p->w, p->taps, tables_x(p), p->R.ptr,
                        p->acc.ptr);
        CK_LAUNCH("k_fwd_rows");
        STAGE_END(TFFR_STAGE_FWD_ROW_FFT);
        STAGE_BEGIN(TFFR_STAGE_INTERP);
        if (y_in) {
            k_unpermute_grad<VT><<<grid_for(p->N, 256), 256, 0, p->stream>>>(p->N, p->perm.ptr, p->acc.ptr, y_in,
                                                                              reinterpret_cast<float*>(values));
            CK_LAUNCH("k_unpermute_grad");
        } else {
            k_unpermute_output<VT><<<grid_for(p->N, 256), 256, 0, p->stream>>>(p->N, p->perm.ptr, p->acc.ptr,
                                                                                p->sD.ptr, apply_weights, values);
            CK_LAUNCH("k_unpermute_output");
        }
        STAGE_END(TFFR_STAGE_INTERP);
    }
    return TFFR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free weights (tffr_weights_noalloc)
//
// Scratch lives in one file-scope device array, held by every GPU that loads
// the library until the process exits: per-block kept counts, a count of
// finished blocks and the total.  In host code the array's name is only a
// stand-in; its device address comes from cudaGetSymbolAddress, looked up
// once per device (with that device current) on the first call there.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 8;
constexpr int kNaPerBlock = kNaThreads * kNaPerThread;          // samples per block
constexpr int kNaMaxBlocks = 32768;
constexpr int64_t kNaMaxN = (int64_t)kNaMaxBlocks * kNaPerBlock;  // 67,108,864 samples

struct NoAllocScratch {
    unsigned int block_kept[kNaMaxBlocks];
    unsigned int done;
    unsigned long long total;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {nullptr};

// D_n for the block's samples (FP64 closed form, no plan-time fit), then the
// block's kept count; the last block to finish adds the counts up.
__global__ void __launch_bounds__(kNaThreads)
k_weights_noalloc(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y, int Mx, int My,
                  WeightArgs A, float* __restrict__ D, NoAllocScratch* __restrict__ sc) {
    __shared__ int s_warp[32];
    __shared__ bool s_last;
    const int64_t base = (int64_t)blockIdx.x * kNaPerBlock;
    int c = 0;
    for (int k = 0; k < kNaPerThread; ++k) {
        const int64_t n = base + (int64_t)k * kNaThreads + threadIdx.x;
        if (n >= N) break;
        float d;
        if (A.mode == 1) d = 1.0f;
        else if (A.mode == 2) d = A.user_D[n];
        else d = weight_exact(lam_x[n], A.separable ? lam_y[n] : 0.0, Mx, My, A);
        D[n] = d;
        c += (d != 0.0f);
    }
    int tot;
    block_exclusive_scan(c, s_warp, &tot);
    if (threadIdx.x == 0) {
        sc->block_kept[blockIdx.x] = (unsigned int)tot;
        __threadfence();
        s_last = (atomicAdd(&sc->done, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long sum = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaThreads) sum += __ldcg(&sc->block_kept[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ unsigned long long s_sum[kNaThreads / 32];
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kNaThreads / 32; ++i) t += s_sum[i];
        sc->total = t;
    }
}

cudaError_t noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = ptr;
    }
    *out = reinterpret_cast<NoAllocScratch*>(g_noalloc_ptr[dev]);
    return cudaSuccess;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void tffr_default_opts(tffr_opts* o) {
    if (!o) return;
    o->sigma = 2;
    o->width = 6;
    o->beta = 0.0;
    o->values = TFFR_VALUES_C64;
    o->layout = TFFR_POINTS_AUTO;
    o->order = TFFR_ORDER_AUTO;
}

void tffr_default_weight_opts(tffr_weight_opts* o) {
    if (!o) return;
    o->mode = TFFR_WEIGHTS_TFFR;
    o->separable = 0;
    o->a = 0.01;
    o->q = 3.0;
    o->tau = 0.97;
    o->user_D = nullptr;
}

const char* tffr_error_string(int s) {
    switch (s) {
        case TFFR_OK: return "ok";
        case TFFR_ERR_INVALID_ARG: return "invalid argument";
        case TFFR_ERR_NOT_READY: return "not ready: set points and weights first";
        case TFFR_ERR_CUDA: return "CUDA error";
        case TFFR_ERR_OOM: return "out of device memory";
        case TFFR_ERR_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* tffr_last_error(tffr_plan_t p) { return p ? p->last_error.c_str() : ""; }

int tffr_plan(tffr_plan_t* out, int Mx, int My, const tffr_opts* opts, tffr_stream_t stream) {
    if (!out) return TFFR_ERR_INVALID_ARG;
    *out = nullptr;
    tffr_opts o;
    tffr_default_opts(&o);
    if (opts) o = *opts;
    if (!is_pow2(Mx) || !is_pow2(My) || Mx < 16 || My < 16 || 2 * Mx > kFftNMax || 2 * My > kFftNMax)
        return TFFR_ERR_INVALID_ARG;
    if (o.sigma != 2) return TFFR_ERR_INVALID_ARG;
    if (o.width < 2 || o.width > 8 || (o.width & 1)) return TFFR_ERR_INVALID_ARG;
    if (o.values < TFFR_VALUES_C64 || o.values > TFFR_VALUES_BF16) return TFFR_ERR_INVALID_ARG;
    if (o.layout < TFFR_POINTS_AUTO || o.layout > TFFR_POINTS_ROWS) return TFFR_ERR_INVALID_ARG;
    if (o.order < TFFR_ORDER_AUTO || o.order > TFFR_ORDER_FINE_ROWS) return TFFR_ERR_INVALID_ARG;
    if (!(o.beta == o.beta) || o.beta > 100.0) return TFFR_ERR_INVALID_ARG;
    tffr_plan_s* p = new (std::nothrow) tffr_plan_s();
    if (!p) return TFFR_ERR_OOM;
    p->Mx = Mx;
    p->My = My;
    p->nx = 2 * Mx;
    p->ny = 2 * My;
    p->lognx = ilog2(p->nx);
    p->logny = ilog2(p->ny);
    p->w = o.width;
    p->beta = o.beta > 0 ? o.beta : 2.30 * o.width;
    p->values = o.values;
    p->layout_hint = o.layout;
    p->order_hint = o.order;
    p->stream = (cudaStream_t)stream;
    fit_taps(p);
    std::memset(&p->wargs, 0, sizeof(p->wargs));
    int s = set_kernel_attributes(p);
    if (s == TFFR_OK) s = upload_tables(p);
    if (s == TFFR_OK) {
        cudaError_t e = grow(p, p->T, (int64_t)Mx * p->ny);
        if (e == cudaSuccess) e = grow(p, p->d_small, 16);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->d_small.ptr, 0, 16 * sizeof(int), p->stream);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_small, 16 * sizeof(int));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->readback, cudaEventDisableTiming);
        if (e == cudaSuccess) e = grow(p, p->d_kept, 1);
        if (e != cudaSuccess) s = cuda_fail(p, e, "tffr_plan: allocation");
    }
    if (s != TFFR_OK) {
        tffr_destroy(p);
        return s;
    }
    *out = p;
    return TFFR_OK;
}

int tffr_destroy(tffr_plan_t p) {
    if (!p) return TFFR_OK;
    cudaStreamSynchronize(p->stream);
    release(p->twh_x); release(p->twl_x); release(p->twh_y); release(p->twl_y); release(p->tt_x); release(p->tt_y);
    release(p->T); release(p->deap_x); release(p->deap_y);
    release(p->d_small); release(p->d_kept); release(p->D);
    release(p->tile_info); release(p->tile_head); release(p->defer);
    release(p->khat); release(p->nwork1); release(p->nwork2);
    release(p->cg_r); release(p->cg_p); release(p->cg_Ap); release(p->cg_y); release(p->cg_s);
    if (p->h_small) cudaFreeHost(p->h_small);
    if (p->readback) cudaEventDestroy(p->readback);
    release(p->row_start); release(p->row_clo); release(p->row_len); release(p->row_ly);
    release(p->row_min); release(p->row_max); release(p->row_end); release(p->row_wy);
    release(p->ell_first);
    release(p->ell_w);
    release(p->bucket_start); release(p->row_fy); release(p->row_lam_y); release(p->row_off); release(p->R);
    release(p->tap_start); release(p->tap_list); release(p->rank_row); release(p->q_ly); release(p->q_wy);
    release(p->lx); release(p->ly); release(p->perm); release(p->slx); release(p->cursor);
    release(p->fx); release(p->fy); release(p->sfx); release(p->sfy); release(p->sD); release(p->acc);
    for (auto& sp : p->prof)
        for (cudaEvent_t e : sp.ev) cudaEventDestroy(e);
    delete p;
    return TFFR_OK;
}

int tffr_plan_get_info(tffr_plan_t p, tffr_plan_info* info) {
    if (!p || !info) return TFFR_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->Mx = p->Mx;
    info->My = p->My;
    info->nx = p->nx;
    info->ny = p->ny;
    info->width = p->w;
    info->beta = p->beta;
    info->N = p->have_points ? p->N : 0;
    info->layout = p->have_points ? p->layout : 0;
    const bool rows = p->have_points && p->layout == TFFR_POINTS_ROWS;
    info->n_rows = rows ? p->P : 0;
    info->row_cells = rows ? p->R_cells : 0;
    info->max_row_cells = rows ? p->max_len : 0;
    info->n_kept = p->have_weights ? p->n_kept : -1;
    info->device_bytes = p->device_bytes;
    info->kernel_launches = p->launches;
    info->pulse_order = (rows && p->pulse_order) ? 1 : 0;
    return TFFR_OK;
}

int tffr_profile(tffr_plan_t p, int enable) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(p->stream));
    for (auto& sp : p->prof) sp.n = 0;
    p->prof_on = enable != 0;
    return TFFR_OK;
}

int tffr_profile_read(tffr_plan_t p, double* ms, int64_t* count, int nstages) {
    if (!p || nstages < 0 || nstages > TFFR_NUM_STAGES) return TFFR_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(p->stream));
    for (int st = 0; st < nstages; ++st) {
        const StageProf& sp = p->prof[st];
        double tot = 0.0;
        for (int64_t i = 0; i < sp.n; ++i) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, sp.ev[2 * i], sp.ev[2 * i + 1]));
            tot += t;
        }
        if (ms) ms[st] = tot;
        if (count) count[st] = sp.n;
    }
    return TFFR_OK;
}

int tffr_set_points(tffr_plan_t p, int64_t N, const double* lam_x, const double* lam_y) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (N < 0 || N >= (int64_t)0x7fffffff) return fail(p, TFFR_ERR_INVALID_ARG, "N out of range");
    if (N > 0 && (!lam_x || !lam_y)) return fail(p, TFFR_ERR_INVALID_ARG, "NULL coordinates");
    p->have_points = false;
    p->have_weights = false;
    p->normal_ready = false;
    p->n_kept = -1;
    p->N = N;
    p->lam_x = lam_x;
    p->lam_y = lam_y;
    if (N == 0) {
        p->layout = TFFR_POINTS_GENERAL;
        p->P = 0;
        p->have_points = true;
        return TFFR_OK;
    }
    STAGE_BEGIN(TFFR_STAGE_POINTS);
    int layout = p->layout_hint;
    int s = TFFR_OK;
    if (layout != TFFR_POINTS_GENERAL) {
        // pulse rows are tried first; a second scan runs only when the row
        // arrays were too small for this set of points
        s = reserve_rows(p, std::max(p->row_cap, (int)std::min<int64_t>(N, 4096)));
        int P = 0;
        if (s == TFFR_OK) s = scan_rows(p, &P);
        if (s != TFFR_OK) return s;
        if (layout == TFFR_POINTS_AUTO) layout = (N >= 8 * (int64_t)P) ? TFFR_POINTS_ROWS : TFFR_POINTS_GENERAL;
        if (layout == TFFR_POINTS_ROWS && P > p->row_cap) {
            s = reserve_rows(p, P);
            if (s == TFFR_OK) s = scan_rows(p, &P);
            if (s != TFFR_OK) return s;
            if (P > p->row_cap) return fail(p, TFFR_ERR_INVALID_ARG, "pulse rows changed between two scans");
        }
    }
    p->layout = layout;
    if (layout == TFFR_POINTS_GENERAL) {
        s = build_general(p);
        if (s != TFFR_OK) return s;
    }
    STAGE_END(TFFR_STAGE_POINTS);
    p->have_points = true;
    return TFFR_OK;
}

int tffr_weights(tffr_plan_t p, const tffr_weight_opts* opts, float* D_out, int64_t* n_kept) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points) return fail(p, TFFR_ERR_NOT_READY, "tffr_weights before tffr_set_points");
    tffr_weight_opts o;
    tffr_default_weight_opts(&o);
    if (opts) o = *opts;
    if (o.mode < TFFR_WEIGHTS_TFFR || o.mode > TFFR_WEIGHTS_USER) return fail(p, TFFR_ERR_INVALID_ARG, "mode");
    if (!(o.q > 0) || !(o.q < 1e6) || !(o.a >= 0) || !(o.a < 1e3) || !(o.tau == o.tau) || !(std::fabs(o.tau) < 1e30))
        return fail(p, TFFR_ERR_INVALID_ARG, "a, q or tau out of range");
    if (o.mode == TFFR_WEIGHTS_USER && !o.user_D && p->N > 0) return fail(p, TFFR_ERR_INVALID_ARG, "user_D");
    const int64_t N = p->N;
    p->have_weights = false;
    p->normal_ready = false;
    p->n_kept = -1;
    WeightArgs& A = p->wargs;
    std::memset(&A, 0, sizeof(A));
    A.mode = o.mode;
    A.separable = o.separable ? 1 : 0;
    A.tau = (float)o.tau;
    A.tau_d = o.tau;
    A.guard = 1e-5f;
    A.a = o.a;
    A.q = o.q;
    A.e_minus = std::exp(-o.a / 2.0);
    A.e_plus = std::exp(o.a / 2.0);
    A.reach = (int)std::ceil(o.q) + 1;
    if (!(p->fit_valid && p->fit_cache.a == A.a && p->fit_cache.q == A.q)) {
        p->fit_cache = A;
        fit_weights(p->fit_cache);
        p->fit_valid = true;
    }
    copy_fit(A, p->fit_cache);
    if (N > 0 && o.mode == TFFR_WEIGHTS_TFFR && p->layout == TFFR_POINTS_ROWS) CK(grow(p, p->defer, N));
    STAGE_BEGIN(TFFR_STAGE_WEIGHTS);
    if (N > 0 && o.mode == TFFR_WEIGHTS_USER) {
        CK(grow(p, p->D, N));
        CK(cudaMemcpyAsync(p->D.ptr, o.user_D, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
        A.user_D = p->D.ptr;
    }
    // Materialise D in the caller's order only when asked for, or for general
    // points (whose kernels read it); the pulse-row kernels evaluate it inline.
    const bool need_D = N > 0 && (D_out || n_kept || p->layout == TFFR_POINTS_GENERAL);
    if (need_D) {
        CK(grow(p, p->D, N));
        CK(cudaMemsetAsync(p->d_kept.ptr, 0, sizeof(unsigned long long), p->stream));
        k_weights<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->lam_x, p->lam_y, p->Mx, p->My, A, p->D.ptr,
                                                          p->d_kept.ptr);
        CK_LAUNCH("k_weights");
        if (p->layout == TFFR_POINTS_GENERAL) {
            k_gather_weights<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->perm.ptr, p->D.ptr, p->sD.ptr);
            CK_LAUNCH("k_gather_weights");
        }
        if (D_out)
            CK(cudaMemcpyAsync(D_out, p->D.ptr, (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
    }
    STAGE_END(TFFR_STAGE_WEIGHTS);
    if (n_kept) {
        unsigned long long k = 0;
        if (N > 0) {
            CK(cudaMemcpyAsync(&k, p->d_kept.ptr, sizeof(k), cudaMemcpyDeviceToHost, p->stream));
            CK(cudaStreamSynchronize(p->stream));
        }
        *n_kept = (int64_t)k;
        p->n_kept = (int64_t)k;
    }
    p->have_weights = true;
    return TFFR_OK;
}

int tffr_adjoint(tffr_plan_t p, const void* values, void* image) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points || !p->have_weights) return fail(p, TFFR_ERR_NOT_READY, "adjoint before points/weights");
    if (!image || (p->N > 0 && !values)) return fail(p, TFFR_ERR_INVALID_ARG, "NULL pointer");
    float2* img = reinterpret_cast<float2*>(image);
    if (p->N == 0) {
        CK(cudaMemsetAsync(img, 0, (size_t)p->Mx * p->My * sizeof(float2), p->stream));
        return TFFR_OK;
    }
    switch (p->values) {
        case TFFR_VALUES_C64: return adjoint_impl<float2>(p, values, img);
        case TFFR_VALUES_C128: return adjoint_impl<double2>(p, values, img);
        case TFFR_VALUES_F16: return adjoint_impl<__half2>(p, values, img);
        default: return adjoint_impl<__nv_bfloat162>(p, values, img);
    }
}

int tffr_forward(tffr_plan_t p, const void* image, void* values, int apply_weights) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points || !p->have_weights) return fail(p, TFFR_ERR_NOT_READY, "forward before points/weights");
    if (!image || (p->N > 0 && !values)) return fail(p, TFFR_ERR_INVALID_ARG, "NULL pointer");
    if (p->N == 0) return TFFR_OK;
    const float2* img = reinterpret_cast<const float2*>(image);
    switch (p->values) {
        case TFFR_VALUES_C128: return forward_impl<double2>(p, img, values, apply_weights);
        default: return forward_impl<float2>(p, img, values, apply_weights);
    }
}

// ---------------------------------------------------------------------------
// Toeplitz normal operator
// ---------------------------------------------------------------------------
namespace {

__global__ void k_normal_inputs(int64_t N, const double* __restrict__ lam_x, const double* __restrict__ lam_y,
                                double* __restrict__ lx2, double* __restrict__ ly2, float2* __restrict__ ones) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        lx2[n] = 2.0 * lam_x[n];
        ly2[n] = 2.0 * lam_y[n];
        ones[n] = make_float2(1.0f, 0.0f);
    }
}

// k(m) for m in [-M, M)^2 (per axis) as the image of a plan with twice the
// sides, coordinates 2 lam, unit samples and this plan's weights D (user
// weights there): that plan's pixel j sits at (j - M) / (2M), and 2 lam times
// it is lam (j - M) / M, so pixel j holds k(j - M).
int normal_kernel_image(tffr_plan_s* p, float2* g) {
    const int64_t N = p->N;
    DevBuf<double> lx2, ly2;
    DevBuf<float2> ones;
    tffr_plan_t q = nullptr;
    int s = TFFR_OK;
    auto cleanup = [&]() {                              // temporaries: not counted in the plan's bytes
        if (q) tffr_destroy(q);
        cudaStreamSynchronize(p->stream);
        p->device_bytes -= (size_t)lx2.cap * sizeof(double) + (size_t)ly2.cap * sizeof(double) +
                           (size_t)ones.cap * sizeof(float2);
        release(lx2); release(ly2); release(ones);
    };
    cudaError_t e = grow(p, lx2, N);
    if (e == cudaSuccess) e = grow(p, ly2, N);
    if (e == cudaSuccess) e = grow(p, ones, N);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(p, e, "tffr_normal_setup: allocation");
    }
    k_normal_inputs<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->lam_x, p->lam_y, lx2.ptr, ly2.ptr, ones.ptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(p, e, "k_normal_inputs");
    }
    tffr_opts o;
    tffr_default_opts(&o);
    o.width = p->w;
    o.beta = p->beta;
    o.values = TFFR_VALUES_C64;
    o.layout = p->layout_hint;
    s = tffr_plan(&q, 2 * p->Mx, 2 * p->My, &o, p->stream);
    if (s == TFFR_OK) s = tffr_set_points(q, N, lx2.ptr, ly2.ptr);
    if (s == TFFR_OK) {
        tffr_weight_opts wo;
        tffr_default_weight_opts(&wo);
        wo.mode = TFFR_WEIGHTS_USER;
        wo.user_D = p->D.ptr;
        s = tffr_weights(q, &wo, nullptr, nullptr);
    }
    if (s == TFFR_OK) s = tffr_adjoint(q, ones.ptr, g);
    if (s != TFFR_OK && q) p->last_error = std::string("tffr_normal_setup: ") + tffr_last_error(q);
    cleanup();
    return s;
}

}  // namespace

// ---------------------------------------------------------------------------
// Conjugate gradients on the weighted normal equations E^H D E f = E^H D y
// (the least-squares refinement of the one-step tFFR image).  Every vector
// operation and every reduction runs on the device; the step sizes are read
// from device scalars, so an iteration needs no host synchronisation.
// ---------------------------------------------------------------------------
namespace {

constexpr int kCgThreads = 256;

// Block sum of one double per thread, added to *out by one atomic per block.
__device__ __forceinline__ void block_add(double v, double* out) {
    __shared__ double s_part[kCgThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kCgThreads / 32; ++i) t += s_part[i];
        atomicAdd(out, t);
    }
}

// x = 0, p = r (r holds b = E^H D y), rr0 += |r|^2.
__global__ void __launch_bounds__(kCgThreads)
k_cg_start(int64_t n, const float2* __restrict__ r, float2* __restrict__ pv, float2* __restrict__ x,
           double* __restrict__ rr0) {
    float acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = r[i];
        pv[i] = v;
        x[i] = make_float2(0.f, 0.f);
        acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
    }
    block_add((double)acc, rr0);
}

// *out += Re sum conj(p) Ap.
__global__ void __launch_bounds__(kCgThreads)
k_cg_dot(int64_t n, const float2* __restrict__ pv, const float2* __restrict__ Ap, double* __restrict__ out) {
    float acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = pv[i], b = Ap[i];
        acc = fmaf(a.x, b.x, fmaf(a.y, b.y, acc));
    }
    block_add((double)acc, out);
}

// alpha = rr_k / pAp_k (0 when pAp_k <= 0); x += alpha p, r -= alpha Ap, rr_next += |r|^2.
__global__ void __launch_bounds__(kCgThreads)
k_cg_step(int64_t n, const double* __restrict__ rr_k, const double* __restrict__ pap_k, float2* __restrict__ x,
          float2* __restrict__ r, const float2* __restrict__ pv, const float2* __restrict__ Ap,
          double* __restrict__ rr_next) {
    const double pap = *pap_k;
    const float alpha = pap > 0.0 ? (float)(*rr_k / pap) : 0.0f;
    float acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 pi = pv[i], api = Ap[i];
        float2 xi = x[i], ri = r[i];
        xi.x = fmaf(alpha, pi.x, xi.x);
        xi.y = fmaf(alpha, pi.y, xi.y);
        ri.x = fmaf(-alpha, api.x, ri.x);
        ri.y = fmaf(-alpha, api.y, ri.y);
        x[i] = xi;
        r[i] = ri;
        acc = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, acc));
    }
    block_add((double)acc, rr_next);
}

// beta = rr_next / rr_k (0 when rr_k <= 0); p = r + beta p.
__global__ void __launch_bounds__(kCgThreads)
k_cg_dir(int64_t n, const double* __restrict__ rr_k, const double* __restrict__ rr_next,
         const float2* __restrict__ r, float2* __restrict__ pv) {
    const double rk = *rr_k;
    const float beta = rk > 0.0 ? (float)(*rr_next / rk) : 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 ri = r[i], pi = pv[i];
        pv[i] = make_float2(fmaf(beta, pi.x, ri.x), fmaf(beta, pi.y, ri.y));
    }
}

// The adjoint in the plan's value type (values: caller's samples).
int adjoint_dispatch(tffr_plan_s* p, const void* values, float2* img, bool weighted) {
    switch (p->values) {
        case TFFR_VALUES_C64: return adjoint_impl<float2>(p, values, img, weighted);
        case TFFR_VALUES_C128: return adjoint_impl<double2>(p, values, img, weighted);
        case TFFR_VALUES_F16: return adjoint_impl<__half2>(p, values, img, weighted);
        default: return adjoint_impl<__nv_bfloat162>(p, values, img, weighted);
    }
}

}  // namespace

int tffr_normal_setup(tffr_plan_t p) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points || !p->have_weights) return fail(p, TFFR_ERR_NOT_READY, "normal setup before points/weights");
    if (4 * p->Mx > kFftNMax || 4 * p->My > kFftNMax)
        return fail(p, TFFR_ERR_INVALID_ARG, "the Toeplitz embedding needs Mx, My <= 2048");
    p->normal_ready = false;
    const int64_t N = p->N;
    const int Mx2 = 2 * p->Mx, My2 = 2 * p->My;
    CK(grow(p, p->khat, (int64_t)Mx2 * My2));
    CK(grow(p, p->nwork1, (int64_t)Mx2 * My2));       // Khat build: all 2My rows; apply: My rows
    CK(grow(p, p->nwork2, (int64_t)Mx2 * p->My));
    if (N == 0) {
        CK(cudaMemsetAsync(p->khat.ptr, 0, (size_t)Mx2 * My2 * sizeof(float2), p->stream));
    } else {
        // D_n in sample order (for USER weights already in p->D)
        CK(grow(p, p->D, N));
        CK(cudaMemsetAsync(p->d_kept.ptr, 0, sizeof(unsigned long long), p->stream));
        k_weights<<<grid_for(N, 256), 256, 0, p->stream>>>(N, p->lam_x, p->lam_y, p->Mx, p->My, p->wargs, p->D.ptr,
                                                          p->d_kept.ptr);
        CK_LAUNCH("k_weights");
        const int s = normal_kernel_image(p, p->khat.ptr);   // k first, transformed in place below
        if (s != TFFR_OK) return s;
        // Khat = FFT2 of k arranged circularly ((-1)^(kx+ky) in frequency) / (4 Mx My)
        launch_fft_rows(p->lognx, -1, My2, p->stream, p->khat.ptr, Mx2, Mx2, tables_x(p), p->nwork1.ptr, Mx2, Mx2);
        CK_LAUNCH("k_fft_rows");
        launch_fft_cols_conv(p->logny, Mx2, p->stream, p->nwork1.ptr, My2, Mx2, tables_y(p), nullptr,
                             1.0f / ((float)Mx2 * (float)My2), p->khat.ptr, My2);
        CK_LAUNCH("k_fft_cols_conv");
    }
    CK(cudaStreamSynchronize(p->stream));
    p->normal_ready = true;
    return TFFR_OK;
}

int tffr_normal_apply(tffr_plan_t p, const void* image_in, void* image_out) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->normal_ready) return fail(p, TFFR_ERR_NOT_READY, "tffr_normal_apply before tffr_normal_setup");
    if (!image_in || !image_out) return fail(p, TFFR_ERR_INVALID_ARG, "NULL pointer");
    const int Mx2 = 2 * p->Mx;
    launch_fft_rows(p->lognx, -1, p->My, p->stream, reinterpret_cast<const float2*>(image_in), p->Mx, p->Mx,
                    tables_x(p), p->nwork1.ptr, Mx2, Mx2);
    CK_LAUNCH("k_fft_rows");
    launch_fft_cols_conv(p->logny, Mx2, p->stream, p->nwork1.ptr, p->My, Mx2, tables_y(p), p->khat.ptr, 0.0f,
                         p->nwork2.ptr, p->My);
    CK_LAUNCH("k_fft_cols_conv");
    launch_fft_rows(p->lognx, +1, p->My, p->stream, p->nwork2.ptr, Mx2, Mx2, tables_x(p),
                    reinterpret_cast<float2*>(image_out), p->Mx, p->Mx);
    CK_LAUNCH("k_fft_rows");
    return TFFR_OK;
}

int tffr_reconstruct(tffr_plan_t p, int64_t N, const double* lam_x, const double* lam_y,
                     const tffr_weight_opts* opts, const void* values, void* image) {
    int st = tffr_set_points(p, N, lam_x, lam_y);
    if (st == TFFR_OK) st = tffr_weights(p, opts, nullptr, nullptr);
    if (st == TFFR_OK) st = tffr_adjoint(p, values, image);
    return st;
}

int tffr_adjoint_unweighted(tffr_plan_t p, const void* values, void* image) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points || !p->have_weights) return fail(p, TFFR_ERR_NOT_READY, "adjoint before points/weights");
    if (!image || (p->N > 0 && !values)) return fail(p, TFFR_ERR_INVALID_ARG, "NULL pointer");
    float2* img = reinterpret_cast<float2*>(image);
    if (p->N == 0) {
        CK(cudaMemsetAsync(img, 0, (size_t)p->Mx * p->My * sizeof(float2), p->stream));
        return TFFR_OK;
    }
    return adjoint_dispatch(p, values, img, false);
}

int tffr_weight_grad(tffr_plan_t p, const void* grad_image, const void* values, float* grad_D) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points || !p->have_weights) return fail(p, TFFR_ERR_NOT_READY, "weight_grad before points/weights");
    if (!grad_image || (p->N > 0 && (!values || !grad_D))) return fail(p, TFFR_ERR_INVALID_ARG, "NULL pointer");
    if (p->N == 0) return TFFR_OK;
    const float2* g = reinterpret_cast<const float2*>(grad_image);
    switch (p->values) {
        case TFFR_VALUES_C64: return forward_impl<float2>(p, g, grad_D, 0, values);
        case TFFR_VALUES_C128: return forward_impl<double2>(p, g, grad_D, 0, values);
        case TFFR_VALUES_F16: return forward_impl<__half2>(p, g, grad_D, 0, values);
        default: return forward_impl<__nv_bfloat162>(p, g, grad_D, 0, values);
    }
}

int tffr_cg(tffr_plan_t p, const void* values, void* image, int iters, int use_toeplitz, double* residuals) {
    if (!p) return TFFR_ERR_INVALID_ARG;
    p->last_error.clear();
    if (!p->have_points || !p->have_weights) return fail(p, TFFR_ERR_NOT_READY, "tffr_cg before points/weights");
    if (use_toeplitz && !p->normal_ready) return fail(p, TFFR_ERR_NOT_READY, "tffr_cg: tffr_normal_setup first");
    if (iters < 0 || iters > 100000) return fail(p, TFFR_ERR_INVALID_ARG, "iters out of range");
    if (!image || (p->N > 0 && !values)) return fail(p, TFFR_ERR_INVALID_ARG, "NULL pointer");
    const int64_t n = (int64_t)p->Mx * p->My;
    float2* x = reinterpret_cast<float2*>(image);
    CK(grow(p, p->cg_r, n));
    CK(grow(p, p->cg_p, n));
    CK(grow(p, p->cg_Ap, n));
    CK(grow(p, p->cg_s, 2 * (int64_t)iters + 1));
    if (!use_toeplitz && p->N > 0) CK(grow(p, p->cg_y, p->N));
    double* rr = p->cg_s.ptr;                          // |r_k|^2, k = 0..iters
    double* pap = p->cg_s.ptr + iters + 1;             // Re <p_k, N p_k>, k < iters
    CK(cudaMemsetAsync(rr, 0, (size_t)(2 * iters + 1) * sizeof(double), p->stream));
    if (p->N == 0) {
        CK(cudaMemsetAsync(p->cg_r.ptr, 0, (size_t)n * sizeof(float2), p->stream));
    } else {
        const int s = adjoint_dispatch(p, values, p->cg_r.ptr, true);       // b = E^H D y
        if (s != TFFR_OK) return s;
    }
    const int blocks = grid_for(n, kCgThreads);
    k_cg_start<<<blocks, kCgThreads, 0, p->stream>>>(n, p->cg_r.ptr, p->cg_p.ptr, x, rr);
    CK_LAUNCH("k_cg_start");
    for (int k = 0; k < iters; ++k) {
        if (use_toeplitz) {
            const int s = tffr_normal_apply(p, p->cg_p.ptr, p->cg_Ap.ptr);
            if (s != TFFR_OK) return s;
        } else if (p->N > 0) {
            int s = forward_impl<float2>(p, p->cg_p.ptr, p->cg_y.ptr, 0);     // E p
            if (s == TFFR_OK) s = adjoint_impl<float2>(p, p->cg_y.ptr, p->cg_Ap.ptr, true);   // E^H D E p
            if (s != TFFR_OK) return s;
        } else {
            CK(cudaMemsetAsync(p->cg_Ap.ptr, 0, (size_t)n * sizeof(float2), p->stream));
        }
        k_cg_dot<<<blocks, kCgThreads, 0, p->stream>>>(n, p->cg_p.ptr, p->cg_Ap.ptr, pap + k);
        CK_LAUNCH("k_cg_dot");
        k_cg_step<<<blocks, kCgThreads, 0, p->stream>>>(n, rr + k, pap + k, x, p->cg_r.ptr, p->cg_p.ptr,
                                                         p->cg_Ap.ptr, rr + k + 1);
        CK_LAUNCH("k_cg_step");
        k_cg_dir<<<blocks, kCgThreads, 0, p->stream>>>(n, rr + k, rr + k + 1, p->cg_r.ptr, p->cg_p.ptr);
        CK_LAUNCH("k_cg_dir");
    }
    if (residuals) {
        std::vector<double> h(iters + 1);
        CK(cudaMemcpyAsync(h.data(), rr, (size_t)(iters + 1) * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
        for (int k = 0; k <= iters; ++k) residuals[k] = std::sqrt(std::max(0.0, h[k]));
    }
    return TFFR_OK;
}

// ---------------------------------------------------------------------------
// Batches of pulse-row patches: one persistent launch per image-size class
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct BatchClass {
    int logn = 0;
    std::vector<int> members;                          // indices into the batch's plans
    BatchPatch* d_patches = nullptr;
    int* d_first = nullptr;                            // row_first[n + 1], fine_first[n + 1], col_first[n + 1]
    int* d_counts = nullptr;                           // next item, done[n], fine_done[n]
    int rows_total = 0, fine_total = 0, cols_total = 0;
    int grid = 0, max_blocks = 1;
    float tuned_ms = 0.0f;                             // the tuner's best time per launch
    FftTables tab;
};

}  // namespace

struct tffr_batch_s {
    cudaStream_t stream = nullptr;
    std::vector<BatchClass> cls;
    BatchPatch* d_patches = nullptr;                   // every patch (the spread launch)
    int* d_row_tag = nullptr;                          // [rows_total] (patch << 16) | pulse row of each spread block
    BatchRow* d_rows = nullptr;                        // [rows_total] each spread block's pulse row
    int rows_total = 0, max_len = 0, w = 6;
    WeightArgs wa;
    TapPoly tp;
    int* d_err = nullptr;                              // [0] error bits, [1] abort flag
    int* d_defer = nullptr;                            // [samples]
    int n = 0;
    int64_t samples = 0;
    unsigned long long wait_ns = 1000000000ull;
    int hold = 0, tuned = 0, sms = 0;
    float spread_ms = 0.0f;                            // the tuner's time of the spread launch
};

namespace {

void batch_free(tffr_batch_s* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (BatchClass& c : b->cls) {
        if (c.d_patches) cudaFree(c.d_patches);
        if (c.d_first) cudaFree(c.d_first);
        if (c.d_counts) cudaFree(c.d_counts);
    }
    if (b->d_patches) cudaFree(b->d_patches);
    if (b->d_row_tag) cudaFree(b->d_row_tag);
    if (b->d_rows) cudaFree(b->d_rows);
    if (b->d_defer) cudaFree(b->d_defer);
    if (b->d_err) cudaFree(b->d_err);
    delete b;
}

BatchClassArgs class_args(const tffr_batch_s* b, const BatchClass& c) {
    BatchClassArgs a;
    const int n = (int)c.members.size();
    a.patches = c.d_patches;
    a.row_first = c.d_first;
    a.fine_first = c.d_first + (n + 1);
    a.col_first = c.d_first + 2 * (n + 1);
    a.npatch = n;
    a.rows_total = c.rows_total;
    a.fine_total = c.fine_total;
    a.total = c.rows_total + c.fine_total + c.cols_total;
    a.next = c.d_counts;
    a.done = c.d_counts + 1;
    a.fine_done = c.d_counts + 1 + n;
    a.err = b->d_err;
    a.wait_ns = b->wait_ns;
    a.hold = b->hold;
    a.tab = c.tab;
    return a;
}

cudaError_t launch_spread(const tffr_batch_s* b) {
    BatchSpreadArgs a;
    a.patches = b->d_patches;
    a.rows = b->d_rows;
    a.row_tag = b->d_row_tag;
    a.npatch = b->n;
    a.wa = b->wa;
    a.tp = b->tp;
    a.defer_item = b->d_defer;
    launch_batch_spread(b->w, b->rows_total, b->max_len, b->stream, a);
    return cudaGetLastError();
}

cudaError_t launch_class(const tffr_batch_s* b, const BatchClass& c) {
    cudaError_t e = cudaMemsetAsync(c.d_counts, 0, (2 * c.members.size() + 1) * sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    launch_batch_fft(c.logn, c.grid, b->stream, class_args(b, c));
    return cudaGetLastError();
}

bool same_weights(const WeightArgs& x, const WeightArgs& y) {
    return x.mode == y.mode && x.separable == y.separable && x.tau_d == y.tau_d && x.a == y.a && x.q == y.q;
}

BatchPatch patch_desc(const tffr_plan_s* p, const void* values, void* image) {
    BatchPatch d;
    d.pulse = p->pulse_order ? 1 : 0;
    d.M = p->Mx;
    d.n = p->nx;
    d.P = p->P;
    d.ldq = (p->P + 3) & ~3;
    d.K = p->ell_k;
    d.row_start = p->row_start.ptr;
    d.row_end = p->row_end.ptr;
    d.row_clo = p->row_clo.ptr;
    d.row_len = p->row_len.ptr;
    d.row_ly = p->row_ly.ptr;
    d.row_fy = p->row_fy.ptr;
    d.row_lam_y = p->row_lam_y.ptr;
    d.rank_row = p->rank_row.ptr;
    d.ell_first = p->ell_first.ptr;
    d.ell_w = p->ell_w.ptr;
    d.deap_x = p->deap_x.ptr;
    d.deap_y = p->deap_y.ptr;
    d.F = p->T.ptr;
    d.tap_start = p->tap_start.ptr;
    d.taps = p->tap_list.ptr;
    d.row_off = p->row_off.ptr;
    d.R = p->R.ptr;
    d.lam_x = p->lam_x;
    d.user_D = p->wargs.mode == TFFR_WEIGHTS_USER ? p->D.ptr : nullptr;
    d.values = reinterpret_cast<const float2*>(values);
    d.image = reinterpret_cast<float2*>(image);
    return d;
}

}  // namespace

extern "C" {

int tffr_batch_create(const tffr_plan_t* plans, int n, const void* const* values, void* const* images,
                      tffr_stream_t stream, tffr_batch_t* out) {
    if (!out) return TFFR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || !values || !images || n < 1) return TFFR_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const tffr_plan_s* p = plans[i];
        if (!p || !values[i] || !images[i]) return TFFR_ERR_INVALID_ARG;
        if (!p->have_points || !p->have_weights) return TFFR_ERR_NOT_READY;
        if (p->layout != TFFR_POINTS_ROWS || p->values != TFFR_VALUES_C64 || p->Mx != p->My || p->P < 1 ||
            !batch_class_supported(p->lognx, p->w))
            return TFFR_ERR_INVALID_ARG;
        // one kernel shape and one weight rule for the whole batch
        if (p->w != plans[0]->w || p->beta != plans[0]->beta || !same_weights(p->wargs, plans[0]->wargs))
            return TFFR_ERR_INVALID_ARG;
        if (p->P >= (1 << 16) || i >= (1 << 15)) return TFFR_ERR_INVALID_ARG;   // the row tags' encoding
    }
    tffr_batch_s* b = new (std::nothrow) tffr_batch_s();
    if (!b) return TFFR_ERR_OOM;
    b->stream = (cudaStream_t)stream;
    b->n = n;
    b->w = plans[0]->w;
    b->wa = plans[0]->wargs;
    b->tp = plans[0]->taps;
    auto bail = [&](cudaError_t e) {
        batch_free(b);
        return e == cudaErrorMemoryAllocation ? TFFR_ERR_OOM : TFFR_ERR_CUDA;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bail(e);
    // the spread launch: every patch, one block per pulse row
    std::vector<BatchPatch> all(n);
    std::vector<int> row_first(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const tffr_plan_s* p = plans[i];
        all[i] = patch_desc(p, values[i], images[i]);
        all[i].defer_off = (int)std::min<int64_t>(b->samples, 0x7fffffff);   // larger batches are rejected below
        row_first[i + 1] = row_first[i] + p->P;
        b->samples += p->N;
        b->max_len = std::max(b->max_len, p->max_len);
        BatchClass* c = nullptr;                          // classes: one line length each
        for (BatchClass& x : b->cls)
            if (x.logn == p->lognx) c = &x;
        if (!c) {
            b->cls.emplace_back();
            c = &b->cls.back();
            c->logn = p->lognx;
            c->tab = tables_x(p);
        }
        c->members.push_back(i);
    }
    b->rows_total = row_first[n];
    std::vector<int> row_tag(std::max(1, b->rows_total));
    for (int i = 0; i < n; ++i)
        for (int r = row_first[i]; r < row_first[i + 1]; ++r) row_tag[r] = (i << 16) | (r - row_first[i]);
    e = cudaMalloc((void**)&b->d_patches, n * sizeof(BatchPatch));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_row_tag, row_tag.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_patches, all.data(), n * sizeof(BatchPatch), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_row_tag, row_tag.data(), row_tag.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_rows, row_tag.size() * sizeof(BatchRow));
    // each spread block's pulse row, from the plans' row arrays once their work is done
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamSynchronize(plans[i]->stream);
    if (e == cudaSuccess && b->rows_total > 0) {
        BatchSpreadArgs ra;
        ra.patches = b->d_patches;
        ra.rows = b->d_rows;
        ra.row_tag = b->d_row_tag;
        ra.npatch = n;
        launch_batch_rows(b->rows_total, b->stream, ra);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) return bail(e);
    for (BatchClass& c : b->cls) {
        const int m = (int)c.members.size();
        std::vector<BatchPatch> hp(m);
        std::vector<int> first(3 * (m + 1), 0);
        for (int j = 0; j < m; ++j) {
            const tffr_plan_s* p = plans[c.members[j]];
            hp[j] = all[c.members[j]];
            const bool pulse = hp[j].pulse != 0;
            first[j + 1] = first[j] + (pulse ? p->P : 0);                          // row items
            first[m + 1 + j + 1] = first[m + 1 + j] + (pulse ? 0 : p->nx);         // fine-row items
            first[2 * (m + 1) + j + 1] = first[2 * (m + 1) + j] + p->Mx;           // column items
        }
        c.rows_total = first[m];
        c.fine_total = first[2 * m + 1];
        c.cols_total = first[3 * m + 2];
        c.max_blocks = std::max(1, batch_max_blocks_per_sm(c.logn));
        c.grid = b->sms * c.max_blocks;
        e = cudaMalloc((void**)&c.d_patches, m * sizeof(BatchPatch));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c.d_first, first.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c.d_counts, (2 * m + 1) * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(c.d_patches, hp.data(), m * sizeof(BatchPatch), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(e);
    }
    e = cudaMalloc((void**)&b->d_err, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_defer, std::max<int64_t>(1, b->samples) * sizeof(int));
    if (e != cudaSuccess) return bail(e);
    if (b->samples >= (int64_t)0x7fffffff) {
        batch_free(b);
        return TFFR_ERR_INVALID_ARG;
    }
    *out = b;
    return TFFR_OK;
}

int tffr_batch_adjoint(tffr_batch_t b) {
    if (!b) return TFFR_ERR_INVALID_ARG;
    if (launch_spread(b) != cudaSuccess) return TFFR_ERR_CUDA;
    for (const BatchClass& c : b->cls)
        if (launch_class(b, c) != cudaSuccess) return TFFR_ERR_CUDA;
    return TFFR_OK;
}

int tffr_batch_wait(tffr_batch_t b) {
    if (!b) return TFFR_ERR_INVALID_ARG;
    int err[2] = {0, 0};
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TFFR_ERR_CUDA;
    if (cudaMemcpy(err, b->d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return TFFR_ERR_CUDA;
    if (err[0] || err[1]) {
        if (cudaMemset(b->d_err, 0, sizeof(err)) != cudaSuccess) return TFFR_ERR_CUDA;
        return TFFR_ERR_TIMEOUT;
    }
    return TFFR_OK;
}

int tffr_batch_set_wait(tffr_batch_t b, double wait_s, int hold_rows) {
    if (!b || !(wait_s > 0.0) || wait_s > 60.0) return TFFR_ERR_INVALID_ARG;
    b->wait_ns = (unsigned long long)(wait_s * 1e9);
    b->hold = hold_rows ? 1 : 0;
    return TFFR_OK;
}

int tffr_batch_tune(tffr_batch_t b, int reps) {
    if (!b || reps < 1 || reps > 1000) return TFFR_ERR_INVALID_ARG;
    if (launch_spread(b) != cudaSuccess) return TFFR_ERR_CUDA;     // the FFT launches read the row buffers
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TFFR_ERR_CUDA;
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess) return TFFR_ERR_CUDA;
    if (cudaEventCreate(&t1) != cudaSuccess) {
        cudaEventDestroy(t0);
        return TFFR_ERR_CUDA;
    }
    int status = TFFR_OK;
    {
        cudaError_t e = cudaEventRecord(t0, b->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_spread(b);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) status = TFFR_ERR_CUDA;
        b->spread_ms = ms / (float)reps;
    }
    for (BatchClass& c : b->cls) {
        if (status != TFFR_OK) break;
        float best = 1e30f;
        int best_grid = c.grid;
        std::vector<int> blocks;                                      // 1, 2, 4, ... and the most that fit
        for (int x = 1; x < c.max_blocks; x *= 2) blocks.push_back(x);
        blocks.push_back(c.max_blocks);
        for (int bps : blocks) {
            c.grid = b->sms * bps;
            cudaError_t e = launch_class(b, c);                       // warm
            if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_class(b, c);
            if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess) {
                status = TFFR_ERR_CUDA;
                break;
            }
            if (ms < best) {
                best = ms;
                best_grid = c.grid;
            }
        }
        c.grid = best_grid;
        c.tuned_ms = best / (float)reps;
        if (status != TFFR_OK) break;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (status == TFFR_OK) {
        b->tuned = 1;
        status = tffr_batch_wait(b);                                  // a timed-out tuning launch shows here
    }
    return status;
}

int tffr_batch_get_info(tffr_batch_t b, tffr_batch_info* info) {
    if (!b || !info) return TFFR_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_patches = b->n;
    info->n_classes = (int)b->cls.size();
    info->samples = b->samples;
    info->width = b->w;
    info->spread_ms = b->spread_ms;
    info->tuned = b->tuned;
    for (int i = 0; i < (int)b->cls.size() && i < TFFR_BATCH_MAX_CLASSES; ++i) {
        const BatchClass& c = b->cls[i];
        info->class_side[i] = (1 << c.logn) / 2;
        info->class_patches[i] = (int)c.members.size();
        info->class_blocks[i] = c.grid;
        info->class_ms[i] = c.tuned_ms;
    }
    return TFFR_OK;
}

int tffr_batch_destroy(tffr_batch_t b) {
    batch_free(b);
    return TFFR_OK;
}

int tffr_weights_noalloc(int64_t N, const double* lam_x, const double* lam_y, int Mx, int My,
                         const tffr_weight_opts* opts, float* D_out, int64_t* n_kept, tffr_stream_t stream) {
    if (N < 0 || N > kNaMaxN || Mx < 1 || My < 1) return TFFR_ERR_INVALID_ARG;
    tffr_weight_opts o;
    tffr_default_weight_opts(&o);
    if (opts) o = *opts;
    if (o.mode < TFFR_WEIGHTS_TFFR || o.mode > TFFR_WEIGHTS_USER) return TFFR_ERR_INVALID_ARG;
    if (!(o.q > 0) || !(o.q < 1e6) || !(o.a >= 0) || !(o.a < 1e3) || !(o.tau == o.tau) || !(std::fabs(o.tau) < 1e30))
        return TFFR_ERR_INVALID_ARG;
    if (N > 0 && (!D_out || (o.mode == TFFR_WEIGHTS_TFFR && !lam_x) ||
                  (o.mode == TFFR_WEIGHTS_TFFR && o.separable && !lam_y) ||
                  (o.mode == TFFR_WEIGHTS_USER && !o.user_D)))
        return TFFR_ERR_INVALID_ARG;
    if (N == 0) {
        if (n_kept) *n_kept = 0;
        return TFFR_OK;
    }
    if (o.mode == TFFR_WEIGHTS_USER) {
        // the kernel reads user_D while it writes D_out: the two ranges must not overlap
        const uintptr_t d0 = reinterpret_cast<uintptr_t>(D_out), u0 = reinterpret_cast<uintptr_t>(o.user_D);
        const uintptr_t bytes = (uintptr_t)N * sizeof(float);
        if (d0 < u0 + bytes && u0 < d0 + bytes) return TFFR_ERR_INVALID_ARG;
    }
    WeightArgs A;
    std::memset(&A, 0, sizeof(A));
    A.mode = o.mode;
    A.separable = o.separable ? 1 : 0;
    A.tau = (float)o.tau;
    A.tau_d = o.tau;
    A.a = o.a;
    A.q = o.q;
    A.e_minus = std::exp(-o.a / 2.0);
    A.e_plus = std::exp(o.a / 2.0);
    A.reach = (int)std::ceil(o.q) + 1;
    A.user_D = o.user_D;
    NoAllocScratch* sc = nullptr;
    if (noalloc_scratch(&sc) != cudaSuccess) return TFFR_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(&sc->done, 0, sizeof(unsigned int), st) != cudaSuccess) return TFFR_ERR_CUDA;
    const int blocks = (int)((N + kNaPerBlock - 1) / kNaPerBlock);
    k_weights_noalloc<<<blocks, kNaThreads, 0, st>>>(N, lam_x, lam_y, Mx, My, A, D_out, sc);
    if (cudaGetLastError() != cudaSuccess) return TFFR_ERR_CUDA;
    if (n_kept) {
        unsigned long long k = 0;
        if (cudaMemcpyAsync(&k, &sc->total, sizeof(k), cudaMemcpyDeviceToHost, st) != cudaSuccess) return TFFR_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return TFFR_ERR_CUDA;
        *n_kept = (int64_t)k;
    }
    return TFFR_OK;
}

}  // extern "C"
