// Instantiations and host launchers of the FFT line kernels, one per line
// length 2^5 .. 2^13 (kept in their own translation unit so that the build
// compiles them in parallel with the rest of the library).

#include <algorithm>

#include "line_kernels.cuh"
#include "line_launch.h"

namespace tffr {

namespace {

template <int LOGN>
size_t line_smem() {
    return line_smem_bytes<LOGN>();
}

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int LOGN>
cudaError_t attrs_for() {
    const size_t b = line_smem<LOGN>();
    cudaError_t e = smem_attr(k_adj_rows<LOGN>, b);
    if (e == cudaSuccess) e = smem_attr(k_adj_rows_general<LOGN>, b);
    if (e == cudaSuccess) e = smem_attr(k_adj_cols<LOGN>, b);
    if (e == cudaSuccess) e = smem_attr(k_fwd_cols<LOGN>, b);
    if (e == cudaSuccess) e = smem_attr(k_fwd_rows<LOGN, true>, b);
    if (e == cudaSuccess) e = smem_attr(k_fwd_rows<LOGN, false>, b);
    if (e == cudaSuccess) e = smem_attr(k_adj_rows_pulse<LOGN>, b);
    if (e == cudaSuccess) e = smem_attr(k_fwd_rows_pulse<LOGN>, b);
    if (e == cudaSuccess) e = smem_attr(k_adj_cols_pulse<LOGN, 1>, line_smem_pulse_cols<LOGN>());
    if (e == cudaSuccess) e = smem_attr(k_adj_cols_pulse<LOGN, 2>, line_smem_pulse_cols<LOGN>());
    if (e == cudaSuccess) e = smem_attr(k_fwd_cols_pulse<LOGN>, line_smem_pulse_cols<LOGN>());
    if (e == cudaSuccess) e = smem_attr(k_fft_rows<LOGN, -1>, b);
    if (e == cudaSuccess) e = smem_attr(k_fft_rows<LOGN, +1>, b);
    if (e == cudaSuccess) e = smem_attr(k_fft_cols_conv<LOGN>, b);
    return e;
}

}  // namespace

#define TFFR_LOGN_SWITCH(logn, CALL) \
    switch (logn) {                  \
        case 5: CALL(5); break;      \
        case 6: CALL(6); break;      \
        case 7: CALL(7); break;      \
        case 8: CALL(8); break;      \
        case 9: CALL(9); break;      \
        case 10: CALL(10); break;    \
        case 11: CALL(11); break;    \
        case 12: CALL(12); break;    \
        default: CALL(13); break;    \
    }

cudaError_t line_set_attributes() {
    cudaError_t e = cudaSuccess;
#define ATTR(LG) if (e == cudaSuccess) e = attrs_for<LG>()
    ATTR(5); ATTR(6); ATTR(7); ATTR(8); ATTR(9); ATTR(10); ATTR(11); ATTR(12); ATTR(13);
#undef ATTR
    return e;
}

void launch_adj_rows(int lognx, int ny, cudaStream_t s, const RowsView& rv, const float2* R, int w,
                     const TapPoly& tp, FftTables tab, const float* deap_x, float2* T) {
#define L(LG) k_adj_rows<LG><<<ny, Line<LG>::T, line_smem<LG>(), s>>>(rv, R, ny, w, tp, tab, deap_x, T)
    TFFR_LOGN_SWITCH(lognx, L)
#undef L
}

void launch_adj_rows_general(int lognx, int ny, cudaStream_t s, const GeneralView& gv, const float2* sval, int w,
                             const TapPoly& tp, FftTables tab, const float* deap_x, float2* T) {
#define L(LG) k_adj_rows_general<LG><<<ny, Line<LG>::T, line_smem<LG>(), s>>>(gv, sval, ny, w, tp, tab, deap_x, T)
    TFFR_LOGN_SWITCH(lognx, L)
#undef L
}

void launch_adj_cols(int logny, int Mx, cudaStream_t s, const float2* T, FftTables tab, const float* deap_y,
                     float2* img) {
#define L(LG) k_adj_cols<LG><<<Mx, Line<LG>::T, line_smem<LG>(), s>>>(T, Mx, tab, deap_y, img)
    TFFR_LOGN_SWITCH(logny, L)
#undef L
}

void launch_fwd_cols(int logny, int Mx, cudaStream_t s, const float2* img, FftTables tab, const float* deap_y,
                     const float* deap_x, float2* T) {
#define L(LG) k_fwd_cols<LG><<<Mx, Line<LG>::T, line_smem<LG>(), s>>>(img, Mx, tab, deap_y, deap_x, T)
    TFFR_LOGN_SWITCH(logny, L)
#undef L
}

void launch_fwd_rows(int lognx, int ny, bool rows, cudaStream_t s, const RowsView& rv, const GeneralView& gv,
                     const float2* T, int w, const TapPoly& tp, FftTables tab, float2* R, float2* acc) {
    if (rows) {
#define L(LG) k_fwd_rows<LG, true><<<ny, Line<LG>::T, line_smem<LG>(), s>>>(rv, gv, T, ny, w, tp, tab, R, acc)
        TFFR_LOGN_SWITCH(lognx, L)
#undef L
    } else {
#define L(LG) k_fwd_rows<LG, false><<<ny, Line<LG>::T, line_smem<LG>(), s>>>(rv, gv, T, ny, w, tp, tab, R, acc)
        TFFR_LOGN_SWITCH(lognx, L)
#undef L
    }
}

void launch_adj_rows_pulse(int lognx, int P, cudaStream_t s, const RowsView& rv, const float2* R, FftTables tab,
                           const float* deap_x, float2* F) {
#define L(LG) k_adj_rows_pulse<LG><<<P, Line<LG>::T, line_smem<LG>(), s>>>(rv, R, tab, deap_x, F)
    TFFR_LOGN_SWITCH(lognx, L)
#undef L
}

void launch_adj_cols_pulse(int logny, int Mx, int P, cudaStream_t s, const float2* F, FftTables tab,
                           const int* ell_first, const float4* ell_w, int K, const float* deap_y, float2* img) {
    // clusters resident at once (two CTAs per SM): the prefetch distance in blocks
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 152;
    }
    const int ahead = std::max(1, sms * 2 / kColCluster);
    if (K <= 4) {
#define L(LG) k_adj_cols_pulse<LG, 1><<<Mx, Line<LG>::T, line_smem_pulse_cols<LG>(), s>>>(F, P, Mx, tab, ell_first, \
                                                                                         ell_w, deap_y, img, ahead)
        TFFR_LOGN_SWITCH(logny, L)
#undef L
    } else {
#define L(LG) k_adj_cols_pulse<LG, 2><<<Mx, Line<LG>::T, line_smem_pulse_cols<LG>(), s>>>(F, P, Mx, tab, ell_first, \
                                                                                         ell_w, deap_y, img, ahead)
        TFFR_LOGN_SWITCH(logny, L)
#undef L
    }
}

void launch_fwd_cols_pulse(int logny, int Mx, int P, cudaStream_t s, const float2* img, FftTables tab,
                           const float* deap_y, const float* deap_x, const int* q_ly, const float* q_wy, int w,
                           float2* F) {
#define L(LG) k_fwd_cols_pulse<LG><<<Mx, Line<LG>::T, line_smem_pulse_cols<LG>(), s>>>(img, Mx, tab, deap_y, deap_x, \
                                                                                      q_ly, q_wy, w, P, F)
    TFFR_LOGN_SWITCH(logny, L)
#undef L
}

void launch_fwd_rows_pulse(int lognx, int P, cudaStream_t s, const RowsView& rv, const float2* F, FftTables tab,
                           float2* R) {
#define L(LG) k_fwd_rows_pulse<LG><<<P, Line<LG>::T, line_smem<LG>(), s>>>(rv, F, tab, R)
    TFFR_LOGN_SWITCH(lognx, L)
#undef L
}

void launch_fft_rows(int logn, int sgn, int rows, cudaStream_t s, const float2* in, int ld_in, int n_in,
                     FftTables tab, float2* out, int ld_out, int n_out) {
    if (sgn < 0) {
#define L(LG) k_fft_rows<LG, -1><<<rows, Line<LG>::T, line_smem<LG>(), s>>>(in, ld_in, n_in, tab, out, ld_out, n_out)
        TFFR_LOGN_SWITCH(logn, L)
#undef L
    } else {
#define L(LG) k_fft_rows<LG, +1><<<rows, Line<LG>::T, line_smem<LG>(), s>>>(in, ld_in, n_in, tab, out, ld_out, n_out)
        TFFR_LOGN_SWITCH(logn, L)
#undef L
    }
}

void launch_fft_cols_conv(int logn, int cols, cudaStream_t s, const float2* in, int n_in, int ld, FftTables tab,
                          const float2* khat, float scale, float2* out, int n_out) {
#define L(LG) k_fft_cols_conv<LG><<<cols, Line<LG>::T, line_smem<LG>(), s>>>(in, n_in, ld, tab, khat, scale, out, n_out)
    TFFR_LOGN_SWITCH(logn, L)
#undef L
}

}  // namespace tffr
