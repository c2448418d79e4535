// Host launchers of the FFT line kernels (compiled in line_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "types.cuh"

namespace tffr {

// Shared-memory limits of every line-kernel instantiation (once per device).
cudaError_t line_set_attributes();

// Pass 1 of the adjoint over the ny fine rows (line length 2^lognx).
void launch_adj_rows(int lognx, int ny, cudaStream_t s, const RowsView& rv, const float2* R, int w,
                     const TapPoly& tp, FftTables tab, const float* deap_x, float2* T);
void launch_adj_rows_general(int lognx, int ny, cudaStream_t s, const GeneralView& gv, const float2* sval, int w,
                             const TapPoly& tp, FftTables tab, const float* deap_x, float2* T);
// Pass 2 of the adjoint over the Mx wanted x modes (line length 2^logny).
void launch_adj_cols(int logny, int Mx, cudaStream_t s, const float2* T, FftTables tab, const float* deap_y,
                     float2* img);
// Forward twin: columns first, then rows.
void launch_fwd_cols(int logny, int Mx, cudaStream_t s, const float2* img, FftTables tab, const float* deap_y,
                     const float* deap_x, float2* T);
void launch_fwd_rows(int lognx, int ny, bool rows, cudaStream_t s, const RowsView& rv, const GeneralView& gv,
                     const float2* T, int w, const TapPoly& tp, FftTables tab, float2* R, float2* acc);

// Pulse-row order (rows layout, P <= M_y): F replaces T, indexed by place q
// in fine-y order (pulse row rv.rank_row[q]).  The adjoint keeps F by blocks
// of four columns, [Mx / 4][ldq][4] with ldq = P rounded up to 4: its x pass,
// block q, writes entry q of every column.  The forward twin keeps F by rows,
// [P][Mx]: its column pass writes row q from the taps of place q (q_ly: y
// cell, q_wy: [P][8] azimuth taps), its x pass reads it.
void launch_adj_rows_pulse(int lognx, int P, cudaStream_t s, const RowsView& rv, const float2* R, FftTables tab,
                           const float* deap_x, float2* F);
// Azimuth taps of the fine rows: fine row r sums weight k of ell_w (slots 0-3
// in ell_w[r], 4-7 in ell_w[2 My + r]) times the place ell_first[r] + k of F's
// column, k < K (places taken modulo P).
void launch_adj_cols_pulse(int logny, int Mx, int P, cudaStream_t s, const float2* F, FftTables tab,
                           const int* ell_first, const float4* ell_w, int K, const float* deap_y, float2* img);
void launch_fwd_cols_pulse(int logny, int Mx, int P, cudaStream_t s, const float2* img, FftTables tab,
                           const float* deap_y, const float* deap_x, const int* q_ly, const float* q_wy, int w,
                           float2* F);
void launch_fwd_rows_pulse(int lognx, int P, cudaStream_t s, const RowsView& rv, const float2* F, FftTables tab,
                           float2* R);

// Toeplitz normal operator: full line transforms (see line_kernels.cuh).
void launch_fft_rows(int logn, int sgn, int rows, cudaStream_t s, const float2* in, int ld_in, int n_in,
                     FftTables tab, float2* out, int ld_out, int n_out);
void launch_fft_cols_conv(int logn, int cols, cudaStream_t s, const float2* in, int n_in, int ld, FftTables tab,
                          const float2* khat, float scale, float2* out, int n_out);

}  // namespace tffr
