// Plain views of plan-owned device arrays, passed to kernels by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tffr {

// One azimuth tap of a pulse row onto a fine row: add wy * R[off + i] to
// fine x cell (clo + i) mod nx, i < len.
struct TapEntry {
    long long off;
    int clo;
    int len;
    float wy;
    int p;
};

// Slots of the fine-row azimuth-tap table (pulse-row order of the FFT passes).
constexpr int kEllMax = 8;

struct RowsView {
    int P;                          // pulse rows
    const int* row_start;           // [P] first sample of the row (rows are contiguous runs)
    const int* row_end;             // [P] one past its last sample
    const int* row_clo;             // [P] first fine x cell of the row buffer
    const int* row_len;             // [P] cells in the row buffer (nx: periodic row)
    const int* row_ly;              // [P] fine y cell floor(2 lam_y)
    const float* row_fy;            // [P] fine y offset in [0, 1]
    const double* row_lam_y;        // [P] lam_y of the row
    const int64_t* row_off;         // [P] offset of the row buffer in R (cells)
    const int* rank_row;            // [P] pulse row at each place in fine-y order (pulse-row order of the adjoint)
    const int* tap_start;           // [ny + 1] taps of each fine row (CSR)
    const TapEntry* taps;           // [P * w]
};

struct GeneralView {
    const int* bucket_start;        // [ny + 1] samples grouped by floor(2 lam_y) mod ny
    const int* perm;                // [N] sorted position -> sample index
    const int* slx;                 // [N] fine x cell, sorted order
    const float* sfx;               // [N] fine x offset, sorted order
    const float* sfy;               // [N] fine y offset, sorted order
    const float* sD;                // [N] weights, sorted order
};

struct FftTables {
    const float2* twh;              // exp(2 pi i 64 h / n), h < max(1, n / 64)
    const float2* twl;              // exp(2 pi i l / n), l < min(64, n)
    const float2* tt;               // exp(2 pi i m / nt), m < nt = min(n, 1024)
};

}  // namespace tffr
