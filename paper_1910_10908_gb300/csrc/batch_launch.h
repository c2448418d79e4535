// Adjoint of a batch of pulse-row patches: device descriptors and the host
// launchers (batch.cu).  One spread launch over every pulse row of every
// patch, then one persistent FFT launch per image-size class over the class's
// row, fine-row and column items, claimed from a device counter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels_points.cuh"
#include "kernels_spread.cuh"
#include "types.cuh"

namespace tffr {

// One patch: the plan's arrays (points, weights, pulse rows, tap table,
// intermediate) and the caller's fixed value and image buffers.  Patches in
// the pulse-row order of the passes (at most M pulse rows) run x-FFT items per
// pulse row and gather the azimuth taps in the column items; the others run
// fine-row items (azimuth taps and x FFT of each of the n fine rows into T),
// then plain column items.
struct BatchPatch {
    int pulse;                          // 1: pulse-row order, 0: fine-row order
    int M, n, P, ldq, K;                // image side (square), fine grid side 2M, pulse rows, F stride, tap slots
    int defer_off;                      // the patch's first slot in the batch's deferred-sample list
    const int* row_start;
    const int* row_end;
    const int* row_clo;
    const int* row_len;
    const int* row_ly;
    const float* row_fy;
    const double* row_lam_y;
    const int* rank_row;                // pulse row at each place in fine-y order
    const int* ell_first;               // [n] first place of each fine row's taps (fine-y order)
    const float4* ell_w;                // [2][n] tap weights of slots 0-3 and 4-7
    const float* deap_x;                // [M]
    const float* deap_y;                // [M]
    float2* F;                          // column-major: pulse-row order F [M][ldq]; fine-row order T [M][n]
    const int* tap_start;               // fine-row order: [n + 1] azimuth taps of each fine row (CSR)
    const TapEntry* taps;
    const int64_t* row_off;             // offset of each pulse row's buffer in R
    float2* R;                          // pulse-row buffers
    const double* lam_x;                // caller's coordinates
    const float* user_D;                // user weights (plan copy) or NULL
    const float2* values;               // caller's samples, complex64
    float2* image;                      // caller's image [M][M]
};

// One pulse row of the batch, for the spread launch (one block each): every
// value its setup needs in one place, so that the block's staging copies
// wait on a single load.
struct BatchRow {
    const double* lam;                  // the row's coordinates (the patch's lam_x + s0)
    const float2* val;                  // the row's samples
    float2* out;                        // the row's buffer in R
    int s0;                             // first sample, as an index into the patch's arrays
    int L;                              // samples
    int clo, len;                       // first fine cell and cells of the row buffer
    int tag;                            // (patch << 16) | pulse row
    int M, n;                           // the patch's image side and fine-grid side
    int d0;                             // the row's region of the deferred-sample list (defer_off + s0)
};

// The spread launch over every pulse row of every patch.
struct BatchSpreadArgs {
    const BatchPatch* patches;          // [npatch] every patch of the batch (npatch < 2^15, rows < 2^16)
    BatchRow* rows;                     // [blocks] each block's pulse row (filled at the batch's creation)
    const int* row_tag;                 // [blocks] (patch << 16) | pulse row of each block
    int npatch;
    WeightArgs wa;                      // the batch's weight evaluation (the patch's M decides the edges)
    TapPoly tp;
    int* defer_item;                    // [samples] per-row regions of the samples for the FP64 decision
};

// Every launch-wide argument of one class's persistent FFT kernel.
struct BatchClassArgs {
    const BatchPatch* patches;          // [npatch] the class's patches
    const int* row_first;               // [npatch + 1] first row item (P each in pulse-row order, else 0)
    const int* fine_first;              // [npatch + 1] first fine-row item (n each in fine-row order, else 0)
    const int* col_first;               // [npatch + 1] first column item of each patch (M each)
    int npatch, rows_total, fine_total, total;   // items: rows, then fine rows, then columns
    int* next;                          // item counter, zero before the launch
    int* done;                          // [npatch] finished row items, zero before the launch
    int* fine_done;                     // [npatch] finished fine-row items, zero before the launch
    int* err;                           // [0] error bits (1: a wait timed out), [1] abort flag
    unsigned long long wait_ns;         // limit of one wait for a patch's rows
    int hold;                           // test hook: items never publish (every wait times out)
    FftTables tab;                      // twiddles of the class's line length
};

// Whether a class (line length 2^logn, spreading width w) is supported.
bool batch_class_supported(int logn, int w);

// Dynamic shared memory of the spread launch for rows of up to max_len cells.
size_t batch_spread_smem(int max_len);

// Kernel attributes (dynamic shared memory) of every instantiation.
cudaError_t batch_set_attributes();

// Blocks of a class's FFT kernel that fit on one SM.
int batch_max_blocks_per_sm(int logn);

void launch_batch_spread(int w, int rows, int max_len, cudaStream_t s, const BatchSpreadArgs& a);
// Fills a.rows[0 .. rows) from the patches' row arrays (after their set_points).
void launch_batch_rows(int rows, cudaStream_t s, const BatchSpreadArgs& a);
void launch_batch_fft(int logn, int grid, cudaStream_t s, const BatchClassArgs& a);

}  // namespace tffr
