// Persistent adjoint of a batch of pulse-row patches: device descriptors and
// the host launcher (batch.cu).  One launch per image-size class runs every
// patch of that class: fused spread + x-FFT items for all pulse rows, then
// column items, claimed from a device counter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels_points.cuh"
#include "types.cuh"

namespace tffr {

// One patch: the plan's arrays (points, weights, pulse rows, tap table,
// intermediate) and the caller's fixed value and image buffers.  Patches in
// the pulse-row order of the passes (at most M pulse rows) run fused spread +
// x FFT items per pulse row and gather the azimuth taps in the column items;
// the others run spread items (row buffers R), then fine-row items (azimuth
// taps and x FFT of each of the n fine rows into T), then plain column items.
struct BatchPatch {
    int pulse;                          // 1: pulse-row order, 0: fine-row order
    int M, n, P, ldq, K;                // image side (square), fine grid side 2M, pulse rows, F stride, tap slots
    const int* row_start;
    const int* row_end;
    const int* row_clo;
    const int* row_len;
    const int* row_ly;
    const float* row_fy;
    const double* row_lam_y;
    const int* rank_row;                // pulse row at each place in fine-y order
    const int2* ell;                    // [K][n] fine-row tap table
    const float* deap_x;                // [M]
    const float* deap_y;                // [M]
    float2* F;                          // pulse-row order: [M / 4][ldq][4]; fine-row order: T [n][M]
    const int* tap_start;               // fine-row order: [n + 1] azimuth taps of each fine row (CSR)
    const TapEntry* taps;
    const int64_t* row_off;             // offset of each pulse row's buffer in R
    float2* R;                          // pulse-row buffers
    const double* lam_x;                // caller's coordinates
    const float* user_D;                // user weights (plan copy) or NULL
    const float2* values;               // caller's samples, complex64
    float2* image;                      // caller's image [M][M]
};

// Every launch-wide argument of one class's kernel.
struct BatchClassArgs {
    const BatchPatch* patches;          // [npatch]
    const int* row_first;               // [npatch + 1] first row item of each patch (P each)
    const int* fine_first;              // [npatch + 1] first fine-row item (n each in fine-row order, else 0)
    const int* col_first;               // [npatch + 1] first column item of each patch (M each)
    int npatch, rows_total, fine_total, total;   // items: rows, then fine rows, then columns
    int* next;                          // item counter, zero before the launch
    int* done;                          // [npatch] finished row items, zero before the launch
    int* fine_done;                     // [npatch] finished fine-row items, zero before the launch
    int* err;                           // [0] error bits (1: a wait timed out), [1] abort flag
    unsigned long long wait_ns;         // limit of one wait for a patch's rows
    int run;                            // samples per thread per spread tile
    int hold;                           // test hook: row items never publish (every wait times out)
    WeightArgs wa;                      // the class's weight evaluation (the patch's Mx decides the edges)
    TapPoly tp;
    FftTables tab;                      // twiddles of the class's line length
};

// Kernel attributes (dynamic shared memory) of every instantiation.
cudaError_t batch_set_attributes();

// Whether a class (line length 2^logn, spreading width w) has a kernel.
bool batch_class_supported(int logn, int w);

// Threads per block and dynamic shared memory of a class's kernel.
int batch_threads(int logn);
size_t batch_smem(int logn);
// Blocks of the class's kernel that fit on one SM.
int batch_max_blocks_per_sm(int logn, int w);

void launch_batch_class(int logn, int w, int grid, cudaStream_t s, const BatchClassArgs& a);

}  // namespace tffr
