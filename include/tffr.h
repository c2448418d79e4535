/*
 * tffr.h -- C ABI of the GB300 tFFR library: the weighted adjoint non-uniform
 * FFT behind thresholded Fourier-frame reconstruction (tFFR) of stripmap SAR
 * data, and its forward twin.
 *
 * What is computed (McKay, Gelb, Jayasuriya, Monga, arXiv 1910.10908):
 *
 *   image   f[jy][jx] = sum_n D_n fhat_n exp(+2 pi i (lam_x[n] x_jx + lam_y[n] y_jy))
 *           with x_j = (j - M/2) / M on the centred pixel grid, no 1/N factor:
 *           Eq. (fstraight) of Sec. II.B with alpha_n = D_n, evaluated the NUFFT
 *           way of Eq. (Anu) (spread with a window, inverse FFT, divide by the
 *           window transform) and Algorithm 1 (per-slice correction, one 2-D IFFT).
 *   weights D_n = R_tau(diag(Psi W)^+) on the range axis (Algorithm 1; Eq. (Psi);
 *           R_tau(x) = x if x >= tau else 0 of Sec. III.B; window
 *           w(x) = exp(-a |x - 1/2|), a = 0.01, tau = 0.97 of Sec. IV).
 *   forward y_n = D_n sum_j f_j exp(-2 pi i lam_n . x_j), the adjoint of the image map.
 *
 * Coordinates lam are in grid units (cycles per image extent), so the image's
 * own Fourier grid is the integers in [-M/2, M/2).  lam_x is the range
 * (non-uniform) axis, lam_y the azimuth (uniform) axis.
 *
 * Conventions shared by every call:
 *  - Every pointer argument marked "device" must point to device memory of
 *    the current CUDA device; the caller owns it and keeps ownership.  The
 *    plan owns all of its internal device buffers and frees them in
 *    tffr_destroy.
 *  - Every call is ordered on the plan's stream.  tffr_adjoint and
 *    tffr_forward never synchronise; tffr_set_points waits for the stream
 *    before it returns (see there); tffr_weights synchronises only when
 *    n_kept is requested.
 *  - The coordinate arrays given to tffr_set_points are used in place (no
 *    copy): they must stay valid and unchanged until the next
 *    tffr_set_points or tffr_destroy on that plan.
 *  - Return value: a tffr_status.  On TFFR_ERR_CUDA the CUDA error text is
 *    available from tffr_last_error(plan).
 *  - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef TFFR_H
#define TFFR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tffr_plan_s* tffr_plan_t;

/* A cudaStream_t passed as an opaque pointer; NULL is the default stream. */
typedef void* tffr_stream_t;

typedef enum {
    TFFR_OK = 0,
    TFFR_ERR_INVALID_ARG = 1, /* bad size, option, pointer, or non-finite coordinate */
    TFFR_ERR_NOT_READY = 2,   /* adjoint/forward before set_points and weights */
    TFFR_ERR_CUDA = 3,        /* a CUDA call failed; see tffr_last_error */
    TFFR_ERR_OOM = 4,         /* device allocation failed */
    TFFR_ERR_TIMEOUT = 5      /* a bounded device wait gave up (the batch's column items wait
                                 for their patch's rows; see tffr_batch_wait) */
} tffr_status;

/* Storage type of the sample values read by tffr_adjoint (and written by
 * tffr_forward).  Arithmetic is FP32 in every case. */
typedef enum {
    TFFR_VALUES_C64 = 0,  /* complex64: float re, im (8 bytes per sample) */
    TFFR_VALUES_C128 = 1, /* complex128: double re, im (16 bytes); forward writes complex128 */
    TFFR_VALUES_F16 = 2,  /* half re, im (4 bytes); forward writes complex64 */
    TFFR_VALUES_BF16 = 3  /* bfloat16 re, im (4 bytes); forward writes complex64 */
} tffr_values;

/* How samples are organised. */
typedef enum {
    TFFR_POINTS_AUTO = 0,    /* pulse rows if runs of equal lam_y average >= 8 samples */
    TFFR_POINTS_GENERAL = 1, /* arbitrary points, bucketed by fine-grid row */
    TFFR_POINTS_ROWS = 2     /* consecutive samples with bit-equal lam_y form one pulse row */
} tffr_points_layout;

/* Order of the two FFT passes on pulse rows.  Both compute the same image
 * (the x transform is linear, so it may come before or after the azimuth
 * taps); the pulse-row order transforms P pulse rows instead of 2 My fine
 * rows and keeps a P x Mx intermediate instead of 2 My x Mx. */
typedef enum {
    TFFR_ORDER_AUTO = 0,      /* pulse rows first when there are at most My of them */
    TFFR_ORDER_FINE_ROWS = 1  /* azimuth taps first, then the x FFT of every fine row */
} tffr_pass_order;

typedef struct {
    int sigma;      /* oversampling of the FFT grid; only 2 is supported */
    int width;      /* spreading-kernel width w in fine cells: 2, 4, 6 or 8 (default 6) */
    double beta;    /* exponential-of-semicircle shape; <= 0 selects 2.30 * width */
    int values;     /* tffr_values (default TFFR_VALUES_C64) */
    int layout;     /* tffr_points_layout (default TFFR_POINTS_AUTO) */
    int order;      /* tffr_pass_order (default TFFR_ORDER_AUTO) */
} tffr_opts;

typedef enum {
    TFFR_WEIGHTS_TFFR = 0, /* D_n = R_tau(1 / G_n), G_n the diagonal of Psi W */
    TFFR_WEIGHTS_UNIT = 1, /* D_n = 1: the plain sum of Eq. (fstraight) */
    TFFR_WEIGHTS_USER = 2  /* D_n given by the caller (device float[N], no threshold) */
} tffr_weight_mode;

typedef struct {
    int mode;             /* tffr_weight_mode */
    int separable;        /* 0: range axis only (Algorithm 1); 1: D = R_tau(1 / (G(lam_x) G(lam_y))) */
    double a;             /* window decay a of w(x) = exp(-a |x - 1/2|), default 0.01 */
    double q;             /* band of W: grid points with |lam - l| < q, default 3 */
    double tau;           /* threshold of R_tau, default 0.97 */
    const float* user_D;  /* device float[N] for TFFR_WEIGHTS_USER, else ignored */
} tffr_weight_opts;

typedef struct {
    int Mx, My;                /* image size */
    int nx, ny;                /* fine (oversampled) grid size, 2 Mx by 2 My */
    int width;
    double beta;
    int64_t N;                 /* samples of the last tffr_set_points */
    int layout;                /* TFFR_POINTS_ROWS or TFFR_POINTS_GENERAL in use (0 before points) */
    int64_t n_rows;            /* pulse rows (rows layout) */
    int64_t row_cells;         /* cells of all pulse-row buffers (rows layout) */
    int max_row_cells;         /* longest pulse-row buffer */
    int64_t n_kept;            /* samples with D_n != 0 after the last tffr_weights (-1 if unknown) */
    size_t device_bytes;       /* device memory held by the plan */
    int64_t kernel_launches;   /* kernels this plan has launched since it was created */
    int pulse_order;           /* 1 when the pulse-row order of the FFT passes is in use */
} tffr_plan_info;

/* Stages of the pipeline, for tffr_profile_read. */
typedef enum {
    TFFR_STAGE_POINTS = 0,     /* tffr_set_points: coordinate reduction, rows or buckets */
    TFFR_STAGE_WEIGHTS = 1,    /* tffr_weights */
    TFFR_STAGE_SPREAD = 2,     /* adjoint: range-axis spread of pulse rows */
    TFFR_STAGE_ROW_FFT = 3,    /* adjoint: azimuth taps + FFT along x + x deapodisation */
    TFFR_STAGE_COL_FFT = 4,    /* adjoint: FFT along y + y deapodisation + image store */
    TFFR_STAGE_FWD_COL_FFT = 5,/* forward: deapodise + FFT along y */
    TFFR_STAGE_FWD_ROW_FFT = 6,/* forward: FFT along x + transposed azimuth taps */
    TFFR_STAGE_INTERP = 7,     /* forward: range-axis interpolation to the samples */
    TFFR_NUM_STAGES = 8
} tffr_stage;

/* Fill the defaults: sigma 2, width 6, beta 2.30 * width, complex64 values, auto layout. */
void tffr_default_opts(tffr_opts* opts);

/* Fill the defaults: tFFR mode, range axis, a = 0.01, q = 3, tau = 0.97 (Sec. IV). */
void tffr_default_weight_opts(tffr_weight_opts* opts);

/*
 * Create a plan for an My x Mx image (Mx, My powers of two, 16 <= M <= 4096).
 * Precomputes in FP64 on the host the FFT twiddles and the deapodisation
 * factors 1 / phi_hat(k / 2M) of the spreading kernel, uploads them, and
 * allocates the Mx x 2My intermediate of the two FFT passes.
 * opts may be NULL (defaults).  stream: the stream every later call uses.
 * Errors: INVALID_ARG for out-of-range sizes or options; OOM; CUDA.
 */
int tffr_plan(tffr_plan_t* out, int Mx, int My, const tffr_opts* opts, tffr_stream_t stream);

/*
 * Set the N sample frequencies (device double[N] each, grid units; Sec. II.A:
 * lam_x range, lam_y azimuth).  The arrays are kept by pointer (see above).
 * Finds the pulse rows (runs of bit-equal lam_y; layout ROWS) or buckets the
 * samples by fine-grid row (layout GENERAL) and sizes the per-row buffers.
 * Every later call reduces a coordinate exactly from its FP64 bits to a fine
 * cell floor(2 lam) and an FP32 offset (at 8192 cells an FP32 coordinate
 * would keep only ~1e-3 cell).
 * N = 0 is allowed (adjoint then returns a zero image).  Invalidates the weights.
 * Errors: INVALID_ARG for N < 0, N >= 2^31, NULL pointers with N > 0, or any
 * |lam| >= 2^28 or non-finite coordinate; OOM; CUDA.  Waits until the stream
 * has finished everything issued before the call and the pass over the
 * coordinates; in layout ROWS the plan's fine-row tap table may still be
 * filled on the stream after the return (that fill reads no caller memory).
 */
int tffr_set_points(tffr_plan_t plan, int64_t N, const double* lam_x, const double* lam_y);

/*
 * Set the frame weights D_n (Algorithm 1: W, Psi and D = R_tau((W Psi)^+),
 * diagonal only).  The plan fits the diagonal G(delta) of the fractional
 * offset once in FP64 and the kernels evaluate D_n inline (FP32 polynomial,
 * with the closed form in FP64 deciding every sample near tau, near the grid
 * edge or on a truncation breakpoint), so the threshold decision is an FP64
 * one.  opts may be NULL (defaults).  USER weights are copied.  D_out
 * (nullable, device float[N]) receives D; n_kept (nullable, host) receives the
 * count of D_n != 0; either makes the call evaluate D for every sample, and
 * n_kept makes it synchronise.
 * Errors: NOT_READY before tffr_set_points; INVALID_ARG for bad options
 * (q <= 0, a < 0, unknown mode, USER mode without user_D); CUDA.
 */
int tffr_weights(tffr_plan_t plan, const tffr_weight_opts* opts, float* D_out, int64_t* n_kept);

/*
 * The tFFR image (the hot path).  values: device, N samples in the plan's
 * value type, in the order given to tffr_set_points.  image: device complex64
 * [My][Mx], row-major, x fastest, fully overwritten.
 * Errors: NOT_READY before tffr_set_points + tffr_weights; INVALID_ARG for
 * NULL pointers; CUDA.
 */
int tffr_adjoint(tffr_plan_t plan, const void* values, void* image);

/*
 * One whole reconstruction (Sec. II.B Eq. (fstraight) with the weights of
 * Algorithm 1): tffr_set_points(plan, N, lam_x, lam_y), tffr_weights(plan,
 * opts, NULL, NULL) and tffr_adjoint(plan, values, image) in one call, with
 * the same arguments, ownership and results as those three.  The adjoint's
 * first launch follows set_points' read-back with no return to the caller in
 * between, so the device does not wait on the caller's own work there.
 * Errors: those of the three calls, from the first that fails (the later ones
 * are then not made).
 */
int tffr_reconstruct(tffr_plan_t plan, int64_t N, const double* lam_x, const double* lam_y,
                     const tffr_weight_opts* opts, const void* values, void* image);

/*
 * The forward twin: values[n] = (apply_weights ? D_n : 1) * sum_j image_j
 * exp(-2 pi i lam_n . x_j).  image: device complex64 [My][Mx].  values:
 * device, N samples (complex128 for the C128 value type, complex64 otherwise).
 * Errors: as tffr_adjoint.
 */
int tffr_forward(tffr_plan_t plan, const void* image, void* values, int apply_weights);

/*
 * The unweighted adjoint f = E^H y (Eq. (fstraight) with alpha_n = 1), the
 * Hermitian transpose of tffr_forward with apply_weights = 0; it serves as that
 * map's backward pass.  Arguments, ordering and errors as tffr_adjoint.
 */
int tffr_adjoint_unweighted(tffr_plan_t plan, const void* values, void* image);

/*
 * Gradient of a real loss L with respect to real frame weights D (the
 * backward of tffr_adjoint in the D argument): for f = E^H D y and
 * grad_image = dL/d conj(f),
 *     grad_D[n] = Re( conj((E grad_image)_n) * y_n ),
 * the unweighted forward twin of grad_image times the samples, fused into the
 * forward's last pass.  grad_image: device complex64 [My][Mx]; values: device,
 * N samples y_n in the plan's value type; grad_D: device float[N], fully
 * overwritten.  Ordered on the plan's stream, no synchronisation.
 * Errors: as tffr_forward.
 */
int tffr_weight_grad(tffr_plan_t plan, const void* grad_image, const void* values, float* grad_D);

/*
 * Conjugate gradients on the weighted normal equations E^H D E f = E^H D y,
 * started from f = 0: the least-squares image refining the one-step tFFR
 * image E^H D y (which is the first CG direction).  E^H D E is applied by the
 * Toeplitz operator when use_toeplitz != 0 (after tffr_normal_setup), else as
 * the unweighted forward twin followed by the weighted adjoint.  Exactly
 * iters iterations run; every vector update and reduction is a kernel on the
 * plan's stream (step sizes are device scalars), so nothing synchronises
 * unless residuals is given.  values: device, N samples in the plan's value
 * type.  image: device complex64 [My][Mx], receives f.  residuals (nullable,
 * host double[iters + 1]): ||b - E^H D E f_k|| by the CG recurrence, k =
 * 0..iters; asking for them synchronises the stream.  The plan keeps three
 * My x Mx work images (and N samples without the Toeplitz operator),
 * allocated on first use.
 * Errors: NOT_READY before points and weights, or use_toeplitz before
 * tffr_normal_setup; INVALID_ARG for NULL pointers or iters outside
 * [0, 100000]; OOM; CUDA.
 */
int tffr_cg(tffr_plan_t plan, const void* values, void* image, int iters, int use_toeplitz, double* residuals);

/*
 * Batches of independent reconstructions (sub-aperture patches of uneven
 * size; the per-slice structure of Algorithm 1 repeated over patches).  A
 * batch takes plans that each have points and weights set (pulse-row layout,
 * complex64 values, square images of side 256, 512 or 1024, one spreading
 * width and one set of weight options for all) and fixed device buffers for
 * each plan's samples and image.  Its adjoint is one spread launch over every
 * pulse row of every patch (the row buffers), then one persistent FFT launch
 * per image side whose blocks claim work items from a device counter: one
 * item per pulse row of the patches in the pulse-row order of the passes (x
 * FFT), one per fine row of the others (more pulse rows than image rows:
 * azimuth taps and x FFT), then one per image column (azimuth taps or the
 * fine rows' column, y FFT, deapodisation, image store).  A column item waits
 * for its patch's rows; the wait is bounded (1 s of device time by default)
 * and a wait that runs out makes every later wait give up, so the launch
 * always ends; tffr_batch_wait then returns TFFR_ERR_TIMEOUT.
 */
typedef struct tffr_batch_s* tffr_batch_t;

#define TFFR_BATCH_MAX_CLASSES 8
typedef struct {
    int n_patches;
    int n_classes;                              /* persistent FFT launches per adjoint: one per image side */
    int64_t samples;                            /* samples of all patches */
    int tuned;                                  /* 1 after tffr_batch_tune */
    int width;                                  /* spreading width of every patch */
    float spread_ms;                            /* the tuner's time of the spread launch (0 untuned) */
    int class_side[TFFR_BATCH_MAX_CLASSES];     /* image side of each class */
    int class_patches[TFFR_BATCH_MAX_CLASSES];  /* patches in the class */
    int class_blocks[TFFR_BATCH_MAX_CLASSES];   /* blocks of the class's persistent launch */
    float class_ms[TFFR_BATCH_MAX_CLASSES];     /* the tuner's best time of the class's launch (0 untuned) */
} tffr_batch_info;

/*
 * Create a batch of n plans.  values[i] (device complex64, plan i's N samples)
 * and images[i] (device complex64 [M][M]) stay the batch's buffers: load new
 * samples into them between adjoints.  The batch keeps pointers into the plans
 * and uses their row buffers and intermediates: recreate it after
 * tffr_set_points or tffr_weights on any of them, and do not run the plans'
 * own adjoints concurrently with it.  stream: the stream tffr_batch_adjoint is
 * ordered on.  Allocates and synchronises (the plans' streams and this one:
 * the batch reads the plans' pulse rows once, into one record per row).
 * Errors: INVALID_ARG (NULL pointers, n < 1, a plan outside the supported
 * layout, value type or sides, or plans with different widths, kernel shapes
 * or weight options); NOT_READY (a plan without points or weights); OOM; CUDA.
 */
int tffr_batch_create(const tffr_plan_t* plans, int n, const void* const* values, void* const* images,
                      tffr_stream_t stream, tffr_batch_t* out);

/* Every patch's adjoint (its plan's weights, Eq. (fstraight) with alpha_n = D_n)
 * into its image.  Ordered on the batch's stream; allocates nothing and does
 * not synchronise, so it can be captured into a CUDA graph.  Errors: CUDA. */
int tffr_batch_adjoint(tffr_batch_t batch);

/* Synchronise the batch's stream and report (and clear) a timed-out wait of an
 * earlier adjoint: TFFR_ERR_TIMEOUT, else TFFR_OK.  Errors: CUDA. */
int tffr_batch_wait(tffr_batch_t batch);

/* Autotuner: for each class, time reps launches of the persistent FFT kernel
 * with every candidate grid (blocks per SM 1, 2, 4, ... up to what fits) and
 * keep the fastest; tffr_batch_get_info reports the choice.  Runs the spread
 * once first; synchronises.  Errors: INVALID_ARG (reps outside [1, 1000]);
 * CUDA; TIMEOUT. */
int tffr_batch_tune(tffr_batch_t batch, int reps);

/* Limit of one wait of a column item for its patch's rows, in seconds of device
 * time (0 < wait_s <= 60; default 1).  hold_rows != 0 makes row items skip
 * publishing their completion, so that every wait runs out: a test of the
 * timeout path that faults and hangs nothing.  Errors: INVALID_ARG. */
int tffr_batch_set_wait(tffr_batch_t batch, double wait_s, int hold_rows);

int tffr_batch_get_info(tffr_batch_t batch, tffr_batch_info* info);

/* Free the batch (after synchronising its streams); the plans stay. NULL is a no-op. */
int tffr_batch_destroy(tffr_batch_t batch);

/*
 * Per-stage timing with CUDA events recorded on the plan's stream around each
 * stage's kernels.  enable != 0 starts (and resets) recording, 0 stops it.
 * Recording costs two event records per stage launch.
 */
int tffr_profile(tffr_plan_t plan, int enable);

/*
 * Synchronise the plan's stream and return, per stage (arrays of length
 * nstages <= TFFR_NUM_STAGES), the summed event time in milliseconds and the
 * number of timed executions since the last tffr_profile(plan, 1).
 * At most 4096 executions per stage are kept; later ones are not timed.
 */
int tffr_profile_read(tffr_plan_t plan, double* ms, int64_t* count, int nstages);

/*
 * Frame weights without a plan and without allocating device memory, for
 * callers that cannot call cudaMalloc at the point where they need weights
 * (for example code that runs while a stream is being captured into a CUDA
 * graph, or under a device-memory budget fixed before it starts).  The paper
 * has no counterpart of this entry point; it is a packaging of the weights
 * step.  D_out (device float[N]) receives the same D_n that tffr_weights
 * computes (FP32 rounding aside: here every sample takes the FP64 closed
 * form, so it is slower); n_kept (nullable, host) receives the count of
 * D_n != 0 and makes the call synchronise the stream.  lam_x / lam_y: device
 * double[N] (lam_y is read only in separable mode); Mx, My: the image sizes
 * whose Fourier grids truncate the sums.
 * Scratch: a fixed array in device memory inside the library (about 132 KB per
 * GPU that loads it, kept until the process exits), so N is limited to
 * 67,108,864 samples; larger N returns INVALID_ARG.  The first call on a
 * device looks the array up (cudaGetSymbolAddress): make that first call
 * before any stream capture.  Every call shares the array, so calls that
 * overlap on the GPU (several streams, several host threads) race: serialise
 * them.
 * In USER mode D_out must not overlap user_D: the kernel reads one while it
 * writes the other, so an overlap returns INVALID_ARG (copy the weights first).
 * n_kept reads the count back with a pageable copy and a stream
 * synchronisation, neither of which may run while the stream is captured:
 * pass n_kept = NULL there.
 * Errors: INVALID_ARG for bad sizes, options, NULL pointers or D_out
 * overlapping user_D; CUDA.
 */
int tffr_weights_noalloc(int64_t N, const double* lam_x, const double* lam_y, int Mx, int My,
                         const tffr_weight_opts* opts, float* D_out, int64_t* n_kept, tffr_stream_t stream);

/*
 * Normal operator of the weighted least-squares image, N = E^H D E, where
 * E[n, j] = exp(-2 pi i lam_n . x_j) and D the plan's weights: tffr_adjoint
 * computes the one-step tFFR image E^H D y (Eq. (fstraight) with alpha_n = D_n),
 * and iterating with N (conjugate gradients on N f = E^H D y) refines it.  N is
 * the convolution of the image with k(m) = sum_n D_n exp(2 pi i lam_n . m / M)
 * (Toeplitz), applied as crop(IFFT2(Khat . FFT2(zero-padded f))) on the
 * 2 My x 2 Mx grid: three passes of line FFTs, independent of N.
 *
 * tffr_normal_setup builds Khat (4 Mx My complex64, owned by the plan) for
 * the current points and weights, through a temporary plan of sides 2 Mx,
 * 2 My (so Mx, My <= 2048); it allocates, synchronises the stream, and must
 * be called again after tffr_set_points or tffr_weights.
 * Errors: NOT_READY before points and weights; INVALID_ARG for Mx or My > 2048;
 * OOM; CUDA.
 */
int tffr_normal_setup(tffr_plan_t plan);

/*
 * image_out = N image_in, both device complex64 [My][Mx], row-major; they may
 * be the same array.  Ordered on the plan's stream, no synchronisation.
 * Errors: NOT_READY before tffr_normal_setup; INVALID_ARG for NULL pointers; CUDA.
 */
int tffr_normal_apply(tffr_plan_t plan, const void* image_in, void* image_out);

/* Query sizes and the state of a plan. */
int tffr_plan_get_info(tffr_plan_t plan, tffr_plan_info* info);

/* Free the plan and every device buffer it owns (after synchronising its stream). NULL is a no-op. */
int tffr_destroy(tffr_plan_t plan);

/* Static text for a status code. */
const char* tffr_error_string(int status);

/* Text of the last error on this plan ("" if none).  Valid until the next call on the plan. */
const char* tffr_last_error(tffr_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* TFFR_H */
