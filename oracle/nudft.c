/*
 * FP64 direct non-uniform DFT: the CPU oracle for the tFFR image.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; it is built by oracle/build.py and used by tests/, the smoke check
 * and the CPU-baseline leg of the benchmark.
 *
 * Definition followed (Section II.B, Eq. (fstraight), with alpha_n := D_n,
 * the tFFR weights of Section III.B):
 *
 *     f(x_jx, y_jy) = sum_n D_n * fhat_n * exp(+2 pi i (lam_x[n] x_jx + lam_y[n] y_jy))
 *
 * on the centred pixel grid x_j = (j - M/2) / M, j = 0..M-1 (image on
 * [-1/2, 1/2)), no 1/N factor.  The forward twin is the plain adjoint of that
 * sum:  y_n = D_n * sum_j f_j exp(-2 pi i lam_n . x_j).
 *
 * Every term is evaluated on its own: phase in FP64, reduced modulo one cycle
 * (exact: the subtraction of floor), then cos/sin of 2 pi times the fraction.
 * No recurrences, no blocking, no FFT.  Parallel over output entries with
 * OpenMP; each output is one plain sequential sum.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

static inline void cis_cycles(double theta, double *c, double *s)
{
    double fr = theta - floor(theta);      /* exact reduction to [0, 1) */
    *c = cos(TWO_PI * fr);
    *s = sin(TWO_PI * fr);
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Image pixels (jx[k], jy[k]) for k < npix.
 * y: interleaved complex128 [N]; D: [N] or NULL (all ones);
 * out: interleaved complex128 [npix].
 */
void oracle_adjoint_pixels(int64_t N, const double *lam_x, const double *lam_y,
                           const double *y, const double *D, int Mx, int My,
                           int64_t npix, const int32_t *jx, const int32_t *jy,
                           double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < npix; ++k) {
        const double x = ((double)jx[k] - (double)(Mx / 2)) / (double)Mx;
        const double yy = ((double)jy[k] - (double)(My / 2)) / (double)My;
        double acc_re = 0.0, acc_im = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            const double d = D ? D[n] : 1.0;
            if (d == 0.0) continue;
            double c, s;
            cis_cycles(lam_x[n] * x + lam_y[n] * yy, &c, &s);
            const double vr = d * y[2 * n], vi = d * y[2 * n + 1];
            acc_re += vr * c - vi * s;
            acc_im += vr * s + vi * c;
        }
        out[2 * k] = acc_re;
        out[2 * k + 1] = acc_im;
    }
}

/*
 * Forward twin at samples idx[k] (k < nidx), or at all N samples if idx is NULL
 * (then nidx must equal N).  img: interleaved complex128 [My][Mx] row-major,
 * x fastest.  D: [N] or NULL.  out: interleaved complex128 [nidx].
 */
void oracle_forward_samples(int64_t N, const double *lam_x, const double *lam_y,
                            const double *img, const double *D, int Mx, int My,
                            int64_t nidx, const int64_t *idx, double *out,
                            int nthreads)
{
    (void)N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < nidx; ++k) {
        const int64_t n = idx ? idx[k] : k;
        const double d = D ? D[n] : 1.0;
        double acc_re = 0.0, acc_im = 0.0;
        if (d != 0.0) {
            for (int jy = 0; jy < My; ++jy) {
                const double yy = ((double)jy - (double)(My / 2)) / (double)My;
                for (int jx = 0; jx < Mx; ++jx) {
                    const double x = ((double)jx - (double)(Mx / 2)) / (double)Mx;
                    double c, s;
                    cis_cycles(lam_x[n] * x + lam_y[n] * yy, &c, &s);
                    /* multiply by exp(-i theta) = c - i s */
                    const double fr = img[2 * ((int64_t)jy * Mx + jx)];
                    const double fi = img[2 * ((int64_t)jy * Mx + jx) + 1];
                    acc_re += fr * c + fi * s;
                    acc_im += fi * c - fr * s;
                }
            }
        }
        out[2 * k] = d * acc_re;
        out[2 * k + 1] = d * acc_im;
    }
}
