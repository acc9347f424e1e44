/*
 * FP64 CPU oracle for the hop-size continuous wavelet transform (CWTH).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it computes (paper Sec. II.A, Eq. 1, discretised with dt = 1 sample;
 * Sec. II.B for the hop):
 *
 *     W_s[k] = a_s^{-1/2} * sum_n x[n] * conj( psi( (n - k*H) / a_s ) ),
 *     k = 0 .. ceil(N/H) - 1,   x[n] = 0 outside [0, N),
 *
 * with the complex Morlet wavelet in the "cmor B-C" convention
 *
 *     psi(t) = (pi*B)^{-1/2} * exp(-t^2 / B) * exp(i*2*pi*C*t).
 *
 * The sum is truncated to |n - kH| <= h_s, h_s = ceil(a_s * sqrt(B*ln(1/eps))),
 * beyond which every tap is below eps relative to the wavelet peak; with
 * truncate = 0 the sum runs over every n in [0, N) (brute force). Terms are
 * accumulated in ascending n, one rounding per multiply and per add
 * (compile with -ffp-contract=off), so a frame's value does not depend on
 * the hop or on which other frames are requested.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* Half-support of the truncated wavelet at scale a (in samples). */
int64_t oracle_half_support(double a, double bandwidth, double eps)
{
    return (int64_t)ceil(a * sqrt(bandwidth * log(1.0 / eps)));
}

int64_t oracle_num_frames(int64_t n, int32_t hop)
{
    if (n <= 0 || hop <= 0)
        return 0;
    return (n + hop - 1) / hop;
}

/*
 * x        : [n] real samples (float64)
 * scales   : [S] scales a_s in samples
 * out_re/im: [S][F] complex coefficients, F = ceil(n / hop)
 * out_mag  : [S][F] |W| (may be NULL)
 * threads  : OpenMP threads (<= 0: library default)
 * returns 0 on success, a negative value on a bad argument or no memory.
 */
int oracle_cwth(const double *x, int64_t n, double bandwidth, double center,
                const double *scales, int32_t S, int32_t hop, double eps,
                int32_t truncate, int32_t threads,
                double *out_re, double *out_im, double *out_mag)
{
    if (!x || !scales || !out_re || !out_im || n <= 0 || S <= 0 || hop <= 0)
        return -1;
    if (!(bandwidth > 0) || !(center > 0) || !(eps > 0 && eps < 1))
        return -1;
    for (int32_t s = 0; s < S; ++s)
        if (!(scales[s] > 0) || !isfinite(scales[s]))
            return -1;

    const int64_t F = oracle_num_frames(n, hop);
    int rc = 0;

    /* Threads of this call only (the process-wide OpenMP default is left as is). */
#ifdef _OPENMP
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif

    for (int32_t s = 0; s < S && rc == 0; ++s) {
        const double a = scales[s];
        int64_t h = truncate ? oracle_half_support(a, bandwidth, eps) : n - 1;
        if (h > n - 1)
            h = n - 1;
        /* Taps g[t] = a^{-1/2} conj(psi(t/a)), t = -h .. h, stored at g[t + h]. */
        double *gre = (double *)malloc(sizeof(double) * (size_t)(2 * h + 1));
        double *gim = (double *)malloc(sizeof(double) * (size_t)(2 * h + 1));
        if (!gre || !gim) {
            free(gre);
            free(gim);
            rc = -2;
            break;
        }
        const double norm = 1.0 / sqrt(a) / sqrt(ORACLE_PI * bandwidth);
        for (int64_t t = -h; t <= h; ++t) {
            const double u = (double)t / a;
            const double env = norm * exp(-(u * u) / bandwidth);
            const double ph = 2.0 * ORACLE_PI * center * u;
            gre[t + h] = env * cos(ph);
            gim[t + h] = -env * sin(ph); /* conjugate */
        }

#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
        for (int64_t k = 0; k < F; ++k) {
            const int64_t b = k * (int64_t)hop;
            int64_t t0 = -h, t1 = h;
            if (b + t0 < 0)
                t0 = -b;
            if (b + t1 > n - 1)
                t1 = n - 1 - b;
            double re = 0.0, im = 0.0;
            for (int64_t t = t0; t <= t1; ++t) {
                const double xv = x[b + t];
                re += xv * gre[t + h];
                im += xv * gim[t + h];
            }
            out_re[(int64_t)s * F + k] = re;
            out_im[(int64_t)s * F + k] = im;
            if (out_mag)
                out_mag[(int64_t)s * F + k] = sqrt(re * re + im * im);
        }
        free(gre);
        free(gim);
    }
    return rc;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
