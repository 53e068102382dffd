/*
 * FP64 reference Range-Doppler compressor -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the oracle that the CUDA path is checked against.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg load it;
 * the product library never links, loads or calls it, and it shares no code,
 * header, table or constant with the CUDA sources.
 *
 * It is deliberately plain and slow: every step is written out as the
 * paper states it, in double precision, with no blocking, fusion or
 * reordering beyond that statement, so that it can be checked by eye.
 *
 *   Range compression (Sec. IV-A, step 1; Sec. II-B):
 *       per azimuth line x:  y = IFFT( FFT(x) . H_r )
 *   Corner turn (Sec. IV-A step 2 / Sec. IV-B: the transpose that turns the
 *       azimuth columns into rows):  out[c][r] = in[r][c]
 *   Azimuth compression (Sec. IV-A, step 4, in the form used here: a full
 *       FFT -> x H_a -> IFFT per range bin after the corner turn).
 *   IFFT (Sec. II-C):  IFFT(X) = (1/N) * sum_k X[k] exp(+2 pi i n k / N);
 *       the paper computes it as conj(FFT(conj X))/N, which is the same value.
 *   Matched filter (Sec. II-B, "pre-computed matched filter"): the reference
 *       chirp c, centred on time index 0 with circular wrap, gives
 *       H = conj(FFT_N(c)), unnormalised.  Correlating with it puts the
 *       compressed peak of a target exactly at the target's position.
 *
 * The FFT is a textbook iterative radix-2 decimation-in-time transform.  Each
 * twiddle factor exp(sign * 2 pi i j / len) is evaluated directly with cos()
 * and sin() for its own index j -- never by a recurrence -- so its error does
 * not grow with the transform length.  A length that is not a power of two
 * takes the O(n^2) sum of the DFT's definition instead, with the twiddle of
 * exponent j*k read from a table of the n roots (entry (j*k) mod n, each
 * evaluated by cos() and sin() of its own index); every function built on the
 * transform (matched filter, line and scene compression) then holds for any
 * length as the same definitions at that length.
 *
 * Data layout: complex numbers are pairs of doubles (re, im), i.e. the
 * memory layout of C99 double complex and of numpy.complex128.  Matrices are
 * row-major.  All entry points return 0 on success and a negative value on a
 * bad argument; none of them allocates memory visible to the caller.
 *
 * Planted mistakes: when compiled with -DORACLE_PLANT=<k> (k >= 1) one
 * deliberate error is introduced (see the ORACLE_PLANT blocks).  The test
 * suite builds each variant in a temporary directory and checks that its
 * pins fail; the default build has ORACLE_PLANT = 0 and no planted error.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

typedef double complex cplx;

static const double kTwoPi = 6.283185307179586476925286766559;
static const double kPi = 3.141592653589793238462643383279;

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transform (definition:  X[k] = sum_n x[n] e^{sign 2 pi i n k / N}). */
/* ------------------------------------------------------------------------ */

/* The DFT of any length n >= 1 by its definition, in place:
 * X[k] = sum_j x[j] w[(j k) mod n], w[m] = e^{sign 2 pi i m / n}. */
static int oracle_dft(int64_t n, cplx *x, int sign)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *y = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!w || !y) {
        free(w);
        free(y);
        return -1;
    }
    for (int64_t m = 0; m < n; ++m) {
        double ang = (double)sign * kTwoPi * (double)m / (double)n;
        w[m] = cos(ang) + I * sin(ang);
    }
    for (int64_t k = 0; k < n; ++k) {
        cplx acc = 0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t e = (j * k) % n;
#if ORACLE_PLANT == 9
            e = (j * k) & (n - 1); /* planted: exponent reduced as if n were a power of two */
#endif
            acc += x[j] * w[e];
        }
        y[k] = acc;
    }
    memcpy(x, y, sizeof(cplx) * (size_t)n);
    free(w);
    free(y);
    return 0;
}

/* In-place unnormalised DFT of length n: the radix-2 FFT when n is a power
 * of two, the definition's O(n^2) sum otherwise.
 * sign = -1: forward transform; sign = +1: inverse kernel (no 1/N). */
int oracle_fft(int64_t n, cplx *x, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1) || !x)
        return -1;
    if (!is_pow2(n))
        return oracle_dft(n, x, sign);
#if ORACLE_PLANT == 1
    sign = -sign; /* planted: wrong exponent sign */
#endif
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1)
            j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    /* butterflies, span len = 2, 4, ..., n */
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        for (int64_t j = 0; j < half; ++j) {
            double ang = (double)sign * kTwoPi * (double)j / (double)len;
            cplx w = cos(ang) + I * sin(ang);
#if ORACLE_PLANT == 2
            if (j == 1) w = conj(w); /* planted: one wrong twiddle */
#endif
            for (int64_t i = 0; i < n; i += len) {
                cplx u = x[i + j];
                cplx v = x[i + j + half] * w;
                x[i + j] = u + v;
                x[i + j + half] = u - v;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Matched filter (Sec. II-B step 3, Sec. IV-A steps 1 and 4).               */
/* ------------------------------------------------------------------------ */

/* H[k] = conj( sum_m c(m) e^{-2 pi i m k / n} ) where the reference chirp
 * sample chirp[j] belongs to time index m = j - n_chirp/2 (the chirp is
 * centred on index 0) and sits at position m mod n of a length-n line. */
int oracle_matched_filter(int64_t n, int64_t n_chirp, const cplx *chirp, cplx *H)
{
    if (n < 1 || n_chirp < 1 || n_chirp > n || !chirp || !H)
        return -1;
    memset(H, 0, sizeof(cplx) * (size_t)n);
    for (int64_t j = 0; j < n_chirp; ++j) {
        int64_t m = j - n_chirp / 2;
#if ORACLE_PLANT == 3
        m = j; /* planted: chirp not centred on index 0 */
#endif
        int64_t pos = ((m % n) + n) % n;
        H[pos] += chirp[j];
    }
    if (oracle_fft(n, H, -1))
        return -1;
    for (int64_t k = 0; k < n; ++k) {
#if ORACLE_PLANT == 4
        continue; /* planted: filter not conjugated */
#endif
        H[k] = conj(H[k]);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fused line compression: y = IFFT(FFT(x) . H), Sec. II-B steps 1-5.        */
/* ------------------------------------------------------------------------ */

/* One line of length n, in place. */
int oracle_compress_line(int64_t n, cplx *x, const cplx *H)
{
    if (n < 1 || !x || !H)
        return -1;
    if (oracle_fft(n, x, -1))
        return -1;
    for (int64_t k = 0; k < n; ++k)
        x[k] *= H[k];
    if (oracle_fft(n, x, +1))
        return -1;
    double inv_n = 1.0 / (double)n;
#if ORACLE_PLANT == 5
    inv_n = 1.0; /* planted: 1/N of the IFFT dropped */
#endif
    for (int64_t k = 0; k < n; ++k)
        x[k] *= inv_n;
    return 0;
}

typedef struct {
    int64_t n_lines, n;
    cplx *data;
    const cplx *H;
    int tid, nthreads, status;
} line_job;

static void *line_worker(void *arg)
{
    line_job *job = (line_job *)arg;
    for (int64_t l = job->tid; l < job->n_lines; l += job->nthreads)
        if (oracle_compress_line(job->n, job->data + l * job->n, job->H))
            job->status = -1;
    return NULL;
}

/* Every one of n_lines contiguous lines of length n, in place.  Line l is
 * handled by worker (l mod nthreads); each line's result is independent of
 * the thread count. */
int oracle_compress_lines(int64_t n_lines, int64_t n, cplx *data, const cplx *H, int nthreads)
{
    if (n_lines < 0 || n < 1 || (n_lines > 0 && !data) || !H)
        return -1;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    if ((int64_t)nthreads > n_lines)
        nthreads = n_lines > 0 ? (int)n_lines : 1;
    line_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (line_job){n_lines, n, data, H, t, nthreads, 0};
    }
    int spawned = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, line_worker, &jobs[t]) != 0)
            break;
        spawned = t;
    }
    /* whatever could not be spawned runs here */
    for (int t = spawned + 1; t < nthreads; ++t)
        line_worker(&jobs[t]);
    line_worker(&jobs[0]);
    for (int t = 1; t <= spawned; ++t)
        pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status)
            return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Corner turn (Sec. IV-A step 2, Sec. IV-B):  out[c][r] = in[r][c].          */
/* ------------------------------------------------------------------------ */

int oracle_corner_turn(int64_t rows, int64_t cols, const cplx *in, cplx *out)
{
    if (rows < 0 || cols < 0 || ((rows * cols) > 0 && (!in || !out)))
        return -1;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
#if ORACLE_PLANT == 6
            if (r == 1 && c == 0) { out[c * rows + r] = in[0]; continue; } /* planted: wrong index */
#endif
            out[c * rows + r] = in[r * cols + c];
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Range-Doppler compression of one scene (Sec. IV-A steps 1, 2, 4).         */
/* ------------------------------------------------------------------------ */

/* raw:   n_az x n_range echo (azimuth-major rows), read only.
 * Hr:    range filter spectrum, n_range values.
 * Ha:    azimuth filter spectrum, l_az values.
 * image: n_range x n_az output (range-bin-major rows).
 * l_az:  azimuth transform length (>= n_az).  When n_az is
 *        smaller the azimuth lines are zero-padded to l_az before the FFT and
 *        cropped back to n_az after the IFFT (circular correlation at length
 *        l_az).  With l_az == n_az this is the plain three-step algorithm. */
int oracle_rda(int64_t n_az, int64_t n_range, int64_t l_az, const cplx *raw, const cplx *Hr,
               const cplx *Ha, cplx *image, int nthreads)
{
    if (n_az < 1 || n_range < 1 || l_az < n_az || !raw || !Hr || !Ha || !image)
        return -1;
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)(n_az * n_range));
    cplx *az = (cplx *)calloc((size_t)(n_range * l_az), sizeof(cplx));
    if (!work || !az) {
        free(work);
        free(az);
        return -1;
    }
    int st = 0;
    /* 1. range compression of every azimuth line */
    memcpy(work, raw, sizeof(cplx) * (size_t)(n_az * n_range));
    st |= oracle_compress_lines(n_az, n_range, work, Hr, nthreads);
    /* 2. corner turn into zero-padded azimuth lines */
    for (int64_t a = 0; a < n_az; ++a)
        for (int64_t r = 0; r < n_range; ++r)
            az[r * l_az + a] = work[a * n_range + r];
    /* 3. azimuth compression of every range bin */
    st |= oracle_compress_lines(n_range, l_az, az, Ha, nthreads);
    /* 4. crop */
    for (int64_t r = 0; r < n_range; ++r)
        memcpy(image + r * n_az, az + r * l_az, sizeof(cplx) * (size_t)n_az);
    free(work);
    free(az);
    return st ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Full Range-Doppler processing with range cell migration correction        */
/* (Sec. IV-A steps 2-4: azimuth FFT, RCMC by sinc interpolation, azimuth    */
/* compression with the range-dependent filter H_a(f_a, R0), azimuth IFFT).  */
/* ------------------------------------------------------------------------ */

/* Azimuth frequency of spectrum index j of an n-point FFT, cycles per line. */
static double az_freq(int64_t j, int64_t n) { return (j < n / 2 ? (double)j : (double)(j - n)) / (double)n; }

/* Range-Doppler migration factor D(f) = sqrt(1 - (f / (kappa v_s))^2): in the
 * range-Doppler domain a target of closest range r0 sits at range r0 / D(f). */
static double migration_d(double f, double kappa, double vs)
{
    double q = f / (kappa * vs);
    return sqrt(1.0 - q * q);
}

/* Interpolation kernel of the RCMC: a sinc of `taps` samples (taps even)
 * under a Hann window, h(x) = sinc(x) * 0.5 (1 + cos(2 pi x / taps)) for
 * |x| < taps / 2, else 0; sinc(x) = sin(pi x) / (pi x). */
static double rcmc_kernel(double x, int taps)
{
    if (fabs(x) >= taps / 2.0)
        return 0.0;
    double s = (x == 0.0) ? 1.0 : sin(kPi * x) / (kPi * x);
    return s * 0.5 * (1.0 + cos(kTwoPi * x / (double)taps));
}

/* RCMC on the range-Doppler data rd[n_range][n_f] (row: range bin, column:
 * azimuth frequency index).  Output bin n at frequency f reads the input at
 * the migrated range n + (r_near + n)(1/D(f) - 1), interpolated with
 * rcmc_kernel over the taps nearest to it; samples outside the range extent
 * count as zero.  taps = 0 copies the data (no correction). */
int oracle_rcmc(int64_t n_range, int64_t n_f, const cplx *rd, cplx *out, double kappa, double vs, double r_near,
                int taps)
{
    if (n_range < 1 || n_f < 1 || !rd || !out || taps < 0 || (taps & 1))
        return -1;
    for (int64_t j = 0; j < n_f; ++j) {
        double d = migration_d(az_freq(j, n_f), kappa, vs);
        for (int64_t n = 0; n < n_range; ++n) {
            if (taps == 0) {
                out[n * n_f + j] = rd[n * n_f + j];
                continue;
            }
            double src = (double)n + (r_near + (double)n) * (1.0 / d - 1.0);
            int64_t k0 = (int64_t)floor(src);
            cplx acc = 0.0;
            for (int64_t k = k0 - taps / 2 + 1; k <= k0 + taps / 2; ++k) {
                if (k < 0 || k >= n_range)
                    continue;
                acc += rcmc_kernel(src - (double)k, taps) * rd[k * n_f + j];
            }
#if ORACLE_PLANT == 7
            acc = rd[n * n_f + j]; /* planted: no correction */
#endif
            out[n * n_f + j] = acc;
        }
    }
    return 0;
}

/* The whole processor: raw[n_az][n_range] -> image[n_range][n_az].
 * 1. range compression with Hr (per azimuth line, as oracle_rda);
 * 2. corner turn; 3. azimuth FFT per range bin;
 * 4. RCMC (oracle_rcmc);
 * 5. azimuth compression: multiply by H_a(f, r) = exp(+2 pi i kappa r D(f)),
 *    r = r_near + n, which cancels the target phase exp(-2 pi i kappa r0 D(f))
 *    of the stationary-phase spectrum, and the azimuth IFFT (1/n_az).
 * n_range, n_az powers of two. */
int oracle_rda_full(int64_t n_az, int64_t n_range, const cplx *raw, const cplx *Hr, double kappa, double vs,
                    double r_near, int taps, cplx *image, int nthreads)
{
    if (!is_pow2(n_az) || !is_pow2(n_range) || !raw || !Hr || !image)
        return -1;
    size_t total = (size_t)(n_az * n_range);
    cplx *work = (cplx *)malloc(sizeof(cplx) * total);
    cplx *rd = (cplx *)malloc(sizeof(cplx) * total);
    if (!work || !rd) {
        free(work);
        free(rd);
        return -1;
    }
    int st = 0;
    memcpy(work, raw, sizeof(cplx) * total);
    st |= oracle_compress_lines(n_az, n_range, work, Hr, nthreads);
    st |= oracle_corner_turn(n_az, n_range, work, rd);                 /* rd[n][m] */
    for (int64_t n = 0; n < n_range; ++n)
        st |= oracle_fft(n_az, rd + n * n_az, -1);                      /* rd[n][f] */
    st |= oracle_rcmc(n_range, n_az, rd, image, kappa, vs, r_near, taps);
    for (int64_t n = 0; n < n_range; ++n) {
        double r = r_near + (double)n;
        cplx *line = image + n * n_az;
        for (int64_t j = 0; j < n_az; ++j) {
            double cyc = kappa * r * migration_d(az_freq(j, n_az), kappa, vs);
            double ph = kTwoPi * (cyc - floor(cyc));
#if ORACLE_PLANT == 8
            ph = -ph; /* planted: filter conjugated */
#endif
            line[j] *= cos(ph) + I * sin(ph);
        }
        st |= oracle_fft(n_az, line, +1);
        for (int64_t j = 0; j < n_az; ++j)
            line[j] /= (double)n_az;
    }
    free(work);
    free(rd);
    return st ? -1 : 0;
}

/* Which planted mistake this compiled copy of the oracle carries (0 = none). */
int oracle_planted(void) { return ORACLE_PLANT; }
