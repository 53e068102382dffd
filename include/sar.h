/*
 * sar.h -- C-ABI of the GB300 (sm_103a) kernel-fused SAR Range-Doppler
 * compression library (libsar.so).
 *
 * The method (Bergach, "From 8 Seconds to 370 ms: Kernel-Fused SAR Imaging
 * ...", arXiv 2604.03585):
 *   - Sec. II-B: per line, load -> FFT -> multiply by the pre-computed matched
 *     filter spectrum -> IFFT -> store, in one kernel, two device-memory
 *     transfers per line.
 *   - Sec. II-C: IFFT(x) = conj(FFT(conj x)) / N, the 1/N folded into the
 *     fused kernel (here: into the stored filter).
 *   - Sec. IV-A/IV-B: Range-Doppler processing of an N_a x N_r scene: range
 *     compression of every azimuth line, a corner turn (global transpose) so
 *     that azimuth columns become rows, and the same fused compression along
 *     azimuth.
 *
 * Conventions for every entry point:
 *   - Complex samples are complex64: interleaved (re, im) float32 pairs,
 *     8 bytes each.  Matrices are row-major and dense.
 *   - Data pointers passed to compute calls are DEVICE pointers of the
 *     current CUDA device, 16-byte aligned; the caller owns them.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Compute
 *     calls only enqueue work on it and return without synchronising the
 *     host; results are ready when the stream reaches that point.
 *   - Every call returns a sar_status.  Argument errors are detected before
 *     anything is enqueued and leave all buffers untouched.  A CUDA error seen
 *     at launch is returned as SAR_ERR_CUDA; an error raised later by the
 *     device surfaces on a later call or on sar_sync().  sar_last_error()
 *     gives a message for the calling thread's last failure.
 *   - No C++ exception crosses this interface.
 *   - Supported line lengths: powers of two from 256 to 16384.
 */
#ifndef SAR_GB300_H
#define SAR_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SAR_API __attribute__((visibility("default")))
#else
#define SAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *sar_stream; /* same type as cudaStream_t */

typedef struct sar_plan_s *sar_plan; /* opaque; immutable after creation; usable from any stream */

typedef enum {
    SAR_OK = 0,
    SAR_ERR_INVALID_ARG = 1,   /* null/misaligned pointer, size out of range, bad flag */
    SAR_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement (e.g. N > 16384) */
    SAR_ERR_OUT_OF_MEMORY = 3, /* a plan allocation failed; nothing was leaked */
    SAR_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
    SAR_ERR_TIMEOUT = 5        /* a bounded device-side wait gave up */
} sar_status;

typedef enum {
    SAR_PREC_FP32 = 0 /* FP32 arithmetic throughout (FP64 only for table phases) */
} sar_precision;

/* Matched filters of a plan (Sec. II-B step 3: "pre-computed matched filter").
 * range_spectrum: device, complex64[n_range]: H_r[k], natural frequency order,
 *                 unnormalised (e.g. conj(FFT(reference range chirp))).
 * az_spectrum:    device, complex64[n_az]:    H_a[k], the same for azimuth
 *                 (one spectrum for every range bin).
 * Both are copied (permuted, with 1/N folded in) into plan-owned memory by
 * sar_plan_create; the caller may free them afterwards. */
typedef struct {
    const void *range_spectrum;
    const void *az_spectrum;
    int32_t precision; /* sar_precision */
    uint32_t flags;    /* must be 0 */
} sar_filters;

/* Create a plan for an n_az x n_range scene (Sec. IV-A, the N_a x N_r data
 * matrix).  n_range and n_az: powers of two in [256, 16384].  Allocates the
 * plan's device tables on the current device, builds them (FP64 twiddle
 * phases rounded to FP32) and synchronises the device once; not for the hot
 * loop.  *out receives the plan, or NULL on failure. */
SAR_API sar_status sar_plan_create(int64_t n_range, int64_t n_az, const sar_filters *filters, sar_plan *out);

/* Release a plan and its device memory.  The caller must make sure no work
 * that uses the plan is still queued.  NULL is accepted. */
SAR_API sar_status sar_plan_destroy(sar_plan plan);

/* Range compression, Sec. IV-A step 1 with the fused kernel of Sec. II-B:
 * every azimuth line x (n_az rows of n_range samples) becomes
 * IFFT(FFT(x) . H_r), in place.  data: device complex64[n_az][n_range]. */
SAR_API sar_status sar_range_compress(sar_plan plan, void *data, sar_stream stream);

/* Corner turn, Sec. IV-A step 2 / Sec. IV-B (the global transpose between
 * the range and azimuth steps): out[c][r] = in[r][c] for in of n_az rows and
 * n_range columns.  in: device complex64[n_az][n_range]; out: device
 * complex64[n_range][n_az]; the two must not overlap.  Bit-exact copy. */
SAR_API sar_status sar_corner_turn(sar_plan plan, const void *in, void *out, sar_stream stream);

/* Azimuth compression, Sec. IV-A step 4 in its full form: every range bin
 * (n_range rows of n_az samples after the corner turn) becomes
 * IFFT(FFT(x) . H_a), in place.  data: device complex64[n_range][n_az]. */
SAR_API sar_status sar_azimuth_compress(sar_plan plan, void *data, sar_stream stream);

/* The three steps in order: range compression in place on raw, corner turn
 * raw -> image, azimuth compression in place on image.
 * raw:   device complex64[n_az][n_range], input; overwritten (range-compressed).
 * image: device complex64[n_range][n_az], output; must not overlap raw. */
SAR_API sar_status sar_rda_process(sar_plan plan, void *raw, void *image, sar_stream stream);

/* Out-of-place range compression: out = IFFT(FFT(in) . H_r) line by line;
 * in is not modified.  in, out: device complex64[n_az][n_range]; in == out is
 * the in-place call, any other overlap is refused. */
SAR_API sar_status sar_range_compress_oop(sar_plan plan, const void *in, void *out, sar_stream stream);

/* The three steps leaving the raw echo intact: range compression raw -> work,
 * corner turn work -> image, azimuth compression in place on image.  Same
 * three kernels and the same HBM traffic as sar_rda_process.
 * raw: device complex64[n_az][n_range] (read only); work: device
 * complex64[n_az][n_range] scratch owned by the caller; image: device
 * complex64[n_range][n_az].  The three buffers must not overlap. */
SAR_API sar_status sar_rda_process_oop(sar_plan plan, const void *raw, void *work, void *image, sar_stream stream);

/* The same three steps on HOST buffers: copies raw to the device, runs
 * sar_rda_process, copies the image back, and returns once the image is in
 * host memory.  raw: host complex64[n_az][n_range] (not modified);
 * image: host complex64[n_range][n_az].  Pinned host memory gives the full
 * copy bandwidth.  The plan allocates its device staging buffers on the first
 * call (2 x n_az x n_range x 8 bytes) and keeps them until destroyed. */
SAR_API sar_status sar_rda_process_host(sar_plan plan, const void *raw, void *image, sar_stream stream);

/* Matched-filter helper (Sec. II-B step 3, Sec. V-A's chirp signal model):
 * writes H[k] = conj(FFT_n(c)) to out (device complex64[n]) where c is the
 * unit-amplitude linear-FM chirp of n_chirp samples and time-bandwidth
 * product tbp, c(m) = exp(i pi (tbp/n_chirp^2) m^2), m = -n_chirp/2 ...
 * n_chirp/2 - 1, centred on index 0 of the length-n line (wrapping).  The
 * chirp phase is evaluated in FP64 on the device and rounded to FP32; the
 * transform is this library's FP32 FFT.  n: power of two in [256, 16384];
 * 1 <= n_chirp <= n; tbp > 0. */
SAR_API sar_status sar_make_lfm_spectrum(int64_t n, int64_t n_chirp, double tbp, void *out, sar_stream stream);

/* Unnormalised DFT of n_lines lines of length n (natural order in and out):
 * out[l][k] = sum_j in[l][j] exp(-+2 pi i j k / n), '+' when inverse != 0
 * (computed as conj(FFT(conj x)), Sec. II-C).  in and out: device
 * complex64[n_lines][n]; in place allowed.  n: power of two in [256, 16384].
 * Exposes the line FFT engine on its own (tests, filter design). */
SAR_API sar_status sar_fft_lines(int64_t n, int64_t n_lines, const void *in, void *out, int inverse, sar_stream stream);

/* sar_fft_lines without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not have device memory
 * allocated on their behalf -- work recorded inside a CUDA stream capture,
 * real-time / on-board processors that fix their device-memory footprint at
 * start-up, applications whose device memory belongs to a pool allocator.
 * Same arguments and results as sar_fft_lines; it calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its twiddle table lives in one
 * fixed device array of 32768 complex64 values (256 KiB, held by every GPU
 * that loads the library until the process exits); every N in [256, 16384]
 * fits, anything needing more is refused with SAR_ERR_UNSUPPORTED.  Every
 * call rewrites that array on its stream before its FFT, and all calls share
 * it: calls that may run at the same time on the GPU (different streams with
 * no ordering between them) race on it, so order them.  The first call on a
 * device looks up the array's address once; make it before any stream
 * capture. */
SAR_API sar_status sar_fft_lines_static(int64_t n, int64_t n_lines, const void *in, void *out, int inverse,
                                        sar_stream stream);

/* Generic corner turn of a rows x cols complex64 matrix (any sizes >= 1):
 * out[c][r] = in[r][c].  Device pointers, non-overlapping. */
SAR_API sar_status sar_transpose(int64_t rows, int64_t cols, const void *in, void *out, sar_stream stream);

/* Wait for `stream` and report any asynchronous device error. */
SAR_API sar_status sar_sync(sar_stream stream);

/* Message describing the calling thread's most recent failure ("" if none). */
SAR_API const char *sar_last_error(void);

/* Library version string. */
SAR_API const char *sar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SAR_GB300_H */
