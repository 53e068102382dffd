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
 *   - Plans, sar_fft_lines and sar_make_lfm_spectrum take any line length in
 *     [2, 8192] besides the powers of two from 256 to 131072 (see
 *     sar_plan_create, sar_fft_lines); the other entry points take those
 *     powers of two.  Lines up to
 *     16384 samples run one line per thread block; longer lines run one line
 *     per thread-block cluster of 2 to 16 blocks exchanging it through
 *     distributed shared memory (sar_range_compress, sar_azimuth_compress,
 *     sar_rda_process[_oop|_host|_unfused], sar_fft_lines,
 *     sar_make_lfm_spectrum, sar_autotune).  The folded corner turn, split
 *     precision, ragged batches, the full processor's azimuth length and
 *     sar_fft_lines_static stop at 16384 (SAR_ERR_UNSUPPORTED above).
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
    SAR_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement (e.g. N > 131072) */
    SAR_ERR_OUT_OF_MEMORY = 3, /* a plan allocation failed; nothing was leaked */
    SAR_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
    SAR_ERR_TIMEOUT = 5        /* a bounded device-side wait gave up */
} sar_status;

typedef enum {
    SAR_PREC_FP32 = 0,   /* FP32 arithmetic throughout (FP64 only for table phases) */
    /* Split precision on the tensor cores (Sec. III's MMA DFT, Eq. (1)-(2),
     * at radix 16): every radix-16 DFT is a real 32 x 32 matrix product of
     * half-precision parts with FP32 accumulation; twiddles, filter and 1/N
     * in FP32.  Line lengths 256 and 4096 only; no folded corner turn. */
    SAR_PREC_FP16X2 = 1, /* x = hi + lo in FP16, products hi*hi + hi*lo + lo*hi, per-group power-of-two scaling */
    SAR_PREC_BF16X2 = 2, /* the same with BF16 parts (16 mantissa bits in total) */
    SAR_PREC_BF16X3 = 3  /* BF16 hi + mid + lo, six products (24 mantissa bits) */
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
    uint32_t flags;    /* 0 or SAR_PLAN_* bits below */
} sar_filters;

/* Plan flags.  By default sar_rda_process folds the corner turn into the
 * range pass where the range schedule supports it (two kernels, 32 bytes of
 * HBM traffic per sample; powers of two up to 16384, and the mixed-radix
 * lengths with a compiled kernel, 1000 ... 8000, with n_az a multiple of 4);
 * this flag keeps the three separate kernels of
 * Sec. IV-A (48 bytes per sample). */
#define SAR_PLAN_UNFOLDED_CORNER_TURN 1u
/* Azimuth-major output: sar_rda_process_oop and sar_rda_process_host return
 * the image as complex64[n_az][n_range] (the raw echo's orientation, as the
 * paper's pipeline transposes back, Sec. IV-B) by a fourth pass, a transpose
 * of the [n_range][n_az] image (16 bytes per sample).  sar_rda_process, which
 * has no scratch buffer, and sar_rda_full refuse such plans
 * (SAR_ERR_INVALID_ARG). */
#define SAR_PLAN_OUT_AZ_MAJOR 2u

/* Create a plan for an n_az x n_range scene (Sec. IV-A, the N_a x N_r data
 * matrix).  n_range and n_az: powers of two in [256, 131072] (above 16384 on
 * thread-block clusters, without the folded corner turn), or any other length
 * in [2, 8192], which gets the exact length-n compression
 * IFFT_n(FFT_n(x) . H):
 *   - lengths whose prime factors are 2, 3, 5 and 7 only (1000, 3000, 5000,
 *     ..., and powers of two below 256) and that split into at most four
 *     radices of 2 ... 16, 20, 25, 32 run the mixed-radix engine at n itself
 *     (twiddles and filter order designed in FP64 at plan time);
 *   - every other length (a prime factor above 7, e.g. 1009, or 7203 =
 *     3 * 7^4) runs a zero-padded linear convolution at the power-of-two
 *     length L >= 2n - 1 (filter FFT_L(IFFT_n(H)) designed in FP64 at plan
 *     time);
 * one fused launch per pass either way, as for powers of two.  The unfused
 * pipeline needs a transform at the length itself (powers of two and the
 * mixed-radix lengths); split precision needs powers of two.  Allocates the
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

/* The three steps: range compression, corner turn raw -> image, azimuth
 * compression in place on image.  With the corner turn folded into the range
 * pass (the default where supported) raw is only read; otherwise (flag
 * SAR_PLAN_UNFOLDED_CORNER_TURN, or a range length without a folded kernel)
 * raw is range-compressed in place first.
 * raw:   device complex64[n_az][n_range], input; may be overwritten.
 * image: device complex64[n_range][n_az], output; must not overlap raw. */
SAR_API sar_status sar_rda_process(sar_plan plan, void *raw, void *image, sar_stream stream);

/* Out-of-place range compression: out = IFFT(FFT(in) . H_r) line by line;
 * in is not modified.  in, out: device complex64[n_az][n_range]; in == out is
 * the in-place call, any other overlap is refused. */
SAR_API sar_status sar_range_compress_oop(sar_plan plan, const void *in, void *out, sar_stream stream);

/* Range compression with the corner turn folded into its store (Sec. IV-A
 * steps 1 and 2 in one kernel): image[r][a] = (IFFT(FFT(raw[a]) . H_r))[r].
 * raw: device complex64[n_az][n_range] (read only); image: device
 * complex64[n_range][n_az].  Only for plans that fold the corner turn
 * (sar_plan_folds_corner_turn); SAR_ERR_UNSUPPORTED otherwise. */
SAR_API sar_status sar_range_compress_ct(sar_plan plan, const void *raw, void *image, sar_stream stream);

/* The three steps leaving the raw echo intact: range compression raw -> work,
 * corner turn work -> image, azimuth compression in place on image (or, when
 * the corner turn is folded into the range pass, raw -> image directly and
 * work is not touched).  The same kernels and HBM traffic as
 * sar_rda_process.
 * raw: device complex64[n_az][n_range] (read only); work: device
 * complex64[n_az][n_range] scratch owned by the caller; image: device
 * complex64[n_range][n_az].  The three buffers must not overlap.  With
 * SAR_PLAN_OUT_AZ_MAJOR the passes leave the [n_range][n_az] image in work
 * and a fourth pass transposes it into image, complex64[n_az][n_range]. */
SAR_API sar_status sar_rda_process_oop(sar_plan plan, const void *raw, void *work, void *image, sar_stream stream);

/* The unfused comparison pipeline the paper's fused kernel replaces (Sec.
 * II-B, Fig. 1 top; Table II's "unfused baseline", here entirely on the
 * GPU): per pass a forward FFT kernel, a spectrum multiply kernel and an
 * inverse FFT kernel, six device-memory transfers per line instead of two.
 * Same arguments, layouts and results (to rounding) as the fused calls;
 * raw is compressed in place. */
SAR_API sar_status sar_range_compress_unfused(sar_plan plan, void *data, sar_stream stream);
SAR_API sar_status sar_azimuth_compress_unfused(sar_plan plan, void *data, sar_stream stream);
SAR_API sar_status sar_rda_process_unfused(sar_plan plan, void *raw, void *image, sar_stream stream);

/* ---- full Range-Doppler processing with RCMC (Sec. IV-A steps 2-4) ----
 * Geometry, in normalised units: kappa = two-way phase cycles per range
 * sample of path (2 dr / lambda); v_s = platform displacement per azimuth line
 * in range samples; r_near = slant range of range bin 0 in range samples.  A
 * target of closest range r0 sits, in the range-Doppler domain, at range
 * r0 / D(f) with D(f) = sqrt(1 - (f / (kappa v_s))^2) (f in cycles per line)
 * and carries the phase exp(-2 pi i kappa r0 D(f)).  kappa * v_s > 0.5.
 * rcmc_taps: 16 (Hann-windowed sinc interpolation) or 0 (no correction).
 * Stores a per-frequency table in the plan (FP64 evaluated, FP32 stored). */
SAR_API sar_status sar_plan_set_geometry(sar_plan plan, double kappa, double v_s, double r_near, int32_t rcmc_taps);

/* RCMC alone (Sec. IV-A step 2, sinc interpolation), in the range-Doppler
 * domain: out[n][j] = sum over the 16 integers k nearest
 * src = n + (r_near + n)(1/D(f_j) - 1) of h(src - k) in[k][j], with
 * h(x) = sinc(x) (1 + cos(2 pi x / 16)) / 2 and rows outside the scene read as
 * zero; f_j = j / n_az for j < n_az / 2, (j - n_az) / n_az above.  in, out:
 * device complex64[n_range][n_az], not overlapping.  Needs a geometry with
 * rcmc_taps = 16 (SAR_ERR_INVALID_ARG otherwise). */
SAR_API sar_status sar_rcmc(sar_plan plan, const void *in, void *out, sar_stream stream);

/* The full processor: range compression and corner turn (raw -> image),
 * azimuth FFT of every range bin (in place), RCMC (image -> work: output bin n
 * at frequency f interpolates the input at n + (r_near + n)(1/D(f) - 1)), and
 * azimuth compression (work -> image): multiply by
 * H_a(f, r) = exp(+2 pi i kappa r D(f)), r = r_near + n, then the inverse FFT
 * (1/n_az).  raw: device complex64[n_az][n_range] (read only); work, image:
 * device complex64[n_range][n_az]; no overlaps.  The first call per line
 * length allocates the library's twiddle tables. */
SAR_API sar_status sar_rda_full(sar_plan plan, const void *raw, void *work, void *image, sar_stream stream);

/* The same three steps on HOST buffers: copies raw to the device, runs
 * sar_rda_process, copies the image back, and returns once the image is in
 * host memory.  raw: host complex64[n_az][n_range] (not modified);
 * image: host complex64[n_range][n_az] ([n_az][n_range] for a plan with
 * SAR_PLAN_OUT_AZ_MAJOR).  Pinned host memory gives the full
 * copy bandwidth.  The plan allocates its device staging buffers on the first
 * call (2 x n_az x n_range x 8 bytes) and keeps them until destroyed.  On a
 * plan that folds the corner turn (image [n_range][n_az], n_az a multiple of
 * 8 x its cluster or block size, n_range of 8) the call is a pipeline on
 * internal copy-in, compute and copy-out streams: the echo arrives in 8
 * blocks of azimuth lines and each block's range pass starts as soon as it
 * has landed; the azimuth pass runs in 8 blocks of range bins, each copied
 * back while the next is computed.  One host-buffer call per plan runs at a
 * time.  A single scene's copies cannot overlap each other (its image needs
 * all of its echo): sar_rda_process_host_n overlaps those of successive
 * scenes. */
SAR_API sar_status sar_rda_process_host(sar_plan plan, const void *raw, void *image, sar_stream stream);

/* n_scenes scenes on host buffers in one call, raws[q] -> images[q], each as
 * sar_rda_process_host computes it (bit for bit).  On a plan whose
 * single-scene call is pipelined the scenes share one pipeline with two
 * device staging sets, scene q in set q mod 2: the echo of scene q + 1 is
 * copied in while the image of scene q is copied out, both directions of the
 * host link at once.  The plan then keeps the second staging set (another
 * 2 x n_az x n_range x 8 bytes) until destroyed.  On other plans the scenes
 * run one after another.  raws: n_scenes host pointers to complex64
 * [n_az][n_range] (not modified); images: n_scenes host pointers to complex64
 * images as for sar_rda_process_host; all non-NULL.  An image may not overlap
 * any echo (SAR_ERR_INVALID_ARG).  One image buffer may serve several scenes:
 * images are written in scene order, so it ends up holding the last of them.
 * n_scenes = 0 does nothing.  Returns once every image is in host memory. */
SAR_API sar_status sar_rda_process_host_n(sar_plan plan, int32_t n_scenes, const void *const *raws,
                                          void *const *images, sar_stream stream);

/* Matched-filter helper (Sec. II-B step 3, Sec. V-A's chirp signal model):
 * writes H[k] = conj(FFT_n(c)) to out (device complex64[n]) where c is the
 * unit-amplitude linear-FM chirp of n_chirp samples and time-bandwidth
 * product tbp, c(m) = exp(i pi (tbp/n_chirp^2) m^2), m = -n_chirp/2 ...
 * n_chirp/2 - 1, centred on index 0 of the length-n line (wrapping).  The
 * chirp phase is evaluated in FP64 on the device and rounded to FP32; the
 * transform is this library's FP32 FFT.  n: power of two in [256, 131072] or
 * any length in [2, 8192];
 * 1 <= n_chirp <= n; tbp > 0. */
SAR_API sar_status sar_make_lfm_spectrum(int64_t n, int64_t n_chirp, double tbp, void *out, sar_stream stream);

/* Point-target echo simulator (the chirp signal model of Sec. V-A with
 * normalised parameters): writes the n_az x n_range complex64 echo of
 * n_targets unit targets at (targets[2k], targets[2k+1]) = (a0, r0), each
 * the product of an azimuth chirp (nc_az samples, time-bandwidth tbp_az) and a
 * range chirp (nc_range, tbp_range) centred on the target (indices modulo the
 * scene size), plus circular complex Gaussian noise of total variance
 * 10^(-snr_db/10) drawn from seed (snr_db = NaN: no noise).  Uses the
 * counter-based splitmix64 / Box-Muller definition of the host generator
 * `sarsim`, so the two agree to the last bit of complex64 up to FP64
 * rounding of log/cos/sin.  targets: host array; out: device
 * complex64[n_az][n_range].  1 <= nc <= n; at most 32 targets. */
SAR_API sar_status sar_simulate_echo(int64_t n_az, int64_t n_range, const int64_t *targets, int32_t n_targets,
                                     int64_t nc_range, double tbp_range, int64_t nc_az, double tbp_az,
                                     double snr_db, uint64_t seed, void *out, sar_stream stream);

/* Unnormalised DFT of n_lines lines of length n (natural order in and out):
 * out[l][k] = sum_j in[l][j] exp(-+2 pi i j k / n), '+' when inverse != 0
 * (computed as conj(FFT(conj x)), Sec. II-C).  in and out: device
 * complex64[n_lines][n]; in place allowed.  n: power of two in [256, 131072],
 * or any other length in [2, 8192]: a length of the mixed-radix engine (prime
 * factors 2, 3, 5, 7; see sar_plan_create) runs its forward passes at n and
 * writes the spectrum in natural order; any other length takes the DFT by
 * Bluestein's identity jk = (j^2 + k^2 - (k-j)^2)/2, a chirp multiply
 * (c_m = exp(-i pi m^2 / n), phases reduced exactly mod 2n in FP64), a linear
 * convolution with conj(c) through the power-of-two engine at L >= 2n - 1
 * (filter designed in FP64 on the first call per length and cached, which
 * allocates) and a chirp multiply of the output, in one kernel.  Either way
 * the first call per length builds and caches its tables (allocates).
 * Exposes the line FFT engine on its own (tests, filter design). */
SAR_API sar_status sar_fft_lines(int64_t n, int64_t n_lines, const void *in, void *out, int inverse, sar_stream stream);

/* sar_fft_lines without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not have device memory
 * allocated on their behalf -- real-time / on-board processors that fix
 * their device-memory footprint at start-up, applications whose device
 * memory belongs to a pool allocator.
 * Same arguments and results as sar_fft_lines; it calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its twiddle table lives in one
 * fixed device array of 32768 complex64 values (256 KiB, held by every GPU
 * that loads the library until the process exits); every N in [256, 16384]
 * fits, anything needing more is refused with SAR_ERR_UNSUPPORTED.  Every
 * call rewrites that array on its stream before its FFT, and all calls share
 * it: calls that may run at the same time on the GPU (different streams with
 * no ordering between them) race on it, so order them.  The first call on a
 * device looks up the array's address once, and the first call at each line
 * length loads that length's kernels (CUDA loads modules lazily by default)
 * and sets their attributes once, so it does more host work than later
 * calls. */
SAR_API sar_status sar_fft_lines_static(int64_t n, int64_t n_lines, const void *in, void *out, int inverse,
                                        sar_stream stream);

/* Generic corner turn of a rows x cols complex64 matrix (any sizes >= 1):
 * out[c][r] = in[r][c].  Device pointers, non-overlapping. */
SAR_API sar_status sar_transpose(int64_t rows, int64_t cols, const void *in, void *out, sar_stream stream);

/* ---- ragged batches ----------------------------------------------------
 * Many strips of different sizes compressed by one CUDA-graph launch.  A
 * strip is a raw echo of n_az azimuth lines by n_range range samples; its
 * azimuth lines are transformed at length L = max(256, next power of two
 * >= n_az), zero-padded, and the image keeps n_az columns (the correlation
 * of the zero-padded lines is circular at length L).  The paper processes one
 * scene size (Sec. IV); batching strips of mixed sizes is this library's
 * extension of the same three steps. */
typedef struct {
    int64_t n_range;            /* power of two in [256, 16384] */
    int64_t n_az;               /* 1 ... 16384 azimuth lines (L <= 16384) */
    const void *raw;            /* device complex64[n_az][n_range], read only */
    void *image;                /* device complex64[n_range][n_az], output */
    const void *range_spectrum; /* device complex64[n_range] */
    const void *az_spectrum;    /* device complex64[L] (complex64[n_az] with SAR_BATCH_EXACT_AZIMUTH) */
} sar_strip;

typedef struct sar_batch_s *sar_batch;

typedef struct {
    int64_t strips;          /* strips in the batch */
    int64_t samples;         /* sum of n_az * n_range */
    int64_t work_bytes;      /* batch-owned scratch (range-compressed strips) */
    int32_t kernels_per_run; /* kernels in the graph */
    int32_t range_classes;   /* distinct (n_range, range spectrum) */
    int32_t azimuth_classes; /* distinct (L, azimuth spectrum) */
} sar_batch_info_t;

/* Group the strips into classes (a class shares a line geometry and a
 * filter: range classes by (n_range, range spectrum), azimuth classes by (L,
 * azimuth spectrum)), build each class's filter and twiddle tables, and
 * capture the whole batch into one CUDA graph.
 * flags 0: the graph is one memset and ONE persistent kernel.  Each resident
 * block (one per SM) takes work items from one list: range items (k azimuth
 * rows of a strip, k = 16384 / n_range, compressed along range and written
 * straight into the corner-turned image, Sec. IV-A steps 1-2) and azimuth
 * items (k range bins, compressed along azimuth in place, Sec. IV-A step 4).
 * A strip's azimuth items wait on a device counter of its finished range
 * lines; that wait is bounded (about a second of SM clock, SAR_WAIT_CYCLES),
 * and a run whose wait ran out is reported by sar_batch_status.  No work
 * buffer.
 * flags SAR_BATCH_MULTI_KERNEL or SAR_BATCH_EXACT_AZIMUTH: see below (one
 * launch per class, a batched corner turn, a work buffer of 8 bytes per raw
 * sample).
 * The strip buffers stay owned by the caller and must outlive the batch; the
 * spectra are copied.  Synchronises the device. */
/* Azimuth lines compressed at exactly their n_az samples (the circular
 * correlation at n_az, as a plan of that length computes it) instead of
 * zero-padded to L: az_spectrum holds n_az values, classes are (n_az, azimuth
 * spectrum), and a length that is not a power of two (at most 8192) runs the
 * zero-padded linear convolution of sar_plan_create, one launch per strip in
 * the graph. */
#define SAR_BATCH_EXACT_AZIMUTH 1u
/* The multi-kernel graph instead of the one persistent kernel, with the same
 * (zero-padded) semantics: one fused launch per class walking a segment
 * table, one batched corner turn, a work buffer of 8 bytes per raw sample.
 * On GB300 it runs the config-4 batch faster than the one-launch kernel,
 * whose blocks are sized for 16384-sample lines (one per SM, the lines of an
 * item advancing together), while the per-class kernels run four or five
 * blocks per SM. */
#define SAR_BATCH_MULTI_KERNEL 2u
/* With SAR_BATCH_MULTI_KERNEL (or SAR_BATCH_EXACT_AZIMUTH): before the graph
 * is captured, time every compiled schedule of each class's power-of-two
 * length (sar_autotune, kind SAR_TUNE_FUSED, 5 repetitions on up to 2^24
 * samples of lines; allocates and synchronises) and give the class the
 * fastest one that has a segment-table kernel (as after sar_autotune, the
 * fastest schedule of each length also becomes its preferred one); without it
 * a class takes the preferred schedule of its length.  Refused
 * (SAR_ERR_INVALID_ARG) for the one-launch kernel, whose line engines are
 * compiled in. */
#define SAR_BATCH_AUTOTUNE 4u
SAR_API sar_status sar_batch_create(const sar_strip *strips, int32_t count, uint32_t flags, sar_batch *out);

/* Compress every strip of the batch: one graph launch on `stream`;
 * asynchronous. */
SAR_API sar_status sar_batch_run(sar_batch batch, sar_stream stream);

/* Synchronise `stream` and report whether a bounded device wait of the
 * one-launch batch kernel ran out in a run since the last call:
 * SAR_ERR_TIMEOUT (the record is then cleared; the images of that run are
 * incomplete, the context stays usable), else SAR_OK.  Every block stops
 * taking work items once a wait has run out, so such a run ends within about
 * one wait bound. */
SAR_API sar_status sar_batch_status(sar_batch batch, sar_stream stream);

/* Sizes of a batch. */
SAR_API sar_status sar_batch_info(sar_batch batch, sar_batch_info_t *info);

/* Release the batch (no run may still be in flight).  NULL is accepted. */
SAR_API sar_status sar_batch_destroy(sar_batch batch);

/* ---- serving ----------------------------------------------------------
 * A continuous-batching request loop (this library's serving layer around
 * the paper's per-scene compression).  Scenes of a few size classes arrive
 * over time; a request is admitted as soon as one of max_inflight slots (CUDA
 * streams) is free and its footprint (raw + image, 16 bytes per sample) fits
 * the HBM budget left by the requests still running.  An admitted request
 * allocates its buffers from the server's stream-ordered memory pool, copies
 * its echo in from the device-resident pool scene of its class (the ingest,
 * part of its latency), runs sar_rda_process with its class's resident plan,
 * optionally copies the image out, frees its buffers and records a completion
 * event.  Requests on different slots overlap on the GPU.  When the oldest
 * waiting request does not fit, later ones that do fit may pass it for at
 * most backfill_s seconds.  With size_priority set, each slot holds one
 * stream per distinct scene size, and a request runs on the one of its
 * class.  Stream priority rises as scene size falls, up to the device's
 * range of priorities.  When SMs free up, the waiting blocks of smaller scenes
 * are dispatched first.  Admission order and every result are unchanged.
 * Priorities only order work on different hardware work queues.  A process
 * that serves with size_priority should therefore set
 * CUDA_DEVICE_MAX_CONNECTIONS=32 before its first CUDA call.  Under the
 * default of 8 queues, slots share queues, and a small request can wait behind
 * a large one queued ahead of it.  The largest class gets the SMs no sooner than
 * the others leave them free.  At high load its latency therefore grows, and
 * under sustained overload it can be starved; with one priority it cannot.
 * aging_s > 0 bounds this.  While some request has been in flight for more
 * than aging_s seconds, only requests of its size or larger are admitted, and
 * the smaller ones wait in the queue until it completes. */
typedef struct {
    int32_t n_classes;                   /* size classes */
    int32_t max_inflight;                /* concurrent requests, 1 ... 256 */
    const int64_t *n_range;              /* [n_classes] powers of two in [256, 131072] */
    const int64_t *n_az;                 /* [n_classes] powers of two in [256, 131072] */
    const void *const *pool;             /* [n_classes] device complex64[n_az][n_range] echoes to ingest */
    const void *const *range_spectrum;   /* [n_classes] device complex64[n_range] */
    const void *const *az_spectrum;      /* [n_classes] device complex64[n_az] */
    int64_t hbm_budget_bytes;            /* admission budget */
    double backfill_s;                   /* how long later requests may pass a blocked head */
    int32_t size_priority;               /* nonzero: smaller scenes on higher-priority streams */
    double aging_s;                      /* > 0: bound on starvation under size_priority (below) */
} sar_server_config;

typedef struct {
    double arrival_s;     /* seconds after the run starts (non-decreasing) */
    int32_t size_class;   /* index of the request's size class */
    void *output;         /* device complex64[n_range][n_az] receiving the image, or NULL */
} sar_request;

typedef struct {
    double arrival_s;     /* as requested (0 in closed loop) */
    double admit_s;       /* host time the request was admitted */
    double done_s;        /* GPU time its work completed; latency = done_s - arrival_s */
    int32_t status;       /* SAR_OK, or the error of this request */
} sar_request_result;

#define SAR_SERVE_OPEN_LOOP 0   /* requests arrive at their arrival_s */
#define SAR_SERVE_CLOSED_LOOP 1 /* every request is waiting at time 0 (saturation) */

typedef struct sar_server_s *sar_server;

/* Create plans for every class (resident until destroy), the slots and the
 * memory pool.  The pool scenes and spectra must stay valid while the
 * server exists. */
SAR_API sar_status sar_server_create(const sar_server_config *config, sar_server *out);

/* Serve n requests and fill results[n]; returns when all are done.  The
 * calling thread runs the loop (admission, completion polling); the device
 * must not be used by anything else meanwhile. */
SAR_API sar_status sar_server_run(sar_server server, const sar_request *requests, int32_t n, int32_t mode,
                                  sar_request_result *results);

/* Release the server (plans, streams, memory pool).  NULL is accepted. */
SAR_API sar_status sar_server_destroy(sar_server server);

/* ---- schedules and the autotuner --------------------------------------
 * A schedule fixes how the fused line kernel of one line length N runs: the
 * samples held per thread (E), the pass radices (N = r1*r2*r3, r3 = 1 for two
 * passes), the lines per thread block, and the resulting block size and
 * shared memory.  Several schedules are compiled per N; which one is fastest
 * depends on the GPU, so a plan takes the process-wide preferred schedule of
 * each length (the first compiled one until sar_autotune or
 * sar_set_preferred_schedule changes it), or names one explicitly.
 * cluster_blocks > 1: one line per cluster of that many blocks; e, r1..r3,
 * threads_per_block and smem_bytes then describe each block's
 * n / cluster_blocks point part of the line. */
typedef struct {
    char name[48];
    int32_t n, e, r1, r2, r3, lines_per_block, threads_per_block, smem_bytes;
    int32_t cluster_blocks;
} sar_schedule_desc;

/* Number of compiled schedules, and the description of schedule `index`
 * (0 <= index < count). */
SAR_API int32_t sar_schedule_count(void);
SAR_API sar_status sar_schedule_get(int32_t index, sar_schedule_desc *out);

/* Make the named schedule the preferred one for its length (process-wide,
 * thread-safe; affects plans created afterwards); if it has a folded
 * range + corner-turn kernel it also becomes the preferred one of that
 * kind. */
SAR_API sar_status sar_set_preferred_schedule(const char *name);

/* sar_plan_create with explicit schedules for the range and azimuth lines
 * (NULL = the preferred schedule of that length).  SAR_ERR_INVALID_ARG if a
 * name is unknown or belongs to another length. */
SAR_API sar_status sar_plan_create_ex(int64_t n_range, int64_t n_az, const sar_filters *filters,
                                      const char *range_schedule, const char *az_schedule, sar_plan *out);

/* Corner-turn kernel choice (process-wide): 0 = the default (32 x 32 tiles
 * of 8-byte accesses), 1 = the same, 2 = 64 x 64 tiles of 16-byte accesses
 * where rows and columns are multiples of 64 (the 32 x 32 kernel elsewhere).
 * The 32 x 32 kernel is the faster on GB300 (4096 x 4096: 47.5 against
 * 49.5 us).  Any other value is refused. */
SAR_API sar_status sar_set_corner_turn_variant(int32_t variant);

/* 1 if sar_rda_process of this plan folds the corner turn into the range
 * pass (two kernels), 0 if it runs three kernels (or plan is NULL). */
SAR_API int32_t sar_plan_folds_corner_turn(sar_plan plan);

/* The schedules a plan runs. */
SAR_API sar_status sar_plan_get_schedules(sar_plan plan, sar_schedule_desc *range, sar_schedule_desc *az);

/* Engine of the split-precision plans (process-wide, thread-safe; takes
 * effect at the next launch): 0 = every radix-16 DFT as tcgen05.mma on the
 * fifth-generation tensor cores, 128 groups x 32 x 32 per instruction, FP32
 * accumulators in tensor memory and the split data written by each thread
 * into its own tensor-memory lane as the A operand (the default); 2 = the
 * same with the A operand in shared-memory tiles; 1 = the warp-level
 * mma.sync.m16n8k16 form, 8 groups per instruction.  Same products, scaling
 * and results within rounding.  SAR_ERR_INVALID_ARG for any other value. */
SAR_API sar_status sar_set_split_engine(int32_t engine);

/* Time every compiled schedule of length n (reps launches each, CUDA events
 * on `stream`, median) and make the fastest the preferred schedule of n for
 * that kind of kernel:
 *   kind SAR_TUNE_FUSED:    the fused line compression on n_lines lines;
 *   kind SAR_TUNE_RANGE_CT: the range pass with the folded corner turn on
 *                           n_lines lines (schedules that have it; n_lines a
 *                           multiple of 4).
 * Returns the winner and its median time in milliseconds; if all_ms is not
 * NULL it receives each candidate's median (up to all_cap values; 0 for a
 * schedule without that kind of kernel), in the order sar_schedule_get lists
 * the schedules of length n.  Allocates (and frees) 2 x n_lines x n x 8 bytes
 * of device memory and synchronises the stream; a tuning call, not for the
 * hot path.  n_lines >= 1, reps >= 1. */
#define SAR_TUNE_FUSED 0
#define SAR_TUNE_RANGE_CT 1
SAR_API sar_status sar_autotune(int64_t n, int64_t n_lines, int32_t reps, int32_t kind, sar_stream stream,
                                sar_schedule_desc *best, float *best_ms, float *all_ms, int32_t all_cap);

/* Synchronise `stream` and report whether any kernel of this plan gave up a
 * bounded device-side wait since the last check (SAR_ERR_TIMEOUT; the lines
 * it was processing were not written), then clear that record.  The
 * persistent kernels bound every wait by about one second of SM clock
 * (SAR_WAIT_CYCLES overrides it when the plan is created). */
SAR_API sar_status sar_plan_status(sar_plan plan, sar_stream stream);

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
