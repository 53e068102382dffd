// Plan-time table builders (device side).
#pragma once
#include "registry.h"

namespace sar {
cudaError_t build_twiddles(const SchedDesc &d, float2 *tw, cudaStream_t st);
cudaError_t build_filter(const SchedDesc &d, const float2 *H, float2 *filt, int32_t *idx_dev, cudaStream_t st);
cudaError_t make_lfm_line(int n, int nc, double tbp, float2 *out, cudaStream_t st);
cudaError_t conjugate(float2 *x, int n, cudaStream_t st);
// unfused comparison path: natural-order filter with 1/N, and the multiply
cudaError_t build_natural_filter(const float2 *H, float2 *dst, int n, cudaStream_t st);
cudaError_t spectrum_multiply(float2 *data, const float2 *h, int64_t n_lines, int64_t n, cudaStream_t st);
cudaError_t launch_transpose(const float2 *in, float2 *out, int64_t rows, int64_t cols, cudaStream_t st);
// 0: automatic (32 x 32 tiles: measured faster on GB300 at 4096^2 and 8192^2),
// 1: always 32 x 32 tiles, 2: 64 x 64 tiles wherever the shape allows
void set_corner_turn_variant(int v);
// split-precision tensor-core line compression (N = 256 or 4096)
cudaError_t launch_mma_compress(int n, int prec, const float2 *in, float2 *out, int64_t n_lines, int64_t ld,
                                const float2 *filt_pos, const float2 *tw, cudaStream_t st);
void mma_filter_positions(int n, int32_t *idx);
// the same on the fifth-generation tensor cores (tcgen05.mma, TMEM
// accumulators); status / wait_cycles bound its completion waits
// (a_in_tmem: the split data as the A operand in tensor memory, written
// with tcgen05.st; else in shared-memory tiles)
cudaError_t launch_mma_tc_compress(int n, int prec, bool a_in_tmem, const float2 *in, float2 *out, int64_t n_lines,
                                   int64_t ld, const float2 *filt_pos, const float2 *tw, int *status,
                                   long long wait_cycles, cudaStream_t st);
// full Range-Doppler processing (RCMC and the range-dependent azimuth filter)
const char *rd_az_schedule(int n);
cudaError_t launch_az_compress_rd(int n, const float2 *in, float2 *out, int64_t n_lines, const float2 *tw,
                                  const void *cols, double r_near, cudaStream_t st);
cudaError_t launch_az_fft_rd(int n, const float2 *in, float2 *out, int64_t n_lines, const float2 *tw, cudaStream_t st);
cudaError_t launch_rcmc(int taps, const float2 *in, float2 *out, int n_range, int n_f, const void *cols,
                        double r_near, int staged_rows, cudaStream_t st);
int rcmc_staged_rows(int n_range, int n_f, double r_near, const void *host_cols);
void rd_columns(int n_f, double kappa, double vs, void *host_cols);
// lines whose length is not a power of two (zero-padded linear convolution)
size_t wrap_filter_scratch_bytes(int n, int L);
cudaError_t build_wrap_filter(const float2 *H, int n, int L, void *scratch, float2 *G, cudaStream_t st);
size_t bluestein_scratch_bytes(int L);
cudaError_t build_bluestein_tables(int n, int L, float2 *chirp, float2 *G, void *scratch, cudaStream_t st);
cudaError_t launch_bluestein(const SchedDesc &d, const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int n,
                             const float2 *filt, const float2 *tw, const float2 *chirp, int inverse, cudaStream_t st);
size_t rd_column_bytes();
int corner_turn_variant();
}  // namespace sar
