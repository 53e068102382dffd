// Host interface of the one-launch ragged batch kernel (batch_persistent.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sar {

// One strip as the kernel sees it.  Range lines are raw rows of n_range
// samples; azimuth lines are image rows of n_az samples, transformed at
// length l_az (zero-padded when n_az < l_az).
struct BStrip {
    const float2 *raw;       // [n_az][n_range], read only
    float2 *image;           // [n_range][n_az]
    const float2 *filt_r, *tw_r;   // range class: filter in register order, twiddles
    const float2 *filt_a, *tw_a;   // azimuth class
    int32_t n_range, n_az, l_az;
    int32_t expect;          // range lines that must be done before an azimuth item runs (n_az)
};

// One work item: `nlines` consecutive lines (line0 ...) of one strip, of one
// kind.  Range lines are azimuth rows; azimuth lines are range bins.
struct BItem {
    int32_t kind;            // 0 range, 1 azimuth
    int32_t strip;
    int32_t line0, nlines;
};

constexpr int kBatchThreads = 512;   // one block per SM

// Lines of length n that one item holds (the block's threads split into
// groups of n / E threads, one line each), or 0 if n is not supported.
int batch_lines_per_item(int n);
// The name of the compiled schedule whose geometry the kernel uses for
// length n (twiddle tables and filter order are built from it), or nullptr.
const char *batch_schedule_name(int n);
// Dynamic shared memory of one block.
int batch_smem_bytes();
// Blocks of the kernel resident on the whole current device (0 on error).
int batch_grid();
// One launch over the item list.  done[n_strips] and next[0] must be zero
// (the caller clears them before every launch); status is set to 5 when a
// bounded wait runs out, and then every block stops taking items.
cudaError_t launch_batch_persistent(const BItem *items, int n_items, const BStrip *strips, int *done, int *next,
                                    int *status, long long wait_cycles, cudaStream_t st);
cudaError_t prepare_batch_persistent();

}  // namespace sar
