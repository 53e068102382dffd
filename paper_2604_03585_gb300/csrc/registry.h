// Schedule registry: every compiled line-engine configuration, with host
// launchers.  A schedule fixes the line length N, the per-thread element
// count E, the pass radices and the number of lines per block (LPB).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sar {

// Extra arguments of the persistent kernels (ignored by the others).
struct FusedCtl {
    int *status;              // device status word: 5 after a timed-out wait, else untouched
    long long wait_cycles;    // bound of every device-side wait, in SM clocks
    int64_t skip_line;        // test hook: never start the copy of this line (-1: off)
};

typedef cudaError_t (*fused_fn)(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                                const float2 *filt, const float2 *tw, const FusedCtl &ctl, cudaStream_t st);
typedef cudaError_t (*dft_fn)(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                              const float2 *tw, int inverse, cudaStream_t st);
typedef cudaError_t (*prep_fn)(void);
// range compression with the corner turn folded into the store: in is
// [n_lines][n] (row stride ld_in), img is [n][ld_img] receiving img[k][l]
typedef cudaError_t (*fused_ct_fn)(const float2 *in, float2 *img, int64_t n_lines, int64_t ld_in, int64_t ld_img,
                                   const float2 *filt, const float2 *tw, cudaStream_t st);

// Fused pass over a segment table (ragged batches); segs/line_begin are
// device arrays (n_seg segments, n_seg + 1 prefix sums of their lines).
struct Seg;
typedef cudaError_t (*seg_fn)(const Seg *segs, const int64_t *line_begin, int n_seg, int64_t n_lines, bool ragged,
                              const float2 *filt, const float2 *tw, cudaStream_t st);

struct SchedDesc {
    const char *name;
    int n, e, r1, r2, r3;   // r3 == 1 for two-pass schedules
    int lpb;                // lines per block
    int threads;            // threads per block = (n / e) * lpb
    int smem_bytes;         // dynamic shared memory per block
    int tw_elems;           // twiddle table length
    int rl;                 // radix of the last pass
    int persistent;         // 1: resident blocks walk the lines, TMA prefetch of the next line
    fused_fn fused;
    dft_fn dft;
    prep_fn prepare;        // raises the dynamic shared-memory limit where needed
    fused_ct_fn fused_ct;   // nullptr: no folded corner turn for this schedule
    int ct_lines;           // lines per block of fused_ct (n_lines must be a multiple)
    seg_fn fused_seg;       // nullptr: no segment-table kernel for this schedule
    int cluster;            // > 1: one line per cluster of this many blocks, N = cluster * (n / cluster);
                            // e, r1..r3, rl, threads and smem_bytes then describe each block's
                            // M = n / cluster point engine, and the twiddle table is the M-point
                            // engine's followed by W_N^{k1 n2} at k1 M + n2 (k1 < cluster, n2 < M)
    int mixed;              // 1: the mixed-radix engine of a 7-smooth length (mixed_radix.h): r1..r3
                            // are its first radices, e is 0, the filter is in the last pass's slot order
};

// All compiled schedules (one table per translation unit).
const SchedDesc *schedules_small(int *count);   // N = 256 .. 1024
const SchedDesc *schedules_2048(int *count);
const SchedDesc *schedules_4096(int *count);        // first: the default of 4096
const SchedDesc *schedules_4096_plain(int *count);
const SchedDesc *schedules_4096_more(int *count);
const SchedDesc *schedules_8192(int *count);
const SchedDesc *schedules_16384(int *count);
const SchedDesc *schedules_cluster(int *count); // N = 32768 ... 131072, one line per cluster

// The preferred schedule for length n, or nullptr.
const SchedDesc *default_schedule(int n);
void set_preferred_schedule(const SchedDesc *d);
const SchedDesc *default_ct_schedule(int n);
void set_preferred_ct_schedule(const SchedDesc *d);
// The schedule that compresses lines of a length n that is not a power of two
// at the engine length L (a power of two >= 2n - 1), or nullptr.  Not part of
// the enumeration below.
const SchedDesc *wrap_schedule(int L);
// Schedule by name, or nullptr.
const SchedDesc *find_schedule(const char *name);
// Visit every schedule.
int schedule_count();
const SchedDesc *schedule_at(int i);

// Host-side permutation of the matched filter into the fused kernel's
// register order: slot j*T + t  (j = s*RL + r)  holds natural frequency
// index k of position P = (t + T*s)*RL + r.  For a cluster schedule, block
// k1's slice (slots k1*M ... k1*M + M - 1) holds k = k1 + C*k_M with k_M the
// M-point engine's index of that slot.
void filter_slot_to_k(const SchedDesc &d, int32_t *idx /* n entries */);

}  // namespace sar
