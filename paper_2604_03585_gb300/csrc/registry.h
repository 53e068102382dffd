// Schedule registry: every compiled line-engine configuration, with host
// launchers.  A schedule fixes the line length N, the per-thread element
// count E, the pass radices and the number of lines per block (LPB).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sar {

typedef cudaError_t (*fused_fn)(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                                const float2 *filt, const float2 *tw, cudaStream_t st);
typedef cudaError_t (*dft_fn)(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                              const float2 *tw, int inverse, cudaStream_t st);
typedef cudaError_t (*prep_fn)(void);

struct SchedDesc {
    const char *name;
    int n, e, r1, r2, r3;   // r3 == 1 for two-pass schedules
    int lpb;                // lines per block
    int threads;            // threads per block = (n / e) * lpb
    int smem_bytes;         // dynamic shared memory per block
    int tw_elems;           // twiddle table length
    int rl;                 // radix of the last pass
    fused_fn fused;
    dft_fn dft;
    prep_fn prepare;        // raises the dynamic shared-memory limit where needed
};

// All compiled schedules (one table per translation unit).
const SchedDesc *schedules_small(int *count);   // N = 256 .. 2048
const SchedDesc *schedules_4096(int *count);
const SchedDesc *schedules_large(int *count);   // N = 8192, 16384

// The default schedule for length n, or nullptr.
const SchedDesc *default_schedule(int n);
// Schedule by name, or nullptr.
const SchedDesc *find_schedule(const char *name);
// Visit every schedule.
int schedule_count();
const SchedDesc *schedule_at(int i);

// Host-side permutation of the matched filter into the fused kernel's
// register order: slot j*T + t  (j = s*RL + r)  holds natural frequency
// index k of position P = (t + T*s)*RL + r.
void filter_slot_to_k(const SchedDesc &d, int32_t *idx /* n entries */);

}  // namespace sar
