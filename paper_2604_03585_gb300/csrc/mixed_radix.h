// Line lengths with prime factors 2, 3, 5, 7 only: the mixed-radix fused
// line engine (mixed_radix.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "registry.h"

namespace sar {

// n in [2, 8192], 7-smooth, and factorable into at most four radices of the
// engine (2 ... 16, 20, 25, 32).
bool mixed_length(int n);
// The engine's descriptor for length n (created on first use, kept for the
// life of the library; not part of the enumerated registry), or nullptr.
const SchedDesc *mixed_schedule(int n);
// The inter-pass twiddle tables of length n (FP64 phases rounded once).
cudaError_t build_mixed_twiddles(int n, float2 *tw, cudaStream_t st);
// idx[P] = the frequency held at position P after the forward passes
// (mixed-radix digit reversal): the filter is stored in that order.
void mixed_positions(int n, int32_t *idx);

}  // namespace sar
