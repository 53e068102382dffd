// The launch and attribute templates of the compiled mixed-radix lengths and
// their table entry (mixed_radix_ct.cu, mixed_radix_ct2.cu).
#pragma once

#include "mixed_radix.cuh"

namespace sar {
namespace mixed {

template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t launch3(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt, const float2* tw,
                    int, cudaStream_t st) {
    constexpr int LPB = kMixedThreads / T, smem = mixed3_smem<N, T, PD>();
    static_assert(smem <= kMixedSmemMax, "within the shared memory the kernel is set up for");
    fused_mixed3_kernel<N, RA, RB, RC, T, MINB, PD>
        <<<(unsigned)((n_lines + LPB - 1) / LPB), kMixedThreads, smem, st>>>(in, out, n_lines, ld, filt, tw);
    return cudaGetLastError();
}
template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t launch3_dft(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                        int pos_off, int inverse, cudaStream_t st) {
    constexpr int LPB = kMixedThreads / T, smem = mixed3_smem<N, T, PD>();
    mixed3_dft_kernel<N, RA, RB, RC, T, MINB, PD><<<(unsigned)((n_lines + LPB - 1) / LPB), kMixedThreads, smem, st>>>(
        in, out, n_lines, ld, valid, tw, pos_off, inverse ? -1.f : 1.f);
    return cudaGetLastError();
}
template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t attr3() {
    cudaError_t e = cudaFuncSetAttribute(fused_mixed3_kernel<N, RA, RB, RC, T, MINB, PD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mixed3_dft_kernel<N, RA, RB, RC, T, MINB, PD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    return e;
}

struct Spec {
    int n, ra, rb, rc, t, minb;
    mixed3_fn launch;
    mixed3_dft_fn launch_dft;
    cudaError_t (*attr)();
};
#define SAR_SPEC(N, RA, RB, RC, T, MB, PD)                                                             \
    Spec{N,  RA, RB, RC, T, MB, &launch3<N, RA, RB, RC, T, MB, PD>, &launch3_dft<N, RA, RB, RC, T, MB, PD>, \
         &attr3<N, RA, RB, RC, T, MB, PD>}

}  // namespace mixed
}  // namespace sar
