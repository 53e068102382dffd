// The launch and attribute templates of the compiled mixed-radix lengths and
// their table entry (mixed_radix_ct.cu, mixed_radix_ct2.cu).
#pragma once

#include "mixed_radix.cuh"
#include "tensor_map.h"

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
// the folded range pass: groups of four lines over n_lines (a multiple of
// 4), 256 / T lines per block, clusters of 4 T / 256 blocks (none for T = 64)
template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t launch3_ct(const float2* in, float2* img, int64_t n_lines, int64_t ld_in, int64_t ld_img,
                       const float2* filt, const float2* tw, cudaStream_t st) {
    constexpr int LPB = kMixedThreads / T, QC = 4 / LPB;
    if (n_lines <= 0) return cudaSuccess;
    if (n_lines % 4 || ld_img % 2) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_lines / LPB), 1, 1);
    cfg.blockDim = dim3(kMixedThreads, 1, 1);
    cfg.dynamicSmemBytes = mixed3_smem<N, T, PD>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = QC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = QC > 1 ? 1 : 0;
    using G = MixedCtGeom<N, T, PD>;
    CUtensorMap m;
    if (image_tensor_map(&m, img, n_lines, N, ld_img, QC, G::BR))
        return cudaLaunchKernelEx(&cfg, fused_mixed3_ct_tma_kernel<N, RA, RB, RC, T, MINB, PD>, in, img, m, ld_in,
                                  ld_img, filt, tw);
    return cudaLaunchKernelEx(&cfg, fused_mixed3_ct_kernel<N, RA, RB, RC, T, MINB, PD>, in, img, ld_in, ld_img, filt,
                              tw);
}
template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t attr3() {
    cudaError_t e = cudaFuncSetAttribute(fused_mixed3_kernel<N, RA, RB, RC, T, MINB, PD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mixed3_dft_kernel<N, RA, RB, RC, T, MINB, PD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fused_mixed3_ct_kernel<N, RA, RB, RC, T, MINB, PD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fused_mixed3_ct_tma_kernel<N, RA, RB, RC, T, MINB, PD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    return e;
}

struct Spec {
    int n, ra, rb, rc, t, minb;
    mixed3_fn launch;
    mixed3_dft_fn launch_dft;
    mixed3_ct_fn launch_ct;
    cudaError_t (*attr)();
};
#define SAR_SPEC(N, RA, RB, RC, T, MB, PD)                                                                 \
    Spec{N, RA, RB, RC, T, MB, &launch3<N, RA, RB, RC, T, MB, PD>, &launch3_dft<N, RA, RB, RC, T, MB, PD>,  \
         &launch3_ct<N, RA, RB, RC, T, MB, PD>, &attr3<N, RA, RB, RC, T, MB, PD>}

}  // namespace mixed
}  // namespace sar
