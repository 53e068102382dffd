// Host launchers for the line-engine kernels (included by the per-size
// instantiation units).
#pragma once

#include "line_engine.cuh"
#include "registry.h"

namespace sar {

template <class SC, int LPB>
constexpr int smem_bytes_of() {
    return LPB * SC::SMEM_ELEMS * (int)sizeof(float2);
}

template <class SC, int LPB>
cudaError_t prepare_sched() {
    constexpr int smem = smem_bytes_of<SC, LPB>();
    if (smem <= 48 * 1024) return cudaSuccess;
    cudaError_t e;
    e = cudaFuncSetAttribute(fused_compress_kernel<SC, LPB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fused_compress_kernel<SC, LPB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(dft_lines_kernel<SC, LPB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(dft_lines_kernel<SC, LPB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class SC, int LPB>
cudaError_t launch_fused(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                         const float2 *filt, const float2 *tw, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    const int64_t blocks = (n_lines + LPB - 1) / LPB;
    constexpr int smem = smem_bytes_of<SC, LPB>();
    if (valid < SC::N)
        fused_compress_kernel<SC, LPB, true><<<(unsigned)blocks, SC::T * LPB, smem, st>>>(in, out, n_lines, ld, valid,
                                                                                         filt, tw);
    else
        fused_compress_kernel<SC, LPB, false><<<(unsigned)blocks, SC::T * LPB, smem, st>>>(in, out, n_lines, ld, valid,
                                                                                          filt, tw);
    return cudaGetLastError();
}

template <class SC, int LPB>
cudaError_t launch_dft(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid, const float2 *tw,
                       int inverse, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    const int64_t blocks = (n_lines + LPB - 1) / LPB;
    constexpr int smem = smem_bytes_of<SC, LPB>();
    if (inverse)
        dft_lines_kernel<SC, LPB, true><<<(unsigned)blocks, SC::T * LPB, smem, st>>>(in, out, n_lines, ld, valid, tw);
    else
        dft_lines_kernel<SC, LPB, false><<<(unsigned)blocks, SC::T * LPB, smem, st>>>(in, out, n_lines, ld, valid, tw);
    return cudaGetLastError();
}

template <class SC, int LPB>
constexpr SchedDesc make_desc(const char *name) {
    return SchedDesc{name,
                     SC::N,
                     SC::E,
                     SC::R1,
                     SC::R2,
                     SC::R3,
                     LPB,
                     SC::T * LPB,
                     smem_bytes_of<SC, LPB>(),
                     SC::TW_ELEMS,
                     SC::RL,
                     &launch_fused<SC, LPB>,
                     &launch_dft<SC, LPB>,
                     &prepare_sched<SC, LPB>};
}

}  // namespace sar
