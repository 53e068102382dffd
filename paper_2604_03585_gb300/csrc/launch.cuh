// Host launchers for the line-engine kernels (included by the per-size
// instantiation units).
#pragma once

#include "persistent.cuh"
#include "streamed.cuh"
#include "registry.h"
#include "tensor_map.h"

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
    if constexpr (SC::MINB > 0) {
        e = cudaFuncSetAttribute(fused_compress_kernel_capped<SC, LPB, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fused_compress_kernel_capped<SC, LPB, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaFuncSetAttribute(fused_compress_kernel<SC, LPB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fused_compress_kernel<SC, LPB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(dft_lines_kernel<SC, LPB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(dft_lines_kernel<SC, LPB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class SC, int LPB>
cudaError_t launch_fused(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                         const float2 *filt, const float2 *tw, const FusedCtl &, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    const int64_t blocks = (n_lines + LPB - 1) / LPB;
    constexpr int smem = smem_bytes_of<SC, LPB>();
    const unsigned grid = (unsigned)blocks, threads = SC::T * LPB;
    if constexpr (SC::MINB > 0) {
        if (valid < SC::N)
            fused_compress_kernel_capped<SC, LPB, true><<<grid, threads, smem, st>>>(in, out, n_lines, ld, valid, filt, tw);
        else
            fused_compress_kernel_capped<SC, LPB, false><<<grid, threads, smem, st>>>(in, out, n_lines, ld, valid, filt, tw);
    } else {
        if (valid < SC::N)
            fused_compress_kernel<SC, LPB, true><<<grid, threads, smem, st>>>(in, out, n_lines, ld, valid, filt, tw);
        else
            fused_compress_kernel<SC, LPB, false><<<grid, threads, smem, st>>>(in, out, n_lines, ld, valid, filt, tw);
    }
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

// --- persistent schedules -----------------------------------------------
template <class SC>
cudaError_t prepare_persistent() {
    constexpr int smem = PersistentLayout<SC>::SMEM_BYTES;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024)
        e = cudaFuncSetAttribute(fused_persistent_kernel<SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return prepare_sched<SC, 1>();   // the plain kernels of the same geometry (ragged lines, FFT)
}

// Resident blocks of the persistent kernel on the whole current device.
template <class SC>
int persistent_grid() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_persistent_kernel<SC>, SC::T,
                                                      PersistentLayout<SC>::SMEM_BYTES);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = per_sm * sms;
    }
    return cached[dev];
}

template <class SC>
cudaError_t launch_persistent(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                              const float2 *filt, const float2 *tw, const FusedCtl &ctl, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (valid < SC::N)   // zero-padded lines take the plain kernel
        return launch_fused<SC, 1>(in, out, n_lines, ld, valid, filt, tw, ctl, st);
    const int resident = persistent_grid<SC>();
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    const int64_t grid = n_lines < resident ? n_lines : resident;
    fused_persistent_kernel<SC><<<(unsigned)grid, SC::T, PersistentLayout<SC>::SMEM_BYTES, st>>>(
        in, out, n_lines, ld, filt, tw, ctl.status, ctl.wait_cycles, ctl.skip_line);
    return cudaGetLastError();
}

template <class SC>
constexpr SchedDesc make_persistent_desc(const char *name) {
    return SchedDesc{name,
                     SC::N,
                     SC::E,
                     SC::R1,
                     SC::R2,
                     SC::R3,
                     1,
                     SC::T,
                     PersistentLayout<SC>::SMEM_BYTES,
                     SC::TW_ELEMS,
                     SC::RL,
                     1,
                     &launch_persistent<SC>,
                     &launch_dft<SC, 1>,
                     &prepare_persistent<SC>,
                     nullptr,
                     0,
                     nullptr};
}

// --- group-streamed schedules ---------------------------------------------
template <class SC, int QL>
constexpr int ct_smem_bytes() {
    return QL * SC::SMEM_ELEMS * (int)sizeof(float2);
}

template <class SC, int LPB, bool ROLL, int QL>
cudaError_t prepare_streamed() {
    constexpr int smem = smem_bytes_of<SC, LPB>();
    cudaError_t e;
    if (smem > 48 * 1024) {
        if constexpr (SC::MINB > 0)
            e = cudaFuncSetAttribute(fused_streamed_kernel_capped<SC, LPB, ROLL>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        else
            e = cudaFuncSetAttribute(fused_streamed_kernel<SC, LPB, ROLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
        if (e != cudaSuccess) return e;
    }
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(fused_seg_kernel<SC, LPB, ROLL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fused_seg_kernel<SC, LPB, ROLL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
    }
    if constexpr (QL > 0) {
        if (ct_smem_bytes<SC, QL>() > 48 * 1024) {
            e = cudaFuncSetAttribute(fused_range_ct_kernel<SC, QL, ROLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     ct_smem_bytes<SC, QL>());
            if (e != cudaSuccess) return e;
        }
    }
    if constexpr (QL < 0) {   // cluster fold: one line of shared memory per block
        constexpr int QC = -QL;
        if (smem_bytes_of<SC, 1>() > 48 * 1024) {
            e = cudaFuncSetAttribute(fused_range_ct_cluster_kernel<SC, QC, ROLL>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes_of<SC, 1>());
            if (e != cudaSuccess) return e;
        }
        if (QC > 8) {
            e = cudaFuncSetAttribute(fused_range_ct_cluster_kernel<SC, QC, ROLL>,
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        if constexpr (ct_tma_ok<SC, QC, ROLL>()) {
            if (smem_bytes_of<SC, 1>() > 48 * 1024) {
                e = cudaFuncSetAttribute(fused_range_ct_tma_kernel<SC, QC, ROLL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes_of<SC, 1>());
                if (e != cudaSuccess) return e;
            }
        }
    }
    return prepare_sched<SC, 1>();
}

template <class SC, int LPB, bool ROLL>
cudaError_t launch_streamed(const float2 *in, float2 *out, int64_t n_lines, int64_t ld, int valid,
                            const float2 *filt, const float2 *tw, const FusedCtl &ctl, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (valid < SC::N) return launch_fused<SC, 1>(in, out, n_lines, ld, valid, filt, tw, ctl, st);
    const int64_t blocks = (n_lines + LPB - 1) / LPB;
    if constexpr (SC::MINB > 0)
        fused_streamed_kernel_capped<SC, LPB, ROLL><<<(unsigned)blocks, SC::T * LPB, smem_bytes_of<SC, LPB>(), st>>>(
            in, out, n_lines, ld, filt, tw);
    else
        fused_streamed_kernel<SC, LPB, ROLL><<<(unsigned)blocks, SC::T * LPB, smem_bytes_of<SC, LPB>(), st>>>(
            in, out, n_lines, ld, filt, tw);
    return cudaGetLastError();
}

template <class SC, bool ROLL, int QL>
cudaError_t launch_range_ct(const float2 *in, float2 *img, int64_t n_lines, int64_t ld_in, int64_t ld_img,
                            const float2 *filt, const float2 *tw, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (n_lines % QL) return cudaErrorInvalidValue;
    fused_range_ct_kernel<SC, QL, ROLL><<<(unsigned)(n_lines / QL), SC::T * QL, ct_smem_bytes<SC, QL>(), st>>>(
        in, img, n_lines, ld_in, ld_img, filt, tw);
    return cudaGetLastError();
}

template <class SC, int QC, bool ROLL>
cudaError_t launch_range_ct_cluster(const float2 *in, float2 *img, int64_t n_lines, int64_t ld_in, int64_t ld_img,
                                    const float2 *filt, const float2 *tw, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (n_lines % QC) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_lines, 1, 1);
    cfg.blockDim = dim3(SC::T, 1, 1);
    cfg.dynamicSmemBytes = smem_bytes_of<SC, 1>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = QC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (ct_tma_ok<SC, QC, ROLL>()) {
        CUtensorMap m;
        if (image_tensor_map(&m, img, n_lines, SC::N, ld_img, 1, 256))
            return cudaLaunchKernelEx(&cfg, fused_range_ct_tma_kernel<SC, QC, ROLL>, in, img, m, ld_in, ld_img, filt,
                                      tw);
    }
    return cudaLaunchKernelEx(&cfg, fused_range_ct_cluster_kernel<SC, QC, ROLL>, in, img, ld_in, ld_img, filt, tw);
}

template <class SC, int LPB, bool ROLL>
cudaError_t launch_seg(const Seg *segs, const int64_t *line_begin, int n_seg, int64_t n_lines, bool ragged,
                       const float2 *filt, const float2 *tw, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_lines + LPB - 1) / LPB);
    if (ragged)
        fused_seg_kernel<SC, LPB, ROLL, true><<<blocks, SC::T * LPB, smem_bytes_of<SC, LPB>(), st>>>(
            segs, line_begin, n_seg, n_lines, filt, tw);
    else
        fused_seg_kernel<SC, LPB, ROLL, false><<<blocks, SC::T * LPB, smem_bytes_of<SC, LPB>(), st>>>(
            segs, line_begin, n_seg, n_lines, filt, tw);
    return cudaGetLastError();
}

// QL > 0: fold with QL lines per block; QL < 0: fold with clusters of -QL blocks
template <class SC, int LPB, bool ROLL, int QL = 0>
constexpr SchedDesc make_streamed_desc(const char *name) {
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
                     0,
                     &launch_streamed<SC, LPB, ROLL>,
                     &launch_dft<SC, 1>,
                     &prepare_streamed<SC, LPB, ROLL, QL>,
                     QL > 0 ? &launch_range_ct<SC, ROLL, (QL > 0 ? QL : 2)>
                            : (QL < 0 ? &launch_range_ct_cluster<SC, (QL < 0 ? -QL : 4), ROLL> : nullptr),
                     QL > 0 ? QL : -QL,
                     &launch_seg<SC, LPB, ROLL>};
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
                     0,
                     &launch_fused<SC, LPB>,
                     &launch_dft<SC, LPB>,
                     &prepare_sched<SC, LPB>,
                     nullptr,
                     0,
                     nullptr};
}

}  // namespace sar
