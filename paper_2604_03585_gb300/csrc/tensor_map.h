// Host-side encoding of the TMA tensor maps the folded range passes store
// their image tiles through.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace sar {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr where the driver does not offer it
typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline encode_tiled_fn encode_tiled() {
    static const encode_tiled_fn f = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (encode_tiled_fn) nullptr;
        return (encode_tiled_fn)p;
    }();
    return f;
}

// Image columns [0, n_lines) of n_rows rows, ld_img complex apart, as a
// tensor of fp32 pairs split into `planes` planes of n_rows / planes rows
// (one per block of a folding cluster; a box that runs past its plane's last
// row is clipped there), boxes of 4 complex x box_rows rows.  False where a
// tensor map cannot describe it (base not 16-byte aligned, odd row pitch, no
// encoder).
inline bool image_tensor_map(CUtensorMap *m, void *img, int64_t n_lines, int64_t n_rows, int64_t ld_img, int planes,
                             int box_rows) {
    const encode_tiled_fn enc = encode_tiled();
    if (!enc || ((uintptr_t)img & 15) || ld_img % 2 || n_rows % planes) return false;
    const int64_t rows = n_rows / planes;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * n_lines), (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)ld_img * 8, (cuuint64_t)(rows * ld_img * 8)};
    const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, 1}, es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, img, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace sar
