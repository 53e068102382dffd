// The mixed-radix fused kernel with registers capped for 2 blocks per SM.
#include "mixed_radix.cuh"

namespace sar {
namespace mixed {
cudaError_t launch_k2(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt,
                      const float2* tw, const MixedGeom& g, int lines_per_block, int smem, cudaStream_t st) {
    return launch_kernel<2>(in, out, n_lines, ld, filt, tw, g, lines_per_block, smem, st);
}
cudaError_t set_smem_k2(int bytes) { return set_smem<2>(bytes); }
}  // namespace mixed
}  // namespace sar
