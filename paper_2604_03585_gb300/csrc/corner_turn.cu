// Corner turn (Sec. IV-A step 2 / Sec. IV-B of the paper: the global
// transpose that turns azimuth columns into rows): out[c][r] = in[r][c].
//
// Tiled through shared memory so that both the HBM reads and the HBM writes
// are coalesced: a block moves a 32 x 32 tile of complex64; each warp reads
// 256 contiguous bytes of a source row and writes 256 contiguous bytes of a
// destination row.  The tile is padded to 33 columns so that the column-wise
// shared-memory reads hit distinct banks (element stride 33 = 1 mod 16).
// Pure data movement: bit-exact.
#include "tables.h"

namespace sar {

constexpr int kTile = 32;
constexpr int kRowsPerPass = 8;   // block = 32 x 8 threads, 4 elements each way

__global__ void __launch_bounds__(kTile * kRowsPerPass)
corner_turn_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, int64_t rows, int64_t cols,
                   int64_t tiles_c) {
    __shared__ float2 tile[kTile][kTile + 1];
    const int64_t tr = blockIdx.x / tiles_c;           // tile row (over `rows`)
    const int64_t tc = blockIdx.x % tiles_c;           // tile column (over `cols`)
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int64_t r0 = tr * kTile, c0 = tc * kTile;
    const bool full = (r0 + kTile <= rows) && (c0 + kTile <= cols);
#pragma unroll
    for (int j = 0; j < kTile; j += kRowsPerPass) {
        const int64_t r = r0 + ty + j, c = c0 + tx;
        if (full || (r < rows && c < cols)) tile[ty + j][tx] = in[r * cols + c];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kTile; j += kRowsPerPass) {
        const int64_t c = c0 + ty + j, r = r0 + tx;       // destination row c, column r
        if (full || (r < rows && c < cols)) out[c * rows + r] = tile[tx][ty + j];
    }
}

cudaError_t launch_transpose(const float2 *in, float2 *out, int64_t rows, int64_t cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int64_t tiles_r = (rows + kTile - 1) / kTile, tiles_c = (cols + kTile - 1) / kTile;
    const int64_t blocks = tiles_r * tiles_c;
    corner_turn_kernel<<<(unsigned)blocks, kTile * kRowsPerPass, 0, st>>>(in, out, rows, cols, tiles_c);
    return cudaGetLastError();
}

}  // namespace sar
