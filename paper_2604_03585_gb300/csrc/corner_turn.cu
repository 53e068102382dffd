// Corner turn (Sec. IV-A step 2 / Sec. IV-B of the paper: the global
// transpose that turns azimuth columns into rows): out[c][r] = in[r][c].
//
// Tiled through shared memory so that both the HBM reads and the HBM writes
// are coalesced: a block moves a 32 x 32 tile of complex64; each warp reads
// 256 contiguous bytes of a source row and writes 256 contiguous bytes of a
// destination row.  The tile is padded to 33 columns so that the column-wise
// shared-memory reads hit distinct banks (element stride 33 = 1 mod 16).
// Pure data movement: bit-exact.
#include <atomic>

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

// Fast path for the scene shapes (rows and cols multiples of 64): a block
// moves a 64 x 64 tile (32 KiB).  Every global access is 16 bytes (two
// complex64) and every warp touches 512 contiguous bytes; the transpose of
// each 2 x 2 block of samples happens in registers, so shared memory is read
// and written in 16-byte chunks only.  Chunk j of tile row r sits at chunk
// r*32 + (j ^ ((r >> 1) & 7)): both the row-wise writes and the paired-row
// reads of a warp hit eight distinct bank groups per 128-byte phase.
constexpr int kBig = 64;

__device__ __forceinline__ int ct_chunk(int r, int j) { return r * 32 + (j ^ ((r >> 1) & 7)); }

__global__ void __launch_bounds__(256)
corner_turn64_kernel(const float4 *__restrict__ in, float4 *__restrict__ out, int64_t rows, int64_t cols,
                     int64_t tiles_c) {
    __shared__ float4 tile[kBig * 32];                 // 64 rows x 32 chunks of 16 B
    const int64_t tr = blockIdx.x / tiles_c, tc = blockIdx.x % tiles_c;
    const int64_t r0 = tr * kBig, c0 = tc * kBig;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cols2 = cols / 2, rows2 = rows / 2;  // rows of 16-byte chunks
    // load: warp w reads tile rows w, w+8, ..., one 512-byte row per instruction
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int r = warp + 8 * k;
        tile[ct_chunk(r, lane)] = in[(r0 + r) * cols2 + c0 / 2 + lane];
    }
    __syncthreads();
    // store: warp w writes output rows c = 2*(w + 8k) and c + 1; lane l covers
    // input rows 2l and 2l + 1 of the tile
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = warp + 8 * k;                    // chunk = columns 2j, 2j+1 of the tile
        const float4 a = tile[ct_chunk(2 * lane, j)];      // (r, c), (r, c+1)
        const float4 b = tile[ct_chunk(2 * lane + 1, j)];  // (r+1, c), (r+1, c+1)
        const int64_t c = c0 + 2 * j;
        out[c * rows2 + r0 / 2 + lane] = make_float4(a.x, a.y, b.x, b.y);
        out[(c + 1) * rows2 + r0 / 2 + lane] = make_float4(a.z, a.w, b.z, b.w);
    }
}

namespace {
std::atomic<int> g_ct_variant{0};
}

void set_corner_turn_variant(int v) { g_ct_variant.store(v); }
int corner_turn_variant() { return g_ct_variant.load(); }

cudaError_t launch_transpose(const float2 *in, float2 *out, int64_t rows, int64_t cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int variant = g_ct_variant.load(std::memory_order_relaxed);
    if (variant != 1 && rows % kBig == 0 && cols % kBig == 0 && ((uintptr_t)in & 15) == 0 &&
        ((uintptr_t)out & 15) == 0 && variant == 2) {
        const int64_t tiles_c = cols / kBig, blocks = (rows / kBig) * tiles_c;
        corner_turn64_kernel<<<(unsigned)blocks, 256, 0, st>>>((const float4 *)in, (float4 *)out, rows, cols,
                                                                tiles_c);
        return cudaGetLastError();
    }
    const int64_t tiles_r = (rows + kTile - 1) / kTile, tiles_c = (cols + kTile - 1) / kTile;
    const int64_t blocks = tiles_r * tiles_c;
    corner_turn_kernel<<<(unsigned)blocks, kTile * kRowsPerPass, 0, st>>>(in, out, rows, cols, tiles_c);
    return cudaGetLastError();
}

}  // namespace sar
