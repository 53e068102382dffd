// A ragged batch in one persistent launch.
//
// Every strip of the batch is two sets of line items: range items (k
// consecutive azimuth rows of the raw echo, compressed along range and
// written straight into the corner-turned image) and azimuth items (k
// consecutive range bins of the image, compressed along azimuth in place).
// One block per SM stays resident and takes items from a single list through
// an atomic counter.  An item holds 16384 samples' worth of lines (8192 at
// length 256): the block's 512 threads split into k groups of T = n / E
// threads, one line each, each group running the group-streamed engine of
// its length with its own named barrier, so one kernel serves every length
// from 256 to 16384 with the register and shared-memory footprint of one
// 16384-sample line.
//
// Corner turn: the k lines of a range item are consecutive azimuth rows, so
// after their inverse transforms (natural order, in shared memory) the block
// writes each range bin's k samples as one k*8-byte run of its image row
// (32 bytes at n_range = 4096, 128 at 1024): the separate transpose and its
// 16 bytes per sample of HBM traffic disappear, without clusters.
//
// Latency: with one block per SM nothing else hides an item's HBM loads, so
// the block that takes item i asks L2 for the rows of item i + gridDim.x
// (one bulk prefetch), which it or a neighbour takes about one item later.
//
// Dependencies: an azimuth item of strip s reads whole image rows, which
// every range item of s writes into.  Range items count their finished lines
// in done[s] (all stores of the block, a block barrier, a device-scope fence,
// then the atomic add); an azimuth item's first thread waits, with an
// acquire load, until done[s] reaches the strip's n_az, and the block reads
// the rows through L2 only (ld.global.cg).  The host orders the list range
// items of strip s + 1 before the azimuth items of strip s, so an item only
// ever waits for items that earlier blocks already took; all blocks are
// resident (one per SM), so those items are being computed and the wait
// ends.  It is bounded all the same: after `wait_cycles` SM clocks the block
// sets *status to 5 (timeout), and every block stops taking items once
// *status is set.  No block waits for another one to start.
#include "batch_persistent.h"
#include "line_engine.cuh"
#include "streamed.cuh"

namespace sar {

namespace {

// the line engines of the batch kernel: E = 32 (E = 16 at n = 256) samples
// per thread, the default geometry of every length
using B256 = Sched<256, 16, 16, 16>;
using B512 = Sched<512, 32, 16, 32>;
using B1024 = Sched<1024, 32, 32, 32>;
using B2048 = Sched<2048, 32, 16, 8, 16>;
using B4096 = Sched<4096, 32, 16, 16, 16>;
using B8192 = Sched<8192, 32, 16, 32, 16>;
using B16384 = Sched<16384, 32, 16, 32, 32>;

// k lines per item and the stride of their shared-memory buffers: one line's
// padded exchange layout plus a shift of 16/k bank pairs (1 for k >= 16), so
// that the transposed store's reads of the k lines at one range bin (k lanes
// of a half-warp) hit distinct bank pairs.  A uniform shift of a line's
// buffer leaves the passes' own access patterns conflict-free.
template <class SC>
struct BGeo {
    static constexpr int K = kBatchThreads / SC::T;
    static_assert(K >= 1 && K * SC::T == kBatchThreads, "lines fill the block");
    static constexpr int SHIFT = K >= 16 ? 1 : 16 / K;
    static constexpr int BS = SC::SMEM_ELEMS + SHIFT;
    static constexpr int SMEM_BYTES = K * BS * (int)sizeof(float2);
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kSmem =
    cmax(cmax(cmax(BGeo<B256>::SMEM_BYTES, BGeo<B512>::SMEM_BYTES), cmax(BGeo<B1024>::SMEM_BYTES, BGeo<B2048>::SMEM_BYTES)),
         cmax(cmax(BGeo<B4096>::SMEM_BYTES, BGeo<B8192>::SMEM_BYTES), BGeo<B16384>::SMEM_BYTES));

// Inverse pass 1 of group-streamed line `lib`: shared memory -> conjugate
// twiddles -> inverse DFT; emit(lo, x) receives natural-order samples
// lo + r*S1.
template <class SC, class Emit>
__device__ __forceinline__ void b_inverse_pass1(const float2* sm, const float2* tw, int t, Emit&& emit) {
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
#pragma unroll 1
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
        emit(lo, x);
    }
}

// Range item: lines line0 .. line0 + nlines - 1 (azimuth rows) of the strip,
// compressed along range and stored transposed into the image.  The item
// routines are not inlined, so that each length gets its own register
// allocation under the block's 128-register budget.
template <class SC>
__device__ __noinline__ void range_item(const BStrip& st, int line0, int nlines, float2* smem) {
    using G = BGeo<SC>;
    constexpr int R1 = SC::R1, S1 = SC::S1;
    const int lib = threadIdx.x / SC::T, t = threadIdx.x % SC::T;
    float2* sm = smem + lib * G::BS;
    if (lib < nlines) {
        const float2* src = st.raw + (int64_t)(line0 + lib) * SC::N;
        streamed_until_last<SC, G::K, true>(src, sm, st.filt_r, st.tw_r, t, lib);
        // natural-order results back into the slots they were read from
        b_inverse_pass1<SC>(sm, st.tw_r, t, [&](int lo, const float2 (&x)[R1]) {
#pragma unroll
            for (int r = 0; r < R1; ++r) sm[smem_pos(lo + r * S1, SC::PADSH)] = x[r];
        });
    }
    __syncthreads();
    // range bin n of the k lines -> image[n][line0 .. line0 + nlines - 1]
    for (int idx = threadIdx.x; idx < SC::N * G::K; idx += kBatchThreads) {
        const int n = idx / G::K, q = idx % G::K;
        if (q < nlines)
            __stcs(st.image + (int64_t)n * st.n_az + line0 + q, smem[q * G::BS + smem_pos(n, SC::PADSH)]);
    }
}

// Azimuth item: range bins line0 .. line0 + nlines - 1 of the image,
// compressed along azimuth in place (transform length l_az, the n_az stored
// samples zero-padded).
template <class SC, bool RAGGED>
__device__ __noinline__ void az_item(const BStrip& st, int line0, int nlines, float2* smem) {
    using G = BGeo<SC>;
    constexpr int R1 = SC::R1, S1 = SC::S1;
    const int lib = threadIdx.x / SC::T, t = threadIdx.x % SC::T;
    float2* sm = smem + lib * G::BS;
    if (lib < nlines) {
        float2* row = st.image + (int64_t)(line0 + lib) * st.n_az;
        const int valid = st.n_az;
        streamed_until_last<SC, G::K, true, RAGGED, true>(row, sm, st.filt_a, st.tw_a, t, lib, valid);
        b_inverse_pass1<SC>(sm, st.tw_a, t, [&](int lo, const float2 (&x)[R1]) {
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int i = lo + r * S1;
                if (!RAGGED || i < valid) __stcs(row + i, x[r]);
            }
        });
    }
}

// one routine per length: lines of n_az = l_az samples take the zero-padding
// path with nothing to pad (one compare per load, one code path per length)
template <class SC>
__device__ __forceinline__ void az_item_any(const BStrip& st, int line0, int nlines, float2* smem) {
    az_item<SC, true>(st, line0, nlines, smem);
}

// Bounded wait of one thread for *ctr >= expect (acquire); false when the
// bound ran out or another block recorded a failure.
__device__ __forceinline__ bool wait_count(const int* ctr, int expect, const int* status, long long wait_cycles) {
    const long long t0 = clock64();
    for (;;) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= expect) return true;
        if (*(volatile const int*)status != 0) return false;
        if (clock64() - t0 > wait_cycles) return false;
        __nanosleep(200);
    }
}

// Bulk L2 prefetch of [p, p + bytes) clipped to whole 16-byte units inside
// the range (the instruction needs a 16-byte-aligned address and size).
__device__ __forceinline__ void prefetch_l2_range(const void* p, int64_t bytes) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + (uintptr_t)bytes) & ~(uintptr_t)15;
    for (uintptr_t q = a; q < e; q += 65536) {
        const uint32_t n = (uint32_t)((e - q) < 65536 ? (e - q) : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}

// The lines item `it` reads: raw rows of a range item, image rows of an
// azimuth item (both contiguous runs).
__device__ __forceinline__ void prefetch_item(const BItem& it, const BStrip& st) {
    if (it.kind == 0)
        prefetch_l2_range(st.raw + (int64_t)it.line0 * st.n_range, (int64_t)it.nlines * st.n_range * 8);
    else
        prefetch_l2_range(st.image + (int64_t)it.line0 * st.n_az, (int64_t)it.nlines * st.n_az * 8);
}

__global__ void __launch_bounds__(kBatchThreads, 1)
batch_persistent_kernel(const BItem* items, int n_items, const BStrip* strips, int* done, int* next, int* status,
                        long long wait_cycles) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ int s_item, s_go;
    for (;;) {
        if (threadIdx.x == 0) {
            int go = *(volatile int*)status == 0;
            const int i = go ? atomicAdd(next, 1) : n_items;
            // the item about one round of all blocks ahead: most likely the
            // next one this block (or a neighbour) takes
            const int j = i + (int)gridDim.x;
            if (go && j < n_items) prefetch_item(items[j], strips[items[j].strip]);
            if (i < n_items && items[i].kind == 1) {
                const BStrip& st = strips[items[i].strip];
                if (!wait_count(done + items[i].strip, st.expect, status, wait_cycles)) {
                    atomicMax(status, 5);
                    go = 0;
                }
            }
            s_item = i;
            s_go = go && i < n_items;
        }
        __syncthreads();
        if (!s_go) break;
        const BItem it = items[s_item];
        const BStrip st = strips[it.strip];
        if (it.kind == 0) {
            switch (st.n_range) {
                case 256: range_item<B256>(st, it.line0, it.nlines, smem); break;
                case 512: range_item<B512>(st, it.line0, it.nlines, smem); break;
                case 1024: range_item<B1024>(st, it.line0, it.nlines, smem); break;
                case 2048: range_item<B2048>(st, it.line0, it.nlines, smem); break;
                case 4096: range_item<B4096>(st, it.line0, it.nlines, smem); break;
                case 8192: range_item<B8192>(st, it.line0, it.nlines, smem); break;
                default: range_item<B16384>(st, it.line0, it.nlines, smem); break;
            }
            __syncthreads();   // every store of the item is issued
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(done + it.strip, it.nlines);
            }
        } else {
            switch (st.l_az) {
                case 256: az_item_any<B256>(st, it.line0, it.nlines, smem); break;
                case 512: az_item_any<B512>(st, it.line0, it.nlines, smem); break;
                case 1024: az_item_any<B1024>(st, it.line0, it.nlines, smem); break;
                case 2048: az_item_any<B2048>(st, it.line0, it.nlines, smem); break;
                case 4096: az_item_any<B4096>(st, it.line0, it.nlines, smem); break;
                case 8192: az_item_any<B8192>(st, it.line0, it.nlines, smem); break;
                default: az_item_any<B16384>(st, it.line0, it.nlines, smem); break;
            }
        }
        __syncthreads();   // the next item overwrites the shared memory and s_item
    }
}

}  // namespace

int batch_lines_per_item(int n) {
    switch (n) {
        case 256: return BGeo<B256>::K;
        case 512: return BGeo<B512>::K;
        case 1024: return BGeo<B1024>::K;
        case 2048: return BGeo<B2048>::K;
        case 4096: return BGeo<B4096>::K;
        case 8192: return BGeo<B8192>::K;
        case 16384: return BGeo<B16384>::K;
        default: return 0;
    }
}

const char *batch_schedule_name(int n) {
    switch (n) {
        case 256: return "n256_e16_r16x16_l8";
        case 512: return "n512_e32_r16x32_l8";
        case 1024: return "n1024_e32_r32x32_l4";
        case 2048: return "n2048_e32_r16x8x16_sr2";
        case 4096: return "n4096_e32_r16x16x16_sr1";
        case 8192: return "n8192_e32_r16x32x16_sr1";
        case 16384: return "n16384_e32_r16x32x32_sr1";
        default: return nullptr;
    }
}

int batch_smem_bytes() { return kSmem; }

cudaError_t prepare_batch_persistent() {
    return cudaFuncSetAttribute(batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

int batch_grid() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, kBatchThreads, kSmem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            return 0;
        }
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = per_sm * sms;
    }
    return cached[dev];
}

cudaError_t launch_batch_persistent(const BItem *items, int n_items, const BStrip *strips, int *done, int *next,
                                    int *status, long long wait_cycles, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const int grid = batch_grid();
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    batch_persistent_kernel<<<(unsigned)(grid < n_items ? grid : n_items), kBatchThreads, kSmem, st>>>(
        items, n_items, strips, done, next, status, wait_cycles);
    return cudaGetLastError();
}

}  // namespace sar
