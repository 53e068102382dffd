// Group-streamed variant of the fused line compression.
//
// Same arithmetic and the same in-place shared-memory geometry as
// fused_compress_kernel (line_engine.cuh), but each pass is executed one
// radix group at a time: load the group's R values (from HBM in the first
// pass, from shared memory otherwise), transform, twiddle, write them back.
// Only one group is live in registers, so a thread that owns several groups
// per pass needs about R complex registers instead of E, and with ROLL the
// loop over groups is not unrolled, which halves the code a warp streams
// through the instruction cache.  In the first pass the next group's HBM
// loads are issued before the current group is transformed, so their latency
// overlaps the arithmetic.
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>

#include "line_engine.cuh"

namespace sar {

template <int R, int S>
__device__ __forceinline__ void grp_smem_load(const float2* sm, int base, int padsh, float2 (&g)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) g[r] = sm[smem_pos(base + r * S, padsh)];
}
template <int R, int S>
__device__ __forceinline__ void grp_smem_store(float2* sm, int base, int padsh, const float2 (&g)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) sm[smem_pos(base + r * S, padsh)] = g[r];
}
template <int R, int S, bool INV>
__device__ __forceinline__ void grp_twiddle(const float2* tw, int lo, float2 (&g)[R]) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * S + lo];
        g[r] = INV ? cmulc(g[r], w) : cmul(g[r], w);
    }
}

// One middle pass (shared memory in, shared memory out) of radix R, stride S.
// FWD: DFT then twiddle; inverse: conjugate twiddle then inverse DFT.
template <class SC, int R, int S, bool INV, bool ROLL>
__device__ __forceinline__ void streamed_mid_pass(float2* sm, const float2* tw, int t) {
    constexpr int G = SC::E / R;
#pragma unroll(ROLL ? 1 : G)
    for (int s = 0; s < G; ++s) {
        const int g = t + SC::T * s;
        const int base = group_base<R, S>(g);
        float2 x[R];
        grp_smem_load<R, S>(sm, base, SC::PADSH, x);
        if (!INV) {
            dft_reg<R, false>(x);
            grp_twiddle<R, S, false>(tw, group_lo<R, S>(g), x);
        } else {
            grp_twiddle<R, S, true>(tw, group_lo<R, S>(g), x);
            dft_reg<R, true>(x);
        }
        grp_smem_store<R, S>(sm, base, SC::PADSH, x);
    }
}

// Everything of the fused line compression except the last inverse pass:
// pass 1 from HBM, the middle passes, the last forward pass with the filter
// multiply and the first inverse pass, and the inverse middle passes.  On
// return the line sits in shared memory ready for the inverse pass 1.
// Element i of a line that holds `valid` stored samples (zero beyond them:
// a zero-padded transform of a ragged line).
// Line samples are read once: streaming loads (evict-first), so that they
// do not push the twiddle and filter tables out of L1.  With L2ONLY the loads
// bypass L1 (ld.global.cg): for data that other SMs wrote earlier in the same
// launch, where an L1 line cached before the write could be stale.
template <bool RAGGED, bool L2ONLY = false>
__device__ __forceinline__ float2 line_at(const float2* src, int i, int valid) {
    if constexpr (RAGGED) {
        if (i >= valid) return make_float2(0.f, 0.f);
    }
    if constexpr (L2ONLY)
        return __ldcg(src + i);
    else
        return __ldcs(src + i);
}

template <class SC, int LPB, bool ROLL, bool RAGGED = false, bool L2ONLY = false>
__device__ __forceinline__ void streamed_until_last(const float2* src, float2* sm, const float2* filt,
                                                    const float2* tw, int t, int lib, int valid = SC::N) {
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    constexpr int RL = SC::RL, GL = SC::E / RL;

    // ---- forward pass 1: HBM -> DFT -> twiddle -> shared memory, with the
    //      next group's loads in flight during the current group's arithmetic
    float2 cur[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) cur[r] = line_at<RAGGED, L2ONLY>(src, t + r * S1, valid);
#pragma unroll(ROLL ? 1 : G1)
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 nxt[R1];
        if (s + 1 < G1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) nxt[r] = line_at<RAGGED, L2ONLY>(src, lo + SC::T + r * S1, valid);
        }
        dft_reg<R1, false>(cur);
        grp_twiddle<R1, S1, false>(tw, lo, cur);
        grp_smem_store<R1, S1>(sm, lo, SC::PADSH, cur);
        if (s + 1 < G1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) cur[r] = nxt[r];
        }
    }
    line_sync<SC, LPB>(lib);
    const float2* tw2 = tw + SC::R1 * SC::S1;
    if constexpr (SC::P == 3) {
        streamed_mid_pass<SC, SC::R2, SC::S2, false, ROLL>(sm, tw2, t);
        line_sync<SC, LPB>(lib);
    }
    // ---- last forward pass, filter, first inverse pass: one group at a time
#pragma unroll(ROLL ? 1 : GL)
    for (int s = 0; s < GL; ++s) {
        const int g = t + SC::T * s;
        float2 x[RL];
        grp_smem_load<RL, 1>(sm, g * RL, SC::PADSH, x);
        dft_reg<RL, false>(x);
#pragma unroll
        for (int r = 0; r < RL; ++r) x[r] = cmul(x[r], filt[(s * RL + r) * SC::T + t]);
        dft_reg<RL, true>(x);
        grp_smem_store<RL, 1>(sm, g * RL, SC::PADSH, x);
    }
    line_sync<SC, LPB>(lib);
    if constexpr (SC::P == 3) {
        streamed_mid_pass<SC, SC::R2, SC::S2, true, ROLL>(sm, tw2, t);
        line_sync<SC, LPB>(lib);
    }
}

template <class SC, int LPB, bool ROLL>
__device__ __forceinline__ void fused_streamed_body(const float2* in, float2* out, int64_t n_lines, int64_t ld,
                                                    const float2* filt, const float2* tw) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    if (line >= n_lines) return;
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    float2* dst = out + line * ld;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    streamed_until_last<SC, LPB, ROLL>(in + line * ld, sm, filt, tw, t, lib);
    // ---- inverse pass 1: shared memory -> twiddle -> inverse DFT -> HBM
#pragma unroll(ROLL ? 1 : G1)
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
#pragma unroll
        for (int r = 0; r < R1; ++r) __stcs(dst + lo + r * S1, x[r]);
    }
}

// Fused line compression over a table of segments (a ragged batch): segment
// k covers lines [line_begin[k], line_begin[k+1]) of the launch; its line j
// is read from in + j*ld_in (valid samples, zero-padded to N) and written to
// out + j*ld_out (the first `valid` samples).  Every line finds its segment
// by binary search over the prefix sums.
struct Seg {
    const float2* in;
    float2* out;
    int64_t ld_in, ld_out;
    int32_t valid, pad;
};

__device__ __forceinline__ int find_seg(const int64_t* line_begin, int n_seg, int64_t g) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (line_begin[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class SC, int LPB, bool ROLL, bool RAGGED>
__global__ void __launch_bounds__(SC::T * LPB)
fused_seg_kernel(const Seg* segs, const int64_t* line_begin, int n_seg, int64_t n_lines, const float2* filt,
                 const float2* tw) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t g = (int64_t)blockIdx.x * LPB + lib;
    if (g >= n_lines) return;
    const int k = find_seg(line_begin, n_seg, g);
    const Seg sg = segs[k];
    const int64_t j = g - line_begin[k];
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    float2* dst = sg.out + j * sg.ld_out;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    streamed_until_last<SC, LPB, ROLL, RAGGED>(sg.in + j * sg.ld_in, sm, filt, tw, t, lib, sg.valid);
#pragma unroll(ROLL ? 1 : G1)
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int i = lo + r * S1;
            if (!RAGGED || i < sg.valid) __stcs(dst + i, x[r]);
        }
    }
}

// Range compression with the corner turn folded into its store (the
// paper's Sec. IV-A steps 1 and 2 in one kernel).  A block compresses QL
// consecutive range lines a0 .. a0+QL-1 (QL = 4); after the inverse pass the
// lines are parked in shared memory in natural order and written out
// transposed: range bin n of the QL lines is one QL*8-byte chunk (with QL = 4
// a full 32-byte HBM sector) of image row n, image[n][a0 .. a0+QL-1].  The separate transpose
// kernel and its 16 bytes per sample of HBM traffic disappear.
// Requires n_lines % QL == 0 and 16-byte aligned rows of the image.
template <class SC, int QL, bool ROLL>
__device__ __forceinline__ void fused_range_ct_body(const float2* in, float2* img, int64_t n_lines, int64_t ld_in,
                                                    int64_t ld_img, const float2* filt, const float2* tw) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t a0 = (int64_t)blockIdx.x * QL;
    const int64_t line = a0 + lib;
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    streamed_until_last<SC, QL, ROLL>(in + line * ld_in, sm, filt, tw, t, lib);
    // ---- inverse pass 1 into registers, then natural order into shared memory
    float2 v[SC::E];
#pragma unroll
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
#pragma unroll
        for (int r = 0; r < R1; ++r) v[s * R1 + r] = x[r];
    }
    line_sync<SC, QL>(lib);
#pragma unroll
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < R1; ++r) sm[lo + r * S1] = v[s * R1 + r];
    }
    __syncthreads();
    // ---- transposed store: one QL*8-byte chunk per range bin
    static_assert(QL == 2 || QL == 4, "chunks of two or four complex64");
    for (int n = threadIdx.x; n < SC::N; n += SC::T * QL) {
        float4* dst = reinterpret_cast<float4*>(img + (int64_t)n * ld_img + a0);
        const float2 c0 = smem_dyn[n], c1 = smem_dyn[SC::SMEM_ELEMS + n];
        dst[0] = make_float4(c0.x, c0.y, c1.x, c1.y);
        if constexpr (QL == 4) {
            const float2 c2 = smem_dyn[2 * SC::SMEM_ELEMS + n], c3 = smem_dyn[3 * SC::SMEM_ELEMS + n];
            dst[1] = make_float4(c2.x, c2.y, c3.x, c3.y);
        }
    }
}

// The fold whose image tiles leave through the tensor memory accelerator:
// after the exchange each block rewrites its receive rows bin-major in place
// (bin j's four samples at 32 j bytes) and one thread stores them as boxes
// of 4 azimuth samples x 256 range bins (cp.async.bulk.tensor over the image
// as a one-plane tensor of fp32 pairs, tensor_map.h), in place of 16 rows of
// 32 bytes per warp store instruction.  For clusters of
// four and the rolled E = 32 engines of up to 256 threads (the E / 2 staged
// float4 take the registers of the line; the unrolled and E = 16 engines run
// the plain fold at fewer registers than this one needs, and at 16384 points,
// one 512-thread block per SM, the wait for the bulk reads before exit leaves
// the SM idle: 0.867 ms per 16384 x 4096 scene against 0.837 with plain
// stores), registers capped so that an SM keeps at least 640 threads of
// lines resident, as the plain fold does.
template <class SC>
__host__ __device__ constexpr int ct_tma_min_blocks() {
    return 640 / SC::T > 0 ? 640 / SC::T : 1;
}
template <class SC, int QC, bool ROLL>
__host__ __device__ constexpr bool ct_tma_ok() {
    return QC == 4 && ROLL && SC::E == 32 && SC::T <= 256 && (SC::N / 4) % 256 == 0 &&
           (SC::N / 4 * 2) % SC::T == 0;
}

// The same fold with one line per block and QC blocks per thread-block
// cluster (QC = 4, 8 or 16).  Block q of the cluster compresses line a0 + q;
// block k owns range bins [k N/QC, (k+1) N/QC) of the image rows.  After a
// cluster barrier (every block is done with its shared memory for the FFT)
// each block pushes its line, straight from the registers of the last pass,
// into the owners' shared memory, line-major (recv[q][j], bin j of line q), so
// that a warp's 32 remote stores form one contiguous 256-byte run.  Remote
// stores do not stall the issuing warp.  After a second barrier (every push
// has landed) each block reads its own shared memory and writes each bin's QC
// samples as one QC*8-byte chunk of image row n, image[n][a0 .. a0+QC-1] (two
// lines, 16 bytes, per lane); no block touches another's shared memory after
// that barrier.  A block needs one line of shared memory, not QC, so an SM
// keeps as many lines in flight as the unfolded kernel.  Launched with a
// cluster dimension of QC.
template <class SC, int QC, bool ROLL, bool TMA = false>
__device__ __forceinline__ void fused_range_ct_cluster_body(const float2* in, float2* img, int64_t ld_in,
                                                            int64_t ld_img, const float2* filt,
                                                            const float2* tw, const CUtensorMap* tmap = nullptr) {
    namespace cg = cooperative_groups;
    extern __shared__ float2 smem_dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int t = threadIdx.x;
    const int rank = (int)cluster.block_rank();
    const int64_t line = blockIdx.x;
    const int64_t a0 = line - rank;
    float2* sm = smem_dyn;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    streamed_until_last<SC, 1, ROLL>(in + line * ld_in, sm, filt, tw, t, 0);
    float2 v[SC::E];
#pragma unroll
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
#pragma unroll
        for (int r = 0; r < R1; ++r) v[s * R1 + r] = x[r];
    }
    static_assert(QC == 4 || QC == 8 || QC == 16, "clusters of 4, 8 or 16 lines");
    constexpr int NQ = SC::N / QC;   // range bins owned by one block
    // receive row of each line, padded by 4 slots: in the transposed read
    // below a half-warp reads bins j = 0..7 of rows 2p and 2p + 1 (p = 0, 1);
    // with rows 2 * RS = 8 (mod 16) bank pairs apart they hit 16 distinct
    // bank pairs (unpadded rows NQ apart put p = 0 and p = 1 on the same ones)
    constexpr int RS = NQ + 4;
    static_assert(QC * RS <= SC::SMEM_ELEMS, "the receive rows fit the line buffer");
    cluster.sync();
    // push: natural-order sample i = lo + r S1 of line a0 + rank goes to
    // block i / NQ, slot rank RS + i mod NQ
#pragma unroll
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int i = lo + r * S1;
            float2* dst = cluster.map_shared_rank(sm, i / NQ);
            dst[rank * RS + i % NQ] = v[s * R1 + r];
        }
    }
    cluster.sync();
    if constexpr (TMA) {
        static_assert(ct_tma_ok<SC, QC, ROLL>(), "four lines, whole boxes of 256 bins");
        constexpr int NIT = NQ * 2 / SC::T;
        float4 w[NIT];
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
            const int idx = t + k * SC::T, j = idx >> 1, p = idx & 1;
            const float2 c0 = sm[(2 * p) * RS + j], c1 = sm[(2 * p + 1) * RS + j];
            w[k] = make_float4(c0.x, c0.y, c1.x, c1.y);
        }
        __syncthreads();
        float4* stg = reinterpret_cast<float4*>(sm);   // bin-major: bin j's four samples at stg[2j], stg[2j + 1]
#pragma unroll
        for (int k = 0; k < NIT; ++k) stg[t + k * SC::T] = w[k];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(stg);
        if (base & 127) {   // a tensor copy wants 128-byte aligned shared memory: plain stores
#pragma unroll
            for (int k = 0; k < NIT; ++k) {
                const int idx = t + k * SC::T, j = idx >> 1, p = idx & 1;
                __stcs(reinterpret_cast<float4*>(img + (int64_t)(rank * NQ + j) * ld_img + a0 + 2 * p), w[k]);
            }
            return;
        }
        if (t == 0) {
#pragma unroll
            for (int c = 0; c < NQ / 256; ++c)
                asm volatile(
                    "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(tmap),
                    "r"(base + c * 256 * 32), "r"((int)(2 * a0)), "r"(rank * NQ + c * 256), "r"(0)
                    : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        return;
    }
    constexpr int LPN = QC / 2;   // lanes per bin, 16 bytes (two lines) each
#pragma unroll 4
    for (int idx = t; idx < NQ * LPN; idx += SC::T) {
        const int j = idx / LPN, p = idx % LPN;
        const float2 c0 = sm[(2 * p) * RS + j], c1 = sm[(2 * p + 1) * RS + j];
        __stcs(reinterpret_cast<float4*>(img + (int64_t)(rank * NQ + j) * ld_img + a0 + 2 * p),
               make_float4(c0.x, c0.y, c1.x, c1.y));
    }
}

template <class SC, int QC, bool ROLL>
__global__ void __launch_bounds__(SC::T)
fused_range_ct_cluster_kernel(const float2* in, float2* img, int64_t ld_in, int64_t ld_img, const float2* filt,
                              const float2* tw) {
    fused_range_ct_cluster_body<SC, QC, ROLL>(in, img, ld_in, ld_img, filt, tw);
}

template <class SC, int QC, bool ROLL>
__global__ void __launch_bounds__(SC::T, ct_tma_min_blocks<SC>())
fused_range_ct_tma_kernel(const float2* in, float2* img, const __grid_constant__ CUtensorMap tmap, int64_t ld_in,
                          int64_t ld_img, const float2* filt, const float2* tw) {
    fused_range_ct_cluster_body<SC, QC, ROLL, true>(in, img, ld_in, ld_img, filt, tw, &tmap);
}

template <class SC, int QL, bool ROLL>
__global__ void __launch_bounds__(SC::T * QL)
fused_range_ct_kernel(const float2* in, float2* img, int64_t n_lines, int64_t ld_in, int64_t ld_img,
                      const float2* filt, const float2* tw) {
    fused_range_ct_body<SC, QL, ROLL>(in, img, n_lines, ld_in, ld_img, filt, tw);
}

template <class SC, int LPB, bool ROLL>
__global__ void __launch_bounds__(SC::T * LPB)
fused_streamed_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt,
                      const float2* tw) {
    fused_streamed_body<SC, LPB, ROLL>(in, out, n_lines, ld, filt, tw);
}
// registers capped so that SC::MINB blocks fit on one SM
template <class SC, int LPB, bool ROLL>
__global__ void __launch_bounds__(SC::T * LPB, SC::MINB)
fused_streamed_kernel_capped(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt,
                             const float2* tw) {
    fused_streamed_body<SC, LPB, ROLL>(in, out, n_lines, ld, filt, tw);
}

}  // namespace sar
