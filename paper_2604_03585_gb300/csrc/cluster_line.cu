// Lines longer than one SM's shared memory: a line of N = C * M samples is
// transformed by a cluster of C thread blocks that exchange it through
// distributed shared memory, so the fused compression of Sec. II-B (load,
// FFT, multiply by the matched filter, IFFT, store: two device-memory
// transfers per line) holds beyond the 16384 samples one block can keep on
// chip (the paper's own kernel stops at the 32 KiB threadgroup memory of its
// GPU, Sec. II-A).
//
// Index split (four-step Cooley-Tukey): n = n1 M + n2, k = k1 + C k2 with
// n1, k1 in [0, C) and n2, k2 in [0, M):
//   X[k1 + C k2] = sum_n2 W_M^{n2 k2} [ W_N^{n2 k1} sum_n1 x[n1 M + n2] W_C^{n1 k1} ].
// Block k1 of the cluster owns frequency residue k1.  The inverse mirrors it:
//   y[n1 M + n2] = sum_k1 W_C^{-n1 k1} [ W_N^{-n2 k1} sum_k2 Y[k1 + C k2] W_M^{-n2 k2} ].
//
// Per line (one cluster):
//  1. block r loads x[n1 M + n2] for every n1 and its quarter (1/C) of n2,
//     n2 in [r Q, r Q + Q), Q = M / C (C runs of Q contiguous samples), takes
//     the C-point DFT over n1 in registers and the twiddle W_N^{n2 k1}, and
//     pushes the value for k1 into block k1's shared memory at position n2
//     (a warp's 32 remote stores are one contiguous run);
//  2. block k1 runs the M-point line engine on what it received: forward
//     passes (digit-reversed spectrum in registers), the filter slice
//     H[k1 + C k2] / N in the same register order, inverse passes (natural n2
//     order), the twiddle W_N^{-n2 k1};
//  3. it pushes each n2 back to the block that owns it, line-major by k1;
//  4. block r takes the C-point inverse DFT over k1 of its n2 and stores
//     y[n1 M + n2] (C runs of Q contiguous samples).
// Cluster barriers: before the first push (every block of the cluster is
// running), after it (the data has landed), before the second push (every
// block is done with its shared memory for the FFT passes) and after it.
// After the last barrier a block touches only its own shared memory.
//
// The stand-alone FFT (sar_fft_lines and the plan-time filter design) uses
// steps 1 and 2's forward passes and stores X[k1 + C k2] through shared
// memory in natural k2 order (stride C in the output line).
#include <cooperative_groups.h>

#include "launch.cuh"
#include "registry.h"

namespace sar {

template <class SC, int C>
struct ClusterGeom {
    static constexpr int M = SC::N, N = M * C, Q = M / C;
    static constexpr int EQ = SC::E / C;   // n2 values per thread in steps 1 and 4
    static_assert(C == 2 || C == 4 || C == 8 || C == 16, "clusters of 2 to 16 blocks");
    static_assert(EQ * SC::T == Q, "each thread takes E / C values of n2 in the cluster steps");
};

__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

// Step 1: C-point DFTs over n1 and the twiddle W_N^{n2 k1}, pushed to block
// k1 at position n2 (PADDED: at the line engine's padded shared-memory slot of
// n2), one n2 at a time (C values live).  roots[k1 M + n2] = W_N^{k1 n2}
// (one contiguous row per k1).  The block announces itself on the cluster barrier at once and waits
// for the others just before its first remote store.
template <class SC, int C, bool RAGGED, bool CONJ_IN, bool PADDED = false>
__device__ __forceinline__ void cluster_first_stage(const float2* src, int valid, const float2* roots, int t,
                                                    int rank, float2* sm,
                                                    cooperative_groups::cluster_group& cluster) {
    using G = ClusterGeom<SC, C>;
    cluster_arrive_relaxed();
#pragma unroll(PADDED ? 2 : G::EQ)
    for (int i = 0; i < G::EQ; ++i) {
        const int n2 = rank * G::Q + t + SC::T * i;
        float2 a[C];
#pragma unroll
        for (int n1 = 0; n1 < C; ++n1) {
            const int idx = n1 * G::M + n2;
            float2 x = (!RAGGED || idx < valid) ? __ldcs(src + idx) : make_float2(0.f, 0.f);
            if (CONJ_IN) x.y = -x.y;
            a[n1] = x;
        }
        dft_reg<C, false>(a);
#pragma unroll
        for (int k1 = 1; k1 < C; ++k1) a[k1] = cmul(a[k1], roots[k1 * G::M + n2]);
        if (i == 0) cluster_wait();   // every block of the cluster is running (the first time round)
#pragma unroll
        for (int k1 = 0; k1 < C; ++k1) cluster.map_shared_rank(sm, k1)[PADDED ? smem_pos(n2, SC::PADSH) : n2] = a[k1];
    }
    cluster.sync();   // the pushes have landed
}

// The received M values, natural n2 order, into pass-1 geometry.
template <class SC>
__device__ __forceinline__ void load_received(const float2* sm, int t, float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / SC::R1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < SC::R1; ++r) v[s * SC::R1 + r] = sm[lo + r * SC::S1];
    }
    __syncthreads();   // the FFT passes reuse the buffer
}

template <class SC, int C, bool RAGGED>
__global__ void __launch_bounds__(SC::T)
cluster_fused_kernel(const float2* in, float2* out, int64_t ld, int valid, const float2* filt, const float2* tw) {
    namespace cg = cooperative_groups;
    using G = ClusterGeom<SC, C>;
    extern __shared__ float2 smem_dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int t = threadIdx.x;
    const int rank = (int)cluster.block_rank();
    const int64_t line = blockIdx.x / C;
    float2* sm = smem_dyn;
    const float2* roots = tw + SC::TW_ELEMS;
    cluster_first_stage<SC, C, RAGGED, false>(in + line * ld, valid, roots, t, rank, sm, cluster);
    float2 v[SC::E];
    load_received<SC>(sm, t, v);
    forward_passes<SC, 1>(v, sm, tw, t, 0);
    filter_multiply<SC>(filt + (int64_t)rank * G::M, t, v);
    inverse_passes<SC, 1>(v, sm, tw, t, 0);
    // v: natural n2 = lo + r S1 in pass-1 geometry; twiddle W_N^{-n2 k1}
#pragma unroll
    for (int s = 0; s < SC::E / SC::R1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < SC::R1; ++r) {
            const int n2 = lo + r * SC::S1;
            v[s * SC::R1 + r] = cmulc(v[s * SC::R1 + r], roots[rank * G::M + n2]);
        }
    }
    cluster.sync();   // every block is done with its shared memory
#pragma unroll
    for (int s = 0; s < SC::E / SC::R1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < SC::R1; ++r) {
            const int n2 = lo + r * SC::S1;
            float2* dst = cluster.map_shared_rank(sm, n2 / G::Q);
            dst[rank * G::Q + n2 % G::Q] = v[s * SC::R1 + r];
        }
    }
    cluster.sync();   // the pushes have landed; only local reads from here on
    float2* dst = out + line * ld;
#pragma unroll
    for (int i = 0; i < G::EQ; ++i) {
        const int q = t + SC::T * i;
        float2 b[C];
#pragma unroll
        for (int k1 = 0; k1 < C; ++k1) b[k1] = sm[k1 * G::Q + q];
        dft_reg<C, true>(b);
#pragma unroll
        for (int n1 = 0; n1 < C; ++n1) {
            const int idx = n1 * G::M + rank * G::Q + q;
            if (!RAGGED || idx < valid) __stcs(dst + idx, b[n1]);
        }
    }
}

// The same compression with the M-point part group-streamed (streamed.cuh:
// one radix group live in registers, rolled group loops), registers capped at
// 128 per thread so that two 256-thread blocks fit on an SM.  Step 1 pushes into the receivers' padded
// shared-memory slots, where the forward pass 1 runs in place like a middle
// pass.  The inverse pass 1 writes its result, times W_N^{-n2 k1}, back in
// place; after a cluster barrier each block pulls its own n2 range from every
// block's shared memory (a receive buffer for a push would cost a second line
// of shared memory), takes the inverse C-point DFTs and stores; a last
// barrier keeps every block's shared memory until all pulls are done.
template <class SC, int C, bool ROLL>
__global__ void __launch_bounds__(SC::T, SC::MINB > 0 ? SC::MINB
                                                    : (65536 / (SC::T * 128) > 1 ? 65536 / (SC::T * 128) : 1))
cluster_streamed_kernel(const float2* in, float2* out, int64_t ld, const float2* filt, const float2* tw) {
    namespace cg = cooperative_groups;
    using G = ClusterGeom<SC, C>;
    extern __shared__ float2 smem_dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int t = threadIdx.x;
    const int rank = (int)cluster.block_rank();
    const int64_t line = blockIdx.x / C;
    float2* sm = smem_dyn;
    const float2* roots = tw + SC::TW_ELEMS;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    constexpr int RL = SC::RL, GL = SC::E / RL;
    cluster_first_stage<SC, C, false, false, true>(in + line * ld, G::N, roots, t, rank, sm, cluster);
    streamed_mid_pass<SC, R1, S1, false, ROLL>(sm, tw, t);
    __syncthreads();
    const float2* tw2 = tw + R1 * S1;
    if constexpr (SC::P == 3) {
        streamed_mid_pass<SC, SC::R2, SC::S2, false, ROLL>(sm, tw2, t);
        __syncthreads();
    }
    // last forward pass, this block's filter slice, first inverse pass
    const float2* fl = filt + (int64_t)rank * G::M;
#pragma unroll(ROLL ? 1 : GL)
    for (int s = 0; s < GL; ++s) {
        const int g = t + SC::T * s;
        float2 x[RL];
        grp_smem_load<RL, 1>(sm, g * RL, SC::PADSH, x);
        dft_reg<RL, false>(x);
#pragma unroll
        for (int r = 0; r < RL; ++r) x[r] = cmul(x[r], fl[(s * RL + r) * SC::T + t]);
        dft_reg<RL, true>(x);
        grp_smem_store<RL, 1>(sm, g * RL, SC::PADSH, x);
    }
    __syncthreads();
    if constexpr (SC::P == 3) {
        streamed_mid_pass<SC, SC::R2, SC::S2, true, ROLL>(sm, tw2, t);
        __syncthreads();
    }
    // inverse pass 1 in place, natural n2 = lo + r S1, times W_N^{-n2 k1}
#pragma unroll(ROLL ? 1 : G1)
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
#pragma unroll
        for (int r = 0; r < R1; ++r) x[r] = cmulc(x[r], roots[rank * G::M + lo + r * S1]);
        grp_smem_store<R1, S1>(sm, lo, SC::PADSH, x);
    }
    cluster.sync();   // every block's inverse result is in place
    float2* dst = out + line * ld;
#pragma unroll 2
    for (int i = 0; i < G::EQ; ++i) {
        const int n2 = rank * G::Q + t + SC::T * i;
        float2 b[C];
#pragma unroll
        for (int k1 = 0; k1 < C; ++k1) b[k1] = cluster.map_shared_rank(sm, k1)[smem_pos(n2, SC::PADSH)];
        dft_reg<C, true>(b);
#pragma unroll
        for (int n1 = 0; n1 < C; ++n1) __stcs(dst + n1 * G::M + n2, b[n1]);
    }
    cluster.sync();   // keep this block's shared memory until every block has pulled
}

// Stand-alone FFT of a line, natural-order output (unnormalised; the inverse
// as conj(FFT(conj x))).  Output lines are dense lines of N.
template <class SC, int C, bool INV>
__global__ void __launch_bounds__(SC::T)
cluster_dft_kernel(const float2* in, float2* out, int64_t ld, int valid, const float2* tw) {
    namespace cg = cooperative_groups;
    using G = ClusterGeom<SC, C>;
    extern __shared__ float2 smem_dyn[];
    cg::cluster_group cluster = cg::this_cluster();
    const int t = threadIdx.x;
    const int rank = (int)cluster.block_rank();
    const int64_t line = blockIdx.x / C;
    float2* sm = smem_dyn;
    cluster_first_stage<SC, C, true, INV>(in + line * ld, valid, tw + SC::TW_ELEMS, t, rank, sm, cluster);
    float2 v[SC::E];
    load_received<SC>(sm, t, v);
    forward_passes<SC, 1>(v, sm, tw, t, 0);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < SC::E / SC::RL; ++s) {
#pragma unroll
        for (int r = 0; r < SC::RL; ++r) {
            const int k2 = natural_index<SC>(t + SC::T * s, r);
            sm[smem_pos(k2, SC::PADSH)] = v[s * SC::RL + r];
        }
    }
    __syncthreads();
    float2* dst = out + line * (int64_t)G::N;
#pragma unroll
    for (int j = 0; j < SC::E; ++j) {
        const int k2 = t + SC::T * j;
        const float2 x = sm[smem_pos(k2, SC::PADSH)];
        dst[rank + C * k2] = INV ? cconj(x) : x;
    }
}

namespace {

template <class SC, int C>
constexpr int cluster_smem() {
    return SC::SMEM_ELEMS * (int)sizeof(float2);
}

template <class K>
cudaError_t cluster_attrs(K kernel, int smem, int c) {
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && c > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <class SC, int C>
cudaError_t prepare_cluster() {
    constexpr int smem = cluster_smem<SC, C>();
    cudaError_t e;
    if ((e = cluster_attrs(cluster_fused_kernel<SC, C, false>, smem, C)) != cudaSuccess) return e;
    if ((e = cluster_attrs(cluster_dft_kernel<SC, C, false>, smem, C)) != cudaSuccess) return e;
    return cluster_attrs(cluster_dft_kernel<SC, C, true>, smem, C);
}

template <class K, class... Args>
cudaError_t launch_on_clusters(K kernel, int64_t n_lines, int threads, int smem, int c, cudaStream_t st,
                               Args... args) {
    const int64_t blocks = n_lines * c;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class SC, int C>
cudaError_t launch_cluster_fused(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid,
                                 const float2* filt, const float2* tw, const FusedCtl&, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    // zero-padded lines (valid < N) arise only in ragged batches, which stop at 16384
    if (valid != ClusterGeom<SC, C>::N) return cudaErrorInvalidValue;
    constexpr int smem = cluster_smem<SC, C>();
    return launch_on_clusters(cluster_fused_kernel<SC, C, false>, n_lines, SC::T, smem, C, st, in, out, ld, valid,
                              filt, tw);
}

template <class SC, int C>
cudaError_t prepare_cluster_streamed() {
    cudaError_t e = cluster_attrs(cluster_streamed_kernel<SC, C, true>, cluster_smem<SC, C>(), C);
    return e == cudaSuccess ? prepare_cluster<SC, C>() : e;
}

template <class SC, int C>
cudaError_t launch_cluster_streamed(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid,
                                    const float2* filt, const float2* tw, const FusedCtl&, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (valid != ClusterGeom<SC, C>::N) return cudaErrorInvalidValue;
    return launch_on_clusters(cluster_streamed_kernel<SC, C, true>, n_lines, SC::T, cluster_smem<SC, C>(), C, st,
                              in, out, ld, filt, tw);
}

template <class SC, int C>
cudaError_t launch_cluster_dft(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid,
                               const float2* tw, int inverse, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    constexpr int smem = cluster_smem<SC, C>();
    if (inverse)
        return launch_on_clusters(cluster_dft_kernel<SC, C, true>, n_lines, SC::T, smem, C, st, in, out, ld, valid,
                                  tw);
    return launch_on_clusters(cluster_dft_kernel<SC, C, false>, n_lines, SC::T, smem, C, st, in, out, ld, valid, tw);
}

template <class SC, int C, bool STREAMED = false>
constexpr SchedDesc make_cluster_desc(const char* name) {
    return SchedDesc{name,
                     ClusterGeom<SC, C>::N,
                     SC::E,
                     SC::R1,
                     SC::R2,
                     SC::R3,
                     1,
                     SC::T,
                     cluster_smem<SC, C>(),
                     SC::TW_ELEMS + ClusterGeom<SC, C>::N,
                     SC::RL,
                     0,
                     STREAMED ? &launch_cluster_streamed<SC, C> : &launch_cluster_fused<SC, C>,
                     &launch_cluster_dft<SC, C>,
                     STREAMED ? &prepare_cluster_streamed<SC, C> : &prepare_cluster<SC, C>,
                     nullptr,
                     0,
                     nullptr,
                     C};
}

using M8192 = Sched<8192, 32, 16, 16, 32>;      // 256 threads, 66 KiB of shared memory per block
using M16384 = Sched<16384, 32, 16, 32, 32>;    // 512 threads, 132 KiB
using M4096 = Sched<4096, 32, 16, 16, 16>;      // 128 threads, 33 KiB, 4 blocks per SM (128 registers)
using M4096b5 = Sched<4096, 32, 16, 16, 16, 5>; // the same, registers capped for 5 blocks per SM
// first of each length: the fastest on GB300 (the autotuner times them all)
const SchedDesc kTable[] = {
    make_cluster_desc<M4096b5, 8, true>("n32768_c8_m4096_e32_sr_b5"),
    make_cluster_desc<M4096, 8, true>("n32768_c8_m4096_e32_sr"),
    make_cluster_desc<M8192, 8, true>("n65536_c8_m8192_e32_sr"),
    make_cluster_desc<M8192, 16, true>("n131072_c16_m8192_e32_sr"),
    make_cluster_desc<M4096, 16, true>("n65536_c16_m4096_e32_sr"),
    make_cluster_desc<M8192, 4, true>("n32768_c4_m8192_e32_sr"),
    make_cluster_desc<M16384, 2, true>("n32768_c2_m16384_e32_sr"),
    make_cluster_desc<M16384, 4, true>("n65536_c4_m16384_e32_sr"),
    make_cluster_desc<M16384, 8, true>("n131072_c8_m16384_e32_sr"),
    make_cluster_desc<M8192, 4>("n32768_c4_m8192_e32"),
    make_cluster_desc<M16384, 2>("n32768_c2_m16384_e32"),
    make_cluster_desc<M8192, 8>("n65536_c8_m8192_e32"),
    make_cluster_desc<M16384, 4>("n65536_c4_m16384_e32"),
    make_cluster_desc<M16384, 8>("n131072_c8_m16384_e32"),
    make_cluster_desc<M8192, 16>("n131072_c16_m8192_e32"),
};

}  // namespace

const SchedDesc* schedules_cluster(int* count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}

}  // namespace sar
