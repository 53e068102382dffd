// Device side of the mixed-radix line engine (see mixed_radix.cu): the
// register DFTs of every radix, the pass routines and the fused kernel.
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>
#include <utility>

#include "launch.cuh"

namespace sar {
namespace mixed {

constexpr int kMixedThreads = 256;

constexpr int kMaxPasses = 4;
constexpr int kMixedSmemMax = 72 * 1024;   // dynamic shared memory the kernel is set up for
constexpr int kRadices[] = {32, 25, 20, 16, 15, 14, 12, 10, 9, 8, 7, 6, 5, 4, 3, 2};

struct MixedGeom {
    int n, P;
    int R[kMaxPasses], S[kMaxPasses], tw_off[kMaxPasses];
    uint32_t M[kMaxPasses];   // ceil(2^32 / S): g / S == umulhi(g, M) for every g < 8192 and 2 <= S <= 8192
                              // (checked exhaustively); 0 for S == 1
    int T;                    // threads per line; kMixedThreads / T lines per block
    int pos_off;              // float2 offset in the table of pos[k] (int32, k < n): the position that
                              // holds frequency k after the forward passes (the plain transform's order)
};

__device__ __forceinline__ int mpad(int p) { return p + (p >> 5); }

// ---- R-point DFT in registers (natural order in and out) -------------------
__host__ __device__ constexpr int small_factor(int L) {
    return L % 4 == 0 ? 4 : L % 2 == 0 ? 2 : L % 3 == 0 ? 3 : L % 5 == 0 ? 5 : L % 7 == 0 ? 7 : L;
}
// position of output k of a length-L DIF over factors small_factor(L), ...
__host__ __device__ constexpr int mpos(int L, int k) {
    return L == 1 ? 0 : ((k % small_factor(L)) * (L / small_factor(L)) + mpos(L / small_factor(L), k / small_factor(L)));
}

// p-point DFT of a[0..p-1] for an odd prime p, by the symmetry of the
// roots: with a_k = x_k + x_{p-k} and b_k = x_k - x_{p-k} (k = 1 .. h,
// h = (p - 1) / 2),
//   y_0 = x_0 + sum_k a_k,
//   y_j = t_j -+ i u_j,  y_{p-j} = t_j +- i u_j   (j = 1 .. h; upper signs
//   forward), t_j = x_0 + sum_k cos(2 pi j k / p) a_k,
//   u_j = sum_k sin(2 pi j k / p) b_k,
// real constants only: about 5 instructions per output at p = 5 instead of
// the 16 of the definition's p - 1 complex products per output.
template <int p, int j, int... K>
__device__ __forceinline__ float2 odd_t(float2 x0, const float2 (&av)[p], std::integer_sequence<int, K...>) {
    float2 t = x0;
    ((t = make_float2(fmaf((float)ct::cos2pi((K + 1) * j, p), av[K + 1].x, t.x),
                      fmaf((float)ct::cos2pi((K + 1) * j, p), av[K + 1].y, t.y))),
     ...);
    return t;
}
template <int p, int j, int... K>
__device__ __forceinline__ float2 odd_u(const float2 (&bv)[p], std::integer_sequence<int, K...>) {
    float2 u = make_float2(0.f, 0.f);
    ((u = make_float2(fmaf((float)ct::sin2pi((K + 1) * j, p), bv[K + 1].x, u.x),
                      fmaf((float)ct::sin2pi((K + 1) * j, p), bv[K + 1].y, u.y))),
     ...);
    return u;
}
template <int p, bool INV, int... J>
__device__ __forceinline__ void dft_odd_outputs(float2 (&a)[p], float2 x0, const float2 (&av)[p],
                                                const float2 (&bv)[p], std::integer_sequence<int, J...>) {
    constexpr int h = (p - 1) / 2;
    float2 y[p];
    (([&] {
         constexpr int j = J + 1;
         const float2 t = odd_t<p, j>(x0, av, std::make_integer_sequence<int, h>{});
         const float2 u = odd_u<p, j>(bv, std::make_integer_sequence<int, h>{});
         // -i u = (u.y, -u.x); +i u = (-u.y, u.x)
         const float2 mi = make_float2(u.y, -u.x);
         y[j] = INV ? csub(t, mi) : cadd(t, mi);
         y[p - j] = INV ? cadd(t, mi) : csub(t, mi);
     }()),
     ...);
#pragma unroll
    for (int k = 1; k < p; ++k) a[k] = y[k];
}
template <int p, bool INV>
__device__ __forceinline__ void dft_odd(float2 (&a)[p]) {
    constexpr int h = (p - 1) / 2;
    float2 av[p], bv[p];
    float2 y0 = a[0];
#pragma unroll
    for (int k = 1; k <= h; ++k) {
        av[k] = cadd(a[k], a[p - k]);
        bv[k] = csub(a[k], a[p - k]);
        y0 = cadd(y0, av[k]);
    }
    const float2 x0 = a[0];
    dft_odd_outputs<p, INV>(a, x0, av, bv, std::make_integer_sequence<int, h>{});
    a[0] = y0;
}

template <int R, int L, int OFF, bool INV, int J, int... K>
__device__ __forceinline__ void mlevel_store(float2 (&v)[R], const float2 (&a)[small_factor(L)],
                                             std::integer_sequence<int, K...>) {
    constexpr int q = L / small_factor(L);
    ((v[OFF + J + K * q] = twiddle_ct<L, J * K, INV>(a[K])), ...);
}
// one butterfly column j of the level of length L at offset OFF: the p
// elements OFF + j + m q (q = L / p), their p-point DFT, twiddles W_L^{j k}
template <int R, int L, int OFF, bool INV, int J>
__device__ __forceinline__ void mlevel_one(float2 (&v)[R]) {
    constexpr int p = small_factor(L), q = L / p;
    float2 a[p];
#pragma unroll
    for (int m = 0; m < p; ++m) a[m] = v[OFF + J + m * q];
    if constexpr (p == 4) {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]), t2 = cadd(a[1], a[3]);
        const float2 t3 = cmul_mi<INV>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[1] = cadd(t1, t3);
        a[2] = csub(t0, t2);
        a[3] = csub(t1, t3);
    } else if constexpr (p == 2) {
        const float2 t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    } else {
        dft_odd<p, INV>(a);
    }
    mlevel_store<R, L, OFF, INV, J>(v, a, std::make_integer_sequence<int, p>{});
}
template <int R, int L, int OFF, bool INV, int... J>
__device__ __forceinline__ void mlevel(float2 (&v)[R], std::integer_sequence<int, J...>) {
    (mlevel_one<R, L, OFF, INV, J>(v), ...);
}
template <int R, int L, int OFF, bool INV, int... K>
__device__ __forceinline__ void mrec_children(float2 (&v)[R], std::integer_sequence<int, K...>);
template <int R, int L, int OFF, bool INV>
__device__ __forceinline__ void mrec(float2 (&v)[R]) {
    if constexpr (L > 1) {
        constexpr int p = small_factor(L), q = L / p;
        mlevel<R, L, OFF, INV>(v, std::make_integer_sequence<int, q>{});
        mrec_children<R, L, OFF, INV>(v, std::make_integer_sequence<int, p>{});
    }
}
template <int R, int L, int OFF, bool INV, int... K>
__device__ __forceinline__ void mrec_children(float2 (&v)[R], std::integer_sequence<int, K...>) {
    constexpr int q = L / small_factor(L);
    (mrec<R, q, OFF + K * q, INV>(v), ...);
}
template <int R, int... K>
__device__ __forceinline__ void munscramble(const float2 (&v)[R], float2 (&o)[R], std::integer_sequence<int, K...>) {
    ((o[K] = v[mpos(R, K)]), ...);
}
// v[k] <- sum_m v[m] exp(-+2 pi i m k / R)
template <int R, bool INV>
__device__ __forceinline__ void dft_any(float2 (&v)[R]) {
    if constexpr (R > 1) {
        mrec<R, R, 0, INV>(v);
        float2 o[R];
        munscramble<R>(v, o, std::make_integer_sequence<int, R>{});
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = o[k];
    }
}

// ---- one group of one pass ---------------------------------------------------
enum MMode { kFirst, kMid, kLast, kInvMid, kInvFirst, kLastDft };

// shared-memory slot of position p: one pad slot per 32 positions, or with
// PADDIV > 0 one per PADDIV positions
template <int PADDIV>
__device__ __forceinline__ int mslot(int p) {
    if constexpr (PADDIV > 0)
        return p + p / PADDIV;
    else
        return mpad(p);
}

// MODE: kFirst global -> DFT -> twiddle -> smem; kMid smem -> DFT -> twiddle
// -> smem; kLast (src global when P == 1) -> DFT -> filter -> IDFT -> smem (or
// global when P == 1); kInvMid smem -> conj twiddle -> IDFT -> smem; kInvFirst
// smem -> conj twiddle -> IDFT -> global; kLastDft smem -> DFT -> smem (the
// last pass of a plain transform).
template <int R, int MODE, bool SINGLE, int PADDIV = 0>
__device__ __forceinline__ void mgroup(int g, int S, uint32_t M, int ng, const float2* src, float2* dst, float2* sm,
                                       const float2* twi, const float2* filt) {
    const int q = M ? (int)__umulhi((uint32_t)g, M) : g;   // M == 0: S == 1
    const int lo = g - q * S, base = q * R * S + lo;
    float2 v[R];
    const bool from_global = MODE == kFirst || (MODE == kLast && SINGLE);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = from_global ? __ldcs(src + base + r * S) : sm[mslot<PADDIV>(base + r * S)];
    if constexpr (MODE == kInvMid || MODE == kInvFirst) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], twi[r * S + lo]);
        dft_any<R, true>(v);
    } else {
        dft_any<R, false>(v);
        if constexpr (MODE == kLast) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = cmul(v[r], filt[r * ng + g]);   // slot of position g R + r
            dft_any<R, true>(v);
        } else if constexpr (MODE == kLastDft) {
            // the spectrum stays in position order
        } else {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twi[r * S + lo]);
        }
    }
    const bool to_global = MODE == kInvFirst || (MODE == kLast && SINGLE);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (to_global)
            __stcs(dst + base + r * S, v[r]);
        else
            sm[mslot<PADDIV>(base + r * S)] = v[r];
    }
}

template <int MODE, bool SINGLE>
__device__ __forceinline__ void mpass(int R, int S, uint32_t M, int n, int t, int T, const float2* src, float2* dst,
                                      float2* sm, const float2* twi, const float2* filt) {
    const int ng = n / R;
#define SAR_MIXED_CASE(RR)                                                                       \
    case RR:                                                                                     \
        for (int g = t; g < ng; g += T) mgroup<RR, MODE, SINGLE>(g, S, M, ng, src, dst, sm, twi, filt); \
        break;
    switch (R) {
        SAR_MIXED_CASE(2)
        SAR_MIXED_CASE(3)
        SAR_MIXED_CASE(4)
        SAR_MIXED_CASE(5)
        SAR_MIXED_CASE(6)
        SAR_MIXED_CASE(7)
        SAR_MIXED_CASE(8)
        SAR_MIXED_CASE(9)
        SAR_MIXED_CASE(10)
        SAR_MIXED_CASE(12)
        SAR_MIXED_CASE(14)
        SAR_MIXED_CASE(15)
        SAR_MIXED_CASE(16)
        SAR_MIXED_CASE(20)
        SAR_MIXED_CASE(25)
        SAR_MIXED_CASE(32)
        default: break;
    }
#undef SAR_MIXED_CASE
}

// Lines of T threads each, kMixedThreads / T lines per block (lines past the
// end still take part in the block's barriers).  MINB: blocks per SM the
// registers are capped for (2, 3 or 4; chosen per length on the host).
template <int MINB>
__global__ void __launch_bounds__(kMixedThreads, MINB)
fused_mixed_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt, const float2* tw,
                   MixedGeom geo) {
    extern __shared__ float2 smem_mixed[];
    const int T = geo.T, lib = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t line = (int64_t)blockIdx.x * (kMixedThreads / T) + lib;
    const bool live = line < n_lines;
    const int n = geo.n, P = geo.P;
    float2* sm = smem_mixed + lib * (n + (n >> 5) + 1);
    const float2* src = in + (live ? line : 0) * ld;
    float2* dst = out + (live ? line : 0) * ld;
    if (P == 1) {
        if (live) mpass<kLast, true>(geo.R[0], 1, 0u, n, t, T, src, dst, sm, tw, filt);
        return;
    }
    if (live) mpass<kFirst, false>(geo.R[0], geo.S[0], geo.M[0], n, t, T, src, dst, sm, tw + geo.tw_off[0], filt);
    __syncthreads();
    for (int i = 1; i < P - 1; ++i) {
        if (live) mpass<kMid, false>(geo.R[i], geo.S[i], geo.M[i], n, t, T, src, dst, sm, tw + geo.tw_off[i], filt);
        __syncthreads();
    }
    if (live) mpass<kLast, false>(geo.R[P - 1], 1, 0u, n, t, T, src, dst, sm, tw, filt);
    __syncthreads();
    for (int i = P - 2; i >= 1; --i) {
        if (live) mpass<kInvMid, false>(geo.R[i], geo.S[i], geo.M[i], n, t, T, src, dst, sm, tw + geo.tw_off[i], filt);
        __syncthreads();
    }
    if (live) mpass<kInvFirst, false>(geo.R[0], geo.S[0], geo.M[0], n, t, T, src, dst, sm, tw + geo.tw_off[0], filt);
}

// The same kernel for one three-pass length fixed at compile time (radices
// RA, RB, RC, T threads per line): every stride, group split and table
// offset becomes a constant, so the per-element index arithmetic of the
// runtime kernel folds away.  Same passes, same arithmetic, same tables and
// filter order; results are bit-identical to the runtime kernel's.
__host__ __device__ constexpr uint32_t split_magic(int S) {
    return S > 1 ? (uint32_t)((((uint64_t)1 << 32) + (uint64_t)S - 1) / (uint64_t)S) : 0u;
}
// PADDIV: the shared-memory padding (0: one slot per 32 positions, as the
// runtime kernel; else one per PADDIV, chosen per length from a simulation
// of every pass's bank pairs); mixed3_smem is the block's shared memory.
template <int N, int T, int PADDIV>
__host__ __device__ constexpr int mixed3_smem() {
    return (kMixedThreads / T) * (N + (PADDIV > 0 ? N / PADDIV : N >> 5) + 1) * (int)sizeof(float2);
}
template <int N, int RA, int RB, int RC, int T, int MINB, int PADDIV>
__global__ void __launch_bounds__(kMixedThreads, MINB)
fused_mixed3_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt,
                    const float2* tw) {
    constexpr int SA = N / RA, SB = SA / RB;
    static_assert(RA * RB * RC == N && SB == RC, "three radices of N");
    static_assert(kMixedThreads % T == 0, "whole lines per block");
    constexpr uint32_t MA = split_magic(SA), MB = split_magic(SB);
    constexpr int LPB = kMixedThreads / T, PADN = mixed3_smem<N, T, PADDIV>() / LPB / (int)sizeof(float2);
    extern __shared__ float2 smem_mixed[];
    const int lib = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    const bool live = line < n_lines;
    float2* sm = smem_mixed + lib * PADN;
    const float2* src = in + (live ? line : 0) * ld;
    float2* dst = out + (live ? line : 0) * ld;
    const float2* twb = tw + RA * SA;   // the second pass's table
    if (live)
        for (int g = t; g < N / RA; g += T)
            mgroup<RA, kFirst, false, PADDIV>(g, SA, MA, N / RA, src, dst, sm, tw, filt);
    __syncthreads();
    if (live)
        for (int g = t; g < N / RB; g += T)
            mgroup<RB, kMid, false, PADDIV>(g, SB, MB, N / RB, src, dst, sm, twb, filt);
    __syncthreads();
    if (live)
        for (int g = t; g < N / RC; g += T)
            mgroup<RC, kLast, false, PADDIV>(g, 1, 0u, N / RC, src, dst, sm, tw, filt);
    __syncthreads();
    if (live)
        for (int g = t; g < N / RB; g += T)
            mgroup<RB, kInvMid, false, PADDIV>(g, SB, MB, N / RB, src, dst, sm, twb, filt);
    __syncthreads();
    if (live)
        for (int g = t; g < N / RA; g += T)
            mgroup<RA, kInvFirst, false, PADDIV>(g, SA, MA, N / RA, src, dst, sm, tw, filt);
}

// The plain transform of the same compile-time length (the forward passes,
// then natural order through the position table after the twiddles; sgn =
// -1 conjugates input and output for the inverse).
template <int N, int RA, int RB, int RC, int T, int MINB, int PADDIV>
__global__ void __launch_bounds__(kMixedThreads, MINB)
mixed3_dft_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                  int pos_off, float sgn) {
    constexpr int SA = N / RA, SB = SA / RB;
    static_assert(RA * RB * RC == N && SB == RC, "three radices of N");
    constexpr uint32_t MA = split_magic(SA), MB = split_magic(SB);
    constexpr int LPB = kMixedThreads / T, PADN = mixed3_smem<N, T, PADDIV>() / LPB / (int)sizeof(float2);
    extern __shared__ float2 smem_mixed[];
    const int lib = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    const bool live = line < n_lines;
    float2* sm = smem_mixed + lib * PADN;
    const float2* src = in + (live ? line : 0) * ld;
    float2* dst = out + (live ? line : 0) * ld;
    const float2* twb = tw + RA * SA;
    if (live)
        for (int p = t; p < N; p += T) {
            const float2 x = p < valid ? __ldcs(src + p) : make_float2(0.f, 0.f);
            sm[mslot<PADDIV>(p)] = make_float2(x.x, sgn * x.y);
        }
    __syncthreads();
    if (live)
        for (int g = t; g < N / RA; g += T)
            mgroup<RA, kMid, false, PADDIV>(g, SA, MA, N / RA, src, dst, sm, tw, tw);
    __syncthreads();
    if (live)
        for (int g = t; g < N / RB; g += T)
            mgroup<RB, kMid, false, PADDIV>(g, SB, MB, N / RB, src, dst, sm, twb, tw);
    __syncthreads();
    if (live)
        for (int g = t; g < N / RC; g += T)
            mgroup<RC, kLastDft, false, PADDIV>(g, 1, 0u, N / RC, src, dst, sm, tw, tw);
    __syncthreads();
    const int32_t* pos = reinterpret_cast<const int32_t*>(tw + pos_off);
    if (live)
        for (int k = t; k < N; k += T) {
            const float2 x = sm[mslot<PADDIV>(pos[k])];
            __stcs(dst + k, make_float2(x.x, sgn * x.y));
        }
}

// The fused compression of a compiled length with the corner turn folded
// into its store (Sec. IV-A steps 1 and 2 in one kernel): four consecutive
// range lines per group, LPB = 256 / T lines per block and QC = 4 / LPB blocks
// per thread-block cluster (one block of four lines for T = 64, clusters of
// two blocks of two for T = 128, of four blocks of one for T = 256).  The
// forward passes, the filter and the inverse middle passes are those of
// fused_mixed3_kernel; the inverse first pass keeps its results in
// registers, and after a barrier (the cluster's, or the block's when QC = 1)
// each line pushes natural-order sample i into the shared memory of block
// i / (N / QC), row = the line's place in the group (rows padded by 4 slots,
// as the power-of-two fold), slot i mod (N / QC).  After a second barrier
// each block writes each of its range bins' four samples as one 32-byte run
// of image row i.  Same arithmetic as the unfolded kernel and the separate
// corner turn: bit-identical images.
template <int N, int T, int PADDIV>
struct MixedCtGeom {
    static constexpr int LPB = kMixedThreads / T, QC = 4 / LPB;
    static constexpr int PADN = mixed3_smem<N, T, PADDIV>() / LPB / (int)sizeof(float2);
    static constexpr int NQ = N / QC, RS = NQ + 4;
    static constexpr int CAP = LPB * PADN;   // float2 of shared memory per block
    // tensor-store boxes: NB boxes of BR bin rows (BR a multiple of 4, so that
    // every box starts 128 bytes aligned; NB BR >= NQ, the last box clipped at
    // the block's plane), staged bin-major in the block's shared memory
    __host__ __device__ static constexpr int box_rows(int nb) { return ((NQ + nb - 1) / nb + 3) / 4 * 4; }
    __host__ __device__ static constexpr int boxes() {
        int nb = (NQ + 255) / 256;
        while (box_rows(nb) > 256 || nb * box_rows(nb) * 4 > CAP) ++nb;
        return nb;
    }
    static constexpr int NB = boxes(), BR = box_rows(NB);
    static constexpr int NIT = (2 * NQ + kMixedThreads - 1) / kMixedThreads;   // float4 staged per thread
    static_assert(BR % 4 == 0 && BR <= 256 && NB * BR >= NQ && (NB - 1) * BR < NQ, "boxes cover the plane once");
    static_assert(NB * BR * 4 <= CAP && 4 * RS <= CAP, "staged boxes and receive rows fit the shared memory");
};

template <int N, int RA, int RB, int RC, int T, int MINB, int PADDIV, bool TMA>
__device__ __forceinline__ void fused_mixed3_ct_body(const float2* in, float2* img, int64_t ld_in, int64_t ld_img,
                                                     const float2* filt, const float2* tw, const CUtensorMap* tmap) {
    namespace cg = cooperative_groups;
    constexpr int LPB = kMixedThreads / T, QC = 4 / LPB;
    static_assert(LPB * QC == 4, "groups of four lines");
    constexpr int SA = N / RA, SB = SA / RB;
    static_assert(RA * RB * RC == N && SB == RC, "three radices of N");
    constexpr uint32_t MA = split_magic(SA), MB = split_magic(SB);
    constexpr int PADN = mixed3_smem<N, T, PADDIV>() / LPB / (int)sizeof(float2);
    constexpr int NQ = N / QC, RS = NQ + 4, GA = (SA + T - 1) / T;
    static_assert(N % QC == 0 && 4 * RS <= LPB * PADN, "four receive rows fit the block's line buffers");
    extern __shared__ float2 smem_mixed[];
    const int lib = threadIdx.x / T, t = threadIdx.x % T;
    int rank = 0;
    if constexpr (QC > 1) rank = (int)cg::this_cluster().block_rank();
    const int64_t a0 = ((int64_t)blockIdx.x - rank) * LPB;   // first line of the group of four
    const int row = rank * LPB + lib;                         // this line's place in the group
    const int64_t line = a0 + row;
    float2* sm = smem_mixed + lib * PADN;
    const float2* src = in + line * ld_in;
    const float2* twb = tw + RA * SA;
    for (int g = t; g < N / RA; g += T) mgroup<RA, kFirst, false, PADDIV>(g, SA, MA, N / RA, src, img, sm, tw, filt);
    __syncthreads();
    for (int g = t; g < N / RB; g += T) mgroup<RB, kMid, false, PADDIV>(g, SB, MB, N / RB, src, img, sm, twb, filt);
    __syncthreads();
    for (int g = t; g < N / RC; g += T) mgroup<RC, kLast, false, PADDIV>(g, 1, 0u, N / RC, src, img, sm, tw, filt);
    __syncthreads();
    for (int g = t; g < N / RB; g += T)
        mgroup<RB, kInvMid, false, PADDIV>(g, SB, MB, N / RB, src, img, sm, twb, filt);
    __syncthreads();
    // inverse first pass into registers: group g < SA holds positions g + r SA
    float2 v[GA][RA];
#pragma unroll
    for (int s = 0; s < GA; ++s) {
        const int g = t + T * s;
        if (g < SA) {
#pragma unroll
            for (int r = 0; r < RA; ++r) v[s][r] = sm[mslot<PADDIV>(g + r * SA)];
#pragma unroll
            for (int r = 1; r < RA; ++r) v[s][r] = cmulc(v[s][r], tw[r * SA + g]);
            dft_any<RA, true>(v[s]);
        }
    }
    if constexpr (QC > 1)
        cg::this_cluster().sync();   // every block is done with its shared memory
    else
        __syncthreads();
#pragma unroll
    for (int s = 0; s < GA; ++s) {
        const int g = t + T * s;
        if (g < SA) {
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const int i = g + r * SA;
                float2* dst = smem_mixed;
                if constexpr (QC > 1) dst = cg::this_cluster().map_shared_rank(smem_mixed, i / NQ);
                dst[row * RS + i % NQ] = v[s][r];
            }
        }
    }
    if constexpr (QC > 1)
        cg::this_cluster().sync();   // the pushes have landed; only local reads from here on
    else
        __syncthreads();
    if constexpr (TMA) {
        // the receive rows rewritten bin-major in place (bin j's four samples
        // at stg[2j], stg[2j + 1]) and stored as NB boxes of the block's plane
        using G = MixedCtGeom<N, T, PADDIV>;
        float4 w[G::NIT];
#pragma unroll
        for (int k = 0; k < G::NIT; ++k) {
            const int idx = threadIdx.x + k * kMixedThreads, j = idx >> 1, p = idx & 1;
            if (idx < NQ * 2) {
                const float2 c0 = smem_mixed[(2 * p) * RS + j], c1 = smem_mixed[(2 * p + 1) * RS + j];
                w[k] = make_float4(c0.x, c0.y, c1.x, c1.y);
            }
        }
        __syncthreads();
        float4* stg = reinterpret_cast<float4*>(smem_mixed);
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(stg);
        if (base & 127) {   // a tensor copy wants 128-byte aligned shared memory: plain stores
#pragma unroll
            for (int k = 0; k < G::NIT; ++k) {
                const int idx = threadIdx.x + k * kMixedThreads, j = idx >> 1, p = idx & 1;
                if (idx < NQ * 2)
                    __stcs(reinterpret_cast<float4*>(img + (int64_t)(rank * NQ + j) * ld_img + a0 + 2 * p), w[k]);
            }
            return;
        }
#pragma unroll
        for (int k = 0; k < G::NIT; ++k) {
            const int idx = threadIdx.x + k * kMixedThreads;
            if (idx < NQ * 2) stg[idx] = w[k];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll 1
            for (int c = 0; c < G::NB; ++c)
                asm volatile(
                    "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(tmap),
                    "r"(base + c * G::BR * 32), "r"((int)(2 * a0)), "r"(c * G::BR), "r"(rank)
                    : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        return;
    }
    for (int idx = threadIdx.x; idx < NQ * 2; idx += kMixedThreads) {
        const int j = idx >> 1, p = idx & 1;
        const float2 c0 = smem_mixed[(2 * p) * RS + j], c1 = smem_mixed[(2 * p + 1) * RS + j];
        __stcs(reinterpret_cast<float4*>(img + (int64_t)(rank * NQ + j) * ld_img + a0 + 2 * p),
               make_float4(c0.x, c0.y, c1.x, c1.y));
    }
}

template <int N, int RA, int RB, int RC, int T, int MINB, int PADDIV>
__global__ void __launch_bounds__(kMixedThreads, MINB)
fused_mixed3_ct_kernel(const float2* in, float2* img, int64_t ld_in, int64_t ld_img, const float2* filt,
                       const float2* tw) {
    fused_mixed3_ct_body<N, RA, RB, RC, T, MINB, PADDIV, false>(in, img, ld_in, ld_img, filt, tw, nullptr);
}

// the same fold with the image tiles written by tensor stores (tmap: the
// image as one plane of N / QC bin rows per block of a cluster)
template <int N, int RA, int RB, int RC, int T, int MINB, int PADDIV>
__global__ void __launch_bounds__(kMixedThreads, MINB)
fused_mixed3_ct_tma_kernel(const float2* in, float2* img, const __grid_constant__ CUtensorMap tmap, int64_t ld_in,
                           int64_t ld_img, const float2* filt, const float2* tw) {
    fused_mixed3_ct_body<N, RA, RB, RC, T, MINB, PADDIV, true>(in, img, ld_in, ld_img, filt, tw, &tmap);
}

// one occupancy variant of the kernel (mixed_radix_k<MINB>.cu)
template <int MINB>
cudaError_t launch_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt,
                          const float2* tw, const MixedGeom& g, int lines_per_block, int smem, cudaStream_t st) {
    fused_mixed_kernel<MINB><<<(unsigned)((n_lines + lines_per_block - 1) / lines_per_block), kMixedThreads, smem,
                               st>>>(in, out, n_lines, ld, filt, tw, g);
    return cudaGetLastError();
}
template <int MINB>
cudaError_t set_smem(int bytes) {
    return cudaFuncSetAttribute(fused_mixed_kernel<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// the variants, one translation unit each (compiled in parallel)
#define SAR_MIXED_VARIANT_DECL(MB)                                                                            \
    cudaError_t launch_k##MB(const float2*, float2*, int64_t, int64_t, const float2*, const float2*,           \
                             const MixedGeom&, int, int, cudaStream_t);                                     \
    cudaError_t set_smem_k##MB(int bytes);
SAR_MIXED_VARIANT_DECL(2)
SAR_MIXED_VARIANT_DECL(3)
SAR_MIXED_VARIANT_DECL(4)
#undef SAR_MIXED_VARIANT_DECL

// The plain transform (mixed_radix_dft.cu): the forward passes, then natural
// order; the inverse as conj(DFT(conj x)), unnormalised.
cudaError_t launch_dft_mixed(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                             int inverse, const MixedGeom& g, int lines_per_block, int smem, cudaStream_t st);
cudaError_t set_smem_dft(int bytes);

// The compile-time specialisations (mixed_radix_ct.cu): the one of length n
// whose radices and threads per line match g, or nullptr.
typedef cudaError_t (*mixed3_fn)(const float2*, float2*, int64_t, int64_t, const float2*, const float2*, int,
                                 cudaStream_t);
typedef cudaError_t (*mixed3_dft_fn)(const float2*, float2*, int64_t, int64_t, int, const float2*, int, int,
                                     cudaStream_t);
typedef cudaError_t (*mixed3_ct_fn)(const float2*, float2*, int64_t, int64_t, int64_t, const float2*, const float2*,
                                    cudaStream_t);
mixed3_fn specialised(const MixedGeom& g);
mixed3_dft_fn specialised_dft(const MixedGeom& g);
// the folded range pass of a compiled length, or nullptr
mixed3_ct_fn specialised_ct(const MixedGeom& g);
// the second table (mixed_radix_ct2.cu), consulted by the two above
mixed3_fn specialised_more(const MixedGeom& g);
mixed3_dft_fn specialised_dft_more(const MixedGeom& g);
mixed3_ct_fn specialised_ct_more(const MixedGeom& g);
cudaError_t prepare_specialised_more();
cudaError_t prepare_specialised();

}  // namespace mixed
}  // namespace sar
