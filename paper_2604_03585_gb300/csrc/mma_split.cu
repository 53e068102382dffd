// Fused line compression with the radix-16 DFTs on the tensor cores, in
// split precision (the paper's Sec. III MMA DFT, Eq. (1)-(2), carried to
// radix 16 and to FP16/BF16 operands with FP32 accumulation).
//
// Every radix-16 stage of the N = 16^P point transform (P = 2 or 3) becomes,
// for 8 groups at a time, the real matrix product
//     [Yr; Yi] = [Fr -Fi; Fi Fr] [Xr; Xi]          (32 x 32 times 32 x 8)
// (Eq. (1)-(2) of the paper for a 16 x 16 DFT matrix F), computed by
// mma.sync.m16n8k16 with FP32 accumulation.  Operands are split into a
// sum of half-precision parts, x = x_hi + x_lo (+ x_mid for BF16 x3), and
// the products hi*hi + hi*lo + lo*hi (BF16 x3: hh + hm + mh + hl + lh + mm)
// recover close to FP32 accuracy.  Each group (one column) is scaled by a
// power of two to |x| < 1 before the split, so FP16 can neither overflow nor
// lose the low part, and unscaled after the product (both exact).  Twiddles,
// the filter multiply and the 1/N stay in FP32.
//
// The line lives in shared memory (the padded in-place layout of the FP32
// engine); each stage reads its groups in the B-fragment layout, multiplies,
// and writes the outputs from the D-fragment layout back to the same
// positions.  One block per line, WARPS warps, 8 groups per warp per step.
#include "../../include/sar.h"
#include "line_engine.cuh"
#include "split_prec.cuh"
#include "registry.h"
#include "tables.h"

namespace sar {

// A fragments of the DFT16 matrix pieces: [level][Fr, Fi, -Fi][4 regs].
template <int PREC>
struct AFrags {
    uint32_t r[3][3][4];
};

template <int PREC>
__device__ __forceinline__ void load_afrags(AFrags<PREC>& A, int lane) {
    const int gid = lane >> 2, tig = lane & 3;
    // fragment register q holds (row, col) pairs:
    //   q0: (gid, 2tig..+1)  q1: (gid+8, 2tig..+1)  q2: (gid, 2tig+8..+9)  q3: (gid+8, 2tig+8..+9)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int row = gid + ((q & 1) ? 8 : 0);
        const int col = 2 * tig + ((q & 2) ? 8 : 0);
        float fr[2], fi[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            // F[m][k] = exp(-2 pi i m k / 16)
            const float2 w = kW16[(row * (col + j)) & 15];
            fr[j] = w.x;
            fi[j] = w.y;
        }
        uint32_t pr[3], pi[3], pn[3];
        split2<PREC>(fr[0], fr[1], pr);
        split2<PREC>(fi[0], fi[1], pi);
        split2<PREC>(-fi[0], -fi[1], pn);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            A.r[l][0][q] = pr[l];
            A.r[l][1][q] = pi[l];
            A.r[l][2][q] = pn[l];
        }
    }
}

// One 8-group step: X (this lane: group gid, elements k = 2tig, 2tig+1,
// 2tig+8, 2tig+9) -> Y (this lane: elements gid, gid+8 of groups 2tig, 2tig+1).
// INV uses conj(F).  Each group is scaled by 2^-e (e from the group's max).
template <int PREC, bool INV>
__device__ __forceinline__ void dft16_mma(const AFrags<PREC>& A, const float2 (&x)[4], float (&yr)[4],
                                          float (&yi)[4], int lane) {
    using TR = SplitTraits<PREC>;
    const int tig = lane & 3;
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) m = fmaxf(m, fmaxf(fabsf(x[j].x), fabsf(x[j].y)));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    const int e = (m > 0.f) ? ilogbf(m) + 1 : 0;
    const float inv = ldexpf(1.f, -e);
    uint32_t br[3][2], bi[3][2];
    {
        uint32_t t0[3], t1[3];
        split2<PREC>(x[0].x * inv, x[1].x * inv, t0);
        split2<PREC>(x[2].x * inv, x[3].x * inv, t1);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            br[l][0] = t0[l];
            br[l][1] = t1[l];
        }
        split2<PREC>(x[0].y * inv, x[1].y * inv, t0);
        split2<PREC>(x[2].y * inv, x[3].y * inv, t1);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            bi[l][0] = t0[l];
            bi[l][1] = t1[l];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) yr[j] = yi[j] = 0.f;
    using PR = Products<TR::LEVELS>;
#pragma unroll
    for (int p = 0; p < PR::COUNT; ++p) {
        const int la = PR::a(p), lb = PR::b(p);
        if (!INV) {
            // Yr = Fr Xr - Fi Xi ; Yi = Fi Xr + Fr Xi
            TR::mma(yr, A.r[la][0], br[lb][0], br[lb][1]);
            TR::mma(yr, A.r[la][2], bi[lb][0], bi[lb][1]);
            TR::mma(yi, A.r[la][1], br[lb][0], br[lb][1]);
            TR::mma(yi, A.r[la][0], bi[lb][0], bi[lb][1]);
        } else {
            // conj(F): Yr = Fr Xr + Fi Xi ; Yi = Fr Xi - Fi Xr
            TR::mma(yr, A.r[la][0], br[lb][0], br[lb][1]);
            TR::mma(yr, A.r[la][1], bi[lb][0], bi[lb][1]);
            TR::mma(yi, A.r[la][2], br[lb][0], br[lb][1]);
            TR::mma(yi, A.r[la][0], bi[lb][0], bi[lb][1]);
        }
    }
    // unscale: output columns are groups 2tig, 2tig+1 (their lanes: 4 * group)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int ec = __shfl_sync(0xffffffffu, e, 4 * (2 * tig + c));
        const float sc = ldexpf(1.f, ec);
        yr[c] *= sc;
        yi[c] *= sc;
        yr[c + 2] *= sc;
        yi[c + 2] *= sc;
    }
}

template <int N>
struct MmaGeom {
    static constexpr int P = (N == 4096) ? 3 : 2;
    static constexpr int G = N / 16;   // groups per pass
    static constexpr int NT = G / 8;   // 8-group steps per pass
    static constexpr int ELEMS = N + N / 16;
};

// One middle pass (shared memory -> shared memory) of stride S.
template <int N, int PREC, bool INV, bool TWID>
__device__ __forceinline__ void mma_pass(const AFrags<PREC>& A, float2* sm, int S, const float2* tw, int warp,
                                         int warps, int lane) {
    const int gid = lane >> 2, tig = lane & 3;
    for (int nt = warp; nt < MmaGeom<N>::NT; nt += warps) {
        const int n = 8 * nt + gid;
        const int base = (n / S) * (16 * S) + (n % S), lo = n % S;
        float2 x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 2 * tig + (j & 1) + ((j & 2) ? 8 : 0);
            x[j] = sm[smem_pos(base + k * S, 4)];
            if (INV && TWID && k > 0) x[j] = cmulc(x[j], tw[k * S + lo]);
        }
        float yr[4], yi[4];
        dft16_mma<PREC, INV>(A, x, yr, yi, lane);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int nn = 8 * nt + 2 * tig + (q & 1);
            const int row = gid + ((q & 2) ? 8 : 0);
            const int bnn = (nn / S) * (16 * S) + (nn % S);
            float2 y = make_float2(yr[q], yi[q]);
            if (!INV && TWID && row > 0) y = cmul(y, tw[row * S + (nn % S)]);
            sm[smem_pos(bnn + row * S, 4)] = y;
        }
    }
}

template <int N, int PREC>
__global__ void __launch_bounds__(128)
mma_compress_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt_pos,
                    const float2* tw) {
    extern __shared__ float2 sm[];
    using GM = MmaGeom<N>;
    const int64_t line = blockIdx.x;
    if (line >= n_lines) return;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31, warps = blockDim.x >> 5;
    AFrags<PREC> A;
    load_afrags<PREC>(A, lane);
    const float2* src = in + line * ld;
    for (int i = t; i < N; i += blockDim.x) sm[smem_pos(i, 4)] = __ldcs(src + i);
    __syncthreads();
    // forward passes with twiddles: strides N/16, N/256 (three passes)
    mma_pass<N, PREC, false, true>(A, sm, N / 16, tw, warp, warps, lane);
    __syncthreads();
    if constexpr (GM::P == 3) {
        mma_pass<N, PREC, false, true>(A, sm, 16, tw + 16 * (N / 16), warp, warps, lane);
        __syncthreads();
    }
    // last forward pass (stride 1), filter, first inverse pass, per 8 groups
    {
        const int gid = lane >> 2, tig = lane & 3;
        for (int nt = warp; nt < GM::NT; nt += warps) {
            float2 x[4];
            const int n = 8 * nt + gid;
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = sm[smem_pos(16 * n + 2 * tig + (j & 1) + ((j & 2) ? 8 : 0), 4)];
            float yr[4], yi[4];
            dft16_mma<PREC, false>(A, x, yr, yi, lane);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int nn = 8 * nt + 2 * tig + (q & 1);
                const int pos = 16 * nn + gid + ((q & 2) ? 8 : 0);
                sm[smem_pos(pos, 4)] = cmul(make_float2(yr[q], yi[q]), filt_pos[pos]);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = sm[smem_pos(16 * n + 2 * tig + (j & 1) + ((j & 2) ? 8 : 0), 4)];
            dft16_mma<PREC, true>(A, x, yr, yi, lane);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int nn = 8 * nt + 2 * tig + (q & 1);
                sm[smem_pos(16 * nn + gid + ((q & 2) ? 8 : 0), 4)] = make_float2(yr[q], yi[q]);
            }
        }
    }
    __syncthreads();
    if constexpr (GM::P == 3) {
        mma_pass<N, PREC, true, true>(A, sm, 16, tw + 16 * (N / 16), warp, warps, lane);
        __syncthreads();
    }
    mma_pass<N, PREC, true, true>(A, sm, N / 16, tw, warp, warps, lane);
    __syncthreads();
    float2* dst = out + line * ld;
    for (int i = t; i < N; i += blockDim.x) __stcs(dst + i, sm[smem_pos(i, 4)]);
}

template <int N, int PREC>
cudaError_t launch_mma(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt_pos,
                       const float2* tw, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    constexpr int smem = MmaGeom<N>::ELEMS * 8;
    constexpr int threads = (N == 4096) ? 128 : 32;
    static bool attr_set = false;
    if (!attr_set && smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(mma_compress_kernel<N, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    mma_compress_kernel<N, PREC><<<(unsigned)n_lines, threads, smem, st>>>(in, out, n_lines, ld, filt_pos, tw);
    return cudaGetLastError();
}

cudaError_t launch_mma_compress(int n, int prec, const float2* in, float2* out, int64_t n_lines, int64_t ld,
                                const float2* filt_pos, const float2* tw, cudaStream_t st) {
    if (n == 4096) {
        if (prec == kF16x2) return launch_mma<4096, kF16x2>(in, out, n_lines, ld, filt_pos, tw, st);
        if (prec == kBF16x2) return launch_mma<4096, kBF16x2>(in, out, n_lines, ld, filt_pos, tw, st);
        if (prec == kBF16x3) return launch_mma<4096, kBF16x3>(in, out, n_lines, ld, filt_pos, tw, st);
    } else if (n == 256) {
        if (prec == kF16x2) return launch_mma<256, kF16x2>(in, out, n_lines, ld, filt_pos, tw, st);
        if (prec == kBF16x2) return launch_mma<256, kBF16x2>(in, out, n_lines, ld, filt_pos, tw, st);
        if (prec == kBF16x3) return launch_mma<256, kBF16x3>(in, out, n_lines, ld, filt_pos, tw, st);
    }
    return cudaErrorInvalidValue;
}

// Position-order filter index of an all-radix-16 transform: position
// P = sum k_i 16^(p-i) holds frequency k = k_1 + 16 k_2 (+ 256 k_3).
void mma_filter_positions(int n, int32_t* idx) {
    const int p = (n == 4096) ? 3 : 2;
    for (int P = 0; P < n; ++P) {
        int rem = P, k = 0, mul = 1;
        int digits[3];
        for (int i = p - 1; i >= 0; --i) {
            digits[i] = rem % 16;
            rem /= 16;
        }
        for (int i = 0; i < p; ++i) {
            k += digits[i] * mul;
            mul *= 16;
        }
        idx[P] = k;
    }
}

}  // namespace sar
