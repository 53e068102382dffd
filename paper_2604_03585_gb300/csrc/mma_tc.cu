// Fused line compression with every radix-16 DFT on the fifth-generation
// tensor cores: tcgen05.mma with the accumulators in tensor memory (TMEM), in
// split precision (the paper's Sec. III MMA DFT, Eq. (1)-(2), carried to
// radix 16 and to FP16 / BF16 operand parts with FP32 accumulation).
//
// The contraction is arranged for the tensor core's shape.  A radix-16 stage
// applies the 16-point DFT F to every group x of 16 complex samples; written
// in reals with (re, im) interleaved, y = F x is a 32 x 32 real matrix times
// a 32-vector.  Stacking the groups of a pass as rows gives
//     Y = X F^T          (128 groups x 32) = (128 x 32)(32 x 32)
// one tcgen05.mma shape with M = 128 (groups), N = 32, K = 32 (two K = 16
// steps).  X is split per group into half-precision parts
// x = 2^e (x_hi + x_lo [+ x_mid]), for FP16 after scaling each group by a
// power of two to |x| < 1 (BF16 has FP32's exponent range: e = 0),
// F into f_hi + f_lo [+ f_mid], and the products
// hi*hi + hi*lo + lo*hi (BF16 x3: hh + hm + mh + hl + lh + mm) accumulate in
// FP32 in TMEM.  Row m of the accumulator is TMEM lane m, so after the MMA
// thread t reads its own group's 16 complex outputs from lane t with one
// tcgen05.ld: the operand layout and the engine's one-group-per-thread layout
// coincide, and no fragment shuffling is needed.
//
// Operands are in this CTA's shared memory in the canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, K-adjacent ones 128 bytes
// apart (LBO), row-group-adjacent ones 512 bytes apart (SBO).  A tiles are
// rewritten by the threads every stage (generic-proxy stores, then a proxy
// fence and a block barrier before one thread issues the MMAs); the B tiles
// (F^T and conj(F)^T at every split level) are written once per block.  One
// thread issues the MMAs and commits them to an mbarrier; every thread waits
// on it (bounded by wait_cycles SM clocks: on a timeout the block records
// status 5, skips the remaining stages, frees its TMEM and returns).
//
// Line geometry: the in-place decimation-in-frequency of the FP32 engine, all
// radix 16 (N = 16^P): pass i works on groups at stride S = N / 16^(i+1),
// twiddles after the forward DFT and before the inverse one, the filter in
// position order between the last forward and the first inverse DFT, 1/N
// folded into the filter.  N = 4096: one line per block, 256 groups (two M
// tiles, 64 TMEM columns); N = 256: eight lines per block, 128 groups (one
// tile, 32 columns).  128 threads, thread t owns group t of every tile.
#include "../../include/sar.h"
#include "line_engine.cuh"
#include "persistent.cuh"
#include "split_prec.cuh"

namespace sar {
namespace {

// ---- tcgen05 (cta_group::1) -------------------------------------------------
__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16 (F16 or BF16 in, F32 out)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the same with A read from tensor memory: K = 16 16-bit elements of row m
// in lane m, columns a .. a + 7 (two elements per 32-bit column, the even K
// index in the low half)
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 16 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// the mbarrier completes one arrival once every MMA this thread issued is done
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
          "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]),
          "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]),
          "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
        : "r"(taddr)
        : "memory");
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: F16 = 0, BF16 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
template <int PREC>
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t m, uint32_t n) {
    constexpr uint32_t fmt = (PREC == kF16x2) ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading and
// stride byte offsets (each >> 4, 14 bits), descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// byte offset of (row, k) in a K-major tile of K = 32 16-bit elements:
// core matrix (row / 8, k / 8) of 8 rows x 16 bytes, 4 per row group
__host__ __device__ constexpr uint32_t km_off(int row, int k) {
    return (uint32_t)(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
constexpr uint32_t kLBO = 128, kSBO = 512;
constexpr uint32_t kATile = 128 * 64;   // 128 rows x 32 K x 2 bytes
constexpr uint32_t kBTile = 32 * 64;    // 32 rows (N) x 32 K x 2 bytes

constexpr uint32_t pow2_at_least(uint32_t v) {
    uint32_t p = 32;
    while (p < v) p <<= 1;
    return p;
}

// ATM: A operand (the split groups) in tensor memory instead of shared memory
template <int N, int PREC, bool ATM>
struct TcGeom {
    static constexpr int LV = SplitTraits<PREC>::LEVELS;
    static constexpr int P = (N == 4096) ? 3 : 2;
    static constexpr int LPB = (N == 4096) ? 1 : 8;   // lines per block
    static constexpr int G = N / 16;                  // groups per line and pass
    static constexpr int GT = G * LPB;                // groups per block and pass
    static constexpr int MT = GT / 128;               // M tiles
    static constexpr int LINE = N + N / 16;           // padded line (one slot per 16)
    static constexpr uint32_t OFF_A = ((LPB * LINE * 8 + 1023) / 1024) * 1024;
    static constexpr uint32_t OFF_B = OFF_A + (ATM ? 0 : MT * LV * kATile);
    static constexpr uint32_t OFF_BAR = OFF_B + 2 * LV * kBTile;
    static constexpr uint32_t SMEM = OFF_BAR + 16;
    // TMEM columns: the accumulators (32 per M tile), then with ATM the A
    // operands (16 columns per tile and split level: 32 16-bit K elements)
    static constexpr uint32_t ACOL = MT * 32;
    static constexpr uint32_t TCOLS = pow2_at_least(ATM ? ACOL + MT * LV * 16 : ACOL);
    static constexpr int MINB = ATM ? (int)(512 / TCOLS) : 1;   // blocks per SM the TMEM allows
    static_assert(GT % 128 == 0, "whole M tiles");
};

// Split one FP32 value into LV half-precision parts (16-bit patterns).
template <int PREC>
__device__ __forceinline__ void split1(float v, uint16_t (&out)[3]) {
    using TR = SplitTraits<PREC>;
    float r = v;
#pragma unroll
    for (int l = 0; l < TR::LEVELS; ++l) {
        const uint32_t p = TR::pack(r, 0.f);
        out[l] = (uint16_t)(p & 0xFFFFu);
        r -= TR::unpack(p).x;
    }
}

template <int N, int PREC, bool ATM>
__global__ void __launch_bounds__(128, TcGeom<N, PREC, ATM>::MINB)
mma_tc_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt_pos, const float2* tw,
              int* status, long long wait_cycles) {
    using GM = TcGeom<N, PREC, ATM>;
    using TR = SplitTraits<PREC>;
    using PR = Products<GM::LV>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* lines = reinterpret_cast<float2*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + GM::OFF_BAR);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(smem_raw + GM::OFF_BAR + 8);
    const int t = threadIdx.x, warp = t >> 5;
    const int64_t line0 = (int64_t)blockIdx.x * GM::LPB;

    if (warp == 0) {
        tc_alloc(s_taddr, GM::TCOLS);
        tc_relinquish();
    }
    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    // B tiles: F^T (forward) and conj(F)^T (inverse) at every split level.
    // Real row k = 2q (+1 for Im x_q) and column n = 2j (+1 for Im y_j) of
    // the 32 x 32 matrix [Re F, -Im F; Im F, Re F], stored K-major as [n][k].
    for (int e = t; e < 2 * 32 * 32; e += 128) {
        const int dir = e >> 10, n = (e >> 5) & 31, k = e & 31;
        const int q = k >> 1, j = n >> 1;
        const float2 w = kW16[(j * q) & 15];   // exp(-2 pi i j q / 16)
        const float c = w.x, s = dir ? -w.y : w.y;
        const float v = (k & 1) == 0 ? ((n & 1) == 0 ? c : s) : ((n & 1) == 0 ? -s : c);
        uint16_t parts[3];
        split1<PREC>(v, parts);
#pragma unroll
        for (int l = 0; l < GM::LV; ++l)
            *reinterpret_cast<uint16_t*>(smem_raw + GM::OFF_B + (dir * GM::LV + l) * kBTile + km_off(n, k)) = parts[l];
    }
    // the lines (zeros for lines past the end)
    for (int l = 0; l < GM::LPB; ++l) {
        const bool have = line0 + l < n_lines;
        const float2* src = in + (line0 + l) * ld;
        for (int i = t; i < N; i += 128)
            lines[l * GM::LINE + smem_pos(i, 4)] = have ? __ldcs(src + i) : make_float2(0.f, 0.f);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *s_taddr;
    const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
    const uint32_t sbase = smem_u32(smem_raw);
    constexpr uint32_t idesc = tc_idesc<PREC>(128, 32);
    uint32_t phase = 0;
    bool ok = true;

    // y = F x (or conj(F) x) for the MT groups of this thread, in place.
    auto dft_round = [&](float2 (&x)[GM::MT][16], bool inv) {
        // FP16 parts need each group scaled into range (a power of two, exact);
        // BF16 has FP32's exponent range and takes the values as they are
        constexpr bool SCALE = PREC == kF16x2;
        int ex[GM::MT];
#pragma unroll
        for (int mt = 0; mt < GM::MT; ++mt) {
            float sc = 1.f;
            ex[mt] = 0;
            if constexpr (SCALE) {
                float m = 0.f;
#pragma unroll
                for (int j = 0; j < 16; ++j) m = fmaxf(m, fmaxf(fabsf(x[mt][j].x), fabsf(x[mt][j].y)));
                ex[mt] = (m > 0.f) ? ilogbf(m) + 1 : 0;
                sc = ldexpf(1.f, -ex[mt]);
            }
            if constexpr (ATM) {
                // row t of the A operand: lane t, 16 columns per split level
                uint32_t v[3][16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    uint32_t pk[3];
                    split2<PREC>(x[mt][j].x * sc, x[mt][j].y * sc, pk);
#pragma unroll
                    for (int l = 0; l < GM::LV; ++l) v[l][j] = pk[l];
                }
#pragma unroll
                for (int l = 0; l < GM::LV; ++l) tc_st16(tlane + GM::ACOL + (mt * GM::LV + l) * 16, v[l]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) {   // K elements 8c .. 8c+7: complex 4c .. 4c+3
                    uint32_t pk[4][3];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        split2<PREC>(x[mt][4 * c + u].x * sc, x[mt][4 * c + u].y * sc, pk[u]);
#pragma unroll
                    for (int l = 0; l < GM::LV; ++l)
                        *reinterpret_cast<uint4*>(smem_raw + GM::OFF_A + (mt * GM::LV + l) * kATile +
                                                  km_off(t, 8 * c)) = make_uint4(pk[0][l], pk[1][l], pk[2][l], pk[3][l]);
                }
            }
        }
        if constexpr (ATM)
            tc_wait_st();
        else
            fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0 && ok) {
            tc_fence_after();
#pragma unroll
            for (int mt = 0; mt < GM::MT; ++mt) {
#pragma unroll
                for (int p = 0; p < PR::COUNT; ++p) {
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const uint32_t b = sbase + GM::OFF_B + ((inv ? 1 : 0) * GM::LV + PR::b(p)) * kBTile + s * 256;
                        if constexpr (ATM) {
                            tc_mma_ts(tbase + 32 * mt, tbase + GM::ACOL + (mt * GM::LV + PR::a(p)) * 16 + 8 * s,
                                      tc_sdesc(b, kLBO, kSBO), idesc, (p > 0 || s > 0) ? 1u : 0u);
                        } else {
                            const uint32_t a = sbase + GM::OFF_A + (mt * GM::LV + PR::a(p)) * kATile + s * 256;
                            tc_mma(tbase + 32 * mt, tc_sdesc(a, kLBO, kSBO), tc_sdesc(b, kLBO, kSBO), idesc,
                                   (p > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                }
            }
            tc_commit(bar);
        }
        if (ok && !mbar_wait_bounded(bar, phase, wait_cycles)) ok = false;
        ok = __syncthreads_and(ok) != 0;   // one decision for the whole block
        phase ^= 1u;
        tc_fence_after();
        if (!ok) return;
#pragma unroll
        for (int mt = 0; mt < GM::MT; ++mt) {
            float d[32];
            tc_ld32(tlane + 32 * mt, d);
            if constexpr (SCALE) {
                const float sc = ldexpf(1.f, ex[mt]);
#pragma unroll
                for (int j = 0; j < 16; ++j) x[mt][j] = make_float2(d[2 * j] * sc, d[2 * j + 1] * sc);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) x[mt][j] = make_float2(d[2 * j], d[2 * j + 1]);
            }
        }
        tc_fence_before();
    };

    // group gt of the block at stride S: group gt % G of line gt / G, whose
    // elements sit at positions base + k*S of that line
    auto base_of = [&](int gt, int S, int& lo) {
        const int g = gt % GM::G;
        lo = g % S;
        return (g / S) * (16 * S) + lo;
    };
    auto line_of = [&](int gt) { return lines + (gt / GM::G) * GM::LINE; };

    float2 x[GM::MT][16];
    // forward passes
#pragma unroll 1
    for (int pass = 0, S = N / 16; pass < GM::P && ok; ++pass, S /= 16) {
        const float2* twp = tw + (pass == 0 ? 0 : 16 * (N / 16));
        int lo[GM::MT], b[GM::MT];
#pragma unroll
        for (int mt = 0; mt < GM::MT; ++mt) {
            b[mt] = base_of(t + 128 * mt, S, lo[mt]);
            const float2* L = line_of(t + 128 * mt);
#pragma unroll
            for (int k = 0; k < 16; ++k) x[mt][k] = L[smem_pos(b[mt] + k * S, 4)];
        }
        dft_round(x, false);
        if (!ok) break;
        if (S > 1) {
#pragma unroll
            for (int mt = 0; mt < GM::MT; ++mt)
#pragma unroll
                for (int k = 1; k < 16; ++k) x[mt][k] = cmul(x[mt][k], twp[k * S + lo[mt]]);
        } else {
            // last pass: filter (position order, 1/N folded in), then the
            // first inverse DFT on the same groups
#pragma unroll
            for (int mt = 0; mt < GM::MT; ++mt)
#pragma unroll
                for (int k = 0; k < 16; ++k) x[mt][k] = cmul(x[mt][k], filt_pos[b[mt] + k]);
            dft_round(x, true);
            if (!ok) break;
        }
#pragma unroll
        for (int mt = 0; mt < GM::MT; ++mt) {
            float2* L = line_of(t + 128 * mt);
#pragma unroll
            for (int k = 0; k < 16; ++k) L[smem_pos(b[mt] + k * S, 4)] = x[mt][k];
        }
        __syncthreads();
    }
    // inverse passes (strides 16, ..., N/16): conjugate twiddles, then the DFT
#pragma unroll 1
    for (int pass = GM::P - 2, S = 16; pass >= 0 && ok; --pass, S *= 16) {
        const float2* twp = tw + (pass == 0 ? 0 : 16 * (N / 16));
        int lo[GM::MT], b[GM::MT];
#pragma unroll
        for (int mt = 0; mt < GM::MT; ++mt) {
            b[mt] = base_of(t + 128 * mt, S, lo[mt]);
            const float2* L = line_of(t + 128 * mt);
#pragma unroll
            for (int k = 0; k < 16; ++k) x[mt][k] = L[smem_pos(b[mt] + k * S, 4)];
#pragma unroll
            for (int k = 1; k < 16; ++k) x[mt][k] = cmulc(x[mt][k], twp[k * S + lo[mt]]);
        }
        dft_round(x, true);
        if (!ok) break;
#pragma unroll
        for (int mt = 0; mt < GM::MT; ++mt) {
            float2* L = line_of(t + 128 * mt);
#pragma unroll
            for (int k = 0; k < 16; ++k) L[smem_pos(b[mt] + k * S, 4)] = x[mt][k];
        }
        __syncthreads();
    }
    if (ok) {
        for (int l = 0; l < GM::LPB; ++l) {
            if (line0 + l >= n_lines) break;
            float2* dst = out + (line0 + l) * ld;
            for (int i = t; i < N; i += 128) __stcs(dst + i, lines[l * GM::LINE + smem_pos(i, 4)]);
        }
    } else if (t == 0) {
        atomicMax(status, 5);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tbase, GM::TCOLS);
}

template <int N, int PREC, bool ATM>
cudaError_t launch_tc(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt_pos,
                      const float2* tw, int* status, long long wait_cycles, cudaStream_t st) {
    using GM = TcGeom<N, PREC, ATM>;
    if (n_lines <= 0) return cudaSuccess;
    static int attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(mma_tc_kernel<N, PREC, ATM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)GM::SMEM);
        if (e != cudaSuccess) return e;
        attr_set[dev] = 1;
    }
    const int64_t blocks = (n_lines + GM::LPB - 1) / GM::LPB;
    mma_tc_kernel<N, PREC, ATM><<<(unsigned)blocks, 128, GM::SMEM, st>>>(in, out, n_lines, ld, filt_pos, tw, status,
                                                                         wait_cycles);
    return cudaGetLastError();
}

template <int N, int PREC>
cudaError_t launch_tc_any(bool atm, const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt_pos,
                          const float2* tw, int* status, long long wait_cycles, cudaStream_t st) {
    return atm ? launch_tc<N, PREC, true>(in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st)
               : launch_tc<N, PREC, false>(in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
}

}  // namespace

cudaError_t launch_mma_tc_compress(int n, int prec, bool a_in_tmem, const float2* in, float2* out, int64_t n_lines,
                                   int64_t ld, const float2* filt_pos, const float2* tw, int* status,
                                   long long wait_cycles, cudaStream_t st) {
    const bool a = a_in_tmem;
    if (n == 4096) {
        if (prec == kF16x2) return launch_tc_any<4096, kF16x2>(a, in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
        if (prec == kBF16x2) return launch_tc_any<4096, kBF16x2>(a, in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
        if (prec == kBF16x3) return launch_tc_any<4096, kBF16x3>(a, in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
    } else if (n == 256) {
        if (prec == kF16x2) return launch_tc_any<256, kF16x2>(a, in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
        if (prec == kBF16x2) return launch_tc_any<256, kBF16x2>(a, in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
        if (prec == kBF16x3) return launch_tc_any<256, kBF16x3>(a, in, out, n_lines, ld, filt_pos, tw, status, wait_cycles, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sar
