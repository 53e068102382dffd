// Split-precision helpers shared by the tensor-core DFT kernels: the
// half-precision formats, the split of an FP32 value into a sum of
// half-precision parts, the products kept, and the 16-point DFT roots.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sar_common.cuh"

namespace sar {

enum SplitPrec { kF16x2 = 1, kBF16x2 = 2, kBF16x3 = 3 };

template <int PREC>
struct SplitTraits;
template <>
struct SplitTraits<kF16x2> {
    static constexpr int LEVELS = 2;
    __device__ static uint32_t pack(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __device__ static float2 unpack(uint32_t v) {
        __half2 h = *reinterpret_cast<__half2*>(&v);
        return __half22float2(h);
    }
    __device__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};
struct BF16Base {
    __device__ static uint32_t pack(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __device__ static float2 unpack(uint32_t v) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
        return __bfloat1622float2(h);
    }
    __device__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};
template <>
struct SplitTraits<kBF16x2> : BF16Base {
    static constexpr int LEVELS = 2;
};
template <>
struct SplitTraits<kBF16x3> : BF16Base {
    static constexpr int LEVELS = 3;
};

// Split a pair of floats into LEVELS packed half-precision parts.
template <int PREC>
__device__ __forceinline__ void split2(float a, float b, uint32_t (&out)[3]) {
    using TR = SplitTraits<PREC>;
    float ra = a, rb = b;
#pragma unroll
    for (int l = 0; l < TR::LEVELS; ++l) {
        out[l] = TR::pack(ra, rb);
        const float2 back = TR::unpack(out[l]);
        ra -= back.x;
        rb -= back.y;
    }
}

// Which products of the parts are kept: (level of A, level of B).
template <int LEVELS>
struct Products;
template <>
struct Products<2> {
    static constexpr int COUNT = 3;
    __host__ __device__ static constexpr int a(int p) { return p == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int b(int p) { return p == 1 ? 1 : 0; }
};
template <>
struct Products<3> {
    static constexpr int COUNT = 6;
    // (0,0) (0,1) (1,0) (0,2) (2,0) (1,1)
    __host__ __device__ static constexpr int a(int p) { return p == 2 ? 1 : p == 4 ? 2 : p == 5 ? 1 : 0; }
    __host__ __device__ static constexpr int b(int p) { return p == 1 ? 1 : p == 3 ? 2 : p == 5 ? 1 : 0; }
};

// exp(-2 pi i j / 16), j = 0..15, evaluated at compile time
#define SAR_W16(j) float2{(float)ct::cos2pi(j, 16), (float)(-ct::sin2pi(j, 16))}
static __constant__ float2 kW16[16] = {SAR_W16(0),  SAR_W16(1),  SAR_W16(2),  SAR_W16(3), SAR_W16(4),  SAR_W16(5),
                                SAR_W16(6),  SAR_W16(7),  SAR_W16(8),  SAR_W16(9), SAR_W16(10), SAR_W16(11),
                                SAR_W16(12), SAR_W16(13), SAR_W16(14), SAR_W16(15)};
#undef SAR_W16

}  // namespace sar
