// Common device helpers for the GB300 SAR compression kernels: complex
// float arithmetic and compile-time twiddle constants.
//
// Twiddle constants used inside the register-resident DFTs are evaluated at
// compile time from their own Taylor series (no library sin/cos), after an
// exact octant reduction of the dyadic angle 2*pi*m/L.  Larger tables are
// generated on the device in FP64 with sincospi() and rounded to FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>

namespace sar {

// ---------------------------------------------------------------------------
// complex float helpers (float2 = interleaved complex64)
// ---------------------------------------------------------------------------
// Complex add and subtract as one packed two-wide FP32 instruction each
// (add / sub .f32x2, sm_100 and later): both halves round exactly as the
// scalar operations do, with half the instructions issued.
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward quarter turn) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 cmul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// compile-time sin/cos of 2*pi*m/L (L a power of two), from the Taylor series
// ---------------------------------------------------------------------------
namespace ct {
constexpr double kPi = 3.14159265358979323846264338327950288;

// sin and cos of theta in [0, pi/4] by their Maclaurin series, summed until
// the terms vanish in double precision (at most ~15 terms here).
__host__ __device__ constexpr double taylor_sin(double t) {
    double term = t, sum = t;
    for (int k = 1; k < 30; ++k) {
        term *= -t * t / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double t) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -t * t / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}
// cos(2 pi f) and sin(2 pi f) for a dyadic fraction f in [0, 1).  Each
// reduction step (half turn, quarter turn, reflection about pi/4) subtracts
// dyadic rationals exactly, so only the final series on [0, pi/4] rounds.
__host__ __device__ constexpr double sin2pi_f(double f);
__host__ __device__ constexpr double cos2pi_f(double f) {
    return f >= 0.5    ? -cos2pi_f(f - 0.5)
           : f >= 0.25 ? -sin2pi_f(f - 0.25)
           : f > 0.125 ? sin2pi_f(0.25 - f)
                       : taylor_cos(2.0 * kPi * f);
}
__host__ __device__ constexpr double sin2pi_f(double f) {
    return f >= 0.5    ? -sin2pi_f(f - 0.5)
           : f >= 0.25 ? cos2pi_f(f - 0.25)
           : f > 0.125 ? cos2pi_f(0.25 - f)
                       : taylor_sin(2.0 * kPi * f);
}
__host__ __device__ constexpr double cos2pi(long long m, long long L) {
    return cos2pi_f(double(((m % L) + L) % L) / double(L));
}
__host__ __device__ constexpr double sin2pi(long long m, long long L) {
    return sin2pi_f(double(((m % L) + L) % L) / double(L));
}
}  // namespace ct

// x * W_L^{M}   (forward, W_L = exp(-2 pi i / L))
// x * W_L^{-M}  (inverse)
// Exact quarter turns cost nothing; everything else is one complex multiply
// by compile-time constants (two FMUL + two FFMA).
template <int L, int M, bool INV>
__device__ __forceinline__ float2 twiddle_ct(float2 x) {
    constexpr int m = ((M % L) + L) % L;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (2 * m == L) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (4 * m == L) {
        return cmul_mi<INV>(x);
    } else if constexpr (4 * m == 3 * L) {
        return cmul_mi<!INV>(x);
    } else {
        constexpr float c = (float)ct::cos2pi(m, L);
        constexpr float s = (float)(INV ? ct::sin2pi(m, L) : -ct::sin2pi(m, L));
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    }
}

// ---------------------------------------------------------------------------
// register-resident DFT of size R (a power of two), in place, natural order
// ---------------------------------------------------------------------------
// Radix-4 (and a final radix-2 where needed) decimation in frequency over a
// float2[R] array with compile-time indices only, so the array never leaves
// registers.  The DIF leaves X[k] at position dif_pos(R, k); the caller reads
// results through that permutation, which costs nothing after unrolling.
__host__ __device__ constexpr int dif_pos(int L, int k) {
    return L == 1 ? 0 : (L == 2 ? (k & 1) : ((k % 4) * (L / 4) + dif_pos(L / 4, k / 4)));
}

template <int R, int L, int OFF, bool INV, int J>
__device__ __forceinline__ void dif4_one(float2 (&v)[R]) {
    constexpr int Q = L / 4;
    const float2 a = v[OFF + J], b = v[OFF + J + Q], c = v[OFF + J + 2 * Q], d = v[OFF + J + 3 * Q];
    const float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d);
    const float2 t3 = cmul_mi<INV>(csub(b, d));
    v[OFF + J] = cadd(t0, t2);
    v[OFF + J + Q] = twiddle_ct<L, J, INV>(cadd(t1, t3));
    v[OFF + J + 2 * Q] = twiddle_ct<L, 2 * J, INV>(csub(t0, t2));
    v[OFF + J + 3 * Q] = twiddle_ct<L, 3 * J, INV>(csub(t1, t3));
}

template <int R, int L, int OFF, bool INV, int... J>
__device__ __forceinline__ void dif4_level(float2 (&v)[R], std::integer_sequence<int, J...>) {
    (dif4_one<R, L, OFF, INV, J>(v), ...);
}

template <int R, int L, int OFF, bool INV>
__device__ __forceinline__ void dif_rec(float2 (&v)[R]) {
    if constexpr (L == 2) {
        const float2 a = v[OFF], b = v[OFF + 1];
        v[OFF] = cadd(a, b);
        v[OFF + 1] = csub(a, b);
    } else if constexpr (L >= 4) {
        constexpr int Q = L / 4;
        dif4_level<R, L, OFF, INV>(v, std::make_integer_sequence<int, Q>{});
        dif_rec<R, Q, OFF, INV>(v);
        dif_rec<R, Q, OFF + Q, INV>(v);
        dif_rec<R, Q, OFF + 2 * Q, INV>(v);
        dif_rec<R, Q, OFF + 3 * Q, INV>(v);
    }
}

template <int R, int... K>
__device__ __forceinline__ void unscramble(const float2 (&v)[R], float2 (&o)[R], std::integer_sequence<int, K...>) {
    ((o[K] = v[dif_pos(R, K)]), ...);
}

// v[k] <- sum_n v[n] exp(-+2 pi i n k / R)   (unnormalised; INV selects +)
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    static_assert(R >= 1 && (R & (R - 1)) == 0, "radix must be a power of two");
    if constexpr (R > 1) {
        dif_rec<R, R, 0, INV>(v);
        float2 o[R];
        unscramble<R>(v, o, std::make_integer_sequence<int, R>{});
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = o[k];
    }
}

}  // namespace sar
