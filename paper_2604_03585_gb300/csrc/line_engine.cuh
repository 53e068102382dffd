// Line FFT engine: one thread group per line, the line held in registers
// between shared-memory exchanges.
//
// A length-N line (N a power of two) is transformed by P = 2 or 3 passes of
// radices R1, R2[, R3] (N = R1*R2[*R3]) in the in-place Cooley-Tukey
// decimation-in-frequency order.  With strides S_i = N / (R1*...*R_i), pass i
// applies an R_i-point DFT to every group of R_i elements at positions
// base + r*S_i and then multiplies element r by W_{R_i S_i}^{lo*r}, where lo
// is the group's offset below S_i.  Positions never move: after the last
// pass, position P = sum_i k_i S_i holds X[k_1 + R1 k_2 + R1 R2 k_3]
// (digit-reversed order).  Each thread owns E = N/T elements and handles E/R_i
// groups per pass; between passes the line goes through shared memory,
// padded with one slot per R_P elements so that every 64-bit warp access
// needs the minimum two wavefronts.
//
// The fused line compression (Sec. II-B of the paper: load, FFT, multiply by
// the matched filter, IFFT, store; two device-memory transfers per line) runs
// the forward passes, multiplies the digit-reversed spectrum by a filter
// stored in exactly that order with 1/N folded in, and runs the inverse as the
// mirror image: conjugate twiddles before each inverse DFT, passes in reverse
// order, ending in natural order.  The inverse's first pass uses the same
// groups as the forward's last pass, so the spectrum never leaves registers
// between the two.  This yields the same values as the paper's
// conjugate-FFT-conjugate inverse (Sec. II-C) without any reordering pass.
#pragma once

#include "sar_common.cuh"

namespace sar {

template <int N_, int E_, int R1_, int R2_, int R3_ = 1, int MINB_ = 0>
struct Sched {
    static constexpr int N = N_, E = E_, T = N_ / E_;
    static constexpr int MINB = MINB_;   // > 0: registers capped for MINB resident blocks per SM
    static constexpr int R1 = R1_, R2 = R2_, R3 = R3_;
    static constexpr int P = (R3_ > 1) ? 3 : 2;
    static constexpr int S1 = N / R1, S2 = S1 / R2, S3 = (P == 3) ? S2 / R3 : 0;
    static constexpr int RL = (P == 3) ? R3 : R2;                 // radix of the last pass
    static constexpr int PADSH = (RL == 16) ? 4 : (RL == 32) ? 5 : (RL == 64) ? 6 : (RL == 8) ? 3 : (RL == 4) ? 2 : 7;
    static constexpr int SMEM_ELEMS = N + (N >> PADSH);            // per line
    static constexpr int TW_ELEMS = R1 * S1 + ((P == 3) ? R2 * S2 : 0);  // twiddle table length
    static_assert(R1 * R2 * R3 == N, "radices must multiply to N");
    static_assert(E % R1 == 0 && E % R2 == 0 && E % R3 == 0, "each radix must divide E");
    static_assert((1 << PADSH) == RL, "unsupported last radix");
    static_assert(P == 2 ? S2 == 1 : S3 == 1, "strides");
};

__device__ __forceinline__ int smem_pos(int p, int padsh) { return p + (p >> padsh); }

// --- pass geometry --------------------------------------------------------
// Pass with radix R and stride S: thread t's s-th group is g = t + T*s, at
// positions base(g) + r*S, base(g) = (g / S) * R * S + g % S.
template <int R, int S>
__device__ __forceinline__ int group_base(int g) { return (g / S) * (R * S) + (g % S); }

template <int R, int S>
__device__ __forceinline__ int group_lo(int g) { return g % S; }

// --- shared-memory exchange ----------------------------------------------
template <class SC, int R, int S>
__device__ __forceinline__ void smem_store(float2* sm, int t, const float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / R; ++s) {
        const int base = group_base<R, S>(t + SC::T * s);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[smem_pos(base + r * S, SC::PADSH)] = v[s * R + r];
    }
}
template <class SC, int R, int S>
__device__ __forceinline__ void smem_load(const float2* sm, int t, float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / R; ++s) {
        const int base = group_base<R, S>(t + SC::T * s);
#pragma unroll
        for (int r = 0; r < R; ++r) v[s * R + r] = sm[smem_pos(base + r * S, SC::PADSH)];
    }
}

// --- DFTs over every group the thread holds ------------------------------
template <class SC, int R, bool INV>
__device__ __forceinline__ void dft_groups(float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / R; ++s) {
        float2 g[R];
#pragma unroll
        for (int r = 0; r < R; ++r) g[r] = v[s * R + r];
        dft_reg<R, INV>(g);
#pragma unroll
        for (int r = 0; r < R; ++r) v[s * R + r] = g[r];
    }
}

// --- inter-pass twiddles: element r of group lo times W^{lo*r} ------------
// table layout tw[r * S + lo] (r = 0 row is unused), FP32 rounded from FP64.
template <class SC, int R, int S, bool INV>
__device__ __forceinline__ void twiddle_groups(const float2* tw, int t, float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / R; ++s) {
        const int lo = group_lo<R, S>(t + SC::T * s);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const float2 w = tw[r * S + lo];
            v[s * R + r] = INV ? cmulc(v[s * R + r], w) : cmul(v[s * R + r], w);
        }
    }
}

// --- global load/store in pass-1 geometry (coalesced: lo = g) -------------
template <class SC, bool RAGGED>
__device__ __forceinline__ void global_load(const float2* src, int valid, int t, float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / SC::R1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < SC::R1; ++r) {
            const int i = lo + r * SC::S1;
            if (RAGGED)
                v[s * SC::R1 + r] = (i < valid) ? src[i] : make_float2(0.f, 0.f);
            else
                v[s * SC::R1 + r] = src[i];
        }
    }
}
template <class SC, bool RAGGED>
__device__ __forceinline__ void global_store(float2* dst, int valid, int t, const float2 (&v)[SC::E]) {
#pragma unroll
    for (int s = 0; s < SC::E / SC::R1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < SC::R1; ++r) {
            const int i = lo + r * SC::S1;
            if (!RAGGED || i < valid) dst[i] = v[s * SC::R1 + r];
        }
    }
}

// --- the matched-filter multiply in last-pass geometry --------------------
// filt[(s*RL + r)*T + t] = H[k(P)] / N for the element at position
// P = g*RL + r, g = t + T*s; coalesced for fixed (s, r).
template <class SC>
__device__ __forceinline__ void filter_multiply(const float2* filt, int t, float2 (&v)[SC::E]) {
#pragma unroll
    for (int j = 0; j < SC::E; ++j) v[j] = cmul(v[j], filt[j * SC::T + t]);
}

// --- line synchronisation among the T threads of one line ----------------
template <class SC, int LPB>
__device__ __forceinline__ void line_sync(int line_in_block) {
    if constexpr (LPB == 1) {
        __syncthreads();
    } else if constexpr (SC::T >= 64) {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + line_in_block), "r"(SC::T) : "memory");
    } else if constexpr (SC::T == 32) {
        __syncwarp();
    } else {
        const unsigned lane = threadIdx.x & 31u;
        const unsigned mask = ((1u << SC::T) - 1u) << (lane & ~(unsigned)(SC::T - 1));
        __syncwarp(mask);
    }
}

// --- forward transform (all passes), leaving the digit-reversed spectrum
//     in registers in last-pass geometry ---------------------------------
template <class SC, int LPB>
__device__ __forceinline__ void forward_passes(float2 (&v)[SC::E], float2* sm, const float2* tw,
                                               int t, int lib) {
    dft_groups<SC, SC::R1, false>(v);
    twiddle_groups<SC, SC::R1, SC::S1, false>(tw, t, v);
    smem_store<SC, SC::R1, SC::S1>(sm, t, v);
    line_sync<SC, LPB>(lib);
    smem_load<SC, SC::R2, SC::S2>(sm, t, v);
    dft_groups<SC, SC::R2, false>(v);
    if constexpr (SC::P == 3) {
        twiddle_groups<SC, SC::R2, SC::S2, false>(tw + SC::R1 * SC::S1, t, v);
        smem_store<SC, SC::R2, SC::S2>(sm, t, v);
        line_sync<SC, LPB>(lib);
        smem_load<SC, SC::R3, SC::S3>(sm, t, v);
        dft_groups<SC, SC::R3, false>(v);
    }
}

// --- inverse transform from the digit-reversed spectrum in last-pass
//     geometry back to natural order in pass-1 geometry (unnormalised) ----
template <class SC, int LPB>
__device__ __forceinline__ void inverse_passes(float2 (&v)[SC::E], float2* sm, const float2* tw,
                                               int t, int lib) {
    if constexpr (SC::P == 3) {
        dft_groups<SC, SC::R3, true>(v);
        smem_store<SC, SC::R3, SC::S3>(sm, t, v);
        line_sync<SC, LPB>(lib);
        smem_load<SC, SC::R2, SC::S2>(sm, t, v);
        twiddle_groups<SC, SC::R2, SC::S2, true>(tw + SC::R1 * SC::S1, t, v);
    }
    dft_groups<SC, SC::R2, true>(v);
    smem_store<SC, SC::R2, SC::S2>(sm, t, v);
    line_sync<SC, LPB>(lib);
    smem_load<SC, SC::R1, SC::S1>(sm, t, v);
    twiddle_groups<SC, SC::R1, SC::S1, true>(tw, t, v);
    dft_groups<SC, SC::R1, true>(v);
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// Every kernel takes n_lines lines of length N; line l starts at
// data + l*ld and holds `valid` (<= N) stored samples: samples beyond `valid`
// are read as zeros and never written (zero-padded transforms).

// Fused line compression, Sec. II-B: y = IFFT(FFT(x) . H), in place allowed.
template <class SC, int LPB, bool RAGGED>
__device__ __forceinline__ void fused_compress_body(const float2* in, float2* out, int64_t n_lines, int64_t ld,
                                                    int valid, const float2* filt, const float2* tw) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    if (line >= n_lines) return;  // whole line groups only: no barrier is left waiting
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    float2 v[SC::E];
    global_load<SC, RAGGED>(in + line * ld, valid, t, v);
    forward_passes<SC, LPB>(v, sm, tw, t, lib);
    filter_multiply<SC>(filt, t, v);
    inverse_passes<SC, LPB>(v, sm, tw, t, lib);
    global_store<SC, RAGGED>(out + line * ld, valid, t, v);
}

// The compiler's own register choice (only the block size is bounded) ...
template <class SC, int LPB, bool RAGGED>
__global__ void __launch_bounds__(SC::T * LPB)
fused_compress_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* filt,
                      const float2* tw) {
    fused_compress_body<SC, LPB, RAGGED>(in, out, n_lines, ld, valid, filt, tw);
}
// ... or registers capped so that SC::MINB blocks fit on one SM.
template <class SC, int LPB, bool RAGGED>
__global__ void __launch_bounds__(SC::T * LPB, SC::MINB)
fused_compress_kernel_capped(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid,
                             const float2* filt, const float2* tw) {
    fused_compress_body<SC, LPB, RAGGED>(in, out, n_lines, ld, valid, filt, tw);
}

// Plain forward (or inverse) DFT of each line, natural order in and out,
// unnormalised.  The inverse uses IFFT(x) = conj(FFT(conj x)) (Sec. II-C).
// Output element k of the last-pass position P is written to its natural
// index k(P).
template <class SC>
__device__ __forceinline__ int natural_index(int g, int r) {
    // position P = g*RL + r = sum k_i S_i  ->  k = k1 + R1 k2 (+ R1 R2 k3)
    const int P = g * SC::RL + r;
    const int k1 = P / SC::S1;
    const int rem = P % SC::S1;
    if constexpr (SC::P == 2) {
        return k1 + SC::R1 * rem;
    } else {
        const int k2 = rem / SC::S2, k3 = rem % SC::S2;
        return k1 + SC::R1 * (k2 + SC::R2 * k3);
    }
}

template <class SC, int LPB, bool INV>
__global__ void __launch_bounds__(SC::T * LPB)
dft_lines_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld,
                 int valid, const float2* tw) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    if (line >= n_lines) return;
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    float2 v[SC::E];
    if (valid < SC::N)
        global_load<SC, true>(in + line * ld, valid, t, v);
    else
        global_load<SC, false>(in + line * ld, valid, t, v);
    if (INV) {
#pragma unroll
        for (int j = 0; j < SC::E; ++j) v[j] = cconj(v[j]);
    }
    forward_passes<SC, LPB>(v, sm, tw, t, lib);
    // natural order through shared memory, then coalesced stores
    line_sync<SC, LPB>(lib);
#pragma unroll
    for (int s = 0; s < SC::E / SC::RL; ++s) {
#pragma unroll
        for (int r = 0; r < SC::RL; ++r) {
            const int k = natural_index<SC>(t + SC::T * s, r);
            sm[smem_pos(k, SC::PADSH)] = v[s * SC::RL + r];
        }
    }
    line_sync<SC, LPB>(lib);
    float2* dst = out + line * SC::N;  // outputs are dense lines of N
#pragma unroll
    for (int j = 0; j < SC::E; ++j) {
        const int k = t + SC::T * j;
        const float2 x = sm[smem_pos(k, SC::PADSH)];
        dst[k] = INV ? cconj(x) : x;
    }
}

}  // namespace sar
