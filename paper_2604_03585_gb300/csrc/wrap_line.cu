// Line lengths that are not powers of two: the exact length-n compression
// y = IFFT_n(FFT_n(x) . H) (Sec. II-B at length n), through the power-of-two
// line engine.  With h = IFFT_n(H), y is the circular convolution x (*)_n h.
// For L a power of two >= 2n - 1 the linear convolution z = x * h (2n - 1
// samples) is exact as z = IFFT_L(FFT_L(x zero-padded to L) . G) with
// G = FFT_L(h zero-padded to L), and the circular result is its wrap,
// y[m] = z[m] + z[m + n].
//
// One fused launch per batch of lines: each line is read once (n samples;
// the zeros up to L are synthesised, not read), the length-L engine runs its
// forward passes, the filter G / L in its register order and its inverse
// passes (streamed.cuh), the last inverse pass leaves z in shared memory, and
// the store adds the two halves.  Two device-memory transfers per line, as for
// powers of two; the arithmetic is that of length L, 2 to 4 times n.
//
// These schedules are kept out of the registry's enumeration (they would be
// wrong for a power-of-two line of length L): plans look them up by L.
#include "launch.cuh"
#include "registry.h"

namespace sar {

template <class SC, int LPB, bool ROLL>
__global__ void __launch_bounds__(SC::T * LPB)
fused_wrap_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, int n, const float2* filt,
                  const float2* tw) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    if (line >= n_lines) return;   // whole line groups only: no barrier is left waiting
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1;
    streamed_until_last<SC, LPB, ROLL, true>(in + line * ld, sm, filt, tw, t, lib, n);
    // inverse pass 1 in place: z in natural order
#pragma unroll(ROLL ? 1 : G1)
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
        grp_smem_store<R1, S1>(sm, lo, SC::PADSH, x);
    }
    line_sync<SC, LPB>(lib);
    // y[m] = z[m] + z[m + n], m + n <= 2n - 1 < L
    float2* dst = out + line * ld;
    for (int m = t; m < n; m += SC::T) {
        const float2 a = sm[smem_pos(m, SC::PADSH)], b = sm[smem_pos(m + n, SC::PADSH)];
        __stcs(dst + m, make_float2(a.x + b.x, a.y + b.y));
    }
}

// The DFT of a line of any length n (Bluestein): with j k = (j^2 + k^2 -
// (k - j)^2) / 2 and c_m = exp(-i pi m^2 / n),
//   X[k] = c_k sum_j (x_j c_j) conj(c_{k-j}),
// a linear convolution of a = x . c (n samples) with conj(c) over lags
// -(n-1) ... n-1, exact through length-L transforms (L >= 2n - 1) as the
// first n outputs of IFFT_L(FFT_L(a padded) . G), G = FFT_L(b), b[m mod L] =
// conj(c_m).  One block per line (LPB lines): the chirped line goes to shared
// memory, the streamed passes of the length-L engine run in place, the last
// inverse pass leaves the convolution there, and the store applies c_k.  INV:
// the inverse kernel as conj(DFT(conj x)).  chirp[m] = c_m, m < n.
template <class SC, int LPB, bool ROLL, bool INV>
__global__ void __launch_bounds__(SC::T * LPB)
bluestein_dft_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, int n, const float2* filt,
                     const float2* tw, const float2* chirp) {
    extern __shared__ float2 smem_dyn[];
    const int lib = threadIdx.x / SC::T;
    const int t = threadIdx.x % SC::T;
    const int64_t line = (int64_t)blockIdx.x * LPB + lib;
    if (line >= n_lines) return;   // whole line groups only: no barrier is left waiting
    float2* sm = smem_dyn + lib * SC::SMEM_ELEMS;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1, RL = SC::RL, GL = SC::E / RL;
    const float2* src = in + line * ld;
    for (int j = t; j < SC::N; j += SC::T) {
        float2 a = make_float2(0.f, 0.f);
        if (j < n) {
            float2 x = __ldcs(src + j);
            if (INV) x.y = -x.y;
            a = cmul(x, chirp[j]);
        }
        sm[smem_pos(j, SC::PADSH)] = a;
    }
    line_sync<SC, LPB>(lib);
    streamed_mid_pass<SC, R1, S1, false, ROLL>(sm, tw, t);
    line_sync<SC, LPB>(lib);
    const float2* tw2 = tw + R1 * S1;
    if constexpr (SC::P == 3) {
        streamed_mid_pass<SC, SC::R2, SC::S2, false, ROLL>(sm, tw2, t);
        line_sync<SC, LPB>(lib);
    }
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
#pragma unroll(ROLL ? 1 : G1)
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 x[R1];
        grp_smem_load<R1, S1>(sm, lo, SC::PADSH, x);
        grp_twiddle<R1, S1, true>(tw, lo, x);
        dft_reg<R1, true>(x);
        grp_smem_store<R1, S1>(sm, lo, SC::PADSH, x);
    }
    line_sync<SC, LPB>(lib);
    float2* dst = out + line * (int64_t)n;   // outputs are dense lines of n
    for (int k = t; k < n; k += SC::T) {
        float2 y = cmul(sm[smem_pos(k, SC::PADSH)], chirp[k]);
        if (INV) y.y = -y.y;
        __stcs(dst + k, y);
    }
}

namespace {

template <class SC, int LPB, bool ROLL>
cudaError_t prepare_wrap() {
    constexpr int smem = smem_bytes_of<SC, LPB>();
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fused_wrap_kernel<SC, LPB, ROLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// `valid` is the line length n; lines are ld apart (ld >= n).
template <class SC, int LPB, bool ROLL>
cudaError_t launch_wrap(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* filt,
                        const float2* tw, const FusedCtl&, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (valid < 1 || 2 * (int64_t)valid - 1 > SC::N || ld < valid) return cudaErrorInvalidValue;
    const int64_t blocks = (n_lines + LPB - 1) / LPB;
    fused_wrap_kernel<SC, LPB, ROLL><<<(unsigned)blocks, SC::T * LPB, smem_bytes_of<SC, LPB>(), st>>>(
        in, out, n_lines, ld, valid, filt, tw);
    return cudaGetLastError();
}

template <class SC, int LPB, bool ROLL>
constexpr SchedDesc make_wrap_desc(const char* name) {
    return SchedDesc{name,
                     SC::N,
                     SC::E,
                     SC::R1,
                     SC::R2,
                     SC::R3,
                     LPB,
                     SC::T * LPB,
                     smem_bytes_of<SC, LPB>(),
                     SC::TW_ELEMS,
                     SC::RL,
                     0,
                     &launch_wrap<SC, LPB, ROLL>,
                     nullptr,
                     &prepare_wrap<SC, LPB, ROLL>,
                     nullptr,
                     0,
                     nullptr,
                     0};
}

const SchedDesc kWrap[] = {
    make_wrap_desc<Sched<256, 16, 16, 16>, 8, false>("wrap_l256_e16_r16x16_s8"),
    make_wrap_desc<Sched<512, 32, 16, 32>, 8, false>("wrap_l512_e32_r16x32_s8"),
    make_wrap_desc<Sched<1024, 32, 32, 32>, 4, false>("wrap_l1024_e32_r32x32_s4"),
    make_wrap_desc<Sched<2048, 16, 16, 8, 16>, 1, false>("wrap_l2048_e16_r16x8x16_s1"),
    make_wrap_desc<Sched<4096, 32, 16, 16, 16>, 1, true>("wrap_l4096_e32_r16x16x16_sr1"),
    make_wrap_desc<Sched<8192, 32, 16, 16, 32>, 1, true>("wrap_l8192_e32_r16x16x32_sr1"),
    make_wrap_desc<Sched<16384, 32, 16, 32, 32>, 1, true>("wrap_l16384_e32_r16x32x32_sr1"),
};

}  // namespace

const SchedDesc* wrap_schedule(int L) {
    for (const SchedDesc& d : kWrap)
        if (d.n == L) return &d;
    return nullptr;
}

namespace {
template <class SC, int LPB, bool ROLL>
cudaError_t launch_bluestein_t(const float2* in, float2* out, int64_t n_lines, int64_t ld, int n, const float2* filt,
                               const float2* tw, const float2* chirp, int inverse, cudaStream_t st) {
    constexpr int smem = smem_bytes_of<SC, LPB>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(bluestein_dft_kernel<SC, LPB, ROLL, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bluestein_dft_kernel<SC, LPB, ROLL, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((n_lines + LPB - 1) / LPB);
    if (inverse)
        bluestein_dft_kernel<SC, LPB, ROLL, true><<<blocks, SC::T * LPB, smem, st>>>(in, out, n_lines, ld, n, filt,
                                                                                   tw, chirp);
    else
        bluestein_dft_kernel<SC, LPB, ROLL, false><<<blocks, SC::T * LPB, smem, st>>>(in, out, n_lines, ld, n, filt,
                                                                                    tw, chirp);
    return cudaGetLastError();
}
}  // namespace

// The DFT of n_lines lines of a length n that is not a power of two (2 <= n,
// 2n - 1 <= L), through the wrap schedule of engine length L = d.n and its
// tables: filt = G / L in the engine's register order, chirp[m] = c_m.
cudaError_t launch_bluestein(const SchedDesc& d, const float2* in, float2* out, int64_t n_lines, int64_t ld, int n,
                             const float2* filt, const float2* tw, const float2* chirp, int inverse, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    if (n < 2 || 2 * (int64_t)n - 1 > d.n || ld < n) return cudaErrorInvalidValue;
    switch (d.n) {
        case 256: return launch_bluestein_t<Sched<256, 16, 16, 16>, 8, false>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
        case 512: return launch_bluestein_t<Sched<512, 32, 16, 32>, 8, false>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
        case 1024: return launch_bluestein_t<Sched<1024, 32, 32, 32>, 4, false>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
        case 2048: return launch_bluestein_t<Sched<2048, 16, 16, 8, 16>, 1, false>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
        case 4096: return launch_bluestein_t<Sched<4096, 32, 16, 16, 16>, 1, true>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
        case 8192: return launch_bluestein_t<Sched<8192, 32, 16, 16, 32>, 1, true>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
        case 16384: return launch_bluestein_t<Sched<16384, 32, 16, 32, 32>, 1, true>(in, out, n_lines, ld, n, filt, tw, chirp, inverse, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sar
