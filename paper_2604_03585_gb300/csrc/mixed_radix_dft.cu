// The plain DFT of a 7-smooth line length on the mixed-radix engine (the
// transform sar_fft_lines computes; the fused compression keeps the
// spectrum in position order, this one returns it in natural order).
//
// A line is staged into its shared-memory slots in natural order (zero beyond
// `valid`, conjugated for the inverse), every forward pass runs in place in
// shared memory (the first as a middle pass), and the spectrum is written out
// in natural order: X[k], k = k_0 + R_0 (k_1 + R_1 (k_2 + ...)), sits at
// position sum_i k_i S_i (a table built with the twiddles; conjugated again
// for the inverse: the inverse is
// conj(DFT(conj x)), unnormalised).  A line is read completely before any of
// it is written, so in == out is safe.
#include "mixed_radix.cuh"

namespace sar {
namespace mixed {

namespace {

// MINB: blocks per SM the registers are capped for (as the fused kernel's
// variants, chosen by length); sgn = -1 for the inverse (conjugation)
template <int MINB>
__global__ void __launch_bounds__(kMixedThreads, MINB)
mixed_dft_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                 MixedGeom geo, float sgn) {
    extern __shared__ float2 smem_mixed[];
    const int T = geo.T, lib = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t line = (int64_t)blockIdx.x * (kMixedThreads / T) + lib;
    const bool live = line < n_lines;
    const int n = geo.n, P = geo.P;
    float2* sm = smem_mixed + lib * (n + (n >> 5) + 1);
    const float2* src = in + (live ? line : 0) * ld;
    float2* dst = out + (live ? line : 0) * ld;
    if (live)
        for (int p = t; p < n; p += T) {
            const float2 x = p < valid ? __ldcs(src + p) : make_float2(0.f, 0.f);
            sm[mpad(p)] = make_float2(x.x, sgn * x.y);
        }
    __syncthreads();
    for (int i = 0; i < P - 1; ++i) {
        if (live) mpass<kMid, false>(geo.R[i], geo.S[i], geo.M[i], n, t, T, src, dst, sm, tw + geo.tw_off[i], tw);
        __syncthreads();
    }
    if (live) mpass<kLastDft, false>(geo.R[P - 1], 1, 0u, n, t, T, src, dst, sm, tw, tw);
    __syncthreads();
    const int32_t* pos = reinterpret_cast<const int32_t*>(tw + geo.pos_off);
    if (live)
        for (int k = t; k < n; k += T) {
            const float2 x = sm[mpad(pos[k])];
            __stcs(dst + k, make_float2(x.x, sgn * x.y));
        }
}

}  // namespace

cudaError_t launch_dft_mixed(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                             int inverse, const MixedGeom& g, int lines_per_block, int smem, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n_lines + lines_per_block - 1) / lines_per_block);
    const float sgn = inverse ? -1.f : 1.f;
    // the fused kernel's register caps by length (n <= 4096: 4 blocks per SM,
    // <= 6000: 3, above: 2)
    if (g.n <= 4096)
        mixed_dft_kernel<4><<<blocks, kMixedThreads, smem, st>>>(in, out, n_lines, ld, valid, tw, g, sgn);
    else if (g.n <= 6000)
        mixed_dft_kernel<3><<<blocks, kMixedThreads, smem, st>>>(in, out, n_lines, ld, valid, tw, g, sgn);
    else
        mixed_dft_kernel<2><<<blocks, kMixedThreads, smem, st>>>(in, out, n_lines, ld, valid, tw, g, sgn);
    return cudaGetLastError();
}

cudaError_t set_smem_dft(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(mixed_dft_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mixed_dft_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mixed_dft_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

}  // namespace mixed
}  // namespace sar
