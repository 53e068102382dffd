// Full Range-Doppler processing with range cell migration correction
// (Sec. IV-A steps 2-4 of the paper: azimuth FFT, RCMC by sinc
// interpolation, azimuth compression with the range-dependent filter
// H_a(f_a, R0), azimuth IFFT).
//
// Geometry (normalised, see sar_plan_set_geometry): a target of closest range
// r0 (in range samples) appears in the range-Doppler domain at r0 / D(f),
// D(f) = sqrt(1 - (f / (kappa v_s))^2), with spectrum phase
// exp(-2 pi i kappa r0 D(f)).  RCMC reads output bin n at frequency f from
// the input at n + (r_near + n)(1/D(f) - 1) through a 16-tap Hann-windowed
// sinc; azimuth compression multiplies by exp(+2 pi i kappa r D(f)),
// r = r_near + n, and applies the inverse FFT (1/N).
//
// Per azimuth frequency index j the plan keeps, computed in FP64 on the host
// and rounded: kappa D(f_j) and 1/D(f_j) - 1, each as an unevaluated float sum
// (hi + lo).  The phase kappa r D of a sample (up to ~1e5 cycles) and the
// migration r (1/D - 1) (up to ~1e2 samples) are then formed in FP32 with an
// exact two-product, so only their fractional parts are rounded; the integer
// range bin n never enters a rounded sum (at n ~ 8000 the FP32 spacing is
// 1e-3 samples, which would cost ~1e-3 relative error on a half-band signal).
#include "../../include/sar.h"
#include "line_engine.cuh"
#include "registry.h"
#include "tables.h"

namespace sar {

struct RdColumn {
    float a_hi, a_lo;       // kappa D(f_j) = a_hi + a_lo
    float mig_hi, mig_lo;   // 1 / D(f_j) - 1 = mig_hi + mig_lo
};

// cos and sin of 2 pi t / 16 for the taps t = -7 ... 8 (index t + 7),
// evaluated at compile time
#define SAR_RC(t) float2{(float)ct::cos2pi(t, 16), (float)ct::sin2pi(t, 16)}
__constant__ float2 kHann16[16] = {SAR_RC(-7), SAR_RC(-6), SAR_RC(-5), SAR_RC(-4), SAR_RC(-3), SAR_RC(-2),
                                   SAR_RC(-1), SAR_RC(0),  SAR_RC(1),  SAR_RC(2),  SAR_RC(3),  SAR_RC(4),
                                   SAR_RC(5),  SAR_RC(6),  SAR_RC(7),  SAR_RC(8)};
#undef SAR_RC

// RCMC, one output sample per thread: out[n][j] = sum_t h(src - k_t) in[k_t][j],
// src = n + (r_near + n)(1/D(f_j) - 1), k_t the 16 integers nearest src,
// h(x) = sinc(x) * 0.5 (1 + cos(2 pi x / 16)).
template <int TAPS>
__global__ void __launch_bounds__(256)
rcmc_kernel(const float2* __restrict__ in, float2* __restrict__ out, int n_range, int n_f, const RdColumn* cols,
            double r_near) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_range * n_f) return;
    const int n = (int)(idx / n_f), j = (int)(idx % n_f);
    const double rd = r_near + (double)n;
    const float r_hi = (float)rd, r_lo = (float)(rd - (double)r_hi);
    const RdColumn c = cols[j];
    // shift = r (mig_hi + mig_lo) = p + e + ..., p the rounded product, e its exact error
    const float p = r_hi * c.mig_hi;
    const float e = fmaf(r_hi, c.mig_hi, -p);
    const float fl = floorf(p);
    float frac = (p - fl) + (e + fmaf(r_hi, c.mig_lo, r_lo * c.mig_hi));   // p - fl is exact
    int k0 = n + (int)fl;
    if (frac < 0.f) { frac += 1.f; k0 -= 1; }
    if (frac >= 1.f) { frac -= 1.f; k0 += 1; }
    float s0, c0, sw, cw;
    sincospif(frac, &s0, &c0);
    sincospif(frac * (2.0f / TAPS), &sw, &cw);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = -TAPS / 2 + 1; t <= TAPS / 2; ++t) {
        const int k = k0 + t;
        if (k < 0 || k >= n_range) continue;
        const float x = frac - (float)t;
        // sin(pi (frac - t)) = (-1)^t sin(pi frac); window 0.5 (1 + cos(2 pi x / TAPS))
        const float sgn = (t & 1) ? -1.f : 1.f;
        const float sinc = (x == 0.f) ? 1.f : sgn * s0 / (3.14159265358979f * x);
        static_assert(TAPS == 16, "the window table holds 16 taps");
        const float2 cs = kHann16[t + 7];
        // cos(2 pi (frac - t) / 16) = cos(2 pi frac/16) cos(2 pi t/16) + sin(2 pi frac/16) sin(2 pi t/16)
        const float win = 0.5f + 0.5f * (cw * cs.x + sw * cs.y);
        const float h = (fabsf(x) < 0.5f * TAPS) ? sinc * win : 0.f;
        const float2 v = in[(int64_t)k * n_f + j];
        acc.x = fmaf(h, v.x, acc.x);
        acc.y = fmaf(h, v.y, acc.y);
    }
    out[idx] = acc;
}

// Azimuth compression of range bin `line` (r = r_near + line): multiply the
// natural-order spectrum by exp(+2 pi i kappa r D(f_j)), inverse FFT through
// conj(FFT(conj .)) (Sec. II-C), 1/N, natural-order coalesced store.
template <class SC>
__global__ void __launch_bounds__(SC::T)
az_compress_rd_kernel(const float2* in, float2* out, int64_t n_lines, const float2* tw, const RdColumn* cols,
                      double r_near) {
    extern __shared__ float2 smem_dyn[];
    const int t = threadIdx.x;
    const int64_t line = blockIdx.x;
    if (line >= n_lines) return;
    float2* sm = smem_dyn;
    const double rd = r_near + (double)line;
    const float r_hi = (float)rd, r_lo = (float)(rd - (double)r_hi);
    float2 v[SC::E];
    const float2* src = in + line * SC::N;
#pragma unroll
    for (int s = 0; s < SC::E / SC::R1; ++s) {
        const int lo = t + SC::T * s;
#pragma unroll
        for (int r = 0; r < SC::R1; ++r) {
            const int j = lo + r * SC::S1;
            const RdColumn c = cols[j];
            const float p = r_hi * c.a_hi;
            const float e = fmaf(r_hi, c.a_hi, -p);           // exact error of the product
            const float frac = (p - rintf(p)) + (e + fmaf(r_hi, c.a_lo, r_lo * c.a_hi));
            float sn, cs;
            sincospif(2.f * frac, &sn, &cs);
            const float2 x = __ldcs(src + j);
            // x * exp(+i phase), conjugated for the forward-transform inverse
            v[s * SC::R1 + r] = cconj(make_float2(fmaf(x.x, cs, -x.y * sn), fmaf(x.x, sn, x.y * cs)));
        }
    }
    forward_passes<SC, 1>(v, sm, tw, t, 0);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < SC::E / SC::RL; ++s) {
#pragma unroll
        for (int r = 0; r < SC::RL; ++r) {
            const int k = natural_index<SC>(t + SC::T * s, r);
            sm[smem_pos(k, SC::PADSH)] = v[s * SC::RL + r];
        }
    }
    __syncthreads();
    constexpr float inv_n = 1.0f / SC::N;
    float2* dst = out + line * SC::N;
#pragma unroll
    for (int i = 0; i < SC::E; ++i) {
        const int k = t + SC::T * i;
        const float2 x = sm[smem_pos(k, SC::PADSH)];
        __stcs(dst + k, make_float2(x.x * inv_n, -x.y * inv_n));
    }
}

namespace {
using A256 = Sched<256, 16, 16, 16>;
using A512 = Sched<512, 32, 16, 32>;
using A1024 = Sched<1024, 32, 32, 32>;
using A2048 = Sched<2048, 16, 16, 16, 8>;
using A4096 = Sched<4096, 32, 16, 16, 16>;
using A8192 = Sched<8192, 32, 16, 16, 32>;
using A16384 = Sched<16384, 32, 16, 32, 32>;

template <class SC>
cudaError_t launch_az(const float2* in, float2* out, int64_t n_lines, const float2* tw, const RdColumn* cols,
                      double r_near, cudaStream_t st) {
    constexpr int smem = SC::SMEM_ELEMS * 8;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(az_compress_rd_kernel<SC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
    }
    az_compress_rd_kernel<SC><<<(unsigned)n_lines, SC::T, smem, st>>>(in, out, n_lines, tw, cols, r_near);
    return cudaGetLastError();
}
}  // namespace

// The schedule whose twiddle tables the azimuth kernel of length n uses.
const char* rd_az_schedule(int n) {
    switch (n) {
        case 256: return "n256_e16_r16x16_l8";
        case 512: return "n512_e32_r16x32_l8";
        case 1024: return "n1024_e32_r32x32_l4";
        case 2048: return "n2048_e16_r16x16x8_l1";
        case 4096: return "n4096_e32_r16x16x16_l1";
        case 8192: return "n8192_e32_r16x16x32_l1";
        case 16384: return "n16384_e32_r16x32x32_l1";
    }
    return nullptr;
}

cudaError_t launch_az_compress_rd(int n, const float2* in, float2* out, int64_t n_lines, const float2* tw,
                                  const void* cols, double r_near, cudaStream_t st) {
    const RdColumn* c = (const RdColumn*)cols;
    switch (n) {
        case 256: return launch_az<A256>(in, out, n_lines, tw, c, r_near, st);
        case 512: return launch_az<A512>(in, out, n_lines, tw, c, r_near, st);
        case 1024: return launch_az<A1024>(in, out, n_lines, tw, c, r_near, st);
        case 2048: return launch_az<A2048>(in, out, n_lines, tw, c, r_near, st);
        case 4096: return launch_az<A4096>(in, out, n_lines, tw, c, r_near, st);
        case 8192: return launch_az<A8192>(in, out, n_lines, tw, c, r_near, st);
        case 16384: return launch_az<A16384>(in, out, n_lines, tw, c, r_near, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rcmc(int taps, const float2* in, float2* out, int n_range, int n_f, const void* cols,
                        double r_near, cudaStream_t st) {
    const int64_t total = (int64_t)n_range * n_f;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    const RdColumn* c = (const RdColumn*)cols;
    if (taps != 16) return cudaErrorInvalidValue;
    rcmc_kernel<16><<<blocks, 256, 0, st>>>(in, out, n_range, n_f, c, r_near);
    return cudaGetLastError();
}

// Host: the per-frequency columns of a geometry, FP64 then rounded.
void rd_columns(int n_f, double kappa, double vs, void* host_cols) {
    RdColumn* c = (RdColumn*)host_cols;
    for (int j = 0; j < n_f; ++j) {
        const double f = (j < n_f / 2 ? (double)j : (double)(j - n_f)) / (double)n_f;
        const double q = f / (kappa * vs);
        const double d = sqrt(1.0 - q * q);
        const double a = kappa * d;
        c[j].a_hi = (float)a;
        c[j].a_lo = (float)(a - (double)c[j].a_hi);
        const double mig = q * q / (d * (1.0 + d));   // 1/D - 1 without cancellation
        c[j].mig_hi = (float)mig;
        c[j].mig_lo = (float)(mig - (double)c[j].mig_hi);
    }
}

size_t rd_column_bytes() { return sizeof(RdColumn); }

}  // namespace sar
