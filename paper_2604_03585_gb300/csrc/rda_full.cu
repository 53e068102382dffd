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
#include "streamed.cuh"
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

// RCMC tiles: 32 frequency columns (one per lane) x 128 range bins per block of
// 8 warps.  A block stages the input rows its outputs touch in shared memory
// (rows n0 + min shift - 7 ... n0 + 127 + max shift + 8, zero outside the
// scene); the host sizes that span from the geometry, and a block whose span
// does not fit reads global memory directly.
constexpr int kRcCols = 32;
constexpr int kRcRows = 128;
constexpr int kRcWarps = 8;
constexpr int kRcMaxStaged = 384;   // 96 KB of staged rows per block

// Source position of output bin n in column c: k0 + frac, frac in [0, 1), for
// r = r_near + n with r_near = rn_hi + rn_lo.  r is formed by a two-sum and the
// shift r (1/D - 1) by a two-product, so only the fractional part is rounded.
__device__ __forceinline__ void rc_locate(int n, const RdColumn& c, float rn_hi, float rn_lo, int& k0, float& frac) {
    const float nf = (float)n;
    const float r_hi = rn_hi + nf;                       // two-sum of rn_hi and n
    const float bb = r_hi - rn_hi;
    const float r_lo = ((rn_hi - (r_hi - bb)) + (nf - bb)) + rn_lo;
    const float p = __fmul_rn(r_hi, c.mig_hi);            // never contracted into the next subtraction
    const float e = fmaf(r_hi, c.mig_hi, -p);             // exact error of the product
    const float fl = floorf(p);
    frac = (p - fl) + (e + fmaf(r_hi, c.mig_lo, r_lo * c.mig_hi));   // p - fl is exact
    k0 = n + (int)fl;
    if (frac < 0.f) { frac += 1.f; k0 -= 1; }
    if (frac >= 1.f) { frac -= 1.f; k0 += 1; }
}

__device__ __forceinline__ float rc_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// (cw, sw) = (cos, sin)(pi frac / 8) and s = sin(pi frac) for frac in (0, 1),
// each to a few FP32 ulps, s relative to its own size near frac = 0 and 1.
// With g = min(frac, 1 - frac) <= 1/2 and theta = pi g / 8 <= pi / 16, sin and
// cos of theta come from their Taylor series (the first omitted terms are below
// 2e-12), s = sin(pi g) = sin(8 theta) from three angle doublings in which
// every cosine stays >= cos(pi / 4) (no cancellation), and for frac > 1/2 the
// window angle is pi / 8 - theta.
__device__ __forceinline__ void rc_trig(float frac, float& cw, float& sw, float& s) {
    const bool flip = frac > 0.5f;
    const float g = flip ? 1.f - frac : frac;   // exact
    const float th = g * 0.392699081698724155f;  // pi / 8
    const float t2 = th * th;
    const float s8 = th * fmaf(t2, fmaf(t2, fmaf(t2, -1.f / 5040.f, 1.f / 120.f), -1.f / 6.f), 1.f);
    const float c8 = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 1.f / 40320.f, -1.f / 720.f), 1.f / 24.f), -0.5f), 1.f);
    float a = 2.f * s8;
    const float s4 = a * c8, c4 = fmaf(-a, s8, 1.f);   // pi g / 4
    a = 2.f * s4;
    const float s2 = a * c4, c2 = fmaf(-a, s4, 1.f);   // pi g / 2
    s = 2.f * s2 * c2;                                   // pi g
    constexpr float C = 0.923879532511286756f, S = 0.382683432365089772f;   // cos, sin of pi / 8
    cw = flip ? fmaf(C, c8, S * s8) : c8;
    sw = flip ? fmaf(S, c8, -C * s8) : s8;
}

// The 16 taps at source position k0 + frac, rows read through row(t) for
// t = -7 ... 8.  Weight h_t = sinc(x) w(x), x = frac - t,
// w(x) = 0.5 (1 + cos(2 pi x / 16)).  With sin(pi x) = (-1)^t sin(pi frac) and
// cos(2 pi x / 16) = cw cos_t + sw sin_t = u_t, cos_t, sin_t the cos and sin of
// 2 pi t / 16:
//   h_t = (sin(pi frac) / (2 pi)) (-1)^t (1 + u_t) / x.
// Taps t and t + 8 share (-1)^t and have u_{t+8} = -u_t.
template <class Row>
__device__ __forceinline__ float2 rc_interp(float frac, Row row) {
    if (frac == 0.f) return row(0);   // h_0 = 1, every other tap sits on a zero of the sinc
    float cw, sw, s;
    rc_trig(frac, cw, sw, s);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = -7; t <= 0; ++t) {
        const float2 cs = kHann16[t + 7];
        const float u = fmaf(cw, cs.x, sw * cs.y);
        const float r1 = rc_rcp(frac - (float)t), r2 = rc_rcp(frac - (float)(t + 8));
        float h1 = fmaf(u, r1, r1), h2 = fmaf(-u, r2, r2);
        if (t & 1) {
            h1 = -h1;
            h2 = -h2;
        }
        const float2 v1 = row(t), v2 = row(t + 8);
        acc.x = fmaf(h1, v1.x, acc.x);
        acc.y = fmaf(h1, v1.y, acc.y);
        acc.x = fmaf(h2, v2.x, acc.x);
        acc.y = fmaf(h2, v2.y, acc.y);
    }
    const float a = s * 0.159154943091895336f;   // sin(pi frac) / (2 pi)
    return make_float2(acc.x * a, acc.y * a);
}

__global__ void __launch_bounds__(kRcCols * kRcWarps)
rcmc_tile_kernel(const float2* __restrict__ in, float2* __restrict__ out, int n_range, int n_f,
                 const RdColumn* __restrict__ cols, float rn_hi, float rn_lo, int staged_rows) {
    extern __shared__ float2 tile[];   // [staged_rows][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * kRcCols + lane;
    const int n0 = blockIdx.y * kRcRows;
    const int n1 = min(n0 + kRcRows, n_range) - 1;
    const bool jok = j < n_f;
    const RdColumn c = cols[jok ? j : n_f - 1];
    // the rows this block reads: the same positions every output computes, so
    // every warp finds the same span
    int k_first, k_last;
    float f_unused;
    rc_locate(n0, c, rn_hi, rn_lo, k_first, f_unused);
    rc_locate(n1, c, rn_hi, rn_lo, k_last, f_unused);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        k_first = min(k_first, __shfl_xor_sync(0xffffffffu, k_first, o));
        k_last = max(k_last, __shfl_xor_sync(0xffffffffu, k_last, o));
    }
    const int lo = k_first - 7, hi = k_last + 8;
    const int span = hi - lo + 1;
    const bool staged = span <= staged_rows;
    if (staged) {
#pragma unroll 4
        for (int rr = warp; rr < span; rr += kRcWarps) {
            const int k = lo + rr;
            tile[rr * kRcCols + lane] =
                (jok && k >= 0 && k < n_range) ? in[(int64_t)k * n_f + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
    }
    if (!jok) return;
    for (int n = n0 + warp; n <= n1; n += kRcWarps) {
        int k0;
        float frac;
        rc_locate(n, c, rn_hi, rn_lo, k0, frac);
        float2 y;
        if (staged) {
            k0 = min(max(k0, lo + 7), hi - 8);   // already within; keeps every read inside the tile
            const float2* b = tile + (k0 - lo) * kRcCols + lane;
            y = rc_interp(frac, [&](int t) { return b[t * kRcCols]; });
        } else {
            y = rc_interp(frac, [&](int t) {
                const int k = k0 + t;
                return (k >= 0 && k < n_range) ? in[(int64_t)k * n_f + j] : make_float2(0.f, 0.f);
            });
        }
        __stcs(out + (int64_t)n * n_f + j, y);
    }
}

// The azimuth kernels of the full processor in group-streamed form: the passes
// before the last run one radix group at a time (R values live, the next
// group's loads in flight during the current group's arithmetic); the last
// pass keeps the line in registers for the scatter to natural order through
// shared memory and the coalesced store.  COMPRESS (range bin `line`,
// r = r_near + line): every sample j is first multiplied by
// exp(+2 pi i frac(kappa r D(f_j))) -- the phase of up to ~1e5 cycles formed
// by an FP32 two-product of r with kappa D(f_j) held as hi + lo, so that only
// its fractional part is rounded -- and conjugated, and the store conjugates
// and scales by 1/N: the inverse FFT of the filtered line through
// conj(FFT(conj .)) (Sec. II-C).  Otherwise the forward FFT of the line (the
// Range-Doppler domain, Sec. IV-A step 2).
template <class SC, bool COMPRESS>
__global__ void __launch_bounds__(SC::T)
az_streamed_kernel(const float2* in, float2* out, int64_t n_lines, const float2* tw, const RdColumn* cols,
                   double r_near) {
    extern __shared__ float2 smem_dyn[];
    const int t = threadIdx.x;
    const int64_t line = blockIdx.x;
    if (line >= n_lines) return;
    float2* sm = smem_dyn;
    constexpr int R1 = SC::R1, S1 = SC::S1, G1 = SC::E / R1, RL = SC::RL, GL = SC::E / RL;
    const float2* src = in + line * SC::N;
    float r_hi = 0.f, r_lo = 0.f;
    if constexpr (COMPRESS) {
        const double rd = r_near + (double)line;
        r_hi = (float)rd;
        r_lo = (float)(rd - (double)r_hi);
    }
    auto sample = [&](int j) -> float2 {
        float2 x = __ldcs(src + j);
        if constexpr (COMPRESS) {
            const RdColumn c = cols[j];
            const float p = __fmul_rn(r_hi, c.a_hi);   // never contracted into p - rint(p)
            const float e = fmaf(r_hi, c.a_hi, -p);    // exact error of the product
            const float frac = (p - rintf(p)) + (e + fmaf(r_hi, c.a_lo, r_lo * c.a_hi));
            float sn, cs;
            sincospif(2.f * frac, &sn, &cs);
            x = cconj(make_float2(fmaf(x.x, cs, -x.y * sn), fmaf(x.x, sn, x.y * cs)));
        }
        return x;
    };
    // pass 1: HBM -> (phase) -> DFT -> twiddle -> shared memory
    float2 cur[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) cur[r] = sample(t + r * S1);
#pragma unroll
    for (int s = 0; s < G1; ++s) {
        const int lo = t + SC::T * s;
        float2 nxt[R1];
        if (s + 1 < G1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) nxt[r] = sample(lo + SC::T + r * S1);
        }
        dft_reg<R1, false>(cur);
        grp_twiddle<R1, S1, false>(tw, lo, cur);
        grp_smem_store<R1, S1>(sm, lo, SC::PADSH, cur);
        if (s + 1 < G1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) cur[r] = nxt[r];
        }
    }
    __syncthreads();
    if constexpr (SC::P == 3) {
        streamed_mid_pass<SC, SC::R2, SC::S2, false, true>(sm, tw + R1 * S1, t);
        __syncthreads();
    }
    // last pass into registers, then natural order through shared memory
    float2 v[SC::E];
#pragma unroll
    for (int s = 0; s < GL; ++s) {
        float2 x[RL];
        grp_smem_load<RL, 1>(sm, (t + SC::T * s) * RL, SC::PADSH, x);
        dft_reg<RL, false>(x);
#pragma unroll
        for (int r = 0; r < RL; ++r) v[s * RL + r] = x[r];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < GL; ++s) {
#pragma unroll
        for (int r = 0; r < RL; ++r) sm[smem_pos(natural_index<SC>(t + SC::T * s, r), SC::PADSH)] = v[s * RL + r];
    }
    __syncthreads();
    constexpr float inv_n = 1.0f / SC::N;
    float2* dst = out + line * SC::N;
#pragma unroll
    for (int i = 0; i < SC::E; ++i) {
        const int k = t + SC::T * i;
        const float2 x = sm[smem_pos(k, SC::PADSH)];
        __stcs(dst + k, COMPRESS ? make_float2(x.x * inv_n, -x.y * inv_n) : x);
    }
}

namespace {
using A256 = Sched<256, 16, 16, 16>;
using A512 = Sched<512, 32, 16, 32>;
using A1024 = Sched<1024, 32, 32, 32>;
using A2048 = Sched<2048, 16, 16, 8, 16>;
using A4096 = Sched<4096, 32, 16, 16, 16>;
using A8192 = Sched<8192, 32, 16, 16, 32>;
using A16384 = Sched<16384, 32, 16, 32, 32>;

template <class SC, bool COMPRESS>
cudaError_t launch_az(const float2* in, float2* out, int64_t n_lines, const float2* tw, const RdColumn* cols,
                      double r_near, cudaStream_t st) {
    constexpr int smem = SC::SMEM_ELEMS * 8;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(az_streamed_kernel<SC, COMPRESS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    az_streamed_kernel<SC, COMPRESS><<<(unsigned)n_lines, SC::T, smem, st>>>(in, out, n_lines, tw, cols, r_near);
    return cudaGetLastError();
}

template <bool COMPRESS>
cudaError_t launch_az_n(int n, const float2* in, float2* out, int64_t n_lines, const float2* tw, const RdColumn* c,
                        double r_near, cudaStream_t st) {
    switch (n) {
        case 256: return launch_az<A256, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
        case 512: return launch_az<A512, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
        case 1024: return launch_az<A1024, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
        case 2048: return launch_az<A2048, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
        case 4096: return launch_az<A4096, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
        case 8192: return launch_az<A8192, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
        case 16384: return launch_az<A16384, COMPRESS>(in, out, n_lines, tw, c, r_near, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

// The schedule whose twiddle tables the azimuth kernel of length n uses.
const char* rd_az_schedule(int n) {
    switch (n) {
        case 256: return "n256_e16_r16x16_l8";
        case 512: return "n512_e32_r16x32_l8";
        case 1024: return "n1024_e32_r32x32_l4";
        case 2048: return "n2048_e16_r16x8x16_l1";
        case 4096: return "n4096_e32_r16x16x16_l1";
        case 8192: return "n8192_e32_r16x16x32_l1";
        case 16384: return "n16384_e32_r16x32x32_l1";
    }
    return nullptr;
}

cudaError_t launch_az_compress_rd(int n, const float2* in, float2* out, int64_t n_lines, const float2* tw,
                                  const void* cols, double r_near, cudaStream_t st) {
    return launch_az_n<true>(n, in, out, n_lines, tw, (const RdColumn*)cols, r_near, st);
}

// Forward FFT of n_lines lines of n (natural order in and out, in place
// allowed) with the twiddles of rd_az_schedule(n).
cudaError_t launch_az_fft_rd(int n, const float2* in, float2* out, int64_t n_lines, const float2* tw,
                             cudaStream_t st) {
    return launch_az_n<false>(n, in, out, n_lines, tw, nullptr, 0.0, st);
}

cudaError_t launch_rcmc(int taps, const float2* in, float2* out, int n_range, int n_f, const void* cols,
                        double r_near, int staged_rows, cudaStream_t st) {
    if (taps != 16 || n_range <= 0 || n_f <= 0) return cudaErrorInvalidValue;
    if (staged_rows > kRcMaxStaged) staged_rows = 0;   // too wide: every block reads global memory
    const size_t smem = (size_t)staged_rows * kRcCols * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(rcmc_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const float rn_hi = (float)r_near, rn_lo = (float)(r_near - (double)rn_hi);
    const dim3 grid((unsigned)((n_f + kRcCols - 1) / kRcCols), (unsigned)((n_range + kRcRows - 1) / kRcRows));
    rcmc_tile_kernel<<<grid, kRcCols * kRcWarps, smem, st>>>(in, out, n_range, n_f, (const RdColumn*)cols, rn_hi,
                                                            rn_lo, staged_rows);
    return cudaGetLastError();
}

// Host: rows a tile must stage, the largest over every tile of the scene:
// 128 bins + 15 taps + the spread of the shift r (1/D - 1) over the tile's
// 32 columns and 128 bins, plus 4 rows of margin for rounding.
int rcmc_staged_rows(int n_range, int n_f, double r_near, const void* host_cols) {
    const RdColumn* c = (const RdColumn*)host_cols;
    double spread = 0;
    for (int g = 0; g < n_f; g += kRcCols) {
        double mn = 1e300, mx = -1e300;
        for (int j = g; j < g + kRcCols && j < n_f; ++j) {
            const double m = (double)c[j].mig_hi + (double)c[j].mig_lo;
            mn = m < mn ? m : mn;
            mx = m > mx ? m : mx;
        }
        for (int n0 = 0; n0 < n_range; n0 += kRcRows) {
            const int n1 = (n0 + kRcRows < n_range ? n0 + kRcRows : n_range) - 1;
            const double d = (r_near + n1) * mx - (r_near + n0) * mn;
            spread = d > spread ? d : spread;
        }
    }
    const double rows = kRcRows + 15 + ceil(spread) + 4;
    return rows > kRcMaxStaged ? kRcMaxStaged + 1 : (int)rows;
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
