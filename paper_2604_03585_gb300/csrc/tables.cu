// Plan-time tables: FP64 twiddle and chirp phases rounded to FP32, and the
// matched filter permuted into the fused kernel's register order.
#include "mixed_radix.h"
#include "tables.h"

namespace sar {

// tw[r*S + lo] = exp(-2 pi i lo r / M) for r in [0, R), lo in [0, S).
// The argument 2*lo*r/M is an exact dyadic rational in FP64; sincospi()
// evaluates the phase in FP64 and the result is rounded once to FP32.
__global__ void twiddle_table_kernel(float2 *tw, int R, int S, int M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * S) return;
    const int r = i / S, lo = i % S;
    const long long e = ((long long)lo * r) % M;
    double s, c;
    sincospi(-2.0 * (double)e / (double)M, &s, &c);
    tw[i] = make_float2((float)c, (float)s);
}

// The four-step twiddles of a line of n = C m samples on a cluster of C
// blocks: out[k1 m + n2] = exp(-2 pi i k1 n2 / n), k1 < C, n2 < m, evaluated
// like the twiddles above (k1 n2 < n, no reduction needed).  Row k1 is the
// twiddle set of one block of the cluster, contiguous in n2, so that a
// warp's consecutive n2 read one run of the table.
__global__ void roots_table_kernel(float2 *out, int n, int m) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const long long e = (long long)(j / m) * (j % m);
    double s, c;
    sincospi(-2.0 * (double)e / (double)n, &s, &c);
    out[j] = make_float2((float)c, (float)s);
}

// One length-n line holding the chirp c(m) = exp(i pi K m^2), K = tbp/nc^2,
// m = -nc/2 ... nc/2 - 1, at position m mod n; zero elsewhere.  The phase in
// units of pi, tbp*m^2/nc^2, is reduced modulo 2 in FP64 before sincospi().
__global__ void lfm_line_kernel(float2 *line, int n, int nc, double tbp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int half = nc / 2;
    long long m;
    bool on = false;
    if (p < nc - half) { m = p; on = true; }
    else if (p >= n - half) { m = (long long)p - n; on = true; }
    if (!on) { line[p] = make_float2(0.f, 0.f); return; }
    const double nc2 = (double)nc * (double)nc;
    const double x = fmod(tbp * (double)(m * m), 2.0 * nc2) / nc2;
    double s, c;
    sincospi(x, &s, &c);
    line[p] = make_float2((float)c, (float)s);
}

__global__ void conj_kernel(float2 *x, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i].y = -x[i].y;
}

// dst[i] = H[idx[i]] * scale   (scale = 1/N, a power of two: exact)
__global__ void gather_scale_kernel(float2 *dst, const float2 *H, const int32_t *idx, int n, float scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 h = H[idx[i]];
    dst[i] = make_float2(h.x * scale, h.y * scale);
}

// data[l][k] *= h[k] for n_lines lines of n (two samples per thread)
__global__ void spectrum_multiply_kernel(float4 *data, const float4 *h, int64_t total2, int64_t n2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total2; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = data[i], w = h[i % n2];
        data[i] = make_float4(fmaf(x.x, w.x, -x.y * w.y), fmaf(x.x, w.y, x.y * w.x), fmaf(x.z, w.z, -x.w * w.w),
                              fmaf(x.z, w.w, x.w * w.z));
    }
}

// dst[k] = H[k] * scale (natural order)
__global__ void scale_copy_kernel(float2 *dst, const float2 *H, int n, float scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_float2(H[i].x * scale, H[i].y * scale);
}

cudaError_t spectrum_multiply(float2 *data, const float2 *h, int64_t n_lines, int64_t n, cudaStream_t st) {
    const int64_t total2 = n_lines * n / 2;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (total2 + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    spectrum_multiply_kernel<<<(unsigned)blocks, 256, 0, st>>>((float4 *)data, (const float4 *)h, total2, n / 2);
    return cudaGetLastError();
}

// --- filter of a line length that is not a power of two -------------------
// roots[e] = exp(sign 2 pi i e / m), e < m, FP64.
__global__ void roots_f64_kernel(double2 *roots, int m, int sign) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    double s, c;
    sincospi((double)sign * 2.0 * (double)e / (double)m, &s, &c);
    roots[e] = make_double2(c, s);
}

// out[j] = scale * sum_{q < n_in} in[q] roots[(j q) mod m], FP64, one warp per
// output j < n_out; in is complex64 (IN_F32) or complex128.
template <bool IN_F32>
__global__ void dft_f64_kernel(const void *in_, int n_in, const double2 *roots, int m, int n_out, double scale,
                               double2 *out64, float2 *out32) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n_out) return;
    double re = 0.0, im = 0.0;
    for (int q = lane; q < n_in; q += 32) {
        double xr, xi;
        if (IN_F32) {
            const float2 v = ((const float2 *)in_)[q];
            xr = v.x;
            xi = v.y;
        } else {
            const double2 v = ((const double2 *)in_)[q];
            xr = v.x;
            xi = v.y;
        }
        const double2 w = roots[((int64_t)j * q) % m];
        re = fma(xr, w.x, fma(-xi, w.y, re));
        im = fma(xr, w.y, fma(xi, w.x, im));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        if (out64) out64[j] = make_double2(re * scale, im * scale);
        if (out32) out32[j] = make_float2((float)(re * scale), (float)(im * scale));
    }
}

size_t wrap_filter_scratch_bytes(int n, int L) { return sizeof(double2) * ((size_t)2 * n + (size_t)L); }

// G = FFT_L(h zero-padded to L), h = IFFT_n(H), both by their definitions in
// FP64 (plan time, O(n L)), G rounded once to FP32.  scratch holds
// wrap_filter_scratch_bytes(n, L) bytes.
cudaError_t build_wrap_filter(const float2 *H, int n, int L, void *scratch, float2 *G, cudaStream_t st) {
    double2 *roots_n = (double2 *)scratch, *h = roots_n + n, *roots_L = h + n;
    roots_f64_kernel<<<(n + 255) / 256, 256, 0, st>>>(roots_n, n, +1);
    roots_f64_kernel<<<(L + 255) / 256, 256, 0, st>>>(roots_L, L, -1);
    dft_f64_kernel<true><<<(n + 7) / 8, 256, 0, st>>>(H, n, roots_n, n, n, 1.0 / (double)n, h, nullptr);
    dft_f64_kernel<false><<<(L + 7) / 8, 256, 0, st>>>(h, n, roots_L, L, L, 1.0, nullptr, G);
    return cudaGetLastError();
}

// --- tables of the DFT of a length that is not a power of two (Bluestein) --
// chirp[m] = c_m = exp(-i pi m^2 / n) for m < n, the phase reduced exactly as
// (m^2 mod 2n) / n before sincospi in FP64; b[m] (m < L) = conj(c_{m'}) for the
// lag m' = m (m < n) or L - m (m > L - n), else 0.
__global__ void bluestein_chirp_kernel(float2 *chirp, double2 *b, int n, int L) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    auto c64 = [n](int64_t k) {
        const int64_t q = (k * k) % (2 * (int64_t)n);
        double s, c;
        sincospi(-(double)q / (double)n, &s, &c);
        return make_double2(c, s);
    };
    if (m < n) {
        const double2 c = c64(m);
        chirp[m] = make_float2((float)c.x, (float)c.y);
        b[m] = make_double2(c.x, -c.y);
    } else if (m > L - n) {
        const double2 c = c64(L - m);
        b[m] = make_double2(c.x, -c.y);
    } else {
        b[m] = make_double2(0.0, 0.0);
    }
}

size_t bluestein_scratch_bytes(int L) { return sizeof(double2) * (size_t)2 * L; }

// chirp (n values) and G = FFT_L(b) (L values, FP64 sums rounded once).
cudaError_t build_bluestein_tables(int n, int L, float2 *chirp, float2 *G, void *scratch, cudaStream_t st) {
    double2 *b = (double2 *)scratch, *roots_L = b + L;
    bluestein_chirp_kernel<<<(L + 255) / 256, 256, 0, st>>>(chirp, b, n, L);
    roots_f64_kernel<<<(L + 255) / 256, 256, 0, st>>>(roots_L, L, -1);
    dft_f64_kernel<false><<<(L + 7) / 8, 256, 0, st>>>(b, L, roots_L, L, L, 1.0, nullptr, G);
    return cudaGetLastError();
}

cudaError_t build_natural_filter(const float2 *H, float2 *dst, int n, cudaStream_t st) {
    scale_copy_kernel<<<(n + 255) / 256, 256, 0, st>>>(dst, H, n, 1.0f / (float)n);
    return cudaGetLastError();
}

cudaError_t build_twiddles(const SchedDesc &d, float2 *tw, cudaStream_t st) {
    if (d.mixed) return build_mixed_twiddles(d.n, tw, st);
    const int M = d.cluster > 1 ? d.n / d.cluster : d.n;   // the per-block engine's length
    const int S1 = M / d.r1;
    int total = d.r1 * S1;
    twiddle_table_kernel<<<(total + 255) / 256, 256, 0, st>>>(tw, d.r1, S1, M);
    if (d.r3 > 1) {
        const int S2 = S1 / d.r2;
        const int t2 = d.r2 * S2;
        twiddle_table_kernel<<<(t2 + 255) / 256, 256, 0, st>>>(tw + total, d.r2, S2, S1);
        total += t2;
    }
    if (d.cluster > 1) roots_table_kernel<<<(d.n + 255) / 256, 256, 0, st>>>(tw + total, d.n, M);
    return cudaGetLastError();
}

cudaError_t build_filter(const SchedDesc &d, const float2 *H, float2 *filt, int32_t *idx_dev, cudaStream_t st) {
    gather_scale_kernel<<<(d.n + 255) / 256, 256, 0, st>>>(filt, H, idx_dev, d.n, 1.0f / (float)d.n);
    return cudaGetLastError();
}

cudaError_t make_lfm_line(int n, int nc, double tbp, float2 *out, cudaStream_t st) {
    lfm_line_kernel<<<(n + 255) / 256, 256, 0, st>>>(out, n, nc, tbp);
    return cudaGetLastError();
}

cudaError_t conjugate(float2 *x, int n, cudaStream_t st) {
    conj_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, n);
    return cudaGetLastError();
}

}  // namespace sar
