// Point-target echo simulator on the device (the chirp signal model of the
// paper's Sec. V-A, with the normalised parameters of the benchmark scenes).
//
// Sample (a, r) of an n_az x n_range echo is
//     sum over targets (a0, r0):  c_a(a - a0) * c_r(r - r0)      (indices mod n)
//   + noise(a * n_range + r)
// with c(m) = exp(i pi (tbp / nc^2) m^2) for m in [-nc/2, nc - nc/2), zero
// outside, and circular complex Gaussian noise of total variance
// 10^(-snr_db/10).  Random numbers are counter-based: value i of stream s under
// seed S is splitmix64(key + (i + 1) * 0x9E3779B97F4A7C15) with
// key = splitmix64(S xor s * 0xD1B54A32D192ED03) (Steele, Lea and Flood,
// OOPSLA 2014; Vigna's finaliser); uniforms take the top 53 bits; noise sample
// j uses uniforms 2j (radius, as 1 - u) and 2j + 1 (angle) in the Box-Muller
// transform.  Every step is evaluated in FP64 without contraction in the same
// order as the host generator, the noise rounded to complex64 before it is
// added, the sum rounded to complex64 at the end.
#include <math.h>

#include "../../include/sar.h"
#include "tables.h"

namespace sar {
sar_status report_error(sar_status st, const char *msg);
sar_status validate_device_ptr(const void *p, const char *what);
}  // namespace sar

namespace {

constexpr int kMaxTargets = 32;

struct Targets {
    int64_t a0[kMaxTargets], r0[kMaxTargets];
    int n;
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t key, uint64_t i) {
    const uint64_t v = mix64(key + (i + 1ULL) * 0x9E3779B97F4A7C15ULL);
    return (double)(v >> 11) * (1.0 / 9007199254740992.0);   // 2^-53
}

// c(m) of a chirp with nc samples and time-bandwidth product tbp, m in
// [-nc/2, nc - nc/2): phase pi * (fmod(tbp m^2, 2 nc^2) / nc^2)
__device__ __forceinline__ void chirp(int64_t m, int64_t nc, double tbp, double &re, double &im) {
    const double md = (double)m;
    const double nc2 = (double)nc * (double)nc;
    const double x = __ddiv_rn(fmod(__dmul_rn(__dmul_rn(tbp, md), md), __dmul_rn(2.0, nc2)), nc2);
    const double arg = __dmul_rn(M_PI, x);
    re = cos(arg);
    im = sin(arg);
}

// offset of sample index p relative to the centre c, wrapped into
// [-nc/2, nc - nc/2), or a value outside that range if not covered
__device__ __forceinline__ int64_t chirp_offset(int64_t p, int64_t c, int64_t n, int64_t nc) {
    int64_t m = ((p - c) % n + n) % n;
    if (m >= nc - nc / 2) m -= n;
    return m;
}

__global__ void simulate_kernel(float2 *out, int64_t n_az, int64_t n_range, Targets tg, int64_t nc_r, double tbp_r,
                                int64_t nc_a, double tbp_a, double noise_sd, int noise, uint64_t key) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_az * n_range) return;
    const int64_t a = idx / n_range, r = idx % n_range;
    double sre = 0.0, sim = 0.0;
    for (int k = 0; k < tg.n; ++k) {
        const int64_t ma = chirp_offset(a, tg.a0[k], n_az, nc_a);
        const int64_t mr = chirp_offset(r, tg.r0[k], n_range, nc_r);
        if (ma < -(nc_a / 2) || ma >= nc_a - nc_a / 2 || mr < -(nc_r / 2) || mr >= nc_r - nc_r / 2) continue;
        double car, cai, crr, cri;
        chirp(ma, nc_a, tbp_a, car, cai);
        chirp(mr, nc_r, tbp_r, crr, cri);
        // (car + i cai)(crr + i cri), products and sums rounded one by one
        sre = __dadd_rn(sre, __dsub_rn(__dmul_rn(car, crr), __dmul_rn(cai, cri)));
        sim = __dadd_rn(sim, __dadd_rn(__dmul_rn(car, cri), __dmul_rn(cai, crr)));
    }
    if (noise) {
        const double u1 = __dsub_rn(1.0, uniform01(key, 2ULL * (uint64_t)idx));
        const double u2 = uniform01(key, 2ULL * (uint64_t)idx + 1ULL);
        const double rad = __dmul_rn(sqrt(__dmul_rn(-2.0, log(u1))), noise_sd);
        const double ang = __dmul_rn(__dmul_rn(2.0, M_PI), u2);
        const float nre = (float)__dmul_rn(rad, cos(ang));
        const float nim = (float)__dmul_rn(rad, sin(ang));
        sre = __dadd_rn(sre, (double)nre);
        sim = __dadd_rn(sim, (double)nim);
    }
    out[idx] = make_float2((float)sre, (float)sim);
}

uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" sar_status sar_simulate_echo(int64_t n_az, int64_t n_range, const int64_t *targets, int32_t n_targets,
                                        int64_t nc_range, double tbp_range, int64_t nc_az, double tbp_az,
                                        double snr_db, uint64_t seed, void *out, sar_stream stream) {
    if (n_az < 1 || n_range < 1 || n_az * n_range > ((int64_t)1 << 34))
        return sar::report_error(SAR_ERR_INVALID_ARG, "scene size out of range");
    if (n_targets < 0 || n_targets > kMaxTargets || (n_targets > 0 && !targets))
        return sar::report_error(SAR_ERR_INVALID_ARG, "0 ... 32 targets");
    if (nc_range < 1 || nc_range > n_range || nc_az < 1 || nc_az > n_az)
        return sar::report_error(SAR_ERR_INVALID_ARG, "chirp lengths must be in [1, n]");
    sar_status st = sar::validate_device_ptr(out, "out");
    if (st != SAR_OK) return st;
    Targets tg{};
    tg.n = n_targets;
    for (int k = 0; k < n_targets; ++k) {
        tg.a0[k] = targets[2 * k];
        tg.r0[k] = targets[2 * k + 1];
    }
    const int noise = !isnan(snr_db);
    const double sd = noise ? sqrt(pow(10.0, -snr_db / 10.0) / 2.0) : 0.0;
    const uint64_t key = host_mix64(seed ^ (2ULL * 0xD1B54A32D192ED03ULL));   // the noise stream
    const int64_t total = n_az * n_range;
    simulate_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        (float2 *)out, n_az, n_range, tg, nc_range, tbp_range, nc_az, tbp_az, sd, noise, key);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, "simulator launch failed");
    return SAR_OK;
}
