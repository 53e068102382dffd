// Line lengths with prime factors 2, 3, 5 and 7 only (1000, 3000, 5000, ...):
// the fused line compression (Sec. II-B: load, FFT, multiply by the matched
// filter, IFFT, store; two device-memory transfers per line) at the line's
// own length, by a mixed-radix decimation-in-frequency engine.
//
// The length is factored into P <= 4 radices R_0 ... R_{P-1} (each at most
// 32, fewest passes first, then the most balanced).  Pass i works on groups
// of R_i elements at stride S_i = n / (R_0 ... R_i): group g sits at
// positions base + r S_i, base = (g / S_i) R_i S_i + g mod S_i, takes an
// R_i-point DFT in registers and (forward passes before the last) multiplies
// element r by W_{R_i S_i}^{(g mod S_i) r}.  Positions never move, so after
// the last pass position P = sum_i k_i S_i holds X[k_0 + R_0 (k_1 + R_1 (k_2
// + ...))] (mixed-radix digit reversal); the filter is stored in exactly that
// position order with 1/n folded in, and the inverse mirrors the passes with
// conjugate twiddles back to natural order.  Twiddles and the filter order
// are designed on the host and in FP64 at plan time.
//
// The radix of a pass is a runtime value (one kernel serves every length):
// each group's work is dispatched on it to a routine compiled for that
// radix, whose register array is indexed only by compile-time constants.  An
// R-point DFT is a recursive decimation in frequency over its smallest factor
// (radix-4, then 2, 3, 5, 7 butterflies; the odd ones through the symmetry
// of their roots), with compile-time twiddles from the same series as the
// power-of-two engine.
//
// Blocks of 256 threads: T threads per line (a power of two covering about
// half the largest group count of a pass), 256 / T lines per block; a line
// lives in shared memory between passes, padded with one slot per 32
// elements.  Group indexes are split by a multiply-high with ceil(2^32 / S)
// instead of an integer division (exact for every index below 2^19).
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "launch.cuh"
#include "mixed_radix.h"
#include "registry.h"

namespace sar {

namespace {

constexpr int kMixedThreads = 256;
constexpr int kMaxPasses = 4;
constexpr int kRadices[] = {32, 25, 20, 16, 15, 14, 12, 10, 9, 8, 7, 6, 5, 4, 3, 2};

struct MixedGeom {
    int n, P;
    int R[kMaxPasses], S[kMaxPasses], tw_off[kMaxPasses];
    uint32_t M[kMaxPasses];   // ceil(2^32 / S): g / S == umulhi(g, M) for every g < 8192 and 2 <= S <= 8192
                              // (checked exhaustively); 0 for S == 1
    int T;                    // threads per line; kMixedThreads / T lines per block
};

__device__ __forceinline__ int mpad(int p) { return p + (p >> 5); }

// ---- R-point DFT in registers (natural order in and out) -------------------
__host__ __device__ constexpr int small_factor(int L) {
    return L % 4 == 0 ? 4 : L % 2 == 0 ? 2 : L % 3 == 0 ? 3 : L % 5 == 0 ? 5 : L % 7 == 0 ? 7 : L;
}
// position of output k of a length-L DIF over factors small_factor(L), ...
__host__ __device__ constexpr int mpos(int L, int k) {
    return L == 1 ? 0 : ((k % small_factor(L)) * (L / small_factor(L)) + mpos(L / small_factor(L), k / small_factor(L)));
}

// p-point DFT of a[0..p-1] for an odd prime p, by the symmetry of the
// roots: with a_k = x_k + x_{p-k} and b_k = x_k - x_{p-k} (k = 1 .. h,
// h = (p - 1) / 2),
//   y_0 = x_0 + sum_k a_k,
//   y_j = t_j -+ i u_j,  y_{p-j} = t_j +- i u_j   (j = 1 .. h; upper signs
//   forward), t_j = x_0 + sum_k cos(2 pi j k / p) a_k,
//   u_j = sum_k sin(2 pi j k / p) b_k,
// real constants only: about 5 instructions per output at p = 5 instead of
// the 16 of the definition's p - 1 complex products per output.
template <int p, int j, int... K>
__device__ __forceinline__ float2 odd_t(float2 x0, const float2 (&av)[p], std::integer_sequence<int, K...>) {
    float2 t = x0;
    ((t = make_float2(fmaf((float)ct::cos2pi((K + 1) * j, p), av[K + 1].x, t.x),
                      fmaf((float)ct::cos2pi((K + 1) * j, p), av[K + 1].y, t.y))),
     ...);
    return t;
}
template <int p, int j, int... K>
__device__ __forceinline__ float2 odd_u(const float2 (&bv)[p], std::integer_sequence<int, K...>) {
    float2 u = make_float2(0.f, 0.f);
    ((u = make_float2(fmaf((float)ct::sin2pi((K + 1) * j, p), bv[K + 1].x, u.x),
                      fmaf((float)ct::sin2pi((K + 1) * j, p), bv[K + 1].y, u.y))),
     ...);
    return u;
}
template <int p, bool INV, int... J>
__device__ __forceinline__ void dft_odd_outputs(float2 (&a)[p], float2 x0, const float2 (&av)[p],
                                                const float2 (&bv)[p], std::integer_sequence<int, J...>) {
    constexpr int h = (p - 1) / 2;
    float2 y[p];
    (([&] {
         constexpr int j = J + 1;
         const float2 t = odd_t<p, j>(x0, av, std::make_integer_sequence<int, h>{});
         const float2 u = odd_u<p, j>(bv, std::make_integer_sequence<int, h>{});
         // -i u = (u.y, -u.x); +i u = (-u.y, u.x)
         const float2 mi = make_float2(u.y, -u.x);
         y[j] = INV ? csub(t, mi) : cadd(t, mi);
         y[p - j] = INV ? cadd(t, mi) : csub(t, mi);
     }()),
     ...);
#pragma unroll
    for (int k = 1; k < p; ++k) a[k] = y[k];
}
template <int p, bool INV>
__device__ __forceinline__ void dft_odd(float2 (&a)[p]) {
    constexpr int h = (p - 1) / 2;
    float2 av[p], bv[p];
    float2 y0 = a[0];
#pragma unroll
    for (int k = 1; k <= h; ++k) {
        av[k] = cadd(a[k], a[p - k]);
        bv[k] = csub(a[k], a[p - k]);
        y0 = cadd(y0, av[k]);
    }
    const float2 x0 = a[0];
    dft_odd_outputs<p, INV>(a, x0, av, bv, std::make_integer_sequence<int, h>{});
    a[0] = y0;
}

template <int R, int L, int OFF, bool INV, int J, int... K>
__device__ __forceinline__ void mlevel_store(float2 (&v)[R], const float2 (&a)[small_factor(L)],
                                             std::integer_sequence<int, K...>) {
    constexpr int q = L / small_factor(L);
    ((v[OFF + J + K * q] = twiddle_ct<L, J * K, INV>(a[K])), ...);
}
// one butterfly column j of the level of length L at offset OFF: the p
// elements OFF + j + m q (q = L / p), their p-point DFT, twiddles W_L^{j k}
template <int R, int L, int OFF, bool INV, int J>
__device__ __forceinline__ void mlevel_one(float2 (&v)[R]) {
    constexpr int p = small_factor(L), q = L / p;
    float2 a[p];
#pragma unroll
    for (int m = 0; m < p; ++m) a[m] = v[OFF + J + m * q];
    if constexpr (p == 4) {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]), t2 = cadd(a[1], a[3]);
        const float2 t3 = cmul_mi<INV>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[1] = cadd(t1, t3);
        a[2] = csub(t0, t2);
        a[3] = csub(t1, t3);
    } else if constexpr (p == 2) {
        const float2 t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    } else {
        dft_odd<p, INV>(a);
    }
    mlevel_store<R, L, OFF, INV, J>(v, a, std::make_integer_sequence<int, p>{});
}
template <int R, int L, int OFF, bool INV, int... J>
__device__ __forceinline__ void mlevel(float2 (&v)[R], std::integer_sequence<int, J...>) {
    (mlevel_one<R, L, OFF, INV, J>(v), ...);
}
template <int R, int L, int OFF, bool INV, int... K>
__device__ __forceinline__ void mrec_children(float2 (&v)[R], std::integer_sequence<int, K...>);
template <int R, int L, int OFF, bool INV>
__device__ __forceinline__ void mrec(float2 (&v)[R]) {
    if constexpr (L > 1) {
        constexpr int p = small_factor(L), q = L / p;
        mlevel<R, L, OFF, INV>(v, std::make_integer_sequence<int, q>{});
        mrec_children<R, L, OFF, INV>(v, std::make_integer_sequence<int, p>{});
    }
}
template <int R, int L, int OFF, bool INV, int... K>
__device__ __forceinline__ void mrec_children(float2 (&v)[R], std::integer_sequence<int, K...>) {
    constexpr int q = L / small_factor(L);
    (mrec<R, q, OFF + K * q, INV>(v), ...);
}
template <int R, int... K>
__device__ __forceinline__ void munscramble(const float2 (&v)[R], float2 (&o)[R], std::integer_sequence<int, K...>) {
    ((o[K] = v[mpos(R, K)]), ...);
}
// v[k] <- sum_m v[m] exp(-+2 pi i m k / R)
template <int R, bool INV>
__device__ __forceinline__ void dft_any(float2 (&v)[R]) {
    if constexpr (R > 1) {
        mrec<R, R, 0, INV>(v);
        float2 o[R];
        munscramble<R>(v, o, std::make_integer_sequence<int, R>{});
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = o[k];
    }
}

// ---- one group of one pass ---------------------------------------------------
enum MMode { kFirst, kMid, kLast, kInvMid, kInvFirst };

// MODE: kFirst global -> DFT -> twiddle -> smem; kMid smem -> DFT -> twiddle
// -> smem; kLast (src global when P == 1) -> DFT -> filter -> IDFT -> smem (or
// global when P == 1); kInvMid smem -> conj twiddle -> IDFT -> smem; kInvFirst
// smem -> conj twiddle -> IDFT -> global.
template <int R, int MODE, bool SINGLE>
__device__ __forceinline__ void mgroup(int g, int S, uint32_t M, const float2* src, float2* dst, float2* sm,
                                       const float2* twi, const float2* filt) {
    const int q = M ? (int)__umulhi((uint32_t)g, M) : g;   // M == 0: S == 1
    const int lo = g - q * S, base = q * R * S + lo;
    float2 v[R];
    const bool from_global = MODE == kFirst || (MODE == kLast && SINGLE);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = from_global ? __ldcs(src + base + r * S) : sm[mpad(base + r * S)];
    if constexpr (MODE == kInvMid || MODE == kInvFirst) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], twi[r * S + lo]);
        dft_any<R, true>(v);
    } else {
        dft_any<R, false>(v);
        if constexpr (MODE == kLast) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = cmul(v[r], filt[base + r]);
            dft_any<R, true>(v);
        } else {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twi[r * S + lo]);
        }
    }
    const bool to_global = MODE == kInvFirst || (MODE == kLast && SINGLE);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (to_global)
            __stcs(dst + base + r * S, v[r]);
        else
            sm[mpad(base + r * S)] = v[r];
    }
}

template <int MODE, bool SINGLE>
__device__ __forceinline__ void mpass(int R, int S, uint32_t M, int n, int t, int T, const float2* src, float2* dst,
                                      float2* sm, const float2* twi, const float2* filt) {
    const int ng = n / R;
#define SAR_MIXED_CASE(RR)                                                                       \
    case RR:                                                                                     \
        for (int g = t; g < ng; g += T) mgroup<RR, MODE, SINGLE>(g, S, M, src, dst, sm, twi, filt); \
        break;
    switch (R) {
        SAR_MIXED_CASE(2)
        SAR_MIXED_CASE(3)
        SAR_MIXED_CASE(4)
        SAR_MIXED_CASE(5)
        SAR_MIXED_CASE(6)
        SAR_MIXED_CASE(7)
        SAR_MIXED_CASE(8)
        SAR_MIXED_CASE(9)
        SAR_MIXED_CASE(10)
        SAR_MIXED_CASE(12)
        SAR_MIXED_CASE(14)
        SAR_MIXED_CASE(15)
        SAR_MIXED_CASE(16)
        SAR_MIXED_CASE(20)
        SAR_MIXED_CASE(25)
        SAR_MIXED_CASE(32)
        default: break;
    }
#undef SAR_MIXED_CASE
}

// Lines of T threads each, kMixedThreads / T lines per block (lines past the
// end still take part in the block's barriers).
__global__ void __launch_bounds__(kMixedThreads)
fused_mixed_kernel(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt, const float2* tw,
                   MixedGeom geo) {
    extern __shared__ float2 smem_mixed[];
    const int T = geo.T, lib = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t line = (int64_t)blockIdx.x * (kMixedThreads / T) + lib;
    const bool live = line < n_lines;
    const int n = geo.n, P = geo.P;
    float2* sm = smem_mixed + lib * (n + (n >> 5) + 1);
    const float2* src = in + (live ? line : 0) * ld;
    float2* dst = out + (live ? line : 0) * ld;
    if (P == 1) {
        if (live) mpass<kLast, true>(geo.R[0], 1, 0u, n, t, T, src, dst, sm, tw, filt);
        return;
    }
    if (live) mpass<kFirst, false>(geo.R[0], geo.S[0], geo.M[0], n, t, T, src, dst, sm, tw + geo.tw_off[0], filt);
    __syncthreads();
    for (int i = 1; i < P - 1; ++i) {
        if (live) mpass<kMid, false>(geo.R[i], geo.S[i], geo.M[i], n, t, T, src, dst, sm, tw + geo.tw_off[i], filt);
        __syncthreads();
    }
    if (live) mpass<kLast, false>(geo.R[P - 1], 1, 0u, n, t, T, src, dst, sm, tw, filt);
    __syncthreads();
    for (int i = P - 2; i >= 1; --i) {
        if (live) mpass<kInvMid, false>(geo.R[i], geo.S[i], geo.M[i], n, t, T, src, dst, sm, tw + geo.tw_off[i], filt);
        __syncthreads();
    }
    if (live) mpass<kInvFirst, false>(geo.R[0], geo.S[0], geo.M[0], n, t, T, src, dst, sm, tw + geo.tw_off[0], filt);
}

// tw[off_i + r S_i + lo] = exp(-2 pi i lo r / (R_i S_i)), FP64 phases rounded
// once (the exponent lo r reduced modulo R_i S_i exactly, in integers)
__global__ void mixed_twiddle_kernel(float2* tw, int R, int S) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= R * S) return;
    const int r = e / S, lo = e % S;
    const int64_t L = (int64_t)R * S;
    const int64_t m = ((int64_t)lo * r) % L;
    double s, c;
    sincospi(-2.0 * (double)m / (double)L, &s, &c);
    tw[e] = make_float2((float)c, (float)s);
}

// ---- host: factorisation, geometry, descriptors ------------------------------
bool seven_smooth(int n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// fewest radices from kRadices multiplying to n; ties: the smallest largest
// radix, then the largest smallest one (balanced passes: similar group counts
// per pass, fewer registers per group); the radices in descending order
void search(int n, int start, std::vector<int>& cur, std::vector<int>& best) {
    if (n == 1) {
        if (best.empty() || cur.size() < best.size() ||
            (cur.size() == best.size() &&
             (cur.front() < best.front() || (cur.front() == best.front() && cur.back() > best.back()))))
            best = cur;
        return;
    }
    if ((int)cur.size() >= kMaxPasses || (!best.empty() && cur.size() + 1 > best.size())) return;
    for (int i = start; i < (int)(sizeof(kRadices) / sizeof(kRadices[0])); ++i) {
        const int r = kRadices[i];
        if (n % r) continue;
        cur.push_back(r);
        search(n / r, i, cur, best);
        cur.pop_back();
    }
}

bool geometry(int n, MixedGeom& g) {
    if (n < 2 || n > 8192 || !seven_smooth(n)) return false;
    std::vector<int> cur, best;
    search(n, 0, cur, best);
    if (best.empty()) return false;
    g.n = n;
    g.P = (int)best.size();
    int rest = n, off = 0, most = 1;
    for (int i = 0; i < kMaxPasses; ++i) {
        g.R[i] = i < g.P ? best[i] : 1;
        if (i < g.P) rest /= g.R[i];
        g.S[i] = i < g.P ? rest : 1;
        g.M[i] = g.S[i] > 1 ? (uint32_t)((((uint64_t)1 << 32) + (uint64_t)g.S[i] - 1) / (uint64_t)g.S[i]) : 0u;
        g.tw_off[i] = off;
        if (i < g.P - 1) off += g.R[i] * g.S[i];
        if (i < g.P && n / g.R[i] > most) most = n / g.R[i];
    }
    // threads per line: a power of two covering about half the largest group
    // count of a pass (one or two groups per thread), 32 ... kMixedThreads
    g.T = 32;
    while (g.T < kMixedThreads && 2 * g.T < most) g.T <<= 1;
    return true;
}

int twiddle_elems(const MixedGeom& g) {
    int e = 0;
    for (int i = 0; i < g.P - 1; ++i) e += g.R[i] * g.S[i];
    return e > 0 ? e : 1;
}

int lines_per_block(const MixedGeom& g) { return kMixedThreads / g.T; }
int smem_bytes(const MixedGeom& g) { return lines_per_block(g) * (g.n + (g.n >> 5) + 1) * (int)sizeof(float2); }

cudaError_t launch_mixed(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* filt,
                         const float2* tw, const FusedCtl&, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    MixedGeom g{};
    if (!geometry(valid, g)) return cudaErrorInvalidValue;
    const int lpb = lines_per_block(g);
    fused_mixed_kernel<<<(unsigned)((n_lines + lpb - 1) / lpb), kMixedThreads, smem_bytes(g), st>>>(in, out, n_lines,
                                                                                                    ld, filt, tw, g);
    return cudaGetLastError();
}

// the largest block shared memory of any length: eight lines of at most
// 1024 samples or one of 8192, about 68 KiB
cudaError_t prepare_mixed() {
    return cudaFuncSetAttribute(fused_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 72 * 1024);
}

struct Entry {
    std::string name;
    SchedDesc desc;
};
std::mutex g_mu;
std::map<int, Entry*> g_descs;   // never freed: the descriptors live as long as the library

}  // namespace

bool mixed_length(int n) {
    MixedGeom g{};
    return geometry(n, g);
}

const SchedDesc* mixed_schedule(int n) {
    MixedGeom g{};
    if (!geometry(n, g)) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_descs.find(n);
    if (it != g_descs.end()) return &it->second->desc;
    Entry* e = new Entry;
    e->name = "n" + std::to_string(n) + "_mixed_r";
    for (int i = 0; i < g.P; ++i) e->name += (i ? "x" : "") + std::to_string(g.R[i]);
    e->desc = SchedDesc{e->name.c_str(), n, 0, g.R[0], g.P > 1 ? g.R[1] : 1, g.P > 2 ? g.R[2] : 1,
                        lines_per_block(g), kMixedThreads, smem_bytes(g), twiddle_elems(g), g.R[g.P - 1], 0,
                        &launch_mixed, nullptr, &prepare_mixed, nullptr, 0, nullptr, 0};
    e->desc.mixed = 1;
    g_descs[n] = e;
    return &e->desc;
}

cudaError_t build_mixed_twiddles(int n, float2* tw, cudaStream_t st) {
    MixedGeom g{};
    if (!geometry(n, g)) return cudaErrorInvalidValue;
    for (int i = 0; i < g.P - 1; ++i) {
        const int cnt = g.R[i] * g.S[i];
        mixed_twiddle_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(tw + g.tw_off[i], g.R[i], g.S[i]);
    }
    return cudaGetLastError();
}

// position P = sum_i k_i S_i -> frequency k_0 + R_0 (k_1 + R_1 (k_2 + ...))
void mixed_positions(int n, int32_t* idx) {
    MixedGeom g{};
    if (!geometry(n, g)) return;
    for (int P = 0; P < n; ++P) {
        int rem = P, digits[kMaxPasses];
        for (int i = 0; i < g.P; ++i) {
            digits[i] = rem / g.S[i];
            rem %= g.S[i];
        }
        int k = 0;
        for (int i = g.P - 1; i >= 0; --i) k = digits[i] + g.R[i] * k;
        idx[P] = k;
    }
}

}  // namespace sar
