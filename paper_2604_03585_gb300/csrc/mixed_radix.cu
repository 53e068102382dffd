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
// + ...))] (mixed-radix digit reversal); the filter is stored in that order
// with 1/n folded in (slot r (n / R_L) + q for position q R_L + r, so that
// the last pass's lanes read it coalesced), and the inverse mirrors the passes with
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
// instead of an integer division (exact for every index below 2^19).  The
// kernel is compiled with registers capped for 2, 3 and 4 blocks per SM
// (mixed_radix_k*.cu) and the variant is chosen by length.
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "mixed_radix.cuh"
#include "mixed_radix.h"
#include "registry.h"

namespace sar {

namespace mixed {
// tw[off_i + r S_i + lo] = exp(-2 pi i lo r / (R_i S_i)), FP64 phases rounded
// once (the exponent lo r reduced modulo R_i S_i exactly, in integers)
// pos[k] = sum_i k_i S_i for k = k_0 + R_0 (k_1 + R_1 (k_2 + ...)): where the
// forward passes leave frequency k
__global__ void mixed_positions_kernel(int32_t* pos, MixedGeom g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    int rem = k, p = 0;
    for (int i = 0; i < g.P; ++i) {
        p += (rem % g.R[i]) * g.S[i];
        rem /= g.R[i];
    }
    pos[k] = p;
}

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

}  // namespace mixed

namespace {
using namespace mixed;

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
    g.pos_off = off;
    // threads per line: a power of two covering about half the largest group
    // count of a pass (one or two groups per thread), 32 ... kMixedThreads
    g.T = 32;
    while (g.T < kMixedThreads && 2 * g.T < most) g.T <<= 1;
    // and the block's lines within the shared memory the kernel is set up for
    while (g.T < kMixedThreads && (kMixedThreads / g.T) * (n + (n >> 5) + 1) * 8 > kMixedSmemMax) g.T <<= 1;
    return true;
}

// the inter-pass twiddles, then the plain transform's position table
int twiddle_elems(const MixedGeom& g) { return g.pos_off + (g.n + 1) / 2; }

int lines_per_block(const MixedGeom& g) { return kMixedThreads / g.T; }
int smem_bytes(const MixedGeom& g) { return lines_per_block(g) * (g.n + (g.n >> 5) + 1) * (int)sizeof(float2); }

// Register cap of the kernel for length n (blocks per SM), measured on GB300
// over 1000 ... 8000: short lines gain from four blocks per SM, long ones lose
// to the spills of the tighter cap while shared memory admits few lines anyway.
int occupancy_variant(int n) { return n <= 4096 ? 4 : n <= 6000 ? 3 : 2; }

cudaError_t launch_mixed(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* filt,
                         const float2* tw, const FusedCtl&, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    MixedGeom g{};
    if (!geometry(valid, g)) return cudaErrorInvalidValue;
    const int lpb = lines_per_block(g), smem = smem_bytes(g);
    // SAR_MIXED_GENERIC=1: the runtime kernel even where a specialisation
    // exists (the two give bit-identical results; tests compare them)
    const char* generic = getenv("SAR_MIXED_GENERIC");
    if (!(generic && generic[0] == '1'))
        if (const mixed3_fn f = specialised(g))
            return f(in, out, n_lines, ld, filt, tw, smem, st);
    switch (occupancy_variant(valid)) {
        case 4: return launch_k4(in, out, n_lines, ld, filt, tw, g, lpb, smem, st);
        case 3: return launch_k3(in, out, n_lines, ld, filt, tw, g, lpb, smem, st);
        default: return launch_k2(in, out, n_lines, ld, filt, tw, g, lpb, smem, st);
    }
}

cudaError_t launch_mixed_dft(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                             int inverse, cudaStream_t st) {
    if (n_lines <= 0) return cudaSuccess;
    MixedGeom g{};   // whole lines: valid is the length (as in launch_mixed)
    if (!geometry(valid, g)) return cudaErrorInvalidValue;
    const char* generic = getenv("SAR_MIXED_GENERIC");
    if (!(generic && generic[0] == '1'))
        if (const mixed3_dft_fn f = specialised_dft(g)) return f(in, out, n_lines, ld, valid, tw, g.pos_off, inverse, st);
    return launch_dft_mixed(in, out, n_lines, ld, valid, tw, inverse, g, lines_per_block(g), smem_bytes(g), st);
}

// the folded range pass of the plan's length (fused_ct of the descriptor):
// the compiled kernel of its length, which exists when the descriptor
// offers this entry.  One entry serves every mixed length, so the length is
// taken from ld_in: raw rows are contiguous lines of n samples on every
// caller of fused_ct.
cudaError_t launch_mixed_ct(const float2* in, float2* img, int64_t n_lines, int64_t ld_in, int64_t ld_img,
                            const float2* filt, const float2* tw, cudaStream_t st) {
    MixedGeom g{};
    if (!geometry((int)ld_in, g)) return cudaErrorInvalidValue;
    const mixed3_ct_fn f = specialised_ct(g);
    if (!f) return cudaErrorInvalidValue;
    return f(in, img, n_lines, ld_in, ld_img, filt, tw, st);
}

cudaError_t prepare_mixed() {
    cudaError_t e = set_smem_k2(kMixedSmemMax);
    if (e == cudaSuccess) e = set_smem_k3(kMixedSmemMax);
    if (e == cudaSuccess) e = set_smem_k4(kMixedSmemMax);
    if (e == cudaSuccess) e = prepare_specialised();
    if (e == cudaSuccess) e = set_smem_dft(kMixedSmemMax);
    return e;
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
                        &launch_mixed, &launch_mixed_dft, &prepare_mixed, nullptr, 0, nullptr, 0};
    e->desc.mixed = 1;
    if (specialised_ct(g)) {   // the folded range pass: groups of four lines
        e->desc.fused_ct = &launch_mixed_ct;
        e->desc.ct_lines = 4;
    }
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
    mixed_positions_kernel<<<(n + 255) / 256, 256, 0, st>>>(reinterpret_cast<int32_t*>(tw + g.pos_off), g);
    return cudaGetLastError();
}

// The filter's slot order: slot j = r (n / R_L) + q holds position P =
// q R_L + r (the last pass's group q, element r; consecutive groups, one per
// lane, read consecutive slots), and position P = sum_i k_i S_i holds
// frequency k_0 + R_0 (k_1 + R_1 (k_2 + ...)).
void mixed_positions(int n, int32_t* idx) {
    MixedGeom g{};
    if (!geometry(n, g)) return;
    const int RL = g.R[g.P - 1], ngl = n / RL;
    for (int j = 0; j < n; ++j) {
        const int P = (j % ngl) * RL + j / ngl;
        int rem = P, digits[kMaxPasses];
        for (int i = 0; i < g.P; ++i) {
            digits[i] = rem / g.S[i];
            rem %= g.S[i];
        }
        int k = 0;
        for (int i = g.P - 1; i >= 0; --i) k = digits[i] + g.R[i] * k;
        idx[j] = k;
    }
}

}  // namespace sar
