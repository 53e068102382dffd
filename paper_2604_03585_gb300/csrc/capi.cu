// C-ABI of libsar: plan lifecycle, argument validation and the entry points
// declared in include/sar.h.  All compute runs in this library's kernels;
// there is no host or library fallback.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <string>
#include <vector>

#include "../../include/sar.h"
#include "mixed_radix.h"
#include "registry.h"
#include "tables.h"

using sar::SchedDesc;

namespace {

thread_local std::string g_last_error;

sar_status fail(sar_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

sar_status cuda_fail(cudaError_t e, const char *what) {
    return fail(SAR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define SAR_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

sar_status check_length(int64_t n, const char *what) {
    if (n < 1) return fail(SAR_ERR_INVALID_ARG, "%s = %lld must be >= 1", what, (long long)n);
    if (!is_pow2(n) || n < 256 || n > 131072)
        return fail(SAR_ERR_UNSUPPORTED, "%s = %lld: supported lengths are powers of two in [256, 131072]", what,
                    (long long)n);
    return SAR_OK;
}

// A plan's line length: a power of two in [256, 131072] (the line engine at
// that length), or any other length in [2, 8192]: the mixed-radix engine at
// the length itself when its prime factors are 2, 3, 5, 7 (mixed_radix.cu),
// else the zero-padded linear convolution at L = max(256, next power of two
// >= 2n - 1) (wrap_line.cu).
bool native_length(int64_t n) { return is_pow2(n) && n >= 256 && n <= 131072; }

sar_status check_plan_length(int64_t n, const char *what) {
    if (n < 1) return fail(SAR_ERR_INVALID_ARG, "%s = %lld must be >= 1", what, (long long)n);
    if (native_length(n) || (n >= 2 && n <= 8192)) return SAR_OK;
    return fail(SAR_ERR_UNSUPPORTED,
                "%s = %lld: supported lengths are powers of two in [256, 131072] and any length in [2, 8192]", what,
                (long long)n);
}

int64_t wrap_length(int64_t n) {
    int64_t L = 256;
    while (L < 2 * n - 1) L <<= 1;
    return L;
}

// A compute pointer must be non-null, 16-byte aligned and device-accessible
// memory of the current device (a host pointer handed to a kernel would
// fault the GPU, so it is refused here).
sar_status check_device_ptr(const void *p, const char *what) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "%s is NULL", what);
    if (((uintptr_t)p) & 15u) return fail(SAR_ERR_INVALID_ARG, "%s is not 16-byte aligned", what);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SAR_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", what, cudaGetErrorName(e));
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(SAR_ERR_INVALID_ARG, "%s is not device memory", what);
    int dev = -1;
    cudaGetDevice(&dev);
    if (a.device != dev) return fail(SAR_ERR_INVALID_ARG, "%s lives on device %d, current device is %d", what,
                                     a.device, dev);
    return SAR_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct LinePlan {
    const SchedDesc *sched = nullptr;
    int64_t n = 0;           // line length (sched->n unless the length is not a power of two)
    float2 *filt = nullptr;  // sched->n complex, register order, 1/sched->n folded in
    float2 *tw = nullptr;    // twiddle tables
    float2 *filt_nat = nullptr;  // n complex, natural order, 1/N folded in (unfused path)
};

// Per-device cache of twiddle tables for the stand-alone FFT entry points.
struct TwiddleCache {
    std::mutex mu;
    std::vector<std::pair<const SchedDesc *, float2 *>> tables[64];
};
TwiddleCache g_tw;

sar_status cached_twiddles(const SchedDesc *d, float2 **out) {
    int dev = 0;
    SAR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(SAR_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_tw.mu);
    for (auto &pr : g_tw.tables[dev])
        if (pr.first == d) {
            *out = pr.second;
            return SAR_OK;
        }
    float2 *tw = nullptr;
    cudaError_t e = cudaMalloc(&tw, sizeof(float2) * (size_t)d->tw_elems);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SAR_ERR_OUT_OF_MEMORY, "twiddle table allocation failed");
    }
    cudaStream_t s;
    SAR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
    e = sar::build_twiddles(*d, tw, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaFree(tw);
        return cuda_fail(e, "twiddle table");
    }
    SAR_CUDA(d->prepare(), "cudaFuncSetAttribute");
    g_tw.tables[dev].push_back({d, tw});
    *out = tw;
    return SAR_OK;
}

// Per-device cache of the tables of the DFT of lengths that are not powers of
// two (Bluestein): the engine schedule of length L, its twiddles, the filter
// FFT_L(conj chirp) / L in the engine's register order, and the chirp.
struct BluesteinCache {
    struct Entry {
        int n;
        const SchedDesc *d;
        float2 *tw, *filt, *chirp;
    };
    std::mutex mu;
    std::vector<Entry> tables[64];
};
BluesteinCache g_bs;

sar_status cached_bluestein(int n, BluesteinCache::Entry *out) {
    int dev = 0;
    SAR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(SAR_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_bs.mu);
    for (auto &en : g_bs.tables[dev])
        if (en.n == n) {
            *out = en;
            return SAR_OK;
        }
    const SchedDesc *d = sar::wrap_schedule((int)wrap_length(n));
    if (!d) return fail(SAR_ERR_UNSUPPORTED, "no engine for length %d", n);
    const int L = d->n;
    const size_t o_f = align_up(sizeof(float2) * (size_t)d->tw_elems);
    const size_t o_c = o_f + align_up(sizeof(float2) * (size_t)L);
    const size_t total = o_c + align_up(sizeof(float2) * (size_t)n);
    const size_t o_g = align_up(sar::bluestein_scratch_bytes(L));
    const size_t o_i = o_g + align_up(sizeof(float2) * (size_t)L);
    const size_t scratch_bytes = o_i + sizeof(int32_t) * (size_t)L;
    char *block = nullptr, *scratch = nullptr;
    if (cudaMalloc(&block, total) != cudaSuccess || cudaMalloc(&scratch, scratch_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(block);
        return fail(SAR_ERR_OUT_OF_MEMORY, "tables of the length-%d DFT", n);
    }
    BluesteinCache::Entry en{n, d, (float2 *)block, (float2 *)(block + o_f), (float2 *)(block + o_c)};
    std::vector<int32_t> idx((size_t)L);
    sar::filter_slot_to_k(*d, idx.data());
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = sar::build_twiddles(*d, en.tw, s);
    if (e == cudaSuccess) e = sar::build_bluestein_tables(n, L, en.chirp, (float2 *)(scratch + o_g), scratch, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scratch + o_i, idx.data(), sizeof(int32_t) * (size_t)L, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sar::build_filter(*d, (const float2 *)(scratch + o_g), en.filt, (int32_t *)(scratch + o_i), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    cudaFree(scratch);
    if (e != cudaSuccess) {
        cudaFree(block);
        return cuda_fail(e, "tables of a DFT length that is not a power of two");
    }
    g_bs.tables[dev].push_back(en);
    *out = en;
    return SAR_OK;
}

bool fault_inject_alloc() {
    const char *v = getenv("SAR_FAULT_INJECT_ALLOC");
    return v && v[0] == '1';
}

// Bound of every device-side wait of a plan's kernels: about one second at
// the GB300's maximum SM clock, or SAR_WAIT_CYCLES.
long long plan_wait_cycles() {
    const char *v = getenv("SAR_WAIT_CYCLES");
    long long c = v ? atoll(v) : 0;
    return c > 0 ? c : 2000000000LL;
}

// Test hook (host-side fault injection): SAR_FAULT_INJECT_SKIP_LINE=<l> makes
// the persistent kernels of plans created while it is set never start the
// copy of line l, so that line's bounded wait runs out.
int64_t plan_skip_line() {
    const char *v = getenv("SAR_FAULT_INJECT_SKIP_LINE");
    return v ? atoll(v) : -1;
}

}  // namespace

// Internal hooks for other translation units of this library: record an
// error for sar_last_error(), and validate a device pointer the same way the
// entry points above do.
namespace sar {
sar_status report_error(sar_status st, const char *msg) { return fail(st, "%s", msg); }
sar_status validate_device_ptr(const void *p, const char *what) { return check_device_ptr(p, what); }
sar_status validate_length(int64_t n, const char *what) { return check_length(n, what); }
}  // namespace sar

struct sar_plan_s {
    int64_t n_range = 0, n_az = 0;
    int device = 0;
    LinePlan range, az;
    int *status = nullptr;  // device word written by timed-out kernels (0 = fine)
    int prec = SAR_PREC_FP32;
    bool fold = false;      // range pass writes the corner-turned image itself
    bool az_major = false;  // image returned as [n_az][n_range] (a fourth pass)
    sar::FusedCtl ctl{};
    void *block = nullptr;  // one device allocation holding every table
    std::mutex host_mu;
    // lazily, for the host-buffer entry points: two staging sets (the second
    // only for calls of several scenes), each an echo and an image
    void *stage_raw[2] = {}, *stage_img[2] = {};
    // lazily, for the chunked host-buffer pipeline: copy-in, compute and
    // copy-out streams, one event per chunk and direction, start / end events,
    // and per staging set the events that free its echo and its image
    static constexpr int kHostChunks = 8;
    cudaStream_t host_copy = nullptr, host_compute = nullptr, host_copy_out = nullptr;
    cudaEvent_t host_ev[2 * kHostChunks + 2] = {};
    cudaEvent_t host_free[4] = {};
    // full Range-Doppler processing (sar_plan_set_geometry)
    void *rd_cols = nullptr;
    double kappa = 0, vs = 0, r_near = 0;
    int taps = 0;
    int rcmc_rows = 0;   // input rows one RCMC tile stages in shared memory
};

// Engine of the split-precision plans (process-wide): 0 = tcgen05.mma with
// TMEM accumulators and the A operand in TMEM, 1 = warp-level mma.sync,
// 2 = tcgen05.mma with the A operand in shared memory.
static std::atomic<int> g_split_engine{0};

extern "C" {

const char *sar_last_error(void) { return g_last_error.c_str(); }

const char *sar_version(void) { return "sar-gb300 0.1 (sm_103a)"; }

sar_status sar_plan_create(int64_t n_range, int64_t n_az, const sar_filters *filters, sar_plan *out) {
    return sar_plan_create_ex(n_range, n_az, filters, nullptr, nullptr, out);
}

sar_status sar_plan_create_ex(int64_t n_range, int64_t n_az, const sar_filters *filters, const char *range_schedule,
                              const char *az_schedule, sar_plan *out) {
    if (!out) return fail(SAR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!filters) return fail(SAR_ERR_INVALID_ARG, "filters is NULL");
    sar_status st;
    if ((st = check_plan_length(n_range, "n_range")) != SAR_OK) return st;
    if ((st = check_plan_length(n_az, "n_az")) != SAR_OK) return st;
    const bool wrap_r = !native_length(n_range), wrap_a = !native_length(n_az);
    if ((wrap_r && range_schedule) || (wrap_a && az_schedule))
        return fail(SAR_ERR_INVALID_ARG, "schedules can be named only for power-of-two lengths");
    if (filters->flags & ~(SAR_PLAN_UNFOLDED_CORNER_TURN | SAR_PLAN_OUT_AZ_MAJOR))
        return fail(SAR_ERR_INVALID_ARG, "filters->flags has unknown bits 0x%x", filters->flags);
    const int prec = filters->precision;
    if (prec < SAR_PREC_FP32 || prec > SAR_PREC_BF16X3)
        return fail(SAR_ERR_INVALID_ARG, "unknown precision %d", prec);
    if (prec != SAR_PREC_FP32 && (!(n_range == 256 || n_range == 4096) || !(n_az == 256 || n_az == 4096)))
        return fail(SAR_ERR_UNSUPPORTED, "split-precision plans need line lengths 256 or 4096");
    if (prec != SAR_PREC_FP32 && (range_schedule || az_schedule))
        return fail(SAR_ERR_INVALID_ARG, "split-precision plans take no schedule names");
    if ((st = check_device_ptr(filters->range_spectrum, "filters->range_spectrum")) != SAR_OK) return st;
    if ((st = check_device_ptr(filters->az_spectrum, "filters->az_spectrum")) != SAR_OK) return st;

    const bool want_fold = !(filters->flags & SAR_PLAN_UNFOLDED_CORNER_TURN) && prec == SAR_PREC_FP32 &&
                           (!wrap_r || sar::mixed_length((int)n_range));
    const SchedDesc *dr = range_schedule ? sar::find_schedule(range_schedule) : nullptr;
    if (wrap_r) {
        dr = sar::mixed_length((int)n_range) ? sar::mixed_schedule((int)n_range)
                                             : sar::wrap_schedule((int)wrap_length(n_range));
    } else if (!range_schedule) {
        dr = want_fold ? sar::default_ct_schedule((int)n_range) : nullptr;
        if (!dr || n_az % dr->ct_lines) dr = sar::default_schedule((int)n_range);
    }
    const SchedDesc *da = wrap_a ? (sar::mixed_length((int)n_az) ? sar::mixed_schedule((int)n_az)
                                                                  : sar::wrap_schedule((int)wrap_length(n_az)))
                                 : az_schedule ? sar::find_schedule(az_schedule) : sar::default_schedule((int)n_az);
    if (range_schedule && (!dr || dr->n != n_range))
        return fail(SAR_ERR_INVALID_ARG, "range schedule '%s' is unknown or not for n_range", range_schedule);
    if (az_schedule && (!da || da->n != n_az))
        return fail(SAR_ERR_INVALID_ARG, "azimuth schedule '%s' is unknown or not for n_az", az_schedule);
    if (prec != SAR_PREC_FP32) {
        // the tensor-core kernel uses the twiddle tables of the all-radix-16 schedules
        dr = sar::find_schedule(n_range == 4096 ? "n4096_e32_r16x16x16_sr1" : "n256_e16_r16x16_l8");
        da = sar::find_schedule(n_az == 4096 ? "n4096_e32_r16x16x16_sr1" : "n256_e16_r16x16_l8");
    }
    if (!dr || !da) return fail(SAR_ERR_UNSUPPORTED, "no compiled schedule for this size");

    sar_plan p = new (std::nothrow) sar_plan_s;
    if (!p) return fail(SAR_ERR_OUT_OF_MEMORY, "host allocation failed");
    p->n_range = n_range;
    p->n_az = n_az;
    cudaGetDevice(&p->device);
    p->range.sched = dr;
    p->az.sched = da;
    p->range.n = n_range;
    p->az.n = n_az;
    p->prec = prec;
    p->fold = want_fold && dr->fused_ct && n_az % dr->ct_lines == 0;
    p->az_major = (filters->flags & SAR_PLAN_OUT_AZ_MAJOR) != 0;

    // one block: filt_r | tw_r | filt_a | tw_a | idx (int32, max engine length) | status | filt_nat_r | filt_nat_a
    const size_t o_fr = 0;
    const size_t o_tr = o_fr + align_up(sizeof(float2) * (size_t)dr->n);
    const size_t o_fa = o_tr + align_up(sizeof(float2) * (size_t)dr->tw_elems);
    const size_t o_ta = o_fa + align_up(sizeof(float2) * (size_t)da->n);
    const size_t o_ix = o_ta + align_up(sizeof(float2) * (size_t)da->tw_elems);
    const size_t o_st = o_ix + align_up(sizeof(int32_t) * (size_t)(dr->n > da->n ? dr->n : da->n));
    const size_t o_nr = o_st + 256;
    const size_t o_na = o_nr + align_up(sizeof(float2) * (size_t)n_range);
    const size_t total = o_na + align_up(sizeof(float2) * (size_t)n_az);
    cudaError_t e = fault_inject_alloc() ? cudaErrorMemoryAllocation : cudaMalloc(&p->block, total);
    if (e != cudaSuccess) {
        if (e != cudaErrorMemoryAllocation) cudaGetLastError();
        else cudaGetLastError();
        delete p;
        return fail(SAR_ERR_OUT_OF_MEMORY, "plan allocation of %zu bytes failed", total);
    }
    char *b = (char *)p->block;
    p->range.filt = (float2 *)(b + o_fr);
    p->range.tw = (float2 *)(b + o_tr);
    p->az.filt = (float2 *)(b + o_fa);
    p->az.tw = (float2 *)(b + o_ta);
    int32_t *idx_dev = (int32_t *)(b + o_ix);
    p->status = (int *)(b + o_st);
    p->range.filt_nat = (float2 *)(b + o_nr);
    p->az.filt_nat = (float2 *)(b + o_na);
    p->ctl = sar::FusedCtl{p->status, plan_wait_cycles(), plan_skip_line()};

    cudaStream_t s = nullptr;
    std::vector<int32_t> idx;
    void *wrap_tmp = nullptr;   // plan-time scratch of the filters of non-power-of-two lengths
    auto cleanup_fail = [&](cudaError_t err, const char *what) {
        if (s) cudaStreamDestroy(s);
        if (wrap_tmp) cudaFree(wrap_tmp);
        cudaFree(p->block);
        delete p;
        return cuda_fail(err, what);
    };
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
        return cleanup_fail(e, "cudaStreamCreate");
    if ((e = cudaMemsetAsync(p->status, 0, sizeof(int), s)) != cudaSuccess) return cleanup_fail(e, "status word");
    // the caller's spectra were produced on the legacy stream or another one:
    // wait for the device once before reading them
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup_fail(e, "cudaDeviceSynchronize");
    const struct {
        LinePlan *lp;
        const void *H;
    } dims[2] = {{&p->range, filters->range_spectrum}, {&p->az, filters->az_spectrum}};
    for (auto &dm : dims) {
        const SchedDesc &d = *dm.lp->sched;
        const int64_t n = dm.lp->n;
        if ((e = d.prepare()) != cudaSuccess) return cleanup_fail(e, "cudaFuncSetAttribute");
        if ((e = sar::build_twiddles(d, dm.lp->tw, s)) != cudaSuccess) return cleanup_fail(e, "twiddle tables");
        idx.assign(d.n, 0);
        sar::filter_slot_to_k(d, idx.data());
        if ((e = cudaMemcpyAsync(idx_dev, idx.data(), sizeof(int32_t) * d.n, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return cleanup_fail(e, "filter index copy");
        const float2 *spectrum = (const float2 *)dm.H;
        if (n != d.n) {
            // length n that is not a power of two: the engine's filter is
            // G = FFT_L(IFFT_n(H) zero-padded to L), L = d.n
            const size_t scratch = sar::wrap_filter_scratch_bytes((int)n, d.n);
            if ((e = cudaMalloc(&wrap_tmp, scratch + sizeof(float2) * (size_t)d.n)) != cudaSuccess) {
                wrap_tmp = nullptr;
                cudaGetLastError();
                return cleanup_fail(e, "filter design scratch");
            }
            float2 *G = (float2 *)((char *)wrap_tmp + scratch);
            if ((e = sar::build_wrap_filter(spectrum, (int)n, d.n, wrap_tmp, G, s)) != cudaSuccess)
                return cleanup_fail(e, "filter design");
            spectrum = G;
        }
        if ((e = sar::build_filter(d, spectrum, dm.lp->filt, idx_dev, s)) != cudaSuccess)
            return cleanup_fail(e, "filter permutation");
        if (n == d.n && (e = sar::build_natural_filter(spectrum, dm.lp->filt_nat, d.n, s)) != cudaSuccess)
            return cleanup_fail(e, "natural-order filter");
        if (prec != SAR_PREC_FP32) {
            // position-order filter of the tensor-core kernel, in place of the
            // register-order one
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup_fail(e, "plan tables");
            sar::mma_filter_positions(d.n, idx.data());
            if ((e = cudaMemcpyAsync(idx_dev, idx.data(), sizeof(int32_t) * d.n, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess)
                return cleanup_fail(e, "filter index copy");
            if ((e = sar::build_filter(d, (const float2 *)dm.H, dm.lp->filt, idx_dev, s)) != cudaSuccess)
                return cleanup_fail(e, "filter permutation");
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup_fail(e, "plan tables");
        if (wrap_tmp) {
            cudaFree(wrap_tmp);
            wrap_tmp = nullptr;
        }
    }
    cudaStreamDestroy(s);
    *out = p;
    return SAR_OK;
}

static void describe(const SchedDesc &d, sar_schedule_desc *o) {
    memset(o, 0, sizeof(*o));
    strncpy(o->name, d.name, sizeof(o->name) - 1);
    o->n = d.n;
    o->e = d.e;
    o->r1 = d.r1;
    o->r2 = d.r2;
    o->r3 = d.r3;
    o->lines_per_block = d.lpb;
    o->threads_per_block = d.threads;
    o->smem_bytes = d.smem_bytes;
    o->cluster_blocks = d.cluster > 1 ? d.cluster : 1;
}

int32_t sar_schedule_count(void) { return sar::schedule_count(); }

sar_status sar_schedule_get(int32_t index, sar_schedule_desc *out) {
    const SchedDesc *d = sar::schedule_at(index);
    if (!d || !out) return fail(SAR_ERR_INVALID_ARG, "schedule index %d out of range or out is NULL", index);
    describe(*d, out);
    return SAR_OK;
}

sar_status sar_set_preferred_schedule(const char *name) {
    const SchedDesc *d = name ? sar::find_schedule(name) : nullptr;
    if (!d) return fail(SAR_ERR_INVALID_ARG, "unknown schedule '%s'", name ? name : "(null)");
    sar::set_preferred_schedule(d);
    return SAR_OK;
}

sar_status sar_set_corner_turn_variant(int32_t v) {
    if (v < 0 || v > 2) return fail(SAR_ERR_INVALID_ARG, "corner-turn variant %d is not 0, 1 or 2", v);
    sar::set_corner_turn_variant(v);
    return SAR_OK;
}

int32_t sar_plan_folds_corner_turn(sar_plan p) { return p && p->fold ? 1 : 0; }

sar_status sar_set_split_engine(int32_t engine) {
    if (engine < 0 || engine > 2) return fail(SAR_ERR_INVALID_ARG, "split engine must be 0, 1 or 2, not %d", engine);
    g_split_engine.store(engine);
    return SAR_OK;
}

sar_status sar_plan_get_schedules(sar_plan p, sar_schedule_desc *range, sar_schedule_desc *az) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (range) describe(*p->range.sched, range);
    if (az) describe(*p->az.sched, az);
    return SAR_OK;
}

sar_status sar_autotune(int64_t n, int64_t n_lines, int32_t reps, int32_t kind, sar_stream stream,
                        sar_schedule_desc *best, float *best_ms, float *all_ms, int32_t all_cap) {
    sar_status st;
    if ((st = check_length(n, "n")) != SAR_OK) return st;
    if (n_lines < 1 || reps < 1) return fail(SAR_ERR_INVALID_ARG, "n_lines and reps must be >= 1");
    if (kind != SAR_TUNE_FUSED && kind != SAR_TUNE_RANGE_CT) return fail(SAR_ERR_INVALID_ARG, "unknown kind %d", kind);
    if (kind == SAR_TUNE_RANGE_CT && n_lines % 4)
        return fail(SAR_ERR_INVALID_ARG, "folded range pass needs n_lines a multiple of 4");
    const size_t bytes = sizeof(float2) * (size_t)n * (size_t)n_lines;
    int cands = 0;
    for (int i = 0; i < sar::schedule_count(); ++i) cands += sar::schedule_at(i)->n == n;
    if (cands == 0) return fail(SAR_ERR_UNSUPPORTED, "no compiled schedule for n = %lld", (long long)n);
    float2 *in = nullptr, *outb = nullptr, *tab = nullptr;
    int max_tw = 0;
    for (int i = 0; i < sar::schedule_count(); ++i)
        if (sar::schedule_at(i)->n == n && sar::schedule_at(i)->tw_elems > max_tw) max_tw = sar::schedule_at(i)->tw_elems;
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&outb, bytes) != cudaSuccess ||
        cudaMalloc(&tab, sizeof(float2) * (size_t)(max_tw + n + 32)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(in);
        cudaFree(outb);
        cudaFree(tab);
        return fail(SAR_ERR_OUT_OF_MEMORY, "autotune buffers (2 x %zu bytes)", bytes);
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const SchedDesc *win = nullptr;
    float win_ms = 0.f;
    cudaError_t e = cudaMemsetAsync(in, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tab, 0, sizeof(float2) * (size_t)(max_tw + n + 32), s);
    const sar::FusedCtl ctl{(int *)(tab + max_tw + n), plan_wait_cycles(), -1};
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<float> times;
    int cand = 0;
    for (int i = 0; i < sar::schedule_count() && e == cudaSuccess; ++i) {
        const SchedDesc &d = *sar::schedule_at(i);
        if (d.n != n) continue;
        const bool ct = kind == SAR_TUNE_RANGE_CT;
        if (ct && !d.fused_ct) {
            if (all_ms && cand < all_cap) all_ms[cand] = 0.f;
            ++cand;
            continue;
        }
        if ((e = d.prepare()) != cudaSuccess) break;
        float2 *tw = tab + n, *filt = tab;
        if ((e = sar::build_twiddles(d, tw, s)) != cudaSuccess) break;
        auto run = [&]() {
            return ct ? d.fused_ct(in, outb, n_lines, n, n_lines, filt, tw, s)
                      : d.fused(in, outb, n_lines, n, (int)n, filt, tw, ctl, s);
        };
        // warm-up, then reps timed launches
        if ((e = run()) != cudaSuccess) break;
        times.clear();
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, s);
            e = run();
            cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            times.push_back(ms);
        }
        if (e != cudaSuccess) break;
        std::sort(times.begin(), times.end());
        const float med = times[times.size() / 2];
        if (all_ms && cand < all_cap) all_ms[cand] = med;
        ++cand;
        if (!win || med < win_ms) {
            win = &d;
            win_ms = med;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(in);
    cudaFree(outb);
    cudaFree(tab);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (!win) return fail(SAR_ERR_UNSUPPORTED, "no schedule of n = %lld has that kind of kernel", (long long)n);
    if (kind == SAR_TUNE_RANGE_CT)
        sar::set_preferred_ct_schedule(win);
    else
        sar::set_preferred_schedule(win);
    if (best) describe(*win, best);
    if (best_ms) *best_ms = win_ms;
    return SAR_OK;
}

sar_status sar_plan_destroy(sar_plan p) {
    if (!p) return SAR_OK;
    cudaFree(p->block);
    for (int b = 0; b < 2; ++b) {
        if (p->stage_raw[b]) cudaFree(p->stage_raw[b]);
        if (p->stage_img[b]) cudaFree(p->stage_img[b]);
    }
    if (p->rd_cols) cudaFree(p->rd_cols);
    if (p->host_copy) cudaStreamDestroy(p->host_copy);
    if (p->host_compute) cudaStreamDestroy(p->host_compute);
    if (p->host_copy_out) cudaStreamDestroy(p->host_copy_out);
    for (cudaEvent_t e : p->host_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : p->host_free)
        if (e) cudaEventDestroy(e);
    delete p;
    return SAR_OK;
}

static sar_status run_fused(const sar_plan_s *p, const LinePlan &lp, int64_t n_lines, const void *in, void *out,
                            cudaStream_t s, const char *what) {
    const SchedDesc &d = *lp.sched;
    if (p->prec != SAR_PREC_FP32) {
        cudaError_t e =
            g_split_engine.load() == 1
                ? sar::launch_mma_compress(d.n, p->prec, (const float2 *)in, (float2 *)out, n_lines, d.n, lp.filt,
                                           lp.tw, s)
                : sar::launch_mma_tc_compress(d.n, p->prec, g_split_engine.load() == 0, (const float2 *)in,
                                              (float2 *)out, n_lines, d.n, lp.filt, lp.tw, p->ctl.status,
                                              p->ctl.wait_cycles, s);
        if (e != cudaSuccess) return cuda_fail(e, what);
        return SAR_OK;
    }
    cudaError_t e = d.fused((const float2 *)in, (float2 *)out, n_lines, lp.n, (int)lp.n, lp.filt, lp.tw, p->ctl, s);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return SAR_OK;
}

sar_status sar_range_compress(sar_plan p, void *data, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st = check_device_ptr(data, "data");
    if (st != SAR_OK) return st;
    return run_fused(p, p->range, p->n_az, data, data, (cudaStream_t)stream, "range compression launch");
}

sar_status sar_azimuth_compress(sar_plan p, void *data, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st = check_device_ptr(data, "data");
    if (st != SAR_OK) return st;
    return run_fused(p, p->az, p->n_range, data, data, (cudaStream_t)stream, "azimuth compression launch");
}

// Range compression straight into the corner-turned image, then the
// azimuth pass in place: two kernels.
static sar_status run_folded(const sar_plan_s *p, const void *raw, void *image, cudaStream_t s) {
    const SchedDesc &d = *p->range.sched;
    cudaError_t e = d.fused_ct((const float2 *)raw, (float2 *)image, p->n_az, p->n_range, p->n_az, p->range.filt,
                               p->range.tw, s);
    if (e != cudaSuccess) return cuda_fail(e, "range compression + corner turn launch");
    return run_fused(p, p->az, p->n_range, image, image, s, "azimuth compression launch");
}

static bool overlaps(const void *a, const void *b, size_t bytes) {
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + bytes && y < x + bytes;
}

sar_status sar_corner_turn(sar_plan p, const void *in, void *out, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st;
    if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
    if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
    if (overlaps(in, out, sizeof(float2) * (size_t)(p->n_az * p->n_range)))
        return fail(SAR_ERR_INVALID_ARG, "in and out overlap");
    cudaError_t e = sar::launch_transpose((const float2 *)in, (float2 *)out, p->n_az, p->n_range, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
    return SAR_OK;
}

// The three passes into image [n_range][n_az] (raw clobbered when unfolded).
static sar_status rda3(sar_plan p, void *raw, void *image, cudaStream_t s) {
    sar_status st;
    if (p->fold) return run_folded(p, raw, image, s);
    if ((st = run_fused(p, p->range, p->n_az, raw, raw, s, "range compression launch")) != SAR_OK) return st;
    cudaError_t e = sar::launch_transpose((const float2 *)raw, (float2 *)image, p->n_az, p->n_range, s);
    if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
    return run_fused(p, p->az, p->n_range, image, image, s, "azimuth compression launch");
}

sar_status sar_rda_process(sar_plan p, void *raw, void *image, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st;
    if ((st = check_device_ptr(raw, "raw")) != SAR_OK) return st;
    if ((st = check_device_ptr(image, "image")) != SAR_OK) return st;
    if (overlaps(raw, image, sizeof(float2) * (size_t)(p->n_az * p->n_range)))
        return fail(SAR_ERR_INVALID_ARG, "raw and image overlap");
    if (p->az_major)
        return fail(SAR_ERR_INVALID_ARG, "azimuth-major output needs a work buffer: use sar_rda_process_oop");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->fold) return run_folded(p, raw, image, s);
    if ((st = run_fused(p, p->range, p->n_az, raw, raw, s, "range compression launch")) != SAR_OK) return st;
    cudaError_t e = sar::launch_transpose((const float2 *)raw, (float2 *)image, p->n_az, p->n_range, s);
    if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
    return run_fused(p, p->az, p->n_range, image, image, s, "azimuth compression launch");
}

sar_status sar_range_compress_oop(sar_plan p, const void *in, void *out, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st;
    if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
    if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
    if (in != out && overlaps(in, out, sizeof(float2) * (size_t)(p->n_az * p->n_range)))
        return fail(SAR_ERR_INVALID_ARG, "in and out partially overlap");
    return run_fused(p, p->range, p->n_az, in, out, (cudaStream_t)stream, "range compression launch");
}

sar_status sar_range_compress_ct(sar_plan p, const void *raw, void *image, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (!p->fold) return fail(SAR_ERR_UNSUPPORTED, "this plan does not fold the corner turn into the range pass");
    sar_status st;
    if ((st = check_device_ptr(raw, "raw")) != SAR_OK) return st;
    if ((st = check_device_ptr(image, "image")) != SAR_OK) return st;
    if (overlaps(raw, image, sizeof(float2) * (size_t)(p->n_az * p->n_range)))
        return fail(SAR_ERR_INVALID_ARG, "raw and image overlap");
    const SchedDesc &d = *p->range.sched;
    cudaError_t e = d.fused_ct((const float2 *)raw, (float2 *)image, p->n_az, p->n_range, p->n_az, p->range.filt,
                               p->range.tw, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "range compression + corner turn launch");
    return SAR_OK;
}

// Range compression and corner turn raw -> image (work as scratch when the
// corner turn is not folded).
static sar_status sar_rda_process_oop_range(sar_plan p, const void *raw, void *work, void *image, cudaStream_t s) {
    if (p->fold) {
        const SchedDesc &d = *p->range.sched;
        cudaError_t e = d.fused_ct((const float2 *)raw, (float2 *)image, p->n_az, p->n_range, p->n_az, p->range.filt,
                                   p->range.tw, s);
        if (e != cudaSuccess) return cuda_fail(e, "range compression + corner turn launch");
        return SAR_OK;
    }
    sar_status st = run_fused(p, p->range, p->n_az, raw, work, s, "range compression launch");
    if (st != SAR_OK) return st;
    cudaError_t e = sar::launch_transpose((const float2 *)work, (float2 *)image, p->n_az, p->n_range, s);
    if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
    return SAR_OK;
}

sar_status sar_rda_process_oop(sar_plan p, const void *raw, void *work, void *image, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st;
    if ((st = check_device_ptr(raw, "raw")) != SAR_OK) return st;
    if ((st = check_device_ptr(work, "work")) != SAR_OK) return st;
    if ((st = check_device_ptr(image, "image")) != SAR_OK) return st;
    const size_t bytes = sizeof(float2) * (size_t)(p->n_az * p->n_range);
    if (overlaps(raw, work, bytes) || overlaps(raw, image, bytes) || overlaps(work, image, bytes))
        return fail(SAR_ERR_INVALID_ARG, "raw, work and image must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->az_major) {
        // the three passes leave the [n_range][n_az] image in work (image as
        // scratch when unfolded), then the fourth pass transposes it back
        if (p->fold) {
            if ((st = run_folded(p, raw, work, s)) != SAR_OK) return st;
        } else {
            if ((st = run_fused(p, p->range, p->n_az, raw, image, s, "range compression launch")) != SAR_OK)
                return st;
            cudaError_t e = sar::launch_transpose((const float2 *)image, (float2 *)work, p->n_az, p->n_range, s);
            if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
            if ((st = run_fused(p, p->az, p->n_range, work, work, s, "azimuth compression launch")) != SAR_OK)
                return st;
        }
        cudaError_t e = sar::launch_transpose((const float2 *)work, (float2 *)image, p->n_range, p->n_az, s);
        if (e != cudaSuccess) return cuda_fail(e, "transpose back launch");
        return SAR_OK;
    }
    if (p->fold) return run_folded(p, raw, image, s);
    if ((st = run_fused(p, p->range, p->n_az, raw, work, s, "range compression launch")) != SAR_OK) return st;
    cudaError_t e = sar::launch_transpose((const float2 *)work, (float2 *)image, p->n_az, p->n_range, s);
    if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
    return run_fused(p, p->az, p->n_range, image, image, s, "azimuth compression launch");
}

// The unfused comparison path (Sec. II-B, the pipeline the fused kernel
// replaces): forward FFT kernel, spectrum multiply kernel, inverse FFT
// kernel, each reading and writing the whole line set (six transfers per
// line instead of two).
static bool unfused_ok(const LinePlan &lp) { return lp.n == lp.sched->n && lp.sched->dft; }
static sar_status unfused_refusal() {
    return fail(SAR_ERR_UNSUPPORTED,
                "the unfused pipeline needs line lengths with their own engine (powers of two, prime factors 2, 3, 5, 7)");
}

static sar_status run_unfused(const sar_plan_s *p, const LinePlan &lp, int64_t n_lines, void *data, cudaStream_t s) {
    const SchedDesc &d = *lp.sched;
    if (!unfused_ok(lp)) return unfused_refusal();
    float2 *tw = nullptr;
    sar_status st = cached_twiddles(&d, &tw);
    if (st != SAR_OK) return st;
    cudaError_t e = d.dft((const float2 *)data, (float2 *)data, n_lines, d.n, d.n, tw, 0, s);
    if (e == cudaSuccess) e = sar::spectrum_multiply((float2 *)data, lp.filt_nat, n_lines, d.n, s);
    if (e == cudaSuccess) e = d.dft((const float2 *)data, (float2 *)data, n_lines, d.n, d.n, tw, 1, s);
    if (e != cudaSuccess) return cuda_fail(e, "unfused pass launch");
    (void)p;
    return SAR_OK;
}

sar_status sar_range_compress_unfused(sar_plan p, void *data, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st = check_device_ptr(data, "data");
    if (st != SAR_OK) return st;
    return run_unfused(p, p->range, p->n_az, data, (cudaStream_t)stream);
}

sar_status sar_azimuth_compress_unfused(sar_plan p, void *data, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st = check_device_ptr(data, "data");
    if (st != SAR_OK) return st;
    return run_unfused(p, p->az, p->n_range, data, (cudaStream_t)stream);
}

sar_status sar_rda_process_unfused(sar_plan p, void *raw, void *image, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    sar_status st;
    if ((st = check_device_ptr(raw, "raw")) != SAR_OK) return st;
    if ((st = check_device_ptr(image, "image")) != SAR_OK) return st;
    if (overlaps(raw, image, sizeof(float2) * (size_t)(p->n_az * p->n_range)))
        return fail(SAR_ERR_INVALID_ARG, "raw and image overlap");
    if (!unfused_ok(p->range) || !unfused_ok(p->az)) return unfused_refusal();
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = run_unfused(p, p->range, p->n_az, raw, s)) != SAR_OK) return st;
    cudaError_t e = sar::launch_transpose((const float2 *)raw, (float2 *)image, p->n_az, p->n_range, s);
    if (e != cudaSuccess) return cuda_fail(e, "corner turn launch");
    return run_unfused(p, p->az, p->n_range, image, s);
}

sar_status sar_plan_set_geometry(sar_plan p, double kappa, double v_s, double r_near, int32_t rcmc_taps) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (!(kappa > 0) || !(v_s > 0) || !(r_near >= 0))
        return fail(SAR_ERR_INVALID_ARG, "kappa, v_s must be > 0 and r_near >= 0");
    if (kappa * v_s <= 0.5)
        return fail(SAR_ERR_INVALID_ARG, "kappa * v_s must exceed 0.5 (every azimuth frequency must migrate)");
    if (rcmc_taps != 0 && rcmc_taps != 16) return fail(SAR_ERR_UNSUPPORTED, "rcmc_taps must be 0 or 16");
    if (p->prec != SAR_PREC_FP32) return fail(SAR_ERR_UNSUPPORTED, "full processing runs in FP32 only");
    std::vector<unsigned char> host(sar::rd_column_bytes() * (size_t)p->n_az);
    sar::rd_columns((int)p->n_az, kappa, v_s, host.data());
    if (!p->rd_cols) {
        if (cudaMalloc(&p->rd_cols, host.size()) != cudaSuccess) {
            cudaGetLastError();
            p->rd_cols = nullptr;
            return fail(SAR_ERR_OUT_OF_MEMORY, "geometry table");
        }
    }
    SAR_CUDA(cudaMemcpy(p->rd_cols, host.data(), host.size(), cudaMemcpyHostToDevice), "geometry table copy");
    p->kappa = kappa;
    p->vs = v_s;
    p->r_near = r_near;
    p->taps = rcmc_taps;
    p->rcmc_rows = sar::rcmc_staged_rows((int)p->n_range, (int)p->n_az, r_near, host.data());
    return SAR_OK;
}

sar_status sar_rcmc(sar_plan p, const void *in, void *out, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (!p->rd_cols || p->taps != 16)
        return fail(SAR_ERR_INVALID_ARG, "the plan has no geometry with 16 RCMC taps (sar_plan_set_geometry)");
    sar_status st;
    if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
    if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
    const size_t bytes = sizeof(float2) * (size_t)(p->n_az * p->n_range);
    if (overlaps(in, out, bytes)) return fail(SAR_ERR_INVALID_ARG, "in and out must not overlap");
    cudaError_t e = sar::launch_rcmc(16, (const float2 *)in, (float2 *)out, (int)p->n_range, (int)p->n_az,
                                     p->rd_cols, p->r_near, p->rcmc_rows, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "RCMC launch");
    return SAR_OK;
}

sar_status sar_rda_full(sar_plan p, const void *raw, void *work, void *image, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (p->az_major) return fail(SAR_ERR_INVALID_ARG, "the full processor writes [n_range][n_az] images only");
    if (!p->rd_cols) return fail(SAR_ERR_INVALID_ARG, "the plan has no geometry (sar_plan_set_geometry)");
    sar_status st;
    if ((st = check_device_ptr(raw, "raw")) != SAR_OK) return st;
    if ((st = check_device_ptr(work, "work")) != SAR_OK) return st;
    if ((st = check_device_ptr(image, "image")) != SAR_OK) return st;
    const size_t bytes = sizeof(float2) * (size_t)(p->n_az * p->n_range);
    if (overlaps(raw, work, bytes) || overlaps(raw, image, bytes) || overlaps(work, image, bytes))
        return fail(SAR_ERR_INVALID_ARG, "raw, work and image must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    const char *az_name = sar::rd_az_schedule((int)p->n_az);
    const SchedDesc *dz = az_name ? sar::find_schedule(az_name) : nullptr;
    if (!dz) return fail(SAR_ERR_UNSUPPORTED, "full processing needs n_az <= 16384");
    float2 *tw_az = nullptr;
    if ((st = cached_twiddles(dz, &tw_az)) != SAR_OK) return st;
    // 1. range compression and corner turn: raw -> image [n_range][n_az]
    if ((st = sar_rda_process_oop_range(p, raw, work, image, s)) != SAR_OK) return st;
    // 2. azimuth FFT of every range bin, in place
    cudaError_t e = sar::launch_az_fft_rd((int)p->n_az, (const float2 *)image, (float2 *)image, p->n_range, tw_az, s);
    if (e != cudaSuccess) return cuda_fail(e, "azimuth FFT launch");
    // 3. RCMC image -> work (or no correction: work <- image)
    if (p->taps)
        e = sar::launch_rcmc(p->taps, (const float2 *)image, (float2 *)work, (int)p->n_range, (int)p->n_az, p->rd_cols,
                             p->r_near, p->rcmc_rows, s);
    else
        e = cudaMemcpyAsync(work, image, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "RCMC launch");
    // 4. azimuth compression with the range-dependent filter and IFFT: work -> image
    e = sar::launch_az_compress_rd((int)p->n_az, (const float2 *)work, (float2 *)image, p->n_range, tw_az, p->rd_cols,
                                   p->r_near, s);
    if (e != cudaSuccess) return cuda_fail(e, "azimuth compression launch");
    return SAR_OK;
}

// The host-buffer path of a folded plan as a pipeline over n scenes: each
// echo arrives in kHostChunks blocks of azimuth lines on the copy-in stream,
// and each block's range pass (with the folded corner turn, into its columns
// of the image) starts on the compute stream as soon as the block has landed;
// the azimuth pass then runs over kHostChunks blocks of range bins, each
// copied back on the copy-out stream while the next is computed.  Scene q
// uses staging set q mod 2, so the echo of scene q + 1 travels to the device
// while the image of scene q travels back: the link carries both directions
// at once, and the compute hides behind the copies.  A set is reused once its
// previous scene's range pass has read the echo and its image has been copied
// out.  Called with p->host_mu held and the staging sets allocated; on an
// error it returns once the internal streams are idle (no copy is left in
// flight from or to the caller's host buffers).
static sar_status host_pipeline_issue(sar_plan p, int n, const void *const *raws, void *const *images,
                                      cudaStream_t s);
static sar_status host_pipeline(sar_plan p, int n, const void *const *raws, void *const *images, cudaStream_t s) {
    const sar_status st = host_pipeline_issue(p, n, raws, images, s);
    if (st != SAR_OK)
        for (cudaStream_t q : {p->host_copy, p->host_compute, p->host_copy_out})
            if (q) cudaStreamSynchronize(q);
    return st;
}

static sar_status host_pipeline_issue(sar_plan p, int n, const void *const *raws, void *const *images,
                                      cudaStream_t s) {
    constexpr int K = sar_plan_s::kHostChunks;
    const SchedDesc &dr = *p->range.sched;
    const int64_t A = p->n_az / K, B = p->n_range / K;
    if (!p->host_copy) {
        SAR_CUDA(cudaStreamCreateWithFlags(&p->host_copy, cudaStreamNonBlocking), "cudaStreamCreate");
        SAR_CUDA(cudaStreamCreateWithFlags(&p->host_compute, cudaStreamNonBlocking), "cudaStreamCreate");
        SAR_CUDA(cudaStreamCreateWithFlags(&p->host_copy_out, cudaStreamNonBlocking), "cudaStreamCreate");
        for (cudaEvent_t &e : p->host_ev) SAR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        for (cudaEvent_t &e : p->host_free)
            SAR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    }
    cudaStream_t si = p->host_copy, sk = p->host_compute, so = p->host_copy_out;
    cudaEvent_t *ev_in = p->host_ev, *ev_out = p->host_ev + K, ev_start = p->host_ev[2 * K],
                ev_end = p->host_ev[2 * K + 1];
    cudaEvent_t *raw_free = p->host_free, *img_free = p->host_free + 2;
    const size_t row_r = sizeof(float2) * (size_t)p->n_range, row_a = sizeof(float2) * (size_t)p->n_az;
    SAR_CUDA(cudaEventRecord(ev_start, s), "cudaEventRecord");
    SAR_CUDA(cudaStreamWaitEvent(si, ev_start, 0), "cudaStreamWaitEvent");
    SAR_CUDA(cudaStreamWaitEvent(sk, ev_start, 0), "cudaStreamWaitEvent");
    SAR_CUDA(cudaStreamWaitEvent(so, ev_start, 0), "cudaStreamWaitEvent");
    for (int q = 0; q < n; ++q) {
        const int b = q & 1;
        float2 *sraw = (float2 *)p->stage_raw[b], *simg = (float2 *)p->stage_img[b];
        if (q >= 2) {
            SAR_CUDA(cudaStreamWaitEvent(si, raw_free[b], 0), "cudaStreamWaitEvent");
            SAR_CUDA(cudaStreamWaitEvent(sk, img_free[b], 0), "cudaStreamWaitEvent");
        }
        for (int k = 0; k < K; ++k) {
            SAR_CUDA(cudaMemcpyAsync(sraw + k * A * p->n_range, (const char *)raws[q] + k * A * row_r, A * row_r,
                                     cudaMemcpyHostToDevice, si),
                     "host-to-device copy");
            SAR_CUDA(cudaEventRecord(ev_in[k], si), "cudaEventRecord");
            SAR_CUDA(cudaStreamWaitEvent(sk, ev_in[k], 0), "cudaStreamWaitEvent");
            cudaError_t e = dr.fused_ct(sraw + k * A * p->n_range, simg + k * A, A, p->n_range, p->n_az,
                                        p->range.filt, p->range.tw, sk);
            if (e != cudaSuccess) return cuda_fail(e, "range compression + corner turn launch");
        }
        SAR_CUDA(cudaEventRecord(raw_free[b], sk), "cudaEventRecord");
        for (int j = 0; j < K; ++j) {
            float2 *rows = simg + j * B * p->n_az;
            sar_status st = run_fused(p, p->az, B, rows, rows, sk, "azimuth compression launch");
            if (st != SAR_OK) return st;
            SAR_CUDA(cudaEventRecord(ev_out[j], sk), "cudaEventRecord");
            SAR_CUDA(cudaStreamWaitEvent(so, ev_out[j], 0), "cudaStreamWaitEvent");
            SAR_CUDA(cudaMemcpyAsync((char *)images[q] + j * B * row_a, rows, B * row_a, cudaMemcpyDeviceToHost, so),
                     "device-to-host copy");
        }
        SAR_CUDA(cudaEventRecord(img_free[b], so), "cudaEventRecord");
    }
    SAR_CUDA(cudaEventRecord(ev_end, so), "cudaEventRecord");
    SAR_CUDA(cudaStreamWaitEvent(s, ev_end, 0), "cudaStreamWaitEvent");
    // the copy-in and compute streams finish before copy-out's last copy;
    // nothing of this call is left on them
    SAR_CUDA(cudaStreamSynchronize(s), "stream synchronise");
    return SAR_OK;
}

// Allocates staging sets 0 ... sets - 1 (each an echo and an image).
static sar_status host_staging(sar_plan p, int sets) {
    const size_t bytes = sizeof(float2) * (size_t)(p->n_az * p->n_range);
    for (int b = 0; b < sets; ++b) {
        if (p->stage_raw[b]) continue;
        void *r = nullptr, *m = nullptr;
        if (cudaMalloc(&r, bytes) != cudaSuccess || cudaMalloc(&m, bytes) != cudaSuccess) {
            cudaGetLastError();
            if (r) cudaFree(r);
            return fail(SAR_ERR_OUT_OF_MEMORY, "staging buffers (2 x %zu bytes)", bytes);
        }
        p->stage_raw[b] = r;
        p->stage_img[b] = m;
    }
    return SAR_OK;
}

// One scene through staging set 0 without the pipeline (plans that do not
// fold the corner turn, azimuth-major output, or block sizes that do not divide).
static sar_status host_serial(sar_plan p, const void *raw, void *image, cudaStream_t s) {
    const size_t bytes = sizeof(float2) * (size_t)(p->n_az * p->n_range);
    SAR_CUDA(cudaMemcpyAsync(p->stage_raw[0], raw, bytes, cudaMemcpyHostToDevice, s), "host-to-device copy");
    sar_status st = rda3(p, p->stage_raw[0], p->stage_img[0], s);
    if (st != SAR_OK) return st;
    const void *result = p->stage_img[0];
    if (p->az_major) {   // the fourth pass, into the staged raw echo (no longer needed)
        cudaError_t e = sar::launch_transpose((const float2 *)p->stage_img[0], (float2 *)p->stage_raw[0], p->n_range,
                                              p->n_az, s);
        if (e != cudaSuccess) return cuda_fail(e, "transpose back launch");
        result = p->stage_raw[0];
    }
    SAR_CUDA(cudaMemcpyAsync(image, result, bytes, cudaMemcpyDeviceToHost, s), "device-to-host copy");
    SAR_CUDA(cudaStreamSynchronize(s), "stream synchronise");
    return SAR_OK;
}

static bool host_pipelined(const sar_plan_s *p) {
    constexpr int K = sar_plan_s::kHostChunks;
    return p->fold && !p->az_major && p->n_az % (K * p->range.sched->ct_lines) == 0 && p->n_range % K == 0;
}

sar_status sar_rda_process_host(sar_plan p, const void *raw, void *image, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (!raw || !image) return fail(SAR_ERR_INVALID_ARG, "raw or image is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(p->host_mu);   // one host-buffer call per plan at a time
    sar_status st;
    if ((st = host_staging(p, 1)) != SAR_OK) return st;
    if (host_pipelined(p)) return host_pipeline(p, 1, &raw, &image, s);
    return host_serial(p, raw, image, s);
}

sar_status sar_rda_process_host_n(sar_plan p, int32_t n_scenes, const void *const *raws, void *const *images,
                                  sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    if (n_scenes < 0) return fail(SAR_ERR_INVALID_ARG, "n_scenes < 0");
    if (n_scenes == 0) return SAR_OK;
    if (!raws || !images) return fail(SAR_ERR_INVALID_ARG, "raws or images is NULL");
    for (int32_t q = 0; q < n_scenes; ++q)
        if (!raws[q] || !images[q]) return fail(SAR_ERR_INVALID_ARG, "raws[%d] or images[%d] is NULL", q, q);
    // an image copied out while a later echo is copied in must not share its memory
    const size_t bytes = sizeof(float2) * (size_t)(p->n_az * p->n_range);
    for (int32_t a = 0; a < n_scenes; ++a)
        for (int32_t b = 0; b < n_scenes; ++b)
            if (overlaps(images[a], raws[b], bytes))
                return fail(SAR_ERR_INVALID_ARG, "images[%d] overlaps raws[%d]", a, b);
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(p->host_mu);
    sar_status st;
    if (!host_pipelined(p)) {
        if ((st = host_staging(p, 1)) != SAR_OK) return st;
        for (int32_t q = 0; q < n_scenes; ++q)
            if ((st = host_serial(p, raws[q], images[q], s)) != SAR_OK) return st;
        return SAR_OK;
    }
    if ((st = host_staging(p, n_scenes > 1 ? 2 : 1)) != SAR_OK) return st;
    return host_pipeline(p, n_scenes, raws, images, s);
}

sar_status sar_fft_lines(int64_t n, int64_t n_lines, const void *in, void *out, int inverse, sar_stream stream) {
    sar_status st;
    if (!native_length(n) && sar::mixed_length((int)n)) {
        // prime factors 2, 3, 5, 7 only: the mixed-radix engine at n itself
        if (n_lines < 0) return fail(SAR_ERR_INVALID_ARG, "n_lines < 0");
        if (n_lines == 0) return SAR_OK;
        if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
        if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
        if (in != out && overlaps(in, out, sizeof(float2) * (size_t)(n * n_lines)))
            return fail(SAR_ERR_INVALID_ARG, "in and out partially overlap");
        const SchedDesc *d = sar::mixed_schedule((int)n);
        float2 *tw = nullptr;
        if ((st = cached_twiddles(d, &tw)) != SAR_OK) return st;
        cudaError_t e = d->dft((const float2 *)in, (float2 *)out, n_lines, n, (int)n, tw, inverse ? 1 : 0,
                               (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "fft launch");
        return SAR_OK;
    }
    if (!native_length(n) && n >= 2 && n <= 8192) {
        // any other length that is not a power of two: Bluestein on the length-L engine
        if (n_lines < 0) return fail(SAR_ERR_INVALID_ARG, "n_lines < 0");
        if (n_lines == 0) return SAR_OK;
        if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
        if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
        if (in != out && overlaps(in, out, sizeof(float2) * (size_t)(n * n_lines)))
            return fail(SAR_ERR_INVALID_ARG, "in and out partially overlap");
        BluesteinCache::Entry en;
        if ((st = cached_bluestein((int)n, &en)) != SAR_OK) return st;
        cudaError_t e = sar::launch_bluestein(*en.d, (const float2 *)in, (float2 *)out, n_lines, n, (int)n, en.filt,
                                              en.tw, en.chirp, inverse ? 1 : 0, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "fft launch");
        return SAR_OK;
    }
    if ((st = check_length(n, "n")) != SAR_OK) return st;
    if (n_lines < 0) return fail(SAR_ERR_INVALID_ARG, "n_lines < 0");
    if (n_lines == 0) return SAR_OK;
    if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
    if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
    const SchedDesc *d = sar::default_schedule((int)n);
    float2 *tw = nullptr;
    if ((st = cached_twiddles(d, &tw)) != SAR_OK) return st;
    // lines are independent, each thread group reads its whole line before
    // writing it: in == out is safe; partial overlap between lines is not
    if (in != out && overlaps(in, out, sizeof(float2) * (size_t)(n * n_lines)))
        return fail(SAR_ERR_INVALID_ARG, "in and out partially overlap");
    cudaError_t e = d->dft((const float2 *)in, (float2 *)out, n_lines, n, (int)n, tw, inverse ? 1 : 0,
                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fft launch");
    return SAR_OK;
}

sar_status sar_make_lfm_spectrum(int64_t n, int64_t n_chirp, double tbp, void *out, sar_stream stream) {
    sar_status st;
    if ((st = check_plan_length(n, "n")) != SAR_OK) return st;
    if (n_chirp < 1 || n_chirp > n) return fail(SAR_ERR_INVALID_ARG, "n_chirp must be in [1, n]");
    if (!(tbp > 0.0)) return fail(SAR_ERR_INVALID_ARG, "tbp must be > 0");
    if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = sar::make_lfm_line((int)n, (int)n_chirp, tbp, (float2 *)out, s);
    if (e != cudaSuccess) return cuda_fail(e, "chirp launch");
    if ((st = sar_fft_lines(n, 1, out, out, 0, stream)) != SAR_OK) return st;
    e = sar::conjugate((float2 *)out, (int)n, s);
    if (e != cudaSuccess) return cuda_fail(e, "conjugate launch");
    return SAR_OK;
}

sar_status sar_transpose(int64_t rows, int64_t cols, const void *in, void *out, sar_stream stream) {
    if (rows < 1 || cols < 1) return fail(SAR_ERR_INVALID_ARG, "rows and cols must be >= 1");
    sar_status st;
    if ((st = check_device_ptr(in, "in")) != SAR_OK) return st;
    if ((st = check_device_ptr(out, "out")) != SAR_OK) return st;
    if (overlaps(in, out, sizeof(float2) * (size_t)(rows * cols)))
        return fail(SAR_ERR_INVALID_ARG, "in and out overlap");
    cudaError_t e = sar::launch_transpose((const float2 *)in, (float2 *)out, rows, cols, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "transpose launch");
    return SAR_OK;
}

sar_status sar_plan_status(sar_plan p, sar_stream stream) {
    if (!p) return fail(SAR_ERR_INVALID_ARG, "plan is NULL");
    int word = 0;
    cudaStream_t s = (cudaStream_t)stream;
    SAR_CUDA(cudaMemcpyAsync(&word, p->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status read");
    SAR_CUDA(cudaStreamSynchronize(s), "stream synchronise");
    if (word == 0) return SAR_OK;
    SAR_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), s), "status reset");
    SAR_CUDA(cudaStreamSynchronize(s), "stream synchronise");
    return fail(SAR_ERR_TIMEOUT, "a device-side wait of this plan's kernels timed out; the affected lines were "
                                 "not written");
}

sar_status sar_sync(sar_stream stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "device error");
    return SAR_OK;
}

}  // extern "C"
