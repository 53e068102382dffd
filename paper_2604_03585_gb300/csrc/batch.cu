// Ragged batches: many strips of different sizes compressed by one CUDA-graph
// launch.
//
// A strip is an n_az x n_range raw echo (n_range a power of two, n_az any
// count); its azimuth lines are transformed at L = max(256, next power of
// two >= n_az), zero-padded, and the image keeps its n_az columns.
//
// Default: one persistent kernel (batch_persistent.cu) walks a list of work
// items -- range items (k azimuth rows of a strip, compressed along range and
// written corner-turned into the image) and azimuth items (k range bins,
// compressed in place) -- with per-strip completion counters between a
// strip's range and azimuth items.  The graph is one memset of the counters
// and that one kernel.  Filters and twiddles are built per class: range
// classes by (n_range, range spectrum), azimuth classes by (L, azimuth
// spectrum), on the kernel's engine geometry of each length.
//
// SAR_BATCH_MULTI_KERNEL, and SAR_BATCH_EXACT_AZIMUTH (azimuth lines at
// exactly n_az, which needs the zero-padded linear convolution of lengths
// that are not powers of two): one fused launch per class walking a segment
// table (one segment per strip,
// the strip's lines concatenated), one batched transpose over all strips, and
// for such lengths one launch per strip, all captured into one graph.  Data
// path per strip there: range compression raw -> work (batch-owned scratch),
// corner turn work -> image, azimuth compression in place on image.  The raw
// echo is only read on both paths.
#include <algorithm>
#include <stdlib.h>
#include <new>
#include <stdio.h>
#include <string.h>
#include <vector>

#include "../../include/sar.h"
#include "batch_persistent.h"
#include "registry.h"
#include "streamed.cuh"
#include "tables.h"

namespace sar {
sar_status report_error(sar_status st, const char *msg);
sar_status validate_device_ptr(const void *p, const char *what);
sar_status validate_length(int64_t n, const char *what);

struct TSeg {
    const float2 *in;
    float2 *out;
    int64_t rows, cols, tiles_c;
};

// Corner turn of every strip in one launch: block b is tile b of the
// concatenated tile lists; 32 x 32 tiles through padded shared memory, as
// corner_turn_kernel.
__global__ void __launch_bounds__(256)
batched_transpose_kernel(const TSeg *segs, const int64_t *tile_begin, int n_seg) {
    __shared__ float2 tile[32][33];
    const int k = find_seg(tile_begin, n_seg, (int64_t)blockIdx.x);
    const TSeg sg = segs[k];
    const int64_t b = (int64_t)blockIdx.x - tile_begin[k];
    const int64_t tr = b / sg.tiles_c, tc = b % sg.tiles_c;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    const int64_t r0 = tr * 32, c0 = tc * 32;
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t r = r0 + ty + j, c = c0 + tx;
        if (r < sg.rows && c < sg.cols) tile[ty + j][tx] = sg.in[r * sg.cols + c];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t c = c0 + ty + j, r = r0 + tx;
        if (r < sg.rows && c < sg.cols) sg.out[c * sg.rows + r] = tile[tx][ty + j];
    }
}

}  // namespace sar

using sar::SchedDesc;

namespace {

int64_t next_pow2(int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct LineClass {
    const SchedDesc *d = nullptr;
    const void *spectrum = nullptr;
    int64_t n = 0;
    bool ragged = false;
    bool wrap = false;   // exact length n that is not a power of two: wrap schedule of length d->n
    std::vector<sar::Seg> segs;
    std::vector<int64_t> begin;   // prefix sums of lines, size segs + 1
    // device
    float2 *filt = nullptr, *tw = nullptr;
    sar::Seg *segs_dev = nullptr;
    int64_t *begin_dev = nullptr;
};

// The preferred schedule of length n that has a segment-table kernel.
const SchedDesc *seg_schedule(int n) {
    const SchedDesc *p = sar::default_schedule(n);
    if (p && p->fused_seg) return p;
    for (int i = 0; i < sar::schedule_count(); ++i)
        if (sar::schedule_at(i)->n == n && sar::schedule_at(i)->fused_seg) return sar::schedule_at(i);
    return nullptr;
}

// SAR_BATCH_AUTOTUNE: the fastest schedule of length n that has a
// segment-table kernel, timed by sar_autotune on `lines` lines of n (every
// compiled schedule of n; the medians come back in the registry's order of
// the schedules of n).  nullptr on any failure (the caller then keeps the
// preferred schedule).
const SchedDesc *tuned_seg_schedule(int n, int64_t lines) {
    std::vector<const SchedDesc *> of_n;
    for (int i = 0; i < sar::schedule_count(); ++i)
        if (sar::schedule_at(i)->n == n) of_n.push_back(sar::schedule_at(i));
    if (of_n.empty()) return nullptr;
    std::vector<float> ms(of_n.size(), 0.f);
    sar_schedule_desc best;
    float best_ms = 0.f;
    if (sar_autotune(n, lines, 5, SAR_TUNE_FUSED, nullptr, &best, &best_ms, ms.data(), (int32_t)ms.size()) != SAR_OK)
        return nullptr;
    const SchedDesc *win = nullptr;
    float win_ms = 0.f;
    for (size_t i = 0; i < of_n.size(); ++i)
        if (of_n[i]->fused_seg && ms[i] > 0.f && (!win || ms[i] < win_ms)) {
            win = of_n[i];
            win_ms = ms[i];
        }
    return win;
}

}  // namespace

struct sar_batch_s {
    std::vector<LineClass> range, az;
    std::vector<sar::TSeg> tsegs;
    std::vector<int64_t> tbegin;
    sar::TSeg *tsegs_dev = nullptr;
    int64_t *tbegin_dev = nullptr;
    void *tables = nullptr;    // filters, twiddles, segment tables
    void *work = nullptr;      // range-compressed strips
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    int64_t samples = 0;       // sum of n_az * n_range
    int32_t launches = 0;      // kernels in the graph
    int64_t strips = 0;
    // one-launch path
    bool persistent = false;
    int32_t n_range_classes = 0, n_az_classes = 0;
    int *status_dev = nullptr;  // 5 after a timed-out wait (sticky until sar_batch_status)
};

static void batch_free(sar_batch b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->tables) cudaFree(b->tables);
    if (b->work) cudaFree(b->work);
    delete b;
}

// Bound of the batch kernel's waits: about one second at the GB300's maximum
// SM clock, or SAR_WAIT_CYCLES.
static long long batch_wait_cycles() {
    const char *v = getenv("SAR_WAIT_CYCLES");
    const long long c = v ? atoll(v) : 0;
    return c > 0 ? c : 2000000000LL;
}

// Test hook (host-side fault injection): SAR_FAULT_INJECT_BATCH_WAIT=<i> makes
// batches created while it is set expect one range line more of strip i than
// it has, so that strip's completion counter never reaches its target and the
// kernel's bounded wait runs out.
static int64_t batch_inject_strip() {
    const char *v = getenv("SAR_FAULT_INJECT_BATCH_WAIT");
    return v ? atoll(v) : -1;
}

// The one-launch batch: classes and their tables, the strip and item tables,
// and a graph of one memset (the counters) and one kernel.
static sar_status create_persistent(const sar_strip *strips, int32_t count, sar_batch b) {
    struct TClass {
        const SchedDesc *d;
        const void *spectrum;
        int64_t n;
        bool range;
        float2 *filt = nullptr, *tw = nullptr;
    };
    std::vector<TClass> cls;
    auto class_of = [&](int64_t n, const void *spec, bool range) -> int {
        for (size_t i = 0; i < cls.size(); ++i)
            if (cls[i].n == n && cls[i].spectrum == spec && cls[i].range == range) return (int)i;
        const char *name = sar::batch_schedule_name((int)n);
        const SchedDesc *d = name ? sar::find_schedule(name) : nullptr;
        if (!d) return -1;
        cls.push_back(TClass{d, spec, n, range});
        if (range)
            ++b->n_range_classes;
        else
            ++b->n_az_classes;
        return (int)cls.size() - 1;
    };
    std::vector<int> rc(count), ac(count);
    std::vector<int64_t> L(count);
    for (int32_t i = 0; i < count; ++i) {
        L[i] = std::max<int64_t>(256, next_pow2(strips[i].n_az));
        if (L[i] > 16384) return sar::report_error(SAR_ERR_UNSUPPORTED, "azimuth transform length above 16384");
        rc[i] = class_of(strips[i].n_range, strips[i].range_spectrum, true);
        ac[i] = class_of(L[i], strips[i].az_spectrum, false);
        if (rc[i] < 0 || ac[i] < 0) return sar::report_error(SAR_ERR_UNSUPPORTED, "no batch engine for a strip length");
    }
    // item list: strips largest first; range items of strip j + 1 before the
    // azimuth items of strip j, so that an azimuth item's strip is finished
    // (or being finished by blocks that took its items earlier) when a block
    // takes it
    std::vector<int32_t> order(count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return strips[x].n_az * strips[x].n_range > strips[y].n_az * strips[y].n_range;
    });
    std::vector<sar::BItem> items;
    auto add_range = [&](int32_t i) {
        const int k = sar::batch_lines_per_item((int)strips[i].n_range);
        for (int64_t a = 0; a < strips[i].n_az; a += k)
            items.push_back(sar::BItem{0, i, (int32_t)a, (int32_t)std::min<int64_t>(k, strips[i].n_az - a)});
    };
    auto add_az = [&](int32_t i) {
        const int k = sar::batch_lines_per_item((int)L[i]);
        for (int64_t r = 0; r < strips[i].n_range; r += k)
            items.push_back(sar::BItem{1, i, (int32_t)r, (int32_t)std::min<int64_t>(k, strips[i].n_range - r)});
    };
    for (int32_t j = 0; j < count; ++j) {
        add_range(order[j]);
        if (j > 0) add_az(order[j - 1]);
    }
    add_az(order[count - 1]);
    if (items.size() > (size_t)0x7fffffff) return sar::report_error(SAR_ERR_UNSUPPORTED, "too many work items");

    // ---- device memory: tables, strips, items, counters, status
    size_t tab = 0;
    auto reserve = [&](size_t bytes) {
        const size_t o = tab;
        tab += align_up(bytes);
        return o;
    };
    std::vector<size_t> off_f, off_t;
    int64_t max_n = 0;
    for (auto &c : cls) {
        off_f.push_back(reserve(sizeof(float2) * c.d->n));
        off_t.push_back(reserve(sizeof(float2) * c.d->tw_elems));
        max_n = std::max<int64_t>(max_n, c.d->n);
    }
    const size_t off_st = reserve(sizeof(sar::BStrip) * count);
    const size_t off_it = reserve(sizeof(sar::BItem) * items.size());
    const size_t off_ctr = reserve(sizeof(int) * ((size_t)count + 1));
    const size_t off_status = reserve(sizeof(int));
    const size_t off_ix = reserve(sizeof(int32_t) * max_n);
    if (cudaMalloc(&b->tables, tab) != cudaSuccess) {
        cudaGetLastError();
        return sar::report_error(SAR_ERR_OUT_OF_MEMORY, "batch tables");
    }
    char *base = (char *)b->tables;
    sar::BStrip *strips_dev = (sar::BStrip *)(base + off_st);
    sar::BItem *items_dev = (sar::BItem *)(base + off_it);
    int *counters = (int *)(base + off_ctr);
    b->status_dev = (int *)(base + off_status);
    int32_t *idx_dev = (int32_t *)(base + off_ix);

    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the caller's spectra are ready
    if (e == cudaSuccess) e = sar::prepare_batch_persistent();
    std::vector<int32_t> idx;
    for (size_t ci = 0; ci < cls.size() && e == cudaSuccess; ++ci) {
        TClass &c = cls[ci];
        c.filt = (float2 *)(base + off_f[ci]);
        c.tw = (float2 *)(base + off_t[ci]);
        if ((e = c.d->prepare()) != cudaSuccess) break;
        if ((e = sar::build_twiddles(*c.d, c.tw, s)) != cudaSuccess) break;
        idx.assign(c.d->n, 0);
        sar::filter_slot_to_k(*c.d, idx.data());
        if ((e = cudaMemcpyAsync(idx_dev, idx.data(), sizeof(int32_t) * c.d->n, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            break;
        if ((e = sar::build_filter(*c.d, (const float2 *)c.spectrum, c.filt, idx_dev, s)) != cudaSuccess) break;
        e = cudaStreamSynchronize(s);   // idx is reused by the next class
    }
    const int64_t inject = batch_inject_strip();
    std::vector<sar::BStrip> bs(count);
    for (int32_t i = 0; i < count; ++i) {
        const sar_strip &st = strips[i];
        bs[i] = sar::BStrip{(const float2 *)st.raw, (float2 *)st.image, cls[rc[i]].filt, cls[rc[i]].tw,
                            cls[ac[i]].filt, cls[ac[i]].tw, (int32_t)st.n_range, (int32_t)st.n_az, (int32_t)L[i],
                            (int32_t)st.n_az + (i == inject ? 1 : 0)};
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(strips_dev, bs.data(), sizeof(sar::BStrip) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(items_dev, items.data(), sizeof(sar::BItem) * items.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status_dev, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    // ---- the graph: clear the counters, one kernel
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaMemsetAsync(counters, 0, sizeof(int) * ((size_t)count + 1), s);
        if (le == cudaSuccess)
            le = sar::launch_batch_persistent(items_dev, (int)items.size(), strips_dev, counters, counters + count,
                                              b->status_dev, batch_wait_cycles(), s);
        b->launches = 1;
        e = cudaStreamEndCapture(s, &b->graph);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        snprintf(msg, sizeof(msg), "batch set-up failed: %s", cudaGetErrorString(e));
        return sar::report_error(SAR_ERR_CUDA, msg);
    }
    b->persistent = true;
    return SAR_OK;
}

extern "C" {

sar_status sar_batch_create(const sar_strip *strips, int32_t count, uint32_t flags, sar_batch *out) {
    if (!out) return sar::report_error(SAR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!strips || count < 1) return sar::report_error(SAR_ERR_INVALID_ARG, "need at least one strip");
    if (flags & ~(SAR_BATCH_EXACT_AZIMUTH | SAR_BATCH_MULTI_KERNEL | SAR_BATCH_AUTOTUNE))
        return sar::report_error(SAR_ERR_INVALID_ARG, "unknown flags");
    const bool exact = (flags & SAR_BATCH_EXACT_AZIMUTH) != 0;
    const bool multi = exact || (flags & SAR_BATCH_MULTI_KERNEL) != 0;
    const bool tune = (flags & SAR_BATCH_AUTOTUNE) != 0;
    if (tune && !multi)
        return sar::report_error(SAR_ERR_INVALID_ARG,
                                 "SAR_BATCH_AUTOTUNE needs the multi-kernel graph (the one-launch kernel's engines are fixed)");
    sar_status st;
    for (int32_t i = 0; i < count; ++i) {
        const sar_strip &s = strips[i];
        if ((st = sar::validate_length(s.n_range, "strip n_range")) != SAR_OK) return st;
        if (s.n_range > 16384)
            return sar::report_error(SAR_ERR_UNSUPPORTED, "strip n_range must be at most 16384");
        if (s.n_az < 1 || s.n_az > 16384)
            return sar::report_error(SAR_ERR_UNSUPPORTED, "strip n_az must be in [1, 16384]");
        const bool az_pow2 = s.n_az >= 256 && (s.n_az & (s.n_az - 1)) == 0;
        if (exact && !az_pow2 && (s.n_az < 2 || s.n_az > 8192))
            return sar::report_error(SAR_ERR_UNSUPPORTED,
                                     "exact azimuth lengths that are not powers of two must be in [2, 8192]");
        if ((st = sar::validate_device_ptr(s.raw, "strip raw")) != SAR_OK) return st;
        if ((st = sar::validate_device_ptr(s.image, "strip image")) != SAR_OK) return st;
        if ((st = sar::validate_device_ptr(s.range_spectrum, "strip range_spectrum")) != SAR_OK) return st;
        if ((st = sar::validate_device_ptr(s.az_spectrum, "strip az_spectrum")) != SAR_OK) return st;
    }
    sar_batch b = new (std::nothrow) sar_batch_s;
    if (!b) return sar::report_error(SAR_ERR_OUT_OF_MEMORY, "host allocation failed");
    cudaGetDevice(&b->device);
    b->strips = count;
    if (!multi) {
        for (int32_t i = 0; i < count; ++i) b->samples += strips[i].n_az * strips[i].n_range;
        const sar_status pst = create_persistent(strips, count, b);
        if (pst != SAR_OK) {
            batch_free(b);
            return pst;
        }
        *out = b;
        return SAR_OK;
    }

    // ---- classes and segment tables (host side)
    size_t work_elems = 0;
    std::vector<size_t> work_off(count);
    for (int32_t i = 0; i < count; ++i) {
        work_off[i] = work_elems;
        work_elems += (size_t)strips[i].n_az * (size_t)strips[i].n_range;
    }
    b->samples = (int64_t)work_elems;
    auto class_of = [](std::vector<LineClass> &cls, int64_t n, const void *spec) -> LineClass & {
        for (auto &c : cls)
            if (c.n == n && c.spectrum == spec) return c;
        cls.emplace_back();
        cls.back().n = n;
        cls.back().spectrum = spec;
        cls.back().begin.push_back(0);
        return cls.back();
    };
    for (int32_t i = 0; i < count; ++i) {
        const sar_strip &s = strips[i];
        const int64_t L = exact ? s.n_az : std::max<int64_t>(256, next_pow2(s.n_az));
        if (L > 16384) {
            batch_free(b);
            return sar::report_error(SAR_ERR_UNSUPPORTED, "azimuth transform length above 16384");
        }
        LineClass &rc = class_of(b->range, s.n_range, s.range_spectrum);
        // out: the strip's slice of the work buffer, filled in below
        rc.segs.push_back(sar::Seg{(const float2 *)s.raw, nullptr, s.n_range, s.n_range, (int32_t)s.n_range, 0});
        rc.begin.push_back(rc.begin.back() + s.n_az);
        LineClass &ac = class_of(b->az, L, s.az_spectrum);
        ac.segs.push_back(sar::Seg{(const float2 *)s.image, (float2 *)s.image, s.n_az, s.n_az, (int32_t)s.n_az, 0});
        ac.begin.push_back(ac.begin.back() + s.n_range);
        if (s.n_az < L) ac.ragged = true;
        if (exact && !(L >= 256 && (L & (L - 1)) == 0)) ac.wrap = true;
        b->tsegs.push_back(sar::TSeg{nullptr, (float2 *)s.image, s.n_az, s.n_range, (s.n_range + 31) / 32});
    }
    b->tbegin.push_back(0);
    for (auto &t : b->tsegs) b->tbegin.push_back(b->tbegin.back() + ((t.rows + 31) / 32) * t.tiles_c);
    for (auto *cls : {&b->range, &b->az})
        for (auto &c : *cls) {
            if (c.wrap) {
                int64_t L = 256;
                while (L < 2 * c.n - 1) L <<= 1;
                c.d = sar::wrap_schedule((int)L);
            } else {
                c.d = nullptr;
                if (tune) {
                    const int64_t lines = c.begin.back() < (1 << 24) / c.n ? c.begin.back() : (1 << 24) / c.n;
                    c.d = tuned_seg_schedule((int)c.n, lines > 0 ? lines : 1);
                }
                if (!c.d) c.d = seg_schedule((int)c.n);
            }
            if (!c.d) {
                batch_free(b);
                return sar::report_error(SAR_ERR_UNSUPPORTED, "no segment-table kernel for a strip length");
            }
        }

    // ---- device memory: one block of tables, one work buffer
    size_t tab = 0;
    auto reserve = [&](size_t bytes) {
        const size_t o = tab;
        tab += align_up(bytes);
        return o;
    };
    std::vector<size_t> off_f, off_t, off_s, off_b;
    int64_t max_n = 0;
    for (auto *cls : {&b->range, &b->az})
        for (auto &c : *cls) {
            off_f.push_back(reserve(sizeof(float2) * c.d->n));
            off_t.push_back(reserve(sizeof(float2) * c.d->tw_elems));
            off_s.push_back(reserve(sizeof(sar::Seg) * c.segs.size()));
            off_b.push_back(reserve(sizeof(int64_t) * c.begin.size()));
            max_n = std::max<int64_t>(max_n, c.d->n);
        }
    const size_t off_ts = reserve(sizeof(sar::TSeg) * b->tsegs.size());
    const size_t off_tb = reserve(sizeof(int64_t) * b->tbegin.size());
    const size_t off_ix = reserve(sizeof(int32_t) * max_n);
    if (cudaMalloc(&b->tables, tab) != cudaSuccess || cudaMalloc(&b->work, sizeof(float2) * work_elems) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return sar::report_error(SAR_ERR_OUT_OF_MEMORY, "batch tables or work buffer");
    }
    char *base = (char *)b->tables;
    size_t ci = 0;
    float2 *work = (float2 *)b->work;
    {
        // range segments write to each strip's slice of the work buffer, which
        // the transpose then reads
        size_t strip = 0;
        std::vector<size_t> seen(b->range.size(), 0);
        for (int32_t i = 0; i < count; ++i) {
            const sar_strip &s = strips[i];
            for (size_t r = 0; r < b->range.size(); ++r) {
                LineClass &c = b->range[r];
                if (c.n == s.n_range && c.spectrum == s.range_spectrum) {
                    c.segs[seen[r]++].out = work + work_off[i];
                    break;
                }
            }
            b->tsegs[strip++].in = work + work_off[i];
        }
    }
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the caller's spectra are ready
    int32_t *idx_dev = (int32_t *)(base + off_ix);
    std::vector<int32_t> idx;
    for (auto *cls : {&b->range, &b->az})
        for (auto &c : *cls) {
            if (e != cudaSuccess) break;
            c.filt = (float2 *)(base + off_f[ci]);
            c.tw = (float2 *)(base + off_t[ci]);
            c.segs_dev = (sar::Seg *)(base + off_s[ci]);
            c.begin_dev = (int64_t *)(base + off_b[ci]);
            ++ci;
            if ((e = c.d->prepare()) != cudaSuccess) break;
            if ((e = sar::build_twiddles(*c.d, c.tw, s)) != cudaSuccess) break;
            idx.assign(c.d->n, 0);
            sar::filter_slot_to_k(*c.d, idx.data());
            if ((e = cudaMemcpyAsync(idx_dev, idx.data(), sizeof(int32_t) * c.d->n, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess)
                break;
            const float2 *spectrum = (const float2 *)c.spectrum;
            void *design = nullptr;
            if (c.wrap) {
                // G = FFT_L(IFFT_n(H) zero-padded to L), designed in FP64
                const size_t scratch = sar::wrap_filter_scratch_bytes((int)c.n, c.d->n);
                if ((e = cudaMalloc(&design, scratch + sizeof(float2) * (size_t)c.d->n)) != cudaSuccess) break;
                float2 *G = (float2 *)((char *)design + scratch);
                if ((e = sar::build_wrap_filter(spectrum, (int)c.n, c.d->n, design, G, s)) != cudaSuccess) {
                    cudaFree(design);
                    break;
                }
                spectrum = G;
            }
            e = sar::build_filter(*c.d, spectrum, c.filt, idx_dev, s);
            if (design) {
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                cudaFree(design);
            }
            if (e != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(c.segs_dev, c.segs.data(), sizeof(sar::Seg) * c.segs.size(), cudaMemcpyHostToDevice,
                                     s)) != cudaSuccess)
                break;
            if ((e = cudaMemcpyAsync(c.begin_dev, c.begin.data(), sizeof(int64_t) * c.begin.size(),
                                     cudaMemcpyHostToDevice, s)) != cudaSuccess)
                break;
            e = cudaStreamSynchronize(s);   // idx is reused by the next class
        }
    b->tsegs_dev = (sar::TSeg *)(base + off_ts);
    b->tbegin_dev = (int64_t *)(base + off_tb);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tsegs_dev, b->tsegs.data(), sizeof(sar::TSeg) * b->tsegs.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tbegin_dev, b->tbegin.data(), sizeof(int64_t) * b->tbegin.size(), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);

    // ---- capture the whole batch into one graph
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        for (auto &c : b->range) {
            if (le == cudaSuccess)
                le = c.d->fused_seg(c.segs_dev, c.begin_dev, (int)c.segs.size(), c.begin.back(), false, c.filt, c.tw, s);
            ++b->launches;
        }
        if (le == cudaSuccess) {
            sar::batched_transpose_kernel<<<(unsigned)b->tbegin.back(), 256, 0, s>>>(b->tsegs_dev, b->tbegin_dev,
                                                                                    (int)b->tsegs.size());
            le = cudaGetLastError();
            ++b->launches;
        }
        const sar::FusedCtl no_ctl{nullptr, 0, -1};
        for (auto &c : b->az) {
            if (c.wrap) {   // one launch per strip of this exact length
                for (size_t k = 0; k < c.segs.size() && le == cudaSuccess; ++k) {
                    const sar::Seg &sg = c.segs[k];
                    le = c.d->fused(sg.in, sg.out, c.begin[k + 1] - c.begin[k], sg.ld_in, sg.valid, c.filt, c.tw,
                                    no_ctl, s);
                    ++b->launches;
                }
                continue;
            }
            if (le == cudaSuccess)
                le = c.d->fused_seg(c.segs_dev, c.begin_dev, (int)c.segs.size(), c.begin.back(), c.ragged, c.filt, c.tw,
                                    s);
            ++b->launches;
        }
        e = cudaStreamEndCapture(s, &b->graph);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        char msg[256];
        snprintf(msg, sizeof(msg), "batch set-up failed: %s", cudaGetErrorString(e));
        return sar::report_error(SAR_ERR_CUDA, msg);
    }
    *out = b;
    return SAR_OK;
}

sar_status sar_batch_run(sar_batch b, sar_stream stream) {
    if (!b) return sar::report_error(SAR_ERR_INVALID_ARG, "batch is NULL");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "graph launch: %s", cudaGetErrorString(e));
        return sar::report_error(SAR_ERR_CUDA, msg);
    }
    return SAR_OK;
}

sar_status sar_batch_info(sar_batch b, sar_batch_info_t *info) {
    if (!b || !info) return sar::report_error(SAR_ERR_INVALID_ARG, "batch or info is NULL");
    info->strips = b->strips;
    info->samples = b->samples;
    info->kernels_per_run = b->launches;
    info->range_classes = b->persistent ? b->n_range_classes : (int32_t)b->range.size();
    info->azimuth_classes = b->persistent ? b->n_az_classes : (int32_t)b->az.size();
    info->work_bytes = b->persistent ? 0 : b->samples * 8;
    return SAR_OK;
}

sar_status sar_batch_status(sar_batch b, sar_stream stream) {
    if (!b) return sar::report_error(SAR_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, cudaGetErrorString(e));
    if (!b->status_dev) return SAR_OK;
    int v = 0;
    if ((e = cudaMemcpy(&v, b->status_dev, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return sar::report_error(SAR_ERR_CUDA, cudaGetErrorString(e));
    if (v == 0) return SAR_OK;
    if ((e = cudaMemset(b->status_dev, 0, sizeof(int))) != cudaSuccess)
        return sar::report_error(SAR_ERR_CUDA, cudaGetErrorString(e));
    return sar::report_error(SAR_ERR_TIMEOUT, "a bounded wait of the batch kernel ran out (a strip's range lines "
                                              "never all completed); the images of that run are incomplete");
}

sar_status sar_batch_destroy(sar_batch b) {
    batch_free(b);
    return SAR_OK;
}

}  // extern "C"
