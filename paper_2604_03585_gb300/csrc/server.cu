// Continuous-batching request loop for scene compression.
//
// Requests (scenes of a few size classes) arrive over time; the loop admits a
// request as soon as a slot (a CUDA stream) is free and its footprint (raw +
// image, 2 x 8 bytes per sample) fits in the HBM budget left by the requests
// still running.  An admitted request allocates its buffers from a dedicated
// stream-ordered memory pool, copies its echo in from the device-resident
// input pool (the ingest, part of its latency), runs the scene compression of
// its size class's plan (plans, filters and tables stay resident), optionally
// copies its image out, frees its buffers stream-ordered and records a
// completion event.  Requests on different slots run concurrently on the GPU.
// A completion poller releases budget and slots; latency = completion time on
// the GPU clock - arrival time.  When the oldest waiting request does not fit
// the remaining budget, later requests that do fit may pass it for at most
// `backfill_s` seconds, after which admission waits for it.  With
// size_priority, a slot holds one stream per size class and a request runs on
// the stream of its class, whose CUDA stream priority rises as the class's
// scene size falls: when SMs free up, the block scheduler dispatches the
// waiting blocks of smaller scenes first (shortest job first at block
// granularity; no work is dropped or reordered within a request).
#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <stdio.h>
#include <vector>

#include "../../include/sar.h"

namespace sar {
sar_status report_error(sar_status st, const char *msg);
sar_status validate_device_ptr(const void *p, const char *what);
}  // namespace sar

namespace {

struct Slot {
    std::vector<cudaStream_t> streams;   // one per priority level in use
    cudaEvent_t done = nullptr;
    int req = -1;
    int64_t footprint = 0;
    double admit_t = 0;   // host time of the request's admission
    int level = 0;        // its class's priority level
};

struct Class {
    int64_t n_range = 0, n_az = 0;
    const void *pool = nullptr;
    sar_plan plan = nullptr;
    int level = 0;   // index of the slot stream its requests run on
    size_t bytes() const { return (size_t)n_range * (size_t)n_az * 8; }
};

}  // namespace

struct sar_server_s {
    std::vector<Class> classes;
    std::vector<Slot> slots;
    cudaMemPool_t mempool = nullptr;
    int64_t budget = 0;
    double backfill_s = 0.05;
    double aging_s = 0;   // 0: no aging
    cudaEvent_t base = nullptr;
};

static void server_free(sar_server s) {
    if (!s) return;
    for (auto &sl : s->slots) {
        if (sl.done) cudaEventDestroy(sl.done);
        for (cudaStream_t st : sl.streams)
            if (st) cudaStreamDestroy(st);
    }
    for (auto &c : s->classes)
        if (c.plan) sar_plan_destroy(c.plan);
    if (s->base) cudaEventDestroy(s->base);
    if (s->mempool) cudaMemPoolDestroy(s->mempool);
    delete s;
}

extern "C" {

sar_status sar_server_create(const sar_server_config *cfg, sar_server *out) {
    if (!out) return sar::report_error(SAR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg || cfg->n_classes < 1 || !cfg->n_range || !cfg->n_az || !cfg->pool || !cfg->range_spectrum ||
        !cfg->az_spectrum)
        return sar::report_error(SAR_ERR_INVALID_ARG, "config needs at least one complete size class");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 256)
        return sar::report_error(SAR_ERR_INVALID_ARG, "max_inflight must be in [1, 256]");
    if (cfg->hbm_budget_bytes <= 0) return sar::report_error(SAR_ERR_INVALID_ARG, "hbm_budget_bytes must be > 0");
    sar_server s = new (std::nothrow) sar_server_s;
    if (!s) return sar::report_error(SAR_ERR_OUT_OF_MEMORY, "host allocation failed");
    s->budget = cfg->hbm_budget_bytes;
    s->backfill_s = cfg->backfill_s > 0 ? cfg->backfill_s : 0.0;
    s->aging_s = cfg->aging_s > 0 ? cfg->aging_s : 0.0;
    sar_status st = SAR_OK;
    for (int32_t k = 0; k < cfg->n_classes && st == SAR_OK; ++k) {
        Class c;
        c.n_range = cfg->n_range[k];
        c.n_az = cfg->n_az[k];
        c.pool = cfg->pool[k];
        if ((st = sar::validate_device_ptr(c.pool, "pool scene")) != SAR_OK) break;
        if ((int64_t)(2 * c.bytes()) > s->budget) {
            st = sar::report_error(SAR_ERR_INVALID_ARG, "a size class does not fit the HBM budget on its own");
            break;
        }
        sar_filters f{cfg->range_spectrum[k], cfg->az_spectrum[k], SAR_PREC_FP32, 0};
        st = sar_plan_create(c.n_range, c.n_az, &f, &c.plan);
        s->classes.push_back(c);
    }
    if (st != SAR_OK) {
        server_free(s);
        return st;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&s->mempool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = ~0ULL;   // keep freed memory in the pool for the next requests
        e = cudaMemPoolSetAttribute(s->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) {
        // no reuse through an inserted wait on another slot's stream: a request
        // would then wait for the request that freed the memory (with size
        // priority, often a starved large one).  Budget is released only after
        // a request's frees have completed, so memory freed by finished
        // requests is reused without a wait and the pool stays within the budget.
        int no = 0;
        e = cudaMemPoolSetAttribute(s->mempool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    // stream priorities: one level per distinct scene size, the smallest size
    // at the greatest priority (numerically lowest), clamped to the device's range
    std::vector<int> prio(1, 0);
    if (cfg->size_priority) {
        int least = 0, greatest = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        std::vector<size_t> sizes;
        for (const Class &c : s->classes) sizes.push_back(c.bytes());
        std::sort(sizes.begin(), sizes.end());
        sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
        prio.assign(sizes.size(), 0);
        for (size_t r = 0; r < sizes.size(); ++r) prio[r] = std::min(greatest + (int)r, least);
        for (Class &c : s->classes)
            c.level = (int)(std::lower_bound(sizes.begin(), sizes.end(), c.bytes()) - sizes.begin());
    }
    s->slots.resize(cfg->max_inflight);
    for (auto &sl : s->slots) {
        sl.streams.assign(prio.size(), nullptr);
        for (size_t r = 0; r < prio.size(); ++r)
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.streams[r], cudaStreamNonBlocking, prio[r]);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.done);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&s->base);
    if (e != cudaSuccess) {
        cudaGetLastError();
        server_free(s);
        return sar::report_error(SAR_ERR_CUDA, "server streams, events or memory pool");
    }
    *out = s;
    return SAR_OK;
}

sar_status sar_server_run(sar_server s, const sar_request *reqs, int32_t n, int32_t mode, sar_request_result *res) {
    if (!s || !reqs || !res || n < 0) return sar::report_error(SAR_ERR_INVALID_ARG, "server, requests or results");
    if (mode != SAR_SERVE_OPEN_LOOP && mode != SAR_SERVE_CLOSED_LOOP)
        return sar::report_error(SAR_ERR_INVALID_ARG, "unknown mode");
    for (int32_t i = 0; i < n; ++i) {
        if (reqs[i].size_class < 0 || reqs[i].size_class >= (int32_t)s->classes.size())
            return sar::report_error(SAR_ERR_INVALID_ARG, "request with an unknown size class");
        if (i && mode == SAR_SERVE_OPEN_LOOP && reqs[i].arrival_s < reqs[i - 1].arrival_s)
            return sar::report_error(SAR_ERR_INVALID_ARG, "arrival times must not decrease");
        res[i] = sar_request_result{mode == SAR_SERVE_CLOSED_LOOP ? 0.0 : reqs[i].arrival_s, -1.0, -1.0, -1};
    }
    using clock = std::chrono::steady_clock;
    if (cudaDeviceSynchronize() != cudaSuccess) return sar::report_error(SAR_ERR_CUDA, "device not idle");
    cudaEventRecord(s->base, s->slots[0].streams[0]);
    cudaEventSynchronize(s->base);
    const auto t0 = clock::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };

    std::deque<int> queue;
    int next = 0, done = 0;
    int64_t used = 0;
    double head_blocked_since = -1.0;
    sar_status fail = SAR_OK;

    auto admit = [&](int i, Slot &sl) -> bool {
        const Class &c = s->classes[reqs[i].size_class];
        const size_t bytes = c.bytes();
        cudaStream_t st = sl.streams[c.level];
        void *raw = nullptr, *img = nullptr;
        if (cudaMallocFromPoolAsync(&raw, bytes, s->mempool, st) != cudaSuccess ||
            cudaMallocFromPoolAsync(&img, bytes, s->mempool, st) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        res[i].admit_s = now_s();
        bool ok = cudaMemcpyAsync(raw, c.pool, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        ok = ok && sar_rda_process(c.plan, raw, img, st) == SAR_OK;
        if (ok && reqs[i].output)
            ok = cudaMemcpyAsync(reqs[i].output, img, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        cudaFreeAsync(raw, st);
        cudaFreeAsync(img, st);
        ok = ok && cudaEventRecord(sl.done, st) == cudaSuccess;
        sl.req = i;
        sl.admit_t = res[i].admit_s;
        sl.level = c.level;
        sl.footprint = (int64_t)(2 * bytes);
        used += sl.footprint;
        res[i].status = ok ? SAR_OK : SAR_ERR_CUDA;
        return ok;
    };

    while (done < n && fail == SAR_OK) {
        const double t = now_s();
        while (next < n && (mode == SAR_SERVE_CLOSED_LOOP || reqs[next].arrival_s <= t)) queue.push_back(next++);
        bool progress = false;
        // completions
        for (auto &sl : s->slots) {
            if (sl.req < 0) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            float ms = 0.f;
            if (q == cudaSuccess && cudaEventElapsedTime(&ms, s->base, sl.done) == cudaSuccess)
                res[sl.req].done_s = ms * 1e-3;
            else
                res[sl.req].status = SAR_ERR_CUDA;
            used -= sl.footprint;
            sl.req = -1;
            ++done;
            progress = true;
        }
        // aging: while a request has been in flight longer than aging_s, only
        // requests of its priority level or lower (its size or larger) are
        // admitted, so the work already queued ahead of it drains and its
        // blocks reach the SMs
        int floor_level = 0;
        if (s->aging_s > 0)
            for (const auto &sl : s->slots)
                if (sl.req >= 0 && t - sl.admit_t > s->aging_s) floor_level = std::max(floor_level, sl.level);
        auto eligible = [&](int j) { return s->classes[reqs[j].size_class].level >= floor_level; };
        // admissions: oldest eligible first; later ones may pass a head that
        // does not fit for at most backfill_s
        for (auto &sl : s->slots) {
            if (sl.req >= 0 || queue.empty()) continue;
            size_t h = 0;
            while (h < queue.size() && h < 256 && !eligible(queue[h])) ++h;
            if (h == queue.size() || h == 256) break;
            int pick = -1;
            size_t pos = h;
            const int head = queue[h];
            const int64_t head_fp = 2 * (int64_t)s->classes[reqs[head].size_class].bytes();
            if (used + head_fp <= s->budget) {
                pick = head;
                head_blocked_since = -1.0;
            } else {
                if (head_blocked_since < 0) head_blocked_since = t;
                if (t - head_blocked_since <= s->backfill_s) {
                    for (size_t k = h + 1; k < queue.size() && k < 256; ++k) {
                        const int j = queue[k];
                        if (eligible(j) && used + 2 * (int64_t)s->classes[reqs[j].size_class].bytes() <= s->budget) {
                            pick = j;
                            pos = k;
                            break;
                        }
                    }
                }
            }
            if (pick < 0) break;
            if (!admit(pick, sl)) {
                fail = sar::report_error(SAR_ERR_CUDA, "request admission failed");
                break;
            }
            queue.erase(queue.begin() + (long)pos);
            progress = true;
        }
        if (!progress && queue.empty() && next < n && mode == SAR_SERVE_OPEN_LOOP) {
            // idle until the next arrival is near (or a completion shows up)
            bool busy = false;
            for (auto &sl : s->slots) busy |= sl.req >= 0;
            if (!busy) {
                const double wait = reqs[next].arrival_s - now_s();
                if (wait > 200e-6) {
                    const auto until = t0 + std::chrono::duration_cast<clock::duration>(
                                                std::chrono::duration<double>(reqs[next].arrival_s - 100e-6));
                    while (clock::now() < until) {
                    }
                }
            }
        }
    }
    cudaDeviceSynchronize();
    return fail;
}

sar_status sar_server_destroy(sar_server s) {
    if (s) cudaDeviceSynchronize();
    server_free(s);
    return SAR_OK;
}

}  // extern "C"
