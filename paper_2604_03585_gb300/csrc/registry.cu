// Schedule lookup and the host-side filter permutation.
#include <string.h>

#include <mutex>

#include "mixed_radix.h"
#include "registry.h"

namespace sar {

namespace {
struct All {
    const SchedDesc *p[96];
    int n = 0;
    All() {
        const SchedDesc *(*tables[])(int *) = {schedules_small,      schedules_2048,      schedules_4096,
                                                  schedules_4096_plain, schedules_4096_more, schedules_8192,
                                                  schedules_16384,      schedules_cluster};
        for (auto f : tables) {
            int c = 0;
            const SchedDesc *t = f(&c);
            for (int i = 0; i < c && n < 96; ++i) p[n++] = &t[i];
        }
    }
};
const All &all() {
    static All a;
    return a;
}
}  // namespace

int schedule_count() { return all().n; }
const SchedDesc *schedule_at(int i) { return (i >= 0 && i < all().n) ? all().p[i] : nullptr; }

const SchedDesc *find_schedule(const char *name) {
    for (int i = 0; i < all().n; ++i)
        if (strcmp(all().p[i]->name, name) == 0) return all().p[i];
    return nullptr;
}

namespace {
std::mutex g_pref_mu;
const SchedDesc *g_preferred[32] = {};      // by log2(n)
const SchedDesc *g_preferred_ct[32] = {};   // folded range pass, by log2(n)
int log2i(int n) {
    int k = 0;
    while ((1 << k) < n && k < 31) ++k;
    return k;
}
}  // namespace

// The preferred schedule of a length: set by the autotuner or the caller,
// otherwise the first compiled schedule of that length.
const SchedDesc *default_schedule(int n) {
    {
        std::lock_guard<std::mutex> lk(g_pref_mu);
        const SchedDesc *p = g_preferred[log2i(n)];
        if (p && p->n == n) return p;
    }
    for (int i = 0; i < all().n; ++i)
        if (all().p[i]->n == n) return all().p[i];
    return nullptr;
}

// The preferred schedule of length n that can fold the corner turn into the
// range pass: the preferred schedule itself if it can, else the first
// compiled one that can, else nullptr.
const SchedDesc *default_ct_schedule(int n) {
    {
        std::lock_guard<std::mutex> lk(g_pref_mu);
        const SchedDesc *q = g_preferred_ct[log2i(n)];
        if (q && q->n == n) return q;
    }
    const SchedDesc *p = default_schedule(n);
    if (p && p->fused_ct) return p;
    for (int i = 0; i < all().n; ++i)
        if (all().p[i]->n == n && all().p[i]->fused_ct) return all().p[i];
    return nullptr;
}

void set_preferred_schedule(const SchedDesc *d) {
    std::lock_guard<std::mutex> lk(g_pref_mu);
    g_preferred[log2i(d->n)] = d;
    if (d->fused_ct) g_preferred_ct[log2i(d->n)] = d;
}

void set_preferred_ct_schedule(const SchedDesc *d) {
    std::lock_guard<std::mutex> lk(g_pref_mu);
    if (d->fused_ct) g_preferred_ct[log2i(d->n)] = d;
}

void filter_slot_to_k(const SchedDesc &d, int32_t *idx) {
    if (d.mixed) {
        mixed_positions(d.n, idx);
        return;
    }
    const int C = d.cluster > 1 ? d.cluster : 1;
    const int N = d.n / C, E = d.e, T = N / E, RL = d.rl;   // N: the per-block engine's length
    const int S1 = N / d.r1;
    const int S2 = S1 / d.r2;
    for (int t = 0; t < T; ++t)
        for (int j = 0; j < E; ++j) {
            const int s = j / RL, r = j % RL;
            const int P = (t + T * s) * RL + r;        // last-pass position
            const int k1 = P / S1, rem = P % S1;
            int k;
            if (d.r3 > 1)
                k = k1 + d.r1 * ((rem / S2) + d.r2 * (rem % S2));
            else
                k = k1 + d.r1 * rem;
            for (int c = 0; c < C; ++c) idx[c * N + j * T + t] = c + C * k;
        }
}

}  // namespace sar
