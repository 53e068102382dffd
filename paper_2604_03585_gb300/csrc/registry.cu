// Schedule lookup and the host-side filter permutation.
#include <string.h>

#include "registry.h"

namespace sar {

namespace {
struct All {
    const SchedDesc *p[64];
    int n = 0;
    All() {
        const SchedDesc *(*tables[])(int *) = {schedules_small, schedules_4096, schedules_large};
        for (auto f : tables) {
            int c = 0;
            const SchedDesc *t = f(&c);
            for (int i = 0; i < c && n < 64; ++i) p[n++] = &t[i];
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

// First compiled schedule of each length is its default.
const SchedDesc *default_schedule(int n) {
    for (int i = 0; i < all().n; ++i)
        if (all().p[i]->n == n) return all().p[i];
    return nullptr;
}

void filter_slot_to_k(const SchedDesc &d, int32_t *idx) {
    const int N = d.n, E = d.e, T = N / E, RL = d.rl;
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
            idx[j * T + t] = k;
        }
}

}  // namespace sar
