// Line-engine instantiations for N = 4096 (64 / 256 threads per line, persistent).
#include "launch.cuh"

namespace sar {
namespace {
using S4096a = Sched<4096, 64, 64, 64>;        // 64 threads per line, one exchange per transform
using S4096b = Sched<4096, 16, 16, 16, 16>;    // 256 threads per line, two exchanges per transform
using S4096c = Sched<4096, 32, 16, 16, 16>;    // 128 threads per line
using S4096g = Sched<4096, 64, 16, 16, 16>;    // 64 threads per line, four groups per pass (streamed only)
// Streamed schedules of 64 and 256 threads per line, and the persistent
// (TMA-prefetching) kernels.
const SchedDesc kTable[] = {
    make_streamed_desc<S4096g, 1, true, 4>("n4096_e64_r16x16x16_sr1"),
    make_streamed_desc<S4096g, 2, true>("n4096_e64_r16x16x16_sr2"),
    make_streamed_desc<S4096b, 1, false, 4>("n4096_e16_r16x16x16_s1"),
    make_persistent_desc<S4096a>("n4096_e64_r64x64_p"),
    make_persistent_desc<S4096b>("n4096_e16_r16x16x16_p"),
    make_persistent_desc<S4096c>("n4096_e32_r16x16x16_p"),
};
}  // namespace

const SchedDesc *schedules_4096_more(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
