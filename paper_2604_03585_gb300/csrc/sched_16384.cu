// Line-engine instantiations for N = 16384 (one line per block).
#include "launch.cuh"

namespace sar {
namespace {
using S16384 = Sched<16384, 32, 16, 32, 32>;   // 512 threads per line, 135 KB shared memory
using S16384c = Sched<16384, 64, 16, 32, 32>;  // 256 threads per line (streamed only)
const SchedDesc kTable[] = {
    make_streamed_desc<S16384, 1, true, -4>("n16384_e32_r16x32x32_sr1"),
    make_desc<S16384, 1>("n16384_e32_r16x32x32_l1"),
    make_streamed_desc<S16384c, 1, true>("n16384_e64_r16x32x32_sr1"),
};
}  // namespace

const SchedDesc *schedules_16384(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
