// Line-engine instantiations for N = 4096.
#include "launch.cuh"

namespace sar {
namespace {
using S4096a = Sched<4096, 64, 64, 64>;        // 64 threads per line, one exchange per transform
using S4096b = Sched<4096, 16, 16, 16, 16>;    // 256 threads per line, two exchanges per transform
const SchedDesc kTable[] = {
    make_desc<S4096a, 1>("n4096_e64_r64x64_l1"),
    make_desc<S4096a, 2>("n4096_e64_r64x64_l2"),
    make_desc<S4096b, 1>("n4096_e16_r16x16x16_l1"),
};
}  // namespace

const SchedDesc *schedules_4096(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
