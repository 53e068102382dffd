// Line-engine instantiations for N = 256 ... 2048 (several lines per block).
#include "launch.cuh"

namespace sar {
namespace {
using S256 = Sched<256, 16, 16, 16>;     // 16 threads per line
using S512 = Sched<512, 32, 16, 32>;     // 16 threads per line
using S1024 = Sched<1024, 32, 32, 32>;   // one warp per line
using S2048 = Sched<2048, 64, 32, 64>;   // one warp per line
const SchedDesc kTable[] = {
    make_desc<S256, 8>("n256_e16_r16x16_l8"),
    make_desc<S512, 8>("n512_e32_r16x32_l8"),
    make_desc<S1024, 4>("n1024_e32_r32x32_l4"),
    make_desc<S2048, 2>("n2048_e64_r32x64_l2"),
};
}  // namespace

const SchedDesc *schedules_small(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
