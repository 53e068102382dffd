// Line-engine instantiations for N = 256 ... 1024 (several lines per block).
#include "launch.cuh"

namespace sar {
namespace {
using S256 = Sched<256, 16, 16, 16>;     // 16 threads per line
using S512 = Sched<512, 32, 16, 32>;     // 16 threads per line
using S1024 = Sched<1024, 32, 32, 32>;   // one warp per line
using S256b = Sched<256, 16, 16, 16>;
using S512b = Sched<512, 16, 16, 8, 4>;       // 32 threads per line, three passes
using S1024b = Sched<1024, 16, 16, 16, 4>;    // 64 threads per line
const SchedDesc kTable[] = {
    make_desc<S256, 8>("n256_e16_r16x16_l8"),
    make_desc<S256b, 16>("n256_e16_r16x16_l16"),
    make_desc<S512, 8>("n512_e32_r16x32_l8"),
    make_desc<S512b, 4>("n512_e16_r16x8x4_l4"),
    make_desc<S1024, 4>("n1024_e32_r32x32_l4"),
    make_desc<S1024b, 2>("n1024_e16_r16x16x4_l2"),
    make_streamed_desc<S1024, 4, false, 4>("n1024_e32_r32x32_s4"),
    make_streamed_desc<S512, 8, false, 4>("n512_e32_r16x32_s8"),
    make_streamed_desc<S256, 8, false, 4>("n256_e16_r16x16_s8"),
    make_persistent_desc<S1024>("n1024_e32_r32x32_p"),
    make_persistent_desc<S1024b>("n1024_e16_r16x16x4_p"),
};
}  // namespace

const SchedDesc *schedules_small(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
