// Line-engine instantiations for N = 2048.
#include "launch.cuh"

namespace sar {
namespace {
using S2048b = Sched<2048, 16, 16, 16, 8>;    // 128 threads per line
using S2048c = Sched<2048, 16, 16, 8, 16>;    // 128 threads per line, last radix 16: minimum wavefronts
using S2048d = Sched<2048, 32, 16, 8, 16>;    // 64 threads per line
// The first schedule of a length is its default (and the first one with a
// folded corner turn the default of the fold): the 16 x 8 x 16 geometry,
// whose every pass takes the minimum two wavefronts per warp access
// (16 x 16 x 8 takes four in its first two passes).
const SchedDesc kTable[] = {
    make_desc<S2048c, 1>("n2048_e16_r16x8x16_l1"),
    make_streamed_desc<S2048d, 2, true, -4>("n2048_e32_r16x8x16_sr2"),
    make_streamed_desc<S2048c, 1, false, -4>("n2048_e16_r16x8x16_s1"),
    make_streamed_desc<S2048d, 4, true>("n2048_e32_r16x8x16_sr4"),
    make_streamed_desc<S2048b, 1, false, -4>("n2048_e16_r16x16x8_s1"),
};
}  // namespace

const SchedDesc *schedules_2048(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
