// Line-engine instantiations for N = 4096 (the group-streamed schedules).
#include "launch.cuh"

namespace sar {
namespace {
using S4096c = Sched<4096, 32, 16, 16, 16>;    // 128 threads per line
using S4096h = Sched<4096, 32, 16, 16, 16, 5>; // as c, capped for 5 blocks per SM (streamed)
using S4096i = Sched<4096, 32, 16, 16, 16, 6>; // as c, capped for 6 blocks per SM (streamed)
// The group-streamed schedules of 128 threads per line; the first is the
// default of the length and of the folded range pass.
const SchedDesc kTable[] = {
    make_streamed_desc<S4096c, 1, true, -4>("n4096_e32_r16x16x16_sr1"),
    make_streamed_desc<S4096c, 1, true, -8>("n4096_e32_r16x16x16_sr1_c8"),
    make_streamed_desc<S4096c, 1, true, -16>("n4096_e32_r16x16x16_sr1_c16"),
    make_streamed_desc<S4096c, 1, true, 4>("n4096_e32_r16x16x16_sr1_q4"),
    make_streamed_desc<S4096c, 1, false>("n4096_e32_r16x16x16_s1"),
    make_streamed_desc<S4096c, 2, true>("n4096_e32_r16x16x16_sr2"),
    make_streamed_desc<S4096h, 1, true>("n4096_e32_r16x16x16_sr1_b5"),
    make_streamed_desc<S4096i, 1, true>("n4096_e32_r16x16x16_sr1_b6"),
};
}  // namespace

const SchedDesc *schedules_4096(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
