// Line-engine instantiations for N = 4096.
#include "launch.cuh"

namespace sar {
namespace {
using S4096a = Sched<4096, 64, 64, 64>;        // 64 threads per line, one exchange per transform
using S4096b = Sched<4096, 16, 16, 16, 16>;    // 256 threads per line, two exchanges per transform
using S4096c = Sched<4096, 32, 16, 16, 16>;    // 128 threads per line
using S4096d = Sched<4096, 64, 64, 64, 1, 6>;  // as a, capped at 168 registers (6 blocks per SM)
using S4096e = Sched<4096, 32, 16, 16, 16, 4>; // as c, capped at 128 registers (4 blocks per SM)
using S4096f = Sched<4096, 16, 16, 16, 16, 3>; // as b, capped at 85 registers (3 blocks per SM)
using S4096g = Sched<4096, 64, 16, 16, 16>;    // 64 threads per line, four groups per pass (streamed only)
using S4096h = Sched<4096, 32, 16, 16, 16, 5>; // as c, capped for 5 blocks per SM (streamed)
using S4096i = Sched<4096, 32, 16, 16, 16, 6>; // as c, capped for 6 blocks per SM (streamed)
const SchedDesc kTable[] = {
    make_streamed_desc<S4096c, 1, true, -4>("n4096_e32_r16x16x16_sr1"),
    make_streamed_desc<S4096c, 1, true, -8>("n4096_e32_r16x16x16_sr1_c8"),
    make_streamed_desc<S4096c, 1, true, -16>("n4096_e32_r16x16x16_sr1_c16"),
    make_streamed_desc<S4096c, 1, true, 4>("n4096_e32_r16x16x16_sr1_q4"),
    make_desc<S4096a, 1>("n4096_e64_r64x64_l1"),
    make_desc<S4096a, 2>("n4096_e64_r64x64_l2"),
    make_desc<S4096d, 1>("n4096_e64_r64x64_l1_b6"),
    make_desc<S4096b, 1>("n4096_e16_r16x16x16_l1"),
    make_desc<S4096b, 2>("n4096_e16_r16x16x16_l2"),
    make_desc<S4096c, 1>("n4096_e32_r16x16x16_l1"),
    make_desc<S4096c, 2>("n4096_e32_r16x16x16_l2"),
    make_desc<S4096e, 1>("n4096_e32_r16x16x16_l1_b4"),
    make_desc<S4096f, 1>("n4096_e16_r16x16x16_l1_b3"),
    make_streamed_desc<S4096c, 1, false>("n4096_e32_r16x16x16_s1"),
    make_streamed_desc<S4096c, 2, true>("n4096_e32_r16x16x16_sr2"),
    make_streamed_desc<S4096h, 1, true>("n4096_e32_r16x16x16_sr1_b5"),
    make_streamed_desc<S4096i, 1, true>("n4096_e32_r16x16x16_sr1_b6"),
    make_streamed_desc<S4096g, 1, true, 4>("n4096_e64_r16x16x16_sr1"),
    make_streamed_desc<S4096g, 2, true>("n4096_e64_r16x16x16_sr2"),
    make_streamed_desc<S4096b, 1, false, 4>("n4096_e16_r16x16x16_s1"),
    make_persistent_desc<S4096a>("n4096_e64_r64x64_p"),
    make_persistent_desc<S4096b>("n4096_e16_r16x16x16_p"),
    make_persistent_desc<S4096c>("n4096_e32_r16x16x16_p"),
};
}  // namespace

const SchedDesc *schedules_4096(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
