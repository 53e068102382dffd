// Line-engine instantiations for N = 8192 (one line per block).
#include "launch.cuh"

namespace sar {
namespace {
using S8192 = Sched<8192, 32, 16, 16, 32>;       // 256 threads per line
using S8192b = Sched<8192, 32, 16, 16, 32, 2>;   // capped at 128 registers: 2 blocks per SM
using S8192c = Sched<8192, 64, 16, 16, 32>;      // 128 threads per line (streamed only)
using S8192d = Sched<8192, 32, 16, 32, 16>;      // 256 threads per line, radix-16 last pass
// first = default: 16 x 32 x 16 (a radix-16 last pass and filter stage)
// measured 11 % faster than the 16 x 16 x 32 schedules
const SchedDesc kTable[] = {
    make_streamed_desc<S8192d, 1, true, -4>("n8192_e32_r16x32x16_sr1"),
    make_streamed_desc<S8192c, 1, true, -4>("n8192_e64_r16x16x32_sr1"),
    make_desc<S8192, 1>("n8192_e32_r16x16x32_l1"),
    make_desc<S8192b, 1>("n8192_e32_r16x16x32_l1_b2"),
    make_persistent_desc<S8192>("n8192_e32_r16x16x32_p"),
    make_streamed_desc<S8192, 1, true, 2>("n8192_e32_r16x16x32_sr1"),
};
}  // namespace

const SchedDesc *schedules_8192(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
