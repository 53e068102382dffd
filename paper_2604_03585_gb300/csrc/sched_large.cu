// Line-engine instantiations for N = 8192 and 16384 (one line per block).
#include "launch.cuh"

namespace sar {
namespace {
using S8192 = Sched<8192, 32, 16, 16, 32>;     // 256 threads per line
using S16384 = Sched<16384, 32, 16, 32, 32>;   // 512 threads per line, 135 KB shared memory
using S8192b = Sched<8192, 32, 16, 16, 32, 2>;   // capped at 128 registers: 2 blocks per SM
using S8192c = Sched<8192, 64, 16, 16, 32>;      // 128 threads per line (streamed only)
using S16384c = Sched<16384, 64, 16, 32, 32>;    // 256 threads per line (streamed only)
const SchedDesc kTable[] = {
    // first per length = default: 8192 as 16 x 32 x 16 (a radix-16 last pass
    // and filter stage) measured 11 % faster than the 16 x 16 x 32 schedules
    make_streamed_desc<Sched<8192, 32, 16, 32, 16>, 1, true, -4>("n8192_e32_r16x32x16_sr1"),
    make_streamed_desc<S8192c, 1, true, -4>("n8192_e64_r16x16x32_sr1"),
    make_streamed_desc<S16384, 1, true, -4>("n16384_e32_r16x32x32_sr1"),
    make_desc<S8192, 1>("n8192_e32_r16x16x32_l1"),
    make_desc<S8192b, 1>("n8192_e32_r16x16x32_l1_b2"),
    make_desc<S16384, 1>("n16384_e32_r16x32x32_l1"),
    make_persistent_desc<S8192>("n8192_e32_r16x16x32_p"),
    make_streamed_desc<S8192, 1, true, 2>("n8192_e32_r16x16x32_sr1"),
    make_streamed_desc<S16384c, 1, true>("n16384_e64_r16x32x32_sr1"),
    make_streamed_desc<Sched<8192, 32, 32, 16, 16>, 1, true>("n8192_e32_r32x16x16_sr1"),
    make_streamed_desc<Sched<16384, 32, 32, 32, 16>, 1, true>("n16384_e32_r32x32x16_sr1"),
    make_streamed_desc<Sched<16384, 64, 16, 64, 16>, 1, true>("n16384_e64_r16x64x16_sr1"),
};
}  // namespace

const SchedDesc *schedules_large(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
