// Line-engine instantiations for N = 4096 (every group live in registers).
#include "launch.cuh"

namespace sar {
namespace {
using S4096a = Sched<4096, 64, 64, 64>;        // 64 threads per line, one exchange per transform
using S4096b = Sched<4096, 16, 16, 16, 16>;    // 256 threads per line, two exchanges per transform
using S4096c = Sched<4096, 32, 16, 16, 16>;    // 128 threads per line
using S4096d = Sched<4096, 64, 64, 64, 1, 6>;  // as a, capped at 168 registers (6 blocks per SM)
using S4096e = Sched<4096, 32, 16, 16, 16, 4>; // as c, capped at 128 registers (4 blocks per SM)
using S4096f = Sched<4096, 16, 16, 16, 16, 3>; // as b, capped at 85 registers (3 blocks per SM)
// Every group of a pass live in registers ("plain"), several geometries.
const SchedDesc kTable[] = {
    make_desc<S4096a, 1>("n4096_e64_r64x64_l1"),
    make_desc<S4096a, 2>("n4096_e64_r64x64_l2"),
    make_desc<S4096d, 1>("n4096_e64_r64x64_l1_b6"),
    make_desc<S4096b, 1>("n4096_e16_r16x16x16_l1"),
    make_desc<S4096b, 2>("n4096_e16_r16x16x16_l2"),
    make_desc<S4096c, 1>("n4096_e32_r16x16x16_l1"),
    make_desc<S4096c, 2>("n4096_e32_r16x16x16_l2"),
    make_desc<S4096e, 1>("n4096_e32_r16x16x16_l1_b4"),
    make_desc<S4096f, 1>("n4096_e16_r16x16x16_l1_b3"),
};
}  // namespace

const SchedDesc *schedules_4096_plain(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
