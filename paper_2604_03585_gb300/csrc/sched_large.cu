// Line-engine instantiations for N = 8192 and 16384 (one line per block).
#include "launch.cuh"

namespace sar {
namespace {
using S8192 = Sched<8192, 32, 16, 16, 32>;     // 256 threads per line
using S16384 = Sched<16384, 32, 16, 32, 32>;   // 512 threads per line, 135 KB shared memory
const SchedDesc kTable[] = {
    make_desc<S8192, 1>("n8192_e32_r16x16x32_l1"),
    make_desc<S16384, 1>("n16384_e32_r16x32x32_l1"),
};
}  // namespace

const SchedDesc *schedules_large(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
