// Line-engine instantiations for N = 256 ... 2048 (several lines per block).
#include "launch.cuh"

namespace sar {
namespace {
using S256 = Sched<256, 16, 16, 16>;     // 16 threads per line
using S512 = Sched<512, 32, 16, 32>;     // 16 threads per line
using S1024 = Sched<1024, 32, 32, 32>;   // one warp per line
using S2048 = Sched<2048, 64, 32, 64>;   // one warp per line
using S256b = Sched<256, 16, 16, 16>;
using S512b = Sched<512, 16, 16, 8, 4>;       // 32 threads per line, three passes
using S1024b = Sched<1024, 16, 16, 16, 4>;    // 64 threads per line
using S2048b = Sched<2048, 16, 16, 16, 8>;    // 128 threads per line
using S2048c = Sched<2048, 16, 16, 8, 16>;    // 128 threads per line, last radix 16: minimum wavefronts
using S2048d = Sched<2048, 32, 16, 8, 16>;    // 64 threads per line
// The first schedule of a length is its default (and the first one with a
// folded corner turn the default of the fold): for 2048 the 16 x 8 x 16
// geometry, whose every pass takes the minimum two wavefronts per warp access
// (16 x 16 x 8 takes four in its first two passes).
const SchedDesc kTable[] = {
    make_desc<S2048c, 1>("n2048_e16_r16x8x16_l1"),
    make_streamed_desc<S2048d, 2, true, -4>("n2048_e32_r16x8x16_sr2"),
    make_streamed_desc<S2048c, 1, false, -4>("n2048_e16_r16x8x16_s1"),
    make_streamed_desc<S2048c, 2, false>("n2048_e16_r16x8x16_s2"),
    make_streamed_desc<S2048d, 4, true>("n2048_e32_r16x8x16_sr4"),
    make_streamed_desc<S2048b, 1, false, -4>("n2048_e16_r16x16x8_s1"),
    make_desc<S256, 8>("n256_e16_r16x16_l8"),
    make_desc<S256b, 16>("n256_e16_r16x16_l16"),
    make_desc<S512, 8>("n512_e32_r16x32_l8"),
    make_desc<S512b, 4>("n512_e16_r16x8x4_l4"),
    make_desc<S1024, 4>("n1024_e32_r32x32_l4"),
    make_desc<S1024b, 2>("n1024_e16_r16x16x4_l2"),
    make_desc<S2048, 2>("n2048_e64_r32x64_l2"),
    make_desc<S2048b, 1>("n2048_e16_r16x16x8_l1"),
    make_streamed_desc<S1024, 4, false, 4>("n1024_e32_r32x32_s4"),
    make_streamed_desc<S512, 8, false, 4>("n512_e32_r16x32_s8"),
    make_streamed_desc<S256, 8, false, 4>("n256_e16_r16x16_s8"),
    make_streamed_desc<S2048b, 2, false>("n2048_e16_r16x16x8_s2"),
    make_persistent_desc<S2048>("n2048_e64_r32x64_p"),
    make_persistent_desc<S2048b>("n2048_e16_r16x16x8_p"),
    make_persistent_desc<S1024>("n1024_e32_r32x32_p"),
    make_persistent_desc<S1024b>("n1024_e16_r16x16x4_p"),
};
}  // namespace

const SchedDesc *schedules_small(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace sar
