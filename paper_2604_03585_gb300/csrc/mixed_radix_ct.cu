// Compile-time specialisations of the mixed-radix fused kernel for common
// three-pass lengths (the runtime kernel serves every other length).  Each
// entry repeats the host geometry of its length (radices, threads per line);
// specialised() hands one out only when they agree.  The register cap (blocks
// per SM) of each is the fastest of 2 ... 5 in a sweep on GB300.
#include "mixed_radix.cuh"

namespace sar {
namespace mixed {

namespace {

template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t launch3(const float2* in, float2* out, int64_t n_lines, int64_t ld, const float2* filt, const float2* tw,
                    int, cudaStream_t st) {
    constexpr int LPB = kMixedThreads / T, smem = mixed3_smem<N, T, PD>();
    static_assert(smem <= kMixedSmemMax, "within the shared memory the kernel is set up for");
    fused_mixed3_kernel<N, RA, RB, RC, T, MINB, PD>
        <<<(unsigned)((n_lines + LPB - 1) / LPB), kMixedThreads, smem, st>>>(in, out, n_lines, ld, filt, tw);
    return cudaGetLastError();
}
template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t launch3_dft(const float2* in, float2* out, int64_t n_lines, int64_t ld, int valid, const float2* tw,
                        int pos_off, int inverse, cudaStream_t st) {
    constexpr int LPB = kMixedThreads / T, smem = mixed3_smem<N, T, PD>();
    mixed3_dft_kernel<N, RA, RB, RC, T, MINB, PD><<<(unsigned)((n_lines + LPB - 1) / LPB), kMixedThreads, smem, st>>>(
        in, out, n_lines, ld, valid, tw, pos_off, inverse ? -1.f : 1.f);
    return cudaGetLastError();
}
template <int N, int RA, int RB, int RC, int T, int MINB, int PD>
cudaError_t attr3() {
    cudaError_t e = cudaFuncSetAttribute(fused_mixed3_kernel<N, RA, RB, RC, T, MINB, PD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mixed3_dft_kernel<N, RA, RB, RC, T, MINB, PD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmemMax);
    return e;
}

struct Spec {
    int n, ra, rb, rc, t, minb;
    mixed3_fn launch;
    mixed3_dft_fn launch_dft;
    cudaError_t (*attr)();
};
#define SAR_SPEC(N, RA, RB, RC, T, MB, PD)                                                             \
    Spec{N,  RA, RB, RC, T, MB, &launch3<N, RA, RB, RC, T, MB, PD>, &launch3_dft<N, RA, RB, RC, T, MB, PD>, \
         &attr3<N, RA, RB, RC, T, MB, PD>}
// padding: one slot per 32 positions except at 8000, one per 20 (the last
// radix: its stride-20 groups then fall on distinct bank pairs; simulated
// wavefronts 1.15 x the conflict-free count against 1.83)
const Spec kSpecs[] = {
    SAR_SPEC(1000, 10, 10, 10, 64, 4, 0),  SAR_SPEC(2000, 20, 10, 10, 128, 4, 0),
    SAR_SPEC(3000, 20, 15, 10, 256, 4, 0), SAR_SPEC(4000, 20, 20, 10, 256, 3, 0),
    SAR_SPEC(5000, 25, 20, 10, 256, 3, 0), SAR_SPEC(6000, 20, 20, 15, 256, 3, 0),
    SAR_SPEC(8000, 20, 20, 20, 256, 2, 20),
};
#undef SAR_SPEC

}  // namespace

static const Spec* find(const MixedGeom& g) {
    if (g.P != 3) return nullptr;
    for (const Spec& s : kSpecs)
        if (s.n == g.n && s.ra == g.R[0] && s.rb == g.R[1] && s.rc == g.R[2] && s.t == g.T) return &s;
    return nullptr;
}

mixed3_fn specialised(const MixedGeom& g) {
    const Spec* s = find(g);
    return s ? s->launch : nullptr;
}

mixed3_dft_fn specialised_dft(const MixedGeom& g) {
    const Spec* s = find(g);
    return s ? s->launch_dft : nullptr;
}

cudaError_t prepare_specialised() {
    for (const Spec& s : kSpecs) {
        const cudaError_t e = s.attr();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mixed
}  // namespace sar
