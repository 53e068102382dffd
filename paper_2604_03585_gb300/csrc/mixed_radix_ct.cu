// Compile-time specialisations of the mixed-radix fused kernel for common
// three-pass lengths (the runtime kernel serves every other length).  Each
// entry repeats the host geometry of its length (radices, threads per line);
// specialised() hands one out only when they agree.  The register cap (blocks
// per SM) of each is the fastest of 2 ... 5 in a sweep on GB300.
#include "mixed_radix_spec.cuh"

namespace sar {
namespace mixed {

namespace {

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
    return s ? s->launch : specialised_more(g);
}

mixed3_dft_fn specialised_dft(const MixedGeom& g) {
    const Spec* s = find(g);
    return s ? s->launch_dft : specialised_dft_more(g);
}

mixed3_ct_fn specialised_ct(const MixedGeom& g) {
    const Spec* s = find(g);
    return s ? s->launch_ct : specialised_ct_more(g);
}

cudaError_t prepare_specialised() {
    for (const Spec& s : kSpecs) {
        const cudaError_t e = s.attr();
        if (e != cudaSuccess) return e;
    }
    return prepare_specialised_more();
}

}  // namespace mixed
}  // namespace sar
