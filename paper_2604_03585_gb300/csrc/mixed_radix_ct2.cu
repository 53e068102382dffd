// More compiled three-pass lengths of the mixed-radix kernels (a second
// translation unit so that the two compile in parallel): round lengths
// between 1200 and 7500 with their host geometry (radices, threads per line)
// and the register cap of their length class (4 blocks per SM up to 4096, 3
// up to 6000, 2 above).
#include "mixed_radix_spec.cuh"

namespace sar {
namespace mixed {

namespace {

const Spec kMore[] = {
    SAR_SPEC(1200, 12, 10, 10, 64, 4, 0),  SAR_SPEC(1500, 15, 10, 10, 128, 4, 0),
    SAR_SPEC(1600, 16, 10, 10, 128, 4, 0), SAR_SPEC(2400, 16, 15, 10, 128, 4, 0),
    SAR_SPEC(2500, 25, 10, 10, 128, 4, 0), SAR_SPEC(3200, 20, 16, 10, 256, 4, 0),
    SAR_SPEC(3500, 25, 14, 10, 256, 4, 0), SAR_SPEC(4500, 20, 15, 15, 256, 3, 0),
    SAR_SPEC(4800, 20, 16, 15, 256, 3, 0), SAR_SPEC(6400, 20, 20, 16, 256, 2, 0),
    SAR_SPEC(7000, 25, 20, 14, 256, 2, 0), SAR_SPEC(7200, 32, 15, 15, 256, 2, 0),
    SAR_SPEC(7500, 25, 20, 15, 256, 2, 0),
};

const Spec* find_more(const MixedGeom& g) {
    if (g.P != 3) return nullptr;
    for (const Spec& s : kMore)
        if (s.n == g.n && s.ra == g.R[0] && s.rb == g.R[1] && s.rc == g.R[2] && s.t == g.T) return &s;
    return nullptr;
}

}  // namespace

mixed3_fn specialised_more(const MixedGeom& g) {
    const Spec* s = find_more(g);
    return s ? s->launch : nullptr;
}

mixed3_dft_fn specialised_dft_more(const MixedGeom& g) {
    const Spec* s = find_more(g);
    return s ? s->launch_dft : nullptr;
}

mixed3_ct_fn specialised_ct_more(const MixedGeom& g) {
    const Spec* s = find_more(g);
    return s ? s->launch_ct : nullptr;
}

cudaError_t prepare_specialised_more() {
    for (const Spec& s : kMore) {
        const cudaError_t e = s.attr();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mixed
}  // namespace sar
