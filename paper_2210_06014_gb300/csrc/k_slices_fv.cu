// k_slices_fv.cu -- factor-pass slice kernels that read v from the per-fiber
// table (one instantiation per (R, J); they never touch the cached products).
#include "slices_impl.cuh"

namespace sft {

void factor_slices_fv(const SliceArgs &g, int R, int J, bool with_maps, const SliceStreams &ss,
                      int sms, int64_t *launches) {
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        factor_slices_t<true, 2, decltype(r_c)::value, decltype(j_c)::value, float>(
            g, with_maps, ss, sms, launches);
    });
}

}  // namespace sft
