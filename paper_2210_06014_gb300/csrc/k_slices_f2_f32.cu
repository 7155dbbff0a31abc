// k_slices_f2_f32.cu -- factor-pass slice kernels, orders up to 3, C stored as float.
#include "slices_impl.cuh"

namespace sft {

void factor_slices_no2_f32(const SliceArgs &g, int R, int J, bool with_maps,
                              const SliceStreams &ss, int sms, int64_t *launches) {
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        factor_slices_t<false, 2, decltype(r_c)::value, decltype(j_c)::value, float>(g, with_maps, ss,
                                                                              sms, launches);
    });
}

}  // namespace sft
