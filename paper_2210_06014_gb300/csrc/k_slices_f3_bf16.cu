// k_slices_f3_bf16.cu -- factor-pass slice kernels, orders up to 4, C stored as __nv_bfloat16.
#include "slices_impl.cuh"

namespace sft {

void factor_slices_no3_bf16(const SliceArgs &g, int R, int J, bool with_maps,
                              const SliceStreams &ss, int sms, int64_t *launches) {
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        factor_slices_t<false, 3, decltype(r_c)::value, decltype(j_c)::value, __nv_bfloat16>(g, with_maps, ss,
                                                                              sms, launches);
    });
}

}  // namespace sft
