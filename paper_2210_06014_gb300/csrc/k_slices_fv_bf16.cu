// k_slices_fv_bf16.cu -- the factor-pass slice kernels reading a bfloat16 v
// table (cached products stored as bfloat16, J_n >= max(8, R/2)); in the fiber
// kernels the element-type parameter is the type of v.
#include "slices_impl.cuh"

namespace sft {

void factor_slices_fv_bf16(const SliceArgs &g, int R, int J, bool with_maps,
                           const SliceStreams &ss, int sms, int64_t *launches) {
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        constexpr int R_ = decltype(r_c)::value, J_ = decltype(j_c)::value;
        if constexpr (J_ >= 8 && J_ / (R_ / 4) >= 2)
            factor_slices_t<true, 2, R_, J_, __nv_bfloat16>(g, with_maps, ss, sms, launches);
    });
}

}  // namespace sft
