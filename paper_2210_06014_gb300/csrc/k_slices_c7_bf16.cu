// k_slices_c7_bf16.cu -- core-pass slice kernel, orders up to 8, C stored as __nv_bfloat16.
#include "slices_impl.cuh"

namespace sft {

int core_slices_no7_bf16(const SliceArgs &g, int R, int J, float *partials, int max_blocks,
                           cudaStream_t st, int sms) {
    int nblk = 1;
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        nblk = core_slices_t<false, 7, decltype(r_c)::value, decltype(j_c)::value, __nv_bfloat16>(
            g, partials, max_blocks, st, sms);
    });
    return nblk;
}

}  // namespace sft
