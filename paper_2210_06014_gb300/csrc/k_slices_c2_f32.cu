// k_slices_c2_f32.cu -- core-pass slice kernel, orders up to 3, C stored as float.
#include "slices_impl.cuh"

namespace sft {

int core_slices_no2_f32(const SliceArgs &g, int R, int J, float *partials, int max_blocks,
                           cudaStream_t st, int sms) {
    int nblk = 1;
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        nblk = core_slices_t<false, 2, decltype(r_c)::value, decltype(j_c)::value, float>(
            g, partials, max_blocks, st, sms);
    });
    return nblk;
}

}  // namespace sft
