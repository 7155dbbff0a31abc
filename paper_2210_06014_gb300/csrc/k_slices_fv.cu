// k_slices_fv.cu -- slice kernels that read v (factor pass) or p (core pass)
// from the per-fiber tables (one instantiation per (R, J); they never touch the
// cached products).  The bfloat16 v table's kernels are in k_slices_fv_bf16.cu.
#include "slices_impl.cuh"

namespace sft {

void factor_slices_fv(const SliceArgs &g, int R, int J, bool vbf16, bool with_maps,
                      const SliceStreams &ss, int sms, int64_t *launches) {
    if (vbf16) {
        factor_slices_fv_bf16(g, R, J, with_maps, ss, sms, launches);
        return;
    }
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        factor_slices_t<true, 2, decltype(r_c)::value, decltype(j_c)::value, float>(
            g, with_maps, ss, sms, launches);
    });
}

int core_slices_fv(const SliceArgs &g, int R, int J, float *partials, int max_blocks,
                   cudaStream_t st, int sms) {
    int nblk = 1;
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        nblk = core_slices_t<true, 2, decltype(r_c)::value, decltype(j_c)::value, float>(
            g, partials, max_blocks, st, sms);
    });
    return nblk;
}

}  // namespace sft
