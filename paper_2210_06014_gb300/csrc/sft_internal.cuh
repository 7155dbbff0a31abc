// sft_internal.cuh -- kernel argument blocks, launch entry points and small
// device helpers shared by the CUDA translation units of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sft.h"

namespace sft {

constexpr int kMaxOrder = SFT_MAX_ORDER;
constexpr unsigned kFull = 0xffffffffu;

// Error flag bits raised by kernels (device int in the workspace).
constexpr int kErrIndex = 1;  // coordinate out of range
constexpr int kErrPerm = 2;   // permutation entry >= nnz
constexpr int kErrWait = 4;   // a bounded wait ran out (tensor-core kernels, batched runner)

// Operands of one pass over the nonzeros of mode n.
struct PassArgs {
    const int32_t *idx[kMaxOrder];  // idx[k][s]
    const float *C[kMaxOrder];      // cached products C^(k), I_k x R
    int32_t dims[kMaxOrder];        // I_k
    int N;                          // order
    int n;                          // mode being updated
    const float *val;               // x_s
    const uint32_t *perm;           // visit order (NULL = storage order)
    int64_t nnz;                    // samples in the whole pass (perm length)
    int64_t base;                   // first visit position of this launch
    int64_t count;                  // visit positions handled by this launch
    float *A;                       // A^(n), I_n x J_n
    float *B;                       // B^(n), J_n x R
    float lr, lam;
    int *err;                       // device error flag
    int cbf16;                      // cached products C^(k) are stored as bfloat16
    // the N-1 modes other than n, in ascending order (set when n >= 0)
    const int32_t *oidx[kMaxOrder];
    const float *oC[kMaxOrder];
    int32_t odims[kMaxOrder];
    // bit q: other mode q's cached-product table is at most kL1TableBytes and
    // its rows are gathered through L1; the rows of larger tables are read
    // from L2 only
    uint32_t ol1;
};

// The slice walks and the fiber table gather one random cached row per other
// mode and position.  Rows of float32 tables with R <= 16 (64-byte rows)
// larger than kL1TableBytes are loaded with ld.global.cg (L2 only), which
// measured faster there than the non-coherent L1 path; bfloat16 tables,
// 128-byte rows (R = 32) and small tables measured faster on the L1 path and
// stay on it.
#ifndef SFT_L1_TABLE_BYTES
#define SFT_L1_TABLE_BYTES (64 * 1024)
#endif
constexpr int64_t kL1TableBytes = SFT_L1_TABLE_BYTES;

inline bool l2_only_rows(int64_t rows, int R, int cbf16) {
    return !cbf16 && R <= 16 && rows * R * 4 > kL1TableBytes;
}

// Workspace pieces used by the deterministic factor path.
struct DetFactorWs {
    int32_t *part_row;   // [chunks][kDetChunk]
    float *part_sum;     // [chunks][kDetChunk][J]
    int32_t *seg_count;  // [chunks]
};

constexpr int kDetChunk = 256;           // samples per CTA in the deterministic factor path
constexpr int64_t kDetMaxBatch = 16384;  // largest deterministic factor minibatch

// ----------------------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after enqueuing.  J and R are validated by
// the caller (sft_api.cu) against the supported set.
cudaError_t launch_refresh(const float *A, const float *B, float *C, int64_t I, int J, int R,
                           bool cbf16, cudaStream_t st, int sms);
cudaError_t launch_factor_hogwild(const PassArgs &a, int J, int R, cudaStream_t st, int sms);
cudaError_t launch_factor_det(const PassArgs &a, int J, int R, const DetFactorWs &ws,
                              cudaStream_t st);
cudaError_t launch_core(const PassArgs &a, int J, int R, float *partials, int nblk,
                        cudaStream_t st);
int core_blocks_for(int64_t count, int sms);
// tensor-core (tcgen05) forms of the refresh and the minibatch core gradient
// for bfloat16 cached products (k_tc.cu)
bool refresh_tc_supported(int J, int R);
// wait_ns: time limit of the kernels' waits on their own copies and MMAs
// (0: give up at once); the drain after an expired wait keeps a 2 s bound.
cudaError_t launch_refresh_tc(const float *A, const float *B, void *C, int64_t I, int J, int R,
                              int *err, uint64_t wait_ns, cudaStream_t st, int sms);
bool core_tc_supported(int J, int R);
cudaError_t launch_core_tc(const PassArgs &a, int J, int R, float *partials, int nblk,
                           uint64_t wait_ns, cudaStream_t st);
cudaError_t launch_core_apply(float *B, const float *partials, int nblk, int JR, int64_t Mb,
                              float lr, float lam, cudaStream_t st);
// Streams of one slice factor pass: `tiles` is the caller's stream; `chains`
// and `maps` may be auxiliary streams forked from it (or the same stream).
struct SliceStreams {
    cudaStream_t tiles, chains, maps;
    cudaEvent_t fork, chains_done, maps_done;  // NULL events: no fork/join
};
// slice (CSF) layout and the passes over it
int64_t slice_sort_length(int64_t nnz);
size_t slice_maps_bytes(int64_t ntiles, int J);
size_t slice_chain_list_offset(int64_t ntiles, int J);
size_t slice_piece_list_offset(int64_t ntiles, int J);
size_t slice_combine_list_offset(int64_t ntiles, int J);
size_t slice_lane_list_offset(int64_t ntiles, int J);
size_t slice_workspace_total(int64_t ntiles, int J, int64_t In);
// the fiber factor pass runs its tiles and short chains with the one-lane
// kernel (k_slices_lanes) when J_n <= 16
constexpr bool slice_lane_kernels(int J) { return J <= 16; }
int slice_tile_length(int64_t nnz, int sms);
int slice_core_tile_length(int64_t nnz, int sms);
cudaError_t launch_expand_rows(const int32_t *row_ptr, int32_t In, int64_t nnz, int32_t *out,
                               cudaStream_t st, int sms);
cudaError_t launch_group_slices(const PassArgs &a, int32_t *const *out_idx, float *out_val,
                                int32_t *row_ptr, unsigned long long *keys, cudaStream_t st,
                                int sms, int64_t *launches);
cudaError_t launch_factor_slices(const PassArgs &a, const int32_t *row_ptr, int64_t W, int64_t Lseq,
                                 bool subslices, bool gram, float *maps, int J, int R, const SliceStreams &ss, int sms,
                                 int64_t *launches);
cudaError_t launch_core_slices(const PassArgs &a, const int32_t *row_ptr, int64_t W, int J, int R,
                               float *partials, int max_blocks, cudaStream_t st, int sms,
                               int64_t *launches);
cudaError_t launch_loss(const PassArgs &a, int R, double *partials, int nblk, double *out2,
                        cudaStream_t st);
int loss_blocks_for(int64_t count, int sms);
cudaError_t launch_predict(const PassArgs &a, int R, float *out, cudaStream_t st, int sms);
// fibers of a slice layout and the factor pass that shares v per fiber (k_fibers.cu)
int64_t fiber_table_capacity(int64_t nnz);
cudaError_t launch_group_fibers(const PassArgs &a, int32_t *fid, int32_t *const *fcoord,
                                void *scratch, int64_t *nfibers, cudaStream_t st, int sms,
                                int64_t *launches);
bool fiber_v_bf16(const PassArgs &a, int J, int R);
cudaError_t launch_fiber_expand(int N, int mode, const int32_t *fid, int64_t nnz, int64_t nfibers,
                                const int32_t *const *fcoord, int32_t *const *out_idx,
                                cudaStream_t st, int sms);
cudaError_t launch_factor_fibers(const PassArgs &a, const int32_t *row_ptr, int64_t W, int64_t Lseq,
                                 bool subslices, bool gram, float *maps, const int32_t *fid, const int32_t *const *fcoord,
                                 int64_t nfibers, float *V, int J, int R, const SliceStreams &ss,
                                 int sms, int64_t *launches);
cudaError_t launch_core_fibers(const PassArgs &a, const int32_t *row_ptr, int64_t W,
                               const int32_t *fid, const int32_t *const *fcoord, int64_t nfibers,
                               float *P,
                               int J, int R, float *partials, int max_blocks, cudaStream_t st,
                               int sms, int64_t *launches, bool fill_p);
// gradient of the sampled loss (k_grad.cu)
struct GradBufs {
    float *dC[kMaxOrder];   // dL/dC^(k), I_k x R float32
    int64_t dims[kMaxOrder];
};
cudaError_t launch_loss_grad(const PassArgs &a, const GradBufs &g, int R, bool accumulate,
                             double *partials, int nblk, double *out, cudaStream_t st, int sms,
                             int64_t *launches);
cudaError_t launch_grad_project(const float *A, const float *B, const float *dC, int64_t I, int J,
                                int R, const double *scale, float *gA, float *gB, float *partials,
                                int max_blocks, cudaStream_t st, int sms, int64_t *launches);

// ----------------------------------------------------------------------------- device helpers
#ifdef __CUDACC__

__device__ __forceinline__ float4 ldg4(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
}

__device__ __forceinline__ float4 ld4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ void mul4(float4 &a, const float4 &b) {
    a.x *= b.x; a.y *= b.y; a.z *= b.z; a.w *= b.w;
}

// Visit position -> storage index, with the permutation bound check.
__device__ __forceinline__ bool sample_at(const PassArgs &a, int64_t pos, int64_t &s) {
    if (a.perm) {
        uint32_t q = __ldg(a.perm + pos);
        if ((int64_t)q >= a.nnz) {
            atomicOr(a.err, kErrPerm);
            return false;
        }
        s = q;
    } else {
        s = pos;
    }
    return true;
}

// Four consecutive cached-product entries starting at element `off` of a C
// array stored as CT (float or bfloat16), widened to float (bf16 -> f32 is
// exact: the bf16 bits are the top half of the f32).
template <typename CT>
__device__ __forceinline__ float4 ldC(const float *base, int64_t off);

template <>
__device__ __forceinline__ float4 ldC<float>(const float *base, int64_t off) {
    return ldg4(base + off);
}

template <>
__device__ __forceinline__ float4 ldC<__nv_bfloat16>(const float *base, int64_t off) {
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(
        reinterpret_cast<const __nv_bfloat16 *>(base) + off));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

// The raw form of four cached-product entries as loaded (float4, or four
// bfloat16 in a uint2) and its widening to float; walks keep the raw form in
// their prefetch rings so that no instruction waits on a gather until the
// value is used.
template <typename CT>
struct CRaw;
template <>
struct CRaw<float> {
    using type = float4;
};
template <>
struct CRaw<__nv_bfloat16> {
    using type = uint2;
};

template <typename CT>
__device__ __forceinline__ typename CRaw<CT>::type ldC_raw(const float *base, int64_t off);

template <>
__device__ __forceinline__ float4 ldC_raw<float>(const float *base, int64_t off) {
    return ldg4(base + off);
}

template <>
__device__ __forceinline__ uint2 ldC_raw<__nv_bfloat16>(const float *base, int64_t off) {
    return __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(base) + off));
}

#ifndef SFT_L1_HINT
#define SFT_L1_HINT 1
#endif

// ldC_raw with the table's cache policy: l1 = through L1 (ld.global.nc), else
// L2 only (ld.global.cg).  The same bits either way.
template <typename CT>
__device__ __forceinline__ typename CRaw<CT>::type ldC_raw_l1(const float *base, int64_t off,
                                                              bool l1);

template <>
__device__ __forceinline__ float4 ldC_raw_l1<float>(const float *base, int64_t off, bool l1) {
    const float4 *p = reinterpret_cast<const float4 *>(base + off);
    return (l1 || !SFT_L1_HINT) ? __ldg(p) : __ldcg(p);
}

template <>
__device__ __forceinline__ uint2 ldC_raw_l1<__nv_bfloat16>(const float *base, int64_t off, bool l1) {
    const uint2 *p = reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(base) + off);
    return (l1 || !SFT_L1_HINT) ? __ldg(p) : __ldcg(p);
}

template <typename CT>
__device__ __forceinline__ typename CRaw<CT>::type c_one();

template <>
__device__ __forceinline__ float4 c_one<float>() {
    return make_float4(1.f, 1.f, 1.f, 1.f);
}

template <>
__device__ __forceinline__ uint2 c_one<__nv_bfloat16>() {
    return make_uint2(0x3f803f80u, 0x3f803f80u);  // four bfloat16 ones
}

__device__ __forceinline__ float4 widen(const float4 &v) { return v; }

__device__ __forceinline__ float4 widen(const uint2 &u) {
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

// Stores four floats as CT at element `off` (bf16: round to nearest even).
template <typename CT>
__device__ __forceinline__ void stC(float *base, int64_t off, float4 v);

template <>
__device__ __forceinline__ void stC<float>(float *base, int64_t off, float4 v) {
    *reinterpret_cast<float4 *>(base + off) = v;
}

template <>
__device__ __forceinline__ void stC<__nv_bfloat16>(float *base, int64_t off, float4 v) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t *>(&lo);
    u.y = *reinterpret_cast<const uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(base) + off) = u;
}

// Load a run of L consecutive floats (L in {1,2,4,8,...}) from a 4L-byte
// aligned address into registers.
template <int L>
__device__ __forceinline__ void load_run(const float *p, float (&r)[L]) {
    if constexpr (L >= 4) {
#pragma unroll
        for (int q = 0; q < L / 4; ++q) {
            float4 v = ld4(p + 4 * q);
            r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
        }
    } else if constexpr (L == 2) {
        float2 v = *reinterpret_cast<const float2 *>(p);
        r[0] = v.x; r[1] = v.y;
    } else {
        r[0] = *p;
    }
}

// Lane mask of the aligned T-lane group that contains `lane`.
template <int T>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if constexpr (T == 32) return kFull;
    else return ((1u << T) - 1u) << (lane & ~(T - 1));
}

// Group sum with an explicit member mask (groups of a warp may diverge).
template <int T>
__device__ __forceinline__ float group_sum_m(float x, unsigned m) {
#pragma unroll
    for (int w = T / 2; w >= 1; w >>= 1) x += __shfl_xor_sync(m, x, w);
    return x;
}

template <int T, int L>
__device__ __forceinline__ void group_reduce_scatter_m(float (&v)[L], int sub, unsigned m) {
#pragma unroll
    for (int w = T / 2; w >= 1; w >>= 1) {
        const int len = (L / T) * 2 * w;
        const bool upper = (sub & w) != 0;
#pragma unroll
        for (int q = 0; q < L / 2; ++q) {
            if (q < len / 2) {
                float send = upper ? v[q] : v[q + len / 2];
                float keep = upper ? v[q + len / 2] : v[q];
                float recv = __shfl_xor_sync(m, send, w);
                v[q] = keep + recv;
            }
        }
    }
}

// Sum over the T lanes of an aligned lane group (T a power of two <= 32).
template <int T>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
    for (int w = T / 2; w >= 1; w >>= 1) x += __shfl_xor_sync(kFull, x, w);
    return x;
}

// Reduce-scatter over the T lanes of a group: on entry every lane holds a
// partial vector v[0..L); on exit lane `sub` holds, in v[0..L/T), the full sum
// of elements [sub*L/T, (sub+1)*L/T).
template <int T, int L>
__device__ __forceinline__ void group_reduce_scatter(float (&v)[L], int sub) {
#pragma unroll
    for (int w = T / 2; w >= 1; w >>= 1) {
        const int len = (L / T) * 2 * w;  // current range length
        const bool upper = (sub & w) != 0;
#pragma unroll
        for (int q = 0; q < L / 2; ++q) {
            if (q < len / 2) {
                float send = upper ? v[q] : v[q + len / 2];
                float keep = upper ? v[q + len / 2] : v[q];
                float recv = __shfl_xor_sync(kFull, send, w);
                v[q] = keep + recv;
            }
        }
    }
}

#endif  // __CUDACC__

}  // namespace sft
