// k_factor.cu -- SGD pass over a factor matrix A^(n) (Algorithm 4; Eq. (9),
// (10)) in the COO form of cuFasterTucker ("reusable intermediates" only).
//
// Per visited nonzero s (T = R/4 lanes, lane `sub` owns r in [4 sub, 4 sub+4)):
//   p_r   = prod_{k != n} C^(k)[i_k][r]            (Eq. (12), cached rows)
//   v     = B^(n) p                                 (partial over the lane's r,
//                                                     then a reduce-scatter: lane
//                                                     `sub` ends with v_j for its
//                                                     J/T slice of j)
//   e     = x_s - a_{i_n} . v                       (group sum of the slices)
//   term  = e v - lambda a_{i_n}                    (Eq. (10), one slice per lane)
//
// Two ways of applying the terms:
//   hogwild        every nonzero adds lr*term to its row at once with vector
//                  atomics (red.global.add.v4.f32); rows are read through L2
//                  (ld.global.cg) so updates by other SMs are seen promptly.
//   deterministic  minibatch rule: all predictions of a minibatch use the rows
//                  as they stood at its start and the terms of a repeated row
//                  are summed in sample order.  One CTA sorts a chunk of 256
//                  samples by (row, position) in shared memory, computes their
//                  terms in that order and sums each run of equal rows; a second
//                  kernel lets the first chunk holding a row add the other
//                  chunks' sums (found by binary search, in chunk order) and
//                  move the row once.
#include "dispatch.cuh"
#include "sft_internal.cuh"

namespace sft {

constexpr int kFacThreads = 256;

// Gather the cached rows of every mode except a.n and multiply them into p
// (lane's 4 entries).  ik[] holds the coordinates.  Up to four row loads are
// in flight per step.
template <int R>
__device__ __forceinline__ float4 hadamard_others(const PassArgs &a, const int32_t (&ik)[kMaxOrder],
                                                  bool ok, int sub) {
    float4 p = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
    for (int k0 = 0; k0 < kMaxOrder; k0 += 4) {
        if (k0 < a.N) {
            float4 c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + u;
                c[u] = (ok && k < a.N && k != a.n) ? (a.cbf16 ? ldC<__nv_bfloat16>(a.C[k], (int64_t)ik[k] * R + 4 * sub)
                                                              : ldg4(a.C[k] + (int64_t)ik[k] * R + 4 * sub))
                                                   : make_float4(1.f, 1.f, 1.f, 1.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) mul4(p, c[u]);
        }
    }
    return p;
}

// Load the coordinates of sample s and check them against the mode lengths;
// `in` receives the coordinate of the updated mode a.n.
__device__ __forceinline__ bool load_coords(const PassArgs &a, int64_t s, bool ok,
                                            int32_t (&ik)[kMaxOrder], int32_t &in) {
    in = 0;
#pragma unroll
    for (int k = 0; k < kMaxOrder; ++k) {
        ik[k] = 0;
        if (ok && k < a.N) {
            ik[k] = __ldg(a.idx[k] + s);
            if ((uint32_t)ik[k] >= (uint32_t)a.dims[k]) {
                atomicOr(a.err, kErrIndex);
                ok = false;
            }
            if (k == a.n) in = ik[k];
        }
    }
    return ok;
}

// vp[j] = sum over the lane's 4 r of B[j][r] p_r, for every j (B in smem).
template <int R, int J>
__device__ __forceinline__ void core_times_partial(const float *sB, const float4 &p, int sub,
                                                   float (&vp)[J]) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
        vp[j] = fmaf(b.x, p.x, fmaf(b.y, p.y, fmaf(b.z, p.z, b.w * p.w)));
    }
}

// --------------------------------------------------------------------------- Hogwild
template <int R, int J>
__global__ void __launch_bounds__(kFacThreads) k_factor_hogwild(PassArgs a) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int GPW = 32 / T;
    __shared__ __align__(16) float sB[J * R];
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = a.B[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1), gw = lane / T;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * GPW; t0 < a.count; t0 += nwarps * GPW) {
        const int64_t pos = t0 + gw;
        bool ok = pos < a.count;
        int64_t s = 0;
        if (ok) ok = sample_at(a, a.base + pos, s);
        int32_t ik[kMaxOrder], in;
        ok = load_coords(a, s, ok, ik, in);
        const float x = ok ? __ldg(a.val + s) : 0.f;
        const float4 p = hadamard_others<R>(a, ik, ok, sub);
        float *arow = a.A + (int64_t)in * J + sub * JL;
        float av[JL];
#pragma unroll
        for (int q = 0; q < JL; ++q) av[q] = 0.f;
        if (ok) {
            if constexpr (JL >= 4) {
#pragma unroll
                for (int q = 0; q < JL / 4; ++q) {
                    float4 v = __ldcg(reinterpret_cast<const float4 *>(arow + 4 * q));
                    av[4 * q] = v.x; av[4 * q + 1] = v.y; av[4 * q + 2] = v.z; av[4 * q + 3] = v.w;
                }
            } else if constexpr (JL == 2) {
                float2 v = __ldcg(reinterpret_cast<const float2 *>(arow));
                av[0] = v.x; av[1] = v.y;
            } else {
                av[0] = __ldcg(arow);
            }
        }
        float vp[J];
        core_times_partial<R, J>(sB, p, sub, vp);
        group_reduce_scatter<T, J>(vp, sub);
        float dot = 0.f;
#pragma unroll
        for (int q = 0; q < JL; ++q) dot = fmaf(av[q], vp[q], dot);
        const float e = x - group_sum<T>(dot);
        if (ok) {
            float d[JL];
#pragma unroll
            for (int q = 0; q < JL; ++q) d[q] = a.lr * (e * vp[q] - a.lam * av[q]);
            if constexpr (JL >= 4) {
#pragma unroll
                for (int q = 0; q < JL / 4; ++q)
                    atomicAdd(reinterpret_cast<float4 *>(arow + 4 * q),
                              make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]));
            } else if constexpr (JL == 2) {
                atomicAdd(reinterpret_cast<float2 *>(arow), make_float2(d[0], d[1]));
            } else {
                atomicAdd(arow, d[0]);
            }
        }
    }
}

cudaError_t launch_factor_hogwild(const PassArgs &a, int J, int R, cudaStream_t st, int sms) {
    const int64_t per_block = (int64_t)kFacThreads / (R / 4);
    int64_t blocks = (a.count + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    SFT_DISPATCH_RJ(R, J, (k_factor_hogwild<R_, J_><<<(int)blocks, kFacThreads, 0, st>>>(a)));
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- deterministic
// Kernel 1: one CTA per chunk of kDetChunk visit positions of the minibatch
// [a.base, a.base + a.count).
template <int R, int J>
__global__ void __launch_bounds__(kDetChunk) k_factor_det_terms(PassArgs a, DetFactorWs ws) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int GPB = kDetChunk / T;  // lane groups per block
    static_assert(kDetChunk == 256, "one thread per chunk sample");
    __shared__ __align__(16) float sB[J * R];
    __shared__ unsigned long long skey[kDetChunk];
    __shared__ __align__(16) float sterm[kDetChunk * J];
    __shared__ int sstart[kDetChunk];
    __shared__ int swarp[kDetChunk / 32];
    const int t = threadIdx.x;
    const int chunk = blockIdx.x;
    const int64_t c0 = (int64_t)chunk * kDetChunk;
    for (int q = t; q < J * R; q += blockDim.x) sB[q] = a.B[q];

    // keys (row << 32 | local position); invalid positions sort last
    unsigned long long key = ~0ull;
    {
        const int64_t pos = c0 + t;
        int64_t s = 0;
        if (pos < a.count && sample_at(a, a.base + pos, s)) {
            const int32_t row = __ldg(a.idx[a.n] + s);
            if ((uint32_t)row < (uint32_t)a.dims[a.n])
                key = ((unsigned long long)(uint32_t)row << 32) | (unsigned)t;
            else
                atomicOr(a.err, kErrIndex);
        }
    }
    skey[t] = key;
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; k <= kDetChunk; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int ixj = t ^ j;
            if (ixj > t) {
                const unsigned long long x = skey[t], y = skey[ixj];
                const bool up = (t & k) == 0;
                if ((x > y) == up) {
                    skey[t] = y;
                    skey[ixj] = x;
                }
            }
            __syncthreads();
        }
    }

    // terms in sorted order
    const int lane = t & 31;
    const int sub = lane & (T - 1);
    for (int q0 = (t / T); q0 < kDetChunk; q0 += GPB) {
        // q0 is uniform over the T lanes of a group; every group runs the same
        // number of iterations (kDetChunk / GPB), so shuffles stay convergent.
        const unsigned long long kq = skey[q0];
        bool ok = kq != ~0ull;
        int64_t s = 0;
        if (ok) ok = sample_at(a, a.base + c0 + (int64_t)(kq & 0xffffffffu), s);
        int32_t ik[kMaxOrder], in;
        ok = load_coords(a, s, ok, ik, in);
        const float x = ok ? __ldg(a.val + s) : 0.f;
        const float4 p = hadamard_others<R>(a, ik, ok, sub);
        float av[JL];
#pragma unroll
        for (int q = 0; q < JL; ++q) av[q] = 0.f;
        if (ok) load_run<JL>(a.A + (int64_t)in * J + sub * JL, av);
        float vp[J];
        core_times_partial<R, J>(sB, p, sub, vp);
        group_reduce_scatter<T, J>(vp, sub);
        float dot = 0.f;
#pragma unroll
        for (int q = 0; q < JL; ++q) dot = fmaf(av[q], vp[q], dot);
        const float e = x - group_sum<T>(dot);
#pragma unroll
        for (int q = 0; q < JL; ++q)
            sterm[q0 * J + sub * JL + q] = ok ? (e * vp[q] - a.lam * av[q]) : 0.f;
    }
    __syncthreads();

    // runs of equal rows
    const unsigned long long kt = skey[t];
    const bool valid = kt != ~0ull;
    const bool start = valid && (t == 0 || (skey[t - 1] >> 32) != (kt >> 32));
    sstart[t] = start ? 1 : 0;
    const unsigned bal = __ballot_sync(kFull, start);
    if (lane == 0) swarp[t >> 5] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < (t >> 5); ++w) before += swarp[w];
    const int seg = before + __popc(bal & ((1u << lane) - 1));
    if (start) {
        const uint32_t row = (uint32_t)(kt >> 32);
        float acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = sterm[t * J + j];
        for (int q = t + 1; q < kDetChunk; ++q) {
            const unsigned long long kq = skey[q];
            if (kq == ~0ull || (uint32_t)(kq >> 32) != row) break;
#pragma unroll
            for (int j = 0; j < J; ++j) acc[j] += sterm[q * J + j];
        }
        ws.part_row[(int64_t)chunk * kDetChunk + seg] = (int32_t)row;
        float *dst = ws.part_sum + ((int64_t)chunk * kDetChunk + seg) * J;
#pragma unroll
        for (int j = 0; j < J; ++j) dst[j] = acc[j];
    }
    if (t == kDetChunk - 1) {
        int total = 0;
        for (int w = 0; w < kDetChunk / 32; ++w) total += swarp[w];
        ws.seg_count[chunk] = total;
    }
}

__device__ __forceinline__ int find_row(const int32_t *rows, int n, int32_t row) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rows[mid] < row) lo = mid + 1; else hi = mid;
    }
    return (lo < n && rows[lo] == row) ? lo : -1;
}

// Kernel 2: the first chunk that holds a row gathers the other chunks' sums
// for it (chunk order) and moves the row once.
template <int J>
__global__ void __launch_bounds__(kDetChunk) k_factor_det_apply(PassArgs a, DetFactorWs ws,
                                                                int nchunks) {
    const int chunk = blockIdx.x;
    const int q = threadIdx.x;
    if (q >= ws.seg_count[chunk]) return;
    const int32_t row = ws.part_row[(int64_t)chunk * kDetChunk + q];
    for (int c = 0; c < chunk; ++c)
        if (find_row(ws.part_row + (int64_t)c * kDetChunk, ws.seg_count[c], row) >= 0) return;
    float acc[J];
    const float *src = ws.part_sum + ((int64_t)chunk * kDetChunk + q) * J;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = src[j];
    for (int c = chunk + 1; c < nchunks; ++c) {
        const int at = find_row(ws.part_row + (int64_t)c * kDetChunk, ws.seg_count[c], row);
        if (at >= 0) {
            const float *o = ws.part_sum + ((int64_t)c * kDetChunk + at) * J;
#pragma unroll
            for (int j = 0; j < J; ++j) acc[j] += o[j];
        }
    }
    float *arow = a.A + (int64_t)row * J;
#pragma unroll
    for (int j = 0; j < J; ++j) arow[j] = fmaf(a.lr, acc[j], arow[j]);
}

cudaError_t launch_factor_det(const PassArgs &a, int J, int R, const DetFactorWs &ws,
                              cudaStream_t st) {
    const int nchunks = (int)((a.count + kDetChunk - 1) / kDetChunk);
    if (nchunks < 1) return cudaSuccess;
    SFT_DISPATCH_RJ(R, J, (k_factor_det_terms<R_, J_><<<nchunks, kDetChunk, 0, st>>>(a, ws)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (J) {
        case 4: k_factor_det_apply<4><<<nchunks, kDetChunk, 0, st>>>(a, ws, nchunks); break;
        case 8: k_factor_det_apply<8><<<nchunks, kDetChunk, 0, st>>>(a, ws, nchunks); break;
        case 16: k_factor_det_apply<16><<<nchunks, kDetChunk, 0, st>>>(a, ws, nchunks); break;
        case 32: k_factor_det_apply<32><<<nchunks, kDetChunk, 0, st>>>(a, ws, nchunks); break;
        default: break;
    }
    return cudaGetLastError();
}

}  // namespace sft
