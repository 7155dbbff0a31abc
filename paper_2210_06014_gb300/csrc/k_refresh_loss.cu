// k_refresh_loss.cu -- the cached-product refresh C^(n) = A^(n) B^(n)
// (Algorithm 3) and the residual sums behind RMSE / MAE (Section
// "Real-world accuracy").
//
// Both kernels are bound by HBM bandwidth: the refresh streams A^(n) in and
// C^(n) out (I_n (J_n + R) * 4 bytes, K = J_n <= 32 is far too short for a
// tensor-core tile to pay), the loss streams the COO set and gathers N rows of
// R floats per nonzero.
#include "dispatch.cuh"
#include "sft_internal.cuh"

namespace sft {

// --------------------------------------------------------------------------- refresh
// T = R/4 lanes per row of C; lane `sub` produces C[i][4 sub .. 4 sub + 3]
// from the whole a row (same addresses across the T lanes) and B^(n) staged in
// shared memory.  Grid-stride over rows; stores are float4 and coalesced.
template <int R, int J, typename CT>
__global__ void __launch_bounds__(256) k_refresh(const float *__restrict__ A,
                                                 const float *__restrict__ B,
                                                 float *__restrict__ C, int64_t I) {
    constexpr int T = R / 4;
    __shared__ __align__(16) float sB[J * R];
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = B[q];
    __syncthreads();
    const int sub = threadIdx.x & (T - 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x / T;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / T; row < I;
         row += stride) {
        float a[J];
#pragma unroll
        for (int q = 0; q < J / 4; ++q) {
            float4 v = ldg4(A + row * J + 4 * q);
            a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
        }
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
            c.x = fmaf(a[j], b.x, c.x);
            c.y = fmaf(a[j], b.y, c.y);
            c.z = fmaf(a[j], b.z, c.z);
            c.w = fmaf(a[j], b.w, c.w);
        }
        stC<CT>(C, row * R + 4 * sub, c);
    }
}

cudaError_t launch_refresh(const float *A, const float *B, float *C, int64_t I, int J, int R,
                           bool cbf16, cudaStream_t st, int sms) {
    const int threads = 256;
    const int64_t rows_per_block = threads / (R / 4);
    int64_t blocks = (I + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (cbf16)
        SFT_DISPATCH_RJ(R, J, (k_refresh<R_, J_, __nv_bfloat16><<<(int)blocks, threads, 0, st>>>(A, B, C, I)));
    else
        SFT_DISPATCH_RJ(R, J, (k_refresh<R_, J_, float><<<(int)blocks, threads, 0, st>>>(A, B, C, I)));
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- loss
// T = R/4 lanes per nonzero, GPW = 32/T nonzeros per warp per step.  Block b
// owns a contiguous span of the set; its warps walk the span in a fixed
// interleave and every lane keeps float64 sums, reduced in a fixed order, so
// the result is bitwise reproducible for a given grid size.
constexpr int kLossThreads = 256;

// NO: a compile-time bound on the order (the rows of a nonzero are held in
// registers, NO float4 per lane).  A group's nonzeros are a two-level
// pipeline: the coordinates of the nonzero after next and the cached rows of
// the next one are in flight while the current one is formed.
template <int R, typename CT, int NO>
__global__ void __launch_bounds__(kLossThreads) k_loss(PassArgs a, double *__restrict__ partials) {
    constexpr int T = R / 4;
    constexpr int GPW = 32 / T;
    constexpr int WARPS = kLossThreads / 32;
    constexpr int64_t STEP = (int64_t)WARPS * GPW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    const int64_t span = (a.count + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = (int64_t)blockIdx.x * span;
    const int64_t p1 = min(a.count, p0 + span);
    double s2 = 0.0, s1 = 0.0;
    struct Coords {
        int32_t ik[NO];
        float x;
        bool ok;
    };
    struct Rows {
        float4 c[NO];
        float x;
        bool ok;
    };
    auto fetch = [&](int64_t pos, Coords &nx) {
        nx.ok = pos < p1;
        int64_t s = 0;
        if (nx.ok) nx.ok = sample_at(a, a.base + pos, s);
#pragma unroll
        for (int k = 0; k < NO; ++k) nx.ik[k] = (nx.ok && k < a.N) ? __ldg(a.idx[k] + s) : 0;
        nx.x = nx.ok ? __ldg(a.val + s) : 0.f;
    };
    // checks a nonzero's coordinates (they have arrived) and issues its row gathers
    auto gather = [&](const Coords &cd, Rows &rw) {
        bool ok = cd.ok;
#pragma unroll
        for (int k = 0; k < NO; ++k)
            if (ok && k < a.N && (uint32_t)cd.ik[k] >= (uint32_t)a.dims[k]) {
                atomicOr(a.err, kErrIndex);
                ok = false;
            }
#pragma unroll
        for (int k = 0; k < NO; ++k)
            rw.c[k] = (ok && k < a.N) ? ldC<CT>(a.C[k], (int64_t)cd.ik[k] * R + 4 * sub)
                                      : make_float4(1.f, 1.f, 1.f, 1.f);
        rw.ok = ok;
        rw.x = ok ? cd.x : 0.f;
    };
    const int64_t q0 = p0 + (int64_t)warp * GPW + gw;
    Coords c1, c2;
    Rows cur;
    fetch(q0, c1);
    fetch(q0 + STEP, c2);
    gather(c1, cur);
    for (int64_t t0 = p0 + (int64_t)warp * GPW; t0 < p1; t0 += STEP) {
        const int64_t q = t0 + gw;
        Coords c3;
        fetch(q + 2 * STEP, c3);
        Rows nx;
        gather(c2, nx);
        float4 p = make_float4(cur.ok ? 1.f : 0.f, cur.ok ? 1.f : 0.f, cur.ok ? 1.f : 0.f,
                               cur.ok ? 1.f : 0.f);
#pragma unroll
        for (int k = 0; k < NO; ++k) mul4(p, cur.c[k]);
        const bool ok = cur.ok;
        const float x = cur.x;
        cur = nx;
        c2 = c3;
        const float xh = group_sum<T>((p.x + p.y) + (p.z + p.w));
        if (ok && sub == 0) {
            const double e = (double)x - (double)xh;
            s2 += e * e;
            s1 += fabs(e);
        }
    }
    // fixed-order reduction: warp tree, then warps in index order
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        s2 += __shfl_xor_sync(kFull, s2, w);
        s1 += __shfl_xor_sync(kFull, s1, w);
    }
    __shared__ double red[WARPS][2];
    if (lane == 0) {
        red[warp][0] = s2;
        red[warp][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t2 = 0.0, t1 = 0.0;
        for (int w = 0; w < WARPS; ++w) {
            t2 += red[w][0];
            t1 += red[w][1];
        }
        partials[2 * blockIdx.x] = t2;
        partials[2 * blockIdx.x + 1] = t1;
    }
}

__global__ void k_loss_final(const double *__restrict__ partials, int nblk, double *out2) {
    // one warp: lane-strided sums, then a fixed tree
    const int lane = threadIdx.x;
    double t2 = 0.0, t1 = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        t2 += partials[2 * b];
        t1 += partials[2 * b + 1];
    }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        t2 += __shfl_xor_sync(kFull, t2, w);
        t1 += __shfl_xor_sync(kFull, t1, w);
    }
    if (lane == 0) {
        out2[0] = t2;
        out2[1] = t1;
    }
}

int loss_blocks_for(int64_t count, int sms) {
    int64_t b = (count + 1023) / 1024;
    const int64_t cap = (int64_t)sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_loss(const PassArgs &a, int R, double *partials, int nblk, double *out2,
                        cudaStream_t st) {
    auto run = [&](auto no_c) {
        constexpr int NO = decltype(no_c)::value;
        if (a.cbf16)
            SFT_DISPATCH_R(R, (k_loss<R_, __nv_bfloat16, NO><<<nblk, kLossThreads, 0, st>>>(a, partials)));
        else
            SFT_DISPATCH_R(R, (k_loss<R_, float, NO><<<nblk, kLossThreads, 0, st>>>(a, partials)));
    };
    if (a.N <= 3) run(ic<3>{});
    else if (a.N <= 4) run(ic<4>{});
    else if (a.N <= 8) run(ic<8>{});
    else run(ic<kMaxOrder>{});
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_loss_final<<<1, 32, 0, st>>>(partials, nblk, out2);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- predict
template <int R, typename CT>
__global__ void __launch_bounds__(kLossThreads) k_predict(PassArgs a, float *__restrict__ out) {
    constexpr int T = R / 4;
    constexpr int GPW = 32 / T;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1), gw = lane / T;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * GPW; t0 < a.count; t0 += nwarps * GPW) {
        const int64_t s = t0 + gw;
        bool ok = s < a.count;
        int32_t ik[kMaxOrder];
#pragma unroll
        for (int k = 0; k < kMaxOrder; ++k) {
            ik[k] = 0;
            if (ok && k < a.N) {
                ik[k] = __ldg(a.idx[k] + s);
                if ((uint32_t)ik[k] >= (uint32_t)a.dims[k]) {
                    atomicOr(a.err, kErrIndex);
                    ok = false;
                }
            }
        }
        float4 p = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
        for (int k0 = 0; k0 < kMaxOrder; k0 += 4) {
            if (k0 < a.N) {
                float4 c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + u;
                    c[u] = (ok && k < a.N) ? ldC<CT>(a.C[k], (int64_t)ik[k] * R + 4 * sub)
                                           : make_float4(1.f, 1.f, 1.f, 1.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) mul4(p, c[u]);
            }
        }
        const float xh = group_sum<T>((p.x + p.y) + (p.z + p.w));
        if (s < a.count && sub == 0) out[s] = ok ? xh : __int_as_float(0x7fc00000);
    }
}

cudaError_t launch_predict(const PassArgs &a, int R, float *out, cudaStream_t st, int sms) {
    const int64_t per_block = (int64_t)kLossThreads / (R / 4);
    int64_t blocks = (a.count + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (a.cbf16)
        SFT_DISPATCH_R(R, (k_predict<R_, __nv_bfloat16><<<(int)blocks, kLossThreads, 0, st>>>(a, out)));
    else
        SFT_DISPATCH_R(R, (k_predict<R_, float><<<(int)blocks, kLossThreads, 0, st>>>(a, out)));
    return cudaGetLastError();
}

}  // namespace sft
