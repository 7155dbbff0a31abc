// k_core.cu -- SGD pass over a core matrix B^(n) (Algorithm 5; Eq. (9), (11)).
//
// Per minibatch the gradient is the contraction
//   G = sum_s e_s a_{i_n(s)} p_s^T        (J_n x M) . (M x R)
// with p_s the Hadamard product of the other modes' cached rows and
// e_s = x_s - a . (B^(n) p_s) taken with B^(n) as it stood at the start of the
// minibatch (Algorithm 5 accumulates first and updates "uniformly" at the end).
//
// Kernel 1 (k_core_grad): lane groups of T = R/4 lanes compute p, e and the
// slices of e*a; each warp stages its GPW samples in shared memory and folds
// them into a warp-private G tile with FFMA (lane = column r, a run of rows).
// A block owns a contiguous span of the minibatch and writes one partial tile;
// everything is summed in a fixed order, so results are bitwise reproducible.
// Kernel 2 (k_core_apply): sums the block partials in a fixed order (float64)
// and applies B += lr (G / M_b - lambda B).
//
// This CUDA-core form is exact in float32 (the float32 parity mode).  With
// bfloat16 cached products and R in {16, 32}, sft_update_core uses the
// tensor-core form of the same contraction instead (k_core_grad_tc, k_tc.cu).
#include "dispatch.cuh"
#include "sft_internal.cuh"

namespace sft {

constexpr int kCoreThreads = 256;
constexpr int kCoreWarps = kCoreThreads / 32;

template <int R, int J>
__global__ void __launch_bounds__(kCoreThreads) k_core_grad(PassArgs a, float *__restrict__ partials) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int GPW = 32 / T;
    constexpr int JR = J * R;
    constexpr int EPL = JR >= 32 ? JR / 32 : 1;  // G entries per lane
    constexpr int STAGE = kCoreWarps * GPW * (J + R);
    constexpr int RED = kCoreWarps * JR;
    constexpr int SMEM = STAGE > RED ? STAGE : RED;
    __shared__ __align__(16) float sB[JR];
    __shared__ __align__(16) float sbuf[SMEM];  // staging during the loop, reduction after
    for (int q = threadIdx.x; q < JR; q += blockDim.x) sB[q] = a.B[q];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    float *sea = sbuf + warp * GPW * (J + R);  // [GPW][J]  e * a
    float *spp = sea + GPW * J;                // [GPW][R]  p
    // G ownership: column r = lane % R, rows [jb, jb + EPL)
    const int r = lane % R;
    const int jb = (lane / R) * EPL;
    const bool active = jb < J;

    float acc[EPL], tot[EPL];
#pragma unroll
    for (int q = 0; q < EPL; ++q) acc[q] = tot[q] = 0.f;

    const int64_t span = (a.count + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = (int64_t)blockIdx.x * span;
    const int64_t p1 = min(a.count, p0 + span);
    int fold = 0;
    for (int64_t t0 = p0 + (int64_t)warp * GPW; t0 < p1; t0 += (int64_t)kCoreWarps * GPW) {
        const int64_t pos = t0 + gw;
        bool ok = pos < p1;
        int64_t s = 0;
        if (ok) ok = sample_at(a, a.base + pos, s);
        int32_t ik[kMaxOrder];
        int32_t in = 0;
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
        const float x = ok ? __ldg(a.val + s) : 0.f;
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
        float av[JL];
#pragma unroll
        for (int q = 0; q < JL; ++q) av[q] = 0.f;
        if (ok) load_run<JL>(a.A + (int64_t)in * J + sub * JL, av);
        // v = B p (partial over the lane's r), reduce-scatter to the lane's j slice
        float vp[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
            vp[j] = fmaf(b.x, p.x, fmaf(b.y, p.y, fmaf(b.z, p.z, b.w * p.w)));
        }
        group_reduce_scatter<T, J>(vp, sub);
        float dot = 0.f;
#pragma unroll
        for (int q = 0; q < JL; ++q) dot = fmaf(av[q], vp[q], dot);
        const float xh = group_sum<T>(dot);  // every lane takes part in the shuffles
        const float e = ok ? x - xh : 0.f;
        // stage e*a (lane's J slice) and p (lane's 4 r)
#pragma unroll
        for (int q = 0; q < JL; ++q) sea[gw * J + sub * JL + q] = e * av[q];
        *reinterpret_cast<float4 *>(&spp[gw * R + 4 * sub]) =
            ok ? p : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        if (active) {
#pragma unroll
            for (int g = 0; g < GPW; ++g) {
                const float pr = spp[g * R + r];
#pragma unroll
                for (int q = 0; q < EPL; ++q) acc[q] = fmaf(sea[g * J + jb + q], pr, acc[q]);
            }
        }
        __syncwarp();
        if (++fold == 16) {  // two-level summation keeps long spans accurate
            fold = 0;
#pragma unroll
            for (int q = 0; q < EPL; ++q) {
                tot[q] += acc[q];
                acc[q] = 0.f;
            }
        }
    }
    __syncthreads();  // staging area becomes the reduction area
    if (active) {
#pragma unroll
        for (int q = 0; q < EPL; ++q) sbuf[warp * JR + (jb + q) * R + r] = tot[q] + acc[q];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < JR; q += blockDim.x) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kCoreWarps; ++w) s += sbuf[w * JR + q];
        partials[(int64_t)blockIdx.x * JR + q] = s;
    }
}

// B += lr (G / M_b - lambda B) with G the sum of the block partials.  A block
// takes 32 entries of G; warp w sums, in float64, the partials of blocks
// w, w + 8, w + 16, ... (lane l: entry l, so the loads are coalesced), and the
// eight warp sums are added in warp order: a fixed order for a given partial
// count, spread over several SMs (one SM's float64 rate made a single-block
// sum of 608 partials take ~90 us).
constexpr int kApplyWarps = 8;

__global__ void __launch_bounds__(kApplyWarps * 32) k_core_apply(float *__restrict__ B,
                                                              const float *__restrict__ partials,
                                                              int nblk, int JR, int64_t Mb,
                                                              float lr, float lam) {
    __shared__ double part[kApplyWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    double g = 0.0;
    if (q < JR) {
#pragma unroll 4
        for (int b = w; b < nblk; b += kApplyWarps) g += (double)__ldg(partials + (int64_t)b * JR + q);
    }
    part[w][lane] = g;
    __syncthreads();
    if (w == 0 && q < JR) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kApplyWarps; ++k) t += part[k][lane];
        const double bq = B[q];
        B[q] = (float)(bq + (double)lr * (t / (double)Mb - (double)lam * bq));
    }
}

// One block per 128 nonzeros (a 4096-nonzero minibatch spreads over 32 SMs),
// at most four per SM (a whole pass).
int core_blocks_for(int64_t count, int sms) {
    int64_t b = (count + 127) / 128;
    const int64_t cap = (int64_t)sms * 4;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_core(const PassArgs &a, int J, int R, float *partials, int nblk,
                        cudaStream_t st) {
    SFT_DISPATCH_RJ(R, J, (k_core_grad<R_, J_><<<nblk, kCoreThreads, 0, st>>>(a, partials)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_core_apply(a.B, partials, nblk, J * R, a.count, a.lr, a.lam, st);
}

cudaError_t launch_core_apply(float *B, const float *partials, int nblk, int JR, int64_t Mb,
                              float lr, float lam, cudaStream_t st) {
    k_core_apply<<<(JR + 31) / 32, kApplyWarps * 32, 0, st>>>(B, partials, nblk, JR, Mb, lr, lam);
    return cudaGetLastError();
}

}  // namespace sft
