// k_grad.cu -- the sampled loss L = 1/2 sum_s e_s^2 over a COO set and its
// gradient with respect to every factor matrix A^(n) and core matrix B^(n).
// It is Eq. (10) and Eq. (11) without the regulariser, summed over the set
// instead of applied per sample.
//
// x^ depends on A^(n) and B^(n) only through the cached product
// C^(n) = A^(n) B^(n) (Eq. (12)), so the chain rule splits the gradient in two.
//
//   k_loss_grad   one pass over the nonzeros for all modes at once.  Each
//                 nonzero gathers its N rows of C, forms x^ and e, and adds
//                   dL/dC^(n)[i_n][r] += -e p^(n)[r],
//                   p^(n)[r] = prod_{k != n} C^(k)[i_k][r],
//                 into dC^(n) for every n.  p^(n) is the product of a prefix
//                 and a suffix of the gathered rows, with no division, so
//                 zero entries need no special case.  The adds are float4 red
//                 operations resolved in L2.  They are the only
//                 order-dependent rounding on this path, so the result is not
//                 bitwise reproducible.
//   k_grad_project  per mode: gA = s dC B^T row by row, and block partials of
//                 gB = s A^T dC.  A and dC tiles are staged in shared memory;
//                 s is the incoming gradient of L, read on the device.
//   k_grad_reduce   sums the gB partials in a fixed order (float64).
// Without dC buffers k_loss_grad computes only the loss.
#include "dispatch.cuh"
#include "sft_internal.cuh"

namespace sft {

constexpr int kGradThreads = 256;

// --------------------------------------------------------------------------- zero
// dC^(n) <- 0 for every mode; blockIdx.y is the mode.
__global__ void k_grad_zero(GradBufs g, int R) {
    const int n = blockIdx.y;
    float4 *p = reinterpret_cast<float4 *>(g.dC[n]);
    const int64_t q4 = g.dims[n] * (int64_t)R / 4;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q4;
         q += (int64_t)gridDim.x * blockDim.x)
        p[q] = z;
}

// --------------------------------------------------------------------------- loss + dC
// T = R/4 lanes per nonzero (lane `sub` owns r in [4 sub, 4 sub + 4)),
// GPW = 32/T nonzeros per warp per step.  NB bounds the order so that the N
// gathered rows and their prefix products stay in registers.
template <int R, int NB, typename CT, bool SCATTER>
__global__ void __launch_bounds__(kGradThreads) k_loss_grad(PassArgs a, GradBufs g,
                                                            double *__restrict__ partials) {
    constexpr int T = R / 4;
    constexpr int GPW = 32 / T;
    constexpr int WARPS = kGradThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    const int64_t span = (a.count + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = (int64_t)blockIdx.x * span;
    const int64_t p1 = min(a.count, p0 + span);
    double s2 = 0.0, s1 = 0.0;
    // The coordinates and value of the next nonzero are loaded one iteration
    // ahead (raw, checked when used), so only the row gathers wait on memory.
    int32_t nik[NB];
    float nx = 0.f;
    auto fetch = [&](int64_t s) {
        const bool in = s < p1;
#pragma unroll
        for (int k = 0; k < NB; ++k) nik[k] = (in && k < a.N) ? __ldg(a.idx[k] + s) : 0;
        nx = in ? __ldg(a.val + s) : 0.f;
    };
    fetch(p0 + (int64_t)warp * GPW + gw);
    for (int64_t t0 = p0 + (int64_t)warp * GPW; t0 < p1; t0 += (int64_t)WARPS * GPW) {
        const int64_t s = t0 + gw;
        bool ok = s < p1;
        int32_t ik[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            ik[k] = nik[k];
            if (ok && k < a.N && (uint32_t)ik[k] >= (uint32_t)a.dims[k]) {
                atomicOr(a.err, kErrIndex);
                ok = false;
            }
        }
        const float x = ok ? nx : 0.f;
        fetch(s + (int64_t)WARPS * GPW);
        float4 c[NB], pre[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k)
            c[k] = (ok && k < a.N) ? ldC<CT>(a.C[k], (int64_t)ik[k] * R + 4 * sub)
                                   : make_float4(1.f, 1.f, 1.f, 1.f);
        float4 run = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            pre[k] = run;
            if (k < a.N) mul4(run, c[k]);
        }
        const float xh = group_sum<T>((run.x + run.y) + (run.z + run.w));
        const float e = ok ? x - xh : 0.f;
        if (ok && sub == 0) {
            s2 += (double)e * (double)e;
            s1 += fabs((double)e);
        }
        if (SCATTER && ok) {
            float4 suf = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
            for (int k = NB - 1; k >= 0; --k) {
                if (k < a.N) {
                    float4 d = pre[k];
                    mul4(d, suf);
                    d.x *= -e; d.y *= -e; d.z *= -e; d.w *= -e;
                    atomicAdd(reinterpret_cast<float4 *>(g.dC[k] + (int64_t)ik[k] * R + 4 * sub), d);
                    mul4(suf, c[k]);
                }
            }
        }
    }
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

// out[0] = 1/2 sum e^2 (the loss L), out[1] = sum |e|; one warp, fixed order.
__global__ void k_loss_grad_final(const double *__restrict__ partials, int nblk, double *out) {
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
        out[0] = 0.5 * t2;
        out[1] = t1;
    }
}

cudaError_t launch_loss_grad(const PassArgs &a, const GradBufs &g, int R, bool accumulate,
                             double *partials, int nblk, double *out, cudaStream_t st, int sms,
                             int64_t *launches) {
    const bool scatter = g.dC[0] != nullptr;
    if (scatter && !accumulate) {
        dim3 grid((unsigned)(sms * 2), (unsigned)a.N);
        k_grad_zero<<<grid, kGradThreads, 0, st>>>(g, R);
        *launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    auto go = [&](auto nb_c) {
        constexpr int NB = decltype(nb_c)::value;
        if (a.cbf16)
            SFT_DISPATCH_R(R, (k_loss_grad<R_, NB, __nv_bfloat16, true><<<nblk, kGradThreads, 0, st>>>(a, g, partials)));
        else
            SFT_DISPATCH_R(R, (k_loss_grad<R_, NB, float, true><<<nblk, kGradThreads, 0, st>>>(a, g, partials)));
    };
    auto go_loss = [&](auto nb_c) {
        constexpr int NB = decltype(nb_c)::value;
        if (a.cbf16)
            SFT_DISPATCH_R(R, (k_loss_grad<R_, NB, __nv_bfloat16, false><<<nblk, kGradThreads, 0, st>>>(a, g, partials)));
        else
            SFT_DISPATCH_R(R, (k_loss_grad<R_, NB, float, false><<<nblk, kGradThreads, 0, st>>>(a, g, partials)));
    };
    if (!scatter) go_loss(ic<16>{});
    else if (a.N <= 4) go(ic<4>{});
    else if (a.N <= 8) go(ic<8>{});
    else go(ic<16>{});
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_loss_grad_final<<<1, 32, 0, st>>>(partials, nblk, out);
    *launches += 1;
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- dC -> gA, gB
// Tiles of TR consecutive rows; A (TR x J) and dC (TR x R) are contiguous in
// memory and staged with float4 loads, rows past I read as zero.
//   gA[i][j] = s sum_r dC[i][r] B[j][r]   (thread per output, coalesced stores)
//   G[j][r] += sum_i A[i][j] dC[i][r]     (thread per G entry, kept in registers)
template <int R, int J>
__global__ void __launch_bounds__(kGradThreads) k_grad_project(const float *__restrict__ A,
                                                               const float *__restrict__ B,
                                                               const float *__restrict__ dC,
                                                               int64_t I,
                                                               const double *__restrict__ scale,
                                                               float *__restrict__ gA,
                                                               float *__restrict__ partials) {
    constexpr int TR = 32;
    constexpr int JR = J * R;
    constexpr int EPT = (JR + kGradThreads - 1) / kGradThreads;
    __shared__ float sB[J][R + 1];
    __shared__ __align__(16) float sA[TR * J];
    __shared__ __align__(16) float sD[TR * R];
    for (int q = threadIdx.x; q < JR; q += blockDim.x) sB[q / R][q % R] = B[q];
    const float sc = scale ? (float)*scale : 1.f;
    float acc[EPT];
#pragma unroll
    for (int m = 0; m < EPT; ++m) acc[m] = 0.f;
    const int64_t tiles = (I + TR - 1) / TR;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = tile * TR;
        const int rows = (int)min((int64_t)TR, I - row0);
        __syncthreads();  // previous tile fully consumed (and sB written on entry)
        for (int q = threadIdx.x; q < TR * J / 4; q += blockDim.x)
            reinterpret_cast<float4 *>(sA)[q] =
                4 * q < rows * J ? ldg4(A + row0 * J + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = threadIdx.x; q < TR * R / 4; q += blockDim.x)
            reinterpret_cast<float4 *>(sD)[q] =
                4 * q < rows * R ? ldg4(dC + row0 * R + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        for (int o = threadIdx.x; o < rows * J; o += blockDim.x) {
            const int row = o / J, j = o % J;
            float t = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) t = fmaf(sD[row * R + r], sB[j][r], t);
            gA[row0 * J + o] = sc * t;
        }
#pragma unroll
        for (int m = 0; m < EPT; ++m) {
            const int q = threadIdx.x + m * kGradThreads;
            if (q < JR) {
                const int j = q / R, r = q % R;
                float t = acc[m];
#pragma unroll 8
                for (int row = 0; row < TR; ++row) t = fmaf(sA[row * J + j], sD[row * R + r], t);
                acc[m] = t;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
        const int q = threadIdx.x + m * kGradThreads;
        if (q < JR) partials[(int64_t)blockIdx.x * JR + q] = acc[m];
    }
}

// A block takes 32 entries of dL/dB; warp w sums (float64) the partials of
// blocks w, w + 8, ... (lane l: entry l), then the warp sums are added in warp
// order: a fixed order, spread over JR / 32 SMs instead of one SM's float64
// units.
constexpr int kReduceWarps = 8;

__global__ void __launch_bounds__(kReduceWarps * 32) k_grad_reduce(const float *__restrict__ partials,
                                                                int nblk, int JR,
                                                                const double *__restrict__ scale,
                                                                float *__restrict__ gB) {
    __shared__ double part[kReduceWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    double t = 0.0;
    if (q < JR) {
#pragma unroll 4
        for (int b = w; b < nblk; b += kReduceWarps) t += (double)__ldg(partials + (int64_t)b * JR + q);
    }
    part[w][lane] = t;
    __syncthreads();
    if (w == 0 && q < JR) {
        double u = 0.0;
#pragma unroll
        for (int k = 0; k < kReduceWarps; ++k) u += part[k][lane];
        gB[q] = (float)((scale ? *scale : 1.0) * u);
    }
}

cudaError_t launch_grad_project(const float *A, const float *B, const float *dC, int64_t I, int J,
                                int R, const double *scale, float *gA, float *gB, float *partials,
                                int max_blocks, cudaStream_t st, int sms, int64_t *launches) {
    int64_t nblk = (I + 31) / 32;
    const int64_t cap = (int64_t)sms * 2 < max_blocks ? (int64_t)sms * 2 : max_blocks;
    if (nblk > cap) nblk = cap;
    if (nblk < 1) nblk = 1;
    SFT_DISPATCH_RJ(R, J, (k_grad_project<R_, J_><<<(int)nblk, kGradThreads, 0, st>>>(
                              A, B, dC, I, scale, gA, partials)));
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int JR = J * R;
    k_grad_reduce<<<(JR + 31) / 32, kReduceWarps * 32, 0, st>>>(partials, (int)nblk, JR, scale, gB);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace sft
