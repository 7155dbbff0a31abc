// k_batch.cu -- one persistent kernel that runs a task list covering many
// independent sparse FastTucker decompositions (each with J_n = R).
//
// CTAs take tasks in list order from a global counter.  A task belongs to a
// phase of one decomposition (a factor pass of mode n, the refresh of C^(n),
// a core pass, its update of B^(n), a loss pass).  The phases of one
// decomposition follow Algorithm 2 and form a chain.  A task first waits
// until the phase it depends on has finished: its counter, decremented by
// every finished task of that phase, reaches zero.  The wait is a bounded
// poll; when the poll limit is reached the kernel raises kErrWait and every
// CTA stops.  The list is a topological order built on the host, so a task
// only ever waits on tasks handed out before it, which are held by running
// CTAs.
//
// Memory ordering: a finished task's writes are published by __syncthreads,
// a device-scope fence and the counter decrement.  The waiting CTA reads the
// counter with ld.acquire.gpu.  Every matrix that a task of the same launch
// may have written (A, B, C) is read through L2 (ld.global.cg), never through
// the non-coherent path.
//
// Task bodies, T = R/4 lanes per nonzero; lane `sub` owns entries
// [4 sub, 4 sub + 4) of every R- (and J = R-) vector:
//   factor   Hogwild SGD on A^(n) rows (Algorithm 4; Eq. (10)): p from the
//            cached rows of the other modes, v = B^(n) p, e = x - a.v,
//            a += lr (e v - lambda a) with vector atomics
//   refresh  C^(n) rows = A^(n) rows B^(n) (Algorithm 3)
//   core     sum over the chunk of e a p^T (Eq. (11)) into a partial slot
//   apply    B^(n) += lr (sum of the slots / nnz - lambda B^(n)) (Algorithm 5)
//   loss     sums of e^2 and |e| of the chunk into a slot; loss-final adds
//            the slots in order
#include "batch_internal.cuh"

// One-ahead gathers of the task loops (1) or gathers at use (0), and the
// minimum resident CTAs per SM asked of the register allocator for the
// kernels of the small ranks (class 0) and of R = 32 (class 1).  Measured on
// the 64-problem workload (epoch ms, class 1 at 1 CTA per SM): gathers at use
// with 3 CTAs per SM for class 0 44.0; 2 CTAs 45.9; 4 CTAs 45.6; one-ahead
// gathers 46.2 (2 CTAs) and 64.1 (3 CTAs, spilling); then class 1 at 2 CTAs
// per SM (128 registers) 38.6.
#ifndef SFT_BATCH_PREFETCH
#define SFT_BATCH_PREFETCH 0
#endif
#ifndef SFT_BATCH_MINB0
#define SFT_BATCH_MINB0 3
#endif
#ifndef SFT_BATCH_MINB1
#define SFT_BATCH_MINB1 2
#endif

namespace sft {

namespace {

constexpr int kWarps = kBatchThreads / 32;

// Cached-product entries through L2 (they may have been refreshed by another
// CTA during this launch).
template <typename CT>
__device__ __forceinline__ float4 ldCcg(const float *base, int64_t off);

template <>
__device__ __forceinline__ float4 ldCcg<float>(const float *base, int64_t off) {
    return __ldcg(reinterpret_cast<const float4 *>(base + off));
}

template <>
__device__ __forceinline__ float4 ldCcg<__nv_bfloat16>(const float *base, int64_t off) {
    const uint2 u = __ldcg(reinterpret_cast<const uint2 *>(
        reinterpret_cast<const __nv_bfloat16 *>(base) + off));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Coordinates and value of the nonzero a lane group visits next, loaded one
// iteration ahead of use (raw); take() checks them and hands them over.
struct NextSample {
    int32_t ik[kBatchMaxOrder];
    float x;
    __device__ __forceinline__ void fetch(const BatchProblem &P, int64_t s, int64_t end) {
        const bool in = s < end;
#pragma unroll
        for (int k = 0; k < kBatchMaxOrder; ++k) ik[k] = (in && k < P.N) ? __ldg(P.idx[k] + s) : 0;
        x = in ? __ldg(P.val + s) : 0.f;
    }
    __device__ __forceinline__ bool take(const BatchProblem &P, bool ok, int n,
                                         int32_t (&out)[kBatchMaxOrder], int32_t &in, float &xo,
                                         int *err) const {
        in = 0;
#pragma unroll
        for (int k = 0; k < kBatchMaxOrder; ++k) {
            out[k] = ik[k];
            if (ok && k < P.N) {
                if ((uint32_t)ik[k] >= (uint32_t)P.dims[k]) {
                    atomicOr(err, kErrIndex);
                    ok = false;
                }
                if (k == n) in = ik[k];
            }
        }
        xo = ok ? x : 0.f;
        return ok;
    }
};

// One nonzero of a lane group with its gathered rows: the lane's 4 entries of
// C^(k)[i_k] for k != skip (skip = -1: every mode) and, where the task needs
// it, of the factor row a_{i_n}.  Loaded one iteration before use, so a lane
// group has two nonzeros' gathers in flight.
struct Gathered {
    float4 c[kBatchMaxOrder];
    float4 a;
    int32_t in;
    float x;
    bool ok;
};

template <int R, typename CT, bool WITH_A>
__device__ __forceinline__ void gather(const BatchProblem &P, const NextSample &nxt, bool valid,
                                       int skip, int sub, Gathered &g, int *err) {
    int32_t ik[kBatchMaxOrder];
    g.ok = nxt.take(P, valid, skip, ik, g.in, g.x, err);
#pragma unroll
    for (int k = 0; k < kBatchMaxOrder; ++k)
        g.c[k] = (g.ok && k < P.N && k != skip) ? ldCcg<CT>(P.C[k], (int64_t)ik[k] * R + 4 * sub)
                                                : make_float4(1.f, 1.f, 1.f, 1.f);
    if constexpr (WITH_A)
        g.a = g.ok ? __ldcg(reinterpret_cast<const float4 *>(P.A[skip] + (int64_t)g.in * R) + sub)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Lane's 4 entries of the product of the gathered rows.
__device__ __forceinline__ float4 product(const Gathered &g) {
    float4 p = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
    for (int k = 0; k < kBatchMaxOrder; ++k) mul4(p, g.c[k]);
    return p;
}

// The lane group's nonzeros of a task, s = begin + warp GPW + gw, then every
// kWarps GPW: body(g) for each with its gathered rows (g.ok false past the
// end).  The loop bound is uniform over the warp.
template <int R, typename CT, bool WITH_A, typename Body>
__device__ __forceinline__ void walk_chunk(const BatchProblem &P, const BatchTask &tk, int skip,
                                           int sub, int gw, int warp, int *err, Body &&body) {
    constexpr int T = R / 4, GPW = 32 / T;
    constexpr int64_t STEP = (int64_t)kWarps * GPW;
    const int64_t s0 = tk.begin + (int64_t)warp * GPW + gw;
    NextSample nxt;
    nxt.fetch(P, s0, tk.end);
    Gathered cur;
    if constexpr (SFT_BATCH_PREFETCH) {
        gather<R, CT, WITH_A>(P, nxt, s0 < tk.end, skip, sub, cur, err);
        nxt.fetch(P, s0 + STEP, tk.end);
    }
    for (int64_t t0 = tk.begin + (int64_t)warp * GPW; t0 < tk.end; t0 += STEP) {
        const int64_t s = t0 + gw;
        if constexpr (SFT_BATCH_PREFETCH) {
            // the next nonzero's gathers go out before this one is formed
            Gathered nx;
            gather<R, CT, WITH_A>(P, nxt, s + STEP < tk.end, skip, sub, nx, err);
            nxt.fetch(P, s + 2 * STEP, tk.end);
            body(cur);
            cur = nx;
        } else {
            gather<R, CT, WITH_A>(P, nxt, s < tk.end, skip, sub, cur, err);
            nxt.fetch(P, s + STEP, tk.end);
            body(cur);
        }
    }
}

// B^(n) (R x R) into shared memory.
template <int R>
__device__ __forceinline__ void stage_B(const float *B, float *sB) {
    for (int q = threadIdx.x; q < R * R / 4; q += blockDim.x)
        reinterpret_cast<float4 *>(sB)[q] = __ldcg(reinterpret_cast<const float4 *>(B) + q);
    __syncthreads();
}

// e for one nonzero: p, then v = B p scattered to the lane's 4 j, x^ = a.v.
// Returns e (0 for an invalid sample); v and a are the lane's slices.
template <int R>
__device__ __forceinline__ float residual(const float *sB, const float4 &p, const float4 &a,
                                          float x, bool ok, int sub, float (&v)[R]) {
    constexpr int T = R / 4;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
        v[j] = fmaf(b.x, p.x, fmaf(b.y, p.y, fmaf(b.z, p.z, b.w * p.w)));
    }
    group_reduce_scatter<T, R>(v, sub);  // v[0..4): entries [4 sub, 4 sub + 4)
    const float dot = fmaf(a.x, v[0], fmaf(a.y, v[1], fmaf(a.z, v[2], a.w * v[3])));
    const float xh = group_sum<T>(dot);
    return ok ? x - xh : 0.f;
}

template <int R, typename CT>
__device__ void task_factor(const BatchProblem &P, const BatchTask &tk, float *sB, int *err) {
    constexpr int T = R / 4;
    stage_B<R>(P.B[tk.mode], sB);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    const int n = tk.mode;
    float *An = P.A[n];
    walk_chunk<R, CT, true>(P, tk, n, sub, gw, warp, err, [&](const Gathered &cur) {
        const float4 p = product(cur);
        const float4 a = cur.a;
        float v[R];
        const float e = residual<R>(sB, p, a, cur.x, cur.ok, sub, v);
        if (cur.ok) {
            float4 d;
            d.x = P.lrA * (e * v[0] - P.lamA * a.x);
            d.y = P.lrA * (e * v[1] - P.lamA * a.y);
            d.z = P.lrA * (e * v[2] - P.lamA * a.z);
            d.w = P.lrA * (e * v[3] - P.lamA * a.w);
            atomicAdd(reinterpret_cast<float4 *>(An + (int64_t)cur.in * R + 4 * sub), d);
        }
    });
}

template <int R, typename CT>
__device__ void task_refresh(const BatchProblem &P, const BatchTask &tk, float *sB) {
    constexpr int T = R / 4;
    stage_B<R>(P.B[tk.mode], sB);
    const int sub = threadIdx.x & (T - 1);
    const float *An = P.A[tk.mode];
    for (int64_t row = tk.begin + threadIdx.x / T; row < tk.end; row += kBatchThreads / T) {
        float a[R];
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const float4 v = __ldcg(reinterpret_cast<const float4 *>(An + row * R) + q);
            a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
        }
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
            c.x = fmaf(a[j], b.x, c.x);
            c.y = fmaf(a[j], b.y, c.y);
            c.z = fmaf(a[j], b.z, c.z);
            c.w = fmaf(a[j], b.w, c.w);
        }
        stC<CT>(P.C[tk.mode], row * R + 4 * sub, c);
    }
}

// Core task.  Shared memory: staging [warp][GPW][R] of e*a and of p during
// the loop, then [warp][R*R] for the fixed-order reduction of G.
template <int R, typename CT>
__device__ void task_core(const BatchProblem &P, const BatchTask &tk, float *sB, float *sbuf,
                          int *err) {
    constexpr int T = R / 4, GPW = 32 / T, RR = R * R;
    constexpr int EPL = RR >= 32 ? RR / 32 : 1;  // G entries per lane
    stage_B<R>(P.B[tk.mode], sB);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    const int n = tk.mode;
    float *sea = sbuf + warp * GPW * 2 * R;  // [GPW][R] e * a
    float *spp = sea + GPW * R;              // [GPW][R] p
    const int r = lane % R;                  // G ownership: column r, rows [jb, jb + EPL)
    const int jb = (lane / R) * EPL;
    const bool active = jb < R;
    float acc[EPL], tot[EPL];
#pragma unroll
    for (int q = 0; q < EPL; ++q) acc[q] = tot[q] = 0.f;
    int fold = 0;
    walk_chunk<R, CT, true>(P, tk, n, sub, gw, warp, err, [&](const Gathered &cur) {
        const bool ok = cur.ok;
        const float4 p = product(cur);
        const float4 a = cur.a;
        float v[R];
        const float e = residual<R>(sB, p, a, cur.x, ok, sub, v);
        *reinterpret_cast<float4 *>(&sea[gw * R + 4 * sub]) =
            make_float4(e * a.x, e * a.y, e * a.z, e * a.w);
        *reinterpret_cast<float4 *>(&spp[gw * R + 4 * sub]) =
            ok ? p : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        if (active) {
#pragma unroll
            for (int g = 0; g < GPW; ++g) {
                const float pr = spp[g * R + r];
#pragma unroll
                for (int q = 0; q < EPL; ++q) acc[q] = fmaf(sea[g * R + jb + q], pr, acc[q]);
            }
        }
        __syncwarp();
        if (++fold == 16) {
            fold = 0;
#pragma unroll
            for (int q = 0; q < EPL; ++q) {
                tot[q] += acc[q];
                acc[q] = 0.f;
            }
        }
    });
    __syncthreads();  // staging becomes the reduction area
    if (active) {
#pragma unroll
        for (int q = 0; q < EPL; ++q) sbuf[warp * RR + (jb + q) * R + r] = tot[q] + acc[q];
    }
    __syncthreads();
    float *out = P.partials + (int64_t)tk.slot * RR;
    for (int q = threadIdx.x; q < RR; q += blockDim.x) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += sbuf[w * RR + q];
        out[q] = s;
    }
}

template <int R>
__device__ void task_apply(const BatchProblem &P, const BatchTask &tk) {
    constexpr int RR = R * R;
    float *B = P.B[tk.mode];
    const double inv = 1.0 / (double)P.nnz;
    for (int q = threadIdx.x; q < RR; q += blockDim.x) {
        double g = 0.0;
        for (int k = 0; k < tk.nslots; ++k) g += (double)__ldcg(P.partials + (int64_t)k * RR + q);
        const double b = __ldcg(B + q);
        B[q] = (float)(b + (double)P.lrB * (g * inv - (double)P.lamB * b));
    }
}

template <int R, typename CT>
__device__ void task_loss(const BatchProblem &P, const BatchTask &tk, double *sred, int *err) {
    constexpr int T = R / 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    double s2 = 0.0, s1 = 0.0;
    walk_chunk<R, CT, false>(P, tk, -1, sub, gw, warp, err, [&](const Gathered &cur) {
        const float4 p = product(cur);
        const float xh = group_sum<T>((p.x + p.y) + (p.z + p.w));
        if (cur.ok && sub == 0) {
            const double e = (double)cur.x - (double)xh;
            s2 += e * e;
            s1 += fabs(e);
        }
    });
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        s2 += __shfl_xor_sync(kFull, s2, w);
        s1 += __shfl_xor_sync(kFull, s1, w);
    }
    if (lane == 0) {
        sred[2 * warp] = s2;
        sred[2 * warp + 1] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t2 = 0.0, t1 = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            t2 += sred[2 * w];
            t1 += sred[2 * w + 1];
        }
        P.lpart[2 * tk.slot] = t2;
        P.lpart[2 * tk.slot + 1] = t1;
    }
}

__device__ void task_loss_final(const BatchProblem &P, const BatchTask &tk) {
    if (threadIdx.x == 0) {
        double t2 = 0.0, t1 = 0.0;
        for (int k = 0; k < tk.nslots; ++k) {
            t2 += __ldcg(P.lpart + 2 * k);
            t1 += __ldcg(P.lpart + 2 * k + 1);
        }
        P.loss_out[0] = t2;
        P.loss_out[1] = t1;
    }
}

template <int R, typename CT>
__device__ void run_task(const BatchProblem &P, const BatchTask &tk, float *sB, float *sbuf,
                         int *err) {
    switch (tk.kind) {
        case kTaskFactor: task_factor<R, CT>(P, tk, sB, err); break;
        case kTaskRefresh: task_refresh<R, CT>(P, tk, sB); break;
        case kTaskCore: task_core<R, CT>(P, tk, sB, sbuf, err); break;
        case kTaskApply: task_apply<R>(P, tk); break;
        case kTaskLoss: task_loss<R, CT>(P, tk, reinterpret_cast<double *>(sbuf), err); break;
        case kTaskLossFin: task_loss_final(P, tk); break;
        default: break;
    }
}

template <typename CT, int CLS>
__global__ void __launch_bounds__(kBatchThreads, CLS == 0 ? SFT_BATCH_MINB0 : SFT_BATCH_MINB1)
    k_batch_run(BatchArgs g) {
    __shared__ __align__(16) float sB[32 * 32];
    __shared__ __align__(16) float sbuf[kWarps * 32 * 32];
    __shared__ __align__(16) BatchProblem sP;  // the task's problem record
    __shared__ int s_task;
    for (;;) {
        if (threadIdx.x == 0) {
            int t = atomicAdd(g.head, 1);
            if (t >= g.ntasks || *(volatile int32_t *)g.abort) {
                t = -1;
            } else {
                const int32_t w = g.tasks[t].wait;
                if (w >= 0) {
                    int64_t polls = 0;
                    while (ld_acquire(g.counters + w) > 0) {
                        if (*(volatile int32_t *)g.abort) {
                            t = -1;
                            break;
                        }
                        if (++polls > g.wait_limit) {
                            atomicOr(g.err, kErrWait);
                            atomicExch(g.abort, 1);
                            t = -1;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
            }
            s_task = t;
        }
        __syncthreads();
        const int t = s_task;
        if (t < 0) break;
        const BatchTask tk = g.tasks[t];
        // the problem record (pointers, sizes, rates) into shared memory, so
        // that the task loops read it there instead of holding it in registers
        static_assert(sizeof(BatchProblem) % 4 == 0, "record copied as words");
        for (int q = threadIdx.x; q < (int)(sizeof(BatchProblem) / 4); q += blockDim.x)
            reinterpret_cast<int32_t *>(&sP)[q] =
                reinterpret_cast<const int32_t *>(g.probs + tk.prob)[q];
        __syncthreads();
        const BatchProblem &P = sP;
        if constexpr (CLS == 0) {
            switch (P.R) {
                case 4: run_task<4, CT>(P, tk, sB, sbuf, g.err); break;
                case 8: run_task<8, CT>(P, tk, sB, sbuf, g.err); break;
                case 16: run_task<16, CT>(P, tk, sB, sbuf, g.err); break;
                default: break;
            }
        } else {
            if (P.R == 32) run_task<32, CT>(P, tk, sB, sbuf, g.err);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicSub(g.counters + tk.done, 1);
        }
    }
}

// Counters back to their starting values and the classes' task cursors to 0.
__global__ void k_batch_reset(BatchArgs g, int32_t *head1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.ncounters; i += gridDim.x * blockDim.x)
        g.counters[i] = g.init[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *g.head = 0;
        *head1 = 0;
        *g.abort = 0;
    }
}

template <typename CT>
int blocks_per_sm(int cls) {
    int n = 0;
    cudaError_t e = cls == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &n, k_batch_run<CT, 0>, kBatchThreads, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &n, k_batch_run<CT, 1>, kBatchThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

template <typename CT>
void launch_class(const BatchArgs &g, int cls, int grid, cudaStream_t st) {
    if (cls == 0) k_batch_run<CT, 0><<<grid, kBatchThreads, 0, st>>>(g);
    else k_batch_run<CT, 1><<<grid, kBatchThreads, 0, st>>>(g);
}

}  // namespace

int batch_blocks_per_sm(bool cbf16, int cls) {
    return cbf16 ? blocks_per_sm<__nv_bfloat16>(cls) : blocks_per_sm<float>(cls);
}

cudaError_t launch_batch(const BatchLaunch &L, bool cbf16, cudaStream_t st, cudaStream_t side,
                         cudaEvent_t fork, cudaEvent_t join) {
    const BatchArgs &g0 = L.cls[0];
    const int rblocks = g0.ncounters > 0 ? (g0.ncounters + 255) / 256 : 1;
    k_batch_reset<<<rblocks, 256, 0, st>>>(g0, L.cls[1].head);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool has0 = L.cls[0].ntasks > 0, has1 = L.cls[1].ntasks > 0;
    auto run = [&](int cls, cudaStream_t s) {
        if (cbf16) launch_class<__nv_bfloat16>(L.cls[cls], cls, L.grid[cls], s);
        else launch_class<float>(L.cls[cls], cls, L.grid[cls], s);
    };
    if (has0 && has1) {
        // the R = 32 kernel (the longer tasks) on the side stream, first
        if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
        run(1, side);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
        run(0, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return cudaStreamWaitEvent(st, join, 0);
    }
    if (has0) run(0, st);
    else if (has1) run(1, st);
    return cudaGetLastError();
}

}  // namespace sft
