// k_tc.cu -- the two dense contractions of the method on the fifth-generation
// tensor cores (tcgen05 MMAs with their float32 accumulators in tensor memory),
// used when the cached products are stored as bfloat16:
//
//   * the refresh C^(n) = A^(n) B^(n) (Algorithm 3): tiles of 128 rows of the
//     float32 master A^(n) are copied into shared memory by TMA, one chain of
//     kind::tf32 MMAs per tile (M = 128 rows, N = R, K = J_n) accumulates in
//     tensor memory, and the epilogue rounds the tile to bfloat16 on its way
//     to C^(n);
//   * the minibatch core gradient G = sum_s e_s a_{i_n(s)} p_s^T of Eq. (11)
//     (Algorithm 5 accumulates it before one uniform update), i.e. the
//     contraction (J_n x M) . (M x R) over the M nonzeros of a minibatch:
//     lane groups form e_s a and p_s of 64 nonzeros at a time, write them as
//     bfloat16 operand tiles (K = nonzero), and one thread issues kind::f16
//     MMAs that accumulate the block's share of G in tensor memory while the
//     next 64 nonzeros are gathered into the other buffer.
//
// Operand tiles are K-major without swizzling: "core matrices" of 8 rows x 16
// bytes, lbo bytes apart along K and sbo bytes apart along M (or N).  Every
// wait on an mbarrier is bounded by a time limit; a wait that runs out sets
// kErrWait in the error flag (reported as SFT_ETIMEOUT), the block stops its
// work, waits once more for what it issued, frees its tensor memory and
// returns.
#include <cuda.h>

#include "dispatch.cuh"
#include "sft_internal.cuh"

namespace sft {
namespace tc {

constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s: the default limit and the drain bound

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor of a K-major operand without swizzling.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0, no swizzle
    return d;
}

// Instruction descriptor: float32 accumulator, A and B of format `fmt` (kind::f16:
// 1 = bfloat16; kind::tf32: 2 = tf32), both K-major, an M x N accumulator.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits until the phase of parity `parity` of barrier b has completed, for at
// most limit_ns; false if the limit ran out.  A limit of 0 gives up without
// looking (the wait has no time at all), which lets a caller make the expiry
// path run on a normal launch.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity,
                                          uint64_t limit_ns = kWaitNs) {
    if (limit_ns == 0) return false;
    if (mbar_test(b, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_test(b, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
        __nanosleep(100);
    }
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 2-D TMA tile load (x = innermost coordinate in elements) completing on bar.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

constexpr int kTmemCols = 32;  // smallest allocation; holds N <= 32 float32 columns

// Whole warp: allocate kTmemCols columns of tensor memory, address to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(slot)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Whole warp (the allocating one).
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "n"(kTmemCols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}

// Arrives on bar once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

// Whole warp: 16 consecutive float32 columns of the warp's 32 tensor-memory
// lanes (thread t receives lane base + t); waits for the load to finish.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

}  // namespace tc

// ============================================================================ refresh
// One CTA of 128 threads per 128-row tile (grid-stride).  Shared memory:
//   sA  : the tile as J/4 column blocks, block q = columns [4q, 4q+4) of the
//         128 rows, 16 bytes per row (one TMA box {4, 128} each, 2 KB); so
//         core matrix (row group g, K block q) sits at q*2048 + g*128:
//         lbo = 2048, sbo = 128;
//   sBt : B^(n)T (R x J) in the same form, core matrix (g, q) at q*16R + g*128.
// kind::tf32 takes K = 8 per MMA, so a tile is J/8 MMAs.
constexpr int kTcRefreshThreads = 128;

template <int R, int J>
__global__ void __launch_bounds__(kTcRefreshThreads) k_refresh_tc(const __grid_constant__ CUtensorMap mapA,
                                                                  const float *__restrict__ B,
                                                                  __nv_bfloat16 *__restrict__ C,
                                                                  int64_t I, int *err,
                                                                  uint64_t wait_ns) {
    static_assert(R == 16 || R == 32, "N = R must be a multiple of 16 for M = 128");
    static_assert(J % 8 == 0, "K = J must be a multiple of 8 for kind::tf32");
    constexpr uint32_t kTileBytes = 128u * J * 4u;
    __shared__ __align__(1024) float sA[128 * J];
    __shared__ __align__(128) float sBt[R * J];
    __shared__ __align__(8) uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int q = threadIdx.x; q < J * R; q += blockDim.x) {
        const int j = q / R, r = q % R;
        sBt[(j >> 2) * 4 * R + (r >> 3) * 32 + (r & 7) * 4 + (j & 3)] = B[q];
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar_tma, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = tc::instr_desc(2, 128, R);
    const int64_t ntiles = (I + 127) / 128;
    uint32_t phase = 0;
    bool ok = true;
    bool tma_pending = false, mma_pending = false;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (threadIdx.x == 0) {
            tc::mbar_expect_tx(&bar_tma, kTileBytes);
#pragma unroll
            for (int q = 0; q < J / 4; ++q)
                tc::tma_load_2d(sA + q * 128 * 4, &mapA, 4 * q, (int32_t)(t * 128), &bar_tma);
        }
        tma_pending = true;
        ok = __syncthreads_and(tc::mbar_wait(&bar_tma, phase, wait_ns));
        if (!ok) break;
        tma_pending = false;
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sBt);
#pragma unroll
            for (int kk = 0; kk < J / 8; ++kk)
                tc::mma_tf32(tmem, tc::desc_kmajor(a0 + kk * 4096u, 2048u, 128u),
                             tc::desc_kmajor(b0 + kk * 32u * R, 16u * R, 128u), idesc, kk > 0);
            tc::mma_commit(&bar_mma);
        }
        mma_pending = true;
        ok = __syncthreads_and(tc::mbar_wait(&bar_mma, phase, wait_ns));
        if (!ok) break;
        mma_pending = false;
        tc::fence_after_sync();
        // epilogue: warp w owns tensor-memory lanes (tile rows) 32w .. 32w+31
        const int64_t row = t * 128 + warp * 32 + lane;
        uint4 out[R / 8];
#pragma unroll
        for (int h = 0; h < R / 16; ++h) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16u * h, v);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                out[2 * h + q] = make_uint4(tc::pack_bf16(v[8 * q + 0], v[8 * q + 1]),
                                            tc::pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                                            tc::pack_bf16(v[8 * q + 4], v[8 * q + 5]),
                                            tc::pack_bf16(v[8 * q + 6], v[8 * q + 7]));
        }
        if (row < I) {
            uint4 *dst = reinterpret_cast<uint4 *>(C + row * R);
#pragma unroll
            for (int q = 0; q < R / 8; ++q) dst[q] = out[q];
        }
        phase ^= 1u;
        tc::fence_before_sync();
        __syncthreads();  // tensor memory and sA are reused by the next tile
        tc::fence_after_sync();
    }
    if (!ok && threadIdx.x == 0) {
        atomicOr(err, kErrWait);
        // one more wait, with the full bound, for the copies / MMAs this block
        // issued, so that shared and tensor memory are released only after them
        if (tma_pending) tc::mbar_wait(&bar_tma, phase);
        if (mma_pending) tc::mbar_wait(&bar_mma, phase);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_free(tmem);
    }
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

}  // namespace

bool refresh_tc_supported(int J, int R) {
    return (R == 16 || R == 32) && (J == 8 || J == 16 || J == 32);
}

cudaError_t launch_refresh_tc(const float *A, const float *B, void *C, int64_t I, int J, int R,
                              int *err, uint64_t wait_ns, cudaStream_t st, int sms) {
    if (!refresh_tc_supported(J, R) || I < 1) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // A^(n): I rows of J float32; boxes of 4 columns x 128 rows
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)J, (cuuint64_t)I};
    const cuuint64_t gstride[1] = {(cuuint64_t)J * sizeof(float)};
    const cuuint32_t box[2] = {4, 128};
    const cuuint32_t estride[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(A), gdim, gstride, box,
            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int64_t ntiles = (I + 127) / 128;
    int64_t blocks = ntiles < (int64_t)sms * 4 ? ntiles : (int64_t)sms * 4;
    auto *Cb = reinterpret_cast<__nv_bfloat16 *>(C);
    switch (R * 100 + J) {
        case 1608: k_refresh_tc<16, 8><<<(int)blocks, kTcRefreshThreads, 0, st>>>(map, B, Cb, I, err, wait_ns); break;
        case 1616: k_refresh_tc<16, 16><<<(int)blocks, kTcRefreshThreads, 0, st>>>(map, B, Cb, I, err, wait_ns); break;
        case 1632: k_refresh_tc<16, 32><<<(int)blocks, kTcRefreshThreads, 0, st>>>(map, B, Cb, I, err, wait_ns); break;
        case 3208: k_refresh_tc<32, 8><<<(int)blocks, kTcRefreshThreads, 0, st>>>(map, B, Cb, I, err, wait_ns); break;
        case 3216: k_refresh_tc<32, 16><<<(int)blocks, kTcRefreshThreads, 0, st>>>(map, B, Cb, I, err, wait_ns); break;
        case 3232: k_refresh_tc<32, 32><<<(int)blocks, kTcRefreshThreads, 0, st>>>(map, B, Cb, I, err, wait_ns); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ============================================================================ core gradient
// 256 threads; lane groups of T = R/4 lanes form one nonzero's p (the lane's
// 4 entries) and e*a (the lane's J/T entries) exactly as the CUDA-core kernel
// does, then write them in bfloat16 into the operand tiles of the current
// buffer at column k (the nonzero's place among the 64 of the batch):
//   A operand (rows j, K = 64): (j/8)*1024 + (k/8)*128 + (j%8)*16 + (k%8)*2
//   B operand (rows r, K = 64): the same formula with r for j
// so lbo = 128, sbo = 1024, and MMA kk (K = 16) starts kk*256 bytes in.  The
// MMA reads 128 rows of A; rows >= J_n hold whatever the buffer region holds
// (zeroed at start) and only produce accumulator rows that are never read.
constexpr int kTcCoreThreads = 256;
constexpr int kTcCoreWarps = kTcCoreThreads / 32;
constexpr int kTcKC = 64;                    // nonzeros per MMA batch
constexpr int kTcABytes = 128 * kTcKC * 2;   // A region (all 128 rows the MMA reads)
constexpr int kTcBBytes = 32 * kTcKC * 2;    // B region (N <= 32 rows)
constexpr int kTcBufBytes = kTcABytes + kTcBBytes;
constexpr int kTcCoreSmem = 2 * kTcBufBytes + 1024;  // two buffers + alignment slack

template <int R, int J, typename CT>
__global__ void __launch_bounds__(kTcCoreThreads) k_core_grad_tc(PassArgs a,
                                                                 float *__restrict__ partials,
                                                                 uint64_t wait_ns) {
    static_assert(R == 16 || R == 32, "N = R must be a multiple of 16 for M = 128");
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int GPW = 32 / T;
    constexpr int NPS = kTcCoreWarps * GPW;  // nonzeros per step of the CTA
    constexpr int STEPS = kTcKC / NPS;       // steps per MMA batch
    static_assert(kTcKC % NPS == 0, "a batch is a whole number of steps");
    constexpr int JR = J * R;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(16) float sB[JR];
    __shared__ __align__(8) uint64_t bar_mma[2];
    __shared__ uint32_t tmem_slot;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (T - 1), gw = lane / T;
    for (int q = threadIdx.x; q < JR; q += blockDim.x) sB[q] = a.B[q];
    for (int q = threadIdx.x; q < 2 * kTcBufBytes / 16; q += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tc::tmem_alloc(&tmem_slot);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar_mma[0], 1);
        tc::mbar_init(&bar_mma[1], 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = tc::instr_desc(1, 128, R);

    const int64_t span = (a.count + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = (int64_t)blockIdx.x * span;
    const int64_t p1 = min(a.count, p0 + span);
    const int64_t nbatch = p1 > p0 ? (p1 - p0 + kTcKC - 1) / kTcKC : 0;
    bool ok = true;
    int64_t c = 0;
    for (; c < nbatch; ++c) {
        const int buf = (int)(c & 1);
        if (c >= 2) {  // the MMAs of batch c - 2 have finished reading this buffer
            ok = __syncthreads_and(
                tc::mbar_wait(&bar_mma[buf], (uint32_t)(((c - 2) >> 1) & 1), wait_ns));
            if (!ok) break;
        }
        uint8_t *tA = smem + buf * kTcBufBytes;
        uint8_t *tB = tA + kTcABytes;
#pragma unroll 1
        for (int stp = 0; stp < STEPS; ++stp) {
            const int k = stp * NPS + warp * GPW + gw;  // column of this nonzero in the batch
            const int64_t pos = p0 + c * kTcKC + k;
            bool v = pos < p1;
            int64_t s = 0;
            if (v) v = sample_at(a, a.base + pos, s);
            int32_t ik[kMaxOrder];
            int32_t in = 0;
#pragma unroll
            for (int q = 0; q < kMaxOrder; ++q) {
                ik[q] = 0;
                if (v && q < a.N) {
                    ik[q] = __ldg(a.idx[q] + s);
                    if ((uint32_t)ik[q] >= (uint32_t)a.dims[q]) {
                        atomicOr(a.err, kErrIndex);
                        v = false;
                    }
                    if (q == a.n) in = ik[q];
                }
            }
            const float x = v ? __ldg(a.val + s) : 0.f;
            float4 p = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
            for (int k0 = 0; k0 < kMaxOrder; k0 += 4) {
                if (k0 < a.N) {
                    float4 cr[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = k0 + u;
                        cr[u] = (v && q < a.N && q != a.n)
                                    ? ldC<CT>(a.C[q], (int64_t)ik[q] * R + 4 * sub)
                                    : make_float4(1.f, 1.f, 1.f, 1.f);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) mul4(p, cr[u]);
                }
            }
            float av[JL];
#pragma unroll
            for (int q = 0; q < JL; ++q) av[q] = 0.f;
            if (v) load_run<JL>(a.A + (int64_t)in * J + sub * JL, av);
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
            const float xh = group_sum<T>(dot);
            const float e = v ? x - xh : 0.f;
            // operand entries of column k (zero for positions past the span)
            const uint32_t kcol = (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 2u;
#pragma unroll
            for (int q = 0; q < JL; ++q) {
                const int j = sub * JL + q;
                *reinterpret_cast<__nv_bfloat16 *>(tA + (j >> 3) * 1024 + (j & 7) * 16 + kcol) =
                    __float2bfloat16_rn(e * av[q]);
            }
            const float pr[4] = {v ? p.x : 0.f, v ? p.y : 0.f, v ? p.z : 0.f, v ? p.w : 0.f};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = 4 * sub + q;
                *reinterpret_cast<__nv_bfloat16 *>(tB + (r >> 3) * 1024 + (r & 7) * 16 + kcol) =
                    __float2bfloat16_rn(pr[q]);
            }
        }
        tc::fence_async_smem();  // operand writes -> the tensor cores' view of shared memory
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_addr(tA), b0 = tc::smem_addr(tB);
#pragma unroll
            for (int kk = 0; kk < kTcKC / 16; ++kk)
                tc::mma_bf16(tmem, tc::desc_kmajor(a0 + kk * 256u, 128u, 1024u),
                             tc::desc_kmajor(b0 + kk * 256u, 128u, 1024u), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(&bar_mma[buf]);
        }
    }
    // the last commit completes once every MMA of the block has
    const int64_t last = c - 1;
    if (ok && last >= 0)
        ok = __syncthreads_and(
            tc::mbar_wait(&bar_mma[last & 1], (uint32_t)((last >> 1) & 1), wait_ns));
    if (!ok) {
        // a wait ran out: flag it, then wait once more, with the full bound, for
        // the MMAs this block issued before anything reads or frees tensor memory
        if (threadIdx.x == 0) {
            atomicOr(a.err, kErrWait);
            if (last >= 0) tc::mbar_wait(&bar_mma[last & 1], (uint32_t)((last >> 1) & 1));
        }
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) {
        // accumulator rows j < J_n <= 32 live in tensor-memory lanes 0..31; a
        // block whose wait ran out contributes zeros
#pragma unroll
        for (int h = 0; h < R / 16; ++h) {
            float g[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) g[q] = 0.f;
            if (ok && last >= 0) tc::tmem_ld16(tmem + 16u * h, g);
            if (lane < J) {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    partials[(int64_t)blockIdx.x * JR + lane * R + 16 * h + q] = g[q];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_free(tmem);
    }
}

bool core_tc_supported(int J, int R) { return (R == 16 || R == 32) && 4 * J >= R; }

cudaError_t launch_core_tc(const PassArgs &a, int J, int R, float *partials, int nblk,
                           uint64_t wait_ns, cudaStream_t st) {
    if (!core_tc_supported(J, R)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kernel) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcCoreSmem);
        if (e == cudaSuccess) kernel<<<nblk, kTcCoreThreads, kTcCoreSmem, st>>>(a, partials, wait_ns);
    };
    switch (R * 100 + J) {
        case 1604: go(k_core_grad_tc<16, 4, __nv_bfloat16>); break;
        case 1608: go(k_core_grad_tc<16, 8, __nv_bfloat16>); break;
        case 1616: go(k_core_grad_tc<16, 16, __nv_bfloat16>); break;
        case 1632: go(k_core_grad_tc<16, 32, __nv_bfloat16>); break;
        case 3208: go(k_core_grad_tc<32, 8, __nv_bfloat16>); break;
        case 3216: go(k_core_grad_tc<32, 16, __nv_bfloat16>); break;
        case 3232: go(k_core_grad_tc<32, 32, __nv_bfloat16>); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_core_apply(a.B, partials, nblk, J * R, a.count, a.lr, a.lam, st);
}

}  // namespace sft
