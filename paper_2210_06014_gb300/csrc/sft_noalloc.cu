// sft_noalloc.cu -- a factor-pass entry point that allocates no device memory.
//
// Some callers cannot hand the library a workspace: for example a plugin
// running inside a host application that owns every byte of device memory
// through its own pool and forbids raw cudaMalloc/cudaFree, or a
// latency-critical loop that must not pay for (or synchronise on) a fresh
// allocation.  For them sft_update_factors_noalloc runs the deterministic
// minibatch factor pass (the same kernels as sft_update_factors with
// deterministic = 1) with its scratch -- the per-chunk row sums of a minibatch
// and the bad-data flag -- in a fixed array of device memory that is part of
// the library image itself.
#include <cmath>
#include <mutex>

#include "sft_internal.cuh"

using namespace sft;

namespace {

constexpr int kNoallocChunks = 16;                              // chunks of kDetChunk samples
constexpr int64_t kNoallocMaxBatch = kNoallocChunks * kDetChunk;  // 4096
constexpr int kNoallocJmax = 32;
constexpr int kNoallocMaxDevices = 64;

struct NoallocScratch {
    int err;
    int pad[63];
    int32_t part_row[kNoallocChunks * kDetChunk];
    float part_sum[kNoallocChunks * kDetChunk * kNoallocJmax];
    int32_t seg_count[kNoallocChunks];
};

std::mutex g_mu;
void *g_addr[kNoallocMaxDevices];  // device address of g_noalloc_scratch, per device

}  // namespace

// The shared scratch (about 529 KB; every GPU that loads the library keeps it
// until the process exits).  In host code this name is only a handle: its
// device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Device address of the scratch on the current device; looked up once per
// device (with that device current) and cached.
static cudaError_t scratch_on_current_device(NoallocScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = (NoallocScratch *)g_addr[dev];
    return cudaSuccess;
}

extern "C" sft_status sft_update_factors_noalloc(int32_t order, const int64_t *dims,
                                                 const int32_t *J, int32_t R, int32_t mode,
                                                 float *A_mode, const float *B_mode,
                                                 float *const *C, const int32_t *const *idx,
                                                 const float *val, const uint32_t *perm,
                                                 int64_t nnz, int64_t batch, float lr,
                                                 float lambda, void *stream) {
    if (order < 2 || order > kMaxOrder || !dims || !J || !C || !idx) return SFT_EINVAL;
    if (mode < 0 || mode >= order) return SFT_EINVAL;
    if (nnz < 0 || nnz > 0x7fffffffLL || batch < 1) return SFT_EINVAL;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return SFT_EINVAL;
    auto rank_ok = [](int v) { return v == 4 || v == 8 || v == 16 || v == 32; };
    if (!rank_ok(R) || !rank_ok(J[mode]) || 4 * J[mode] < R) return SFT_ENOTSUP;
    if (batch > kNoallocMaxBatch) return SFT_ENOTSUP;  // the scratch holds 4096-sample batches
    if (!A_mode || !B_mode || ((uintptr_t)A_mode & 15u) || ((uintptr_t)B_mode & 15u))
        return SFT_EINVAL;
    for (int k = 0; k < order; ++k) {
        if (dims[k] < 1 || dims[k] > 0x7fffffffLL) return SFT_EINVAL;
        if (!C[k] || ((uintptr_t)C[k] & 15u)) return SFT_EINVAL;
        if (nnz > 0 && !idx[k]) return SFT_EINVAL;
    }
    if (nnz > 0 && !val) return SFT_EINVAL;
    if (nnz == 0) return SFT_OK;

    cudaStream_t st = (cudaStream_t)stream;
    // The call reads the bad-data flag back and waits for the stream, which a
    // stream capture cannot hold: refuse before touching anything.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SFT_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return SFT_ENOTSUP;
    NoallocScratch *sc = nullptr;
    if (scratch_on_current_device(&sc) != cudaSuccess) return SFT_ECUDA;
    if (cudaMemsetAsync(&sc->err, 0, sizeof(int), st) != cudaSuccess) return SFT_ECUDA;

    PassArgs a{};
    for (int k = 0; k < order; ++k) {
        a.idx[k] = idx[k];
        a.C[k] = C[k];
        a.dims[k] = (int32_t)dims[k];
    }
    a.N = order;
    a.n = mode;
    a.val = val;
    a.perm = perm;
    a.nnz = nnz;
    a.A = A_mode;
    a.B = const_cast<float *>(B_mode);
    a.lr = lr;
    a.lam = lambda;
    a.err = &sc->err;
    DetFactorWs ws{sc->part_row, sc->part_sum, sc->seg_count};
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        a.base = b0;
        a.count = nnz - b0 < batch ? nnz - b0 : batch;
        if (launch_factor_det(a, J[mode], R, ws, st) != cudaSuccess) return SFT_ECUDA;
    }
    int flag = 0;
    if (cudaMemcpyAsync(&flag, &sc->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SFT_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SFT_ECUDA;
    return flag ? SFT_EINVAL : SFT_OK;
}
