// sft_api.cu -- host side of the C ABI declared in include/sft.h: argument
// validation, workspace carving and the launch sequence of each call.
// Nothing here computes on the host; every step of the method is a kernel.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>

#include "sft_internal.cuh"

using namespace sft;

struct sft_ctx {
    int N = 0;
    int R = 0;
    int deterministic = 0;
    int cbf16 = 0;  // cached products stored as bfloat16 (SFT_BF16)
    int64_t dims[kMaxOrder] = {};
    int32_t J[kMaxOrder] = {};
    float *A[kMaxOrder] = {};
    float *B[kMaxOrder] = {};
    float *C[kMaxOrder] = {};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 1;
    // workspace pieces
    int *err = nullptr;
    double *loss_out = nullptr;
    double *loss_partials = nullptr;
    int loss_max_blocks = 0;
    float *core_partials = nullptr;
    int core_max_blocks = 0;
    DetFactorWs det{};
    int64_t det_max_chunks = 0;
    int jmax = 0;
    int64_t launches = 0;
    cudaStream_t aux[2] = {nullptr, nullptr};  // forked streams of the slice factor pass
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int64_t slice_tile = 0;        // 0 = automatic
    int64_t slice_max_direct = 0;  // 0 = automatic
    int64_t slice_lseq_mode[kMaxOrder] = {};  // per-mode choice of sft_autotune_slices (0 = none)
    int tensor_cores = 1;  // tcgen05 refresh / core gradient for bfloat16 cached products
    uint64_t tc_wait_ns = 2000000000ull;  // limit of the tensor-core kernels' waits
    int long_slices = SFT_LONG_MAPS;      // how the slice factor pass runs long slices
    int blocked_chains = 1;               // long chains of the fiber pass in 32-position blocks
    std::string last_error;
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool supported_rank(int v) { return v == 4 || v == 8 || v == 16 || v == 32; }

int device_sms(int *device_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (device_out) *device_out = dev;
    return sms;
}

// Fixed part of the workspace: error flag, loss output and partials, core
// partials.  Followed by the deterministic-factor chunk arrays.
struct Layout {
    size_t err, loss_out, loss_partials, core_partials, det;
    size_t fixed_bytes;
    size_t per_chunk_bytes;
};

Layout make_layout(int sms, int jmax, int R) {
    Layout L{};
    size_t off = 0;
    L.err = off;
    off = align_up(off + sizeof(int));
    L.loss_out = off;
    off = align_up(off + 2 * sizeof(double));
    L.loss_partials = off;
    off = align_up(off + (size_t)sms * 8 * 2 * sizeof(double));
    L.core_partials = off;
    off = align_up(off + (size_t)sms * 4 * jmax * R * sizeof(float));
    L.det = off;
    L.fixed_bytes = off;
    L.per_chunk_bytes = (size_t)kDetChunk * sizeof(int32_t)          // part_row
                        + (size_t)kDetChunk * jmax * sizeof(float)   // part_sum
                        + sizeof(int32_t);                           // seg_count
    return L;
}

const char *check_config(const sft_config *cfg, sft_status *st) {
    *st = SFT_EINVAL;
    if (!cfg) return "config is NULL";
    if (cfg->order < 2 || cfg->order > kMaxOrder) return "order must be in [2, 16]";
    if (!cfg->dims || !cfg->J) return "dims / J arrays are NULL";
    if (cfg->R < 1) return "R must be positive";
    for (int n = 0; n < cfg->order; ++n) {
        if (cfg->dims[n] < 1 || cfg->dims[n] > 0x7fffffffLL) return "each I_n must be in [1, 2^31)";
        if (cfg->J[n] < 1) return "each J_n must be positive";
    }
    if (cfg->prec != SFT_FP32 && cfg->prec != SFT_BF16) return "unknown precision";
    *st = SFT_ENOTSUP;
    if (!supported_rank(cfg->R)) return "R must be one of 4, 8, 16, 32";
    for (int n = 0; n < cfg->order; ++n) {
        if (!supported_rank(cfg->J[n])) return "each J_n must be one of 4, 8, 16, 32";
        if (4 * cfg->J[n] < cfg->R) return "4 * J_n must be >= R";
    }
    *st = SFT_OK;
    return nullptr;
}

sft_status fail(sft_ctx *c, sft_status st, const std::string &msg) {
    if (c) c->last_error = msg;
    return st;
}

sft_status cuda_fail(sft_ctx *c, cudaError_t e, const char *where) {
    return fail(c, SFT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Common validation of a pass over a COO set.
sft_status check_set(sft_ctx *c, const int32_t *const *idx, const float *val, int64_t nnz) {
    if (!idx) return fail(c, SFT_EINVAL, "idx array is NULL");
    for (int k = 0; k < c->N; ++k)
        if (!idx[k] && nnz > 0) return fail(c, SFT_EINVAL, "idx[k] is NULL");
    if (!val && nnz > 0) return fail(c, SFT_EINVAL, "val is NULL");
    if (nnz < 0 || nnz > 0x7fffffffLL) return fail(c, SFT_EINVAL, "nnz must be in [0, 2^31)");
    return SFT_OK;
}

PassArgs pass_args(const sft_ctx *c, int mode, const int32_t *const *idx, const float *val,
                   const uint32_t *perm, int64_t nnz, float lr, float lam) {
    PassArgs a{};
    for (int k = 0; k < c->N; ++k) {
        a.idx[k] = idx[k];
        a.C[k] = c->C[k];
        a.dims[k] = (int32_t)c->dims[k];
    }
    a.N = c->N;
    a.n = mode;
    a.val = val;
    a.perm = perm;
    a.nnz = nnz;
    a.base = 0;
    a.count = nnz;
    if (mode >= 0) {
        a.A = c->A[mode];
        a.B = c->B[mode];
        int q = 0;
        for (int k = 0; k < c->N; ++k) {
            if (k == mode) continue;
            a.oidx[q] = idx[k];
            a.oC[q] = c->C[k];
            a.odims[q] = (int32_t)c->dims[k];
            if (!l2_only_rows(c->dims[k], c->R, c->cbf16)) a.ol1 |= 1u << q;
            ++q;
        }
    }
    a.lr = lr;
    a.lam = lam;
    a.err = c->err;
    a.cbf16 = c->cbf16;
    return a;
}

}  // namespace

extern "C" {

size_t sft_workspace_bytes(const sft_config *cfg, int64_t max_batch) {
    sft_status st;
    if (check_config(cfg, &st)) return 0;
    int sms = device_sms(nullptr);
    if (sms < 1) return 0;
    int jmax = 0;
    for (int n = 0; n < cfg->order; ++n) jmax = cfg->J[n] > jmax ? cfg->J[n] : jmax;
    Layout L = make_layout(sms, jmax, cfg->R);
    int64_t b = max_batch < 1 ? 1 : (max_batch > kDetMaxBatch ? kDetMaxBatch : max_batch);
    int64_t chunks = (b + kDetChunk - 1) / kDetChunk;
    return L.fixed_bytes + (size_t)chunks * L.per_chunk_bytes + kAlign;
}

sft_status sft_init(const sft_config *cfg, float *const *A, float *const *B, void *const *C,
                    void *const *A_lo, void *workspace, size_t workspace_bytes, sft_ctx **out) {
    if (!out) return SFT_EINVAL;
    *out = nullptr;
    sft_status st;
    if (check_config(cfg, &st)) return st;
    if (!A || !B || !C) return SFT_EINVAL;
    if (A_lo) return SFT_EINVAL;
    for (int n = 0; n < cfg->order; ++n) {
        if (!A[n] || !B[n] || !C[n]) return SFT_EINVAL;
        if (!aligned16(A[n]) || !aligned16(B[n]) || !aligned16(C[n])) return SFT_EINVAL;
    }
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0) return SFT_EINVAL;
    int device = 0;
    int sms = device_sms(&device);
    if (sms < 1) return SFT_ECUDA;
    sft_ctx *c = new (std::nothrow) sft_ctx;
    if (!c) return SFT_ENOMEM;
    c->N = cfg->order;
    c->R = cfg->R;
    c->deterministic = cfg->deterministic ? 1 : 0;
    c->cbf16 = cfg->prec == SFT_BF16 ? 1 : 0;
    c->stream = (cudaStream_t)cfg->stream;
    c->device = device;
    c->sms = sms;
    for (int n = 0; n < c->N; ++n) {
        c->dims[n] = cfg->dims[n];
        c->J[n] = cfg->J[n];
        c->A[n] = A[n];
        c->B[n] = B[n];
        c->C[n] = (float *)C[n];
        c->jmax = c->J[n] > c->jmax ? c->J[n] : c->jmax;
    }
    Layout L = make_layout(sms, c->jmax, c->R);
    if (workspace_bytes < L.fixed_bytes + L.per_chunk_bytes) {
        delete c;
        return SFT_ENOMEM;
    }
    char *ws = (char *)workspace;
    c->err = (int *)(ws + L.err);
    c->loss_out = (double *)(ws + L.loss_out);
    c->loss_partials = (double *)(ws + L.loss_partials);
    c->loss_max_blocks = sms * 8;
    c->core_partials = (float *)(ws + L.core_partials);
    c->core_max_blocks = sms * 4;
    c->det_max_chunks = (int64_t)((workspace_bytes - L.fixed_bytes) / L.per_chunk_bytes);
    if (c->det_max_chunks * kDetChunk > kDetMaxBatch) c->det_max_chunks = kDetMaxBatch / kDetChunk;
    char *d = ws + L.det;
    c->det.part_row = (int32_t *)d;
    d += (size_t)c->det_max_chunks * kDetChunk * sizeof(int32_t);
    c->det.part_sum = (float *)d;
    d += (size_t)c->det_max_chunks * kDetChunk * c->jmax * sizeof(float);
    c->det.seg_count = (int32_t *)d;
    cudaError_t e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) {
        delete c;
        return SFT_ECUDA;
    }
    // auxiliary streams for the concurrent kernels of a slice factor pass; if
    // they cannot be created everything runs on the caller's stream
    bool aux_ok = true;
    // aux[0]: chains; aux[1]: maps, the longest of the three kernels, at the
    // highest stream priority so that its blocks are scheduled first
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        prio_greatest = prio_least = 0;
    }
    aux_ok = cudaStreamCreateWithFlags(&c->aux[0], cudaStreamNonBlocking) == cudaSuccess;
    if (aux_ok)
        aux_ok = cudaStreamCreateWithPriority(&c->aux[1], cudaStreamNonBlocking, prio_greatest) ==
                 cudaSuccess;
    for (int i = 0; i < 3 && aux_ok; ++i)
        aux_ok = cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!aux_ok) {
        cudaGetLastError();
        for (int i = 0; i < 2; ++i) if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
        for (int i = 0; i < 3; ++i) if (c->ev[i]) cudaEventDestroy(c->ev[i]);
        c->aux[0] = c->aux[1] = nullptr;
        c->ev[0] = c->ev[1] = c->ev[2] = nullptr;
    }
    *out = c;
    return SFT_OK;
}

sft_status sft_refresh_C(sft_ctx *c, int32_t mode) {
    if (!c) return SFT_EINVAL;
    if (mode < -1 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    for (int n = 0; n < c->N; ++n) {
        if (mode >= 0 && n != mode) continue;
        cudaError_t e;
        if (c->cbf16 && c->tensor_cores && refresh_tc_supported(c->J[n], c->R))
            e = launch_refresh_tc(c->A[n], c->B[n], c->C[n], c->dims[n], c->J[n], c->R, c->err,
                                  c->tc_wait_ns, c->stream, c->sms);
        else
            e = launch_refresh(c->A[n], c->B[n], c->C[n], c->dims[n], c->J[n], c->R,
                               c->cbf16 != 0, c->stream, c->sms);
        c->launches += 1;
        if (e != cudaSuccess) return cuda_fail(c, e, "refresh launch");
    }
    return SFT_OK;
}

sft_status sft_update_factors(sft_ctx *c, int32_t mode, const int32_t *const *idx,
                              const float *val, const uint32_t *perm, int64_t nnz, int64_t batch,
                              float lr, float lambda) {
    if (!c) return SFT_EINVAL;
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    sft_status st = check_set(c, idx, val, nnz);
    if (st != SFT_OK) return st;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return fail(c, SFT_EINVAL, "lr / lambda not finite");
    if (nnz == 0) return SFT_OK;
    PassArgs a = pass_args(c, mode, idx, val, perm, nnz, lr, lambda);
    if (!c->deterministic) {
        cudaError_t e = launch_factor_hogwild(a, c->J[mode], c->R, c->stream, c->sms);
        c->launches += 1;
        if (e != cudaSuccess) return cuda_fail(c, e, "factor launch");
        return SFT_OK;
    }
    if (batch < 1) return fail(c, SFT_EINVAL, "batch must be >= 1");
    if (batch > c->det_max_chunks * kDetChunk)
        return fail(c, SFT_ENOTSUP, "deterministic factor batch larger than the workspace allows "
                                    "(at most 16384 and the max_batch given to sft_workspace_bytes)");
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        a.base = b0;
        a.count = nnz - b0 < batch ? nnz - b0 : batch;
        cudaError_t e = launch_factor_det(a, c->J[mode], c->R, c->det, c->stream);
        c->launches += 2;
        if (e != cudaSuccess) return cuda_fail(c, e, "deterministic factor launch");
    }
    return SFT_OK;
}

sft_status sft_update_core(sft_ctx *c, int32_t mode, const int32_t *const *idx, const float *val,
                           const uint32_t *perm, int64_t nnz, int64_t batch, float lr,
                           float lambda) {
    if (!c) return SFT_EINVAL;
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    sft_status st = check_set(c, idx, val, nnz);
    if (st != SFT_OK) return st;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return fail(c, SFT_EINVAL, "lr / lambda not finite");
    if (batch < 1) return fail(c, SFT_EINVAL, "batch must be >= 1");
    if (nnz == 0) return SFT_OK;
    PassArgs a = pass_args(c, mode, idx, val, perm, nnz, lr, lambda);
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        a.base = b0;
        a.count = nnz - b0 < batch ? nnz - b0 : batch;
        int nblk = core_blocks_for(a.count, c->sms);
        if (nblk > c->core_max_blocks) nblk = c->core_max_blocks;
        const bool tc = c->cbf16 && c->tensor_cores && core_tc_supported(c->J[mode], c->R);
        cudaError_t e = tc ? launch_core_tc(a, c->J[mode], c->R, c->core_partials, nblk,
                                            c->tc_wait_ns, c->stream)
                           : launch_core(a, c->J[mode], c->R, c->core_partials, nblk, c->stream);
        c->launches += 2;
        if (e != cudaSuccess) return cuda_fail(c, e, "core launch");
    }
    return SFT_OK;
}

static sft_status loss_enqueue(sft_ctx *c, const int32_t *const *idx, const float *val,
                               int64_t nnz, double *out2) {
    sft_status st = check_set(c, idx, val, nnz);
    if (st != SFT_OK) return st;
    PassArgs a = pass_args(c, -1, idx, val, nullptr, nnz, 0.f, 0.f);
    int nblk = loss_blocks_for(nnz, c->sms);
    if (nblk > c->loss_max_blocks) nblk = c->loss_max_blocks;
    cudaError_t e = launch_loss(a, c->R, c->loss_partials, nblk, out2, c->stream);
    c->launches += 2;
    if (e != cudaSuccess) return cuda_fail(c, e, "loss launch");
    return SFT_OK;
}

static sft_status read_flag(sft_ctx *c) {
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the error flag");
    if (flag) {
        cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
        cudaStreamSynchronize(c->stream);
        std::string m = "a kernel skipped bad data:";
        if (flag & kErrIndex) m += " coordinate out of range;";
        if (flag & kErrPerm) m += " permutation entry >= nnz;";
        if (flag & kErrWait) {
            m += " a tensor-core kernel gave up waiting for its copies / MMAs;";
            return fail(c, SFT_ETIMEOUT, m);
        }
        return fail(c, SFT_EINVAL, m);
    }
    return SFT_OK;
}

sft_status sft_loss(sft_ctx *c, const int32_t *const *idx, const float *val, int64_t nnz,
                    double *sse, double *sae) {
    if (!c) return SFT_EINVAL;
    if (!sse || !sae) return fail(c, SFT_EINVAL, "sse / sae are NULL");
    sft_status st = loss_enqueue(c, idx, val, nnz, c->loss_out);
    if (st != SFT_OK) return st;
    double h[2] = {0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(h, c->loss_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "loss readback");
    st = read_flag(c);
    if (st != SFT_OK) return st;
    *sse = h[0];
    *sae = h[1];
    return SFT_OK;
}

sft_status sft_loss_async(sft_ctx *c, const int32_t *const *idx, const float *val, int64_t nnz,
                          double *out2) {
    if (!c) return SFT_EINVAL;
    if (!out2) return fail(c, SFT_EINVAL, "out2 is NULL");
    return loss_enqueue(c, idx, val, nnz, out2);
}

sft_status sft_predict(sft_ctx *c, const int32_t *const *idx, int64_t nnz, float *out) {
    if (!c) return SFT_EINVAL;
    if (!idx) return fail(c, SFT_EINVAL, "idx array is NULL");
    for (int k = 0; k < c->N; ++k)
        if (!idx[k] && nnz > 0) return fail(c, SFT_EINVAL, "idx[k] is NULL");
    if (!out && nnz > 0) return fail(c, SFT_EINVAL, "out is NULL");
    if (nnz < 0 || nnz > 0x7fffffffLL) return fail(c, SFT_EINVAL, "nnz must be in [0, 2^31)");
    if (nnz == 0) return SFT_OK;
    PassArgs a = pass_args(c, -1, idx, nullptr, nullptr, nnz, 0.f, 0.f);
    cudaError_t e = launch_predict(a, c->R, out, c->stream, c->sms);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "predict launch");
    return SFT_OK;
}

sft_status sft_loss_grad_C(sft_ctx *c, const int32_t *const *idx, const float *val, int64_t nnz,
                           float *const *dC, int32_t accumulate, double *loss_out) {
    if (!c) return SFT_EINVAL;
    sft_status st = check_set(c, idx, val, nnz);
    if (st != SFT_OK) return st;
    if (dC)
        for (int n = 0; n < c->N; ++n)
            if (!dC[n] || !aligned16(dC[n]))
                return fail(c, SFT_EINVAL, "dC[n] is NULL or not 16-byte aligned");
    if (!loss_out || ((uintptr_t)loss_out & 7u)) return fail(c, SFT_EINVAL, "loss_out is NULL or misaligned");
    PassArgs a = pass_args(c, -1, idx, val, nullptr, nnz, 0.f, 0.f);
    GradBufs g{};
    for (int n = 0; n < c->N; ++n) {
        g.dC[n] = dC ? dC[n] : nullptr;
        g.dims[n] = c->dims[n];
    }
    int nblk = loss_blocks_for(nnz, c->sms);
    if (nblk > c->loss_max_blocks) nblk = c->loss_max_blocks;
    cudaError_t e = launch_loss_grad(a, g, c->R, accumulate != 0, c->loss_partials, nblk, loss_out,
                                     c->stream, c->sms, &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "loss gradient launch");
    return SFT_OK;
}

sft_status sft_grad_AB(sft_ctx *c, const float *const *dC, const double *scale, float *const *gA,
                       float *const *gB) {
    if (!c) return SFT_EINVAL;
    if (!dC || !gA || !gB) return fail(c, SFT_EINVAL, "dC / gA / gB array is NULL");
    for (int n = 0; n < c->N; ++n) {
        if (!dC[n] || !gA[n] || !gB[n]) return fail(c, SFT_EINVAL, "dC[n] / gA[n] / gB[n] is NULL");
        if (!aligned16(dC[n])) return fail(c, SFT_EINVAL, "dC[n] is not 16-byte aligned");
    }
    if (scale && ((uintptr_t)scale & 7u)) return fail(c, SFT_EINVAL, "scale is misaligned");
    for (int n = 0; n < c->N; ++n) {
        cudaError_t e = launch_grad_project(c->A[n], c->B[n], dC[n], c->dims[n], c->J[n], c->R,
                                            scale, gA[n], gB[n], c->core_partials,
                                            c->core_max_blocks, c->stream, c->sms, &c->launches);
        if (e != cudaSuccess) return cuda_fail(c, e, "gradient projection launch");
    }
    return SFT_OK;
}

sft_status sft_epoch(sft_ctx *c, const int32_t *const *idx, const float *val, int64_t nnz,
                     const uint32_t *const *perm_factor, const uint32_t *const *perm_core,
                     int64_t batch_factor, int64_t batch_core, float lr_A, float lambda_A,
                     float lr_B, float lambda_B) {
    if (!c) return SFT_EINVAL;
    for (int n = 0; n < c->N; ++n) {
        sft_status st = sft_update_factors(c, n, idx, val, perm_factor ? perm_factor[n] : nullptr,
                                           nnz, batch_factor, lr_A, lambda_A);
        if (st != SFT_OK) return st;
        st = sft_refresh_C(c, n);
        if (st != SFT_OK) return st;
    }
    for (int n = 0; n < c->N; ++n) {
        sft_status st = sft_update_core(c, n, idx, val, perm_core ? perm_core[n] : nullptr, nnz,
                                        batch_core, lr_B, lambda_B);
        if (st != SFT_OK) return st;
        st = sft_refresh_C(c, n);
        if (st != SFT_OK) return st;
    }
    return SFT_OK;
}

// ----------------------------------------------------------------------------- slices

static int64_t slice_W(const sft_ctx *c, int64_t nnz) {
    return c->slice_tile > 0 ? c->slice_tile : slice_tile_length(nnz, c->sms);
}

static int64_t slice_core_W(const sft_ctx *c, int64_t nnz) {
    return c->slice_tile > 0 ? c->slice_tile : slice_core_tile_length(nnz, c->sms);
}

// Chain length of the slice factor pass: a crossing slice of at most Lseq
// nonzeros is run whole as one element-by-element chain, a longer one runs its
// first Lseq nonzeros as a chain and the rest through composed maps.  Lseq is
// 0 (every crossing slice through maps) or at least one tile (so that a tile
// holds at most one map piece per slot).  The default, 2 tiles, is replaced per
// mode by sft_autotune_slices.
static int64_t slice_Lseq(const sft_ctx *c, int mode, int64_t W, int64_t nnz) {
    (void)nnz;
    const int64_t tuned = c->slice_lseq_mode[mode];
    int64_t L;
    if (tuned != 0) L = tuned < 0 ? 0 : tuned;
    else if (c->slice_max_direct > 0) L = c->slice_max_direct;
    else if (c->slice_max_direct < 0) L = 0;
    else L = 2 * W;
    return L > 0 && L < W ? W : L;
}

size_t sft_slices_scratch_bytes(int64_t nnz) {
    if (nnz < 0) return 0;
    return (size_t)slice_sort_length(nnz) * sizeof(unsigned long long);
}

sft_status sft_group_slices(sft_ctx *c, int32_t mode, const int32_t *const *idx, const float *val,
                            const uint32_t *perm, int64_t nnz, int32_t *const *out_idx,
                            float *out_val, int32_t *out_row_ptr, void *scratch,
                            size_t scratch_bytes) {
    if (!c) return SFT_EINVAL;
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    sft_status st = check_set(c, idx, val, nnz);
    if (st != SFT_OK) return st;
    if (!out_idx || !out_val || !out_row_ptr) return fail(c, SFT_EINVAL, "output arrays are NULL");
    for (int k = 0; k < c->N; ++k)
        if (!out_idx[k]) return fail(c, SFT_EINVAL, "out_idx[k] is NULL");
    if (!scratch || scratch_bytes < sft_slices_scratch_bytes(nnz) || ((uintptr_t)scratch & 15u))
        return fail(c, SFT_EINVAL, "scratch missing, misaligned or smaller than sft_slices_scratch_bytes");
    PassArgs a = pass_args(c, mode, idx, val, perm, nnz, 0.f, 0.f);
    cudaError_t e = launch_group_slices(a, out_idx, out_val, out_row_ptr,
                                        (unsigned long long *)scratch, c->stream, c->sms,
                                        &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "slice layout launch");
    return SFT_OK;
}

sft_status sft_slices_expand_rows(sft_ctx *c, int32_t mode, const int32_t *row_ptr, int64_t nnz,
                                  int32_t *out) {
    if (!c) return SFT_EINVAL;
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    if (nnz < 0 || nnz > 0x7fffffffLL) return fail(c, SFT_EINVAL, "nnz must be in [0, 2^31)");
    if (nnz == 0) return SFT_OK;
    if (!row_ptr || !out) return fail(c, SFT_EINVAL, "row_ptr or out is NULL");
    cudaError_t e = launch_expand_rows(row_ptr, (int32_t)c->dims[mode], nnz, out, c->stream, c->sms);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "row expansion launch");
    return SFT_OK;
}

size_t sft_slices_workspace_bytes(const sft_ctx *c, int32_t mode, int64_t nnz) {
    if (!c || mode < 0 || mode >= c->N || nnz < 0) return 0;
    const int64_t W = slice_W(c, nnz);
    const int64_t ntiles = (nnz + W - 1) / W;
    // the piece maps, the pass's chain list, its piece list and its one-lane
    // work list
    return slice_workspace_total(ntiles, c->J[mode], c->dims[mode]);
}

static sft_status check_slices(sft_ctx *c, int32_t mode, const int32_t *const *sidx,
                               const float *sval, const int32_t *row_ptr, int64_t nnz) {
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    sft_status st = check_set(c, sidx, sval, nnz);
    if (st != SFT_OK) return st;
    if (!row_ptr) return fail(c, SFT_EINVAL, "row_ptr is NULL");
    return SFT_OK;
}

sft_status sft_update_factors_slices(sft_ctx *c, int32_t mode, const int32_t *const *sidx,
                                     const float *sval, const int32_t *row_ptr, int64_t nnz,
                                     float lr, float lambda, void *workspace,
                                     size_t workspace_bytes) {
    if (!c) return SFT_EINVAL;
    sft_status st = check_slices(c, mode, sidx, sval, row_ptr, nnz);
    if (st != SFT_OK) return st;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return fail(c, SFT_EINVAL, "lr / lambda not finite");
    if (nnz == 0) return SFT_OK;
    if (!workspace || workspace_bytes < sft_slices_workspace_bytes(c, mode, nnz) ||
        ((uintptr_t)workspace & 15u))
        return fail(c, SFT_EINVAL, "workspace missing, misaligned or smaller than sft_slices_workspace_bytes");
    PassArgs a = pass_args(c, mode, sidx, sval, nullptr, nnz, lr, lambda);
    const int64_t W = slice_W(c, nnz);
    SliceStreams ss{c->stream, c->aux[0], c->aux[1], c->ev[0], c->ev[1], c->ev[2]};
    cudaError_t e = launch_factor_slices(a, row_ptr, W, slice_Lseq(c, mode, W, nnz),
                                         c->long_slices == SFT_LONG_SUBSLICES, false,
                                         (float *)workspace,
                                         c->J[mode], c->R, ss, c->sms, &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "slice factor launch");
    return SFT_OK;
}

sft_status sft_update_core_slices(sft_ctx *c, int32_t mode, const int32_t *const *sidx,
                                  const float *sval, const int32_t *row_ptr, int64_t nnz,
                                  int64_t batch, float lr, float lambda) {
    if (!c) return SFT_EINVAL;
    sft_status st = check_slices(c, mode, sidx, sval, row_ptr, nnz);
    if (st != SFT_OK) return st;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return fail(c, SFT_EINVAL, "lr / lambda not finite");
    if (batch < 1) return fail(c, SFT_EINVAL, "batch must be >= 1");
    if (nnz == 0) return SFT_OK;
    PassArgs a = pass_args(c, mode, sidx, sval, nullptr, nnz, lr, lambda);
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        a.base = b0;
        a.count = nnz - b0 < batch ? nnz - b0 : batch;
        cudaError_t e = launch_core_slices(a, row_ptr, slice_core_W(c, a.count), c->J[mode], c->R,
                                           c->core_partials, c->core_max_blocks, c->stream, c->sms,
                                           &c->launches);
        if (e != cudaSuccess) return cuda_fail(c, e, "slice core launch");
    }
    return SFT_OK;
}

size_t sft_fibers_scratch_bytes(int64_t nnz) {
    if (nnz < 0) return 0;
    return (size_t)fiber_table_capacity(nnz) * 20 + 256;
}

sft_status sft_group_fibers(sft_ctx *c, int32_t mode, const int32_t *const *sidx, int64_t nnz,
                            int32_t *fid, int32_t *const *fcoord, int64_t *nfibers, void *scratch,
                            size_t scratch_bytes) {
    if (!c) return SFT_EINVAL;
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    if (!sidx) return fail(c, SFT_EINVAL, "sidx array is NULL");
    for (int k = 0; k < c->N; ++k)
        if (!sidx[k] && nnz > 0) return fail(c, SFT_EINVAL, "sidx[k] is NULL");
    if (nnz < 0 || nnz > 0x7fffffffLL) return fail(c, SFT_EINVAL, "nnz must be in [0, 2^31)");
    if (!nfibers) return fail(c, SFT_EINVAL, "nfibers is NULL");
    if ((!fid || !fcoord) && nnz > 0) return fail(c, SFT_EINVAL, "fid / fcoord are NULL");
    for (int k = 0; k < c->N && nnz > 0; ++k)
        if (k != mode && !fcoord[k]) return fail(c, SFT_EINVAL, "fcoord[k] is NULL for a mode k != mode");
    if (!scratch || scratch_bytes < sft_fibers_scratch_bytes(nnz) || ((uintptr_t)scratch & 15u))
        return fail(c, SFT_EINVAL, "scratch missing, misaligned or smaller than sft_fibers_scratch_bytes");
    // the fiber key is the exact linear index of the other modes' coordinates
    double prod = 1.0;
    for (int k = 0; k < c->N; ++k)
        if (k != mode) prod *= (double)c->dims[k];
    if (prod >= 4.0e18)
        return fail(c, SFT_ENOTSUP, "product of the other modes' lengths must be below 4e18");
    *nfibers = 0;
    if (nnz == 0) return SFT_OK;
    PassArgs a = pass_args(c, mode, sidx, nullptr, nullptr, nnz, 0.f, 0.f);
    cudaError_t e = launch_group_fibers(a, fid, fcoord, scratch, nfibers, c->stream, c->sms,
                                        &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "fiber layout");
    return read_flag(c);
}

sft_status sft_fibers_expand_coords(sft_ctx *c, int32_t mode, const int32_t *fid, int64_t nnz,
                                    const int32_t *const *fcoord, int64_t nfibers,
                                    int32_t *const *out_idx) {
    if (!c) return SFT_EINVAL;
    if (mode < 0 || mode >= c->N) return fail(c, SFT_EINVAL, "mode out of range");
    if (nnz < 0 || nnz > 0x7fffffffLL) return fail(c, SFT_EINVAL, "nnz must be in [0, 2^31)");
    if (nfibers < 0 || nfibers > nnz) return fail(c, SFT_EINVAL, "nfibers must be in [0, nnz]");
    if (nnz == 0) return SFT_OK;
    if (!fid || !fcoord || !out_idx) return fail(c, SFT_EINVAL, "fid, fcoord or out_idx is NULL");
    for (int k = 0; k < c->N; ++k)
        if (k != mode && (!fcoord[k] || !out_idx[k]))
            return fail(c, SFT_EINVAL, "fcoord[k] or out_idx[k] is NULL for a mode k != mode");
    cudaError_t e = launch_fiber_expand(c->N, mode, fid, nnz, nfibers, fcoord, out_idx, c->stream,
                                        c->sms);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "fiber coordinate expansion launch");
    return SFT_OK;
}

sft_status sft_update_factors_fibers(sft_ctx *c, int32_t mode, const int32_t *const *sidx,
                                     const float *sval, const int32_t *row_ptr, int64_t nnz,
                                     const int32_t *fid, const int32_t *const *fcoord,
                                     int64_t nfibers,
                                     float *V, float lr, float lambda, void *workspace,
                                     size_t workspace_bytes) {
    if (!c) return SFT_EINVAL;
    sft_status st = check_slices(c, mode, sidx, sval, row_ptr, nnz);
    if (st != SFT_OK) return st;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return fail(c, SFT_EINVAL, "lr / lambda not finite");
    if (nnz == 0) return SFT_OK;
    if (!fid || !fcoord || !V || nfibers < 0 || nfibers > nnz)
        return fail(c, SFT_EINVAL, "fid / fcoord / V missing or nfibers outside [0, nnz]");
    for (int k = 0; k < c->N; ++k)
        if (k != mode && !fcoord[k]) return fail(c, SFT_EINVAL, "fcoord[k] is NULL for a mode k != mode");
    if (!aligned16(V)) return fail(c, SFT_EINVAL, "V must be 16-byte aligned");
    if (!workspace || workspace_bytes < sft_slices_workspace_bytes(c, mode, nnz) ||
        ((uintptr_t)workspace & 15u))
        return fail(c, SFT_EINVAL, "workspace missing, misaligned or smaller than sft_slices_workspace_bytes");
    PassArgs a = pass_args(c, mode, sidx, sval, nullptr, nnz, lr, lambda);
    const int64_t W = slice_W(c, nnz);
    SliceStreams ss{c->stream, c->aux[0], c->aux[1], c->ev[0], c->ev[1], c->ev[2]};
    cudaError_t e = launch_factor_fibers(a, row_ptr, W, slice_Lseq(c, mode, W, nnz),
                                         c->long_slices == SFT_LONG_SUBSLICES,
                                         c->blocked_chains != 0, (float *)workspace,
                                         fid, fcoord, nfibers, V, c->J[mode], c->R, ss, c->sms,
                                         &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "fiber factor launch");
    return SFT_OK;
}

sft_status sft_update_core_fibers(sft_ctx *c, int32_t mode, const int32_t *const *sidx,
                                  const float *sval, const int32_t *row_ptr, int64_t nnz,
                                  int64_t batch, const int32_t *fid, const int32_t *const *fcoord,
                                  int64_t nfibers, float *P, float lr, float lambda) {
    if (!c) return SFT_EINVAL;
    sft_status st = check_slices(c, mode, sidx, sval, row_ptr, nnz);
    if (st != SFT_OK) return st;
    if (!std::isfinite(lr) || !std::isfinite(lambda)) return fail(c, SFT_EINVAL, "lr / lambda not finite");
    if (batch < 1) return fail(c, SFT_EINVAL, "batch must be >= 1");
    if (nnz == 0) return SFT_OK;
    if (!fid || !fcoord || !P || nfibers < 0 || nfibers > nnz)
        return fail(c, SFT_EINVAL, "fid / fcoord / P missing or nfibers outside [0, nnz]");
    for (int k = 0; k < c->N; ++k)
        if (k != mode && !fcoord[k]) return fail(c, SFT_EINVAL, "fcoord[k] is NULL for a mode k != mode");
    if (!aligned16(P)) return fail(c, SFT_EINVAL, "P must be 16-byte aligned");
    PassArgs a = pass_args(c, mode, sidx, sval, nullptr, nnz, lr, lambda);
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        a.base = b0;
        a.count = nnz - b0 < batch ? nnz - b0 : batch;
        cudaError_t e = launch_core_fibers(a, row_ptr, slice_core_W(c, a.count), fid, fcoord, nfibers, P,
                                           c->J[mode], c->R, c->core_partials, c->core_max_blocks,
                                           c->stream, c->sms, &c->launches, b0 == 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "fiber core launch");
    }
    return SFT_OK;
}

sft_status sft_set_slice_tiling(sft_ctx *c, int64_t tile, int64_t max_direct) {
    if (!c) return SFT_EINVAL;
    if (tile < 0) return fail(c, SFT_EINVAL, "tile must be >= 0");
    c->slice_tile = tile;
    c->slice_max_direct = max_direct;  // < 0: every crossing slice goes through maps
    for (int n = 0; n < kMaxOrder; ++n) c->slice_lseq_mode[n] = 0;
    return SFT_OK;
}

sft_status sft_set_tensor_cores(sft_ctx *c, int32_t enable) {
    if (!c) return SFT_EINVAL;
    c->tensor_cores = enable ? 1 : 0;
    return SFT_OK;
}

sft_status sft_set_blocked_chains(sft_ctx *c, int32_t enable) {
    if (!c) return SFT_EINVAL;
    c->blocked_chains = enable ? 1 : 0;
    return SFT_OK;
}

sft_status sft_set_long_slices(sft_ctx *c, int32_t how) {
    if (!c) return SFT_EINVAL;
    if (how != SFT_LONG_MAPS && how != SFT_LONG_SUBSLICES)
        return fail(c, SFT_EINVAL, "long-slice mode must be SFT_LONG_MAPS or SFT_LONG_SUBSLICES");
    c->long_slices = how;
    return SFT_OK;
}

sft_status sft_set_tc_wait_limit(sft_ctx *c, int64_t limit_ns) {
    if (!c) return SFT_EINVAL;
    if (limit_ns < 0 || limit_ns > 60000000000LL)
        return fail(c, SFT_EINVAL, "tensor-core wait limit must be in [0, 60 s]");
    c->tc_wait_ns = (uint64_t)limit_ns;
    return SFT_OK;
}

sft_status sft_autotune_slices(sft_ctx *c, int32_t mode, const int32_t *const *sidx,
                               const float *sval, const int32_t *row_ptr, int64_t nnz,
                               const int32_t *fid, const int32_t *const *fcoord, int64_t nfibers,
                               float *V, float lr, float lambda, void *workspace,
                               size_t workspace_bytes, void *scratch, size_t scratch_bytes,
                               int64_t *lseq_out) {
    if (!c) return SFT_EINVAL;
    sft_status st = check_slices(c, mode, sidx, sval, row_ptr, nnz);
    if (st != SFT_OK) return st;
    const size_t abytes = (size_t)c->dims[mode] * c->J[mode] * sizeof(float);
    if (!scratch || scratch_bytes < abytes || ((uintptr_t)scratch & 15u))
        return fail(c, SFT_EINVAL, "scratch missing, misaligned or smaller than I_mode * J_mode floats");
    if (nnz == 0) return SFT_OK;
    const bool fibers = fid != nullptr;
    const int64_t W = slice_W(c, nnz);
    // candidate chain lengths (a slice up to it runs whole, a longer one runs
    // that many positions as its head): W and the default 2W, the powers of
    // two from 1024 to 65536 and the midpoints 1.5 x 2^k between them, and
    // every crossing slice whole
    int64_t cands[24];
    int nc = 0;
    cands[nc++] = W;
    cands[nc++] = 2 * W;
    for (int64_t L = 1024; L <= 65536; L *= 2) {
        if (L > 2 * W) cands[nc++] = L;
        if (L < 65536 && 3 * L / 2 > 2 * W) cands[nc++] = 3 * L / 2;
    }
    cands[nc++] = (int64_t)1 << 40;
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "event");
    if (cudaEventCreate(&t1) != cudaSuccess) {
        cudaEventDestroy(t0);
        return cuda_fail(c, cudaGetLastError(), "event");
    }
    const int64_t keep = c->slice_lseq_mode[mode];
    cudaError_t e = cudaMemcpyAsync(scratch, c->A[mode], abytes, cudaMemcpyDeviceToDevice, c->stream);
    float best = -1.f;
    int64_t best_L = 2 * W;
    for (int i = 0; i < nc && e == cudaSuccess && st == SFT_OK; ++i) {
        c->slice_lseq_mode[mode] = cands[i];
        for (int rep = 0; rep < 2 && st == SFT_OK; ++rep) {  // the second run is timed
            if (rep == 1) cudaEventRecord(t0, c->stream);
            st = fibers ? sft_update_factors_fibers(c, mode, sidx, sval, row_ptr, nnz, fid, fcoord,
                                                    nfibers, V, lr, lambda, workspace,
                                                    workspace_bytes)
                        : sft_update_factors_slices(c, mode, sidx, sval, row_ptr, nnz, lr, lambda,
                                                    workspace, workspace_bytes);
            if (rep == 1) cudaEventRecord(t1, c->stream);
            e = cudaMemcpyAsync(c->A[mode], scratch, abytes, cudaMemcpyDeviceToDevice, c->stream);
        }
        if (st != SFT_OK || e != cudaSuccess) break;
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && (best < 0.f || ms < best)) {
            best = ms;
            best_L = cands[i];
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != SFT_OK) {
        c->slice_lseq_mode[mode] = keep;
        return st;
    }
    if (e != cudaSuccess) {
        c->slice_lseq_mode[mode] = keep;
        return cuda_fail(c, e, "slice autotune");
    }
    c->slice_lseq_mode[mode] = best_L;
    if (lseq_out) *lseq_out = best_L;
    return read_flag(c);
}

sft_status sft_sync(sft_ctx *c, int64_t timeout_ms) {
    if (!c) return SFT_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(c, e, "stream query");
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (ms > timeout_ms) return fail(c, SFT_ETIMEOUT, "stream still busy at the timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return read_flag(c);
}

sft_status sft_set_stream(sft_ctx *c, void *stream) {
    if (!c) return SFT_EINVAL;
    c->stream = (cudaStream_t)stream;
    return SFT_OK;
}

const char *sft_last_error(const sft_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

int64_t sft_launch_count(const sft_ctx *c) { return c ? c->launches : 0; }

void sft_destroy(sft_ctx *c) {
    if (!c) return;
    for (int i = 0; i < 2; ++i) if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
    for (int i = 0; i < 3; ++i) if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    delete c;
}

}  // extern "C"
