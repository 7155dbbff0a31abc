/*
 * sft.h -- C ABI of the GB300 (sm_103a) sparse FastTucker SGD library.
 *
 * The library runs the hot path of cuFasterTucker (arXiv 2210.06014) in the
 * "reusable intermediates, COO storage" form the paper calls
 * cuFasterTucker_COO (Section "Experimental Settings"):
 *
 *   sft_refresh_C       C^(n) = A^(n) B^(n)             Algorithm 3; Algorithm 2
 *   sft_update_factors  SGD pass over A^(n)             Algorithm 4; Eq. (9), (10)
 *   sft_update_core     SGD pass over B^(n)             Algorithm 5; Eq. (9), (11)
 *   sft_loss            sum of squared / absolute       Section "Real-world accuracy"
 *                       residuals over a set            (test RMSE and MAE)
 *
 * Notation: a tensor of order N with mode lengths I_n, factor matrices
 * A^(n) (I_n x J_n), Kruskal-form core matrices B^(n) (J_n x R), cached
 * products C^(n) = A^(n) B^(n) (I_n x R).  A nonzero s has coordinates
 * (i_0 .. i_{N-1}) and value x_s; its prediction is
 *   x^_s = sum_r prod_k C^(k)[i_k][r]                    (Eq. (1) through Eq. (12)).
 *
 * Memory: every array is a *device* pointer owned by the caller (e.g. torch
 * tensors); the library borrows them and frees nothing it did not allocate.
 * Matrices are dense row-major, 16-byte aligned, with no padding: A[n] has
 * I_n*J_n float32, B[n] J_n*R float32, C[n] I_n*R float32 (bfloat16 with
 * SFT_BF16).  A COO set is given as
 * N device pointers idx[k] (int32, nnz entries each, 0 <= idx[k][s] < I_k) and
 * val (float32, nnz entries).  An optional permutation perm (uint32, nnz
 * entries, a permutation of 0..nnz-1) gives the order in which the nonzeros
 * are visited; NULL means storage order.
 *
 * Asynchrony: every call except sft_loss, sft_sync and sft_destroy only
 * enqueues kernels on the configured CUDA stream and returns.  Argument errors
 * are detected on the host before anything is launched (SFT_EINVAL).  Bad
 * data found by a kernel (an index out of range, a permutation entry >= nnz) is
 * skipped by that kernel and recorded in a device flag that sft_sync and
 * sft_loss report as SFT_EINVAL.  No call aborts, throws or hangs: sft_sync
 * gives up after its timeout with SFT_ETIMEOUT.
 *
 * Supported shapes on the CUDA path: 2 <= N <= 16, R in {4, 8, 16, 32},
 * J_n in {4, 8, 16, 32} with 4*J_n >= R, I_n < 2^31, nnz < 2^31.  Other shapes
 * return SFT_ENOTSUP.
 */
#ifndef SFT_H
#define SFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFT_MAX_ORDER 16

typedef struct sft_ctx sft_ctx; /* opaque; created by sft_init, freed by sft_destroy */

typedef enum {
    SFT_OK = 0,
    SFT_EINVAL = 1,   /* bad argument, or bad data flagged by a kernel */
    SFT_ENOMEM = 2,   /* workspace too small / host allocation failed */
    SFT_ECUDA = 3,    /* a CUDA runtime call failed (message in sft_last_error) */
    SFT_ETIMEOUT = 4, /* sft_sync gave up before the stream drained */
    SFT_ENOTSUP = 5   /* shape or mode not supported by the CUDA path */
} sft_status;

typedef enum {
    SFT_FP32 = 0, /* A, B, C float32 */
    SFT_BF16 = 1  /* C stored as bfloat16 (rounded to nearest even by sft_refresh_C);
                     A and B stay float32 (master copies).  The gathers widen C to
                     float32; the refresh and the COO core gradient run on tensor
                     cores (see sft_set_tensor_cores), everything else in float32. */
} sft_precision;

typedef struct {
    int32_t order;         /* N, 2..16 */
    const int64_t *dims;   /* host array [N]: I_n */
    const int32_t *J;      /* host array [N]: J_n */
    int32_t R;             /* Kruskal rank of the core */
    int32_t prec;          /* sft_precision */
    int32_t deterministic; /* 1: minibatch rule with fixed-order sums (bitwise
                              reproducible, matches the FP64 oracle);
                              0: Hogwild factor rows (Algorithm 4 style) */
    void *stream;          /* cudaStream_t to enqueue on (NULL = legacy stream) */
} sft_config;

/* Bytes of device workspace sft_init needs for this configuration when no
 * minibatch is larger than max_batch.  Returns 0 for an invalid config. */
size_t sft_workspace_bytes(const sft_config *cfg, int64_t max_batch);

/* Create a context.  A, B, C: host arrays of N device pointers (see header
 * comment for layout).  A_lo must be NULL (reserved; the bfloat16 form keeps
 * no copy of A).
 * workspace: device buffer of at least sft_workspace_bytes(cfg, max_batch)
 * bytes, 256-byte aligned, owned by the caller and not touched by anyone else
 * while the context lives.  The context copies cfg and the pointer arrays.
 * On success *out receives the context; on failure *out is NULL. */
sft_status sft_init(const sft_config *cfg, float *const *A, float *const *B, void *const *C,
                    void *const *A_lo, void *workspace, size_t workspace_bytes, sft_ctx **out);

/* C^(mode) = A^(mode) B^(mode) (Algorithm 3); mode = -1 refreshes every mode.
 * The caller refreshes a mode after each pass over it, as Algorithm 2 does. */
sft_status sft_refresh_C(sft_ctx *ctx, int32_t mode);

/* One SGD pass over A^(mode) (Algorithm 2, factor module; Eq. (9)-(10)).
 * For each visited nonzero s: p_r = prod_{k != mode} C^(k)[i_k][r],
 * v = B^(mode) p, e = x_s - a_{i_mode} . v, and the row moves by
 * lr * (e v - lambda a_{i_mode}).
 *   deterministic = 1: the visit order is cut into minibatches of `batch`
 *     samples (last one shorter); inside a minibatch every prediction uses the
 *     rows as they stood at its start and the terms of a repeated row are summed
 *     (no 1/batch factor).  batch must be <= min(max_batch, 16384).
 *   deterministic = 0: every nonzero reads its row and adds its own term at
 *     once with atomic adds, many nonzeros concurrently (Hogwild); `batch` is
 *     ignored.
 * C^(mode) is not read and not refreshed. */
sft_status sft_update_factors(sft_ctx *ctx, int32_t mode, const int32_t *const *idx,
                              const float *val, const uint32_t *perm, int64_t nnz, int64_t batch,
                              float lr, float lambda);

/* One SGD pass over B^(mode) (Algorithm 2, core module; Eq. (9), (11)).
 * For each minibatch of `batch` samples (last one shorter, size M_b), with
 * B^(mode) as it stood at its start: G = sum_s e_s a_{i_mode(s)} p_s^T and
 * B^(mode) += lr * (G / M_b - lambda B^(mode)).  batch = nnz gives the single
 * update per pass of Algorithm 5.  Sums are in a fixed order in both modes.
 * batch must be <= max_batch or equal to nnz.  With SFT_BF16 and R in {16, 32}
 * the contraction G runs on the tensor cores (sft_set_tensor_cores). */
sft_status sft_update_core(sft_ctx *ctx, int32_t mode, const int32_t *const *idx,
                           const float *val, const uint32_t *perm, int64_t nnz, int64_t batch,
                           float lr, float lambda);

/* Sum of squared and of absolute residuals x_s - sum_r prod_k C^(k)[i_k][r]
 * over the nnz nonzeros, accumulated in float64 in a fixed order.  sse/sae are
 * HOST pointers; the call waits for the stream and also reports any bad-data
 * flag raised by earlier kernels. */
sft_status sft_loss(sft_ctx *ctx, const int32_t *const *idx, const float *val, int64_t nnz,
                    double *sse, double *sae);

/* As sft_loss, but writes {sse, sae} to the DEVICE buffer out2 (two doubles)
 * and does not wait. */
sft_status sft_loss_async(sft_ctx *ctx, const int32_t *const *idx, const float *val, int64_t nnz,
                          double *out2);

/* Predictions x^_s = sum_r prod_k C^(k)[i_k][r] (Eq. (1) via Eq. (12)) for
 * the nnz nonzeros, written to the DEVICE array out (float32, nnz entries).
 * Enqueues only.  Used to fill in missing entries once the model is fitted. */
sft_status sft_predict(sft_ctx *ctx, const int32_t *const *idx, int64_t nnz, float *out);

/* One epoch of Algorithm 2: for every mode a factor pass then a refresh of
 * that mode, then for every mode a core pass then a refresh.  perm_factor /
 * perm_core: host arrays of N device permutation pointers (or NULL for storage
 * order everywhere; individual entries may be NULL).  Enqueues only. */
sft_status sft_epoch(sft_ctx *ctx, const int32_t *const *idx, const float *val, int64_t nnz,
                     const uint32_t *const *perm_factor, const uint32_t *const *perm_core,
                     int64_t batch_factor, int64_t batch_core, float lr_A, float lambda_A,
                     float lr_B, float lambda_B);

/* ---------------------------------------------------------------------------
 * Gradient of the sampled loss.  L = 1/2 sum_s e_s^2 over a COO set is the
 * data term of the objective in Section "Sparse FastTucker Decomposition"
 * (the factor 2 absorbed, as in Eq. (10)/(11)).  Its gradient with respect to
 * A^(n) and B^(n) is Eq. (10) and Eq. (11) without the regulariser, summed
 * over the set.  Because x^ depends on A^(n), B^(n) only through
 * C^(n) = A^(n) B^(n) (Eq. (12)), it is computed in two calls:
 *   dL/dC^(n) = -sum_s e_s [rows i_n(s)] p^(n)_s  (one pass, all modes),
 *   dL/dA^(n) = dL/dC^(n) B^(n)T,  dL/dB^(n) = A^(n)T dL/dC^(n).
 * Both read C^(k) as it stands; call sft_refresh_C(ctx, -1) first if A or B
 * changed.
 * ------------------------------------------------------------------------- */

/* loss_out (DEVICE, 8-byte aligned, 2 doubles) receives {L, sum_s |e_s|}.
 * dC: host array of N device pointers; dC[n] is I_n x R float32 row-major,
 * 16-byte aligned, owned by the caller; dC = NULL computes loss_out only.  accumulate = 0 overwrites dC (zeroed
 * first); accumulate != 0 adds to what is there.  The per-row sums use float
 * atomic adds, so dC is not bitwise reproducible from run to run (with either
 * value of the config's deterministic flag); loss_out is.  Coordinates out
 * of range are skipped and raise the error flag that sft_sync reports.
 * Enqueues only. */
sft_status sft_loss_grad_C(sft_ctx *ctx, const int32_t *const *idx, const float *val, int64_t nnz,
                           float *const *dC, int32_t accumulate, double *loss_out);

/* gA[n] = s dC[n] B^(n)T (I_n x J_n) and gB[n] = s A^(n)T dC[n] (J_n x R) for
 * every mode, float32, overwritten; s = *scale, a DEVICE double (the incoming
 * gradient of L), or 1 when scale is NULL.  dC[n] as produced by
 * sft_loss_grad_C.  gB is summed over row blocks in a fixed order.
 * Enqueues only. */
sft_status sft_grad_AB(sft_ctx *ctx, const float *const *dC, const double *scale, float *const *gA,
                       float *const *gB);

/* ---------------------------------------------------------------------------
 * Slice layout.  A "slice" of mode n is the set of nonzeros that share the
 * coordinate i_n -- the first level of the CSF tree of Section "Tensor
 * Storage Format".  The sliced copy of a COO set holds the same nonzeros
 * ordered by (i_n, visit position): slice i occupies positions
 * [row_ptr[i], row_ptr[i+1]) and keeps the caller's visit order inside.
 * ------------------------------------------------------------------------- */

/* Bytes of device scratch sft_group_slices needs for nnz nonzeros. */
size_t sft_slices_scratch_bytes(int64_t nnz);

/* Build the slice layout of mode `mode` on the device (a stable radix sort of
 * (i_mode, position) keys by i_mode, then a gather).  out_idx: N device arrays of nnz
 * int32; out_val: nnz float32; out_row_ptr: I_mode + 1 int32.  perm as in
 * sft_update_factors (NULL = storage order).  Nonzeros with a coordinate out
 * of range are moved behind the last slice and flagged (SFT_EINVAL at the next
 * sft_sync).  Enqueues only. */
sft_status sft_group_slices(sft_ctx *ctx, int32_t mode, const int32_t *const *idx, const float *val,
                            const uint32_t *perm, int64_t nnz, int32_t *const *out_idx,
                            float *out_val, int32_t *out_row_ptr, void *scratch,
                            size_t scratch_bytes);

/* Writes the mode-`mode` coordinate of every position of a slice layout from
 * its row pointer alone: out[p] = r for row_ptr[r] <= p < row_ptr[r + 1], -1
 * for positions after the last slice (the bad-data tail of sft_group_slices).
 * row_ptr: DEVICE, I_mode + 1 int32 as sft_group_slices writes it (row_ptr[0]
 * = 0, non-decreasing); out: DEVICE, nnz int32, written.  Lets a caller keep
 * or ship a layout without its mode-`mode` coordinate array (it equals this
 * expansion) and rebuild it on the device.  Enqueues only; SFT_EINVAL for a
 * bad mode, nnz or NULL pointers (nnz = 0 does nothing). */
sft_status sft_slices_expand_rows(sft_ctx *ctx, int32_t mode, const int32_t *row_ptr, int64_t nnz,
                                  int32_t *out);

/* Bytes of device workspace sft_update_factors_slices needs for a slice layout
 * of nnz nonzeros of mode `mode` under the context's current tiling. */
size_t sft_slices_workspace_bytes(const sft_ctx *ctx, int32_t mode, int64_t nnz);

/* One factor pass over A^(mode) on a slice layout, element by element
 * (Algorithm 4; Eq. (9)-(10) with batch 1): every slice's nonzeros are run in
 * their stored order, so the result equals the sequential pass over the visit
 * order that built the layout (slices of one mode never interact during a
 * factor pass).  Long slices are cut into tile-sized pieces composed as affine
 * maps and applied in order (same recurrence, re-associated).  Deterministic:
 * the only atomics collect the lists of slices, tile interiors and map pieces
 * to run, whose order affects no result.  workspace: device buffer of sft_slices_workspace_bytes bytes
 * (the piece maps and that list).  Enqueues only. */
sft_status sft_update_factors_slices(sft_ctx *ctx, int32_t mode, const int32_t *const *sidx,
                                     const float *sval, const int32_t *row_ptr, int64_t nnz,
                                     float lr, float lambda, void *workspace,
                                     size_t workspace_bytes);

/* One core pass over B^(mode) on a slice layout (Algorithm 5; Eq. (9), (11)):
 * minibatches are consecutive ranges of `batch` positions of the layout
 * (batch = nnz: one update per pass).  G is accumulated per slice run as
 * a_i (sum_s e_s p_s)^T.  Deterministic.  Enqueues only. */
sft_status sft_update_core_slices(sft_ctx *ctx, int32_t mode, const int32_t *const *sidx,
                                  const float *sval, const int32_t *row_ptr, int64_t nnz,
                                  int64_t batch, float lr, float lambda);

/* ---------------------------------------------------------------------------
 * Fibers: the shared intermediate variables of Section "Reusable Intermediate
 * Variables" (Eq. (12)-(13)).  A fiber of mode n is a tuple (i_k)_{k != n};
 * its nonzeros share p = prod_{k != n} C^(k)[i_k] and v = B^(n) p.
 * ------------------------------------------------------------------------- */

/* Bytes of device scratch sft_group_fibers needs (a hash table of at least
 * twice nnz slots, 20 bytes each). */
size_t sft_fibers_scratch_bytes(int64_t nnz);

/* For the slice layout of mode n (sidx: N device pointers from
 * sft_group_slices), writes fid[pos] (DEVICE int32, nnz entries) = the fiber of
 * each position, numbered 0..nfibers-1, and the fibers' coordinates:
 * fcoord (host array of N device pointers; the entry for `mode` is ignored)
 * with fcoord[k][f] = i_k of fiber f (DEVICE int32, room for nnz entries).
 * *nfibers (HOST) receives the count.  The numbering depends on thread
 * scheduling; the fibers themselves do not.  Synchronises the stream.
 * SFT_ENOTSUP if the product of the other modes' lengths is 4e18 or more (the
 * fiber key is their exact linear index).  Coordinates out of range get
 * fid -1 and are reported as SFT_EINVAL. */
sft_status sft_group_fibers(sft_ctx *ctx, int32_t mode, const int32_t *const *sidx, int64_t nnz,
                            int32_t *fid, int32_t *const *fcoord, int64_t *nfibers, void *scratch,
                            size_t scratch_bytes);

/* Rebuilds the other modes' coordinate arrays of a slice layout from its fiber
 * table: every position of fiber f holds that fiber's tuple (Eq. (12)), so for
 * each k != mode, out_idx[k][p] = fcoord[k][fid[p]]; a position whose fid is
 * not in [0, nfibers) (the -1 that sft_group_fibers gives bad data) gets -1 in
 * every such k.  fid: DEVICE, nnz int32; fcoord: host array of N device
 * pointers (the entry for `mode` is ignored), each with nfibers int32; out_idx:
 * host array of N device pointers (the entry for `mode` is ignored), each nnz
 * int32, written.  With sft_slices_expand_rows this lets a caller keep or ship
 * a layout as values, row_ptr, fid and fcoord only and rebuild its coordinate
 * arrays on the device.  Enqueues only; SFT_EINVAL for a bad mode, nnz or
 * nfibers (0 <= nfibers <= nnz) or NULL pointers (nnz = 0 does nothing). */
sft_status sft_fibers_expand_coords(sft_ctx *ctx, int32_t mode, const int32_t *fid, int64_t nnz,
                                    const int32_t *const *fcoord, int64_t nfibers,
                                    int32_t *const *out_idx);

/* sft_update_factors_slices with v formed once per fiber: first
 * V[f][0..J_n) = B^(n) p_f for every fiber (V: DEVICE float32, nfibers x J_n,
 * 16-byte aligned, caller-owned), then the element-by-element slice pass reads
 * v from V.  fid / fcoord / nfibers from sft_group_fibers on the same layout.
 * v is formed with the same operations in the same order as the per-nonzero
 * path, so the result is the same.  Enqueues only. */
sft_status sft_update_factors_fibers(sft_ctx *ctx, int32_t mode, const int32_t *const *sidx,
                                     const float *sval, const int32_t *row_ptr, int64_t nnz,
                                     const int32_t *fid, const int32_t *const *fcoord,
                                     int64_t nfibers, float *V, float lr, float lambda,
                                     void *workspace,
                                     size_t workspace_bytes);

/* sft_update_core_slices with p formed once per fiber: first
 * P[f][0..R) = prod_{k != n} C^(k)[i_k(f)] (P: DEVICE float32, nfibers x R,
 * 16-byte aligned, caller-owned; it does not depend on B^(n), so one fill
 * serves every minibatch of the pass), then the core pass reads p from P.
 * Same result as the per-nonzero path.  Enqueues only. */
sft_status sft_update_core_fibers(sft_ctx *ctx, int32_t mode, const int32_t *const *sidx,
                                  const float *sval, const int32_t *row_ptr, int64_t nnz,
                                  int64_t batch, const int32_t *fid,
                                  const int32_t *const *fcoord, int64_t nfibers, float *P,
                                  float lr, float lambda);

/* Tiling of the slice passes: tile = positions per work item (0 = automatic),
 * max_direct = chain length: a slice that crosses a tile boundary and has at
 * most max_direct nonzeros is run element by element, whole, by one lane
 * group; a longer one runs its first max_direct nonzeros that way and the rest
 * through composed affine maps applied to the row the head leaves
 * (0 = automatic, two tiles; < 0 = none: every crossing slice goes through
 * maps; values between 0 and one tile are raised to one tile).  Results do
 * not depend on it beyond rounding. */
sft_status sft_set_slice_tiling(sft_ctx *ctx, int64_t tile, int64_t max_direct);

/* Tensor cores for the two dense contractions when the cached products are
 * bfloat16 (SFT_BF16); on by default.  With enable != 0:
 *   sft_refresh_C (J_n in {8, 16, 32}, R in {16, 32}): C^(n) = A^(n) B^(n) by
 *     tcgen05 MMAs of kind tf32 (tiles of A^(n) copied by TMA; float32
 *     accumulation; C^(n) rounded to bfloat16 as before);
 *   sft_update_core (R in {16, 32}): the minibatch core gradient
 *     G = sum_s e_s a p_s^T of Eq. (11) as the contraction (J_n x M).(M x R) by
 *     tcgen05 MMAs of kind f16 with bfloat16 operands e_s a and p_s and a
 *     float32 accumulator per block; the block partials are summed in float64
 *     in a fixed order, as on the CUDA-core path.
 * With enable = 0 (or other shapes) the float32 CUDA-core kernels run.  The
 * float32 configuration (SFT_FP32) never uses tensor cores.  A wait of a
 * tensor-core kernel that runs out (2 s) is reported as SFT_ETIMEOUT by the
 * next sft_sync / sft_loss. */
sft_status sft_set_tensor_cores(sft_ctx *ctx, int32_t enable);

/* Time limit, in nanoseconds, of the tensor-core kernels' waits on their own
 * TMA copies and MMAs (mbarrier waits of the main loop; default 2 s, at most
 * 60 s).  A wait that runs out makes the kernel flag it, stop, wait once more
 * -- always with the full 2 s bound -- for the copies and MMAs it issued,
 * free its tensor memory and return; the next sft_sync / sft_loss reports
 * SFT_ETIMEOUT and the context stays usable.  The result of the call whose
 * wait ran out is not valid: a refresh leaves C^(n) partly stale, a core pass
 * moves B^(n) by a partial gradient (blocks whose wait ran out add nothing).  limit_ns = 0 gives up without waiting,
 * so that the expiry path can be made to run on a normal launch (this is how
 * it is tested).  Does not affect the float32 kernels. */
sft_status sft_set_tc_wait_limit(sft_ctx *ctx, int64_t limit_ns);

/* How the slice factor pass runs a long slice (a crossing slice longer than
 * max_direct):
 *   SFT_LONG_MAPS (default): exactly, in Algorithm 4's element order -- its
 *     first max_direct nonzeros as a chain, the rest cut at tile boundaries
 *     into pieces composed as affine maps and applied in order;
 *   SFT_LONG_SUBSLICES: as the paper's B-CSF storage treats a heavy slice
 *     (Section "Tensor Storage Format"; its sub-slices are walked
 *     concurrently): every tile-sized piece is walked element by element from
 *     the row as it stands when the walk starts, and its change is added to
 *     the row with atomic adds.  Pieces of one row overlap in time (Hogwild
 *     within the row), so the result depends on scheduling. */
/* Blocked chains in the fiber factor pass (sft_update_factors_fibers, J_n in
 * {8, 16, 32}, lr * lambda < 0.5; on by default): a chain of at least 4096
 * nonzeros is run by one warp 32 nonzeros at a time -- the block's steps
 * solved as a triangular system over its Gram matrix V V^T (TF32 tensor-core
 * MMAs with a high/low split, float32 accumulation), the row moved once per
 * block.  The same recurrence re-associated: results agree with the
 * element-by-element form to rounding, not bitwise.  enable = 0 runs every
 * chain element by element. */
sft_status sft_set_blocked_chains(sft_ctx *ctx, int32_t enable);

#define SFT_LONG_MAPS 0
#define SFT_LONG_SUBSLICES 1
sft_status sft_set_long_slices(sft_ctx *ctx, int32_t how);

/* Per-mode autotuner of the slice factor pass: times the pass of `mode` with
 * several limits on the length of a crossing slice that is run whole as one
 * chain (W, 2W, 1024, 1536, 2048, 3072, .. 49152, 65536, and every crossing
 * slice whole; W is the factor pass's tile length; a longer slice
 * runs that many nonzeros as a chain and the rest through maps) and keeps the
 * fastest for this mode.  It overrides the tiling's
 * max_direct for that mode until sft_set_slice_tiling is called again.  Every
 * trial starts from the same A^(mode): it is saved to scratch (DEVICE,
 * >= I_mode * J_mode floats, 16-byte aligned) first and restored after each
 * trial, so the model is left as it was.  fid / fcoord / nfibers / V as for
 * sft_update_factors_fibers, or fid = NULL for the per-nonzero path.  The
 * choice does not change any result beyond rounding order.  Synchronous;
 * *lseq_out (HOST, may be NULL) receives the chosen limit. */
sft_status sft_autotune_slices(sft_ctx *ctx, int32_t mode, const int32_t *const *sidx,
                               const float *sval, const int32_t *row_ptr, int64_t nnz,
                               const int32_t *fid, const int32_t *const *fcoord, int64_t nfibers,
                               float *V, float lr, float lambda, void *workspace,
                               size_t workspace_bytes, void *scratch, size_t scratch_bytes,
                               int64_t *lseq_out);

/* ---------------------------------------------------------------------------
 * Factor pass without any device allocation.  The paper has no counterpart to
 * this call; it exists for callers that cannot allocate device memory -- e.g.
 * a plugin inside a host application that owns all device memory through its
 * own pool and forbids cudaMalloc/cudaFree, or a latency-critical loop that
 * must not allocate -- and so cannot give sft_init a workspace.
 *
 * It runs the same deterministic minibatch factor pass as sft_update_factors
 * with deterministic = 1 (same kernels, same result), taking every operand
 * directly: the order, mode lengths dims[N], ranks J[N] and R; mode; the
 * device matrices A_mode (I_mode x J_mode, updated in place), B_mode
 * (J_mode x R) and C[N] (I_k x R, the cached products, FLOAT32: the layout of
 * an SFT_FP32 decomposition; bfloat16 products are not accepted here); the
 * COO set idx[N], val, optional perm, nnz; batch, lr, lambda (finite); the
 * cudaStream_t `stream`.
 * Its scratch (the per-chunk row sums of a minibatch and the bad-data flag) is
 * a fixed ~529 KB array of device memory inside the library image, kept by
 * every GPU that loads the library until the process exits; no call allocates,
 * frees, or calls an allocating routine.
 *   - batch must be 1..4096 (the scratch holds one minibatch of at most 4096
 *     nonzeros); a larger batch returns SFT_ENOTSUP and does nothing;
 *   - the first call on a device looks up the array's device address (with that
 *     device current) and caches it;
 *   - every call reads the bad-data flag back and waits for `stream` before it
 *     returns, so it cannot be recorded into a CUDA graph: on a stream that is
 *     being captured it returns SFT_ENOTSUP before enqueuing anything;
 *   - all calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and must not be issued;
 *   - SFT_EINVAL is returned after the wait if a kernel flagged bad data
 *     (coordinates out of range, permutation entries >= nnz), which was then
 *     skipped.
 * Returns SFT_EINVAL / SFT_ENOTSUP for bad or unsupported arguments before any
 * launch, SFT_ECUDA on a CUDA error. */
sft_status sft_update_factors_noalloc(int32_t order, const int64_t *dims, const int32_t *J,
                                      int32_t R, int32_t mode, float *A_mode, const float *B_mode,
                                      float *const *C, const int32_t *const *idx, const float *val,
                                      const uint32_t *perm, int64_t nnz, int64_t batch, float lr,
                                      float lambda, void *stream);

/* Wait for the stream, at most timeout_ms milliseconds (< 0: no limit).
 * Returns SFT_ETIMEOUT if work is still running, SFT_EINVAL if a kernel
 * flagged bad data (the flag is then cleared), SFT_ECUDA on a CUDA error. */
sft_status sft_sync(sft_ctx *ctx, int64_t timeout_ms);

/* Change the stream later calls enqueue on. */
sft_status sft_set_stream(sft_ctx *ctx, void *stream);

/* Human-readable message of the last failure on this context ("" if none).
 * Valid until the next call on the context. */
const char *sft_last_error(const sft_ctx *ctx);

/* Number of kernels this context has launched so far. */
int64_t sft_launch_count(const sft_ctx *ctx);

/* Free the context (host memory only).  Does not synchronise. */
void sft_destroy(sft_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SFT_H */
