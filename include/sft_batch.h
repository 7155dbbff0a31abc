/*
 * sft_batch.h -- many independent sparse FastTucker decompositions trained
 * together by one graph launch per epoch (GB300, sm_103a).
 *
 * The paper trains one tensor at a time.  This interface runs the same epoch
 * of Algorithm 2 on a set of unrelated problems at once: every problem's
 * factor passes (Algorithm 4; Eq. (9), (10)), refreshes of C^(n)
 * (Algorithm 3) and core passes (Algorithm 5; Eq. (9), (11)), in the paper's
 * order within a problem.  The paper has no counterpart for the batching
 * itself.
 *
 * How it runs: the library cuts every pass into tasks (`chunk` nonzeros, or
 * 4096 rows of C) and orders all tasks of all problems with a list scheduler
 * (problems with the most remaining work first).  That order respects each
 * problem's chain of passes.  The problems are split by rank into two
 * classes (R <= 16 and R = 32), each with its own list and its own
 * persistent kernel compiled for those ranks only; the two kernels run side
 * by side and hand their tasks out in list order.  A task whose predecessor
 * pass is still running waits on a device counter with a bounded poll.  The
 * reset of the counters plus the persistent kernels are captured once as a
 * CUDA graph and replayed every epoch.  sft_batch_autotune picks `chunk` and the CTAs per SM by timing
 * epochs.
 *
 * Update rules (as the single-problem calls with deterministic = 0):
 *   factor rows   Hogwild, per nonzero: a += lr_A (e v - lambda_A a), applied
 *                 with float atomic adds, so rows are not bitwise
 *                 reproducible and order effects differ from a sequential run
 *   core          one update per pass over all of the problem's nonzeros:
 *                 B += lr_B (sum_s e_s a_s p_s^T / nnz - lambda_B B), the
 *                 chunk partials summed in a fixed order (float64)
 * Shapes: 2 <= N <= 8, J_n = R for every mode, R in {4, 8, 16, 32},
 * I_n < 2^31, 1 <= nnz < 2^31.  Other shapes return SFT_ENOTSUP (SFT_EINVAL
 * for nnz < 1).
 *
 * Memory: as in sft.h, every array is a device pointer owned by the caller
 * (A[n] I_n x R, B[n] R x R float32, C[n] I_n x R float32 or bfloat16 per
 * `prec`, idx[n] int32 and val float32 with nnz entries, all row-major,
 * 16-byte aligned).  The caller also provides the workspace (device, 256-byte
 * aligned) sized by sft_batch_workspace_bytes.  The handle owns host metadata,
 * two private streams and two events used for graph capture, and the
 * instantiated graphs.
 *
 * Errors: argument errors return before any launch.  Bad coordinates are
 * skipped by the kernel and reported by sft_batch_sync / sft_batch_loss as
 * SFT_EINVAL.  A dependency wait that runs out of polls stops the kernel and
 * is reported as SFT_ETIMEOUT.
 */
#ifndef SFT_BATCH_H
#define SFT_BATCH_H

#include "sft.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sft_batch sft_batch; /* opaque */

typedef struct {
    int32_t order;               /* N, 2..8 */
    const int64_t *dims;         /* host array [N]: I_n */
    int32_t R;                   /* rank; J_n = R for every mode */
    float *const *A;             /* host array [N] of device pointers, I_n x R */
    float *const *B;             /* host array [N] of device pointers, R x R */
    void *const *C;              /* host array [N] of device pointers, I_n x R (prec) */
    const int32_t *const *idx;   /* host array [N] of device pointers, nnz each */
    const float *val;            /* device, nnz */
    int64_t nnz;
    float lr_A, lambda_A, lr_B, lambda_B;
} sft_batch_problem;

/* Device workspace for a batch whose passes are cut into tasks of at least
 * min_chunk nonzeros (min_chunk >= 256).  0 on invalid arguments. */
size_t sft_batch_workspace_bytes(int32_t nprob, const sft_batch_problem *probs, int64_t min_chunk);

/* Creates the handle: validates every problem, copies the problem table to
 * the workspace, builds the task lists for `chunk` (>= min_chunk given to
 * sft_batch_workspace_bytes; 0 = min_chunk) and `blocks_per_sm` CTAs per SM
 * (0 = as many as fit), and captures the graphs.  prec: sft_precision of C.
 * stream: cudaStream_t every later call enqueues on.  Enqueues nothing. */
sft_status sft_batch_create(int32_t nprob, const sft_batch_problem *probs, int32_t prec,
                            int64_t min_chunk, int64_t chunk, int32_t blocks_per_sm,
                            void *workspace, size_t workspace_bytes, void *stream,
                            sft_batch **out);

/* Enqueues C^(n) = A^(n) B^(n) for every mode of every problem. */
sft_status sft_batch_refresh(sft_batch *b);

/* Enqueues one epoch of Algorithm 2 for every problem (one graph launch). */
sft_status sft_batch_epoch(sft_batch *b);

/* Residual sums over each problem's own nonzeros with its current C:
 * out (HOST, 2 * nprob doubles) receives {sum e^2, sum |e|} per problem.
 * Synchronises the stream; reports kernel-flagged errors. */
sft_status sft_batch_loss(sft_batch *b, double *out);

/* Bytes of device scratch sft_batch_autotune needs (a copy of every A and B). */
size_t sft_batch_snapshot_bytes(const sft_batch *b);

/* Times `epochs` epochs (after one warm-up epoch) for each candidate chunk
 * (chunk, 2, 4 and 8 times the workspace's min_chunk) and CTAs per SM (1, 2,
 * as many as fit) and keeps the fastest.  Every A and B is saved to scratch
 * (device, >= sft_batch_snapshot_bytes, 16-byte aligned) first and restored
 * after each candidate, then C is refreshed, so the model is left as it was.
 * Synchronous.  chunk_out / bps_out (host, may be NULL) receive the choice. */
sft_status sft_batch_autotune(sft_batch *b, void *scratch, size_t scratch_bytes, int32_t epochs,
                              int64_t *chunk_out, int32_t *bps_out);

/* Waits for the stream (SFT_ETIMEOUT after timeout_ms; < 0 = no limit) and
 * reports kernel-flagged errors. */
sft_status sft_batch_sync(sft_batch *b, int64_t timeout_ms);

/* Polls (of at least 256 ns each) after which a task stops waiting for the
 * pass it depends on; the kernel then stops and sft_batch_sync reports
 * SFT_ETIMEOUT.  Default 2^24 (several seconds).  Applies to graphs built
 * afterwards: call before sft_batch_autotune or re-create.  polls >= 1. */
sft_status sft_batch_set_wait_limit(sft_batch *b, int64_t polls);

/* Failure injection for tests, done on the host: hold = 1 makes the first
 * pass of problem `prob` in the epoch list wait for one task more than it
 * has, so the passes after it can never start and their waits run out (the
 * kernel stops, SFT_ETIMEOUT); hold = 0 undoes it.  Nothing faults. */
sft_status sft_batch_hold_pass(sft_batch *b, int32_t prob, int32_t hold);

/* Graph launches enqueued so far (one per refresh, epoch, loss; each runs
 * the persistent kernel of every rank class that has tasks). */
int64_t sft_batch_launch_count(const sft_batch *b);

/* Tasks in one epoch's list with the current chunk. */
int64_t sft_batch_epoch_tasks(const sft_batch *b);

/* One record of a task list, as sft_batch_plan reports it.  kind: 0 factor
 * chunk, 1 refresh rows, 2 core chunk, 3 core update, 4 loss chunk, 5 loss
 * total.  wait / done: index of the pass counter the task waits on (-1 none)
 * and the one it decrements.  [begin, end): nonzeros (or rows of C^(mode)). */
typedef struct {
    int32_t prob, kind, mode, wait, done, slot, nslots, pad;
    int64_t begin, end;
} sft_batch_task_info;

/* Host only (no GPU needed): the task list sft_batch_create builds for
 * plan 0 (epoch), 1 (refresh) or 2 (loss) with tasks of `chunk` nonzeros:
 * the tasks of the problems with R <= 16, then those of the problems with
 * R = 32 (each part run by its own persistent kernel), each part ordered
 * for `workers` CTAs.  Writes at most cap records to out (host) and
 * returns the full task count, or -1 on invalid arguments. */
int64_t sft_batch_plan(int32_t nprob, const sft_batch_problem *probs, int32_t plan, int64_t chunk,
                       int32_t workers, sft_batch_task_info *out, int64_t cap);

const char *sft_batch_last_error(const sft_batch *b);
void sft_batch_destroy(sft_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* SFT_BATCH_H */
