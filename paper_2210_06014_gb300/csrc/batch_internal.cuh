// batch_internal.cuh -- device-side records of the batched runner (many
// independent decompositions driven by one persistent kernel): the problem
// table, the task list and the kernel arguments.  Shared by k_batch.cu (the
// kernel) and sft_batch.cu (plan building, graph capture, autotuning).
#pragma once

#include <stdint.h>

#include "sft_internal.cuh"

namespace sft {

constexpr int kBatchMaxOrder = 8;
constexpr int kBatchThreads = 256;

// One decomposition.  J_n = R for every mode.  Pointers are device pointers
// borrowed from the caller; C[k] holds float or bfloat16 entries.
struct BatchProblem {
    const int32_t *idx[kBatchMaxOrder];
    float *A[kBatchMaxOrder];
    float *B[kBatchMaxOrder];
    float *C[kBatchMaxOrder];
    int32_t dims[kBatchMaxOrder];
    const float *val;
    float *partials;   // core-gradient partials, one R x R slot per core task
    double *lpart;     // loss partials, two doubles per loss task
    double *loss_out;  // {sum e^2, sum |e|}
    int64_t nnz;
    int32_t N, R;
    float lrA, lamA, lrB, lamB;
};

enum BatchKind : int32_t {
    kTaskFactor = 0,   // Hogwild SGD over a chunk of nonzeros (Algorithm 4; Eq. (10))
    kTaskRefresh = 1,  // rows [begin, end) of C^(n) = A^(n) B^(n) (Algorithm 3)
    kTaskCore = 2,     // core-gradient partial of a chunk (Eq. (11)) into slot `slot`
    kTaskApply = 3,    // B^(n) += lr (sum of `nslots` partials / nnz - lambda B^(n)) (Algorithm 5)
    kTaskLoss = 4,     // residual sums of a chunk into loss slot `slot`
    kTaskLossFin = 5,  // sum of `nslots` loss slots into loss_out
};

struct BatchTask {
    int32_t prob;
    int32_t kind;
    int32_t mode;
    int32_t wait;     // counter that must reach 0 before the task starts (-1: none)
    int32_t done;     // counter decremented when the task has finished
    int32_t slot;     // partial slot written by a core / loss task
    int32_t nslots;   // slots summed by an apply / loss-final task
    int32_t pad;
    int64_t begin, end;
};

struct BatchArgs {
    const BatchProblem *probs;
    const BatchTask *tasks;
    int32_t ntasks;
    int32_t *counters;      // live counters of this plan
    const int32_t *init;    // their starting values
    int32_t ncounters;
    int32_t *head;          // next task to hand out
    int32_t *abort;         // set when a wait gave up; every CTA then stops
    int *err;               // error flag bits (kErrIndex, kErrWait)
    int64_t wait_limit;     // polls before a wait gives up
};

// kErrWait (sft_internal.cuh): a dependency wait ran out of polls

// Problems are split by R into classes, each run by its own persistent
// kernel compiled for those R only, so that the kernel of the small ranks
// is not held at the register count of R = 32: class 0 holds R <= 16,
// class 1 R = 32.  The two kernels share the plan's counters (problems of
// different classes never wait on each other) and run side by side.
constexpr int kBatchClasses = 2;
inline int batch_class(int R) { return R <= 16 ? 0 : 1; }

struct BatchLaunch {
    BatchArgs cls[kBatchClasses];  // tasks, count and head of each class (same counters)
    int grid[kBatchClasses];       // persistent CTAs of each class's kernel
};

// Counter reset, then the class kernels that have tasks (class 1 on `side`,
// forked from and joined back to `st` with the two events).
cudaError_t launch_batch(const BatchLaunch &L, bool cbf16, cudaStream_t st, cudaStream_t side,
                         cudaEvent_t fork, cudaEvent_t join);
int batch_blocks_per_sm(bool cbf16, int cls);

}  // namespace sft
