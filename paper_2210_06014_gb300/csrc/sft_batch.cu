// sft_batch.cu -- host side of include/sft_batch.h: validation, the task
// lists of the persistent kernel in k_batch.cu, their order (a list
// scheduler), CUDA-graph capture and the autotuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sft_batch.h"
#include "batch_internal.cuh"

using namespace sft;

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kRowChunk = 4096;     // rows of C per refresh task
constexpr int64_t kMinChunk = 256;
constexpr int64_t kWaitLimit = 1 << 24; // polls of >= 256 ns: several seconds

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct HostProblem {
    int N = 0, R = 0;
    int64_t dims[kBatchMaxOrder] = {};
    int64_t nnz = 0;
    float *A[kBatchMaxOrder] = {};
    float *B[kBatchMaxOrder] = {};
    float *C[kBatchMaxOrder] = {};
    const int32_t *idx[kBatchMaxOrder] = {};
    const float *val = nullptr;
    float lrA = 0, lamA = 0, lrB = 0, lamB = 0;
};

enum PlanId { kPlanEpoch = 0, kPlanRefresh = 1, kPlanLoss = 2, kPlans = 3 };

// Upper bounds of a plan's task and counter counts for a given chunk.
struct PlanSize {
    int64_t tasks = 0, counters = 0;
};

PlanSize plan_size(const std::vector<HostProblem> &ps, int plan, int64_t chunk) {
    PlanSize s;
    for (const HostProblem &p : ps) {
        const int64_t nt = cdiv(p.nnz, chunk);
        int64_t rows = 0;
        for (int n = 0; n < p.N; ++n) rows += cdiv(p.dims[n], kRowChunk);
        if (plan == kPlanEpoch) {
            s.tasks += 2 * p.N * nt + 2 * rows + p.N;
            s.counters += 5 * p.N;
        } else if (plan == kPlanRefresh) {
            s.tasks += rows;
            s.counters += p.N;
        } else {
            s.tasks += nt + 1;
            s.counters += 2;
        }
    }
    return s;
}

// Workspace layout (byte offsets).
struct Layout {
    size_t probs = 0, err = 0, abort = 0, head = 0;
    size_t tasks[kPlans] = {}, counters[kPlans] = {}, init[kPlans] = {};
    int64_t cap_tasks[kPlans] = {}, cap_counters[kPlans] = {};
    std::vector<size_t> partials, lpart;  // per problem
    size_t loss_out = 0;
    size_t total = 0;
};

Layout make_layout(const std::vector<HostProblem> &ps, int64_t min_chunk) {
    Layout L;
    size_t off = 0;
    L.probs = off;
    off = align_up(off + ps.size() * sizeof(BatchProblem));
    L.err = off;
    off = align_up(off + sizeof(int));
    L.abort = off;
    off = align_up(off + sizeof(int32_t));
    L.head = off;
    off = align_up(off + kPlans * kBatchClasses * sizeof(int32_t));
    for (int pl = 0; pl < kPlans; ++pl) {
        PlanSize s = plan_size(ps, pl, min_chunk);
        L.cap_tasks[pl] = s.tasks;
        L.cap_counters[pl] = s.counters;
        L.tasks[pl] = off;
        off = align_up(off + (size_t)s.tasks * sizeof(BatchTask));
        L.counters[pl] = off;
        off = align_up(off + (size_t)s.counters * sizeof(int32_t));
        L.init[pl] = off;
        off = align_up(off + (size_t)s.counters * sizeof(int32_t));
    }
    for (const HostProblem &p : ps) {
        L.partials.push_back(off);
        off = align_up(off + (size_t)cdiv(p.nnz, min_chunk) * p.R * p.R * sizeof(float));
        L.lpart.push_back(off);
        off = align_up(off + (size_t)(cdiv(p.nnz, min_chunk) + 1) * 2 * sizeof(double));
    }
    L.loss_out = off;
    off = align_up(off + ps.size() * 2 * sizeof(double));
    L.total = off;
    return L;
}

const char *check_problems(int32_t nprob, const sft_batch_problem *probs, int prec,
                           sft_status *st, std::vector<HostProblem> *out) {
    *st = SFT_EINVAL;
    if (nprob < 1 || !probs) return "need at least one problem";
    if (prec != SFT_FP32 && prec != SFT_BF16) return "unknown precision";
    std::vector<HostProblem> ps;
    for (int32_t i = 0; i < nprob; ++i) {
        const sft_batch_problem &q = probs[i];
        HostProblem p;
        if (q.order < 2) return "order must be >= 2";
        if (q.order > kBatchMaxOrder) {
            *st = SFT_ENOTSUP;
            return "order must be <= 8 in a batch";
        }
        if (!(q.R == 4 || q.R == 8 || q.R == 16 || q.R == 32)) {
            *st = SFT_ENOTSUP;
            return "R must be one of 4, 8, 16, 32";
        }
        if (!q.dims || !q.A || !q.B || !q.C || !q.idx || !q.val) return "a problem has NULL arrays";
        if (q.nnz < 1 || q.nnz > 0x7fffffffLL) return "each problem needs 1 <= nnz < 2^31";
        if (!std::isfinite(q.lr_A) || !std::isfinite(q.lambda_A) || !std::isfinite(q.lr_B) ||
            !std::isfinite(q.lambda_B))
            return "learning rates / lambdas must be finite";
        p.N = q.order;
        p.R = q.R;
        p.nnz = q.nnz;
        p.val = q.val;
        p.lrA = q.lr_A;
        p.lamA = q.lambda_A;
        p.lrB = q.lr_B;
        p.lamB = q.lambda_B;
        for (int n = 0; n < p.N; ++n) {
            if (q.dims[n] < 1 || q.dims[n] > 0x7fffffffLL) return "each I_n must be in [1, 2^31)";
            if (!q.A[n] || !q.B[n] || !q.C[n] || !q.idx[n]) return "a problem has NULL arrays";
            if (((uintptr_t)q.A[n] | (uintptr_t)q.B[n] | (uintptr_t)q.C[n]) & 15u)
                return "A, B and C must be 16-byte aligned";
            p.dims[n] = q.dims[n];
            p.A[n] = q.A[n];
            p.B[n] = q.B[n];
            p.C[n] = (float *)q.C[n];
            p.idx[n] = q.idx[n];
        }
        ps.push_back(p);
    }
    *out = std::move(ps);
    *st = SFT_OK;
    return nullptr;
}

// One pass of one problem: `ntasks` tasks of `per` units each (the last one
// shorter) over `total` units.
struct Phase {
    int prob, kind, mode;
    int64_t total, per;
    int ntasks;
    double cost;      // estimated time of one task (arbitrary units)
    int counter;      // counter of this phase (index within the plan)
    int wait;         // counter of the phase it waits for (-1: none)
    int nslots;       // apply / loss-final: tasks of the preceding phase
    double rest = 0;  // estimated work from this phase to the end of its chain
};

double nnz_cost(const HostProblem &p, int64_t n) {
    return 2000.0 + (double)n * (p.N * p.R / 4.0 + p.R * p.R / 8.0);
}
double row_cost(const HostProblem &p, int64_t rows) {
    return 2000.0 + (double)rows * p.R * p.R / 16.0;
}

// Phase chains of every problem for a plan.
std::vector<std::vector<Phase>> make_phases(const std::vector<HostProblem> &ps, int plan,
                                            int64_t chunk) {
    std::vector<std::vector<Phase>> chains(ps.size());
    int counter = 0;
    for (size_t pi = 0; pi < ps.size(); ++pi) {
        const HostProblem &p = ps[pi];
        std::vector<Phase> &ch = chains[pi];
        auto add = [&](int kind, int mode, int64_t total, int64_t per, double cost_one,
                       bool chained, int nslots) {
            Phase ph{};
            ph.prob = (int)pi;
            ph.kind = kind;
            ph.mode = mode;
            ph.total = total;
            ph.per = per;
            ph.ntasks = (int)cdiv(total, per);
            ph.cost = cost_one;
            ph.counter = counter++;
            ph.wait = (chained && !ch.empty()) ? ch.back().counter : -1;
            ph.nslots = nslots;
            ch.push_back(ph);
        };
        const int64_t nchunks = cdiv(p.nnz, chunk);
        if (plan == kPlanEpoch) {
            for (int n = 0; n < p.N; ++n) {
                add(kTaskFactor, n, p.nnz, chunk, nnz_cost(p, std::min(chunk, p.nnz)), true, 0);
                add(kTaskRefresh, n, p.dims[n], kRowChunk,
                    row_cost(p, std::min(kRowChunk, p.dims[n])), true, 0);
            }
            for (int n = 0; n < p.N; ++n) {
                add(kTaskCore, n, p.nnz, chunk, nnz_cost(p, std::min(chunk, p.nnz)), true, 0);
                add(kTaskApply, n, 1, 1, 2000.0 + nchunks * p.R * p.R / 64.0, true, (int)nchunks);
                add(kTaskRefresh, n, p.dims[n], kRowChunk,
                    row_cost(p, std::min(kRowChunk, p.dims[n])), true, 0);
            }
        } else if (plan == kPlanRefresh) {
            for (int n = 0; n < p.N; ++n)
                add(kTaskRefresh, n, p.dims[n], kRowChunk,
                    row_cost(p, std::min(kRowChunk, p.dims[n])), false, 0);
        } else {
            add(kTaskLoss, -1, p.nnz, chunk, nnz_cost(p, std::min(chunk, p.nnz)), true, 0);
            add(kTaskLossFin, -1, 1, 1, 2000.0 + nchunks, true, (int)nchunks);
        }
        double rest = 0;
        for (int k = (int)ch.size() - 1; k >= 0; --k) {
            rest += ch[k].cost * ch[k].ntasks;
            ch[k].rest = rest;
        }
    }
    return chains;
}

// List scheduling of the phase chains on `workers` CTAs: whenever a CTA is
// free it takes the next task of the ready phase with the most remaining work
// in its chain.  The dispatch order is a topological order of the task graph
// (a task is emitted only after every task of the phase it waits for has
// been emitted), which is what the persistent kernel's waits rely on.
// Only the chains of problems with use[p] set are scheduled; `init` (sized by
// the caller to every counter of the plan) receives their counters' starting
// values.
std::vector<BatchTask> order_tasks(std::vector<std::vector<Phase>> &chains,
                                   const std::vector<char> &use, int workers,
                                   std::vector<int32_t> *init) {
    struct Ready {
        double rest;
        int prob, k;
        bool operator<(const Ready &o) const { return rest < o.rest; }
    };
    struct Event {
        double t;
        int prob, k;
        bool operator>(const Event &o) const { return t > o.t; }
    };
    std::priority_queue<Ready> ready;
    std::priority_queue<Event, std::vector<Event>, std::greater<Event>> events;
    std::vector<std::vector<int>> dispatched(chains.size()), finished(chains.size());
    for (size_t p = 0; p < chains.size(); ++p) {
        dispatched[p].assign(chains[p].size(), 0);
        finished[p].assign(chains[p].size(), 0);
    }
    // a chain's first phase with tasks is ready at once (phases without
    // tasks cannot occur: every problem has nnz >= 1 and I_n >= 1)
    for (size_t p = 0; p < chains.size(); ++p) {
        if (!use[p]) continue;
        for (const Phase &ph : chains[p]) (*init)[ph.counter] = ph.ntasks;
        for (size_t k = 0; k < chains[p].size(); ++k) {
            const bool head = chains[p][k].wait < 0;
            if (head) ready.push({chains[p][k].rest, (int)p, (int)k});
        }
    }
    std::vector<BatchTask> out;
    int idle = workers < 1 ? 1 : workers;
    double now = 0;
    for (;;) {
        while (idle > 0 && !ready.empty()) {
            Ready r = ready.top();
            Phase &ph = chains[r.prob][r.k];
            const int i = dispatched[r.prob][r.k]++;
            BatchTask t{};
            t.prob = ph.prob;
            t.kind = ph.kind;
            t.mode = ph.mode;
            t.wait = ph.wait;
            t.done = ph.counter;
            t.slot = i;
            t.nslots = ph.nslots;
            t.begin = (int64_t)i * ph.per;
            t.end = std::min(ph.total, t.begin + ph.per);
            out.push_back(t);
            events.push({now + ph.cost, r.prob, r.k});
            --idle;
            if (dispatched[r.prob][r.k] == ph.ntasks) ready.pop();
        }
        if (events.empty()) break;
        Event e = events.top();
        events.pop();
        now = e.t;
        ++idle;
        if (++finished[e.prob][e.k] == chains[e.prob][e.k].ntasks) {
            // the phases chained to this one become ready
            const int c = chains[e.prob][e.k].counter;
            for (size_t k = 0; k < chains[e.prob].size(); ++k)
                if (chains[e.prob][k].wait == c) ready.push({chains[e.prob][k].rest, e.prob, (int)k});
        }
    }
    return out;
}

int count_counters(const std::vector<std::vector<Phase>> &chains) {
    int n = 0;
    for (const auto &c : chains) n += (int)c.size();
    return n;
}

// The plan's task list: the list of class 0 (R <= 16) followed by that of
// class 1 (R = 32), each scheduled on its own kernel's CTAs; n[c] = tasks of
// class c.
std::vector<BatchTask> class_lists(const std::vector<HostProblem> &ps,
                                   std::vector<std::vector<Phase>> &chains,
                                   const int (&workers)[kBatchClasses], std::vector<int32_t> *init,
                                   int64_t (&n)[kBatchClasses]) {
    init->assign(count_counters(chains), 0);
    std::vector<BatchTask> out;
    for (int c = 0; c < kBatchClasses; ++c) {
        std::vector<char> use(ps.size(), 0);
        for (size_t p = 0; p < ps.size(); ++p) use[p] = batch_class(ps[p].R) == c;
        std::vector<BatchTask> t = order_tasks(chains, use, workers[c], init);
        n[c] = (int64_t)t.size();
        out.insert(out.end(), t.begin(), t.end());
    }
    return out;
}

}  // namespace

struct sft_batch {
    std::vector<HostProblem> ps;
    int cbf16 = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;   // private stream for graph capture
    cudaStream_t side = nullptr;  // ... and its fork for the second class kernel
    cudaEvent_t fork = nullptr, join = nullptr;
    int device = 0, sms = 1;
    int max_bps[kBatchClasses] = {1, 1};
    char *ws = nullptr;
    Layout L;
    int64_t min_chunk = kMinChunk, chunk = kMinChunk;
    int bps = 1;
    int64_t wait_limit = kWaitLimit;
    std::vector<int32_t> epoch_init;   // starting counters of the epoch list (host copy)
    std::vector<int32_t> epoch_first;  // per problem: counter of its first epoch pass
    BatchLaunch args[kPlans] = {};
    cudaGraphExec_t exec[kPlans] = {nullptr, nullptr, nullptr};
    int64_t launches = 0;
    std::string last_error;
};

namespace {

sft_status fail(sft_batch *b, sft_status st, const std::string &m) {
    if (b) b->last_error = m;
    return st;
}

sft_status cuda_fail(sft_batch *b, cudaError_t e, const char *where) {
    return fail(b, SFT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void drop_graphs(sft_batch *b) {
    for (int pl = 0; pl < kPlans; ++pl) {
        if (b->exec[pl]) cudaGraphExecDestroy(b->exec[pl]);
        b->exec[pl] = nullptr;
    }
}

// Graphs, streams, events and the handle itself.
void release(sft_batch *b) {
    drop_graphs(b);
    if (b->join) cudaEventDestroy(b->join);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

// Builds the three task lists for (chunk, bps), uploads them and captures
// one graph per list (counter reset + the persistent kernel of each class;
// bps is capped by each class kernel's occupancy).
sft_status build_plans(sft_batch *b, int64_t chunk, int bps) {
    // the old lists and graphs may still be in use by enqueued work
    cudaError_t se = cudaStreamSynchronize(b->stream);
    if (se != cudaSuccess) return cuda_fail(b, se, "stream synchronize");
    drop_graphs(b);
    b->chunk = chunk;
    b->bps = bps;
    int grid[kBatchClasses];
    for (int c = 0; c < kBatchClasses; ++c) grid[c] = b->sms * std::min(bps, b->max_bps[c]);
    for (int pl = 0; pl < kPlans; ++pl) {
        auto chains = make_phases(b->ps, pl, chunk);
        std::vector<int32_t> init;
        int64_t ncls[kBatchClasses];
        std::vector<BatchTask> tasks = class_lists(b->ps, chains, grid, &init, ncls);
        if ((int64_t)tasks.size() > b->L.cap_tasks[pl] || (int64_t)init.size() > b->L.cap_counters[pl])
            return fail(b, SFT_ENOMEM, "task list larger than the workspace allows");
        BatchTask *dt = (BatchTask *)(b->ws + b->L.tasks[pl]);
        int32_t *dc = (int32_t *)(b->ws + b->L.counters[pl]);
        int32_t *di = (int32_t *)(b->ws + b->L.init[pl]);
        cudaError_t e = cudaMemcpy(dt, tasks.data(), tasks.size() * sizeof(BatchTask),
                                   cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(di, init.data(), init.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(b, e, "task list upload");
        BatchLaunch &bl = b->args[pl];
        int64_t base = 0;
        for (int c = 0; c < kBatchClasses; ++c) {
            BatchArgs &g = bl.cls[c];
            g.probs = (const BatchProblem *)(b->ws + b->L.probs);
            g.tasks = dt + base;
            g.ntasks = (int32_t)ncls[c];
            g.counters = dc;
            g.init = di;
            g.ncounters = (int32_t)init.size();
            g.head = (int32_t *)(b->ws + b->L.head) + pl * kBatchClasses + c;
            g.abort = (int32_t *)(b->ws + b->L.abort);
            g.err = (int *)(b->ws + b->L.err);
            g.wait_limit = b->wait_limit;
            bl.grid[c] = grid[c];
            base += ncls[c];
        }
        if (pl == kPlanEpoch) {
            b->epoch_init = init;
            b->epoch_first.assign(b->ps.size(), -1);
            for (size_t p = 0; p < chains.size(); ++p)
                if (!chains[p].empty()) b->epoch_first[p] = chains[p][0].counter;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(b, e, "graph capture");
        cudaError_t le = launch_batch(bl, b->cbf16 != 0, b->cap, b->side, b->fork, b->join);
        e = cudaStreamEndCapture(b->cap, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(b, le, "batch launch capture");
        }
        if (e != cudaSuccess) return cuda_fail(b, e, "graph capture");
        e = cudaGraphInstantiate(&b->exec[pl], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(b, e, "graph instantiate");
    }
    return SFT_OK;
}

sft_status run_plan(sft_batch *b, int pl) {
    cudaError_t e = cudaGraphLaunch(b->exec[pl], b->stream);
    b->launches += 1;
    if (e != cudaSuccess) return cuda_fail(b, e, "graph launch");
    return SFT_OK;
}

sft_status wait_stream(sft_batch *b, int64_t timeout_ms) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(b->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(b, e, "stream query");
        if (timeout_ms >= 0) {
            const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                                std::chrono::steady_clock::now() - t0).count();
            if (ms > timeout_ms) return fail(b, SFT_ETIMEOUT, "stream still busy at the timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, b->ws + b->L.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(b, e, "reading the error flag");
    if (flag) {
        cudaMemset(b->ws + b->L.err, 0, sizeof(int));
        if (flag & kErrWait)
            return fail(b, SFT_ETIMEOUT, "a task gave up waiting for the pass it depends on");
        return fail(b, SFT_EINVAL, "a kernel skipped bad data: coordinate out of range");
    }
    return SFT_OK;
}

}  // namespace

extern "C" {

size_t sft_batch_workspace_bytes(int32_t nprob, const sft_batch_problem *probs, int64_t min_chunk) {
    if (min_chunk < kMinChunk) return 0;
    std::vector<HostProblem> ps;
    sft_status st;
    if (check_problems(nprob, probs, SFT_FP32, &st, &ps)) return 0;
    return make_layout(ps, min_chunk).total + kAlign;
}

sft_status sft_batch_create(int32_t nprob, const sft_batch_problem *probs, int32_t prec,
                            int64_t min_chunk, int64_t chunk, int32_t blocks_per_sm,
                            void *workspace, size_t workspace_bytes, void *stream,
                            sft_batch **out) {
    if (!out) return SFT_EINVAL;
    *out = nullptr;
    std::vector<HostProblem> ps;
    sft_status st;
    if (check_problems(nprob, probs, prec, &st, &ps)) return st;
    if (min_chunk < kMinChunk) return SFT_EINVAL;
    if (chunk == 0) chunk = min_chunk;
    if (chunk < min_chunk) return SFT_EINVAL;
    if (blocks_per_sm < 0) return SFT_EINVAL;
    if (!workspace || ((uintptr_t)workspace % kAlign) != 0) return SFT_EINVAL;
    Layout L = make_layout(ps, min_chunk);
    if (workspace_bytes < L.total) return SFT_ENOMEM;
    sft_batch *b = new (std::nothrow) sft_batch;
    if (!b) return SFT_ENOMEM;
    b->ps = std::move(ps);
    b->cbf16 = prec == SFT_BF16 ? 1 : 0;
    b->stream = (cudaStream_t)stream;
    b->ws = (char *)workspace;
    b->L = L;
    b->min_chunk = min_chunk;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release(b);
        return SFT_ECUDA;
    }
    for (int c = 0; c < kBatchClasses; ++c) b->max_bps[c] = batch_blocks_per_sm(b->cbf16 != 0, c);
    const int maxb = std::max(b->max_bps[0], b->max_bps[1]);
    int bps = blocks_per_sm == 0 ? maxb : std::min<int>(blocks_per_sm, maxb);
    // problem table
    std::vector<BatchProblem> table(b->ps.size());
    for (size_t i = 0; i < b->ps.size(); ++i) {
        const HostProblem &p = b->ps[i];
        BatchProblem &q = table[i];
        std::memset(&q, 0, sizeof(q));
        for (int n = 0; n < p.N; ++n) {
            q.idx[n] = p.idx[n];
            q.A[n] = p.A[n];
            q.B[n] = p.B[n];
            q.C[n] = p.C[n];
            q.dims[n] = (int32_t)p.dims[n];
        }
        q.val = p.val;
        q.partials = (float *)(b->ws + L.partials[i]);
        q.lpart = (double *)(b->ws + L.lpart[i]);
        q.loss_out = (double *)(b->ws + L.loss_out) + 2 * i;
        q.nnz = p.nnz;
        q.N = p.N;
        q.R = p.R;
        q.lrA = p.lrA;
        q.lamA = p.lamA;
        q.lrB = p.lrB;
        q.lamB = p.lamB;
    }
    cudaError_t e = cudaMemcpy(b->ws + L.probs, table.data(), table.size() * sizeof(BatchProblem),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->ws + L.err, 0, sizeof(int));
    if (e != cudaSuccess) {
        release(b);
        return SFT_ECUDA;
    }
    st = build_plans(b, chunk, bps);
    if (st != SFT_OK) {
        release(b);
        return st;
    }
    *out = b;
    return SFT_OK;
}

sft_status sft_batch_refresh(sft_batch *b) {
    if (!b) return SFT_EINVAL;
    return run_plan(b, kPlanRefresh);
}

sft_status sft_batch_epoch(sft_batch *b) {
    if (!b) return SFT_EINVAL;
    return run_plan(b, kPlanEpoch);
}

sft_status sft_batch_loss(sft_batch *b, double *out) {
    if (!b) return SFT_EINVAL;
    if (!out) return fail(b, SFT_EINVAL, "out is NULL");
    sft_status st = run_plan(b, kPlanLoss);
    if (st != SFT_OK) return st;
    st = wait_stream(b, -1);
    if (st != SFT_OK) return st;
    cudaError_t e = cudaMemcpy(out, b->ws + b->L.loss_out, b->ps.size() * 2 * sizeof(double),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(b, e, "loss readback");
    return SFT_OK;
}

size_t sft_batch_snapshot_bytes(const sft_batch *b) {
    if (!b) return 0;
    size_t s = 0;
    for (const HostProblem &p : b->ps)
        for (int n = 0; n < p.N; ++n)
            s += align_up((size_t)p.dims[n] * p.R * sizeof(float)) +
                 align_up((size_t)p.R * p.R * sizeof(float));
    return s;
}

static cudaError_t snapshot(sft_batch *b, char *scratch, bool restore) {
    size_t off = 0;
    for (const HostProblem &p : b->ps) {
        for (int n = 0; n < p.N; ++n) {
            const size_t a = (size_t)p.dims[n] * p.R * sizeof(float);
            const size_t bb = (size_t)p.R * p.R * sizeof(float);
            cudaError_t e = restore
                ? cudaMemcpyAsync(p.A[n], scratch + off, a, cudaMemcpyDeviceToDevice, b->stream)
                : cudaMemcpyAsync(scratch + off, p.A[n], a, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return e;
            off += align_up(a);
            e = restore
                ? cudaMemcpyAsync(p.B[n], scratch + off, bb, cudaMemcpyDeviceToDevice, b->stream)
                : cudaMemcpyAsync(scratch + off, p.B[n], bb, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return e;
            off += align_up(bb);
        }
    }
    return cudaSuccess;
}

sft_status sft_batch_autotune(sft_batch *b, void *scratch, size_t scratch_bytes, int32_t epochs,
                              int64_t *chunk_out, int32_t *bps_out) {
    if (!b) return SFT_EINVAL;
    if (!scratch || scratch_bytes < sft_batch_snapshot_bytes(b) || ((uintptr_t)scratch & 15u))
        return fail(b, SFT_EINVAL, "scratch missing, misaligned or smaller than sft_batch_snapshot_bytes");
    if (epochs < 1) return fail(b, SFT_EINVAL, "epochs must be >= 1");
    char *snap = (char *)scratch;
    cudaError_t e = snapshot(b, snap, false);
    if (e != cudaSuccess) return cuda_fail(b, e, "snapshot");
    std::vector<int64_t> chunks;
    int64_t maxnnz = 0;
    for (const HostProblem &p : b->ps) maxnnz = std::max(maxnnz, p.nnz);
    for (int k = 0; k < 4; ++k) {
        const int64_t c = b->min_chunk << k;
        if (k > 0 && c > std::max<int64_t>(maxnnz, b->min_chunk)) break;
        chunks.push_back(c);
    }
    std::vector<int> bpss;
    const int maxb = std::max(b->max_bps[0], b->max_bps[1]);
    for (int v : {1, 2, maxb})
        if (v <= maxb && std::find(bpss.begin(), bpss.end(), v) == bpss.end()) bpss.push_back(v);
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess) return cuda_fail(b, cudaGetLastError(), "event");
    if (cudaEventCreate(&t1) != cudaSuccess) {
        cudaEventDestroy(t0);
        return cuda_fail(b, cudaGetLastError(), "event");
    }
    float best = -1.f;
    int64_t best_chunk = b->chunk;
    int best_bps = b->bps;
    sft_status st = SFT_OK;
    for (int64_t c : chunks) {
        for (int v : bpss) {
            st = build_plans(b, c, v);
            if (st != SFT_OK) break;
            st = run_plan(b, kPlanEpoch);  // warm-up
            if (st != SFT_OK) break;
            cudaEventRecord(t0, b->stream);
            for (int i = 0; i < epochs && st == SFT_OK; ++i) st = run_plan(b, kPlanEpoch);
            cudaEventRecord(t1, b->stream);
            if (st != SFT_OK) break;
            e = snapshot(b, snap, true);
            if (e != cudaSuccess) {
                st = cuda_fail(b, e, "restore");
                break;
            }
            st = wait_stream(b, -1);
            if (st != SFT_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            if (best < 0.f || ms < best) {
                best = ms;
                best_chunk = c;
                best_bps = v;
            }
        }
        if (st != SFT_OK) break;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != SFT_OK) {
        snapshot(b, snap, true);
        return st;
    }
    st = build_plans(b, best_chunk, best_bps);
    if (st != SFT_OK) return st;
    st = run_plan(b, kPlanRefresh);
    if (st != SFT_OK) return st;
    st = wait_stream(b, -1);
    if (st != SFT_OK) return st;
    if (chunk_out) *chunk_out = best_chunk;
    if (bps_out) *bps_out = best_bps;
    return SFT_OK;
}

sft_status sft_batch_sync(sft_batch *b, int64_t timeout_ms) {
    if (!b) return SFT_EINVAL;
    return wait_stream(b, timeout_ms);
}

int64_t sft_batch_plan(int32_t nprob, const sft_batch_problem *probs, int32_t plan, int64_t chunk,
                       int32_t workers, sft_batch_task_info *out, int64_t cap) {
    static_assert(sizeof(sft_batch_task_info) == sizeof(BatchTask), "task record layout");
    std::vector<HostProblem> ps;
    sft_status st;
    if (check_problems(nprob, probs, SFT_FP32, &st, &ps)) return -1;
    if (plan < 0 || plan >= kPlans || chunk < kMinChunk || workers < 1 || cap < 0) return -1;
    auto chains = make_phases(ps, plan, chunk);
    std::vector<int32_t> init;
    int64_t ncls[kBatchClasses];
    const int w[kBatchClasses] = {workers, workers};
    std::vector<BatchTask> tasks = class_lists(ps, chains, w, &init, ncls);
    const int64_t n = (int64_t)tasks.size();
    if (out && cap > 0) std::memcpy(out, tasks.data(), (size_t)std::min(n, cap) * sizeof(BatchTask));
    return n;
}

sft_status sft_batch_set_wait_limit(sft_batch *b, int64_t polls) {
    if (!b) return SFT_EINVAL;
    if (polls < 1) return fail(b, SFT_EINVAL, "polls must be >= 1");
    b->wait_limit = polls;
    return build_plans(b, b->chunk, b->bps);
}

sft_status sft_batch_hold_pass(sft_batch *b, int32_t prob, int32_t hold) {
    if (!b) return SFT_EINVAL;
    if (prob < 0 || prob >= (int32_t)b->ps.size()) return fail(b, SFT_EINVAL, "prob out of range");
    const int c = b->epoch_first[prob];
    if (c < 0) return fail(b, SFT_EINVAL, "problem has no epoch pass");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "stream synchronize");
    const int32_t v = b->epoch_init[c] + (hold ? 1 : 0);
    int32_t *di = (int32_t *)(b->ws + b->L.init[kPlanEpoch]);
    e = cudaMemcpy(di + c, &v, sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(b, e, "counter upload");
    return SFT_OK;
}

int64_t sft_batch_launch_count(const sft_batch *b) { return b ? b->launches : 0; }

int64_t sft_batch_epoch_tasks(const sft_batch *b) {
    if (!b) return 0;
    int64_t n = 0;
    for (int c = 0; c < kBatchClasses; ++c) n += b->args[kPlanEpoch].cls[c].ntasks;
    return n;
}

const char *sft_batch_last_error(const sft_batch *b) { return b ? b->last_error.c_str() : "null handle"; }

void sft_batch_destroy(sft_batch *b) {
    if (!b) return;
    release(b);
}

}  // extern "C"
