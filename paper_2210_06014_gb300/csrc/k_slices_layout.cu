// k_slices_layout.cu -- the factor and core passes over nonzeros grouped into the
// mode-n slices of the tensor (all nonzeros that share i_n, kept in visit
// order), the CSF layout of Section "Tensor Storage Format".
//
// Layout.  k_slice_keys / k_rs_* (a stable radix sort by i_n of keys that
// start in position order) / k_slice_gather / k_slice_rowptr order the visit
// positions by (i_n, position), so the order inside a slice is the visit order,
// and copy the COO arrays into that order; row_ptr[i] is the first position
// of slice i.
//
// Factor pass (Eq. (9)-(10), element by element as in Algorithm 4).  During a
// factor pass over mode n a nonzero reads and writes only a_{i_n}; slices are
// independent, and running every slice's nonzeros one after another in visit
// order reproduces the element-by-element rule exactly.  Positions are cut
// into tiles of W; then
//   - the slices inside a tile (its interior) are run directly: the row stays
//     in registers, each nonzero does e = x - a.(B p), a += lr (e v - lambda a);
//   - a slice that crosses tile boundaries and has at most Lseq nonzeros is
//     run directly, whole, as one chain;
//   - a longer slice runs its first Lhead = Lseq nonzeros as a chain (its head)
//     and the rest (its map region) split at the tile boundaries.  One step is
//     the affine map a -> M_t a + c_t with M_t = (1 - lr lambda) I - lr v v^T
//     and c_t = lr x v, so each piece is composed into one map (M, c) in
//     parallel (k_slices_maps); k_slices_compose multiplies blocks of
//     consecutive piece maps and k_slices_combine applies them to the row, in
//     order, after its head.  This is the same recurrence, re-associated.
// With the fiber table and J_n <= 16 the interiors and the chains are one
// work list sorted by length (k_lane_count / k_lane_scatter) that a
// persistent kernel walks one item per lane (k_slices_lanes); chains of
// 4096+ positions go to the blocked kernel (k_slices_gram).  Otherwise lane
// groups of R/4 lanes walk them (k_slices_tiles / k_slices_chains).  The
// atomics only build the lists, whose order affects no result: the pass is
// bitwise reproducible.
//
// Core pass (Eq. (9), (11), Algorithm 5).  With A^(n) fixed,
//   G = sum_s e_s a_{i_n(s)} p_s^T = sum_slices a_i (sum_{s in slice} e_s p_s)^T,
// so a group keeps q = sum e_s p_s over the run of a slice inside its tile and
// adds a_i q^T to its shared-memory tile of G once per run.  x^_s = (B^T a).p_s
// uses w = B^T a computed once per run.
#include "slices_impl.cuh"

namespace sft {


// ============================================================================ layout
__global__ void k_slice_keys(const int32_t *__restrict__ rowidx, const uint32_t *__restrict__ perm,
                             int64_t nnz, int32_t In, unsigned long long *__restrict__ keys,
                             int64_t P, int *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        unsigned long long key = ~0ull;
        if (i < nnz) {
            int64_t s = i;
            uint32_t row = (uint32_t)In;  // invalid samples sort after every slice
            bool ok = true;
            if (perm) {
                const uint32_t q = perm[i];
                if ((int64_t)q >= nnz) {
                    atomicOr(err, kErrPerm);
                    ok = false;
                } else {
                    s = q;
                }
            }
            if (ok) {
                const uint32_t r = (uint32_t)rowidx[s];
                if (r >= (uint32_t)In) atomicOr(err, kErrIndex);
                else row = r;
            }
            key = ((unsigned long long)row << 32) | (unsigned long long)i;
        }
        keys[i] = key;
    }
}

// Stable LSD radix sort of the keys by their row (the high 32 bits), 4 bits
// per pass.  The keys start in position order, so after the passes they are
// ordered by (row, position): every slice keeps the visit order.  A pass:
// k_rs_count counts the digits of each tile of kRsTile keys, k_rs_scan turns
// the counts (digit-major: digit d of every tile, then digit d + 1) into
// output offsets, and k_rs_scatter moves each tile's keys to their offsets,
// in order within a digit (the ranks are per-thread counts scanned across
// the block's threads in thread order, each thread holding consecutive keys).
constexpr int kRsThreads = 256;
constexpr int kRsPerThread = 12;
constexpr int kRsTile = kRsThreads * kRsPerThread;
constexpr int kRsDigits = 16;

__device__ __forceinline__ int rs_digit(unsigned long long key, int shift) {
    return (int)((key >> (32 + shift)) & (kRsDigits - 1));
}

__global__ void __launch_bounds__(kRsThreads) k_rs_count(const unsigned long long *__restrict__ in,
                                                         int64_t n, int shift, int64_t ntiles,
                                                         unsigned int *__restrict__ hist) {
    __shared__ unsigned int h[kRsDigits];
    if (threadIdx.x < kRsDigits) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const int64_t j = base + i;
        if (j < n) atomicAdd(&h[rs_digit(in[j], shift)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kRsDigits) hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive prefix sum of m counts in place, one block of 1024 threads (each
// thread sums a contiguous run, the runs' sums are scanned across the block).
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned int *__restrict__ v, int64_t m) {
    __shared__ unsigned int part[1024];
    const int64_t per = (m + 1023) / 1024;
    const int64_t lo = (int64_t)threadIdx.x * per;
    const int64_t hi = lo + per < m ? lo + per : m;
    unsigned int sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += v[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
        const unsigned int y = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned int run = part[threadIdx.x] - sum;
    for (int64_t i = lo; i < hi; ++i) {
        const unsigned int c = v[i];
        v[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const unsigned long long *__restrict__ in,
                                                           unsigned long long *__restrict__ out,
                                                           int64_t n, int shift, int64_t ntiles,
                                                           const unsigned int *__restrict__ offs) {
    // the tile, padded by one key per thread's run so the runs' reads spread
    // over the banks; then per digit and thread the count, scanned in place
    __shared__ unsigned long long sk[kRsTile + kRsThreads];
    __shared__ unsigned int cnt[kRsDigits][kRsThreads + 1];
    __shared__ unsigned int goff[kRsDigits];
    const int t = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = t; i < kRsTile; i += kRsThreads) {
        const int64_t j = base + i;
        sk[i + i / kRsPerThread] = j < n ? in[j] : ~0ull;
    }
    for (int d = 0; d < kRsDigits; ++d) cnt[d][t] = 0;
    if (t < kRsDigits) goff[t] = offs[(int64_t)t * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned long long *mine = sk + t * (kRsPerThread + 1);
    const int64_t first = base + (int64_t)t * kRsPerThread;  // this thread's first key
#pragma unroll 4
    for (int i = 0; i < kRsPerThread; ++i)
        if (first + i < n) cnt[rs_digit(mine[i], shift)][t] += 1u;
    __syncthreads();
    // exclusive scan of cnt[d][0..255] for every digit: warp w takes digits
    // 2w and 2w + 1, each lane a run of 8 threads
    {
        const int w = t >> 5, lane = t & 31;
#pragma unroll
        for (int dd = 0; dd < 2; ++dd) {
            const int d = 2 * w + dd;
            unsigned int c[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = cnt[d][lane * 8 + q];
                sum += c[q];
            }
            unsigned int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            unsigned int run = incl - sum;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                cnt[d][lane * 8 + q] = run;
                run += c[q];
            }
        }
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < kRsPerThread; ++i) {
        if (first + i < n) {
            const unsigned long long key = mine[i];
            const int d = rs_digit(key, shift);
            const unsigned int r = cnt[d][t]++;
            out[goff[d] + r] = key;
        }
    }
}

struct SliceOut {
    int32_t *idx[kMaxOrder];
    float *val;
};

__global__ void k_slice_gather(PassArgs a, const unsigned long long *__restrict__ keys, SliceOut o) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.nnz; t += stride) {
        const unsigned long long key = keys[t];
        const uint32_t row = (uint32_t)(key >> 32);
        const int64_t pos = (int64_t)(key & 0xffffffffu);
        if (row >= (uint32_t)a.dims[a.n]) {
            for (int k = 0; k < a.N; ++k) o.idx[k][t] = -1;
            o.val[t] = 0.f;
            continue;
        }
        const int64_t s = a.perm ? (int64_t)a.perm[pos] : pos;
        for (int k = 0; k < a.N; ++k) o.idx[k][t] = a.idx[k][s];
        o.val[t] = a.val[s];
    }
}

__global__ void k_slice_rowptr(const unsigned long long *__restrict__ keys, int64_t nnz, int32_t In,
                               int32_t *__restrict__ row_ptr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= In; r += stride) {
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(keys[mid] >> 32) < r) lo = mid + 1; else hi = mid;
        }
        row_ptr[r] = (int32_t)lo;
    }
}

// Scratch of the layout build: two key buffers of nnz and the digit counts
// of every tile (as unsigned long long units).
int64_t slice_sort_length(int64_t nnz) {
    const int64_t ntiles = (nnz + kRsTile - 1) / kRsTile;
    return 2 * nnz + (kRsDigits * ntiles + 1) / 2 + 2;
}

cudaError_t launch_group_slices(const PassArgs &a, int32_t *const *out_idx, float *out_val,
                                int32_t *row_ptr, unsigned long long *keys, cudaStream_t st,
                                int sms, int64_t *launches) {
    const int64_t n = a.nnz;
    const int th = 256;
    auto grid = [&](int64_t m) {
        int64_t b = (m + th - 1) / th;
        const int64_t cap = (int64_t)sms * 16;
        return (int)(b < 1 ? 1 : (b > cap ? cap : b));
    };
    unsigned long long *kin = keys, *kout = keys + n;
    unsigned int *hist = reinterpret_cast<unsigned int *>(keys + 2 * n);
    const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    k_slice_keys<<<grid(n), th, 0, st>>>(a.idx[a.n], a.perm, n, a.dims[a.n], kin, n, a.err);
    *launches += 1;
    // rows run up to I_n (bad coordinates sort after every slice)
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) <= (int64_t)a.dims[a.n]) ++bits;
    for (int shift = 0; shift < bits && n > 0; shift += 4) {
        k_rs_count<<<(int)ntiles, kRsThreads, 0, st>>>(kin, n, shift, ntiles, hist);
        k_rs_scan<<<1, 1024, 0, st>>>(hist, kRsDigits * ntiles);
        k_rs_scatter<<<(int)ntiles, kRsThreads, 0, st>>>(kin, kout, n, shift, ntiles, hist);
        *launches += 3;
        unsigned long long *tmp = kin;
        kin = kout;
        kout = tmp;
    }
    keys = kin;
    SliceOut o{};
    for (int k = 0; k < a.N; ++k) o.idx[k] = out_idx[k];
    o.val = out_val;
    k_slice_gather<<<grid(a.nnz), th, 0, st>>>(a, keys, o);
    k_slice_rowptr<<<grid((int64_t)a.dims[a.n] + 1), th, 0, st>>>(keys, a.nnz, a.dims[a.n], row_ptr);
    *launches += 2;
    return cudaGetLastError();
}


// ============================================================================ long slices: combine
// Pieces of a long slice (one per tile it touches) are grouped into blocks of
// Bc = ceil(sqrt(K)) consecutive pieces (K pieces in all).  k_slices_compose
// folds each block into one map, in place in the slot of its first piece
// (X = P_last; X = X o P for the earlier pieces: X.M <- X.M P.M,
// X.c <- X.M P.c + X.c), and k_slices_combine applies the block maps to the
// row in order.  Lane `sub` owns rows [sub*JL, (sub+1)*JL) of X.

__device__ __forceinline__ int64_t block_len(int64_t K) {
    int64_t b = (int64_t)sqrtf((float)K);
    while (b * b < K) ++b;
    return b < 1 ? 1 : b;
}

// Slot of a long slice's piece in tile t, its map region starting at hs.
__device__ __forceinline__ int piece_slot(int64_t hs, int64_t t, int64_t W) {
    return hs < t * W ? 0 : 1;
}

// The long slice whose map piece in tile t is in slot `side` (see map_piece).
__device__ __forceinline__ bool long_piece(const SliceArgs &g, int64_t t, int side, int32_t &r,
                                           int64_t &s, int64_t &e, int64_t &hs) {
    int64_t q0, q1;
    return map_piece(g, t, side, r, s, e, hs, q0, q1);
}

constexpr int kComposeGroups = 8;  // lane groups per block of k_slices_compose

// Form for J = 32 or lanes holding more than 4 rows (J/T > 4).  X (the running block map,
// rows of X.M then X.c) lives in shared memory; lane
// `sub` owns columns [sub*JL, (sub+1)*JL) of X.M and rows [sub*JL, ...) of X.c.
// Each product X <- X o P first pulls the lane's column slice of P.M and all of
// P.c into registers (one memory latency per product), then computes the new
// columns from the whole of X; a group barrier separates reads from writes.
template <int R, int J>
__global__ void __launch_bounds__(kComposeGroups * (R / 4)) k_slices_compose_smem(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int MS = J * J + J;
    __shared__ __align__(16) float sX[kComposeGroups * MS];
    const int sub = threadIdx.x & (T - 1);
    const int gid = threadIdx.x / T;
    const unsigned m = group_mask<T>(threadIdx.x & 31);
    float *X = sX + gid * MS;
    const int64_t groups = (int64_t)gridDim.x * kComposeGroups;
    for (int64_t t = (int64_t)blockIdx.x * kComposeGroups + gid; t < g.ntiles; t += groups) {
        for (int side = 0; side < 2; ++side) {
            int32_t r;
            int64_t s, e, hs;
            if (!long_piece(g, t, side, r, s, e, hs)) continue;
            const int64_t t0 = hs / g.W, t1 = (e - 1) / g.W;
            const int64_t Bc = block_len(t1 - t0 + 1);
            if ((t - t0) % Bc != 0) continue;
            const int64_t tl = min(t + Bc - 1, t1);
            if (tl == t) continue;  // a block of one piece is already its own map
            const float *P = g.maps + (tl * 2 + piece_slot(hs, tl, g.W)) * (int64_t)MS;
            for (int j = 0; j < J; ++j)
#pragma unroll
                for (int q = 0; q < JL; ++q) X[j * J + sub * JL + q] = __ldcg(P + j * J + sub * JL + q);
#pragma unroll
            for (int q = 0; q < JL; ++q) X[J * J + sub * JL + q] = __ldcg(P + J * J + sub * JL + q);
            __syncwarp(m);
            for (int64_t u = tl - 1; u >= t; --u) {
                P = g.maps + (u * 2 + piece_slot(hs, u, g.W)) * (int64_t)MS;
                float pc[J];          // all of P.c
                float pm[J][JL];      // the lane's columns of P.M
#pragma unroll
                for (int l = 0; l < J; ++l) {
                    pc[l] = __ldcg(P + J * J + l);
#pragma unroll
                    for (int q = 0; q < JL; ++q) pm[l][q] = __ldcg(P + l * J + sub * JL + q);
                }
                // new X.c for the lane's rows (reads rows of the old X.M)
                float nc[JL];
#pragma unroll
                for (int q = 0; q < JL; ++q) {
                    const int j = sub * JL + q;
                    float acc = X[J * J + j];
#pragma unroll
                    for (int l = 0; l < J; ++l) acc = fmaf(X[j * J + l], pc[l], acc);
                    nc[q] = acc;
                }
                // one row of X.M at a time: read it whole, then write the lane's columns
#pragma unroll 1
                for (int j = 0; j < J; ++j) {
                    float nrow[JL];
#pragma unroll
                    for (int q = 0; q < JL; ++q) nrow[q] = 0.f;
#pragma unroll
                    for (int l = 0; l < J; ++l) {
                        const float xjl = X[j * J + l];
#pragma unroll
                        for (int q = 0; q < JL; ++q) nrow[q] = fmaf(xjl, pm[l][q], nrow[q]);
                    }
                    __syncwarp(m);
#pragma unroll
                    for (int q = 0; q < JL; ++q) X[j * J + sub * JL + q] = nrow[q];
                    __syncwarp(m);
                }
#pragma unroll
                for (int q = 0; q < JL; ++q) X[J * J + sub * JL + q] = nc[q];
                __syncwarp(m);
            }
            float *out = g.maps + (t * 2 + piece_slot(hs, t, g.W)) * (int64_t)MS;
            for (int j = 0; j < J; ++j)
#pragma unroll
                for (int q = 0; q < JL; ++q) out[j * J + sub * JL + q] = X[j * J + sub * JL + q];
#pragma unroll
            for (int q = 0; q < JL; ++q) out[J * J + sub * JL + q] = X[J * J + sub * JL + q];
            __syncwarp(m);
        }
    }
}

// Form for J <= 16 and J/T <= 4.  X (the running block map) lives in registers: lane `sub` holds rows
// [sub*JL, (sub+1)*JL) of X.M and of X.c.  The group stages each piece map P in
// shared memory with cp.async, two buffers deep (the next P is in flight while
// the current product runs); every lane reads P whole (broadcast) and forms its
// rows of X o P:  X.M <- X.M P.M,  X.c <- X.M P.c + X.c, each entry summed
// over l in ascending order.
template <int R, int J>
__global__ void __launch_bounds__(kComposeGroups * (R / 4)) k_slices_compose(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int MS = J * J + J;
    constexpr int CH = MS / 4;  // 16-byte chunks of one map
    __shared__ __align__(16) float sP[kComposeGroups * 2 * MS];
    const int sub = threadIdx.x & (T - 1);
    const int gid = threadIdx.x / T;
    const unsigned m = group_mask<T>(threadIdx.x & 31);
    float *buf = sP + gid * 2 * MS;
    auto stage = [&](const float *P, float *dst) {
        for (int c = sub; c < CH; c += T) {
            const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + 4 * c));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(P + 4 * c)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int64_t groups = (int64_t)gridDim.x * kComposeGroups;
    for (int64_t t = (int64_t)blockIdx.x * kComposeGroups + gid; t < g.ntiles; t += groups) {
        for (int side = 0; side < 2; ++side) {
            int32_t r;
            int64_t s, e, hs;
            if (!long_piece(g, t, side, r, s, e, hs)) continue;
            const int64_t t0 = hs / g.W, t1 = (e - 1) / g.W;
            const int64_t Bc = block_len(t1 - t0 + 1);
            if ((t - t0) % Bc != 0) continue;
            const int64_t tl = min(t + Bc - 1, t1);
            if (tl == t) continue;  // a block of one piece is already its own map
            auto map_of = [&](int64_t u) {
                return g.maps + (u * 2 + piece_slot(hs, u, g.W)) * (int64_t)MS;
            };
            stage(map_of(tl - 1), buf);
            float X[JL][J], Xc[JL];
            {
                const float *P = map_of(tl);
#pragma unroll
                for (int q = 0; q < JL; ++q) {
#pragma unroll
                    for (int k = 0; k < J; k += 4) {
                        const float4 v = __ldcg(reinterpret_cast<const float4 *>(
                            P + (sub * JL + q) * J + k));
                        X[q][k] = v.x; X[q][k + 1] = v.y; X[q][k + 2] = v.z; X[q][k + 3] = v.w;
                    }
                    Xc[q] = __ldcg(P + J * J + sub * JL + q);
                }
            }
            int cur = 0;
            for (int64_t u = tl - 1; u >= t; --u) {
                if (u > t) {
                    stage(map_of(u - 1), buf + (cur ^ 1) * MS);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                } else {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                }
                __syncwarp(m);  // every lane's chunks of P have landed
                const float *P = buf + cur * MS;
#pragma unroll
                for (int q = 0; q < JL; ++q) {
                    float nrow[J];
#pragma unroll
                    for (int k = 0; k < J; ++k) nrow[k] = 0.f;
                    float acc = Xc[q];
#pragma unroll
                    for (int l = 0; l < J; ++l) {
                        const float x = X[q][l];
#pragma unroll
                        for (int k = 0; k < J; k += 4) {
                            const float4 pv = *reinterpret_cast<const float4 *>(P + l * J + k);
                            nrow[k] = fmaf(x, pv.x, nrow[k]);
                            nrow[k + 1] = fmaf(x, pv.y, nrow[k + 1]);
                            nrow[k + 2] = fmaf(x, pv.z, nrow[k + 2]);
                            nrow[k + 3] = fmaf(x, pv.w, nrow[k + 3]);
                        }
                        acc = fmaf(x, P[J * J + l], acc);
                    }
#pragma unroll
                    for (int k = 0; k < J; ++k) X[q][k] = nrow[k];
                    Xc[q] = acc;
                }
                __syncwarp(m);  // P fully read before its buffer is refilled
                cur ^= 1;
            }
            float *out = map_of(t);
#pragma unroll
            for (int q = 0; q < JL; ++q) {
#pragma unroll
                for (int k = 0; k < J; k += 4)
                    *reinterpret_cast<float4 *>(out + (sub * JL + q) * J + k) =
                        make_float4(X[q][k], X[q][k + 1], X[q][k + 2], X[q][k + 3]);
                out[J * J + sub * JL + q] = Xc[q];
            }
        }
    }
}

template <int R, int J>
__global__ void __launch_bounds__(kSliceThreads) k_slices_combine(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int MS = J * J + J;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const unsigned m = group_mask<T>(lane);
    const int64_t groups = (int64_t)gridDim.x * (kSliceThreads / T);
    for (int64_t item = (int64_t)blockIdx.x * (kSliceThreads / T) + threadIdx.x / T;
         item < g.ntiles - 1; item += groups) {
        int32_t r;
        int64_t s, e;
        if (!first_boundary_slice(g, item + 1, r, s, e) || e - s <= g.Lseq) continue;
        // the row after the slice's head (run by the chain kernel), then the
        // block maps of its map region [hs, e) in order
        float *arow = g.a.A + (int64_t)r * J + sub * JL;
        float av[JL];
        load_run<JL>(arow, av);
        const int64_t hs = s + g.Lhead;
        const int64_t t0 = hs / g.W, t1 = (e - 1) / g.W;
        const int64_t Bc = block_len(t1 - t0 + 1);
        for (int64_t t = t0; t <= t1; t += Bc) {
            const float *mp = g.maps + (t * 2 + piece_slot(hs, t, g.W)) * (int64_t)MS;
            float full[J];
#pragma unroll
            for (int k = 0; k < J; ++k) full[k] = __shfl_sync(m, av[k % JL], k / JL, T);
#pragma unroll
            for (int q = 0; q < JL; ++q) {
                const float *row = mp + (sub * JL + q) * J;
                float acc = __ldcg(mp + J * J + sub * JL + q);
#pragma unroll
                for (int k4 = 0; k4 < J / 4; ++k4) {
                    const float4 v = __ldcg(reinterpret_cast<const float4 *>(row) + k4);
                    acc = fmaf(v.x, full[4 * k4], acc);
                    acc = fmaf(v.y, full[4 * k4 + 1], acc);
                    acc = fmaf(v.z, full[4 * k4 + 2], acc);
                    acc = fmaf(v.w, full[4 * k4 + 3], acc);
                }
                av[q] = acc;
            }
        }
        if constexpr (JL >= 4) {
#pragma unroll
            for (int q = 0; q < JL / 4; ++q)
                *reinterpret_cast<float4 *>(arow + 4 * q) =
                    make_float4(av[4 * q], av[4 * q + 1], av[4 * q + 2], av[4 * q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < JL; ++q) arow[q] = av[q];
        }
    }
}

// ============================================================================ launchers
// Tile lengths of the factor and core passes, clamped to [32, 2048].  Measured
// on the ratings tensor (90M nonzeros, 152 SMs): the factor pass is fastest at
// nnz / (SMs * 1024) (578 positions: fewer pieces to compose), the core pass at
// nnz / (SMs * 4096) (144 positions).
#ifndef SFT_FACTOR_TILE_DIV
#define SFT_FACTOR_TILE_DIV 1024
#endif
#ifndef SFT_CORE_TILE_DIV
#define SFT_CORE_TILE_DIV 4096
#endif

static int clamp_tile(int64_t W) { return (int)(W < 32 ? 32 : (W > 2048 ? 2048 : W)); }

int slice_tile_length(int64_t nnz, int sms) {
    return clamp_tile(nnz / ((int64_t)sms * SFT_FACTOR_TILE_DIV));
}

int slice_core_tile_length(int64_t nnz, int sms) {
    return clamp_tile(nnz / ((int64_t)sms * SFT_CORE_TILE_DIV));
}

// The pass's chain list: every crossing slice (one that spans a tile
// boundary) of at most Lseq nonzeros, and, when long slices have a head
// (Lhead > 0), every longer crossing slice too (for its head).  A chain of at
// least gram_min positions (gram_min > 0) is stored from the back of the list
// (count[1]) for the blocked-chain kernel, shorter ones from the front
// (count[0]) unless gram_only (the one-lane kernel takes them from its own
// work list); the list has room for `cap` entries (one per tile boundary).
__global__ void k_chain_list(const int32_t *__restrict__ row_ptr, int32_t In, int64_t W,
                             int64_t Lseq, int64_t Lhead, int64_t nnz, int64_t gram_min,
                             int gram_only, int64_t cap, int32_t *list, unsigned int *count) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < In;
         r += (int64_t)gridDim.x * blockDim.x) {
        bool gram;
        const int64_t run = chain_run(row_ptr, (int32_t)r, W, Lseq, Lhead, nnz, gram_min, &gram);
        if (run <= 0) continue;
        if (gram)
            list[cap - 1 - atomicAdd(&count[1], 1u)] = (int32_t)r;
        else if (!gram_only)
            list[atomicAdd(&count[0], 1u)] = (int32_t)r;
    }
}

// list_ws: 16 bytes of counts, then room for one row per tile boundary.
cudaError_t launch_chain_list(SliceArgs &g, void *list_ws, bool gram_only, cudaStream_t st,
                              int sms, int64_t *launches) {
    g.nchains = (unsigned int *)list_ws;
    g.chains = (int32_t *)((char *)list_ws + 16);
    cudaError_t e = cudaMemsetAsync(g.nchains, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int32_t In = g.a.dims[g.a.n];
    int64_t blocks = (In + 255) / 256;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    if (blocks < 1) blocks = 1;
    k_chain_list<<<(int)blocks, 256, 0, st>>>(g.row_ptr, In, g.W, g.Lseq, g.Lhead, g.a.nnz,
                                               g.gram ? kGramMin : 0, gram_only ? 1 : 0,
                                               g.ntiles < 1 ? 1 : g.ntiles, g.chains, g.nchains);
    *launches += 1;
    return cudaGetLastError();
}

// The one-lane kernel's work list, sorted by length: the interiors of the
// tiles and the chains below the blocked kernel's threshold, as item * 2 +
// kind, grouped by length class (longest first; order within a class
// arbitrary: every item writes only its own rows, so the order affects no
// result).  Item k of the enumeration: k < ntiles is tile k, else row
// k - ntiles.
__device__ __forceinline__ int64_t lane_item_len(const SliceArgs &g, int64_t k, int64_t gram_min,
                                                 uint32_t *item) {
    if (k < g.ntiles) {
        int64_t q0, q1;
        if (!tile_inner(g, k, q0, q1)) {
            atomicOr(g.a.err, kErrIndex);
            return 0;
        }
        *item = (uint32_t)(k << 1);
        return q1 - q0;
    }
    const int64_t r = k - g.ntiles;
    bool gram;
    const int64_t run = chain_run(g.row_ptr, (int32_t)r, g.W, g.Lseq, g.Lhead, g.a.nnz, gram_min,
                                  &gram);
    *item = (uint32_t)((r << 1) | 1);
    return gram ? 0 : run;
}

constexpr int kLaneListThreads = 256;

// Pass 1: items per length class (block histograms, added to lane_cnt[0..]).
__global__ void __launch_bounds__(kLaneListThreads) k_lane_count(SliceArgs g, int64_t gram_min) {
    __shared__ unsigned int h[kLaneBuckets];
    for (int b = threadIdx.x; b < kLaneBuckets; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int64_t n = g.ntiles + g.a.dims[g.a.n];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t item;
        const int64_t len = lane_item_len(g, k, gram_min, &item);
        if (len > 0) atomicAdd(&h[lane_bucket(len)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kLaneBuckets; b += blockDim.x)
        if (h[b]) atomicAdd(&g.lane_cnt[b], h[b]);
}

// Pass 2: every block counts its own items per class again, reserves a range
// of each class from the cursors (lane_cnt[kLaneBuckets + b]), and places its
// items in it.  The class starts are the prefix sums of the pass-1 counts.
__global__ void __launch_bounds__(kLaneListThreads) k_lane_scatter(SliceArgs g, int64_t gram_min) {
    __shared__ unsigned int start[kLaneBuckets];  // class starts, then this block's range starts
    __shared__ unsigned int h[kLaneBuckets];
    if (threadIdx.x < 32) {  // exclusive prefix sum of the class counts, 4 classes per lane
        unsigned int c[kLaneBuckets / 32], run = 0;
#pragma unroll
        for (int i = 0; i < kLaneBuckets / 32; ++i) {
            c[i] = g.lane_cnt[threadIdx.x * (kLaneBuckets / 32) + i];
            run += c[i];
        }
        unsigned int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)threadIdx.x >= o) incl += y;
        }
        unsigned int off = incl - run;
#pragma unroll
        for (int i = 0; i < kLaneBuckets / 32; ++i) {
            start[threadIdx.x * (kLaneBuckets / 32) + i] = off;
            off += c[i];
        }
    }
    for (int b = threadIdx.x; b < kLaneBuckets; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int64_t n = g.ntiles + g.a.dims[g.a.n];
    const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = k0; k < n; k += stride) {
        uint32_t item;
        const int64_t len = lane_item_len(g, k, gram_min, &item);
        if (len > 0) atomicAdd(&h[lane_bucket(len)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kLaneBuckets; b += blockDim.x) {
        const unsigned int mine = h[b];
        start[b] += mine ? atomicAdd(&g.lane_cnt[kLaneBuckets + b], mine) : 0u;
        h[b] = 0;
    }
    __syncthreads();
    for (int64_t k = k0; k < n; k += stride) {
        uint32_t item;
        const int64_t len = lane_item_len(g, k, gram_min, &item);
        if (len <= 0) continue;
        const int b = lane_bucket(len);
        g.lane_items[start[b] + atomicAdd(&h[b], 1u)] = item;
    }
}

// list_ws: the class counts, cursors and grab counter (2 kLaneBuckets + 4
// words), then room for one item per tile and one per row of the mode.
cudaError_t launch_lane_list(SliceArgs &g, void *list_ws, cudaStream_t st, int sms,
                             int64_t *launches) {
    g.lane_cnt = (unsigned int *)list_ws;
    g.lane_items = (uint32_t *)((char *)list_ws + (2 * kLaneBuckets + 4) * sizeof(unsigned int));
    cudaError_t e = cudaMemsetAsync(g.lane_cnt, 0, (2 * kLaneBuckets + 4) * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int64_t n = g.ntiles + g.a.dims[g.a.n];
    int64_t blocks = (n + kLaneListThreads - 1) / kLaneListThreads;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    if (blocks < 1) blocks = 1;
    const int64_t gram_min = g.gram ? kGramMin : 0;
    k_lane_count<<<(int)blocks, kLaneListThreads, 0, st>>>(g, gram_min);
    k_lane_scatter<<<(int)blocks, kLaneListThreads, 0, st>>>(g, gram_min);
    *launches += 2;
    return cudaGetLastError();
}

size_t slice_maps_bytes(int64_t ntiles, int J) {
    return (size_t)(ntiles < 1 ? 1 : ntiles) * 2 * (size_t)(J * J + J) * sizeof(float);
}

// Workspace of a slice factor pass: the piece maps, the chain list (a count
// and one row per tile), the piece list (two counts and two entries per
// tile), then the one-lane work list, each part starting on a 16-byte
// boundary.
size_t slice_chain_list_offset(int64_t ntiles, int J) { return slice_maps_bytes(ntiles, J); }

size_t slice_piece_list_offset(int64_t ntiles, int J) {
    const size_t o = slice_chain_list_offset(ntiles, J) + 16 + (size_t)(ntiles < 1 ? 1 : ntiles) * 4;
    return (o + 15) / 16 * 16;
}

size_t slice_lane_list_offset(int64_t ntiles, int J) {
    const size_t o = slice_piece_list_offset(ntiles, J) + 16 + (size_t)(ntiles < 1 ? 1 : ntiles) * 2 * 4;
    return (o + 15) / 16 * 16;
}

// The lane list needs the mode's length I_n too (one item per row at most).
size_t slice_workspace_total(int64_t ntiles, int J, int64_t In) {
    return slice_lane_list_offset(ntiles, J) + (2 * kLaneBuckets + 4) * sizeof(unsigned int) +
           (size_t)((ntiles < 1 ? 1 : ntiles) + (In < 0 ? 0 : In)) * 4;
}

// The pass's map pieces into the piece list: full-tile pieces from the front,
// shorter ones from the back (each piece writes only its own map slot, so the
// order of the list affects no result).
__global__ void k_piece_list(SliceArgs g) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        for (int side = 0; side < 2; ++side) {
            int32_t r;
            int64_t s, e, hs, q0, q1;
            if (!map_piece(g, t, side, r, s, e, hs, q0, q1)) continue;
            const int32_t entry = (int32_t)(t * 2 + side);
            if (q1 - q0 == g.W) g.pieces[atomicAdd(&g.npieces[0], 1u)] = entry;
            else g.pieces[2 * g.ntiles - 1 - atomicAdd(&g.npieces[1], 1u)] = entry;
        }
    }
}

// The map pieces of the pass into g.pieces / g.npieces (list_ws: the piece
// list part of the workspace).
cudaError_t launch_piece_list(SliceArgs &g, void *list_ws, cudaStream_t st, int sms,
                              int64_t *launches) {
    g.npieces = (unsigned int *)list_ws;
    g.pieces = (int32_t *)((char *)list_ws + 16);
    cudaError_t e = cudaMemsetAsync(g.npieces, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = (g.ntiles + 255) / 256;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    if (blocks < 1) blocks = 1;
    k_piece_list<<<(int)blocks, 256, 0, st>>>(g);
    *launches += 1;
    return cudaGetLastError();
}

template <typename F>
static void dispatch_nb(int N, F &&f) {
    // the template argument is the number of other-mode slots (>= N - 1)
    if (N <= 3) f(ic<2>{});
    else if (N <= 4) f(ic<3>{});
    else if (N <= 8) f(ic<7>{});
    else f(ic<15>{});
}

cudaError_t launch_factor_slices(const PassArgs &a, const int32_t *row_ptr, int64_t W, int64_t Lseq,
                                 bool subslices, bool gram, float *maps, int J, int R,
                                 const SliceStreams &ss_in, int sms, int64_t *launches) {
    (void)gram;  // the blocked chains read v from the fiber table
    SliceStreams ss = ss_in;
    const cudaStream_t st = ss.tiles;
    const bool fork = ss.fork && ss.chains_done && ss.maps_done && ss.chains && ss.maps &&
                      ss.chains != st && ss.maps != st;
    if (fork) {
        cudaEventRecord(ss.fork, st);
        cudaStreamWaitEvent(ss.chains, ss.fork, 0);
        cudaStreamWaitEvent(ss.maps, ss.fork, 0);
    } else {
        ss.chains = ss.maps = st;
    }
    SliceArgs g{};
    g.a = a;
    g.row_ptr = row_ptr;
    g.W = W;
    g.Lseq = Lseq;
    g.Lhead = subslices ? 0 : Lseq;
    g.subslices = subslices ? 1 : 0;
    g.ntiles = (a.nnz + W - 1) / W;
    g.maps = maps;
    const bool with_maps = maps != nullptr;
    {
        cudaError_t e = launch_chain_list(g, (char *)maps + slice_chain_list_offset(g.ntiles, J),
                                          false, ss.chains, sms, launches);
        if (e == cudaSuccess && with_maps && !subslices)
            e = launch_piece_list(g, (char *)maps + slice_piece_list_offset(g.ntiles, J), ss.maps,
                                  sms, launches);
        if (e != cudaSuccess) return e;
    }
    if (a.cbf16) {
        if (a.N <= 3) factor_slices_no2_bf16(g, R, J, with_maps, ss, sms, launches);
        else if (a.N <= 4) factor_slices_no3_bf16(g, R, J, with_maps, ss, sms, launches);
        else if (a.N <= 8) factor_slices_no7_bf16(g, R, J, with_maps, ss, sms, launches);
        else factor_slices_no15_bf16(g, R, J, with_maps, ss, sms, launches);
    } else {
        if (a.N <= 3) factor_slices_no2_f32(g, R, J, with_maps, ss, sms, launches);
        else if (a.N <= 4) factor_slices_no3_f32(g, R, J, with_maps, ss, sms, launches);
        else if (a.N <= 8) factor_slices_no7_f32(g, R, J, with_maps, ss, sms, launches);
        else factor_slices_no15_f32(g, R, J, with_maps, ss, sms, launches);
    }
    if (fork) {
        cudaEventRecord(ss.chains_done, ss.chains);
        cudaEventRecord(ss.maps_done, ss.maps);
        cudaStreamWaitEvent(st, ss.chains_done, 0);
        cudaStreamWaitEvent(st, ss.maps_done, 0);
    }
    if (with_maps && !subslices && g.ntiles > 1) {
        cudaError_t e = launch_slice_combine(g, J, R, st, sms);
        *launches += 2;
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Compose the piece maps of long slices in blocks, then apply them in order
// to the rows (after the map kernel has finished).
cudaError_t launch_slice_combine(const SliceArgs &g, int J, int R, cudaStream_t st, int sms) {
    dispatch_rj(R, J, [&](auto r_c, auto j_c) {
        constexpr int R_ = decltype(r_c)::value, J_ = decltype(j_c)::value;
        const int gpb = kSliceThreads / (R_ / 4);
        const int cth = kComposeGroups * (R_ / 4);
        if constexpr (J_ <= 16 && J_ / (R_ / 4) <= 4) {
            const int gc = grid_for(k_slices_compose<R_, J_>, cth, 0, kComposeGroups, g.ntiles, sms);
            k_slices_compose<R_, J_><<<gc, cth, 0, st>>>(g);
        } else {
            const int gc = grid_for(k_slices_compose_smem<R_, J_>, cth, 0, kComposeGroups, g.ntiles,
                                    sms);
            k_slices_compose_smem<R_, J_><<<gc, cth, 0, st>>>(g);
        }
        const int gb = grid_for(k_slices_combine<R_, J_>, kSliceThreads, 0, gpb, g.ntiles, sms);
        k_slices_combine<R_, J_><<<gb, kSliceThreads, 0, st>>>(g);
    });
    return cudaGetLastError();
}

cudaError_t launch_core_slices(const PassArgs &a, const int32_t *row_ptr, int64_t W, int J, int R,
                               float *partials, int max_blocks, cudaStream_t st, int sms,
                               int64_t *launches) {
    SliceArgs g{};
    g.a = a;
    g.row_ptr = row_ptr;
    g.W = W;
    g.Lseq = 0;
    g.ntiles = (a.count + W - 1) / W;
    g.maps = nullptr;
    int nblk;
    if (a.cbf16) {
        if (a.N <= 3) nblk = core_slices_no2_bf16(g, R, J, partials, max_blocks, st, sms);
        else if (a.N <= 4) nblk = core_slices_no3_bf16(g, R, J, partials, max_blocks, st, sms);
        else if (a.N <= 8) nblk = core_slices_no7_bf16(g, R, J, partials, max_blocks, st, sms);
        else nblk = core_slices_no15_bf16(g, R, J, partials, max_blocks, st, sms);
    } else {
        if (a.N <= 3) nblk = core_slices_no2_f32(g, R, J, partials, max_blocks, st, sms);
        else if (a.N <= 4) nblk = core_slices_no3_f32(g, R, J, partials, max_blocks, st, sms);
        else if (a.N <= 8) nblk = core_slices_no7_f32(g, R, J, partials, max_blocks, st, sms);
        else nblk = core_slices_no15_f32(g, R, J, partials, max_blocks, st, sms);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 2;
    return launch_core_apply(a.B, partials, nblk, J * R, a.count, a.lr, a.lam, st);
}

}  // namespace sft
