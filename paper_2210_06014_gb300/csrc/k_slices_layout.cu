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
//     parallel (k_slices_maps); k_slices_compose_w multiplies blocks of
//     consecutive piece maps and k_slices_combine_w applies them to the row, in
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


// The mode-n coordinates of a slice layout from its row_ptr alone (every
// position of slice r holds r).  A warp takes a span of 32 x kExpandPer
// consecutive positions; lane l writes positions l, l + 32, ... of it (stores
// coalesced across the warp), finds the slice of its first position by binary
// search and then only steps r forward past the slice ends it crosses.
constexpr int kExpandPer = 64;

__global__ void k_expand_rows(const int32_t *__restrict__ row_ptr, int32_t In, int64_t nnz,
                              int32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int64_t kSpan = 32 * kExpandPer;
    for (int64_t c0 = warp * kSpan; c0 < nnz; c0 += nwarps * kSpan) {
        const int64_t c1 = min(nnz, c0 + kSpan);
        int64_t p = c0 + lane;
        if (p >= c1) continue;
        // last r with row_ptr[r] <= p (row_ptr is non-decreasing, row_ptr[0] = 0)
        int32_t lo = 0, hi = In;
        while (lo < hi) {
            const int32_t mid = (int32_t)(((int64_t)lo + hi + 1) >> 1);
            if (__ldg(row_ptr + mid) <= p) lo = mid; else hi = mid - 1;
        }
        int32_t r = lo;
        int64_t next = r < In ? __ldg(row_ptr + r + 1) : nnz;
        for (; p < c1; p += 32) {
            while (p >= next && r < In) {
                ++r;
                next = r < In ? __ldg(row_ptr + r + 1) : nnz;
            }
            out[p] = r < In ? r : -1;  // positions after the last slice (bad data) get -1
        }
    }
}

cudaError_t launch_expand_rows(const int32_t *row_ptr, int32_t In, int64_t nnz, int32_t *out,
                               cudaStream_t st, int sms) {
    if (nnz <= 0) return cudaSuccess;
    const int64_t span = 32 * kExpandPer;
    int64_t b = ((nnz + span - 1) / span + 7) / 8;  // 8 warps per block
    if (b > (int64_t)sms * 8) b = (int64_t)sms * 8;
    k_expand_rows<<<(int)b, 256, 0, st>>>(row_ptr, In, nnz, out);
    return cudaGetLastError();
}

// ============================================================================ long slices: combine
// Pieces of a long slice (one per tile it touches) are grouped into blocks of
// Bc = ceil(sqrt(K)) consecutive pieces (K pieces in all).  k_slices_compose_w
// folds each block into one map, in place in the slot of its first piece
// (X = P_last; X = X o P for the earlier pieces: X.M <- X.M P.M,
// X.c <- X.M P.c + X.c), and k_slices_combine_w applies the block maps to the
// row in order.

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

// ---------------------------------------------------------------------------- one warp per chain
// The block products of the composition and the block-map applications are
// sequential chains; the longest chain (the longest
// slice: Bc = ceil(sqrt(K)) products, K up to ~1e4 pieces on a Zipf mode)
// sets their time.  These forms give each chain a whole warp, taken from
// lists built by k_long_list (every long slice, and every block start of its
// map region), so a product or an application is short and no warp idles on
// the tiles that start no block.  The arithmetic (each entry's sums in
// ascending order) is that of the lane-group forms, bit for bit.

// Lane layout of a J x J map over one warp: LPR lanes per row, CPL columns
// per lane (J = 4 uses 16 lanes).
template <int J>
struct WarpMap {
    static constexpr int LPR = (32 / J) < J ? (32 / J) : J;
    static constexpr int CPL = J / LPR;
    static constexpr int LANES = J * LPR;
};
constexpr int kWarpMapWarps = 4;   // warps per block of the warp-per-chain kernels
constexpr int kCombineRing = 4;    // block maps staged ahead by k_slices_combine_w (J <= 16)

// The long slices of the pass (rows, into longs) and the block starts of their
// map regions (t * 2 + slot, into starts).  counts[0] / counts[1] receive the
// two lengths.
__global__ void k_long_list(SliceArgs g, int32_t *longs, int32_t *starts, unsigned int *counts) {
    const int32_t In = g.a.dims[g.a.n];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < In;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g.row_ptr[r], e = g.row_ptr[r + 1];
        if (s < 0 || s >= e || e > g.a.nnz) continue;
        if (e - s <= g.Lseq || s / g.W == (e - 1) / g.W) continue;  // not long / not crossing
        const int64_t hs = s + g.Lhead;
        if (hs >= e) continue;
        longs[atomicAdd(&counts[0], 1u)] = (int32_t)r;
        const int64_t t0 = hs / g.W, t1 = (e - 1) / g.W;
        const int64_t Bc = block_len(t1 - t0 + 1);
        for (int64_t t = t0; t <= t1; t += Bc)
            if (min(t + Bc - 1, t1) > t)  // a block of one piece is already its own map
                starts[atomicAdd(&counts[1], 1u)] = (int32_t)(t * 2 + piece_slot(hs, t, g.W));
    }
}

template <int J>
__global__ void __launch_bounds__(kWarpMapWarps * 32) k_slices_compose_w(SliceArgs g,
                                                                       const int32_t *starts,
                                                                       const unsigned int *count) {
    using WM = WarpMap<J>;
    constexpr int MS = J * J + J;
    constexpr int CH = MS / 4;  // 16-byte chunks of one map
    constexpr int CPL = WM::CPL;
    __shared__ __align__(16) float sP[kWarpMapWarps][2][MS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane / WM::LPR, part = lane % WM::LPR, c0 = part * CPL;
    const bool act = lane < WM::LANES;
    const int rbase = lane - part;  // first lane of this lane's row
    const int64_t n = (int64_t)*count;
    auto stage = [&](const float *P, float *dst) {
        for (int c = lane; c < CH; c += 32) {
            const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + 4 * c));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(P + 4 * c)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int64_t k = (int64_t)blockIdx.x * kWarpMapWarps + warp; k < n;
         k += (int64_t)gridDim.x * kWarpMapWarps) {
        const int32_t entry = starts[k];
        const int64_t t = entry >> 1;
        const int side = entry & 1;
        int32_t row;
        int64_t s, e, hs;
        if (t >= g.ntiles || !long_piece(g, t, side, row, s, e, hs)) continue;
        const int64_t t0 = hs / g.W, t1 = (e - 1) / g.W;
        const int64_t Bc = block_len(t1 - t0 + 1);
        const int64_t tl = min(t + Bc - 1, t1);
        if (tl == t || (t - t0) % Bc != 0) continue;
        auto map_of = [&](int64_t u) {
            return g.maps + (u * 2 + piece_slot(hs, u, g.W)) * (int64_t)MS;
        };
        stage(map_of(tl - 1), sP[warp][0]);
        // X = the last piece's map; every lane of a row holds the whole row
        float X[J], Xc = 0.f;
        {
            const float *P = map_of(tl);
#pragma unroll
            for (int l = 0; l < J; l += 4) {
                const float4 v = act ? __ldcg(reinterpret_cast<const float4 *>(P + r * J + l))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                X[l] = v.x; X[l + 1] = v.y; X[l + 2] = v.z; X[l + 3] = v.w;
            }
            if (act) Xc = __ldcg(P + J * J + r);
        }
        int cur = 0;
        for (int64_t u = tl - 1; u >= t; --u) {
            if (u > t) {
                stage(map_of(u - 1), sP[warp][cur ^ 1]);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncwarp();  // every lane's chunks of P have landed
            const float *P = sP[warp][cur];
            // X <- X o P on the lane's columns: X.M <- X.M P.M, X.c <- X.M P.c + X.c
            float nx[CPL];
#pragma unroll
            for (int q = 0; q < CPL; ++q) nx[q] = 0.f;
            float acc = Xc;
#pragma unroll
            for (int l = 0; l < J; ++l) {
                const float x = X[l];
                if constexpr (CPL % 4 == 0) {
#pragma unroll
                    for (int q = 0; q < CPL; q += 4) {
                        const float4 pv = *reinterpret_cast<const float4 *>(P + l * J + c0 + q);
                        nx[q] = fmaf(x, pv.x, nx[q]);
                        nx[q + 1] = fmaf(x, pv.y, nx[q + 1]);
                        nx[q + 2] = fmaf(x, pv.z, nx[q + 2]);
                        nx[q + 3] = fmaf(x, pv.w, nx[q + 3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < CPL; ++q) nx[q] = fmaf(x, P[l * J + c0 + q], nx[q]);
                }
                acc = fmaf(x, P[J * J + l], acc);
            }
            __syncwarp();  // P fully read before its buffer is refilled
            // the whole new row back into every lane of the row
#pragma unroll
            for (int j = 0; j < J; ++j) X[j] = __shfl_sync(0xffffffffu, nx[j % CPL], rbase + j / CPL);
            Xc = acc;
            cur ^= 1;
        }
        if (act) {
            float *out = map_of(t);
#pragma unroll
            for (int j = 0; j < J; ++j)  // the lane's columns (no run-time register index)
                if (j / CPL == part) out[r * J + j] = X[j];
            if (part == 0) out[J * J + r] = Xc;
        }
        __syncwarp();
    }
}

// Applies the block maps of each long slice's map region, in order, to the
// row its head left: lane j < J forms entry j (c_j, then the row's dot product
// in ascending order), the block maps staged kCombineRing ahead with cp.async.
template <int J>
__global__ void __launch_bounds__(kWarpMapWarps * 32) k_slices_combine_w(SliceArgs g,
                                                                       const int32_t *longs,
                                                                       const unsigned int *count) {
    constexpr int MS = J * J + J;
    constexpr int CH = MS / 4;
    constexpr int D = J <= 16 ? kCombineRing : 2;
    __shared__ __align__(16) float sM[kWarpMapWarps][D][MS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = (int64_t)*count;
    for (int64_t k = (int64_t)blockIdx.x * kWarpMapWarps + warp; k < n;
         k += (int64_t)gridDim.x * kWarpMapWarps) {
        const int32_t r = longs[k];
        if (r < 0 || r >= g.a.dims[g.a.n]) continue;
        const int64_t s = __ldg(g.row_ptr + r), e = __ldg(g.row_ptr + r + 1);
        if (!slice_ok(g, s, e)) continue;
        const int64_t hs = s + g.Lhead;
        const int64_t t0 = hs / g.W, t1 = (e - 1) / g.W;
        const int64_t Bc = block_len(t1 - t0 + 1);
        const int64_t nb = (t1 - t0) / Bc + 1;  // block maps, at t0, t0 + Bc, ...
        auto map_of = [&](int64_t b) {
            const int64_t t = t0 + b * Bc;
            return g.maps + (t * 2 + piece_slot(hs, t, g.W)) * (int64_t)MS;
        };
        auto stage = [&](int64_t b) {
            if (b < nb) {
                const float *P = map_of(b);
                float *dst = sM[warp][b % D];
                for (int c = lane; c < CH; c += 32) {
                    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + 4 * c));
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d),
                                 "l"(P + 4 * c)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        float *arow = g.a.A + (int64_t)r * J;
        float a[J];
#pragma unroll
        for (int l = 0; l < J; l += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(arow + l);
            a[l] = v.x; a[l + 1] = v.y; a[l + 2] = v.z; a[l + 3] = v.w;
        }
        for (int64_t b = 0; b < D - 1; ++b) stage(b);
        for (int64_t b = 0; b < nb; ++b) {
            stage(b + D - 1);
            asm volatile("cp.async.wait_group %0;" ::"n"(D - 1) : "memory");
            __syncwarp();  // block map b has landed
            const float *M = sM[warp][b % D];
            float acc = 0.f;
            if (lane < J) {
                acc = M[J * J + lane];
#pragma unroll
                for (int l = 0; l < J; l += 4) {
                    const float4 v = *reinterpret_cast<const float4 *>(M + lane * J + l);
                    acc = fmaf(v.x, a[l], acc);
                    acc = fmaf(v.y, a[l + 1], acc);
                    acc = fmaf(v.z, a[l + 2], acc);
                    acc = fmaf(v.w, a[l + 3], acc);
                }
            }
            __syncwarp();  // map b read before its slot is refilled
#pragma unroll
            for (int l = 0; l < J; ++l) a[l] = __shfl_sync(0xffffffffu, acc, l);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int l = 0; l < J; ++l)  // lane l writes entry l (no run-time register index)
            if (lane == l) arow[l] = a[l];
        __syncwarp();
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
// tile), the combine lists, then the one-lane work list, each part starting
// on a 16-byte boundary.
size_t slice_chain_list_offset(int64_t ntiles, int J) { return slice_maps_bytes(ntiles, J); }

size_t slice_piece_list_offset(int64_t ntiles, int J) {
    const size_t o = slice_chain_list_offset(ntiles, J) + 16 + (size_t)(ntiles < 1 ? 1 : ntiles) * 4;
    return (o + 15) / 16 * 16;
}

// The combine lists: two counts, then a row per long slice (at most one per
// tile boundary) and a block start per piece (at most two per tile).
size_t slice_combine_list_offset(int64_t ntiles, int J) {
    const size_t o = slice_piece_list_offset(ntiles, J) + 16 + (size_t)(ntiles < 1 ? 1 : ntiles) * 2 * 4;
    return (o + 15) / 16 * 16;
}

size_t slice_lane_list_offset(int64_t ntiles, int J) {
    const size_t o = slice_combine_list_offset(ntiles, J) + 16 + (size_t)(ntiles < 1 ? 1 : ntiles) * 3 * 4;
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
    (void)R;
    char *base = (char *)g.maps + slice_combine_list_offset(g.ntiles, J);
    unsigned int *counts = (unsigned int *)base;
    int32_t *longs = (int32_t *)(base + 16);
    int32_t *starts = longs + (g.ntiles < 1 ? 1 : g.ntiles);
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int32_t In = g.a.dims[g.a.n];
    int64_t lb = ((int64_t)In + 255) / 256;
    if (lb > (int64_t)sms * 4) lb = (int64_t)sms * 4;
    if (lb < 1) lb = 1;
    k_long_list<<<(int)lb, 256, 0, st>>>(g, longs, starts, counts);
    auto run = [&](auto j_c) {
        constexpr int J_ = decltype(j_c)::value;
        const int gc = grid_for(k_slices_compose_w<J_>, kWarpMapWarps * 32, 0, kWarpMapWarps,
                                (int64_t)1 << 30, sms);
        k_slices_compose_w<J_><<<gc, kWarpMapWarps * 32, 0, st>>>(g, starts, counts + 1);
        const int gb = grid_for(k_slices_combine_w<J_>, kWarpMapWarps * 32, 0, kWarpMapWarps,
                                (int64_t)1 << 30, sms);
        k_slices_combine_w<J_><<<gb, kWarpMapWarps * 32, 0, st>>>(g, longs, counts);
    };
    switch (J) {
        case 4: run(ic<4>{}); break;
        case 8: run(ic<8>{}); break;
        case 16: run(ic<16>{}); break;
        case 32: run(ic<32>{}); break;
        default: break;
    }
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
