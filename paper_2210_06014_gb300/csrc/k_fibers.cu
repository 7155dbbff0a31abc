// k_fibers.cu -- fibers of a slice layout and their shared vectors, the
// "shared intermediate variables" of cuFasterTucker (Section "Reusable
// Intermediate Variables", Eq. (12)-(13)).
//
// For mode n a fiber is a tuple (i_k)_{k != n}.  All nonzeros of one fiber
// share p = prod_{k != n} C^(k)[i_k] and v = B^(n) p, and during a factor pass
// over mode n neither C^(k != n) nor B^(n) changes, so v can be formed once
// per fiber at the start of the pass instead of once per nonzero.
//
// Fiber ids (layout time): the exact 64-bit linear key of the tuple is
// inserted into an open-addressing table (atomicCAS, linear probing, bounded
// by the table size, which is at least twice the number of nonzeros), which
// also keeps the first layout position of each fiber (atomicMin); fibers are
// then numbered in the order of their first positions (a scan over the
// positions), so that a walk over the layout meets fibers it has not seen
// before in increasing order and reads their v rows as a stream.  Ids do not
// depend on scheduling, and each fiber's v does not depend on its id.
//
// Per pass: k_fiber_v forms every fiber's v with the same arithmetic, in the
// same order, as the per-nonzero path (product of the other modes' rows in
// ascending mode order, partial products with B over the lane's r, group
// reduce-scatter), so the fiber path gives the same bits.
#include "slices_impl.cuh"

namespace sft {

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kFibThreads = 256;

__device__ __forceinline__ unsigned long long mix_key(unsigned long long z) {
    // SplitMix64 finaliser (Steele, Lea, Flood 2014), used only to spread keys
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebull;
    z ^= z >> 31;
    return z;
}

struct FiberKeyArgs {
    const int32_t *oidx[kMaxOrder];
    int32_t odims[kMaxOrder];
    unsigned long long stride[kMaxOrder];
    int no;  // number of other modes
};

struct FiberCoords {
    const int32_t *c[kMaxOrder];  // [q][f]: coordinate of other mode q of fiber f
};
struct FiberCoordsOut {
    int32_t *c[kMaxOrder];
};

__global__ void k_fiber_clear(unsigned long long *table, int32_t *slot_pos, int64_t cap) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (int64_t)gridDim.x * blockDim.x) {
        table[i] = kEmpty;
        slot_pos[i] = 0x7fffffff;
    }
}

// slot_of[t] = table slot of position t's fiber (-1 for bad coordinates);
// slot_pos[slot] = the fiber's first layout position (its representative).
__global__ void k_fiber_insert(FiberKeyArgs f, int64_t nnz, unsigned long long *table,
                               int32_t *slot_pos, int64_t cap, int32_t *slot_of, int *err) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = 0;
        bool ok = true;
        for (int q = 0; q < f.no; ++q) {
            const int32_t i = f.oidx[q][t];
            if ((uint32_t)i >= (uint32_t)f.odims[q]) ok = false;
            else key += (unsigned long long)i * f.stride[q];
        }
        if (!ok) {
            atomicOr(err, kErrIndex);
            slot_of[t] = -1;
            continue;
        }
        int64_t h = (int64_t)(mix_key(key) & (unsigned long long)(cap - 1));
        int32_t slot = -1;
        for (int64_t probe = 0; probe < cap; ++probe) {
            const unsigned long long prev = atomicCAS(table + h, kEmpty, key);
            if (prev == kEmpty || prev == key) {
                atomicMin(slot_pos + h, (int32_t)t);
                slot = (int32_t)h;
                break;
            }
            h = (h + 1) & (cap - 1);
        }
        if (slot < 0) atomicOr(err, kErrIndex);  // unreachable: cap >= 2 nnz
        slot_of[t] = slot;
    }
}

// Numbering in the order of first positions.  A position is a representative
// when it is its fiber's first position; kScanBlock positions per block.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ bool is_rep(const int32_t *slot_of, const int32_t *slot_pos, int64_t t,
                                       int64_t nnz) {
    if (t >= nnz) return false;
    const int32_t s = slot_of[t];
    return s >= 0 && slot_pos[s] == (int32_t)t;
}

// counts[b] = representatives among positions [b * kScanBlock, (b + 1) * kScanBlock)
__global__ void __launch_bounds__(kScanBlock) k_fiber_count(const int32_t *slot_of,
                                                            const int32_t *slot_pos, int64_t nnz,
                                                            int32_t *counts) {
    __shared__ int32_t wsum[kScanBlock / 32];
    const int64_t t = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const unsigned b = __ballot_sync(kFull, is_rep(slot_of, slot_pos, t, nnz));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t c = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) c += wsum[w];
        counts[blockIdx.x] = c;
    }
}

// Exclusive prefix sums of the block counts (one block, in place), and the
// total into *count.
__global__ void __launch_bounds__(1024) k_fiber_scan(int32_t *counts, int64_t nblocks,
                                                     unsigned long long *count) {
    __shared__ long long carry;
    __shared__ int32_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nblocks; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < nblocks ? counts[i] : 0;
        // inclusive scan inside the warp, then across warps
        int32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, x, d);
            if ((threadIdx.x & 31) >= d) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int32_t w = wsum[threadIdx.x];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, w, d);
                if ((int)threadIdx.x >= d) w += y;
            }
            wsum[threadIdx.x] = w;
        }
        __syncthreads();
        const int32_t before = (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0) + x - v;
        if (i < nblocks) counts[i] = (int32_t)(carry + before);
        __syncthreads();
        if (threadIdx.x == 1023) carry += before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = (unsigned long long)carry;
}

// Ids of the representatives: block offset + rank inside the block.
__global__ void __launch_bounds__(kScanBlock) k_fiber_number(const int32_t *slot_of,
                                                             const int32_t *slot_pos, int64_t nnz,
                                                             const int32_t *offsets,
                                                             int32_t *slot_fid, int32_t *rep) {
    __shared__ int32_t wsum[kScanBlock / 32];
    const int64_t t = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const bool r = is_rep(slot_of, slot_pos, t, nnz);
    const unsigned b = __ballot_sync(kFull, r);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = __popc(b);
    __syncthreads();
    if (r) {
        int32_t before = offsets[blockIdx.x];
        for (int w = 0; w < warp; ++w) before += wsum[w];
        before += __popc(b & ((1u << lane) - 1u));
        slot_fid[slot_of[t]] = before;
        rep[before] = (int32_t)t;
    }
}

__global__ void k_fiber_remap(int32_t *fid, int64_t nnz, const int32_t *slot_fid) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = fid[t];
        fid[t] = s >= 0 ? slot_fid[s] : -1;
    }
}

// fcoord[q][f] = coordinate of other mode q of fiber f (read at its
// representative position), so the per-pass kernels read them sequentially.
__global__ void k_fiber_coords(FiberKeyArgs f, const int32_t *rep,
                               const unsigned long long *count, FiberCoordsOut out) {
    const int64_t nf = (int64_t)*count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t pos = rep[i];
        for (int q = 0; q < f.no; ++q) out.c[q][i] = f.oidx[q][pos];
    }
}

// Gathers the lane's 4 entries of every other mode's cached row of a fiber
// whose coordinates are in ci (checked here; bad ones leave the fiber out).
template <int R, typename CT, int NO>
__device__ __forceinline__ bool fiber_rows(const PassArgs &a, const int32_t (&ci)[NO], bool ok,
                                           int sub, Rows<NO, CT> &w) {
    bool bad = false;
#pragma unroll
    for (int q = 0; q < NO; ++q)
        if (ok && q < a.N - 1 && (uint32_t)ci[q] >= (uint32_t)a.odims[q]) bad = true;
    if (ok && bad) atomicOr(a.err, kErrIndex);
    ok = ok && !bad;
#pragma unroll
    for (int q = 0; q < NO; ++q)
        w.r[q] = (ok && q < a.N - 1) ? ldC_raw_l1<CT>(a.oC[q], (int64_t)ci[q] * R + 4 * sub,
                                                       (a.ol1 >> q) & 1u)
                                     : c_one<CT>();
    return ok;
}

// V[f] = B^(n) prod_{k != n} C^(k)[i_k(f)] for every fiber; T = R/4 lanes per
// fiber, lane `sub` writes entries [sub*J/T, (sub+1)*J/T).  NO bounds the
// number of other modes.  For NO <= 3 a group forms two fibers' v per
// iteration (f and f + stride: each float4 of B read from shared memory serves
// both) while the next pair's coordinates and cached rows are in flight;
// otherwise one fiber per iteration, its coordinates loaded one ahead.
// The lane's JL entries of a fiber's v into the table, as float or rounded
// to bfloat16 (nearest even).
template <typename VT, int JL>
__device__ __forceinline__ void store_v(void *V, int64_t off, const float (&vq)[JL]) {
    if constexpr (sizeof(VT) == 4) {
        store_run<JL>(static_cast<float *>(V) + off, vq);
    } else if constexpr (JL == 1) {
        static_cast<__nv_bfloat16 *>(V)[off] = __float2bfloat16_rn(vq[0]);
    } else {
        uint32_t w[JL / 2];
#pragma unroll
        for (int q = 0; q < JL / 2; ++q) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(vq[2 * q], vq[2 * q + 1]);
            w[q] = *reinterpret_cast<const uint32_t *>(&h);
        }
        __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(V) + off;
        if constexpr (JL == 8) *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        else if constexpr (JL == 4) *reinterpret_cast<uint2 *>(dst) = make_uint2(w[0], w[1]);
        else *reinterpret_cast<uint32_t *>(dst) = w[0];
    }
}

template <int R, int J, typename CT, int NO, typename VT>
__global__ void __launch_bounds__(kFibThreads, (NO <= 3 && J <= 16) ? 3 : 1) k_fiber_v(PassArgs a, FiberCoords fc,
                                                         int64_t nfibers, void *V) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr bool PIPE = NO <= 3;
    __shared__ __align__(16) float sB[J * R];
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = a.B[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const int64_t stride = (int64_t)gridDim.x * (kFibThreads / T);
    // every group of a warp runs the same number of iterations (full-mask shuffles)
    const int64_t first = (int64_t)blockIdx.x * (kFibThreads / T) + threadIdx.x / T;
    const int64_t warp_first = first - (lane / T);
    int32_t nc[NO];
    auto fetch = [&](int64_t f) {
#pragma unroll
        for (int q = 0; q < NO; ++q) nc[q] = (f < nfibers && q < a.N - 1) ? __ldg(fc.c[q] + f) : 0;
    };
    auto emit = [&](int64_t f, bool ok, const Rows<NO, CT> &w) {
        const float4 p = product<NO, CT>(w);
        float vp[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
            vp[j] = fmaf(b.x, p.x, fmaf(b.y, p.y, fmaf(b.z, p.z, b.w * p.w)));
        }
        group_reduce_scatter<T, J>(vp, sub);
        float vq[JL];
#pragma unroll
        for (int q = 0; q < JL; ++q) vq[q] = vp[q];
        if (ok) store_v<VT, JL>(V, f * J + sub * JL, vq);
    };
    if constexpr (PIPE) {
        // two fibers per group and iteration (f and f + stride): every float4 of
        // B read from shared memory serves both products
        int32_t ncB[NO];
        auto fetch2 = [&](int64_t f) {
            fetch(f);
#pragma unroll
            for (int q = 0; q < NO; ++q)
                ncB[q] = (f + stride < nfibers && q < a.N - 1) ? __ldg(fc.c[q] + f + stride) : 0;
        };
        auto rows2 = [&](int64_t f, Rows<NO, CT> &wa, bool &oka, Rows<NO, CT> &wb, bool &okb) {
            int32_t ca[NO], cb[NO];
#pragma unroll
            for (int q = 0; q < NO; ++q) {
                ca[q] = nc[q];
                cb[q] = ncB[q];
            }
            fetch2(f + 2 * stride);
            oka = fiber_rows<R, CT, NO>(a, ca, f < nfibers, sub, wa);
            okb = fiber_rows<R, CT, NO>(a, cb, f + stride < nfibers, sub, wb);
        };
        fetch2(first);
        Rows<NO, CT> wa, wb;
        bool oka, okb;
        rows2(first, wa, oka, wb, okb);
        for (int64_t f0 = warp_first; f0 < nfibers; f0 += 2 * stride) {
            const int64_t f = f0 + lane / T;
            Rows<NO, CT> na, nb;
            bool okna, oknb;
            rows2(f + 2 * stride, na, okna, nb, oknb);
            const float4 pa = product<NO, CT>(wa), pb = product<NO, CT>(wb);
            float va[J], vb[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
                va[j] = fmaf(b.x, pa.x, fmaf(b.y, pa.y, fmaf(b.z, pa.z, b.w * pa.w)));
                vb[j] = fmaf(b.x, pb.x, fmaf(b.y, pb.y, fmaf(b.z, pb.z, b.w * pb.w)));
            }
            group_reduce_scatter<T, J>(va, sub);
            group_reduce_scatter<T, J>(vb, sub);
            float qa[JL], qb[JL];
#pragma unroll
            for (int q = 0; q < JL; ++q) {
                qa[q] = va[q];
                qb[q] = vb[q];
            }
            if (oka) store_v<VT, JL>(V, f * J + sub * JL, qa);
            if (okb) store_v<VT, JL>(V, (f + stride) * J + sub * JL, qb);
            wa = na;
            wb = nb;
            oka = okna;
            okb = oknb;
        }
    } else {
        fetch(first);
        for (int64_t f0 = warp_first; f0 < nfibers; f0 += stride) {
            const int64_t f = f0 + lane / T;
            int32_t ci[NO];
#pragma unroll
            for (int q = 0; q < NO; ++q) ci[q] = nc[q];
            fetch(f + stride);
            Rows<NO, CT> w;
            const bool ok = fiber_rows<R, CT, NO>(a, ci, f < nfibers, sub, w);
            emit(f, ok, w);
        }
    }
}

// P[f] = prod_{k != n} C^(k)[i_k(f)] (R floats) for every fiber: the core
// pass's p, in the same product order as the per-nonzero walk.
template <int R, typename CT>
__global__ void __launch_bounds__(kFibThreads) k_fiber_p(PassArgs a, FiberCoords fc,
                                                         int64_t nfibers, float *P) {
    constexpr int T = R / 4;
    constexpr int NO = kMaxOrder - 1;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const int64_t stride = (int64_t)gridDim.x * (kFibThreads / T);
    const int64_t first = (int64_t)blockIdx.x * (kFibThreads / T) + threadIdx.x / T;
    int32_t nc[NO];
    auto fetch = [&](int64_t f) {
#pragma unroll
        for (int q = 0; q < NO; ++q) nc[q] = (f < nfibers && q < a.N - 1) ? __ldg(fc.c[q] + f) : 0;
    };
    fetch(first);
    for (int64_t f = first; f < nfibers; f += stride) {
        int32_t ci[NO];
#pragma unroll
        for (int q = 0; q < NO; ++q) ci[q] = nc[q];
        fetch(f + stride);
        Rows<NO, CT> w;
        if (fiber_rows<R, CT, NO>(a, ci, true, sub, w))
            *reinterpret_cast<float4 *>(P + f * R + 4 * sub) = product<NO, CT>(w);
    }
}

}  // namespace

int64_t fiber_table_capacity(int64_t nnz) {
    int64_t cap = 1024;
    while (cap < 2 * nnz) cap <<= 1;
    return cap;
}

cudaError_t launch_group_fibers(const PassArgs &a, int32_t *fid, int32_t *const *fcoord,
                                void *scratch, int64_t *nfibers, cudaStream_t st, int sms,
                                int64_t *launches) {
    const int64_t cap = fiber_table_capacity(a.nnz);
    char *p = (char *)scratch;
    unsigned long long *table = (unsigned long long *)p;
    p += cap * sizeof(unsigned long long);
    int32_t *slot_pos = (int32_t *)p;
    p += cap * sizeof(int32_t);
    int32_t *slot_fid = (int32_t *)p;
    p += cap * sizeof(int32_t);
    int32_t *rep = (int32_t *)p;
    p += cap * sizeof(int32_t);
    unsigned long long *count = (unsigned long long *)p;
    FiberKeyArgs f{};
    FiberCoordsOut out{};
    f.no = a.N - 1;
    unsigned long long s = 1;
    for (int q = f.no - 1; q >= 0; --q) {
        f.oidx[q] = a.oidx[q];
        f.odims[q] = a.odims[q];
        f.stride[q] = s;
        s *= (unsigned long long)a.odims[q];
    }
    for (int k = 0, q = 0; k < a.N; ++k)
        if (k != a.n) out.c[q++] = fcoord[k];
    const int blocks = sms * 8;
    k_fiber_clear<<<blocks, kFibThreads, 0, st>>>(table, slot_pos, cap);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_fiber_insert<<<blocks, kFibThreads, 0, st>>>(f, a.nnz, table, slot_pos, cap, fid, a.err);
    // number the fibers in the order of their first positions; the block counts
    // use the upper half of `rep` (rep needs at most nnz <= cap / 2 entries)
    const int64_t nb = (a.nnz + kScanBlock - 1) / kScanBlock;
    int32_t *counts = rep + cap / 2;
    if (nb > 0) {
        k_fiber_count<<<(int)nb, kScanBlock, 0, st>>>(fid, slot_pos, a.nnz, counts);
        k_fiber_scan<<<1, 1024, 0, st>>>(counts, nb, count);
        k_fiber_number<<<(int)nb, kScanBlock, 0, st>>>(fid, slot_pos, a.nnz, counts, slot_fid, rep);
    }
    k_fiber_remap<<<blocks, kFibThreads, 0, st>>>(fid, a.nnz, slot_fid);
    k_fiber_coords<<<blocks, kFibThreads, 0, st>>>(f, rep, count, out);
    *launches += 7;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unsigned long long h = 0;
    e = cudaMemcpyAsync(&h, count, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *nfibers = (int64_t)h;
    return e;
}

// The other modes' coordinates of every layout position from its fiber: all
// positions of fiber f share the tuple fcoord[.][f] (Eq. (12)), so
// out[q][p] = fcoord[q][fid[p]]; a position outside every fiber (fid outside
// [0, nfibers): the bad data sft_group_fibers marks -1) gets -1.  fid is read
// once and each output written once, coalesced; the fcoord reads follow fid,
// which numbers fibers by first position, so they stay local.
__global__ void k_fiber_expand(const int32_t *__restrict__ fid, int64_t nnz, int64_t nf,
                               FiberCoords in, FiberCoordsOut out, int no) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = __ldg(fid + p);
        const bool ok = 0 <= f && f < nf;
        for (int q = 0; q < no; ++q) out.c[q][p] = ok ? __ldg(in.c[q] + f) : -1;
    }
}

cudaError_t launch_fiber_expand(int N, int mode, const int32_t *fid, int64_t nnz, int64_t nfibers,
                                const int32_t *const *fcoord, int32_t *const *out_idx,
                                cudaStream_t st, int sms) {
    if (nnz <= 0) return cudaSuccess;
    FiberCoords in{};
    FiberCoordsOut out{};
    int no = 0;
    for (int k = 0; k < N; ++k)
        if (k != mode) {
            in.c[no] = fcoord[k];
            out.c[no] = out_idx[k];
            ++no;
        }
    int64_t b = (nnz + kFibThreads - 1) / kFibThreads;
    if (b > (int64_t)sms * 8) b = (int64_t)sms * 8;
    k_fiber_expand<<<(int)b, kFibThreads, 0, st>>>(fid, nnz, nfibers, in, out, no);
    return cudaGetLastError();
}

// v is stored as bfloat16 when the cached products are (SFT_BF16) and each lane
// of a T = R/4 group holds at least two entries of a row (J_n >= R/2, J_n >= 8).
bool fiber_v_bf16(const PassArgs &a, int J, int R) {
    return a.cbf16 && J >= 8 && J / (R / 4) >= 2;
}

static FiberCoords fiber_coords(const PassArgs &a, const int32_t *const *fcoord) {
    FiberCoords fc{};
    for (int k = 0, q = 0; k < a.N; ++k)
        if (k != a.n) fc.c[q++] = fcoord[k];
    return fc;
}

cudaError_t launch_factor_fibers(const PassArgs &a, const int32_t *row_ptr, int64_t W, int64_t Lseq,
                                 bool subslices, bool gram, float *maps, const int32_t *fid,
                                 const int32_t *const *fcoord,
                                 int64_t nfibers, float *V, int J, int R, const SliceStreams &ss_in,
                                 int sms, int64_t *launches) {
    SliceStreams ss = ss_in;
    const cudaStream_t st = ss.tiles;
    // 1. v of every fiber (stored as bfloat16 when the cached products are, and
    // every lane of a group holds at least two entries of a row)
    const bool vbf16 = fiber_v_bf16(a, J, R);
    if (nfibers > 0) {
        const int64_t per_block = kFibThreads / (R / 4);
        int64_t blocks = (nfibers + per_block - 1) / per_block;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        const FiberCoords fc = fiber_coords(a, fcoord);
        constexpr int NG = kMaxOrder - 1;
        using bf = __nv_bfloat16;
        if (a.cbf16 && a.N <= 3 && vbf16)
            SFT_DISPATCH_RJ(R, J, (k_fiber_v<R_, J_, bf, 2, bf><<<(int)blocks, kFibThreads, 0, st>>>(a, fc, nfibers, V)));
        else if (a.cbf16 && vbf16)
            SFT_DISPATCH_RJ(R, J, (k_fiber_v<R_, J_, bf, NG, bf><<<(int)blocks, kFibThreads, 0, st>>>(a, fc, nfibers, V)));
        else if (a.cbf16 && a.N <= 3)
            SFT_DISPATCH_RJ(R, J, (k_fiber_v<R_, J_, bf, 2, float><<<(int)blocks, kFibThreads, 0, st>>>(a, fc, nfibers, V)));
        else if (a.cbf16)
            SFT_DISPATCH_RJ(R, J, (k_fiber_v<R_, J_, bf, NG, float><<<(int)blocks, kFibThreads, 0, st>>>(a, fc, nfibers, V)));
        else if (a.N <= 3)
            SFT_DISPATCH_RJ(R, J, (k_fiber_v<R_, J_, float, 2, float><<<(int)blocks, kFibThreads, 0, st>>>(a, fc, nfibers, V)));
        else
            SFT_DISPATCH_RJ(R, J, (k_fiber_v<R_, J_, float, NG, float><<<(int)blocks, kFibThreads, 0, st>>>(a, fc, nfibers, V)));
        *launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // 2. the slice factor pass reading v from the table
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
    // blocked chains: J_n with an MMA shape, alpha = 1 - lr lambda well away from 0,
    // float32 v
    g.gram = (gram && !vbf16 && (J == 8 || J == 16 || J == 32) && a.lr * a.lam < 0.5f) ? 1 : 0;
    g.ntiles = (a.nnz + W - 1) / W;
    g.maps = maps;
    g.fid = fid;
    g.V = V;
    g.nfibers = nfibers;
    const bool with_maps = maps != nullptr;
    {
        // with the one-lane kernel (J_n <= 16) the chain list keeps only the
        // blocked chains; the lane kernel builds its own sorted work list
        cudaError_t e = launch_chain_list(g, (char *)maps + slice_chain_list_offset(g.ntiles, J),
                                          slice_lane_kernels(J), ss.chains, sms, launches);
        if (e == cudaSuccess && with_maps && !subslices)
            e = launch_piece_list(g, (char *)maps + slice_piece_list_offset(g.ntiles, J), ss.maps,
                                  sms, launches);
        if (e != cudaSuccess) return e;
    }
    factor_slices_fv(g, R, J, vbf16, with_maps, ss, sms, launches);
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

cudaError_t launch_core_fibers(const PassArgs &a, const int32_t *row_ptr, int64_t W,
                               const int32_t *fid, const int32_t *const *fcoord, int64_t nfibers,
                               float *P,
                               int J, int R, float *partials, int max_blocks, cudaStream_t st,
                               int sms, int64_t *launches, bool fill_p) {
    if (fill_p && nfibers > 0) {
        const int64_t per_block = kFibThreads / (R / 4);
        int64_t blocks = (nfibers + per_block - 1) / per_block;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        if (a.cbf16)
            SFT_DISPATCH_R(R, (k_fiber_p<R_, __nv_bfloat16><<<(int)blocks, kFibThreads, 0, st>>>(a, fiber_coords(a, fcoord), nfibers, P)));
        else
            SFT_DISPATCH_R(R, (k_fiber_p<R_, float><<<(int)blocks, kFibThreads, 0, st>>>(a, fiber_coords(a, fcoord), nfibers, P)));
        *launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    SliceArgs g{};
    g.a = a;
    g.row_ptr = row_ptr;
    g.W = W;
    g.Lseq = 0;
    g.ntiles = (a.count + W - 1) / W;
    g.maps = nullptr;
    g.fid = fid;
    g.V = P;
    g.nfibers = nfibers;
    const int nblk = core_slices_fv(g, R, J, partials, max_blocks, st, sms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 2;
    return launch_core_apply(a.B, partials, nblk, J * R, a.count, a.lr, a.lam, st);
}

}  // namespace sft
