// slices_impl.cuh -- kernels of the passes over the slice (CSF) layout; see
// k_slices_layout.cu for the layout, the description of the method and the
// launchers.  Included by the per-order translation units k_slices_f*.cu /
// k_slices_c*.cu, which instantiate them for one bound on the order.
#pragma once

#include "dispatch.cuh"
#include "sft_internal.cuh"

// Minimum resident blocks per SM requested from the register allocator: the
// slice kernels are latency bound, so occupancy is traded against a few spills
// for J <= 16; J = 32 keeps more registers.
#define SFT_DIRECT_MINB 2
#define SFT_MAPS_MINB (J >= 32 ? 1 : 2)
#ifndef SFT_CORE_MINB
#define SFT_CORE_MINB (J >= 32 ? 2 : 4)
#endif
#ifndef SFT_MAP_RING_D
#define SFT_MAP_RING_D 4
#endif
// one-lane walks: packed partial sums of a . v
#ifndef SFT_LANE_DOT_PACKED
#define SFT_LANE_DOT_PACKED 1
#endif
// prefetch distance (positions) of the one-lane walks of the sorted work list
#ifndef SFT_LANE_P
#define SFT_LANE_P 8
#endif

namespace sft {

// ============================================================================ shared pieces
// NO = number of "other" mode slots (modes != n), a compile-time bound on N-1.
// A Sample holds the raw loads of one position; nothing consumes them until
// the position's cached rows are gathered D steps later, so issuing the loads
// never waits on memory.
template <int NO>
struct Sample {
    int32_t i[NO];
    int32_t row;  // coordinate of mode n (loaded only by walks that need it)
    float x;
    bool valid;   // the position exists (a property of the range, not of the data)
};

template <int NO, bool WITH_ROW = false>
__device__ __forceinline__ void load_sample(const PassArgs &a, int64_t t, bool valid, Sample<NO> &c) {
    c.valid = valid;
#pragma unroll
    for (int q = 0; q < NO; ++q) c.i[q] = (valid && q < a.N - 1) ? __ldg(a.oidx[q] + t) : 0;
    c.row = (WITH_ROW && valid) ? __ldg(a.idx[a.n] + t) : -1;
    c.x = valid ? __ldg(a.val + t) : 0.f;
}

// The lane's raw entries of every other mode's cached row of one position.
template <int NO, typename CT>
struct Rows {
    typename CRaw<CT>::type r[NO];
};

// Checks the coordinates of a sample (they have arrived by now), reports bad
// data, and gathers the lane's float4 of every other mode's cached row.
template <int NO, int R, typename CT, bool WITH_ROW = false>
__device__ __forceinline__ void load_rows(const PassArgs &a, const Sample<NO> &c, int sub,
                                          Rows<NO, CT> &w, bool &ok, int32_t &row) {
    bool bad = false;
#pragma unroll
    for (int q = 0; q < NO; ++q)
        if (q < a.N - 1) bad |= (uint32_t)c.i[q] >= (uint32_t)a.odims[q];
    row = c.row;
    if (WITH_ROW && (uint32_t)row >= (uint32_t)a.dims[a.n]) {
        bad = true;  // samples with a bad own coordinate sit after the last slice
        row = -1;
    }
    if (c.valid && bad) atomicOr(a.err, kErrIndex);
    ok = c.valid && !bad;
#pragma unroll
    for (int q = 0; q < NO; ++q)
        w.r[q] = (ok && q < a.N - 1) ? ldC_raw_l1<CT>(a.oC[q], (int64_t)c.i[q] * R + 4 * sub,
                                                       (a.ol1 >> q) & 1u)
                                     : c_one<CT>();
}

// prod_q of the rows, widened to float as they are consumed
template <int NO, typename CT>
__device__ __forceinline__ float4 product(const Rows<NO, CT> &w) {
    float4 p = widen(w.r[0]);
#pragma unroll
    for (int q = 1; q < NO; ++q) mul4(p, widen(w.r[q]));
    return p;
}

// One entry of the element step a <- a + lr (e v - lambda a) (Eq. (10)),
// with its roundings spelled out so that every kernel that runs the step
// (lane groups or one lane per chain) produces the same bits.
__device__ __forceinline__ float row_step(float a, float e, float v, float lr, float lam) {
    return __fmaf_rn(lr, __fmaf_rn(-lam, a, __fmul_rn(e, v)), a);
}

// Prefetch depth of the slice walks: coordinates and cached rows of the next
// D positions are in flight while the current one is computed.
template <int NO, int DMAX>
struct WalkDepth {
    static constexpr int base = NO <= 2 ? 4 : (NO <= 3 ? 3 : (NO <= 7 ? 2 : 1));
    static constexpr int value = base < DMAX ? base : DMAX;
};

// Calls body(x, ok, p) for slice-ordered positions [s0, s1) in order, where p
// is the lane's 4 entries of prod_{k != n} C^(k)[i_k][:] and ok says whether
// the position's data was valid.
template <int NO, int R, typename CT, int DMAX, bool WITH_ROW, typename Body>
__device__ __forceinline__ void walk(const PassArgs &a, int64_t s0, int64_t s1, int sub,
                                     Body &&body) {
    // Two-level ring: the cached rows of positions t .. t+D-1 and the raw
    // coordinates of positions t+D .. t+2D-1 are in flight; a row gather is
    // issued D steps after its coordinates and consumed D steps after that.
    constexpr int D = WalkDepth<NO, DMAX>::value;
    Rows<NO, CT> ring[D];
    float rx[D];
    bool rok[D];
    int32_t rrow[D];
    Sample<NO> cring[D];
    {
        Sample<NO> tmp[D];
#pragma unroll
        for (int u = 0; u < D; ++u) load_sample<NO, WITH_ROW>(a, s0 + u, s0 + u < s1, tmp[u]);
#pragma unroll
        for (int u = 0; u < D; ++u)
            load_sample<NO, WITH_ROW>(a, s0 + D + u, s0 + D + u < s1, cring[u]);
#pragma unroll
        for (int u = 0; u < D; ++u) {
            load_rows<NO, R, CT, WITH_ROW>(a, tmp[u], sub, ring[u], rok[u], rrow[u]);
            rx[u] = tmp[u].x;
        }
    }
    for (int64_t t = s0; t < s1; t += D) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
            if (t + u < s1) {
                body(rrow[u], rx[u], rok[u], product<NO, CT>(ring[u]));
                // position t + u + D: its coordinates arrived D steps ago
                load_rows<NO, R, CT, WITH_ROW>(a, cring[u], sub, ring[u], rok[u], rrow[u]);
                rx[u] = cring[u].x;
                load_sample<NO, WITH_ROW>(a, t + u + 2 * D, t + u + 2 * D < s1, cring[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------- cp.async
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if constexpr (BYTES >= 16) {
#pragma unroll
        for (int q = 0; q < BYTES / 16; ++q)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16 * q),
                         "l"(static_cast<const char *>(src) + 16 * q)
                         : "memory");
    } else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES)
                     : "memory");
}

// N entries of a v row of type VT (float or bfloat16) from shared memory,
// widened to float (bfloat16 -> float is exact: the bits are the top half).
template <typename VT, int N>
__device__ __forceinline__ void ld_v_smem(const void *src, float (&out)[N]) {
    if constexpr (sizeof(VT) == 4) {
        const float *p = static_cast<const float *>(src);
        if constexpr (N % 4 == 0) {
#pragma unroll
            for (int q = 0; q < N; q += 4) {
                const float4 t = *reinterpret_cast<const float4 *>(p + q);
                out[q] = t.x; out[q + 1] = t.y; out[q + 2] = t.z; out[q + 3] = t.w;
            }
        } else if constexpr (N == 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p);
            out[0] = t.x; out[1] = t.y;
        } else {
            out[0] = p[0];
        }
    } else {
        const uint32_t *p = static_cast<const uint32_t *>(src);
        if constexpr (N % 8 == 0) {
#pragma unroll
            for (int q = 0; q < N; q += 8) {
                const uint4 t = *reinterpret_cast<const uint4 *>(p + q / 2);
                const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    out[q + 2 * k] = __uint_as_float(w[k] << 16);
                    out[q + 2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
                }
            }
        } else if constexpr (N == 4) {
            const uint2 t = *reinterpret_cast<const uint2 *>(p);
            out[0] = __uint_as_float(t.x << 16); out[1] = __uint_as_float(t.x & 0xffff0000u);
            out[2] = __uint_as_float(t.y << 16); out[3] = __uint_as_float(t.y & 0xffff0000u);
        } else {
            static_assert(N == 2, "bfloat16 v rows are read at least two entries at a time");
            out[0] = __uint_as_float(p[0] << 16); out[1] = __uint_as_float(p[0] & 0xffff0000u);
        }
    }
}

struct SliceArgs {
    PassArgs a;              // idx / val in slice order, perm unused
    const int32_t *row_ptr;  // I_n + 1 slice starts
    int64_t W;               // tile length
    int64_t Lseq;            // 0, or >= W: crossing slices up to this length run whole as
                             // one chain; longer ones are long slices
    int64_t Lhead;           // head of a long slice run as a chain before its map region
                             // (= Lseq for the exact maps; 0 for sub-slices)
    int subslices;           // long slices as concurrent sub-slices (no maps)
    // the pass's map pieces, as t * 2 + slot: full-tile pieces, then shorter
    // ones (built by k_piece_list, so that the groups of a warp run pieces of
    // the same length side by side)
    int32_t *pieces;         // [2 * ntiles] full pieces from the front, short from the back
    unsigned int *npieces;   // [0]: full pieces, [1]: short pieces
    int64_t ntiles;
    float *maps;             // [ntiles][2][J*J + J]
    // crossing slices of at most Lseq nonzeros (built per pass by k_chain_list)
    int32_t *chains;         // their rows, in no particular order (blocked chains from the back)
    unsigned int *nchains;   // [0]: chains for the lane kernels, [1]: for the blocked kernel
    int gram;                // long chains run by the blocked (Gram) kernel
    // work list of the one-lane kernel (built per pass by k_lane_count /
    // k_lane_scatter): tile interiors and chains, longest first
    uint32_t *lane_items;    // item * 2 + kind (0: interior of tile item, 1: chain of row item)
    unsigned int *lane_cnt;  // [kLaneBuckets] items per length class, [kLaneBuckets] scatter
                             // cursors, then the grab counter
    // fiber-shared v (set for the fiber variant of the factor pass)
    const int32_t *fid;      // fiber of every slice position (-1: bad data)
    const void *V;           // [nfibers][J]: v = B^(n) p of every fiber (float, or bfloat16
                             // when the context stores v that way; P of the core pass: float)
    int64_t nfibers;
};

// The lane's J/T entries of v = B^(n) p from the lane's 4 entries of p: a
// partial matrix-vector product over the lane's r, then a reduce-scatter over
// the group (lane `sub` ends with entries [sub*J/T, (sub+1)*J/T)).
template <int R, int J>
__device__ __forceinline__ void v_from_p(const float *sB, const float4 &p, int sub, unsigned m,
                                         float (&vq)[J / (R / 4)]) {
    constexpr int T = R / 4;
    float vp[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
        vp[j] = fmaf(b.x, p.x, fmaf(b.y, p.y, fmaf(b.z, p.z, b.w * p.w)));
    }
    group_reduce_scatter_m<T, J>(vp, sub, m);
#pragma unroll
    for (int q = 0; q < J / T; ++q) vq[q] = vp[q];
}

// Walk over slice positions [s0, s1) that reads v from the per-fiber table
// instead of gathering the other modes' rows: the ring holds the fiber ids of
// positions t+D..t+2D-1 and the lane's v entries of positions t..t+D-1.
template <int R, int J, int DMAX, bool WITH_ROW, typename Body>
__device__ __forceinline__ void walk_v(const SliceArgs &g, int64_t s0, int64_t s1, int sub,
                                       Body &&body) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int D = DMAX < 4 ? DMAX : 4;
    const PassArgs &a = g.a;
    struct Raw {
        int32_t f, row;
        float x;
        bool valid;
    };
    auto load_raw = [&](int64_t t, bool valid, Raw &c) {
        c.valid = valid;
        c.f = valid ? __ldg(g.fid + t) : -1;
        c.row = (WITH_ROW && valid) ? __ldg(a.idx[a.n] + t) : -1;
        c.x = valid ? __ldg(a.val + t) : 0.f;
    };
    auto load_v = [&](const Raw &c, float (&v)[JL], bool &ok, int32_t &row) {
        bool bad = (uint64_t)(int64_t)c.f >= (uint64_t)g.nfibers;
        row = c.row;
        if (WITH_ROW && (uint32_t)row >= (uint32_t)a.dims[a.n]) {
            bad = true;
            row = -1;
        }
        if (c.valid && bad) atomicOr(a.err, kErrIndex);
        ok = c.valid && !bad;
        const float *src = static_cast<const float *>(g.V) + (int64_t)(ok ? c.f : 0) * J + sub * JL;
        if constexpr (JL >= 4) {
#pragma unroll
            for (int q = 0; q < JL / 4; ++q) {
                const float4 u = ok ? ldg4(src + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
                v[4 * q] = u.x; v[4 * q + 1] = u.y; v[4 * q + 2] = u.z; v[4 * q + 3] = u.w;
            }
        } else if constexpr (JL == 2) {
            const float2 u = ok ? __ldg(reinterpret_cast<const float2 *>(src)) : make_float2(0.f, 0.f);
            v[0] = u.x; v[1] = u.y;
        } else {
            v[0] = ok ? __ldg(src) : 0.f;
        }
    };
    float ring[D][JL];
    float rx[D];
    bool rok[D];
    int32_t rrow[D];
    Raw cring[D];
    {
        Raw tmp[D];
#pragma unroll
        for (int u = 0; u < D; ++u) load_raw(s0 + u, s0 + u < s1, tmp[u]);
#pragma unroll
        for (int u = 0; u < D; ++u) load_raw(s0 + D + u, s0 + D + u < s1, cring[u]);
#pragma unroll
        for (int u = 0; u < D; ++u) {
            load_v(tmp[u], ring[u], rok[u], rrow[u]);
            rx[u] = tmp[u].x;
        }
    }
    for (int64_t t = s0; t < s1; t += D) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
            if (t + u < s1) {
                body(rrow[u], rx[u], rok[u], ring[u]);
                load_v(cring[u], ring[u], rok[u], rrow[u]);
                rx[u] = cring[u].x;
                load_raw(t + u + 2 * D, t + u + 2 * D < s1, cring[u]);
            }
        }
    }
}

// Deep shared-memory prefetch ring of the element-by-element walks over the
// fiber table (tiles and chains).  A chain step depends on the previous one
// only through the row, and every input of a position (fiber id, value, own
// coordinate, v) is known in advance, so a chain runs as fast as its
// arithmetic once the inputs are staged far enough ahead of use: P positions
// of v (one lane copies its J/T floats of each) and 2P positions of the
// scalars (lane 0 copies the fiber id, the value and, with WITH_ROW, the
// coordinate of mode n), all with cp.async, one commit group per step.  The v
// copy of position q needs its fiber id, which was copied P steps earlier.
// Per lane group: (P+1) * J floats of v slots and 3 (2P+1) words of scalar
// slots.  A slot is refilled one step after it was read (its readers have
// passed the __syncwarp at the top of the next step).
template <int J, int P>
struct DeepRing {
    static constexpr int DV = P + 1;      // v slots
    static constexpr int DS = 2 * P + 1;  // scalar slots
    // 4-byte words per lane group, rounded up to 16 bytes so that every
    // group's ring (and so every v slot) starts 16-byte aligned
    static constexpr int words = (DV * J + 3 * DS + 3) / 4 * 4;
};

constexpr int kDeepP = 16;  // prefetch distance (positions) of the deep walk

template <int R, int J, int P, bool WITH_ROW, typename VT, typename Body>
__device__ __forceinline__ void walk_v_deep(const SliceArgs &g, float *ring, int64_t s0,
                                            int64_t s1, int sub, unsigned m, Body &&body) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int DV = DeepRing<J, P>::DV;
    constexpr int DS = DeepRing<J, P>::DS;
    const PassArgs &a = g.a;
    float *vr = ring;                                             // [DV][J]
    int32_t *fr = reinterpret_cast<int32_t *>(ring + DV * J);     // [DS] fiber ids
    float *xr = ring + DV * J + DS;                               // [DS] values
    int32_t *rr = reinterpret_cast<int32_t *>(ring + DV * J + 2 * DS);  // [DS] coordinates
    const int64_t n = s1 - s0;
    auto scalars = [&](int64_t q, int slot) {  // lane 0: position q into scalar slot
        if (sub == 0 && q < n) {
            cp_async<4>(fr + slot, g.fid + s0 + q);
            cp_async<4>(xr + slot, a.val + s0 + q);
            if constexpr (WITH_ROW) cp_async<4>(rr + slot, a.idx[a.n] + s0 + q);
        }
    };
    auto vcopy = [&](int64_t q, int fslot, int vslot) {  // every lane: its part of v of q
        if (q < n) {
            const int32_t f = fr[fslot];
            if ((uint64_t)(int64_t)f < (uint64_t)g.nfibers)
                cp_async<JL * (int)sizeof(VT)>(
                    reinterpret_cast<char *>(vr + vslot * J) + sub * JL * sizeof(VT),
                    static_cast<const char *>(g.V) + ((int64_t)f * J + sub * JL) * sizeof(VT));
        }
    };
    // prologue: scalars of 0 .. P-1 (landed before anything else), then the v
    // of 0 .. P-1 and the scalars of P .. 2P-1, one commit group per position
    for (int q = 0; q < P; ++q) scalars(q, q);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp(m);
    for (int q = 0; q < P; ++q) {
        vcopy(q, q, q);
        scalars(q + P, q + P);
        cp_async_commit();
    }
    int vs = 0;       // v slot of position i
    int ss = 0;       // scalar slot of position i
    int fs = P;       // scalar slot of position i + P
    int row_pf = -1;  // last coordinate whose factor row was prefetched
    for (int64_t i = 0; i < n; ++i) {
        cp_async_wait<P - 1>();  // this lane's copies of step i - P have landed
        __syncwarp(m);           // ... and lane 0's scalars; slots of i - 1 are free
        const int32_t f = fr[ss];
        const float x = xr[ss];
        int32_t row = WITH_ROW ? rr[ss] : -1;
        float vq[JL];
        ld_v_smem<VT, JL>(reinterpret_cast<const char *>(vr + vs * J) + sub * JL * sizeof(VT), vq);
        if constexpr (WITH_ROW) {
            // a coordinate P positions ahead that starts a new slice: bring its
            // factor row towards the SM (L2) before the walk switches to it
            const int32_t rn = rr[fs];
            if (sub == 0 && i + P < n && rn != row_pf && (uint32_t)rn < (uint32_t)a.dims[a.n]) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.A + (int64_t)rn * J));
                row_pf = rn;
            }
        }
        const int prev_vs = vs == 0 ? DV - 1 : vs - 1;  // slot of i - 1 == slot of i + P
        const int prev_ss = ss == 0 ? DS - 1 : ss - 1;  // slot of i - 1 == slot of i + 2P
        vcopy(i + P, fs, prev_vs);
        scalars(i + 2 * P, prev_ss);
        cp_async_commit();
        bool bad = (uint64_t)(int64_t)f >= (uint64_t)g.nfibers;
        if (WITH_ROW && (uint32_t)row >= (uint32_t)a.dims[a.n]) {
            bad = true;
            row = -1;
        }
        if (bad && sub == 0) atomicOr(a.err, kErrIndex);
        if (bad) {
#pragma unroll
            for (int q = 0; q < JL; ++q) vq[q] = 0.f;
        }
        body(row, x, !bad, vq);
        vs = vs + 1 == DV ? 0 : vs + 1;
        ss = ss + 1 == DS ? 0 : ss + 1;
        fs = fs + 1 == DS ? 0 : fs + 1;
    }
    cp_async_wait<0>();
    __syncwarp(m);
}

// Calls step(row, x, ok, vq) for positions [s0, s1) in order, where vq is the
// lane's J/T entries of v: computed from the gathered rows (FV = false) or
// read from the per-fiber table (FV = true).
template <bool FV, int NB, int R, int J, typename CT, int DMAX, bool WITH_ROW, typename Step>
__device__ __forceinline__ void walk_steps(const SliceArgs &g, const float *sB, int64_t s0,
                                           int64_t s1, int sub, unsigned m, Step &&step,
                                           float *deep = nullptr) {
    constexpr int JL = J / (R / 4);
    if constexpr (FV) {
        if (deep)
            walk_v_deep<R, J, kDeepP, WITH_ROW, CT>(g, deep, s0, s1, sub, m, step);
        else
            walk_v<R, J, DMAX, WITH_ROW>(g, s0, s1, sub, step);
    } else {
        walk<NB, R, CT, DMAX, WITH_ROW>(g.a, s0, s1, sub,
                                        [&](int32_t row, float x, bool ok, const float4 &p) {
                                            float vq[JL];
                                            v_from_p<R, J>(sB, p, sub, m, vq);
                                            step(row, x, ok, vq);
                                        });
    }
}

// Slice [s, e) of row r is consistent with the layout and the position bounds.
__device__ __forceinline__ bool slice_ok(const SliceArgs &g, int64_t s, int64_t e) {
    return 0 <= s && s < e && e <= g.a.nnz;
}

template <int L>
__device__ __forceinline__ void store_run(float *p, const float (&r)[L]) {
    if constexpr (L >= 4) {
#pragma unroll
        for (int q = 0; q < L / 4; ++q)
            *reinterpret_cast<float4 *>(p + 4 * q) =
                make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    } else if constexpr (L == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
    } else {
        p[0] = r[0];
    }
}

// ============================================================================ factor: direct run
// Runs positions [s0, s1) of slice r element by element.  The lane holds the
// JL entries [sub*JL, (sub+1)*JL) of a_r.  The next position's coordinates and
// cached rows are loaded while the current one is computed.
template <bool FV, int NB, int R, int J, typename CT>
__device__ __forceinline__ void run_direct(const SliceArgs &g, const float *sB, int32_t r,
                                           int64_t s0, int64_t s1, int sub, unsigned m,
                                           float *deep) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    const PassArgs &a = g.a;
    float av[JL];
    float *arow = a.A + (int64_t)r * J + sub * JL;
    load_run<JL>(arow, av);
    // One-step software pipeline: v of position t does not depend on the row,
    // so it is computed while the row update of position t-1 (which needs the
    // row) is still in flight; the pending step is applied in the next call.
    float vq[JL];
    float xq = 0.f;
    bool okq = false, have = false;
    auto apply = [&]() {
        float dot = 0.f;
#pragma unroll
        for (int q = 0; q < JL; ++q) dot = fmaf(av[q], vq[q], dot);
        const float e = xq - group_sum_m<T>(dot, m);
        if (okq) {
#pragma unroll
            for (int q = 0; q < JL; ++q) av[q] = row_step(av[q], e, vq[q], a.lr, a.lam);
        }
    };
    walk_steps<FV, NB, R, J, CT, 4, false>(g, sB, s0, s1, sub, m,
                                           [&](int32_t, float x, bool ok, const float (&v)[JL]) {
        if (have) apply();
#pragma unroll
        for (int q = 0; q < JL; ++q) vq[q] = v[q];
        xq = x;
        okq = ok;
        have = true;
    }, deep);
    if (have) apply();
    store_run<JL>(arow, av);
}

// Finds the crossing slice whose first tile boundary is b (1 <= b < ntiles).
__device__ __forceinline__ bool first_boundary_slice(const SliceArgs &g, int64_t b, int32_t &r,
                                                     int64_t &s, int64_t &e) {
    const int64_t q = b * g.W;
    if (q >= g.a.nnz) return false;
    const int32_t *rowidx = g.a.idx[g.a.n];
    r = __ldg(rowidx + q);
    if ((uint32_t)r >= (uint32_t)g.a.dims[g.a.n] || __ldg(rowidx + q - 1) != r) return false;
    s = __ldg(g.row_ptr + r);
    e = __ldg(g.row_ptr + r + 1);
    if (!slice_ok(g, s, e) || s >= q || e <= q) {
        atomicOr(g.a.err, kErrIndex);
        return false;
    }
    return s / g.W + 1 == b;
}

constexpr int kSliceThreads = 256;

// Slices inside tiles.  Every lane group walks its tile's positions in order
// (the same trip count and code path for all groups of a warp), skipping the
// tile's first run if its slice started before the tile and its last run if
// its slice continues after it; the factor row is switched in place whenever
// the slice changes.
// Dynamic shared memory of the direct kernels in the fiber variant: one deep
// prefetch ring per lane group (none in the per-nonzero variant).
template <bool FV, int R, int J>
constexpr size_t direct_smem() {
    return FV ? (size_t)(kSliceThreads / (R / 4)) * DeepRing<J, kDeepP>::words * 4 : 0;
}

template <bool FV, int NB, int R, int J, typename CT>
__global__ void __launch_bounds__(kSliceThreads, SFT_DIRECT_MINB) k_slices_tiles(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    __shared__ __align__(16) float sB[J * R];
    extern __shared__ __align__(16) float dyn_ring[];
    float *deep = FV ? dyn_ring + (threadIdx.x / T) * DeepRing<J, kDeepP>::words : nullptr;
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = g.a.B[q];
    __syncthreads();
    const PassArgs &a = g.a;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const unsigned m = group_mask<T>(lane);
    const int64_t groups = (int64_t)gridDim.x * (kSliceThreads / T);
    const int32_t *rowidx = a.idx[a.n];
    const uint32_t In = (uint32_t)a.dims[a.n];
    for (int64_t t = (int64_t)blockIdx.x * (kSliceThreads / T) + threadIdx.x / T; t < g.ntiles;
         t += groups) {
        const int64_t p0 = t * g.W;
        const int64_t p1 = min(a.nnz, p0 + g.W);
        int64_t q0 = p0, q1 = p1;
        bool bad = false;
        const int32_t r0 = __ldg(rowidx + p0);
        if (p0 > 0 && (uint32_t)r0 < In && __ldg(rowidx + p0 - 1) == r0) {
            const int64_t e0 = __ldg(g.row_ptr + r0 + 1);
            if (e0 <= p0 || e0 > a.nnz) bad = true;
            else q0 = min(e0, p1);
        }
        const int32_t r1 = __ldg(rowidx + p1 - 1);
        if (p1 < a.nnz && (uint32_t)r1 < In && __ldg(rowidx + p1) == r1) {
            const int64_t s1 = __ldg(g.row_ptr + r1);
            if (s1 < 0 || s1 > p1 - 1) bad = true;
            else q1 = max(s1, q0);
        }
        if (bad) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
        if (q0 >= q1) continue;
        int32_t cur = -1;
        float av[JL];
#pragma unroll
        for (int q = 0; q < JL; ++q) av[q] = 0.f;
        walk_steps<FV, NB, R, J, CT, 4, true>(g, sB, q0, q1, sub, m,
                                              [&](int32_t row, float x, bool ok,
                                                  const float (&vq)[JL]) {
            if (row != cur) {  // the slice changes: write the finished row, read the next
                if (cur >= 0) store_run<JL>(a.A + (int64_t)cur * J + sub * JL, av);
                cur = row;
                if (cur >= 0) load_run<JL>(a.A + (int64_t)cur * J + sub * JL, av);
            }
            float dot = 0.f;
#pragma unroll
            for (int q = 0; q < JL; ++q) dot = fmaf(av[q], vq[q], dot);
            const float e = x - group_sum_m<T>(dot, m);
            if (ok) {
#pragma unroll
                for (int q = 0; q < JL; ++q) av[q] = row_step(av[q], e, vq[q], a.lr, a.lam);
            }
        }, deep);
        if (cur >= 0) store_run<JL>(a.A + (int64_t)cur * J + sub * JL, av);
    }
}

// ============================================================================ factor: one lane per chain
// In the fiber variant with J_n <= 16 an element-by-element chain (a tile's
// short slices, a crossing slice run whole, the head of a long slice) is run by
// one lane holding the whole row: its step (a . v, the residual, the row
// update) needs no shuffle, and the lane stages its own inputs with cp.async
// into a private ring (no group synchronisation).  The sum a . v is taken in
// the order the T = R/4-lane groups of the other kernels take it (sequential
// over each group lane's J/T entries, then the butterfly of the group sum), so
// the rows come out bitwise equal to the lane-group kernels and to the
// per-nonzero path.
template <int T, int J>
__device__ __forceinline__ float group_order_dot(const float (&a)[J], const float (&v)[J]) {
    constexpr int JL = J / T;
    float p[T];
    if constexpr (T % 2 == 0 && SFT_LANE_DOT_PACKED) {
        // two group lanes' partial sums at a time with packed FMAs (each half
        // an ordinary fused multiply-add, in the same order as a lane's sum)
#pragma unroll
        for (int l = 0; l < T; l += 2) {
            float2 d = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < JL; ++q)
                d = __ffma2_rn(make_float2(a[l * JL + q], a[(l + 1) * JL + q]),
                               make_float2(v[l * JL + q], v[(l + 1) * JL + q]), d);
            p[l] = d.x;
            p[l + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int l = 0; l < T; ++l) {
            float d = 0.f;
#pragma unroll
            for (int q = 0; q < JL; ++q) d = fmaf(a[l * JL + q], v[l * JL + q], d);
            p[l] = d;
        }
    }
    // butterfly: at distance w every member adds its partner's value
#pragma unroll
    for (int w = T / 2; w >= 1; w >>= 1) {
        float nxt[T];
#pragma unroll
        for (int l = 0; l < T; ++l) nxt[l] = p[l] + p[l ^ w];
#pragma unroll
        for (int l = 0; l < T; ++l) p[l] = nxt[l];
    }
    return p[0];
}

// Per-lane ring of the one-lane walks: P positions of v (J floats, plus J
// floats of the factor row at positions where a new slice starts, for the tile
// walk) and 2P positions of the scalars (fiber id, value, mode-n coordinate).
template <int J, int P, bool ROWS>
struct LaneRing {
    // a slot is refilled two positions after it was read
    static constexpr int DV = P + 2;
    static constexpr int DS = 2 * P + 2;
    static constexpr int VW = ROWS ? 2 * J : J;  // floats per v slot
    static constexpr int words = (DV * VW + 3 * DS + 3) / 4 * 4;  // 16-byte multiple
};

constexpr int kLaneThreads = 64;  // block size of the one-lane kernels

// Calls body(row, x, ok, v, newrow) for positions [s0, s1) in order: v = the
// position's v (J floats); with ROWS, row = its mode-n coordinate and newrow =
// the pass-start value of that row's factor row (valid where the coordinate
// differs from the previous position's).
template <int J, int P, bool ROWS, typename VT, typename Body>
__device__ __forceinline__ void walk_lane(const SliceArgs &g, float *ring, int64_t s0, int64_t s1,
                                          Body &&body) {
    using LR = LaneRing<J, P, ROWS>;
    constexpr int DV = LR::DV, DS = LR::DS, VW = LR::VW;
    static_assert(P % 2 == 0, "two positions per wait");
    const PassArgs &a = g.a;
    float *vr = ring;
    int32_t *fr = reinterpret_cast<int32_t *>(ring + DV * VW);
    float *xr = ring + DV * VW + DS;
    int32_t *rr = reinterpret_cast<int32_t *>(ring + DV * VW + 2 * DS);
    const int n = (int)(s1 - s0);  // a walk stays inside one pass (< 2^31 positions)
    const int32_t *fid = g.fid + s0;
    const float *val = a.val + s0;
    const int32_t *rowi = a.idx[a.n] + s0;
    const uint32_t In = (uint32_t)a.dims[a.n];
    const uint32_t nf = (uint32_t)g.nfibers;  // < 2^31 (one fiber per position at most)
    int32_t last_row = -1;  // coordinate of the last position whose v copy was issued
    auto scalars = [&](int q, int slot) {
        if (q < n) {
            cp_async<4>(fr + slot, fid + q);
            cp_async<4>(xr + slot, val + q);
            if constexpr (ROWS) cp_async<4>(rr + slot, rowi + q);
        }
    };
    auto vcopy = [&](int q, int fslot, int vslot) {
        if (q < n) {
            const int32_t f = fr[fslot];
            if ((uint32_t)f < nf)
                cp_async<J * (int)sizeof(VT)>(vr + vslot * VW,
                                              static_cast<const char *>(g.V) +
                                                  (int64_t)f * J * (int64_t)sizeof(VT));
            if constexpr (ROWS) {
                const int32_t r = rr[fslot];
                if (r != last_row && (uint32_t)r < In)
                    cp_async<J * 4>(vr + vslot * VW + J, a.A + (int64_t)r * J);
                last_row = r;
            }
        }
    };
    auto use = [&](int ss, int vs) {
        const int32_t f = fr[ss];
        const float x = xr[ss];
        int32_t row = ROWS ? rr[ss] : -1;
        float v[J];
        const float *src = vr + vs * VW;
        ld_v_smem<VT, J>(src, v);
        bool ok = (uint32_t)f < nf;
        if (ROWS && (uint32_t)row >= In) {
            ok = false;
            row = -1;
        }
        if (!ok) atomicOr(a.err, kErrIndex);
        body(row, x, ok, v, src + J);  // reads the slot before it is refilled
    };
    auto next = [](int x, int D) { return x + 1 == D ? 0 : x + 1; };
    for (int q = 0; q < P; ++q) scalars(q, q);
    cp_async_commit();
    cp_async_wait<0>();
    for (int q = 0; q < P; ++q) {
        vcopy(q, q, q);
        scalars(q + P, q + P);
        cp_async_commit();
    }
    int vs = 0, ss = 0;             // slots of position i
    int fs = P;                     // scalar slot of position i + P
    int rv = DV - 2, rs = DS - 2;   // slots of position i - 2, refilled at step i
    auto advance = [&]() {
        vs = next(vs, DV); ss = next(ss, DS); fs = next(fs, DS);
        rv = next(rv, DV); rs = next(rs, DS);
    };
    for (int i = 0; i < n; i += 2) {
        cp_async_wait<P - 2>();  // this lane's copies of steps i - P and i + 1 - P have landed
        use(ss, vs);             // position i
        vcopy(i + P, fs, rv);
        scalars(i + 2 * P, rs);
        cp_async_commit();
        advance();
        if (i + 1 < n) use(ss, vs);  // position i + 1
        vcopy(i + 1 + P, fs, rv);
        scalars(i + 1 + 2 * P, rs);
        cp_async_commit();
        advance();
    }
    cp_async_wait<0>();
}

// One element step on a whole row held by one lane: the same operations as
// the lane-group kernels (sum order of a T-lane group, then
// a += lr (e v - lambda a)).
template <int T, int J>
__device__ __forceinline__ void lane_step(const PassArgs &a, float (&av)[J], const float (&v)[J],
                                          float x, bool ok) {
    const float e = x - group_order_dot<T, J>(av, v);
    if (ok) {
        // row_step on pairs of entries with packed float32 operations (the
        // same roundings as row_step entry by entry)
        const float2 e2 = make_float2(e, e), nl = make_float2(-a.lam, -a.lam),
                     lr = make_float2(a.lr, a.lr);
#pragma unroll
        for (int q = 0; q < J; q += 2) {
            const float2 aq = make_float2(av[q], av[q + 1]);
            const float2 d = __ffma2_rn(nl, aq, __fmul2_rn(e2, make_float2(v[q], v[q + 1])));
            const float2 r = __ffma2_rn(lr, d, aq);
            av[q] = r.x;
            av[q + 1] = r.y;
        }
    }
}

// The interior [q0, q1) of tile t: its positions minus the slices that cross
// either of its boundaries (those run as chains or through maps).  False on a
// slice layout that contradicts the coordinates (the caller flags it).
__device__ __forceinline__ bool tile_inner(const SliceArgs &g, int64_t t, int64_t &q0,
                                           int64_t &q1) {
    const PassArgs &a = g.a;
    const int32_t *rowidx = a.idx[a.n];
    const uint32_t In = (uint32_t)a.dims[a.n];
    const int64_t p0 = t * g.W;
    const int64_t p1 = min(a.nnz, p0 + g.W);
    q0 = p0;
    q1 = p1;
    const int32_t r0 = __ldg(rowidx + p0);
    if (p0 > 0 && (uint32_t)r0 < In && __ldg(rowidx + p0 - 1) == r0) {
        const int64_t e0 = __ldg(g.row_ptr + r0 + 1);
        if (e0 <= p0 || e0 > a.nnz) return false;
        q0 = min(e0, p1);
    }
    const int32_t r1 = __ldg(rowidx + p1 - 1);
    if (p1 < a.nnz && (uint32_t)r1 < In && __ldg(rowidx + p1) == r1) {
        const int64_t s1 = __ldg(g.row_ptr + r1);
        if (s1 < 0 || s1 > p1 - 1) return false;
        q1 = max(s1, q0);
    }
    return true;
}

// The part of row r's slice that runs as one element-by-element chain: the
// whole slice if it crosses a tile boundary and has at most Lseq nonzeros, its
// first Lhead nonzeros if it is longer (and long slices have heads); else
// none (run = 0).  gram_min > 0: chains of at least gram_min positions belong
// to the blocked kernel and are left out too.
__device__ __forceinline__ int64_t chain_run(const int32_t *row_ptr, int32_t r, int64_t W,
                                             int64_t Lseq, int64_t Lhead, int64_t nnz,
                                             int64_t gram_min, bool *gram) {
    const int64_t s = row_ptr[r], e = row_ptr[r + 1];
    *gram = false;
    if (Lseq <= 0 || s < 0 || s >= e || e > nnz) return 0;
    if (e - s > Lseq && Lhead <= 0) return 0;
    if (s / W == (e - 1) / W) return 0;  // inside one tile: the tile's interior
    const int64_t run = e - s <= Lseq ? e - s : Lhead;
    *gram = gram_min > 0 && run >= gram_min;
    return run;
}

// Length class of a work item, longest first: 4 classes per octave (class
// 4 floor(log2 len) + the two bits after the leading one), reversed.
constexpr int kLaneBuckets = 128;
__device__ __forceinline__ int lane_bucket(int64_t len) {
    const uint64_t u = (uint64_t)len;
    const int lz = 63 - __clzll(u);
    const int q = lz >= 2 ? (int)((u >> (lz - 2)) & 3u) : (int)((u << (2 - lz)) & 3u);
    const int b = 4 * lz + q;
    return kLaneBuckets - 1 - (b < kLaneBuckets ? b : kLaneBuckets - 1);
}

// Positions [q0, q1) of a work-list item (false: nothing to run, or bad data,
// which is flagged).
__device__ __forceinline__ bool lane_item_range(const SliceArgs &g, uint32_t item, int64_t &q0,
                                                int64_t &q1) {
    const int64_t x = (int64_t)(item >> 1);
    if (item & 1u) {  // a chain: row x
        if (x >= g.a.dims[g.a.n]) return false;
        const int64_t s = __ldg(g.row_ptr + x), e = __ldg(g.row_ptr + x + 1);
        if (!slice_ok(g, s, e)) return false;
        q0 = s;
        q1 = e - s <= g.Lseq ? e : min(e, s + g.Lhead);
        return q1 > q0;
    }
    if (x >= g.ntiles) return false;
    if (!tile_inner(g, x, q0, q1)) {
        atomicOr(g.a.err, kErrIndex);
        return false;
    }
    return q1 > q0;
}

// The one-lane element-by-element walks of the pass -- tile interiors (runs of
// whole slices) and chains (crossing slices, heads of long slices) -- from the
// work list sorted by length: each warp takes the next 32 items, one per lane,
// so the lanes of a warp walk about as many positions and the longest items
// start first.  The factor row of each new slice is staged in the lane's ring
// with the position that starts it; the finished row is written back when the
// slice ends.
template <int R, int J, typename VT>
__global__ void __launch_bounds__(kLaneThreads) k_slices_lanes(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int P = SFT_LANE_P;
    using LR = LaneRing<J, P, true>;
    extern __shared__ __align__(16) float lane_ring[];
    float *ring = lane_ring + threadIdx.x * LR::words;
    const PassArgs &a = g.a;
    const int lane = threadIdx.x & 31;
    unsigned total = 0;
    for (int b = lane; b < kLaneBuckets; b += 32) total += g.lane_cnt[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    unsigned *grab = g.lane_cnt + 2 * kLaneBuckets;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(grab, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const unsigned k = base + (unsigned)lane;
        int64_t q0 = 0, q1 = 0;
        if (k >= total || !lane_item_range(g, g.lane_items[k], q0, q1)) continue;
        int32_t cur = -1;
        float av[J];
#pragma unroll
        for (int q = 0; q < J; ++q) av[q] = 0.f;
        walk_lane<J, P, true, VT>(g, ring, q0, q1,
                                  [&](int32_t row, float x, bool ok, const float (&v)[J],
                                      const float *newrow) {
            if (row != cur) {  // the slice changes: write the finished row, take the next
                if (cur >= 0) store_run<J>(a.A + (int64_t)cur * J, av);
                cur = row;
                if (cur >= 0) load_run<J>(newrow, av);
            }
            lane_step<T, J>(a, av, v, x, ok);
        });
        if (cur >= 0) store_run<J>(a.A + (int64_t)cur * J, av);
    }
}

// ============================================================================ factor: blocked chains
// A long element-by-element chain (a crossing slice run whole, or the head of
// a long slice) is run by one warp, 32 positions at a time.  With every v of a
// block known in advance, the block's steps collapse to a triangular solve:
// writing a_t for the row before the t-th position of the block, c_t for the
// number of valid positions before it, alpha = 1 - lr lambda, beta = lr/alpha,
// u_t = a_0 . v_t and G_tk = v_t . v_k, the scaled residuals
// g_t = e_t / alpha^c_t satisfy
//   g_t = x_t alpha^-c_t - u_t - beta sum_{k < t} G_tk g_k
// (Eq. (10) applied position after position, Algorithm 4's order), and the row
// after the block is a_B = alpha^c_B (a_0 + beta sum_t g_t v_t).  The Gram
// block G = V V^T (32 x 32, K = J_n) is a real contraction: it runs on the
// tensor cores (mma.sync m16n8k8, TF32 operands split into high and low
// parts, three products, float32 accumulation: about float32 accuracy); the
// solve is 32 broadcast-and-FMA steps across the warp, the sums over the block
// are float32.  The inputs are staged PB blocks ahead with cp.async (fiber
// ids 2 PB blocks ahead).  Invalid positions (bad fiber id, or past the end of
// the chain) have v = 0 and are not counted in c_t.
constexpr int kGramWarps = 4;      // chains (warps) per block
constexpr int kGramPB = 3;         // prefetch distance in 32-position blocks
constexpr int64_t kGramMin = 4096;  // shortest chain given to the blocked kernel

template <int J>
struct GramSmem {
    static constexpr int SV = J + 4;           // v row stride (conflict-free fragment loads)
    static constexpr int SG = 36;              // Gram row stride
    static constexpr int NVB = kGramPB + 1;    // v / x block slots
    static constexpr int NFB = 2 * kGramPB + 1;  // fiber-id block slots
    static constexpr int v_words = NVB * 32 * SV;
    static constexpr int x_words = NVB * 32;
    static constexpr int f_words = NFB * 32;
    static constexpr int g_words = 32 * SG;
    static constexpr int w_words = 32;
    static constexpr int words = v_words + x_words + f_words + g_words + w_words;  // per warp
    static constexpr size_t bytes = (size_t)kGramWarps * words * 4 + 2 * 33 * 4;    // + alpha tables
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// G' = V (beta V)^T for the 32 x J block V (rows = positions, stride SV), into
// sg (row-major, stride SG).  Fragments of m16n8k8 (TF32): A rows gid, gid + 8
// and columns tig, tig + 4 of a 16 x 8 tile; B rows (k) tig, tig + 4 and
// column gid; D rows gid, gid + 8 and columns 2 tig, 2 tig + 1
// (gid = lane / 4, tig = lane % 4).
template <int J>
__device__ __forceinline__ void gram_block(const float *vb, float beta, float *sg, int lane) {
    constexpr int SV = GramSmem<J>::SV, SG = GramSmem<J>::SG;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.f;
#pragma unroll
    for (int kk = 0; kk < J / 8; ++kk) {
        uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const float x[4] = {vb[(16 * mi + gid) * SV + 8 * kk + tig],
                                vb[(16 * mi + gid + 8) * SV + 8 * kk + tig],
                                vb[(16 * mi + gid) * SV + 8 * kk + tig + 4],
                                vb[(16 * mi + gid + 8) * SV + 8 * kk + tig + 4]};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ah[mi][q] = to_tf32(x[q]);
                al[mi][q] = to_tf32(x[q] - __uint_as_float(ah[mi][q]));
            }
        }
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const float y[2] = {beta * vb[(8 * ni + gid) * SV + 8 * kk + tig],
                                beta * vb[(8 * ni + gid) * SV + 8 * kk + tig + 4]};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                bh[ni][q] = to_tf32(y[q]);
                bl[ni][q] = to_tf32(y[q] - __uint_as_float(bh[ni][q]));
            }
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                mma_tf32(acc[mi][ni], al[mi], bh[ni]);
                mma_tf32(acc[mi][ni], ah[mi], bl[ni]);
                mma_tf32(acc[mi][ni], ah[mi], bh[ni]);
            }
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int r0 = 16 * mi + gid, c0 = 8 * ni + 2 * tig;
            *reinterpret_cast<float2 *>(sg + r0 * SG + c0) = make_float2(acc[mi][ni][0], acc[mi][ni][1]);
            *reinterpret_cast<float2 *>(sg + (r0 + 8) * SG + c0) =
                make_float2(acc[mi][ni][2], acc[mi][ni][3]);
        }
}

// The chains of at least kGramMin positions from the back of the chain list,
// one per warp.
template <int J>
__global__ void __launch_bounds__(kGramWarps * 32) k_slices_gram(SliceArgs g) {
    using GS = GramSmem<J>;
    constexpr int SV = GS::SV, SG = GS::SG, NVB = GS::NVB, NFB = GS::NFB, PB = kGramPB;
    extern __shared__ __align__(16) float gram_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *apow = gram_smem + kGramWarps * GS::words;  // alpha^k, k = 0..32
    float *ainv = apow + 33;                            // alpha^-k
    const PassArgs &a = g.a;
    const float alpha = 1.f - a.lr * a.lam;
    const float beta = a.lr / alpha;
    if (threadIdx.x == 0) {
        float p = 1.f, q = 1.f;
        const float ai = 1.f / alpha;
        for (int k = 0; k <= 32; ++k) {
            apow[k] = p;
            ainv[k] = q;
            p *= alpha;
            q *= ai;
        }
    }
    __syncthreads();
    float *base = gram_smem + warp * GS::words;
    float *vbuf = base;                                        // [NVB][32][SV]
    float *xbuf = vbuf + GS::v_words;                          // [NVB][32]
    int32_t *fbuf = reinterpret_cast<int32_t *>(xbuf + GS::x_words);  // [NFB][32]
    float *sg = reinterpret_cast<float *>(fbuf + GS::f_words);  // [32][SG]
    float *wv = sg + GS::g_words;                               // [32]
    const uint32_t nf = (uint32_t)g.nfibers;
    const int64_t nlong = (int64_t)g.nchains[1];
    const int64_t cap = g.ntiles;  // list capacity: long chains are stored from the back
    const int64_t warps = (int64_t)gridDim.x * kGramWarps;
    // chains fill the blocks in order (four per block), so that blocks past the
    // list exit at once and give their shared memory back to the other kernels
    for (int64_t c = (int64_t)blockIdx.x * kGramWarps + warp; c < nlong; c += warps) {
        const int32_t r = __ldg(g.chains + cap - 1 - c);
        if ((uint32_t)r >= (uint32_t)a.dims[a.n]) continue;
        const int64_t s = __ldg(g.row_ptr + r), e = __ldg(g.row_ptr + r + 1);
        if (!slice_ok(g, s, e)) continue;
        const int64_t e1 = e - s <= g.Lseq ? e : min(e, s + g.Lhead);
        const int n = (int)(e1 - s);
        const int nb = (n + 31) >> 5;
        const int32_t *fid = g.fid + s;
        const float *val = a.val + s;
        // staging of block b: fiber ids (2 PB blocks ahead), then v and x (PB ahead)
        auto fids = [&](int b) {
            const int p = 32 * b + lane;
            if (b < nb && p < n) cp_async<4>(fbuf + (b % NFB) * 32 + lane, fid + p);
        };
        auto vx = [&](int b) {
            if (b >= nb) return;
            const int p = 32 * b + lane;
            float *dst = vbuf + (b % NVB) * 32 * SV + lane * SV;
            const int32_t f = p < n ? fbuf[(b % NFB) * 32 + lane] : -1;
            if (p < n && (uint32_t)f < nf) {
                cp_async<J * 4>(dst, static_cast<const float *>(g.V) + (int64_t)f * J);
                cp_async<4>(xbuf + (b % NVB) * 32 + lane, val + p);
            } else {
#pragma unroll
                for (int q = 0; q < J; q += 4)
                    *reinterpret_cast<float4 *>(dst + q) = make_float4(0.f, 0.f, 0.f, 0.f);
                xbuf[(b % NVB) * 32 + lane] = 0.f;
            }
        };
        for (int b = 0; b < PB; ++b) fids(b);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        for (int b = 0; b < PB; ++b) {
            vx(b);
            fids(b + PB);
            cp_async_commit();
        }
        // the row, in every lane
        float av[J];
        {
            const float *arow = a.A + (int64_t)r * J;
#pragma unroll
            for (int q = 0; q < J; q += 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(arow + q);
                av[q] = t4.x; av[q + 1] = t4.y; av[q + 2] = t4.z; av[q + 3] = t4.w;
            }
        }
        float a_own = 0.f;  // av[lane % J] after the last block
        for (int b = 0; b < nb; ++b) {
            cp_async_wait<PB - 1>();  // this lane's copies of block b have landed
            __syncwarp();             // ... and every lane's; slots of block b - 1 are free
            vx(b + PB);
            fids(b + 2 * PB);
            cp_async_commit();
            const float *vb = vbuf + (b % NVB) * 32 * SV;
            const int p = 32 * b + lane;
            const int32_t f = p < n ? fbuf[(b % NFB) * 32 + lane] : -1;
            const bool valid = p < n && (uint32_t)f < nf;
            if (p < n && !valid) atomicOr(a.err, kErrIndex);
            const unsigned mask = __ballot_sync(kFull, valid);
            // u = a . v of the lane's position (the solve's right-hand side)
            float vl[J];
#pragma unroll
            for (int q = 0; q < J; q += 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(vb + lane * SV + q);
                vl[q] = t4.x; vl[q + 1] = t4.y; vl[q + 2] = t4.z; vl[q + 3] = t4.w;
            }
            float u0 = 0.f, u1 = 0.f;
#pragma unroll
            for (int q = 0; q < J; q += 2) {
                u0 = fmaf(av[q], vl[q], u0);
                u1 = fmaf(av[q + 1], vl[q + 1], u1);
            }
            const int ct = __popc(mask & ((1u << lane) - 1u));
            float rr = valid ? fmaf(xbuf[(b % NVB) * 32 + lane], ainv[ct], -(u0 + u1)) : 0.f;
            // G' = beta V V^T on the tensor cores, then the lane's row of it
            gram_block<J>(vb, beta, sg, lane);
            __syncwarp();
            float h[32];
#pragma unroll
            for (int k = 0; k < 32; k += 4) {
                const float4 t4 = *reinterpret_cast<const float4 *>(sg + lane * SG + k);
                h[k] = t4.x; h[k + 1] = t4.y; h[k + 2] = t4.z; h[k + 3] = t4.w;
            }
            // forward substitution: g_k is final in lane k when step k is reached
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float gk = __shfl_sync(kFull, rr, k);
                if (lane > k) rr = fmaf(-h[k], gk, rr);
            }
            // the row after the block: alpha^c_B (a + beta sum_t g_t v_t)
            wv[lane] = valid ? rr : 0.f;
            __syncwarp();
            float sj;
            {
                constexpr int SPL = 32 / J;  // lanes per entry j, each summing 32/SPL positions
                const int j = lane % J, part = lane / J;
                float acc = 0.f;
#pragma unroll
                for (int t = part * (32 / SPL); t < (part + 1) * (32 / SPL); ++t)
                    acc = fmaf(wv[t], vb[t * SV + j], acc);
#pragma unroll
                for (int w = J; w < 32; w <<= 1) acc += __shfl_xor_sync(kFull, acc, w);
                sj = acc;
            }
            const float ab = apow[__popc(mask)];
            float aj = av[0];  // av[lane % J], selected without a dynamic register index
#pragma unroll
            for (int q = 1; q < J; ++q)
                if ((lane % J) == q) aj = av[q];
            const float anew = ab * fmaf(beta, sj, aj);
            a_own = anew;
#pragma unroll
            for (int q = 0; q < J; ++q) av[q] = __shfl_sync(kFull, anew, q);
            __syncwarp();  // sg / wv are rewritten by the next block
        }
        cp_async_wait<0>();
        __syncwarp();
        if (lane < J && nb > 0) a.A[(int64_t)r * J + lane] = a_own;
    }
}

template <int R, int J>
constexpr bool lane_kernels() {
    return J <= 16;
}

// Crossing slices, one per lane group: a slice of at most Lseq nonzeros is
// run whole, a longer one its first Lseq nonzeros (its head); the groups take
// the slices of the pass's chain list in turn, so every group of every warp
// has work while the list lasts.
template <bool FV, int NB, int R, int J, typename CT>
__global__ void __launch_bounds__(kSliceThreads, SFT_DIRECT_MINB) k_slices_chains(SliceArgs g) {
    constexpr int T = R / 4;
    __shared__ __align__(16) float sB[J * R];
    extern __shared__ __align__(16) float dyn_ring[];
    float *deep = FV ? dyn_ring + (threadIdx.x / T) * DeepRing<J, kDeepP>::words : nullptr;
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = g.a.B[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const unsigned m = group_mask<T>(lane);
    const int64_t groups = (int64_t)gridDim.x * (kSliceThreads / T);
    const int64_t n = (int64_t)*g.nchains;
    // entry c goes to block c % gridDim.x: a short list spreads over every SM
    // instead of filling the first blocks (a chain is a dependent sequence, so
    // chains sharing an SM share its issue slots)
    for (int64_t c = (int64_t)(threadIdx.x / T) * gridDim.x + blockIdx.x; c < n; c += groups) {
        const int32_t r = __ldg(g.chains + c);
        if ((uint32_t)r >= (uint32_t)g.a.dims[g.a.n]) continue;
        const int64_t s = __ldg(g.row_ptr + r), e = __ldg(g.row_ptr + r + 1);
        if (!slice_ok(g, s, e)) continue;
        // a slice of at most Lseq nonzeros whole; a longer one its first Lseq
        // (the rest goes through maps, applied to the row this leaves)
        run_direct<FV, NB, R, J, CT>(g, sB, r, s, e - s <= g.Lseq ? e : min(e, s + g.Lhead), sub,
                                     m, deep);
    }
}

// ============================================================================ factor: long slices
// Shared-memory prefetch ring of the fiber-shared v for the map walk: D slots
// of J floats per lane group.  Lane `sub` copies its J/T floats of a row with
// cp.async P = D - 1 positions ahead of their use (one commit group per step),
// the fiber id of a position is loaded D steps before its copy is issued and
// the value D steps before it is used, so no step waits on memory.  A slot is
// refilled one step after it was read; the __syncwarp at the top of every step
// orders the group's reads of a slot before its refill.
template <int R, int J>
struct MapRing {
    static constexpr int GPB = 256 / (R / 4);  // lane groups per block of the map kernel
    static constexpr int DMAX = SFT_MAP_RING_D;
    static constexpr int D = GPB * DMAX * J * 4 <= 32768 ? DMAX : 2;
    static constexpr bool use = GPB * D * J * 4 <= 32768;  // else the register walk
};

// Calls step(v, vl, x, ok) for slice positions [s0, s1) in order: v = all J
// entries of the position's fiber v (shared memory), vl = the lane's J/T.
template <int R, int J, typename VT, typename Step>
__device__ __forceinline__ void walk_v_ring(const SliceArgs &g, float *ring, int64_t s0, int64_t s1,
                                            int sub, unsigned m, Step &&step) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int D = MapRing<R, J>::D;
    constexpr int P = D - 1;
    const PassArgs &a = g.a;
    const int64_t n = s1 - s0;
    int32_t fr[D];     // fiber ids, slot q % D holds position q until its copy is issued
    float xr[D];       // values, slot q % D holds position q until it is used
    uint32_t okm = 0;  // bit q % D: position q is valid
    auto issue = [&](int64_t q, int32_t f) {  // copy v of position q into slot q % D
        const bool valid = q < n;
        const bool good = (uint64_t)(int64_t)f < (uint64_t)g.nfibers;
        if (valid && !good) atomicOr(a.err, kErrIndex);
        const int slot = (int)(q % D);
        okm = (okm & ~(1u << slot)) | ((valid && good) ? (1u << slot) : 0u);
        if (valid && good)
            cp_async<JL * (int)sizeof(VT)>(
                reinterpret_cast<char *>(ring + slot * J) + sub * JL * sizeof(VT),
                static_cast<const char *>(g.V) + ((int64_t)f * J + sub * JL) * sizeof(VT));
        cp_async_commit();
    };
    auto ld_fid = [&](int64_t q) { return q < n ? __ldg(g.fid + s0 + q) : -1; };
    auto ld_x = [&](int64_t q) { return q < n ? __ldg(a.val + s0 + q) : 0.f; };
    // prologue: copies of positions 0 .. P-1, fiber ids of P .. P+D-1, values of 0 .. D-1
    {
        int32_t f0[P];
#pragma unroll
        for (int q = 0; q < P; ++q) f0[q] = ld_fid(q);
#pragma unroll
        for (int q = 0; q < D; ++q) fr[(P + q) % D] = ld_fid(P + q);
#pragma unroll
        for (int q = 0; q < D; ++q) xr[q] = ld_x(q);
#pragma unroll
        for (int q = 0; q < P; ++q) issue(q, f0[q]);
    }
    for (int64_t b = 0; b < n; b += D) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const int64_t i = b + u;
            if (i < n) {  // uniform over the group
                cp_async_wait<P - 1>();  // this lane's copy of position i has landed
                __syncwarp(m);           // ... and every lane's; slot (i-1) % D is free
                const int sq = (u + P) % D;  // slot of position i + P (static)
                issue(i + P, fr[sq]);
                fr[sq] = ld_fid(i + P + D);
                float v[J], vl[JL];
                const float *src = ring + u * J;  // slot i % D == u (b is a multiple of D)
                ld_v_smem<VT, J>(src, v);
                ld_v_smem<VT, JL>(reinterpret_cast<const char *>(src) + sub * JL * sizeof(VT), vl);
                const float x = xr[u];
                const bool ok = (okm >> u) & 1u;
                xr[u] = ld_x(i + D);
                step(v, vl, x, ok);
            }
        }
    }
    cp_async_wait<0>();
    __syncwarp(m);
}

// Composes the steps of positions [s0, s1) of one slice into the affine map
// (M, c) with a_after = M a_before + c.  The lane holds columns
// [sub*JC, (sub+1)*JC) of M (all J rows) and rows [sub*JL, (sub+1)*JL) of c.
// Every lane has the whole v of a step (read from the shared-memory ring in
// the fiber variant; all-gathered over the group from the walk's J/T entries
// otherwise: exact copies either way, independent of M), so the M recurrence
// (w = v^T M on the lane's columns, then the rank-1 update) needs no
// cross-lane reduction; only v . c is summed over the group.  The arithmetic
// is the same in both variants, so their results are bitwise equal.
template <bool FV, int NB, int R, int J, typename CT>
__device__ __forceinline__ void compose_map(const SliceArgs &g, const float *sB, float *ring,
                                            int64_t s0, int64_t s1, int sub, unsigned m,
                                            float *out) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;  // entries of v and rows of c per lane
    constexpr int JC = J / T;  // columns of M per lane
    const PassArgs &a = g.a;
    // The map is kept as M = alpha^n M', c = alpha^n c' (n = steps since the
    // last fold), so one step is a pure rank-1 FFMA update:
    //   M' <- M' + v (nvc w),  w = v^T M',  nvc = -lr/alpha,
    //   c' <- c' + v (nvc s) + lr x alpha^-(n+1) v,  s = v . c';
    // the factor alpha^n is folded back in at the end, and earlier only if it
    // falls below 2^-20 (large lr * lambda), so alpha^-(n+1) stays bounded.
    const float alpha = 1.f - a.lr * a.lam;
    const float ainv = 1.f / alpha;
    const float nvc = -a.lr * ainv;
    float apow = 1.f, pw = ainv;
    float M[J][JC], cv[JL];
#pragma unroll
    for (int q = 0; q < J; ++q) {
#pragma unroll
        for (int k = 0; k < JC; ++k) M[q][k] = (sub * JC + k == q) ? 1.f : 0.f;
    }
#pragma unroll
    for (int q = 0; q < JL; ++q) cv[q] = 0.f;
    auto fold = [&]() {
#pragma unroll
        for (int q = 0; q < J; ++q) {
#pragma unroll
            for (int k = 0; k < JC; ++k) M[q][k] *= apow;
        }
#pragma unroll
        for (int q = 0; q < JL; ++q) cv[q] *= apow;
        apow = 1.f;
        pw = ainv;
    };
    auto apply = [&](const float (&v)[J], const float (&vl)[JL], float x, bool ok) {
        // w = v^T M' on the lane's columns (two partial sums each); columns are
        // taken in pairs with packed float32 FMAs (each half is an ordinary
        // fused multiply-add, so the sums are the same as column by column)
        float w[JC];
        if constexpr (JC % 2 == 0) {
#pragma unroll
            for (int k = 0; k < JC; k += 2) {
                float2 e0 = make_float2(0.f, 0.f), e1 = e0;
#pragma unroll
                for (int q = 0; q < J; q += 2) {
                    e0 = __ffma2_rn(make_float2(v[q], v[q]), make_float2(M[q][k], M[q][k + 1]), e0);
                    e1 = __ffma2_rn(make_float2(v[q + 1], v[q + 1]),
                                    make_float2(M[q + 1][k], M[q + 1][k + 1]), e1);
                }
                w[k] = e0.x + e1.x;
                w[k + 1] = e0.y + e1.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < JC; ++k) {
                float e0 = 0.f, e1 = 0.f;
#pragma unroll
                for (int q = 0; q < J; q += 2) {
                    e0 = fmaf(v[q], M[q][k], e0);
                    e1 = fmaf(v[q + 1], M[q + 1][k], e1);
                }
                w[k] = e0 + e1;
            }
        }
        float sc = 0.f;
#pragma unroll
        for (int q = 0; q < JL; ++q) sc = fmaf(vl[q], cv[q], sc);
        sc = group_sum_m<T>(sc, m);
        if (ok) {
            const float xs = a.lr * x * pw;
            const float ns = nvc * sc;
#pragma unroll
            for (int k = 0; k < JC; ++k) w[k] *= nvc;
            if constexpr (JC % 2 == 0) {
#pragma unroll
                for (int q = 0; q < J; ++q) {
#pragma unroll
                    for (int k = 0; k < JC; k += 2) {
                        const float2 r = __ffma2_rn(make_float2(v[q], v[q]),
                                                    make_float2(w[k], w[k + 1]),
                                                    make_float2(M[q][k], M[q][k + 1]));
                        M[q][k] = r.x;
                        M[q][k + 1] = r.y;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < J; ++q) {
#pragma unroll
                    for (int k = 0; k < JC; ++k) M[q][k] = fmaf(v[q], w[k], M[q][k]);
                }
            }
#pragma unroll
            for (int q = 0; q < JL; ++q) cv[q] = fmaf(xs, vl[q], fmaf(vl[q], ns, cv[q]));
            apow *= alpha;
            pw *= ainv;
            if (apow < 0x1p-20f) fold();
        }
    };
    if constexpr (FV && MapRing<R, J>::use) {
        walk_v_ring<R, J, CT>(g, ring, s0, s1, sub, m, apply);
    } else {
        // One-step software pipeline: v of position t (independent of M) is
        // computed while the rank-1 update of position t-1 is applied.
        float vq[JL];
        float xq = 0.f;
        bool okq = false, have = false;
        auto gathered = [&]() {
            float v[J];
#pragma unroll
            for (int s = 0; s < T; ++s) {
#pragma unroll
                for (int q = 0; q < JL; ++q) v[s * JL + q] = __shfl_sync(m, vq[q], s, T);
            }
            apply(v, vq, xq, okq);
        };
        // prefetch depth 1: with the pipelined step a deeper ring spills at the
        // 128-register bound (measured)
        walk_steps<FV, NB, R, J, CT, 1, false>(g, sB, s0, s1, sub, m,
                                                  [&](int32_t, float x0, bool ok0,
                                                      const float (&v)[JL]) {
            if (have) gathered();
#pragma unroll
            for (int q = 0; q < JL; ++q) vq[q] = v[q];
            xq = x0;
            okq = ok0;
            have = true;
        });
        if (have) gathered();
    }
    fold();
#pragma unroll
    for (int q = 0; q < J; ++q) store_run<JC>(out + q * J + sub * JC, M[q]);
    store_run<JL>(out + J * J + sub * JL, cv);
}

// The map piece of tile t on `side` (slot).  A crossing slice longer than
// Lseq (a long slice) runs its first Lhead positions as a chain (k_slices_chains)
// and its map region [hs, e), hs = s + Lhead, through composed affine maps, one
// piece per tile the region touches:
//   slot 0: the region started before the tile: piece [p0, min(e, p1));
//   slot 1: the region starts inside the tile: piece [hs, min(e, p1)).
// With Lhead >= W only the slice holding the tile's first position p0 can have
// a piece in the tile (a slice starting inside the tile has its region start
// at least W later).  With Lhead = 0 the slot-1 piece belongs to the slice
// holding the last position p1 - 1.  Lhead is 0 or at least W (the callers
// enforce it), so the two slots never clash.
__device__ __forceinline__ bool map_piece(const SliceArgs &g, int64_t t, int side, int32_t &r,
                                          int64_t &s, int64_t &e, int64_t &hs, int64_t &q0,
                                          int64_t &q1) {
    const int64_t p0 = t * g.W;
    const int64_t p1 = min(g.a.nnz, p0 + g.W);
    const int64_t at = (side == 0 || g.Lhead > 0) ? p0 : p1 - 1;
    r = __ldg(g.a.idx[g.a.n] + at);
    if ((uint32_t)r >= (uint32_t)g.a.dims[g.a.n]) return false;
    s = __ldg(g.row_ptr + r);
    e = __ldg(g.row_ptr + r + 1);
    if (!slice_ok(g, s, e) || at < s || at >= e) {
        atomicOr(g.a.err, kErrIndex);
        return false;
    }
    if (e - s <= g.Lseq || (s >= p0 && e <= p1)) return false;  // not long / not crossing
    hs = s + g.Lhead;
    if (side == 0) {
        if (hs >= p0) return false;
        q0 = p0;
    } else {
        if (hs < p0 || hs >= p1 || hs >= e) return false;
        q0 = hs;
    }
    q1 = min(e, p1);
    return true;
}

// One group per map piece of the piece list (full pieces first).
template <bool FV, int NB, int R, int J, typename CT>
__global__ void __launch_bounds__(kSliceThreads, SFT_MAPS_MINB) k_slices_maps(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int GPB = kSliceThreads / T;
    constexpr bool RINGED = FV && MapRing<R, J>::use;
    constexpr int RING = RINGED ? GPB * MapRing<R, J>::D * J : 4;  // v prefetch rings
    __shared__ __align__(16) float sB[J * R];
    __shared__ __align__(16) float sring[RING];
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = g.a.B[q];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const unsigned m = group_mask<T>(lane);
    float *ring = RINGED ? sring + (threadIdx.x / T) * (MapRing<R, J>::D * J) : nullptr;
    const int64_t groups = (int64_t)gridDim.x * GPB;
    const int64_t nfull = (int64_t)g.npieces[0], nshort = (int64_t)g.npieces[1];
    for (int64_t k = (int64_t)blockIdx.x * GPB + threadIdx.x / T; k < nfull + nshort;
         k += groups) {
        const int32_t entry = k < nfull ? __ldg(g.pieces + k)
                                        : __ldg(g.pieces + 2 * g.ntiles - 1 - (k - nfull));
        const int64_t t = entry >> 1;
        const int side = entry & 1;
        int32_t r;
        int64_t s, e, hs, q0, q1;
        if (t >= g.ntiles || !map_piece(g, t, side, r, s, e, hs, q0, q1)) continue;
        compose_map<FV, NB, R, J, CT>(g, sB, ring, q0, q1, sub, m,
                                      g.maps + (t * 2 + side) * (int64_t)(J * J + J));
    }
}

// Long slices in the paper's B-CSF manner (Section "Tensor Storage Format":
// heavy slices cut into sub-slices that are walked concurrently), used instead
// of the exact maps when the context asks for sub-slices: every map piece
// (here a sub-slice of at most W nonzeros) is walked element by element from
// the row as it stands in memory when the walk starts, and its change to the
// row is added back with vector atomics.  Sub-slices of one row overlap in
// time, so the result depends on scheduling (Hogwild within a row); it is
// checked by the per-epoch RMSE only.
template <bool FV, int NB, int R, int J, typename CT>
__global__ void __launch_bounds__(kSliceThreads, SFT_DIRECT_MINB) k_slices_subs(SliceArgs g) {
    constexpr int T = R / 4;
    constexpr int JL = J / T;
    constexpr int GPB = kSliceThreads / T;
    __shared__ __align__(16) float sB[J * R];
    extern __shared__ __align__(16) float dyn_ring[];
    float *deep = FV ? dyn_ring + (threadIdx.x / T) * DeepRing<J, kDeepP>::words : nullptr;
    for (int q = threadIdx.x; q < J * R; q += blockDim.x) sB[q] = g.a.B[q];
    __syncthreads();
    const PassArgs &a = g.a;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const unsigned m = group_mask<T>(lane);
    const int64_t groups = (int64_t)gridDim.x * GPB;
    for (int64_t t = (int64_t)blockIdx.x * GPB + threadIdx.x / T; t < g.ntiles; t += groups) {
        for (int side = 0; side < 2; ++side) {
            int32_t r;
            int64_t s, e, hs, q0, q1;
            if (!map_piece(g, t, side, r, s, e, hs, q0, q1)) continue;
            float *arow = a.A + (int64_t)r * J + sub * JL;
            float a0[JL], av[JL];
#pragma unroll
            for (int q = 0; q < JL; ++q) av[q] = a0[q] = __ldcg(arow + q);
            walk_steps<FV, NB, R, J, CT, 4, false>(g, sB, q0, q1, sub, m,
                                                   [&](int32_t, float x, bool ok,
                                                       const float (&vq)[JL]) {
                float dot = 0.f;
#pragma unroll
                for (int q = 0; q < JL; ++q) dot = fmaf(av[q], vq[q], dot);
                const float ev = x - group_sum_m<T>(dot, m);
                if (ok) {
#pragma unroll
                    for (int q = 0; q < JL; ++q) av[q] = row_step(av[q], ev, vq[q], a.lr, a.lam);
                }
            }, deep);
            if constexpr (JL >= 4) {
#pragma unroll
                for (int q = 0; q < JL; q += 4)
                    atomicAdd(reinterpret_cast<float4 *>(arow + q),
                              make_float4(av[q] - a0[q], av[q + 1] - a0[q + 1],
                                          av[q + 2] - a0[q + 2], av[q + 3] - a0[q + 3]));
            } else {
#pragma unroll
                for (int q = 0; q < JL; ++q) atomicAdd(arow + q, av[q] - a0[q]);
            }
        }
    }
}

// ============================================================================ core
// Dynamic shared memory: B (J*R) then one G tile (J*R) per lane group.
constexpr int kCoreSliceThreads = 128;

template <bool FV, int NB, int R, int J, typename CT>
__global__ void __launch_bounds__(kCoreSliceThreads, SFT_CORE_MINB) k_slices_core(SliceArgs g,
                                                                   float *__restrict__ partials) {
    constexpr int T = R / 4;
    constexpr int GPB = kCoreSliceThreads / T;
    constexpr int JR = J * R;
    extern __shared__ __align__(16) float smem[];
    float *sB = smem;
    float *sG = smem + JR;
    for (int q = threadIdx.x; q < JR; q += blockDim.x) sB[q] = g.a.B[q];
    for (int q = threadIdx.x; q < GPB * JR; q += blockDim.x) sG[q] = 0.f;
    __syncthreads();
    const PassArgs &a = g.a;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);
    const int gid = threadIdx.x / T;
    const unsigned m = group_mask<T>(lane);
    float *myG = sG + gid * JR;
    const int64_t lo = a.base, hi = a.base + a.count;  // minibatch range of positions
    const int64_t ntiles = (a.count + g.W - 1) / g.W;
    const int64_t groups = (int64_t)gridDim.x * GPB;
    for (int64_t t = (int64_t)blockIdx.x * GPB + gid; t < ntiles; t += groups) {
        const int64_t p0 = lo + t * g.W;
        const int64_t p1 = min(hi, p0 + g.W);
        int32_t cur = -1;
        float arow[J];
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f), qv = w;
#pragma unroll
        for (int j = 0; j < J; ++j) arow[j] = 0.f;
        // G[j][4 sub .. 4 sub + 3] += a_j q for the finished run (the lane's columns)
        auto flush = [&]() {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                float4 *gp = reinterpret_cast<float4 *>(&myG[j * R + 4 * sub]);
                float4 v = *gp;
                v.x = fmaf(arow[j], qv.x, v.x);
                v.y = fmaf(arow[j], qv.y, v.y);
                v.z = fmaf(arow[j], qv.z, v.z);
                v.w = fmaf(arow[j], qv.w, v.w);
                *gp = v;
            }
        };
        auto step = [&](int32_t row, float x0, bool ok0, const float4 &p) {
            if (row != cur) {  // a new run: close the last one, read a and w = B^T a
                if (cur >= 0) flush();
                cur = row;
                qv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (cur >= 0) {
                    load_run<J>(a.A + (int64_t)cur * J, arow);
                    w = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float4 b = *reinterpret_cast<const float4 *>(&sB[j * R + 4 * sub]);
                        w.x = fmaf(arow[j], b.x, w.x);
                        w.y = fmaf(arow[j], b.y, w.y);
                        w.z = fmaf(arow[j], b.z, w.z);
                        w.w = fmaf(arow[j], b.w, w.w);
                    }
                }
            }
            const float part = fmaf(w.x, p.x, fmaf(w.y, p.y, fmaf(w.z, p.z, w.w * p.w)));
            const float xh = group_sum_m<T>(part, m);
            const float ev = ok0 ? x0 - xh : 0.f;
            qv.x = fmaf(ev, p.x, qv.x);
            qv.y = fmaf(ev, p.y, qv.y);
            qv.z = fmaf(ev, p.z, qv.z);
            qv.w = fmaf(ev, p.w, qv.w);
        };
        if constexpr (FV) {
            // p of every position read from the per-fiber table (g.V holds P here)
            walk_v<R, R, 4, true>(g, p0, p1, sub,
                                  [&](int32_t row, float x0, bool ok0, const float (&pq)[4]) {
                                      step(row, x0, ok0, make_float4(pq[0], pq[1], pq[2], pq[3]));
                                  });
        } else {
            walk<NB, R, CT, 4, true>(a, p0, p1, sub, step);
        }
        if (cur >= 0) flush();
    }
    __syncthreads();
    for (int q = threadIdx.x; q < JR; q += blockDim.x) {
        float acc = 0.f;
        for (int k = 0; k < GPB; ++k) acc += sG[k * JR + q];
        partials[(int64_t)blockIdx.x * JR + q] = acc;
    }
}

cudaError_t launch_lane_list(SliceArgs &g, void *list_ws, cudaStream_t st, int sms,
                             int64_t *launches);

template <typename K>
inline int grid_for(K kernel, int threads, size_t smem, int64_t items_per_block, int64_t items,
                    int sms) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t b = (items + items_per_block - 1) / items_per_block;
    const int64_t cap = (int64_t)sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// The three kernels touch disjoint data (chains and tiles write different
// factor rows, maps write only the map workspace), so they may run on three
// streams at once.
template <bool FV, int NB, int R, int J, typename CT>
void factor_slices_t(const SliceArgs &g, bool with_maps, const SliceStreams &ss, int sms,
                     int64_t *launches) {
    const int gpb = kSliceThreads / (R / 4);
    constexpr size_t dsm = direct_smem<FV, R, J>();
    if (g.subslices && g.ntiles > 1) {
        if (dsm > 0)
            cudaFuncSetAttribute(k_slices_subs<FV, NB, R, J, CT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        const int gs = grid_for(k_slices_subs<FV, NB, R, J, CT>, kSliceThreads, dsm, gpb,
                                g.ntiles, sms);
        k_slices_subs<FV, NB, R, J, CT><<<gs, kSliceThreads, dsm, ss.maps>>>(g);
        *launches += 1;
    }
    // maps first: it is the longest of the three, so its blocks take the SMs first
    if (with_maps && !g.subslices && g.ntiles > 1) {
        const int gm = grid_for(k_slices_maps<FV, NB, R, J, CT>, kSliceThreads, 0, gpb, g.ntiles,
                                sms);
        k_slices_maps<FV, NB, R, J, CT><<<gm, kSliceThreads, 0, ss.maps>>>(g);
        *launches += 1;
    }
    if constexpr (FV && lane_kernels<R, J>()) {
        static_assert(slice_lane_kernels(J), "host and device agree on the lane kernel");
        // blocked chains exist only if a chain may reach kGramMin positions
        const bool gram = g.gram && g.Lseq >= kGramMin;
        if (g.ntiles > 1) {
            if constexpr (J == 8 || J == 16 || J == 32) {
                if (gram) {
                    // the blocked chains first, on their own stream: they are the
                    // longest dependent sequences of the pass
                    cudaFuncSetAttribute(k_slices_gram<J>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GramSmem<J>::bytes);
                    const int gg = grid_for(k_slices_gram<J>, kGramWarps * 32, GramSmem<J>::bytes,
                                            kGramWarps, g.ntiles - 1, sms);
                    k_slices_gram<J><<<gg, kGramWarps * 32, GramSmem<J>::bytes, ss.chains>>>(g);
                    *launches += 1;
                }
            }
        }
        // tile interiors and the other chains: the sorted work list, then one
        // persistent launch of the one-lane kernel
        SliceArgs gl = g;
        if (launch_lane_list(gl, (char *)g.maps + slice_lane_list_offset(g.ntiles, J), ss.tiles, sms,
                             launches) != cudaSuccess)
            return;
        constexpr size_t lsm = (size_t)kLaneThreads * LaneRing<J, SFT_LANE_P, true>::words * 4;
        cudaFuncSetAttribute(k_slices_lanes<R, J, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lsm);
        const int gl_blocks = grid_for(k_slices_lanes<R, J, CT>, kLaneThreads, lsm, 1,
                                       (int64_t)1 << 30, sms);
        k_slices_lanes<R, J, CT><<<gl_blocks, kLaneThreads, lsm, ss.tiles>>>(gl);
        *launches += 1;
        return;
    }
    if (dsm > 0) {
        cudaFuncSetAttribute(k_slices_chains<FV, NB, R, J, CT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        cudaFuncSetAttribute(k_slices_tiles<FV, NB, R, J, CT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    }
    if (g.ntiles > 1) {
        // the list holds at most one slice per tile boundary
        const int gch = grid_for(k_slices_chains<FV, NB, R, J, CT>, kSliceThreads, dsm, gpb,
                                 g.ntiles - 1, sms);
        k_slices_chains<FV, NB, R, J, CT><<<gch, kSliceThreads, dsm, ss.chains>>>(g);
        *launches += 1;
    }
    const int gd = grid_for(k_slices_tiles<FV, NB, R, J, CT>, kSliceThreads, dsm, gpb, g.ntiles,
                            sms);
    k_slices_tiles<FV, NB, R, J, CT><<<gd, kSliceThreads, dsm, ss.tiles>>>(g);
    *launches += 1;
}

template <bool FV, int NB, int R, int J, typename CT>
int core_slices_t(const SliceArgs &g, float *partials, int max_blocks, cudaStream_t st,
                         int sms) {
    constexpr int T = R / 4;
    const size_t smem = (size_t)(1 + kCoreSliceThreads / T) * J * R * sizeof(float);
    cudaFuncSetAttribute(k_slices_core<FV, NB, R, J, CT>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nblk = grid_for(k_slices_core<FV, NB, R, J, CT>, kCoreSliceThreads, smem,
                        kCoreSliceThreads / T, g.ntiles, sms);
    if (nblk > max_blocks) nblk = max_blocks;
    k_slices_core<FV, NB, R, J, CT><<<nblk, kCoreSliceThreads, smem, st>>>(g, partials);
    return nblk;
}


// Per-order wrappers (defined in k_slices_f<NO>.cu / k_slices_c<NO>.cu).
// Per-(order bound, C type) wrappers, one translation unit each
// (k_slices_f<NO>_<ct>.cu, k_slices_c<NO>_<ct>.cu) so they compile in parallel.
#define SFT_SLICE_WRAPPERS(NO, CTN)                                                         \
    void factor_slices_no##NO##_##CTN(const SliceArgs &g, int R, int J, bool with_maps,    \
                                      const SliceStreams &ss, int sms, int64_t *launches);  \
    int core_slices_no##NO##_##CTN(const SliceArgs &g, int R, int J, float *partials,      \
                                   int max_blocks, cudaStream_t st, int sms);
SFT_SLICE_WRAPPERS(2, f32)
SFT_SLICE_WRAPPERS(3, f32)
SFT_SLICE_WRAPPERS(7, f32)
SFT_SLICE_WRAPPERS(15, f32)
SFT_SLICE_WRAPPERS(2, bf16)
SFT_SLICE_WRAPPERS(3, bf16)
SFT_SLICE_WRAPPERS(7, bf16)
SFT_SLICE_WRAPPERS(15, bf16)
#undef SFT_SLICE_WRAPPERS
cudaError_t launch_slice_combine(const SliceArgs &g, int J, int R, cudaStream_t st, int sms);
cudaError_t launch_chain_list(SliceArgs &g, void *list_ws, bool gram_only, cudaStream_t st,
                              int sms, int64_t *launches);
cudaError_t launch_piece_list(SliceArgs &g, void *list_ws, cudaStream_t st, int sms,
                              int64_t *launches);
// fiber-shared v (k_slices_fv.cu): one instantiation per (R, J)
void factor_slices_fv(const SliceArgs &g, int R, int J, bool vbf16, bool with_maps,
                      const SliceStreams &ss, int sms, int64_t *launches);
void factor_slices_fv_bf16(const SliceArgs &g, int R, int J, bool with_maps,
                           const SliceStreams &ss, int sms, int64_t *launches);
int core_slices_fv(const SliceArgs &g, int R, int J, float *partials, int max_blocks,
                   cudaStream_t st, int sms);

}  // namespace sft
