// Frontier kernels of the hot path (sm_103a): propagation sweeps (Alg. 2 as a
// push from changed vertices) and cover levels (Alg. 3).
//
// Work of a level = a "light" queue, walked as a flat edge space (sum of the
// queued vertices' degrees), plus, for propagation, a "heavy" queue of
// in-degree hubs.  The units (the heavy vertices first, then slices of
// `light_batches` 32-edge batches) go one to each warp, and, when a level has
// more units than warps, the rest are claimed from one counter.  Each queued
// vertex carries a change mask (one bit per
// simulation): only simulations that changed at the previous level are pushed
// (propagation) or expanded (cover).
//
// Light vertex, per in-edge (propagation) or out-edge (cover): lanes resolve
// 32 edges (stored edge hash, threshold, candidate range of Eq. hash_prob over
// the sorted X), then the batch's 16-simulation chunks that hold a changed
// simulation are dealt to the lanes; a chunk moves 16 register bytes with one
// 16-byte load and merges them with a byte-wise max (Eq. sketch-merge) through
// CAS on 4-byte words, only where a register improves.
//
// Heavy vertex v (weighted-cascade or uniform model, threshold below 2^26):
// every in-edge of v has the same threshold, and in-rows are sorted by edge
// hash, so the in-edges live in simulation j are inside one hash interval
// (the edge hash must agree with X_j above the threshold's top bit).  Each
// changed simulation costs two binary searches in v's row plus the live
// candidates, instead of a scan of all in-edges.
#include <cooperative_groups.h>

#include "im_launch.h"

namespace im {

constexpr int kFBlock = 256;
// per-lane statistics counters: 32 bits (a lane's counts over one phase stay
// far below 2^32) keep registers free in the frontier loops; warp sums are 64-bit
using StatT = uint32_t;
// resident blocks per SM the frontier kernels are compiled for (register cap);
// the work is latency-bound, so more resident warps hide more of it
#ifndef IM_PHASE_MIN_BLOCKS
#define IM_PHASE_MIN_BLOCKS 4
#endif
#ifndef IM_LEVEL_MIN_BLOCKS
#define IM_LEVEL_MIN_BLOCKS 4
#endif
constexpr int kPhaseMinBlocks = IM_PHASE_MIN_BLOCKS;
constexpr int kLevelMinBlocks = IM_LEVEL_MIN_BLOCKS;

__device__ __forceinline__ unsigned long long wsum(unsigned long long x) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, s);
    return x;
}

// Last queue entry whose offset is <= f (warp-wide 32-ary search).
__device__ __forceinline__ int32_t covering_entry(const QEntry* __restrict__ q, int32_t count, int64_t f) {
    int32_t lo = 0, hi = count;
    const int lane = (int)lane_id();
    while (hi - lo > 1) {
        const int32_t step = (hi - lo + 31) >> 5;
        const int64_t idx = (int64_t)lo + (int64_t)step * (lane + 1);
        const bool le = idx < hi && (int64_t)__ldcg(&q[idx].off) <= f;
        const int c = __popc(__ballot_sync(0xFFFFFFFFu, le));
        const int32_t nlo = lo + step * c;
        const int32_t nhi = (c < 32) ? (int32_t)min((int64_t)hi, (int64_t)lo + (int64_t)step * (c + 1)) : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Warp-aggregated append to a queue with a packed (count << 38 | edges) counter.
__device__ __forceinline__ void append(bool want, int32_t v, int32_t rp, int32_t deg, uint32_t aux,
                                       QEntry* __restrict__ q, unsigned long long* ctr, int32_t cap,
                                       uint32_t* err) {
    const unsigned wm = __ballot_sync(0xFFFFFFFFu, want);
    if (wm == 0u) return;
    const int lane = (int)lane_id();
    const int d = want ? deg : 0;
    int incl = d;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
        if (lane >= s) incl += y;
    }
    const int totd = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long base = 0;
    if (lane == 0)
        base = atomicAdd(ctr, ((unsigned long long)__popc(wm) << kCountShift) | (unsigned long long)totd);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (want) {
        const int32_t slot = (int32_t)(base >> kCountShift) + __popc(wm & ((1u << lane) - 1u));
        if (slot < cap) {
            QEntry e;
            e.v = v;
            e.rp = rp;
            e.off = (int32_t)(base & kEdgeMask) + (incl - d);
            e.aux = aux;
            q[slot] = e;
        } else {
            atomicOr(err, kErrQueue);
        }
    }
}

// 16 change bits -> 4 words of byte masks (0xFF where the bit is set).
__device__ __forceinline__ uint32_t bits_to_bytes(uint32_t b4) {
    return ((b4 * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// Non-zero bytes of a word -> 4 bits.
__device__ __forceinline__ uint32_t bytes_to_bits(uint32_t d) {
    const uint32_t t = (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
    return ((t >> 7) * 0x10204080u) >> 28;
}

// Where a vertex whose registers changed goes for the next propagation
// level: the heavy queue when it is an in-degree hub whose in-edges share one
// small threshold, else the light queue.
template <int KIND>
__device__ __forceinline__ bool is_heavy(int32_t deg, uint32_t thr, int32_t heavy_indeg) {
    if constexpr (KIND == kWC || KIND == kUniform)
        return deg > heavy_indeg && thr > 0u && thr < (1u << 26);
    else
        return false;
}

// 16-byte compare-and-swap (PTX atom.cas.b128, sm_90 and later): returns the
// piece found at p; it was replaced by nw when it equalled cmp.
__device__ __forceinline__ uint4 cas16(uint8_t* p, uint4 cmp, uint4 nw) {
    const unsigned long long c_lo = (unsigned long long)cmp.x | ((unsigned long long)cmp.y << 32);
    const unsigned long long c_hi = (unsigned long long)cmp.z | ((unsigned long long)cmp.w << 32);
    const unsigned long long n_lo = (unsigned long long)nw.x | ((unsigned long long)nw.y << 32);
    const unsigned long long n_hi = (unsigned long long)nw.z | ((unsigned long long)nw.w << 32);
    unsigned long long o_lo, o_hi;
    asm volatile(
        "{\n\t.reg .b128 d, b, c;\n\t"
        "mov.b128 b, {%2, %3};\n\t"
        "mov.b128 c, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], b, c;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(o_lo), "=l"(o_hi)
        : "l"(c_lo), "l"(c_hi), "l"(n_lo), "l"(n_hi), "l"(p)
        : "memory");
    return make_uint4((uint32_t)o_lo, (uint32_t)(o_lo >> 32), (uint32_t)o_hi, (uint32_t)(o_hi >> 32));
}

// Byte-wise max of cand into the 16 register bytes at trow (16-byte aligned)
// through 16-byte CAS, the merged words nw (byte_max of tg and cand) already
// known; a retry (the piece changed meanwhile) merges into what it found.
// Returns the changed registers as 16 bits.
__device__ __forceinline__ uint32_t merge_chunk_nw(uint8_t* trow, const uint32_t cand[4], uint4 tg,
                                                  const uint32_t nw[4], StatT& n_cas, uint32_t* err) {
    uint4 cur = tg;
    uint4 nv = make_uint4(nw[0], nw[1], nw[2], nw[3]);
    for (int tries = 0;; ++tries) {
        if (nv.x == cur.x && nv.y == cur.y && nv.z == cur.z && nv.w == cur.w) return 0u;
        const uint4 prev = cas16(trow, cur, nv);
        if (prev.x == cur.x && prev.y == cur.y && prev.z == cur.z && prev.w == cur.w) {
            ++n_cas;
            return bytes_to_bits(nv.x ^ cur.x) | (bytes_to_bits(nv.y ^ cur.y) << 4) |
                   (bytes_to_bits(nv.z ^ cur.z) << 8) | (bytes_to_bits(nv.w ^ cur.w) << 12);
        }
        if (tries >= kCasRetryLimit) {
            atomicOr(err, kErrCasLimit);
            return 0u;
        }
        cur = prev;
        nv = make_uint4(byte_max(cur.x, cand[0]), byte_max(cur.y, cand[1]), byte_max(cur.z, cand[2]),
                        byte_max(cur.w, cand[3]));
    }
}

__device__ __forceinline__ uint32_t merge_chunk(uint8_t* trow, const uint32_t cand[4], uint4 tg,
                                               StatT& n_cas, uint32_t* err) {
    const uint32_t nw[4] = {byte_max(tg.x, cand[0]), byte_max(tg.y, cand[1]), byte_max(tg.z, cand[2]),
                            byte_max(tg.w, cand[3])};
    return merge_chunk_nw(trow, cand, tg, nw, n_cas, err);
}

// Registers of cand (ranks, no visited bytes) above those of t: 0x80 in each
// such byte.  (t | 0x80) - c never borrows across bytes because every byte of
// c is below 0x80.
__device__ __forceinline__ uint32_t raise_hi(uint32_t t, uint32_t c) {
    return ~((t | 0x80808080u) - c) & 0x80808080u;
}

// Two bits per change word: bit 0 = a simulation of its low 16 changed, bit 1
// = of its high 16 (one bit per 16-simulation chunk).
__device__ __forceinline__ uint32_t halves_nonzero(uint32_t w) {
    return ((w & 0xFFFFu) != 0u ? 1u : 0u) | ((w >> 16) != 0u ? 2u : 0u);
}

// Chunks of vertex v with a changed simulation: bits 0..31 in lo, 32..63 in
// hi.  The change words are also kept in `keep` (words <= kKeepWords).
constexpr int kKeepWords = 8;
__device__ __forceinline__ void chunk_change_mask(const uint32_t* __restrict__ chg, int32_t v, int words,
                                                  uint32_t& lo, uint32_t& hi, uint32_t* keep) {
    lo = 0u;
    hi = 0u;
    const uint32_t* row = chg + (size_t)v * words;
    if (words >= 4) {
        for (int q = 0; q < (words >> 2); ++q) {
            const uint4 w4 = __ldcg(reinterpret_cast<const uint4*>(row) + q);
            if (words <= kKeepWords) {
                keep[4 * q] = w4.x; keep[4 * q + 1] = w4.y; keep[4 * q + 2] = w4.z; keep[4 * q + 3] = w4.w;
            }
            const uint32_t b = halves_nonzero(w4.x) | (halves_nonzero(w4.y) << 2) | (halves_nonzero(w4.z) << 4) |
                               (halves_nonzero(w4.w) << 6);
            if (q < 4) lo |= b << (8 * q);
            else hi |= b << (8 * (q - 4));
        }
    } else {
        for (int w = 0; w < words; ++w) {
            const uint32_t x = __ldcg(row + w);
            keep[w] = x;
            lo |= halves_nonzero(x) << (2 * w);
        }
    }
}

// Position of the r-th (0-based) set bit of the 64-bit mask (lo, hi).
__device__ __forceinline__ int nth_chunk(uint32_t lo, uint32_t hi, int r) {
    const int cl = __popc(lo);
    uint32_t m = r < cl ? lo : hi;
    // an edge is live in a few consecutive chunks: clearing the r lowest set
    // bits takes a handful of steps
    for (int t = r < cl ? r : r - cl; t > 0; --t) m &= m - 1u;
    return (r < cl ? 0 : 32) + __ffs((int)m) - 1;
}

// Vertex-format enqueue (warp-collective): vertex o, whose registers changed
// this level, joins the next level's queue once (enqueue stamp), hubs of the
// propagation in the heavy queue.
template <int KIND, int MODE>
__device__ __forceinline__ void vertex_enqueue(const GraphDev& g, const LevelArgs& a, bool changed, int32_t o) {
    bool want = false;
    int32_t rp = 0, deg = 0;
    uint32_t aux = 0u;
    bool heavy = false;
    if (changed) {
        // the enqueue stamp and the row words are fetched together
        const int32_t* rpp = MODE != kCover ? g.rp_in : g.rp_out;
        rp = __ldg(rpp + o);
        deg = __ldg(rpp + o + 1);
        if constexpr (MODE != kCover && KIND == kWC) aux = __ldg(g.thr_v + o);
        want = atomicExch(a.gen + o, a.gen_next) != a.gen_next;
        deg -= rp;
        if constexpr (MODE == kPush)
            heavy = is_heavy<KIND>(deg, KIND == kWC ? aux : g.thr_uniform, a.heavy_indeg);
        want = want && deg > 0;
    }
    append(want && !heavy, o, rp, deg, aux, a.ql_out, a.cl_out, a.vq_cap, a.err);
    if constexpr (MODE == kPush) append(want && heavy, o, rp, deg, aux, a.qh_out, a.ch_out, a.vq_cap, a.err);
}

// Enqueue in two steps around the register update, so that its round trips
// overlap the update's: `issue` starts the loads and atomics for target o
// whose 16 registers of chunk c the item raises (imp, predicted from the
// target piece it loaded: a register another thread raises first changed this
// level all the same), `finish` appends (warp-collective).
struct EnqueueState {
    int32_t rp = 0, deg = 0;
    uint32_t aux = 0u, old = 0u, os = 0u, oe = 0u;
    bool fresh = false;
};

template <int KIND, int MODE>
__device__ __forceinline__ EnqueueState vertex_enqueue_issue(const GraphDev& g, const LevelArgs& a, int32_t o,
                                                             uint32_t c, uint32_t imp) {
    EnqueueState q;
    if (imp) {
        // a cover reads the word's previous bits (newly_visited counts from them)
        if constexpr (MODE == kCover)
            q.old = atomicOr(a.chg_next + (size_t)o * a.words + (c >> 1), imp << ((c & 1u) * 16u));
        else
            red_or(a.chg_next + (size_t)o * a.words + (c >> 1), imp << ((c & 1u) * 16u));
        const int32_t* rpp = MODE != kCover ? g.rp_in : g.rp_out;
        q.rp = __ldg(rpp + o);
        q.deg = __ldg(rpp + o + 1);
        if constexpr (MODE != kCover && KIND == kWC) q.aux = __ldg(g.thr_v + o);
        q.fresh = atomicExch(a.gen + o, a.gen_next) != a.gen_next;
    }
    return q;
}

template <int KIND, int MODE>
__device__ __forceinline__ void vertex_enqueue_finish(const GraphDev& g, const LevelArgs& a, bool changed,
                                                      int32_t o, const EnqueueState& q) {
    const int32_t deg = q.deg - q.rp;
    bool heavy = false;
    if constexpr (MODE == kPush)
        heavy = changed && is_heavy<KIND>(deg, KIND == kWC ? q.aux : g.thr_uniform, a.heavy_indeg);
    const bool want = changed && q.fresh && deg > 0;
    append(want && !heavy, o, q.rp, deg, q.aux, a.ql_out, a.cl_out, a.vq_cap, a.err);
    if constexpr (MODE == kPush) append(want && heavy, o, q.rp, deg, q.aux, a.qh_out, a.ch_out, a.vq_cap, a.err);
}

// Affected-set search (incremental rebuild): marks the simulations of
// chunk c in which target o becomes affected (cand: 0xFF bytes where o is
// reached along a live edge and its register is not visited); returns the
// 16 bits that were not marked before.
__device__ __forceinline__ uint32_t mark_affected(const LevelArgs& a, const uint32_t cand[4], int32_t o, uint32_t c,
                                                  StatT& st_new) {
    uint32_t b16 = 0u;
#pragma unroll
    for (int w = 0; w < 4; ++w) b16 |= bytes_to_bits(cand[w]) << (4 * w);
    if (!b16) return 0u;
    const uint32_t sh = (c & 1u) * 16u;
    const uint32_t old = atomicOr(a.aff + (size_t)o * a.words + (c >> 1), b16 << sh);
    const uint32_t fresh = b16 & ~(old >> sh) & 0xFFFFu;
    st_new += (unsigned)__popc(fresh);
    if (old == 0u && a.awl) {
        // the word's first bit: list it (one append for the lanes here together)
        cooperative_groups::coalesced_group grp = cooperative_groups::coalesced_threads();
        unsigned int base = 0u;
        if (grp.thread_rank() == 0) base = atomicAdd(a.awl_count, grp.size());
        base = grp.shfl(base, 0);
        a.awl[base + grp.thread_rank()] = (uint32_t)o * (uint32_t)a.words + (c >> 1);
    }
    return fresh;
}

// Cover: registers newly visited since the last build (the next incremental
// rebuild starts from them).
__device__ __forceinline__ void note_newly_visited(const LevelArgs& a, int32_t o, uint32_t c, uint32_t nbits) {
    if (a.nv && nbits) red_or(a.nv + (size_t)o * a.words + (c >> 1), nbits << ((c & 1u) * 16u));
}

// Forward declarations (bucket mode, below).
__device__ __forceinline__ uint32_t bucket_start(const uint32_t* __restrict__ end, int64_t b);
__device__ __forceinline__ void bucket_append(bool want, uint32_t b, uint32_t start, uint32_t len,
                                              QEntry* __restrict__ q, unsigned long long* ctr,
                                              unsigned long long* overflow, int32_t cap, bool guard);

// Bucket-format enqueue (warp-collective): the change bits nbits (16, of
// chunk c) of vertex o are set; the first change of that chunk this level
// (the returned bits tell) queues the bucket (o, c) unless it is empty (an
// empty bucket's bits are never read).
__device__ __forceinline__ void bucket_enqueue(const LevelArgs& a, bool changed, int32_t o, uint32_t c,
                                               uint32_t nbits) {
    bool want = false;
    uint32_t ob = 0u, os = 0u, oe = 0u;
    if (changed) {
        const uint32_t sh = (c & 1u) * 16u;
        ob = (uint32_t)o * (uint32_t)a.chunks + c;
        oe = __ldcg(a.bk_end + ob);
        os = bucket_start(a.bk_end, ob);
        const uint32_t old = atomicOr(a.chg_next + (size_t)o * a.words + (c >> 1), nbits << sh);
        want = ((old >> sh) & 0xFFFFu) == 0u && oe > os;
    }
    bucket_append(want, ob, os, oe - os, a.ql_out, a.cl_out, a.ch_out, a.bq_cap, a.bq_guard != 0);
}

__device__ __forceinline__ EnqueueState bucket_enqueue_issue(const LevelArgs& a, int32_t o, uint32_t c,
                                                             uint32_t imp) {
    EnqueueState q;
    if (imp) {
        const uint32_t ob = (uint32_t)o * (uint32_t)a.chunks + c;
        q.oe = __ldcg(a.bk_end + ob);
        q.os = bucket_start(a.bk_end, ob);
        q.old = atomicOr(a.chg_next + (size_t)o * a.words + (c >> 1), imp << ((c & 1u) * 16u));
    }
    return q;
}

__device__ __forceinline__ void bucket_enqueue_finish(const LevelArgs& a, bool changed, int32_t o, uint32_t c,
                                                      const EnqueueState& q) {
    const uint32_t sh = (c & 1u) * 16u;
    const bool want = changed && ((q.old >> sh) & 0xFFFFu) == 0u && q.oe > q.os;
    bucket_append(want, (uint32_t)o * (uint32_t)a.chunks + c, q.os, q.oe - q.os, a.ql_out, a.cl_out, a.ch_out,
                  a.bq_cap, a.bq_guard != 0);
}

// Dense-format output (a propagation level that walks every vertex, while the
// frontier stays large): a raised register only sets its change bits (no
// reply needed), and the lane counts its raised items; no queue entry, no
// enqueue stamp, no row words.  Each warp adds its count to the next level's
// counter once, at the end of the level (dense_count_flush).  The next level
// walks every vertex again and reads the change bits.
template <int MODE>
__device__ __forceinline__ uint32_t dense_enqueue_issue(const LevelArgs& a, int32_t o, uint32_t c, uint32_t imp) {
    if (!imp) return 0u;
    uint32_t* w = a.chg_next + (size_t)o * a.words + (c >> 1);
    if constexpr (MODE == kCover) return atomicOr(w, imp << ((c & 1u) * 16u));
    red_or(w, imp << ((c & 1u) * 16u));
    return 0u;
}

// The registers a cover item visits first: a register becomes visited at
// exactly one level (a later level's target load sees the mark), every item
// that visits it at that level sets its change bit, and the one whose
// atomicOr found the bit clear counts it (old: the change word before).
__device__ __forceinline__ void newly_visited(const LevelArgs& a, int32_t o, uint32_t c, uint32_t imp, uint32_t old,
                                              StatT& st_new) {
    const uint32_t fresh = imp & ~(old >> ((c & 1u) * 16u)) & 0xFFFFu;
    if (!fresh) return;
    const unsigned k = (unsigned)__popc(fresh);
    st_new += k;
    if (a.gcount) red_add(a.gcount + __ldg(a.gid + o), (unsigned long long)k);
}

__device__ __forceinline__ void dense_count_flush(const LevelArgs& a, StatT n) {
    unsigned long long s = n;
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, k);
    if (s && lane_id() == 0) atomicAdd(a.cl_out, s << kCountShift);
}

// ---------------------------------------------------------------------------
// Light units: a slice of 32-edge batches of the flat edge space.
// ---------------------------------------------------------------------------
template <int KIND, int MODE>
__device__ __forceinline__ void light_slice(const GraphDev& g, const LevelArgs& a, const QEntry* __restrict__ qlin,
                                            const uint32_t* sX,
                                            const uint16_t* sTab, int64_t b0, int64_t b1, int32_t nl,
                                            int64_t El, StatT& st_chunks,
                                            StatT& st_cas, StatT& st_new,
                                            StatT& st_batches, StatT& st_dealt,
                                            StatT& st_live, bool skip_heavy, uint32_t (*sKeep)[kKeepWords], bool out_b,
                                            bool out_d, StatT* st_chg, StatT& st_draised, bool all_sims) {
    const int lane = (int)lane_id();
    const int J = a.J, words = a.words;
    const int64_t fend = min(El, b1 << 5);
    int64_t f0 = b0 << 5;
    int32_t qi = f0 == 0 ? 0 : covering_entry(qlin, nl, f0);
    // queue window of the first batch; later windows are prefetched one batch ahead
    int4 raw = make_int4(0, 0, 0x7FFFFFFF, 0);
    if (qi + lane < nl) raw = __ldcg(reinterpret_cast<const int4*>(qlin) + qi + lane);
    for (; f0 < fend; f0 += 32) {
        const int32_t wi = qi + lane;
        const bool wvalid = wi < nl;
        const int64_t rel = (int64_t)raw.z - f0;
        const int c0 = __popc(__ballot_sync(0xFFFFFFFFu, wvalid && rel <= 0));
        const unsigned starts =
            __reduce_or_sync(0xFFFFFFFFu, (wvalid && rel >= 1 && rel <= 31) ? (1u << rel) : 0u);
        const int myw = c0 - 1 + __popc(starts & ((2u << lane) - 1u));
        const int32_t qv = chk(__shfl_sync(0xFFFFFFFFu, raw.x, myw), g.n, a.err);
        const int32_t qrp = __shfl_sync(0xFFFFFFFFu, raw.y, myw);
        const int32_t qoff = __shfl_sync(0xFFFFFFFFu, raw.z, myw);
        const uint32_t qaux = (uint32_t)__shfl_sync(0xFFFFFFFFu, raw.w, myw);
        // the window of the next batch: the entry covering f0 + 32
        const int n32 = __popc(__ballot_sync(0xFFFFFFFFu, wvalid && rel <= 32));
        int32_t qn = qi + n32 - 1;
        if (n32 == 32 && qi + 32 < nl) {
            if ((int64_t)__ldcg(&qlin[qi + 32].off) <= f0 + 32) qn = qi + 32;
        }
        int4 rawn = make_int4(0, 0, 0x7FFFFFFF, 0);
        if (f0 + 32 < fend && qn + lane < nl) rawn = __ldcg(reinterpret_cast<const int4*>(qlin) + qn + lane);
        // this lane's edge: live chunk mask, source and hash are fetched at
        // once (one round trip with the change words below)
        const int64_t f = f0 + lane;
        int64_t e = (int64_t)qrp + (f - qoff);
        int32_t o = 0;
        uint32_t h = 0, thr = 0;
        uint32_t m_lo = 0u, m_hi = 0u;
        if (f < fend) {
            e = chk(e, g.m, a.err);
            m_lo = __ldg(a.lcm_lo + e);
            if (a.lcm_hi) m_hi = __ldg(a.lcm_hi + e);
            if constexpr (MODE != kCover) {
                o = chk(__ldg(g.src_in + e), g.n, a.err);
                h = __ldg(g.h_in + e);
                if constexpr (KIND == kExplicit) thr = __ldg(g.thr_in + e);
            } else {
                o = chk(__ldg(g.col_out + e), g.n, a.err);
                h = __ldg(g.h_out + e);
                if constexpr (KIND == kExplicit || KIND == kWC) thr = edge_threshold<KIND, false>(g, 0u, 0u, e, 0u);
            }
        }
        // chunks with a changed simulation of each queue entry this batch uses
        uint32_t cm_lo = 0xFFFFFFFFu, cm_hi = 0xFFFFFFFFu;
        const bool used = wvalid && rel <= 31 && lane >= c0 - 1;

        __syncwarp();
        if (!a.all_changed && used && (!all_sims || st_chg))
            chunk_change_mask(a.chg_cur, chk(raw.x, g.n, a.err), words, cm_lo, cm_hi, sKeep[lane]);
        // a walk over every vertex counts the changed ones (the previous
        // level's output had no queue): once each, where its row starts
        if (st_chg && used && rel >= 0 && (cm_lo | cm_hi) != 0u) ++*st_chg;
        // all_sims: the walk pushes every live simulation of every vertex,
        // changed or not (what a source raised earlier in this same walk then
        // moves on at once)
        if (all_sims) { cm_lo = 0xFFFFFFFFu; cm_hi = 0xFFFFFFFFu; }
        if constexpr (MODE == kPush) {
            // dense walk: the heavy queue pushes the hubs
            if (skip_heavy && used) {
                const int32_t deg = __ldg(g.rp_in + raw.x + 1) - raw.y;
                if (is_heavy<KIND>(deg, KIND == kWC ? (uint32_t)raw.w : g.thr_uniform, a.heavy_indeg)) {
                    cm_lo = 0u;
                    cm_hi = 0u;
                }
            }
        }
        __syncwarp();
        m_lo &= __shfl_sync(0xFFFFFFFFu, cm_lo, myw);
        m_hi &= __shfl_sync(0xFFFFFFFFu, cm_hi, myw);
        const int nch = __popc(m_lo) + __popc(m_hi);
        if (nch) {
            if constexpr (MODE != kCover) {
                if constexpr (KIND != kExplicit) thr = edge_threshold<KIND, true>(g, (uint32_t)o, (uint32_t)qv, e, qaux);
            } else {
                if constexpr (KIND != kExplicit && KIND != kWC)
                    thr = edge_threshold<KIND, false>(g, (uint32_t)qv, (uint32_t)o, e, 0u);
            }
        }
        if (nch) ++st_live;
        int incl = nch;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
            if (lane >= s) incl += y;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const int excl = incl - nch;
        if (lane == 0) { ++st_batches; st_dealt += (unsigned)total; }
        for (int base = 0; base < total; base += 32) {
            const int k = base + lane;
            int i = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int ic = __shfl_sync(0xFFFFFFFFu, incl, i + s - 1);
                if (ic <= k) i += s;
            }
            if (i > 31) i = 31;
            const int ex_i = __shfl_sync(0xFFFFFFFFu, excl, i);
            const int w_i = __shfl_sync(0xFFFFFFFFu, myw, i);
            const uint32_t ml_i = __shfl_sync(0xFFFFFFFFu, m_lo, i);
            const uint32_t mh_i = __shfl_sync(0xFFFFFFFFu, m_hi, i);
            const int32_t o_i = __shfl_sync(0xFFFFFFFFu, o, i);
            const int32_t q_i = __shfl_sync(0xFFFFFFFFu, qv, i);
            const uint32_t h_i = __shfl_sync(0xFFFFFFFFu, h, i);
            const uint32_t t_i = __shfl_sync(0xFFFFFFFFu, thr, i);
            uint32_t nbits = 0u, imp = 0u, any = 0u;
            int chunk = 0;
            EnqueueState eq;
            if (k < total) {
                chunk = chk(nth_chunk(ml_i, mh_i, k - ex_i), a.chunks, a.err);
                uint32_t chb = 0xFFFFu;
                if (!a.all_changed && !all_sims) {
                    const uint32_t cw = words <= kKeepWords ? sKeep[w_i][chunk >> 1]
                                                            : __ldcg(a.chg_cur + (size_t)q_i * words + (chunk >> 1));
                    chb = (cw >> ((chunk & 1) * 16)) & 0xFFFFu;
                }
                if (chb) {
                    const uint4* xs = reinterpret_cast<const uint4*>(sX + chunk * 16);
                    const uint8_t* srow = a.M + (size_t)q_i * J + chunk * 16;
                    uint8_t* trow = a.M + (size_t)o_i * J + chunk * 16;
                    const uint4 src = ld_cg16(srow);
                    const uint4 tg = ld_cg16(trow);
                    const uint32_t sw[4] = {src.x, src.y, src.z, src.w};
                    const uint32_t tw[4] = {tg.x, tg.y, tg.z, tg.w};
                    uint32_t cand[4], nwv[4];
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const uint32_t L = live4(xs[w], h_i, t_i) & bits_to_bytes((chb >> (4 * w)) & 0xFu);
                        if constexpr (MODE == kPush) cand[w] = sw[w] & L & ~visited_bytes(sw[w]);
                        else if constexpr (MODE == kCover) cand[w] = L & visited_bytes(sw[w]) & ~visited_bytes(tw[w]);
                        else cand[w] = L & ~visited_bytes(tw[w]);
                        any |= cand[w];
                        // registers this item raises, as the loaded target piece shows
                        if constexpr (MODE == kPush) {
                            const uint32_t gt = raise_hi(tw[w], cand[w]) >> 7;
                            imp |= ((gt * 0x10204080u) >> 28) << (4 * w);
                            const uint32_t m = gt * 0xFFu;
                            nwv[w] = (tw[w] & ~m) | (cand[w] & m);
                        } else if constexpr (MODE == kCover) {
                            imp |= bytes_to_bits(cand[w]) << (4 * w);
                        }
                    }
                    if constexpr (MODE == kAffect) imp = mark_affected(a, cand, o_i, (uint32_t)chunk, st_new);
                    // the enqueue's loads and atomics go out before the register update
                    if (out_d) eq.old = dense_enqueue_issue<MODE>(a, o_i, (uint32_t)chunk, imp);
                    else eq = out_b ? bucket_enqueue_issue(a, o_i, (uint32_t)chunk, imp)
                                    : vertex_enqueue_issue<KIND, MODE>(g, a, o_i, (uint32_t)chunk, imp);
                    if (MODE != kAffect && any) {
                        ++st_chunks;
                        if constexpr (MODE == kPush) {
                            nbits = merge_chunk_nw(trow, cand, tg, nwv, st_cas, a.err);
                        } else {
                            // the visited marks go out without a reply; the
                            // change word's previous bits count the new ones
                            red_or_piece(trow, cand);
                            newly_visited(a, o_i, (uint32_t)chunk, imp, eq.old, st_new);
                            note_newly_visited(a, o_i, (uint32_t)chunk, imp);
                        }
                    }
                }
            }
            (void)nbits;
            // enqueue what changed: the vertex, or its chunk's bucket
            if (out_d) st_draised += imp != 0u ? 1u : 0u;
            else if (out_b) bucket_enqueue_finish(a, imp != 0u, o_i, (uint32_t)chunk, eq);
            else vertex_enqueue_finish<KIND, MODE>(g, a, imp != 0u, o_i, eq);
        }
        qi = qn;
        raw = rawn;
    }
}

// First index in [lo, hi) with h[index] >= key.  h is sorted ascending and
// holds edge hashes, spread uniformly over [0, 2^31): a few interpolation
// probes (each keeping every value of [lo, hi) inside [vlo, vhi]) shrink the
// range to a handful of entries, then bisection finishes (and bounds the
// worst case).
__device__ __forceinline__ int32_t lower_bound_h(const uint32_t* __restrict__ h, int32_t lo, int32_t hi,
                                                 uint32_t key) {
    uint32_t vlo = 0u, vhi = 0x7FFFFFFFu;
    for (int it = 0; it < 4 && hi - lo > 8; ++it) {
        const uint64_t span = (uint64_t)(vhi - vlo) + 1u;
        int64_t g = lo + (int64_t)(((uint64_t)(key - vlo) * (uint64_t)(hi - lo)) / span);
        if (g >= hi) g = hi - 1;
        const uint32_t x = __ldg(h + g);
        if (x < key) { lo = (int32_t)g + 1; vlo = x; }
        else { hi = (int32_t)g; vhi = x; }
    }
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(h + mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Heavy unit: one in-degree hub, its changed simulations dealt to the lanes.
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void heavy_vertex(const GraphDev& g, const LevelArgs& a, const uint32_t* sX,
                                             QEntry ent, StatT& st_chunks,
                                             StatT& st_cas, bool out_b) {
    const int lane = (int)lane_id();
    const int J = a.J, words = a.words;
    const int32_t v = chk(ent.v, g.n, a.err);
    const int32_t rb = ent.rp;
    const int32_t re = __ldg(g.rp_in + v + 1);
    const uint32_t thr = KIND == kWC ? ent.aux : g.thr_uniform;
    const int t1 = 32 - __clz((int)thr);  // t + 1, thr in (0, 2^26)
    // changed simulations of v whose source register can still raise a target
    uint32_t cw = 0u;
    if (lane < words) {
        cw = a.all_changed ? 0xFFFFFFFFu : __ldcg(a.chg_cur + (size_t)v * words + lane);
        if (cw) {
            const uint8_t* srow = a.M + (size_t)v * J + lane * 32;
            const uint4 s0 = ld_cg16(srow), s1 = ld_cg16(srow + 16);
            const uint32_t sw[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
            uint32_t useful = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                // a register is useful when it is neither visited nor 0
                const uint32_t nz = bytes_to_bits(sw[q]);
                const uint32_t vis = bytes_to_bits(visited_bytes(sw[q]));
                useful |= (nz & ~vis) << (4 * q);
            }
            cw &= useful;
        }
    }
    const int cnt = __popc(cw);
    int incl = cnt;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
        if (lane >= s) incl += y;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const int excl = incl - cnt;
    for (int base = 0; base < total; base += 32) {
        const int k = base + lane;
        int i = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            const int ic = __shfl_sync(0xFFFFFFFFu, incl, i + s - 1);
            if (ic <= k) i += s;
        }
        if (i > 31) i = 31;
        const uint32_t word = __shfl_sync(0xFFFFFFFFu, cw, i);
        const int ex_i = __shfl_sync(0xFFFFFFFFu, excl, i);
        int32_t a0 = 0, a1 = 0;
        int j = 0;
        uint32_t val = 0u, Xj = 0u;
        if (k < total) {
            const int bit = (int)__fns(word, 0u, k - ex_i + 1);
            j = i * 32 + bit;
            val = a.M[(size_t)v * J + j];
            Xj = sX[j];
            const uint32_t lo_key = (Xj >> t1) << t1;
            const uint32_t hi_key = lo_key + (1u << t1);
            a0 = lower_bound_h(g.h_in, rb, re, lo_key);
            a1 = lower_bound_h(g.h_in, a0, re, hi_key);
            ++st_chunks;
        }
        int ncand = a1 - a0;
        int maxc = ncand;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) maxc = max(maxc, __shfl_xor_sync(0xFFFFFFFFu, maxc, s));
        for (int c = 0; c < maxc; ++c) {
            bool changed = false;
            int32_t u = 0;
            if (c < ncand) {
                const int32_t e = chk(a0 + c, g.m, a.err);
                const uint32_t h = __ldg(g.h_in + e);
                if ((Xj ^ h) < thr) {
                    u = chk(__ldg(g.src_in + e), g.n, a.err);
                    unsigned int* addr = reinterpret_cast<unsigned int*>(a.M + (((size_t)u * J + j) & ~(size_t)3));
                    const uint32_t b = val << (8 * (j & 3));
                    uint32_t cur = __ldcg(addr);
                    uint32_t nw = byte_max(cur, b);
                    int tries = 0;
                    while (nw != cur) {
                        const uint32_t prev = atomicCAS(addr, cur, nw);
                        if (prev == cur) { changed = true; ++st_cas; break; }
                        cur = prev;
                        nw = byte_max(cur, b);
                        if (++tries > kCasRetryLimit) { atomicOr(a.err, kErrCasLimit); break; }
                    }
                    if (changed && !out_b) red_or(a.chg_next + (size_t)u * words + (j >> 5), 1u << (j & 31));
                }
            }
            if (out_b) bucket_enqueue(a, changed, u, (uint32_t)(j >> 4), 1u << (j & 15));
            else vertex_enqueue<KIND, kPush>(g, a, changed, u);
        }
    }
}

// ---------------------------------------------------------------------------
// Bucket mode.  A level's work is a set of buckets (v, chunk c) whose 16
// change bits are set; a bucket's entries are exactly the edges of v live in
// a simulation of c, with their live masks, so no edge is visited for a chunk
// that did not change and no live test runs.  Flat positions walk the queue's
// buckets (offsets from the packed counter), or, on a level that walks every
// bucket (level 0 of a build, or a queue that overflowed), the entry array
// itself.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bucket_start(const uint32_t* __restrict__ end, int64_t b) {
    return b > 0 ? __ldcg(end + b - 1) : 0u;
}

// Last bucket r in [lo, hi) with start(r) <= f (start(lo) <= f), warp-wide.
__device__ __forceinline__ int64_t bucket_of_warp(const uint32_t* __restrict__ end, int64_t lo, int64_t hi,
                                                  int64_t f) {
    const int lane = (int)lane_id();
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t idx = lo + step * (lane + 1);
        const bool le = idx < hi && (int64_t)bucket_start(end, idx) <= f;
        const int c = __popc(__ballot_sync(0xFFFFFFFFu, le));
        const int64_t nlo = lo + step * c;
        const int64_t nhi = (c < 32) ? min(hi, lo + step * (c + 1)) : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

__device__ __forceinline__ int64_t bucket_of_thread(const uint32_t* __restrict__ end, int64_t lo, int64_t hi,
                                                    int64_t f) {
    while (hi - lo > 1) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)bucket_start(end, mid) <= f) lo = mid; else hi = mid;
    }
    return lo;
}

// Warp-aggregated append of buckets; a full queue raises its level's
// overflow word instead (the next level then walks every bucket).
__device__ __forceinline__ void bucket_append(bool want, uint32_t b, uint32_t start, uint32_t len,
                                              QEntry* __restrict__ q, unsigned long long* ctr,
                                              unsigned long long* overflow, int32_t cap, bool guard) {
    const unsigned wm = __ballot_sync(0xFFFFFFFFu, want);
    if (wm == 0u) return;
    const int lane = (int)lane_id();
    const int d = want ? (int)len : 0;
    int incl = d;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
        if (lane >= s) incl += y;
    }
    const int totd = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long base = ~0ull;
    if (lane == 0) {
        // on graphs whose level could append 2^26 buckets (the count field's
        // width), a queue already at capacity is not grown further
        if (!guard || (int32_t)(__ldcg(ctr) >> kCountShift) < cap)
            base = atomicAdd(ctr, ((unsigned long long)__popc(wm) << kCountShift) | (unsigned long long)totd);
        else
            atomicOr(overflow, 1ull);
    }
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base == ~0ull || !want) return;
    const int32_t slot = (int32_t)(base >> kCountShift) + __popc(wm & ((1u << lane) - 1u));
    if (slot < cap) {
        QEntry e;
        e.v = (int32_t)b;
        e.rp = (int32_t)start;
        e.off = (int32_t)(base & kEdgeMask) + (incl - d);
        e.aux = len;
        q[slot] = e;
    } else {
        atomicOr(overflow, 1ull);
    }
}

// A speculative continuation of a level (the chains of small levels): the
// bucket (o, c) a lane just raised, processed again at once by the same warp
// with the raised bits.  The bucket is also queued for the next level as
// usual, so the continuation only adds propagation of values the registers
// already hold (max-merges of valid values are safe in any order and number):
// a chain of small buckets then advances several hops per level.
struct InlineCand {
    bool ok = false;
    uint32_t b = 0u, start = 0u, len = 0u, bits = 0u;
};
constexpr int kChainCap = 32;        // continuation stack entries per warp
constexpr uint32_t kChainMaxLen = 32;  // bucket entries a continuation may take (one batch)

// One position of a bucket walk: bucket bkt (vertex u, chunk c), list entry
// e, change bits chb of the chunk (valid false: a lane past the walk's end,
// which still joins the warp-wide enqueue).  ic: the raised target bucket,
// when its first change this level queued it and it is small enough to
// continue at once.
template <int KIND, int MODE>
__device__ __forceinline__ void bucket_pos(const GraphDev& g, const LevelArgs& a, bool valid, uint32_t bkt,
                                           int64_t e, uint32_t chb, StatT& st_chunks,
                                           StatT& st_cas, StatT& st_new,
                                           StatT& st_dealt, bool out_b, InlineCand& ic) {
    const int J = a.J;
    const uint32_t C = (uint32_t)a.chunks;
    if (valid) bkt = chk(bkt, a.nbuckets, a.err);
    const uint32_t u = bkt / C, c = bkt % C;
    uint32_t nbits = 0u;
    int32_t o = 0;
    // the entry and the source piece are fetched with the change bits
    uint32_t m16 = 0u;
    uint4 src = make_uint4(0u, 0u, 0u, 0u);
    if (valid) {
#ifdef IM_BOUNDS_CHECK
        e = chk(e, (int64_t)__ldcg(a.bk_end + a.nbuckets - 1), a.err);
#endif
        o = chk(__ldg(a.bk_other + e), g.n, a.err);
        m16 = __ldg(a.bk_mask + e);
        src = ld_cg16(a.M + (size_t)u * J + c * 16);
    }
    uint32_t imp = 0u;
    uint4 tg = make_uint4(0u, 0u, 0u, 0u);
    uint32_t cand[4] = {0u, 0u, 0u, 0u};
    uint32_t any = 0u;
    uint8_t* trow = a.M + (size_t)o * J + c * 16;
    if (valid && chb) {
        ++st_dealt;
        m16 &= chb;
        tg = ld_cg16(trow);
        const uint32_t sw[4] = {src.x, src.y, src.z, src.w};
        const uint32_t tw[4] = {tg.x, tg.y, tg.z, tg.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t L = bits_to_bytes((m16 >> (4 * w)) & 0xFu);
            if constexpr (MODE == kPush) cand[w] = sw[w] & L & ~visited_bytes(sw[w]);
            else if constexpr (MODE == kCover) cand[w] = L & visited_bytes(sw[w]) & ~visited_bytes(tw[w]);
            else cand[w] = L & ~visited_bytes(tw[w]);
            any |= cand[w];
            // registers this item raises, as the loaded target piece shows
            if constexpr (MODE == kPush) imp |= bytes_to_bits(byte_max(tw[w], cand[w]) ^ tw[w]) << (4 * w);
            else if constexpr (MODE == kCover) imp |= bytes_to_bits(cand[w]) << (4 * w);
        }
        if constexpr (MODE == kAffect) imp = mark_affected(a, cand, o, c, st_new);
    }
    // the enqueue's loads and atomics go out before the register update
    const EnqueueState eq = out_b ? bucket_enqueue_issue(a, o, c, imp)
                                  : vertex_enqueue_issue<KIND, MODE>(g, a, o, c, imp);
    if (MODE != kAffect) {
        if (any) {
            ++st_chunks;
            if constexpr (MODE == kPush) {
                nbits = merge_chunk(trow, cand, tg, st_cas, a.err);
            } else {
                red_or_piece(trow, cand);
                newly_visited(a, o, c, imp, eq.old, st_new);
                note_newly_visited(a, o, c, imp);
            }
        }
    }
    (void)nbits;
    // enqueue what changed: the target's bucket of this chunk, or the
    // target vertex
    if (out_b) {
        bucket_enqueue_finish(a, imp != 0u, o, c, eq);
        const uint32_t sh = (c & 1u) * 16u;
        if (imp != 0u && ((eq.old >> sh) & 0xFFFFu) == 0u && eq.oe > eq.os && eq.oe - eq.os <= kChainMaxLen) {
            ic.ok = true;
            ic.b = (uint32_t)o * C + c;
            ic.start = eq.os;
            ic.len = eq.oe - eq.os;
            ic.bits = imp;
        }
    } else {
        vertex_enqueue_finish<KIND, MODE>(g, a, imp != 0u, o, eq);
    }
}

// Pushes the warp's continuation candidates (depth d) on its stack; the ones
// that find it full are left to the next level.
__device__ __forceinline__ void chain_push(int4* stk, int& sp, const InlineCand& ic, int d) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, ic.ok);
    if (!m) return;
    const int lane = (int)lane_id();
    const int pos = sp + __popc(m & ((1u << lane) - 1u));
    if (ic.ok && pos < kChainCap)
        stk[pos] = make_int4((int)ic.b, (int)ic.start, (int)ic.len, (int)(ic.bits | ((uint32_t)d << 16)));
    sp = min(kChainCap, sp + __popc(m));
    __syncwarp();
}

// Runs the warp's continuations (last pushed first) while its budget of
// `chain` continuations this level lasts; a continuation pushes its own
// raised buckets.  What is left on the stack is dropped (the next level has
// it queued).
template <int KIND, int MODE>
__device__ __forceinline__ void chain_drain(const GraphDev& g, const LevelArgs& a, int4* stk, int& sp, int chain,
                                            int& used, StatT& st_chunks, StatT& st_cas,
                                            StatT& st_new, StatT& st_batches,
                                            StatT& st_dealt, bool out_b) {
    const int lane = (int)lane_id();
    for (; sp > 0 && used < chain; ++used) {
        --sp;
        const int4 it = stk[sp];
        __syncwarp();
        const uint32_t len = (uint32_t)it.z, bits = (uint32_t)it.w & 0xFFFFu;
        const int d = (int)((uint32_t)it.w >> 16);
        for (uint32_t off = 0; off < len; off += 32) {
            if (lane == 0) ++st_batches;
            InlineCand ic;
            bucket_pos<KIND, MODE>(g, a, off + (uint32_t)lane < len, (uint32_t)it.x,
                                   (int64_t)(uint32_t)it.y + off + lane, bits, st_chunks, st_cas, st_new, st_dealt,
                                   out_b, ic);
            chain_push(stk, sp, ic, d + 1);
        }
    }
    sp = 0;
}

// One bucket-mode unit: flat positions [b0*32, b1*32) of the level's walk.
template <int KIND, int MODE>
__device__ __forceinline__ void bucket_slice(const GraphDev& g, const LevelArgs& a, const QEntry* __restrict__ qlin,
                                             int64_t b0, int64_t b1, int32_t nq, int64_t E, bool dense,
                                             StatT& st_chunks, StatT& st_cas,
                                             StatT& st_new, StatT& st_batches,
                                             StatT& st_dealt, bool out_b, int chain,
                                             bool all_bits) {
    const int lane = (int)lane_id();
    const int words = a.words;
    const uint32_t C = (uint32_t)a.chunks;
    const int64_t nb = a.nbuckets;
    __shared__ int4 sChain[kFBlock / 32][kChainCap];
    int sp = 0, chain_used = 0;
    const uint16_t* chg16 = reinterpret_cast<const uint16_t*>(a.chg_cur);
    const int64_t fend = min(E, b1 << 5);
    int64_t f0 = b0 << 5;
    int32_t qi = 0;
    int4 raw = make_int4(0, 0, 0x7FFFFFFF, 0);
    int64_t bk0 = 0;
    if (!dense) {
        qi = f0 == 0 ? 0 : covering_entry(qlin, nq, f0);
        if (qi + lane < nq) raw = __ldcg(reinterpret_cast<const int4*>(qlin) + qi + lane);
    } else {
        bk0 = bucket_of_warp(a.bk_end, 0, nb, f0);
    }
    for (; f0 < fend; f0 += 32) {
        const int64_t f = f0 + lane;
        uint32_t bkt = 0u;
        int64_t e = f;
        uint32_t chb = 0u;
        if (!dense) {
            const int32_t wi = qi + lane;
            const bool wvalid = wi < nq;
            const int64_t rel = (int64_t)raw.z - f0;
            const int c0 = __popc(__ballot_sync(0xFFFFFFFFu, wvalid && rel <= 0));
            const unsigned starts =
                __reduce_or_sync(0xFFFFFFFFu, (wvalid && rel >= 1 && rel <= 31) ? (1u << rel) : 0u);
            const int myw = c0 - 1 + __popc(starts & ((2u << lane) - 1u));
            // change bits of each window entry's chunk
            // (all_bits: every simulation of the chunk, skipping the load)
            uint32_t cwl = 0u;
            if (wvalid && rel <= 31 && lane >= c0 - 1) {
                const uint32_t bw = (uint32_t)raw.x;
                cwl = all_bits ? 0xFFFFu : chg16[(size_t)(bw / C) * words * 2 + (bw % C)];
            }
            bkt = (uint32_t)__shfl_sync(0xFFFFFFFFu, raw.x, myw);
            const int32_t qrp = __shfl_sync(0xFFFFFFFFu, raw.y, myw);
            const int32_t qoff = __shfl_sync(0xFFFFFFFFu, raw.z, myw);
            chb = __shfl_sync(0xFFFFFFFFu, cwl, myw);
            e = (int64_t)(uint32_t)qrp + (f - qoff);
            // the window of the next batch: the entry covering f0 + 32
            const int n32 = __popc(__ballot_sync(0xFFFFFFFFu, wvalid && rel <= 32));
            int32_t qn = qi + n32 - 1;
            if (n32 == 32 && qi + 32 < nq) {
                if ((int64_t)__ldcg(&qlin[qi + 32].off) <= f0 + 32) qn = qi + 32;
            }
            int4 rawn = make_int4(0, 0, 0x7FFFFFFF, 0);
            if (f0 + 32 < fend && qn + lane < nq) rawn = __ldcg(reinterpret_cast<const int4*>(qlin) + qn + lane);
            qi = qn;
            raw = rawn;
        } else {
            // windows of 32 bucket starts from bk0: a position takes the last
            // bucket starting at or before it once a later start is known to
            // exceed it; unresolved positions (a run of empty buckets) move
            // on with the next window, 31 buckets further
            int64_t base = bk0;
            int64_t bf = bk0;
            bool done = f >= fend;
            for (;;) {
                const int64_t bl = base + lane;
                const uint32_t beg = bl < nb ? bucket_start(a.bk_end, bl) : 0xFFFFFFFFu;
                const uint32_t b31 = __shfl_sync(0xFFFFFFFFu, beg, 31);
                int i = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const uint32_t bb = __shfl_sync(0xFFFFFFFFu, beg, (i + s) & 31);
                    if (i + s <= 31 && (int64_t)bb <= f) i += s;
                }
                uint32_t cwl = 0xFFFFu;
                if (!a.all_changed && bl < nb) cwl = chg16[(size_t)(bl / C) * words * 2 + (bl % C)];
                const uint32_t cw_i = __shfl_sync(0xFFFFFFFFu, cwl, i);
                if (!done && (i < 31 || (int64_t)b31 > f || base + 32 >= nb)) {
                    bf = base + i;
                    chb = cw_i;
                    done = true;
                }
                if (__all_sync(0xFFFFFFFFu, done)) break;
                base += 31;
            }
            bkt = (uint32_t)bf;
            bk0 = __shfl_sync(0xFFFFFFFFu, bf, 31);
            if (a.gflag && chb) {
                // a batch rebuild walks only the graphs whose rule fired
                if (!__ldg(a.gflag + __ldg(a.gid + bkt / C))) chb = 0u;
            }
        }
        if (lane == 0) ++st_batches;
        InlineCand ic;
        bucket_pos<KIND, MODE>(g, a, f < fend, bkt, e, chb, st_chunks, st_cas, st_new, st_dealt, out_b, ic);
        if (chain > 0) {
            chain_push(sChain[threadIdx.x >> 5], sp, ic, 1);
            chain_drain<KIND, MODE>(g, a, sChain[threadIdx.x >> 5], sp, chain, chain_used, st_chunks, st_cas,
                                    st_new, st_batches, st_dealt, out_b);
        }
    }
}

struct LevelStats {
    StatT chunks = 0, cas = 0, fresh = 0, hsims = 0, batches = 0, dealt = 0, live = 0, bentries = 0, chg = 0;
};

// Clears the change bits read by the level before the previous one.
__device__ __forceinline__ void clear_prev_bits(const LevelArgs& a, int64_t warp, int64_t nwarps) {
    if (!a.chg_prev) return;
    const int lane = (int)lane_id();
    const int32_t nlp = a.cl_prev ? (int32_t)(__ldcg(a.cl_prev) >> kCountShift) : 0;
    auto clear_all = [&](int64_t nw) {
        for (int64_t i = warp * 32 + lane; i < nw; i += nwarps * 32) a.chg_prev[i] = 0u;
    };
    if (a.fmt_prev && __ldcg(a.fmt_prev) == kFmtDense) {
        // a level without a queue (dense format): every change word
        clear_all((int64_t)a.vq_cap * a.words);
        return;
    }
    if (a.fmt_prev && __ldcg(a.fmt_prev) == kFmtBucket) {
        // bucket queue: each entry owns the 16 change bits of its chunk; a
        // queue that overflowed (its level walked every bucket) clears all
        const bool overflow = nlp > a.bq_cap || (a.ch_prev && __ldcg(a.ch_prev) != 0ull);
        if (overflow) {
            clear_all((int64_t)a.nbuckets / a.chunks * a.words);
            return;
        }
        uint16_t* h16 = reinterpret_cast<uint16_t*>(a.chg_prev);
        for (int64_t i = warp * 32 + lane; i < nlp; i += nwarps * 32) {
            const uint32_t b = chk((uint32_t)__ldcg(&a.ql_prev[i].v), a.nbuckets, a.err);
            const uint32_t u = b / (uint32_t)a.chunks, c = b % (uint32_t)a.chunks;
            h16[(size_t)u * a.words * 2 + c] = 0;
        }
        return;
    }
    const int32_t nhp = a.ch_prev ? (int32_t)(__ldcg(a.ch_prev) >> kCountShift) : 0;
    for (int64_t i = warp; i < (int64_t)nlp + nhp; i += nwarps) {
        const int32_t v = chk(i < nlp ? __ldcg(&a.ql_prev[i].v) : __ldcg(&a.qh_prev[i - nlp].v), a.vq_cap, a.err);
        if (lane < a.words) a.chg_prev[(size_t)v * a.words + lane] = 0u;
    }
}

// Clearing the previous level's change bits as claimable units (taken by the
// warps that find no work, off the critical path of the ones that do): mode 1
// vertex entries (all words of each), 2 bucket entries (their 16 bits), 3 the
// whole buffer (an overflowed bucket queue); 32 entries or 1024 words a unit.
struct ClearPlan {
    int mode = 0;
    int64_t n = 0, units = 0, nl = 0;
};

__device__ __forceinline__ ClearPlan clear_plan(const LevelArgs& a, unsigned long long pl, unsigned long long ph,
                                                int pfmt) {
    ClearPlan c;
    if (!a.chg_prev) return c;
    const int32_t nlp = (int32_t)(pl >> kCountShift);
    if (pfmt == kFmtDense) {
        c.mode = 3;
        c.n = (int64_t)a.vq_cap * a.words;
        c.units = (c.n + 1023) >> 10;
        return c;
    }
    if (pfmt == kFmtBucket) {
        if (nlp > a.bq_cap || ph != 0ull) {
            c.mode = 3;
            c.n = (int64_t)a.nbuckets / a.chunks * a.words;
            c.units = (c.n + 1023) >> 10;
        } else {
            c.mode = 2;
            c.n = nlp;
            c.units = (c.n + 31) >> 5;
        }
    } else {
        c.mode = 1;
        c.nl = nlp;
        c.n = (int64_t)nlp + (int64_t)(ph >> kCountShift);
        c.units = (c.n + 31) >> 5;
    }
    return c;
}

__device__ __forceinline__ void clear_unit(const LevelArgs& a, const ClearPlan& c, int64_t u) {
    const int lane = (int)lane_id();
    if (c.mode == 3) {
        for (int64_t i = (u << 10) + lane; i < min(c.n, (u + 1) << 10); i += 32) a.chg_prev[i] = 0u;
    } else if (c.mode == 2) {
        const int64_t i = (u << 5) + lane;
        if (i < c.n) {
            const uint32_t b = chk((uint32_t)__ldcg(&a.ql_prev[i].v), a.nbuckets, a.err);
            const uint32_t v = b / (uint32_t)a.chunks, ch = b % (uint32_t)a.chunks;
            reinterpret_cast<uint16_t*>(a.chg_prev)[(size_t)v * a.words * 2 + ch] = 0;
        }
    } else if (c.mode == 1) {
        const int64_t i = (u << 5) + lane;
        if (i < c.n) {
            const int32_t v = chk(i < c.nl ? __ldcg(&a.ql_prev[i].v) : __ldcg(&a.qh_prev[i - c.nl].v), a.vq_cap, a.err);
            for (int w = 0; w < a.words; ++w) a.chg_prev[(size_t)v * a.words + w] = 0u;
        }
    }
}

// Units of a level: each warp first takes a fixed unit, spread over the
// blocks (the k-th warps of all blocks before any (k+1)-th warp, so a small
// level runs on many SMs), then, when the level has more units than warps,
// claims further ones from the level's counter.  A warp without a unit makes
// no atomic: a small level costs no contended claims.
struct UnitCursor {
    int64_t unit, total, nwarps;
    __device__ __forceinline__ UnitCursor(int64_t total_units) {
        nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        unit = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
        total = total_units;
    }
    __device__ __forceinline__ bool valid() const { return unit < total; }
    __device__ __forceinline__ void next(unsigned int* claim) {
        if (total <= nwarps) { unit = total; return; }
        unsigned int c = 0;
        if (lane_id() == 0) c = atomicAdd(claim, 1u);
        unit = nwarps + (int64_t)__shfl_sync(0xFFFFFFFFu, c, 0);
    }
};

// Work of one level: heavy vertices first, then slices of light batches, taken through
// a UnitCursor.  BK: the sketch may have bucketed lists (false: edge scans
// only, so the bucket code is compiled out and the scan loops keep more
// registers).
template <int KIND, int MODE, bool BK>
__device__ __forceinline__ void level_work(const GraphDev& g, const LevelArgs& a, const uint32_t* sX,
                                           const uint16_t* sTab, int64_t warp, LevelStats& ls,
                                           uint32_t (*sKeep)[kKeepWords], unsigned long long cl,
                                           unsigned long long ch, int in_fmt, const ClearPlan& cp) {
    const bool in_b = in_fmt == kFmtBucket;
    const int lane = (int)lane_id();
    // output format: bucket entries once the level's input work is small
    // against the graph (the bucketed lists then skip the edges of unchanged
    // chunks), vertex entries otherwise
    auto out_bucket = [&](int64_t work) {
        // the affected-set search is sparse in simulations: bucket queues
        // whenever the sketch has the lists
        if (!BK) return false;
        if (MODE == kAffect) return a.bk_end != nullptr;
        return a.bk_end != nullptr && a.bucket_div > 0 && work * a.bucket_div < g.m;
    };
    if (BK && in_b) {
        // the queue's buckets, or every bucket when the queue overflowed
        // (ch = overflow word)
        const int32_t nq = (int32_t)(cl >> kCountShift);
        const bool dense = a.all_changed || nq > a.bq_cap || ch != 0ull;
        const int64_t E = dense ? (int64_t)__ldcg(a.bk_end + a.nbuckets - 1) : (int64_t)(cl & kEdgeMask);
        const bool out_b = out_bucket(E);
        if (a.fmt_out && blockIdx.x == 0 && threadIdx.x == 0) *a.fmt_out = out_b ? 1 : 0;
        const int64_t nbl = (E + 31) >> 5;
        const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        const int64_t lb = max((int64_t)1, min((int64_t)a.light_batches, nbl / nwarps));
        const int64_t units = (nbl + lb - 1) / lb;
        if (units + cp.units == 0) return;
        // continuations on levels of at most one batch a warp (not in covers,
        // whose small levels fan out rather than chain)
        const int chain = (MODE != kCover && a.chain > 0 && out_b && !dense && nbl <= nwarps) ? a.chain : 0;
        // on such small levels a propagation or cover takes every simulation of
        // a queued chunk, not only the changed ones (one dependent load less
        // per hop): a simulation that did not change was pushed along every
        // live edge when it last did, so its targets already hold at least its
        // value (a visited one's targets are visited), and it raises nothing
        const bool all_bits = MODE != kAffect && !dense && nbl <= nwarps && a.gflag == nullptr;
        if (warp == 0 && lane == 0) {
            atomicAdd(a.stats + (MODE == kPush ? kStSweepBuckets : kStCoverVertices), (unsigned long long)nq);
            // the input of a level after the first: what the previous level changed
            if (MODE == kPush && a.cl_prev) atomicAdd(a.stats + kStSweepChangedBuckets, (unsigned long long)nq);
            if (MODE == kCover) atomicAdd(a.stats + kStCoverEdges, (unsigned long long)E);
            atomicAdd(a.stats + (MODE == kPush ? kStSweepLevels : kStCoverLevels), 1ull);
        }
        for (UnitCursor uc(units + cp.units); uc.valid(); uc.next(a.claim)) {
            const int64_t unit = uc.unit;
            if (unit >= units) {
                clear_unit(a, cp, unit - units);
                continue;
            }
            const int64_t b0 = unit * lb;
            const int64_t b1 = min(nbl, b0 + lb);
            bucket_slice<KIND, MODE>(g, a, a.ql_in, b0, b1, nq, E, dense, ls.chunks, ls.cas, ls.fresh,
                                     ls.batches, ls.bentries, out_b, chain, all_bits);
        }
        return;
    }
    int32_t nl = (int32_t)(cl >> kCountShift);
    const int32_t nl_in = nl;  // the input's count (raised items after a dense-format level)
    int64_t El = (int64_t)(cl & kEdgeMask);
    int32_t nh = (int32_t)(ch >> kCountShift);
    const QEntry* ql = a.ql_in;
    // dense level: walk every vertex with in-edges (propagation) or out-edges
    // (cover) in vertex order (contiguous CSR reads); vertices without changed
    // simulations produce no chunks.  A propagation level goes dense when its
    // frontier holds more than n_dense / dense_div vertices, a cover level when
    // its frontier's out-edges exceed m / dense_div (a cascade's frontier is
    // few hubs with most edges).  A dense-format input (no queue: its count is
    // the raised items) is always walked this way.
    constexpr bool kDenseMode = MODE == kPush || MODE == kCover;
    const bool in_d = kDenseMode && in_fmt == kFmtDense;
    bool dense = in_d;
    if (kDenseMode && a.q_dense && a.dense_div > 0 && (nl + nh) > 0) {
        if (MODE == kPush && ((int64_t)(nl + nh) * a.dense_div > (int64_t)a.n_dense || a.all_changed)) dense = true;
        if (MODE == kCover && El * a.dense_div > g.m) dense = true;
    }
    // the output of a dense walk stays in dense format while the frontier is
    // large: the input's vertices (or, after a dense-format level, its raised
    // items, several per vertex) above n_dense / dense_div
    bool out_d = false;
    if (kDenseMode && dense && a.dense_out)
        out_d = in_d ? (int64_t)nl * a.dense_div > 4 * (int64_t)a.n_dense : true;
    if (dense) {
        ql = a.q_dense;
        nl = a.n_dense;
        El = a.e_dense;
        if (in_d) nh = 0;
    }
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // a small level scans the hubs' in-edges as a second flat edge space
    // (split over many warps) instead of searching per changed simulation:
    // the searches' chains of dependent loads would set the level's latency
    const int64_t Eh = in_d ? 0 : (int64_t)(ch & kEdgeMask);
    // a dense-format output scans the hubs' in-edges in the walk (the hub path
    // would enqueue them), so the heavy queue is not used then
    if (out_d && nh > 0) nh = 0;
    const bool hscan = MODE == kPush && nh > 0 && El + Eh <= nwarps * 32 * 4;
    const int64_t nbl = (El + 31) >> 5;
    const int64_t nbh = hscan ? (Eh + 31) >> 5 : 0;
    // batches per claim: the tuned value, fewer when the level has fewer
    // batches than warps (shorter chains on small levels)
    const int64_t lb = max((int64_t)1, min((int64_t)a.light_batches, (nbl + nbh) / nwarps));
    const int64_t lunits = (nbl + lb - 1) / lb;
    const int64_t hunits = (nbh + lb - 1) / lb;
    const int64_t nhv = hscan ? 0 : (int64_t)nh;  // hubs searched per changed simulation
    const int64_t total = nhv + lunits + hunits;
    const bool out_b = !out_d && out_bucket(El + Eh);
    if (a.fmt_out && blockIdx.x == 0 && threadIdx.x == 0) *a.fmt_out = out_d ? kFmtDense : (out_b ? kFmtBucket : kFmtVertex);
    if (total + cp.units == 0) return;
    if (warp == 0 && lane == 0) {
        atomicAdd(a.stats + (MODE == kPush ? kStSweepVertices : kStCoverVertices),
                  (unsigned long long)(nl + nh));
        // the input of a level after the first: the vertices the previous
        // level changed (the queues' own counts, also on a dense walk; after
        // a dense-format level the walk counts them)
        if (MODE == kPush && a.cl_prev && !in_d)
            atomicAdd(a.stats + kStSweepChanged, (cl >> kCountShift) + (ch >> kCountShift));
        atomicAdd(a.stats + (MODE == kPush ? kStSweepEdges : kStCoverEdges), (unsigned long long)(El + (hscan ? Eh : 0)));
        atomicAdd(a.stats + (MODE == kPush ? kStSweepLevels : kStCoverLevels), 1ull);
        if (MODE == kPush) atomicAdd(a.stats + kStSweepHeavy, (unsigned long long)nhv);
    }
    StatT draised = 0;  // raised items of a dense-format output
    // dense_all: a dense walk pushes every live simulation while the frontier
    // is large (a vertex queue that went dense, or a dense-format input with
    // more than two raised items per vertex): what a vertex raised earlier in
    // the walk then moves on in the same level; a small dense-format input (a
    // rebuild's second level) pushes only what changed
    // A dense cover walk (dense_all bit 1) pushes every visited simulation of
    // every vertex: a register visited at an earlier level, or by an earlier
    // cover, has every live successor visited already (a cover's visited set
    // is closed under live edges once it ends), so it marks nothing, and what
    // a vertex visited earlier in the walk moves on in the same level
    const bool all_sims = (MODE == kPush && dense && (a.dense_all & 1) != 0 &&
                           (!in_d || (int64_t)nl_in > 2 * (int64_t)a.n_dense)) ||
                          (MODE == kCover && dense && (a.dense_all & 2) != 0);
    for (UnitCursor uc(total + cp.units); uc.valid(); uc.next(a.claim)) {
        const int64_t unit = uc.unit;
        if (unit >= total) {
            clear_unit(a, cp, unit - total);
        } else if (unit < nhv) {
            if constexpr (MODE == kPush && (KIND == kWC || KIND == kUniform)) {
                const int4 raw = __ldcg(reinterpret_cast<const int4*>(a.qh_in) + unit);
                QEntry ent;
                ent.v = raw.x; ent.rp = raw.y; ent.off = raw.z; ent.aux = (uint32_t)raw.w;
                heavy_vertex<KIND>(g, a, sX, ent, ls.hsims, ls.cas, out_b);
            }
        } else if ((int64_t)unit < nhv + lunits) {
            const int64_t lu = (int64_t)unit - nhv;
            const int64_t b0 = lu * lb;
            const int64_t b1 = min(nbl, b0 + lb);
            light_slice<KIND, MODE>(g, a, ql, sX, sTab, b0, b1, nl, El, ls.chunks, ls.cas, ls.fresh,
                                    ls.batches, ls.dealt, ls.live, dense && nh > 0, sKeep, out_b, out_d,
                                    MODE == kPush && in_d ? &ls.chg : nullptr, draised, all_sims);
        } else {
            const int64_t hu = (int64_t)unit - nhv - lunits;
            const int64_t b0 = hu * lb;
            const int64_t b1 = min(nbh, b0 + lb);
            light_slice<KIND, MODE>(g, a, a.qh_in, sX, sTab, b0, b1, nh, Eh, ls.chunks, ls.cas, ls.fresh,
                                    ls.batches, ls.dealt, ls.live, false, sKeep, out_b, false, nullptr, draised, false);
        }
    }
    if (out_d) dense_count_flush(a, draised);
}

template <int MODE>
__device__ __forceinline__ void flush_stats(const LevelArgs& a, LevelStats& ls) {
    const unsigned long long chunks = wsum(ls.chunks), cas = wsum(ls.cas), fresh = wsum(ls.fresh),
                             hsims = wsum(ls.hsims), batches = wsum(ls.batches), dealt = wsum(ls.dealt),
                             live = wsum(ls.live), bentries = wsum(ls.bentries), chg = wsum(ls.chg);
    if (lane_id() == 0) {
        if constexpr (MODE == kPush) {
            if (chg) atomicAdd(a.stats + kStSweepChanged, chg);
            if (bentries) atomicAdd(a.stats + kStSweepBucketEntries, bentries);
            if (live) atomicAdd(a.stats + kStSweepLiveEdges, live);
            if (batches) atomicAdd(a.stats + kStSweepBatches, batches);
            if (dealt) atomicAdd(a.stats + kStSweepDealt, dealt);
            if (chunks) atomicAdd(a.stats + kStSweepChunks, chunks);
            if (cas) atomicAdd(a.stats + kStSweepCas, cas);
            if (hsims) atomicAdd(a.stats + kStSweepHeavySims, hsims);
        } else if constexpr (MODE == kCover) {
            if (chunks) atomicAdd(a.stats + kStCoverChunks, chunks);
            if (fresh) {
                atomicAdd(a.stats + kStCoverNew, fresh);
                atomicAdd(a.count, fresh);
            }
        } else {
            if (fresh) atomicAdd(a.stats + kStAffected, fresh);
        }
    }
    ls = LevelStats();
}

__device__ __forceinline__ void load_tables(const LevelArgs& a, uint32_t* sX, uint16_t* sTab) {
    for (int i = threadIdx.x; i < a.J; i += blockDim.x) sX[i] = __ldg(a.X + i);
    for (int i = threadIdx.x; i < kTabSize; i += blockDim.x) sTab[i] = __ldg(a.tab + i);
    __syncthreads();
}

// One level per launch (used when the host traces every level).
template <int KIND, int MODE>
__global__ void __launch_bounds__(kFBlock, kLevelMinBlocks) k_level(GraphDev g, LevelArgs a) {
    __shared__ __align__(16) uint32_t sX[kMaxJ];
    __shared__ uint16_t sTab[kTabSize];
    __shared__ uint32_t sKeep[kFBlock / 32][32][kKeepWords];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long cl = __ldcg(a.cl_in);
    const unsigned long long ch = a.ch_in ? __ldcg(a.ch_in) : 0ull;
    const int in_fmt = a.fmt_in != nullptr ? (int)__ldcg(a.fmt_in) : kFmtVertex;
    if ((cl >> kCountShift) == 0 && (ch >> kCountShift) == 0 && !a.all_changed) {
        clear_prev_bits(a, warp, nwarps);
        return;
    }
    load_tables(a, sX, sTab);
    LevelStats ls;
    // the previous level's change bits (read by no one any more) are cleared
    // by the warps that find no work
    const ClearPlan cp = clear_plan(a, a.cl_prev ? __ldcg(a.cl_prev) : 0ull, a.ch_prev ? __ldcg(a.ch_prev) : 0ull,
                                    a.fmt_prev != nullptr ? (int)__ldcg(a.fmt_prev) : kFmtVertex);
    level_work<KIND, MODE, true>(g, a, sX, sTab, warp, ls, sKeep[threadIdx.x >> 5], cl, ch, in_fmt, cp);
    flush_stats<MODE>(a, ls);
}

// Grid-wide barrier of a cooperative launch: arrival counter + generation
// word.  Every wait is bounded by `limit_ns` of global time (0: a block that
// has to wait gives up at its first poll); a block that gives up raises
// kErrBarrier and the abort word, and all blocks leave the phase at their
// next barrier.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(unsigned int* arrive, volatile unsigned int* gen, volatile unsigned int* abort_flag,
                             uint32_t* err, unsigned long long limit_ns, unsigned int g0) {
    // one arrival counter (the last block to arrive resets it and advances
    // the generation); the waits poll only the generation word, with the
    // abort word and the clock at the first poll and every 32nd
    __syncthreads();
    __shared__ bool ok;
    if (threadIdx.x == 0) {
        ok = true;
        // g0: the generation word's value before this barrier (it counts the
        // barriers passed, so the caller knows it without a read)
        __threadfence();
        bool last = false;
        if (atomicAdd(arrive, 1u) == gridDim.x - 1u) {
            *arrive = 0u;
            __threadfence();
            atomicAdd((unsigned int*)gen, 1u);
            last = true;
        }
        if (!last) {
            const unsigned long long t0 = global_ns();
            unsigned int it = 0;
            while (*gen == g0) {
                if ((it++ & 31u) == 0u) {
                    if (*abort_flag) { ok = false; break; }
                    if (global_ns() - t0 >= limit_ns) {
                        atomicOr(err, kErrBarrier);
                        *abort_flag = 1u;
                        ok = false;
                        break;
                    }
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok;
}

// All levels of one phase in one cooperative launch: level t uses queue
// buffers t % 3 as in k_level; a grid barrier separates levels; the phase
// ends when both queues of the next level are empty.  BK as in level_work.
template <int KIND, int MODE, bool BK>
__global__ void __launch_bounds__(kFBlock, kPhaseMinBlocks) k_phase(GraphDev g, PhaseArgs p) {
    __shared__ __align__(16) uint32_t sX[kMaxJ];
    __shared__ uint16_t sTab[kTabSize];
    __shared__ uint32_t sKeep[kFBlock / 32][32][kKeepWords];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    LevelArgs a = p.base;
    load_tables(a, sX, sTab);
    LevelStats ls;
    int t = 0;
    if (p.level_ns && blockIdx.x == 0 && threadIdx.x == 0) p.level_ns[0] = global_ns();
    // counters and format of the level's input queue, read once after the
    // barrier that precedes it
    unsigned long long pre_l = __ldcg(&p.ctr[0].x), pre_h = __ldcg(&p.ctr[0].y);
    int pre_f = p.fmt != nullptr ? (int)__ldcg(p.fmt) : kFmtVertex;
    // the previous level's input counters and format (its bits are cleared now)
    unsigned long long prev_l = 0ull, prev_h = 0ull;
    int prev_f = kFmtVertex;
    for (; t < p.max_levels; ++t) {
        const int bi = t % 3, bo = (t + 1) % 3, bp = (t + 2) % 3;
        a.ql_in = p.ql[bi];
        a.cl_in = &p.ctr[t].x;
        a.qh_in = p.qh[bi];
        a.ch_in = &p.ctr[t].y;
        a.ql_out = p.ql[bo];
        a.cl_out = &p.ctr[t + 1].x;
        a.qh_out = p.qh[bo];
        a.ch_out = &p.ctr[t + 1].y;
        if (t >= 1) {
            a.ql_prev = p.ql[bp];
            a.cl_prev = &p.ctr[t - 1].x;
            a.qh_prev = p.qh[bp];
            a.ch_prev = &p.ctr[t - 1].y;
            a.chg_prev = p.chg[bp];
        } else {
            a.ql_prev = nullptr; a.cl_prev = nullptr; a.qh_prev = nullptr; a.ch_prev = nullptr;
            a.chg_prev = nullptr;
        }
        a.chg_cur = p.chg[bi];
        a.chg_next = p.chg[bo];
        a.all_changed = (t == 0 && p.all_first) ? 1 : 0;
        a.claim = p.claim + t;
        a.gen_next = p.gen_base + t;
        a.fmt_in = p.fmt ? p.fmt + t : nullptr;
        a.fmt_out = p.fmt ? p.fmt + t + 1 : nullptr;
        a.fmt_prev = (p.fmt && t >= 1) ? p.fmt + t - 1 : nullptr;
        // the previous level's change bits are cleared by the warps that find
        // no work this level
        const ClearPlan cp = clear_plan(a, prev_l, prev_h, prev_f);
        level_work<KIND, MODE, BK>(g, a, sX, sTab, warp, ls, sKeep[threadIdx.x >> 5], pre_l, pre_h, pre_f, cp);
        prev_l = pre_l;
        prev_h = pre_h;
        prev_f = pre_f;
        if (!grid_barrier(p.bar_arrive, p.bar_gen, p.abort_flag, a.err, p.limit_ns, (unsigned int)t))
            break;
        if (p.level_ns && blockIdx.x == 0 && threadIdx.x == 0) p.level_ns[t + 1] = global_ns();
        pre_l = __ldcg(&p.ctr[t + 1].x);
        pre_h = __ldcg(&p.ctr[t + 1].y);
        pre_f = p.fmt != nullptr ? (int)__ldcg(p.fmt + t + 1) : kFmtVertex;
        if ((pre_l >> kCountShift) == 0 && (pre_h >> kCountShift) == 0) { ++t; break; }
    }
    // the last queue read (t - 1) still has its change bits; clearing them
    // leaves every change mask zero for the next phase
    if (t >= 1 && t < p.max_levels && !*(volatile unsigned int*)p.abort_flag) {
        const int bl = (t - 1) % 3;
        a.ql_prev = p.ql[bl];
        a.cl_prev = &p.ctr[t - 1].x;
        a.qh_prev = p.qh[bl];
        a.ch_prev = &p.ctr[t - 1].y;
        a.chg_prev = p.chg[bl];
        a.fmt_prev = p.fmt ? p.fmt + t - 1 : nullptr;
        clear_prev_bits(a, warp, nwarps);
    }
    flush_stats<MODE>(a, ls);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *p.levels_out = t;
        // a frontier that did not empty within the level limit is an error the
        // host reads with the others (it may read it only after later launches)
        if (t >= p.max_levels) atomicOr(a.err, kErrLevels);
    }
}

int phase_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 152, per_sm = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase<kWC, kPush, true>, kFBlock, 0);
        int pc = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_phase<kWC, kCover, true>, kFBlock, 0);
        if (pc < per_sm) per_sm = pc;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_phase<kWC, kAffect, true>, kFBlock, 0);
        if (pc < per_sm) per_sm = pc;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_phase<kTrivalency, kPush, false>, kFBlock, 0);
        if (pc < per_sm) per_sm = pc;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_phase<kWC, kCover, false>, kFBlock, 0);
        if (pc < per_sm) per_sm = pc;
        for (int kd : {0, 2, 3}) {
            int q = 0;
            if (kd == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_phase<kUniform, kPush, true>, kFBlock, 0);
            if (kd == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_phase<kTrivalency, kPush, true>, kFBlock, 0);
            if (kd == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_phase<kExplicit, kPush, true>, kFBlock, 0);
            if (q < per_sm) per_sm = q;
        }
        if (per_sm < 1 || !coop) per_sm = 0;
        grid = sms * per_sm;
    }
    return grid;
}

template <int KIND, int MODE>
static cudaError_t coop_launch(const GraphDev& g, const PhaseArgs& p, int grid, cudaStream_t st) {
    void* args[] = {(void*)&g, (void*)&p};
    // edge-scan sketches (no bucketed lists) run the variant without the bucket code
    const void* fn = p.base.bk_end != nullptr ? (const void*)k_phase<KIND, MODE, true>
                                              : (const void*)k_phase<KIND, MODE, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kFBlock), args, 0, st);
}

cudaError_t launch_phase(int kind, int mode, const GraphDev& g, const PhaseArgs& p, int grid,
                         cudaStream_t st) {
    if (mode == kPush) {
        switch (kind) {
            case kUniform: return coop_launch<kUniform, kPush>(g, p, grid, st);
            case kWC: return coop_launch<kWC, kPush>(g, p, grid, st);
            case kTrivalency: return coop_launch<kTrivalency, kPush>(g, p, grid, st);
            default: return coop_launch<kExplicit, kPush>(g, p, grid, st);
        }
    }
    if (mode == kAffect) {
        switch (kind) {
            case kUniform: return coop_launch<kUniform, kAffect>(g, p, grid, st);
            case kWC: return coop_launch<kWC, kAffect>(g, p, grid, st);
            case kTrivalency: return coop_launch<kTrivalency, kAffect>(g, p, grid, st);
            default: return coop_launch<kExplicit, kAffect>(g, p, grid, st);
        }
    }
    switch (kind) {
        case kUniform: return coop_launch<kUniform, kCover>(g, p, grid, st);
        case kWC: return coop_launch<kWC, kCover>(g, p, grid, st);
        case kTrivalency: return coop_launch<kTrivalency, kCover>(g, p, grid, st);
        default: return coop_launch<kExplicit, kCover>(g, p, grid, st);
    }
}

int level_grid() {
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 152, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<kWC, kPush>, kFBlock, 0);
        if (per_sm < 1) per_sm = 1;
        grid = sms * per_sm;
    }
    return grid;
}

template <int MODE>
static cudaError_t launch_level_mode(int kind, const GraphDev& g, const LevelArgs& a, int grid,
                                     cudaStream_t st) {
    switch (kind) {
        case kUniform: k_level<kUniform, MODE><<<grid, kFBlock, 0, st>>>(g, a); break;
        case kWC: k_level<kWC, MODE><<<grid, kFBlock, 0, st>>>(g, a); break;
        case kTrivalency: k_level<kTrivalency, MODE><<<grid, kFBlock, 0, st>>>(g, a); break;
        default: k_level<kExplicit, MODE><<<grid, kFBlock, 0, st>>>(g, a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_level(int kind, int mode, const GraphDev& g, const LevelArgs& a, int grid,
                         cudaStream_t st) {
    if (mode == kAffect) return launch_level_mode<kAffect>(kind, g, a, grid, st);
    return mode == kPush ? launch_level_mode<kPush>(kind, g, a, grid, st)
                         : launch_level_mode<kCover>(kind, g, a, grid, st);
}

// ---------------------------------------------------------------------------
// Live chunk masks (once per sketch: the simulations and thresholds are fixed
// for its lifetime).  Bit c of edge e is set iff the edge is live (Eq.
// hash_prob) in at least one simulation of chunk c (sorted simulations 16c ..
// 16c+15).  A level then reads 4 bytes of an edge to learn which of its
// source's changed chunks can move registers; the edge's id, hash and
// threshold are read only for those.
//
// Work split by edges, not rows (a hub's edges spread over many warps): a
// warp takes 512 consecutive edges, finds the row of the first by a 32-ary
// search of the row starts, then for each 32 edges loads the starts of the
// next 32 rows and every lane picks its row among them (a lane whose edge
// lies past those rows, after a run of empty rows, searches on its own).
// ---------------------------------------------------------------------------
// (kLcmEdgesPerWarp, row_of_warp and the row walks are in im_device.cuh.)

// Live masks of one edge over every chunk that holds a candidate simulation:
// fn(c, m16) for each chunk c with m16 != 0 (bit i: simulation 16c + i live).
template <class F>
__device__ __forceinline__ void edge_chunk_masks(uint32_t h, uint32_t thr, int J, const uint32_t* sX,
                                                 const uint16_t* sTab, F&& fn) {
    if (thr >= 0x80000000u) {
        for (int c = 0; c < (J >> 4); ++c) fn(c, 0xFFFFu);
        return;
    }
    if (thr == 0u) return;
    int lo, hi;
    candidate_range(h, thr, J, sX, sTab, lo, hi);
    for (int c = lo >> 4; hi > lo && c <= ((hi - 1) >> 4); ++c) {
        uint32_t m16 = 0u;
        const int j1 = min(hi, 16 * c + 16);
        for (int j = max(lo, 16 * c); j < j1; ++j)
            if ((sX[j] ^ h) < thr) m16 |= 1u << (j - 16 * c);
        if (m16) fn(c, m16);
    }
}

// Chunks of one edge with at least one live simulation: bits c of lo (c <
// 32) and hi (c >= 32).  A chunk's scan stops at its first live simulation
// (sorted X puts an edge's candidates in a few consecutive chunks).
__device__ __forceinline__ void edge_live_chunks(uint32_t h, uint32_t thr, int J, const uint32_t* sX,
                                                 const uint16_t* sTab, uint32_t& lo_mask, uint32_t& hi_mask) {
    lo_mask = 0u;
    hi_mask = 0u;
    if (thr >= 0x80000000u) {
        const int C = J >> 4;
        lo_mask = C >= 32 ? 0xFFFFFFFFu : ((1u << C) - 1u);
        hi_mask = C > 32 ? (C >= 64 ? 0xFFFFFFFFu : ((1u << (C - 32)) - 1u)) : 0u;
        return;
    }
    if (thr == 0u) return;
    int lo, hi;
    candidate_range(h, thr, J, sX, sTab, lo, hi);
    for (int c = lo >> 4; hi > lo && c <= ((hi - 1) >> 4); ++c) {
        const int j1 = min(hi, 16 * c + 16);
        for (int j = max(lo, 16 * c); j < j1; ++j)
            if ((sX[j] ^ h) < thr) {
                if (c < 32) lo_mask |= 1u << c;
                else hi_mask |= 1u << (c - 32);
                break;
            }
    }
}

// Every edge of one CSR orientation with its row (the owner vertex), the
// other endpoint, hash and threshold, edge-balanced over warps:
// fn(e, row, other, h, thr) once per edge.
template <int KIND, int MODE, class F>
__device__ __forceinline__ void for_each_edge(const GraphDev& g, F&& fn) {
    const int32_t* rp = MODE == kPush ? g.rp_in : g.rp_out;
    walk_rows(rp, g.n, g.m, [&](int64_t e, int32_t v) {
        uint32_t h, thr;
        int32_t other;
        if constexpr (MODE == kPush) {
            other = __ldg(g.src_in + e);
            h = __ldg(g.h_in + e);
            const uint32_t aux = KIND == kWC ? __ldg(g.thr_v + v) : 0u;
            if (KIND == kTrivalency && g.tri_b) {
                const int2 tb = __ldg(g.tri_b + v);
                const int cls = (e >= tb.x ? 1 : 0) + (e >= tb.y ? 1 : 0);
                thr = cls == 0 ? g.tri_thr[0] : (cls == 1 ? g.tri_thr[1] : g.tri_thr[2]);
            } else {
                thr = edge_threshold<KIND, true>(g, (uint32_t)other, (uint32_t)v, e, aux);
            }
        } else {
            other = __ldg(g.col_out + e);
            h = __ldg(g.h_out + e);
            thr = edge_threshold<KIND, false>(g, (uint32_t)v, (uint32_t)other, e, 0u);
        }
        fn(e, v, other, h, thr);
    });
}

__device__ __forceinline__ void load_sims(const uint32_t* X, const uint16_t* tab, int J, uint32_t* sX,
                                          uint16_t* sTab) {
    for (int i = threadIdx.x; i < J; i += blockDim.x) sX[i] = __ldg(X + i);
    for (int i = threadIdx.x; i < kTabSize; i += blockDim.x) sTab[i] = __ldg(tab + i);
    __syncthreads();
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(kFBlock) k_live_chunks(GraphDev g, const uint32_t* __restrict__ X,
                                                         const uint16_t* __restrict__ tab, int J,
                                                         uint32_t* __restrict__ lo_out,
                                                         uint32_t* __restrict__ hi_out) {
    __shared__ __align__(16) uint32_t sX[kMaxJ];
    __shared__ uint16_t sTab[kTabSize];
    load_sims(X, tab, J, sX, sTab);
    for_each_edge<KIND, MODE>(g, [&](int64_t e, int32_t, int32_t, uint32_t h, uint32_t thr) {
        uint32_t mlo, mhi;
        edge_live_chunks(h, thr, J, sX, sTab, mlo, mhi);
        lo_out[e] = mlo;
        if (hi_out) hi_out[e] = mhi;
    });
}

// Bucketed live lists: pass 0 counts, pass 1 places (see launch_buckets).
// Edges are walked in row order and a row's edges are sorted by hash, so the
// lanes of a warp often share a bucket (same row, nearby simulations): the
// count pass makes one atomic per bucket and chunk for those lanes together;
// the place pass takes positions one entry at a time (its stores follow).
template <int KIND, int MODE, int PASS>
__global__ void __launch_bounds__(kFBlock) k_buckets(GraphDev g, const uint32_t* __restrict__ X,
                                                     const uint16_t* __restrict__ tab, int J,
                                                     uint32_t* __restrict__ cnt_or_end,
                                                     int32_t* __restrict__ other_out,
                                                     uint16_t* __restrict__ mask_out) {
    __shared__ __align__(16) uint32_t sX[kMaxJ];
    __shared__ uint16_t sTab[kTabSize];
    load_sims(X, tab, J, sX, sTab);
    const int C = J >> 4;
    if constexpr (PASS == 1) {
        for_each_edge<KIND, MODE>(g, [&](int64_t, int32_t v, int32_t other, uint32_t h, uint32_t thr) {
            edge_chunk_masks(h, thr, J, sX, sTab, [&](int c, uint32_t m16) {
                const uint32_t pos = atomicAdd(cnt_or_end + (int64_t)v * C + c, 1u);
                other_out[pos] = other;
                mask_out[pos] = (uint16_t)m16;
            });
        });
        return;
    }
    const int32_t* rp = MODE == kPush ? g.rp_in : g.rp_out;
    walk_rows_all([rp](int32_t r) -> int64_t { return (int64_t)__ldg(rp + r); }, g.n, g.m,
                  [&](int64_t e, int32_t v, bool valid) {
        uint32_t lo = 0u, hi = 0u;
        if (valid) {
            uint32_t h, thr;
            if constexpr (MODE == kPush) {
                const int32_t other = __ldg(g.src_in + e);
                h = __ldg(g.h_in + e);
                const uint32_t aux = KIND == kWC ? __ldg(g.thr_v + v) : 0u;
                thr = edge_threshold<KIND, true>(g, (uint32_t)other, (uint32_t)v, e, aux);
            } else {
                const int32_t other = __ldg(g.col_out + e);
                h = __ldg(g.h_out + e);
                thr = edge_threshold<KIND, false>(g, (uint32_t)v, (uint32_t)other, e, 0u);
            }
            edge_live_chunks(h, thr, J, sX, sTab, lo, hi);
        }
        uint32_t ul = __reduce_or_sync(0xFFFFFFFFu, lo), uh = __reduce_or_sync(0xFFFFFFFFu, hi);
        while (ul | uh) {
            int c;
            if (ul) { c = __ffs(ul) - 1; ul &= ul - 1; }
            else { c = 32 + __ffs(uh) - 1; uh &= uh - 1; }
            const bool mine = ((c < 32 ? lo >> c : hi >> (c - 32)) & 1u) != 0u;
            const long long key = mine ? (long long)v * C + c : -1ll;
            const unsigned grp = __match_any_sync(0xFFFFFFFFu, key);
            if (mine && (int)lane_id() == __ffs(grp) - 1) atomicAdd(cnt_or_end + key, (unsigned)__popc(grp));
        }
    });
}

// Warp fill rate of the live tests (Table 6 analogue).  For every in-edge:
// the simulations where it is live, counted once; the 32-simulation warps
// (draw order) that hold one of them — a kernel testing every simulation in
// draw order runs those warps; and the 32-simulation warps (sorted order,
// aligned) that hold one of them — a kernel over the sorted candidate range
// runs those.  out[0] += edges, out[1] += live (edge, simulation) pairs,
// out[2] += active draw-order warps, out[3] += active sorted-order warps,
// out[4] += candidate simulations (the sorted range's width).
template <int KIND>
__global__ void __launch_bounds__(kFBlock) k_fill_rate(GraphDev g, uint64_t seed, const uint32_t* __restrict__ X,
                                                       const uint16_t* __restrict__ tab, int J,
                                                       unsigned long long* __restrict__ out) {
    __shared__ __align__(16) uint32_t sX[kMaxJ];
    __shared__ uint16_t sTab[kTabSize];
    __shared__ uint16_t sDraw[kMaxJ];  // draw index of the simulation at each sorted position
    __shared__ uint32_t sRaw[kMaxJ];
    load_sims(X, tab, J, sX, sTab);
    for (int d = threadIdx.x; d < J; d += blockDim.x)
        sRaw[d] = (uint32_t)splitmix_at(seed, (uint64_t)d) & 0x7FFFFFFFu;
    __syncthreads();
    for (int d = threadIdx.x; d < J; d += blockDim.x) {
        // the stable sort position of draw d (the order the sketch uses)
        const uint32_t x = sRaw[d];
        int r = 0;
        for (int i = 0; i < J; ++i) r += (sRaw[i] < x) || (sRaw[i] == x && i < d);
        sDraw[r] = (uint16_t)d;
    }
    __syncthreads();
    unsigned long long edges = 0, live = 0, wdraw = 0, wsort = 0, cands = 0;
    for_each_edge<KIND, kPush>(g, [&](int64_t, int32_t, int32_t, uint32_t h, uint32_t thr) {
        ++edges;
        int lo = 0, hi = 0;
        if (thr >= 0x80000000u) { lo = 0; hi = J; }
        else if (thr > 0u) candidate_range(h, thr, J, sX, sTab, lo, hi);
        cands += (unsigned long long)(hi - lo);
        uint32_t draw_warps = 0u;   // bit w: draw-order warp w has a live simulation
        uint32_t sort_warps = 0u;   // bit w: sorted-order warp w has one
        for (int j = lo; j < hi; ++j) {
            if ((sX[j] ^ h) < thr) {
                ++live;
                sort_warps |= 1u << (j >> 5);
                draw_warps |= 1u << (sDraw[j] >> 5);
            }
        }
        wdraw += (unsigned long long)__popc(draw_warps);
        wsort += (unsigned long long)__popc(sort_warps);
    });
    edges = wsum(edges); live = wsum(live); wdraw = wsum(wdraw); wsort = wsum(wsort); cands = wsum(cands);
    if (lane_id() == 0) {
        atomicAdd(out + 0, edges);
        atomicAdd(out + 1, live);
        atomicAdd(out + 2, wdraw);
        atomicAdd(out + 3, wsort);
        atomicAdd(out + 4, cands);
    }
}

cudaError_t launch_fill_rate(int kind, const GraphDev& g, uint64_t seed, const uint32_t* X, const uint16_t* tab,
                             int J, unsigned long long* out, cudaStream_t st) {
    if (g.m == 0) return cudaSuccess;
    const int64_t groups = (g.m + kLcmEdgesPerWarp - 1) / kLcmEdgesPerWarp;
    const int64_t want = (groups + (kFBlock / 32) - 1) / (kFBlock / 32);
    const int grid = (int)max((int64_t)1, min(want, (int64_t)level_grid()));
    switch (kind) {
        case kUniform: k_fill_rate<kUniform><<<grid, kFBlock, 0, st>>>(g, seed, X, tab, J, out); break;
        case kWC: k_fill_rate<kWC><<<grid, kFBlock, 0, st>>>(g, seed, X, tab, J, out); break;
        case kTrivalency: k_fill_rate<kTrivalency><<<grid, kFBlock, 0, st>>>(g, seed, X, tab, J, out); break;
        default: k_fill_rate<kExplicit><<<grid, kFBlock, 0, st>>>(g, seed, X, tab, J, out); break;
    }
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t live_chunks_mode(int kind, const GraphDev& g, const uint32_t* X, const uint16_t* tab, int J,
                                    uint32_t* lo, uint32_t* hi, int grid, cudaStream_t st) {
    switch (kind) {
        case kUniform: k_live_chunks<kUniform, MODE><<<grid, kFBlock, 0, st>>>(g, X, tab, J, lo, hi); break;
        case kWC: k_live_chunks<kWC, MODE><<<grid, kFBlock, 0, st>>>(g, X, tab, J, lo, hi); break;
        case kTrivalency: k_live_chunks<kTrivalency, MODE><<<grid, kFBlock, 0, st>>>(g, X, tab, J, lo, hi); break;
        default: k_live_chunks<kExplicit, MODE><<<grid, kFBlock, 0, st>>>(g, X, tab, J, lo, hi); break;
    }
    return cudaGetLastError();
}

template <int MODE, int PASS>
static cudaError_t buckets_mode(int kind, const GraphDev& g, const uint32_t* X, const uint16_t* tab, int J,
                                uint32_t* ce, int32_t* other, uint16_t* mask, int grid, cudaStream_t st) {
    switch (kind) {
        case kUniform: k_buckets<kUniform, MODE, PASS><<<grid, kFBlock, 0, st>>>(g, X, tab, J, ce, other, mask); break;
        case kWC: k_buckets<kWC, MODE, PASS><<<grid, kFBlock, 0, st>>>(g, X, tab, J, ce, other, mask); break;
        case kTrivalency: k_buckets<kTrivalency, MODE, PASS><<<grid, kFBlock, 0, st>>>(g, X, tab, J, ce, other, mask); break;
        default: k_buckets<kExplicit, MODE, PASS><<<grid, kFBlock, 0, st>>>(g, X, tab, J, ce, other, mask); break;
    }
    return cudaGetLastError();
}

static int edge_walk_grid(const GraphDev& g) {
    const int64_t groups = (g.m + kLcmEdgesPerWarp - 1) / kLcmEdgesPerWarp;
    const int64_t want = (groups + (kFBlock / 32) - 1) / (kFBlock / 32);
    return (int)max((int64_t)1, min(want, (int64_t)level_grid()));
}

// Nonzero entries of cnt[0..n) added to *out (one atomic per block).
__global__ void __launch_bounds__(kFBlock) k_count_nonzero(const uint32_t* __restrict__ cnt, int64_t n,
                                                           unsigned long long* out) {
    __shared__ unsigned long long part[kFBlock / 32];
    unsigned long long c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < n; i += stride) {
        if (i + 4 <= n && ((n & 3) == 0)) {
            const uint4 q = __ldcs(reinterpret_cast<const uint4*>(cnt + i));
            c += (q.x != 0u) + (q.y != 0u) + (q.z != 0u) + (q.w != 0u);
        } else {
            for (int64_t k = i; k < min(n, i + 4); ++k) c += __ldcs(cnt + k) != 0u;
        }
    }
    c = wsum(c);
    if (lane_id() == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kFBlock / 32; ++w) t += part[w];
        if (t) atomicAdd(out, t);
    }
}

cudaError_t launch_buckets(int pass, int kind, int mode, const GraphDev& g, const uint32_t* X,
                           const uint16_t* tab, int J, uint32_t* cnt_or_end, unsigned long long* nonempty,
                           int32_t* other, uint16_t* mask, cudaStream_t st) {
    if (g.m == 0) return cudaSuccess;
    const int grid = edge_walk_grid(g);
    cudaError_t e;
    if (mode == kPush)
        e = pass == 0 ? buckets_mode<kPush, 0>(kind, g, X, tab, J, cnt_or_end, other, mask, grid, st)
                      : buckets_mode<kPush, 1>(kind, g, X, tab, J, cnt_or_end, other, mask, grid, st);
    else
        e = pass == 0 ? buckets_mode<kCover, 0>(kind, g, X, tab, J, cnt_or_end, other, mask, grid, st)
                      : buckets_mode<kCover, 1>(kind, g, X, tab, J, cnt_or_end, other, mask, grid, st);
    if (e != cudaSuccess || pass != 0) return e;
    // the nonempty buckets, counted after the pass (not by a contended
    // counter in it)
    const int64_t nb = (int64_t)g.n * (J >> 4);
    k_count_nonzero<<<152 * 4, kFBlock, 0, st>>>(cnt_or_end, nb, nonempty);
    return cudaGetLastError();
}

cudaError_t launch_live_chunks(int kind, int mode, const GraphDev& g, const uint32_t* X, const uint16_t* tab,
                               int J, uint32_t* lo, uint32_t* hi, cudaStream_t st) {
    if (g.m == 0) return cudaSuccess;
    const int grid = edge_walk_grid(g);
    return mode == kPush ? live_chunks_mode<kPush>(kind, g, X, tab, J, lo, hi, grid, st)
                         : live_chunks_mode<kCover>(kind, g, X, tab, J, lo, hi, grid, st);
}

// ---------------------------------------------------------------------------
// Level-0 queues of a build: every vertex with in-edges, hubs to the heavy queue.
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(kFBlock) k_init_queues(GraphDev g, LevelArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < g.n; v0 += stride) {
        const int64_t v = v0 + threadIdx.x;
        bool want = false, heavy = false;
        int32_t rp = 0, deg = 0;
        uint32_t aux = 0u;
        if (v < g.n) {
            rp = g.rp_in[v];
            deg = g.rp_in[v + 1] - rp;
            if constexpr (KIND == kWC) aux = g.thr_v[v];
            heavy = is_heavy<KIND>(deg, KIND == kWC ? aux : g.thr_uniform, a.heavy_indeg);
            want = deg > 0 && (!a.gflag || a.gflag[a.gid[v]]);
        }
        append(want && !heavy, (int32_t)v, rp, deg, aux, a.ql_out, a.cl_out, g.n, a.err);
        append(want && heavy, (int32_t)v, rp, deg, aux, a.qh_out, a.ch_out, g.n, a.err);
    }
}

cudaError_t launch_init_queues(int kind, const GraphDev& g, const LevelArgs& a, cudaStream_t st) {
    const int grid = 152 * 8;
    switch (kind) {
        case kUniform: k_init_queues<kUniform><<<grid, kFBlock, 0, st>>>(g, a); break;
        case kWC: k_init_queues<kWC><<<grid, kFBlock, 0, st>>>(g, a); break;
        case kTrivalency: k_init_queues<kTrivalency><<<grid, kFBlock, 0, st>>>(g, a); break;
        default: k_init_queues<kExplicit><<<grid, kFBlock, 0, st>>>(g, a); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Incremental rebuild (Alg. 4's rebuild computed exactly on the registers it
// can change).  After covers since the last build, a non-visited register
// (u, j) changes at the rebuild only if u reaches, along live edges of
// simulation j through non-visited vertices, a vertex visited since the last
// build: otherwise u's reach set avoiding the visited vertices is the same as
// at the last build (whatever a visited vertex reaches is visited).  The
// affected registers are found by a search from the newly visited ones along
// in-edges (kAffect levels), reset to the vertex's own rank, raised by a pull
// over their out-edges (whose other registers hold final values), and the
// propagation then runs from the affected registers only.
// ---------------------------------------------------------------------------

// Level-0 bucket entries (warp-collective; lanes with valid false add
// none): for each chunk c of vertex v whose 16 bits in `bits` are nonzero and
// whose bucket (of a's orientation) is nonempty, the bucket goes to the queue
// (q, ctr, overflow word) and, with chg, the bits to that change mask.  The
// warp's (vertex, chunk) items are dealt one per lane (their bucket bounds
// load in parallel); one reservation per warp keeps queue order and edge
// offsets in step.
__device__ __forceinline__ void bucket_level0(const LevelArgs& a, bool valid, int32_t v,
                                              const uint32_t* __restrict__ bits, uint32_t* chg, QEntry* q,
                                              unsigned long long* ctr, unsigned long long* overflow) {
    const int lane = (int)lane_id();
    uint32_t cm_lo = 0u, cm_hi = 0u;
    if (valid)
        for (int w = 0; w < a.words; ++w) {
            const uint32_t hb = halves_nonzero(__ldcg(bits + (size_t)v * a.words + w));
            if (w < 16) cm_lo |= hb << (2 * w);
            else cm_hi |= hb << (2 * (w - 16));
        }
    const int nch = __popc(cm_lo) + __popc(cm_hi);
    int incl = nch;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
        if (lane >= s) incl += y;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0) return;
    const int excl = incl - nch;
    // the item of lane `lane` in the round starting at `base`: its bucket and bounds
    auto item = [&](int base, int64_t& b, uint32_t& st, uint32_t& en) -> bool {
        const int k = base + lane;
        int i = 0;
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            const int ic = __shfl_sync(0xFFFFFFFFu, incl, i + s - 1);
            if (ic <= k) i += s;
        }
        if (i > 31) i = 31;
        const int ex_i = __shfl_sync(0xFFFFFFFFu, excl, i);
        const uint32_t lo_i = __shfl_sync(0xFFFFFFFFu, cm_lo, i), hi_i = __shfl_sync(0xFFFFFFFFu, cm_hi, i);
        const int32_t v_i = __shfl_sync(0xFFFFFFFFu, v, i);
        if (k >= total) return false;
        const int c = nth_chunk(lo_i, hi_i, k - ex_i);
        b = (int64_t)v_i * a.chunks + c;
        st = bucket_start(a.bk_end, b);
        en = __ldcg(a.bk_end + b);
        return en > st;
    };
    // pass 1: the warp's nonempty buckets and their entries
    uint32_t w_cnt = 0u, w_len = 0u;
    for (int base = 0; base < total; base += 32) {
        int64_t b = 0;
        uint32_t st = 0u, en = 0u;
        const bool ne = item(base, b, st, en);
        w_cnt += (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, ne));
        w_len += __reduce_add_sync(0xFFFFFFFFu, ne ? en - st : 0u);
    }
    unsigned long long gb = ~0ull;
    if (lane == 0 && w_cnt) {
        if (a.bq_guard && (int32_t)(__ldcg(ctr) >> kCountShift) >= a.bq_cap) atomicOr(overflow, 1ull);
        else gb = atomicAdd(ctr, ((unsigned long long)w_cnt << kCountShift) | (unsigned long long)w_len);
    }
    gb = __shfl_sync(0xFFFFFFFFu, gb, 0);
    // pass 2: the entries (a warp refused by a full queue still sets its
    // change bits: the level then walks every bucket)
    int32_t slot = gb == ~0ull ? 0 : (int32_t)(gb >> kCountShift);
    uint32_t off = gb == ~0ull ? 0u : (uint32_t)(gb & kEdgeMask);
    const uint16_t* b16 = reinterpret_cast<const uint16_t*>(bits);
    uint16_t* h16 = reinterpret_cast<uint16_t*>(chg);
    for (int base = 0; base < total; base += 32) {
        int64_t b = 0;
        uint32_t st = 0u, en = 0u;
        const bool ne = item(base, b, st, en);
        const uint32_t len = ne ? en - st : 0u;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, ne);
        uint32_t lincl = len;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, lincl, s);
            if (lane >= s) lincl += y;
        }
        if (ne) {
            const uint32_t u = (uint32_t)(b / a.chunks), c = (uint32_t)(b % a.chunks);
            const uint16_t bits16 = __ldcg(b16 + (size_t)u * a.words * 2 + c);
            if (h16) h16[(size_t)u * a.words * 2 + c] = bits16;
            const int32_t my = slot + __popc(m & ((1u << lane) - 1u));
            if (gb != ~0ull) {
                if (my < a.bq_cap) {
                    // (a bucket entry's last word: the chunk's bits here, unused by the
                    // level walks, read by the pull)
                    QEntry e;
                    e.v = (int32_t)b; e.rp = (int32_t)st; e.off = (int32_t)(off + lincl - len); e.aux = bits16;
                    q[my] = e;
                } else {
                    atomicOr(overflow, 1ull);
                }
            }
        }
        slot += __popc(m);
        off += __shfl_sync(0xFFFFFFFFu, lincl, 31);
    }
}

// Level-0 vertex entry of v whose change bits are `bits` (one thread): the
// bits go to the change mask; want tells whether v has in-edges and a bit.
template <int KIND>
__device__ __forceinline__ void vertex_level0(const GraphDev& g, const LevelArgs& a, int32_t v,
                                              const uint32_t* __restrict__ bits, bool& want, int32_t& rp,
                                              int32_t& deg, uint32_t& aux, bool& heavy, bool push) {
    want = false;
    heavy = false;
    rp = g.rp_in[v];
    deg = g.rp_in[v + 1] - rp;
    aux = 0u;
    if constexpr (KIND == kWC) aux = g.thr_v[v];
    if (deg <= 0) return;
    uint32_t any = 0u;
    for (int w = 0; w < a.words; ++w) any |= __ldcg(bits + (size_t)v * a.words + w);
    if (!any) return;
    for (int w = 0; w < a.words; ++w) a.chg_next[(size_t)v * a.words + w] = __ldcg(bits + (size_t)v * a.words + w);
    if (push) heavy = is_heavy<KIND>(deg, KIND == kWC ? aux : g.thr_uniform, a.heavy_indeg);
    want = true;
}

// Level 0 of the affected-set search: the newly visited registers (nv).
template <int KIND>
__global__ void __launch_bounds__(kFBlock) k_affect_init(GraphDev g, LevelArgs a, const uint32_t* __restrict__ nv,
                                                         int buckets) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < g.n; v0 += stride) {
        const int64_t v = v0 + threadIdx.x;
        if (buckets) {
            bucket_level0(a, v < g.n, (int32_t)v, nv, a.chg_next, a.ql_out, a.cl_out, a.ch_out);
            continue;
        }
        bool want = false, heavy = false;
        int32_t rp = 0, deg = 0;
        uint32_t aux = 0u;
        if (v < g.n) vertex_level0<KIND>(g, a, (int32_t)v, nv, want, rp, deg, aux, heavy, false);
        append(want, (int32_t)v, rp, deg, aux, a.ql_out, a.cl_out, g.n, a.err);
    }
}

// Affected registers back to the vertex's own rank (Alg. 1); every vertex with
// one goes to `list` with its out-degree and the chunks of its affected bits,
// and, with out-bucket lists (o.bk_end), its affected chunks' out-buckets to
// the pull queue (pq, pctr[0] packed counter, pctr[1] overflow word).
__global__ void __launch_bounds__(kFBlock) k_reset_affected(uint8_t* __restrict__ M, int32_t n, int J, int words,
                                                            const uint32_t* __restrict__ salt,
                                                            const int32_t* __restrict__ hkey,
                                                            const uint32_t* __restrict__ aff, const int32_t* __restrict__ rp_out,
                                                            int32_t* __restrict__ list, int32_t* __restrict__ ldeg,
                                                            uint2* __restrict__ lmask, unsigned int* __restrict__ list_count,
                                                            LevelArgs o, QEntry* pq, unsigned long long* pctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += stride) {
        const int64_t v = v0 + threadIdx.x;
        const int lane = (int)lane_id();
        bool listed = false;
        uint2 lm = make_uint2(0u, 0u);
        uint32_t nzw = 0u;  // words of v with an affected bit (words <= 32)
        if (v < n) {
            uint32_t am_lo = 0u, am_hi = 0u;
            for (int w = 0; w < words; ++w) {
                const uint32_t b = __ldcg(aff + (size_t)v * words + w);
                const uint32_t hb = halves_nonzero(b);
                if (w < 16) am_lo |= hb << (2 * w);
                else am_hi |= hb << (2 * (w - 16));
                if (b) nzw |= 1u << w;
            }
            listed = (am_lo | am_hi) != 0u;
            lm = make_uint2(am_lo, am_hi);
        }
        // the resets, dealt one (vertex, word) a lane: a vertex affected in
        // many simulations spreads over many lanes
        const int nz = __popc(nzw);
        int incl = nz;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
            if (lane >= s) incl += y;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const int excl = incl - nz;
        for (int base = 0; base < total; base += 32) {
            const int k = base + lane;
            int i = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int ic = __shfl_sync(0xFFFFFFFFu, incl, i + s - 1);
                if (ic <= k) i += s;
            }
            if (i > 31) i = 31;
            const int ex_i = __shfl_sync(0xFFFFFFFFu, excl, i);
            const uint32_t nzw_i = __shfl_sync(0xFFFFFFFFu, nzw, i);
            const int64_t v_i = v - lane + i;  // the owner lane's vertex
            if (k < total) {
                const int w = (int)__fns(nzw_i, 0u, k - ex_i + 1);
                const uint32_t ku = mm3_k(hkey ? (uint32_t)hkey[v_i] : (uint32_t)v_i);
                uint32_t b = __ldcg(aff + (size_t)v_i * words + w);
                while (b) {
                    const int j = 32 * w + __ffs(b) - 1;
                    b &= b - 1;
                    M[(size_t)v_i * J + j] = (uint8_t)rank_of(ku, __ldg(salt + j));
                }
            }
        }
        // one list reservation per warp
        const unsigned wm = __ballot_sync(0xFFFFFFFFu, listed);
        if (wm) {
            unsigned int base = 0u;
            if (lane == 0) base = atomicAdd(list_count, (unsigned)__popc(wm));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (listed) {
                const unsigned int i = base + __popc(wm & ((1u << lane) - 1u));
                list[i] = (int32_t)v;
                ldeg[i] = rp_out[v + 1] - rp_out[v];
                lmask[i] = lm;
            }
        }
        if (o.bk_end) bucket_level0(o, v < n, (int32_t)v, aff, nullptr, pq, pctr, pctr + 1);
    }
}

// Pull of the affected registers of the listed vertices over their
// out-edges, edge-balanced (a hub's out-edges spread over many warps):
// M[u][j] = max(M[u][j], M[w][j]) for every live (u -> w) in an affected
// simulation j with w not visited, merged by CAS.
template <int KIND>
__global__ void __launch_bounds__(kFBlock) k_pull_affected(GraphDev g, LevelArgs a, const int32_t* __restrict__ list,
                                                           const int32_t* __restrict__ loff,
                                                           const uint2* __restrict__ lmask, int32_t count) {
    const int64_t total = __ldcg(loff + count);
    __shared__ __align__(16) uint32_t sX[kMaxJ];
    __shared__ uint16_t sTab[kTabSize];
    load_sims(a.X, a.tab, a.J, sX, sTab);
    const int J = a.J, words = a.words;
    StatT n_cas = 0;
    walk_rows(loff, count, total, [&](int64_t f, int32_t row) {
        const int32_t u = chk(__ldg(list + row), g.n, a.err);
        const int64_t e = chk((int64_t)__ldg(g.rp_out + u) + (f - __ldg(loff + row)), g.m, a.err);
        const uint2 am = __ldg(lmask + row);
        uint32_t m_lo = __ldg(a.lcm_lo + e) & am.x;
        uint32_t m_hi = a.lcm_hi ? (__ldg(a.lcm_hi + e) & am.y) : 0u;
        if (!(m_lo | m_hi)) return;
        const int32_t w = chk(__ldg(g.col_out + e), g.n, a.err);
        const uint32_t h = __ldg(g.h_out + e);
        const uint32_t thr = edge_threshold<KIND, false>(g, (uint32_t)u, (uint32_t)w, e, 0u);
        const uint32_t* au = a.aff + (size_t)u * words;
        while (m_lo | m_hi) {
            int c;
            if (m_lo) { c = __ffs(m_lo) - 1; m_lo &= m_lo - 1; }
            else { c = 32 + __ffs(m_hi) - 1; m_hi &= m_hi - 1; }
            const uint32_t a16 = (__ldcg(au + (c >> 1)) >> ((c & 1) * 16)) & 0xFFFFu;
            const uint4* xs = reinterpret_cast<const uint4*>(sX + c * 16);
            const uint4 pw = ld_cg16(a.M + (size_t)w * J + c * 16);
            const uint32_t pv[4] = {pw.x, pw.y, pw.z, pw.w};
            uint32_t cand[4];
            uint32_t any = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t L = live4(xs[q], h, thr) & bits_to_bytes((a16 >> (4 * q)) & 0xFu);
                cand[q] = pv[q] & L & ~visited_bytes(pv[q]);
                any |= cand[q];
            }
            if (!any) continue;
            uint8_t* urow = a.M + (size_t)u * J + c * 16;
            merge_chunk(urow, cand, ld_cg16(urow), n_cas, a.err);
        }
    });
}

// The same pull over the out-bucket lists (a: out orientation): the queue
// holds the affected chunks' buckets; positions of one bucket (one register
// piece M[u][16c..16c+16)) are max-combined across the warp first, so one lane
// per bucket and batch merges.
__global__ void __launch_bounds__(kFBlock) k_pull_buckets(LevelArgs a, const QEntry* __restrict__ q,
                                                          const unsigned long long* __restrict__ pctr) {
    const unsigned long long cv = __ldcg(pctr);
    const int32_t nq = (int32_t)(cv >> kCountShift);
    const int64_t total = (int64_t)(cv & kEdgeMask);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(a.stats + kStPullBuckets, (unsigned long long)nq);
        atomicAdd(a.stats + kStPullEntries, (unsigned long long)total);
    }
    const int J = a.J;
    const uint32_t C = (uint32_t)a.chunks;
    const int lane = (int)lane_id();
    StatT n_cas = 0;
    walk_rows_all([&](int32_t r) -> int64_t { return r < nq ? (int64_t)__ldg(&q[r].off) : total; }, nq, total,
                  [&](int64_t f, int32_t r, bool valid) {
        uint32_t cand[4] = {0u, 0u, 0u, 0u};
        uint32_t b = 0xFFFFFFFFu;
        if (valid) {
            const int4 raw = __ldg(reinterpret_cast<const int4*>(q) + r);
            b = chk((uint32_t)raw.x, a.nbuckets, a.err);
            const uint32_t c = b % C;
            int64_t e = (int64_t)(uint32_t)raw.y + (f - raw.z);
#ifdef IM_BOUNDS_CHECK
            e = chk(e, (int64_t)__ldcg(a.bk_end + a.nbuckets - 1), a.err);
#endif
            const int32_t w = chk(__ldg(a.bk_other + e), a.vq_cap, a.err);
            const uint32_t a16 = (uint32_t)raw.w;  // the chunk's affected bits, from the queue entry
            const uint32_t m16 = __ldg(a.bk_mask + e) & a16;
            if (m16) {
                const uint4 pw = ld_cg16(a.M + (size_t)w * J + c * 16);
                const uint32_t pv[4] = {pw.x, pw.y, pw.z, pw.w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    cand[k] = pv[k] & bits_to_bytes((m16 >> (4 * k)) & 0xFu) & ~visited_bytes(pv[k]);
            }
        }
        if (!__any_sync(0xFFFFFFFFu, (cand[0] | cand[1] | cand[2] | cand[3]) != 0u)) return;
        // segmented max over runs of lanes with the same bucket
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t bo = __shfl_down_sync(0xFFFFFFFFu, b, s);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t x = __shfl_down_sync(0xFFFFFFFFu, cand[k], s);
                if (lane + s < 32 && bo == b) cand[k] = byte_max(cand[k], x);
            }
        }
        const uint32_t bp = __shfl_up_sync(0xFFFFFFFFu, b, 1);
        if (!valid || (lane > 0 && bp == b)) return;
        if (!(cand[0] | cand[1] | cand[2] | cand[3])) return;
        uint8_t* urow = a.M + (size_t)(b / C) * J + (b % C) * 16;
        merge_chunk(urow, cand, ld_cg16(urow), n_cas, a.err);
    });
}

// Level 0 of the propagation after the pull: the listed vertices, their
// affected bits as the change mask (bucket entries in bucket mode).
template <int KIND>
__global__ void __launch_bounds__(kFBlock) k_push_init_list(GraphDev g, LevelArgs a, const int32_t* __restrict__ list,
                                                            const unsigned int* __restrict__ list_count, int buckets) {
    const int64_t cnt = (int64_t)__ldcg(list_count);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < cnt; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const int32_t v = i < cnt ? chk(__ldcg(list + i), g.n, a.err) : 0;
        if (buckets) {
            bucket_level0(a, i < cnt, v, a.aff, a.chg_next, a.ql_out, a.cl_out, a.ch_out);
            continue;
        }
        bool want = false, heavy = false;
        int32_t rp = 0, deg = 0;
        uint32_t aux = 0u;
        if (i < cnt) vertex_level0<KIND>(g, a, v, a.aff, want, rp, deg, aux, heavy, true);
        append(want && !heavy, v, rp, deg, aux, a.ql_out, a.cl_out, g.n, a.err);
        append(want && heavy, v, rp, deg, aux, a.qh_out, a.ch_out, g.n, a.err);
    }
}

// Bucket entries for listed words (warp-collective): word item it = v * words
// + w (valid lanes) gives chunks 2w, 2w+1; each chunk whose 16 bits in `bits`
// are nonzero and whose bucket (a's orientation) is nonempty is queued (its
// bits in the entry's last word), and, with chg, its bits go to that change
// mask.
__device__ __forceinline__ void bucket_words(const LevelArgs& a, bool valid, uint32_t it,
                                             const uint32_t* __restrict__ bits, uint32_t* chg, QEntry* q,
                                             unsigned long long* ctr, unsigned long long* overflow) {
    const int lane = (int)lane_id();
    const uint32_t v = valid ? it / (uint32_t)a.words : 0u, w = valid ? it % (uint32_t)a.words : 0u;
    const uint32_t word = valid ? __ldcg(bits + it) : 0u;
    uint16_t* h16 = reinterpret_cast<uint16_t*>(chg);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const uint32_t b16 = (word >> (16 * half)) & 0xFFFFu;
        const int64_t b = (int64_t)v * a.chunks + 2 * w + half;
        uint32_t st = 0u, en = 0u;
        if (b16) {
            st = bucket_start(a.bk_end, b);
            en = __ldcg(a.bk_end + b);
        }
        const bool ne = b16 != 0u && en > st;
        if (ne && h16) h16[(size_t)it * 2 + half] = (uint16_t)b16;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, ne);
        if (!m) continue;
        const uint32_t len = ne ? en - st : 0u;
        uint32_t incl = len;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
            if (lane >= s) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        unsigned long long gb = ~0ull;
        if (lane == 0) {
            if (a.bq_guard && (int32_t)(__ldcg(ctr) >> kCountShift) >= a.bq_cap) atomicOr(overflow, 1ull);
            else gb = atomicAdd(ctr, ((unsigned long long)__popc(m) << kCountShift) | (unsigned long long)tot);
        }
        gb = __shfl_sync(0xFFFFFFFFu, gb, 0);
        if (!ne || gb == ~0ull) continue;
        const int32_t slot = (int32_t)(gb >> kCountShift) + __popc(m & ((1u << lane) - 1u));
        if (slot < a.bq_cap) {
            QEntry e;
            e.v = (int32_t)b; e.rp = (int32_t)st; e.off = (int32_t)((gb & kEdgeMask) + incl - len); e.aux = b16;
            q[slot] = e;
        } else {
            atomicOr(overflow, 1ull);
        }
    }
}

// Reset of the listed affected words to their vertices' own ranks (Alg. 1),
// and the pull queue of their chunks' out-buckets (o: out orientation).
__global__ void __launch_bounds__(kFBlock) k_reset_words(uint8_t* __restrict__ M, int J, const uint32_t* __restrict__ salt,
                                                         const int32_t* __restrict__ hkey, const uint32_t* __restrict__ aff,
                                                         const uint32_t* __restrict__ awl,
                                                         const unsigned int* __restrict__ awl_count, LevelArgs o,
                                                         QEntry* pq, unsigned long long* pctr) {
    const int64_t cnt = (int64_t)__ldcg(awl_count);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < cnt; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool valid = i < cnt;
        const uint32_t it = valid ? chk(__ldcg(awl + i), (int64_t)o.vq_cap * o.words, o.err) : 0u;
        if (valid) {
            const uint32_t v = it / (uint32_t)o.words, w = it % (uint32_t)o.words;
            const uint32_t ku = mm3_k(hkey ? (uint32_t)hkey[v] : v);
            uint32_t b = __ldcg(aff + it);
            while (b) {
                const int j = 32 * (int)w + __ffs(b) - 1;
                b &= b - 1;
                M[(size_t)v * J + j] = (uint8_t)rank_of(ku, __ldg(salt + j));
            }
        }
        bucket_words(o, valid, it, aff, nullptr, pq, pctr, pctr + 1);
    }
}

// Level 0 of the propagation after the pull from the listed words: their
// chunks' in-buckets, the affected bits as the change mask.
__global__ void __launch_bounds__(kFBlock) k_push_init_words(LevelArgs a, const uint32_t* __restrict__ awl,
                                                             const unsigned int* __restrict__ awl_count) {
    const int64_t cnt = (int64_t)__ldcg(awl_count);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < cnt; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool valid = i < cnt;
        const uint32_t it = valid ? __ldcg(awl + i) : 0u;
        bucket_words(a, valid, it, a.aff, a.chg_next, a.ql_out, a.cl_out, a.ch_out);
    }
}

cudaError_t launch_incremental(int step, int kind, const GraphDev& g, const LevelArgs& a, const IncrArgs& x,
                               cudaStream_t st) {
    const int grid = 152 * 8;
    switch (step) {
        case 0:
            switch (kind) {
                case kUniform: k_affect_init<kUniform><<<grid, kFBlock, 0, st>>>(g, a, x.nv, x.buckets); break;
                case kWC: k_affect_init<kWC><<<grid, kFBlock, 0, st>>>(g, a, x.nv, x.buckets); break;
                case kTrivalency: k_affect_init<kTrivalency><<<grid, kFBlock, 0, st>>>(g, a, x.nv, x.buckets); break;
                default: k_affect_init<kExplicit><<<grid, kFBlock, 0, st>>>(g, a, x.nv, x.buckets); break;
            }
            break;
        case 1:
            if (x.words_list) {
                k_reset_words<<<grid, kFBlock, 0, st>>>(a.M, a.J, x.salt, x.hkey, a.aff, x.awl, x.awl_count, a, x.pq,
                                                        x.pctr);
                break;
            }
            k_reset_affected<<<grid, kFBlock, 0, st>>>(a.M, g.n, a.J, a.words, x.salt, x.hkey, a.aff, g.rp_out,
                                                       x.list, x.ldeg, x.lmask, x.list_count, a, x.pq, x.pctr);
            break;
        case 2: {
            if (!x.pull_buckets && x.count == 0) break;
            const int pg = grid;
            if (x.pull_buckets) {
                k_pull_buckets<<<pg, kFBlock, 0, st>>>(a, x.pq, x.pctr);
                break;
            }
            switch (kind) {
                case kUniform: k_pull_affected<kUniform><<<pg, kFBlock, 0, st>>>(g, a, x.list, x.loff, x.lmask, x.count); break;
                case kWC: k_pull_affected<kWC><<<pg, kFBlock, 0, st>>>(g, a, x.list, x.loff, x.lmask, x.count); break;
                case kTrivalency: k_pull_affected<kTrivalency><<<pg, kFBlock, 0, st>>>(g, a, x.list, x.loff, x.lmask, x.count); break;
                default: k_pull_affected<kExplicit><<<pg, kFBlock, 0, st>>>(g, a, x.list, x.loff, x.lmask, x.count); break;
            }
            break;
        }
        default:
            if (x.words_list) {
                k_push_init_words<<<grid, kFBlock, 0, st>>>(a, x.awl, x.awl_count);
                break;
            }
            switch (kind) {
                case kUniform: k_push_init_list<kUniform><<<grid, kFBlock, 0, st>>>(g, a, x.list, x.list_count, x.buckets); break;
                case kWC: k_push_init_list<kWC><<<grid, kFBlock, 0, st>>>(g, a, x.list, x.list_count, x.buckets); break;
                case kTrivalency: k_push_init_list<kTrivalency><<<grid, kFBlock, 0, st>>>(g, a, x.list, x.list_count, x.buckets); break;
                default: k_push_init_list<kExplicit><<<grid, kFBlock, 0, st>>>(g, a, x.list, x.list_count, x.buckets); break;
            }
            break;
    }
    return cudaGetLastError();
}

}  // namespace im
