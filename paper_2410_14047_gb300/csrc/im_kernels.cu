// Kernels of the sketch-based IM hot path for GB300 (sm_103a).
//
//   k_sims         per-simulation draws X_j, salt_j, FASST sort, range table   (Sec. 2.2, Sec. 4.1)
//   k_fill         Fill-Sketches: M[u][j] = rank of u in simulation j         (Alg. 1, Eq. sketch-init)
//   (im_frontier.cu holds the propagation sweeps and cover levels)
//   k_pick         Sketchwise-Sum + argmax + seed init of the cover        (Eq. gpu-sketch-int, Alg. 4)
//   k_mc_*         independent-cascade Monte-Carlo spread (Sec. 5.1 oracle)
//
// The Monte-Carlo levels walk the flat out-edge space of their queue (sum of
// the queued vertices' out-degrees); each warp owns an equal slice of it, so a
// hub's edges are spread over many warps.
#include <cstdio>

#include "im_launch.h"

namespace im {

constexpr int kBlock = 256;
constexpr int kWarpsPerBlock = kBlock / 32;

// ---------------------------------------------------------------------------
// a1: simulations.  One block; thread j draws SplitMix64 output j, X_j = low 31
// bits, salt_j = high 32 bits; rank-sort by (X, j) (stable); sTab[b] = number
// of X below b << 19.
// ---------------------------------------------------------------------------
__global__ void k_sims(uint64_t seed, int J, uint32_t* X, uint32_t* salt, uint16_t* tab) {
    __shared__ uint32_t sx[kMaxJ];
    __shared__ uint32_t sorted[kMaxJ];
    const int j = threadIdx.x;
    uint32_t x = 0, s = 0;
    if (j < J) {
        const uint64_t z = splitmix_at(seed, (uint64_t)j);
        x = (uint32_t)z & 0x7FFFFFFFu;
        s = (uint32_t)(z >> 32);
        sx[j] = x;
    }
    __syncthreads();
    if (j < J) {
        int r = 0;
        for (int i = 0; i < J; ++i) {
            const uint32_t xi = sx[i];
            r += (xi < x) || (xi == x && i < j);
        }
        sorted[r] = x;
        X[r] = x;
        salt[r] = s;
    }
    __syncthreads();
    for (int b = j; b < kTabSize; b += blockDim.x) {
        const uint32_t key = (uint32_t)b << (31 - kTabBits);
        int lo = 0, hi = J;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sorted[mid] < key) lo = mid + 1; else hi = mid;
        }
        tab[b] = (uint16_t)lo;
    }
}

cudaError_t launch_sims(uint64_t seed, int J, uint32_t* X, uint32_t* salt, uint16_t* tab,
                        cudaStream_t st) {
    k_sims<<<1, kMaxJ, 0, st>>>(seed, J, X, salt, tab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a3: Fill-Sketches (Alg. 1).  Thread per 16-byte chunk of a register row;
// non-visited bytes get the vertex's rank, visited bytes are kept.
// ---------------------------------------------------------------------------
// FRESH: the registers were never written (a new sketch), none is visited:
// every register is written without reading the row first.
template <bool FRESH>
__global__ void __launch_bounds__(kBlock) k_fill(uint8_t* __restrict__ M, int32_t n, int J,
                                                 const uint32_t* __restrict__ salt) {
    const int cpr_log = __ffs(J >> 4) - 1;  // chunks per row = J/16, a power of two
    const int64_t total = (int64_t)n << cpr_log;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)(c >> cpr_log);
        const int ch = (int)(c & ((1 << cpr_log) - 1));
        uint4* p = reinterpret_cast<uint4*>(M + (size_t)u * J + ch * 16);
        const uint4 cur = FRESH ? make_uint4(0u, 0u, 0u, 0u) : *p;
        const uint32_t ku = mm3_k(u);
        const uint4* sl = reinterpret_cast<const uint4*>(salt + ch * 16);
        uint32_t w[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 s4 = __ldg(sl + q);
            const uint32_t r = rank_of(ku, s4.x) | (rank_of(ku, s4.y) << 8) |
                               (rank_of(ku, s4.z) << 16) | (rank_of(ku, s4.w) << 24);
            const uint32_t vis = visited_bytes(w[q]);
            w[q] = (w[q] & vis) | (r & ~vis);
        }
        *p = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__global__ void __launch_bounds__(kBlock) k_fill_flagged(uint8_t* __restrict__ M, int32_t n, int J,
                                                         const uint32_t* __restrict__ salt,
                                                         const int32_t* __restrict__ gid,
                                                         const uint8_t* __restrict__ gflag,
                                                         const int32_t* __restrict__ hkey) {
    const int cpr_log = __ffs(J >> 4) - 1;
    const int64_t total = (int64_t)n << cpr_log;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)(c >> cpr_log);
        if (!gflag[gid[u]]) continue;
        const int ch = (int)(c & ((1 << cpr_log) - 1));
        uint4* p = reinterpret_cast<uint4*>(M + (size_t)u * J + ch * 16);
        const uint4 cur = *p;
        const uint32_t ku = mm3_k((uint32_t)hkey[u]);  // rank of the graph's own vertex id
        const uint4* sl = reinterpret_cast<const uint4*>(salt + ch * 16);
        uint32_t w[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 s4 = __ldg(sl + q);
            const uint32_t r = rank_of(ku, s4.x) | (rank_of(ku, s4.y) << 8) |
                               (rank_of(ku, s4.z) << 16) | (rank_of(ku, s4.w) << 24);
            const uint32_t vis = visited_bytes(w[q]);
            w[q] = (w[q] & vis) | (r & ~vis);
        }
        *p = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

cudaError_t launch_fill_flagged(uint8_t* M, int32_t n, int J, const uint32_t* salt, const int32_t* gid,
                                const uint8_t* gflag, const int32_t* hkey, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t total = (int64_t)n * (J / 16);
    int64_t grid = (total + kBlock - 1) / kBlock;
    if (grid > 152 * 16) grid = 152 * 16;
    k_fill_flagged<<<(int)grid, kBlock, 0, st>>>(M, n, J, salt, gid, gflag, hkey);
    return cudaGetLastError();
}

cudaError_t launch_fill(uint8_t* M, int32_t n, int J, const uint32_t* salt, bool fresh, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t total = (int64_t)n * (J / 16);
    int64_t grid = (total + kBlock - 1) / kBlock;
    if (grid > 152 * 16) grid = 152 * 16;
    if (fresh) k_fill<true><<<(int)grid, kBlock, 0, st>>>(M, n, J, salt);
    else k_fill<false><<<(int)grid, kBlock, 0, st>>>(M, n, J, salt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Flat-edge-space helpers.
// ---------------------------------------------------------------------------

// Index of the last queue entry whose offset is <= f (a warp-wide 32-ary search).
__device__ __forceinline__ int32_t find_covering(const QEntry* __restrict__ q, int32_t count,
                                                 int64_t f) {
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

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, s);
    return x;
}

// ---------------------------------------------------------------------------
// a5 / a6: Sketchwise-Sum + argmax (Alg. 4) + seed init of the cover.
// S_u = sum_j 2^(32 - M[u][j]) with visited = 2^32 (exact uint64); the pick
// is the smallest (S_u, u) over vertices not yet picked.  A warp covers
// 32 / LPR rows at once (LPR = min(J/16, 32) lanes per row, 16 bytes a lane).
// The last block to finish reduces the per-block minima, records the seed
// and its estimate J*2^32/(phi*S), marks its row visited and queues it for
// the cover.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t shr_clamped(uint32_t x, uint32_t s) {
    // PTX shr.u32 clamps shift amounts above 32 to 32 (result 0)
    uint32_t r;
    asm("shr.u32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(s));
    return r;
}

__device__ __forceinline__ unsigned long long row_terms16(uint4 q) {
    // ranks 1..32 give 2^(32-r) = 0x80000000 >> (r - 1), at most 2^31: summed
    // in 64 bits; rank 0 and visited (0xFF) give 2^32: counted per word from
    // its zero and visited bytes (r - 1 wraps above 31 there, and the
    // clamped shift adds 0)
    unsigned long long lo = 0;
    uint32_t big = 0;
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t nz = (((w[i] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w[i]) & 0x80808080u;
        big += (uint32_t)__popc((~nz & 0x80808080u) | (w[i] & 0x80808080u));
#pragma unroll
        for (int b = 0; b < 4; ++b) lo += shr_clamped(0x80000000u, __byte_perm(w[i], 0u, 0x4440u | b) - 1u);
    }
    return ((unsigned long long)big << 32) + lo;
}

// Sum of the row owned by this lane's segment; valid in every lane of the segment.
__device__ __forceinline__ unsigned long long row_sum(const uint8_t* __restrict__ M, int J,
                                                      int32_t row, int lpr, int cpl, int seg_lane) {
    unsigned long long s = 0;
    const uint8_t* p = M + (size_t)row * J;
    for (int c = 0; c < cpl; ++c) {
        const int chunk = seg_lane + c * lpr;
        s += row_terms16(__ldcg(reinterpret_cast<const uint4*>(p) + chunk));
    }
    for (int off = lpr >> 1; off >= 1; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    return s;
}

__device__ __forceinline__ void lex_min(unsigned long long& S, int32_t& u, unsigned long long oS,
                                        int32_t ou) {
    if (oS < S || (oS == S && ou < u)) { S = oS; u = ou; }
}

// Bucket mode: queues the seed's out-buckets whose chunk has newly visited
// simulations (level 0 of its cover); a chunk without live out-edges keeps
// no change bits.  One thread; chg_row = the seed's change words.
__device__ void cover_seed_buckets(int32_t s, uint32_t* chg_row, int C, const uint32_t* bk_end, QEntry* q,
                                   unsigned long long* ctr) {
    uint16_t* h16 = reinterpret_cast<uint16_t*>(chg_row);
    uint32_t k = 0, len_sum = 0;
    for (int c = 0; c < C; ++c) {
        if (!h16[c]) continue;
        const int64_t b = (int64_t)s * C + c;
        const uint32_t st = b > 0 ? bk_end[b - 1] : 0u, en = bk_end[b];
        if (en > st) { ++k; len_sum += en - st; }
        else h16[c] = 0;
    }
    if (k == 0) return;
    const unsigned long long base = atomicAdd(ctr, ((unsigned long long)k << kCountShift) | len_sum);
    uint32_t slot = (uint32_t)(base >> kCountShift), off = (uint32_t)(base & kEdgeMask);
    for (int c = 0; c < C; ++c) {
        if (!h16[c]) continue;
        const int64_t b = (int64_t)s * C + c;
        const uint32_t st = b > 0 ? bk_end[b - 1] : 0u, en = bk_end[b];
        QEntry e;
        e.v = (int32_t)(uint32_t)b; e.rp = (int32_t)st; e.off = (int32_t)off; e.aux = en - st;
        q[slot++] = e;
        off += en - st;
    }
}

// Marks row s visited and queues s as level 0 of a cover (one block).
__device__ void cover_seed_block(uint8_t* M, int J, int32_t s, const int32_t* rp_out, QEntry* q,
                                 unsigned long long* ctr, uint32_t* chg0, unsigned long long* count,
                                 const uint32_t* bk_end = nullptr, int C = 0, uint32_t* nv = nullptr) {
    __shared__ unsigned int newly_sh;
    if (threadIdx.x == 0) newly_sh = 0;
    __syncthreads();
    unsigned int newly = 0;
    uint8_t* row = M + (size_t)s * J;
    const int Jr = (J + 31) & ~31;
    const int words = Jr >> 5;
    for (int j = threadIdx.x; j < Jr; j += blockDim.x) {
        const bool fresh = j < J && row[j] != kVisited;
        if (fresh) { row[j] = (uint8_t)kVisited; ++newly; }
        // change mask of the seed at cover level 0: its newly visited simulations
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, fresh);
        if ((j & 31) == 0) {
            chg0[(size_t)s * words + (j >> 5)] = bits;
            // registers newly visited since the last build (incremental rebuilds)
            if (nv && bits) atomicOr(nv + (size_t)s * words + (j >> 5), bits);
        }
    }
    newly = (unsigned)warp_sum(newly);
    if (lane_id() == 0 && newly) atomicAdd(&newly_sh, newly);
    __syncthreads();
    if (threadIdx.x == 0 && bk_end) {
        const unsigned int nw = newly_sh;
        if (nw) atomicAdd(count, (unsigned long long)nw);
        *ctr = 0ull;
        if (nw) cover_seed_buckets(s, chg0 + (size_t)s * words, C, bk_end, q, ctr);
    } else if (threadIdx.x == 0) {
        const unsigned int nw = newly_sh;
        if (nw) atomicAdd(count, (unsigned long long)nw);
        const int32_t rp = rp_out[s];
        const int32_t deg = rp_out[s + 1] - rp;
        if (nw && deg > 0) {
            QEntry e;
            e.v = s; e.rp = rp; e.off = 0; e.aux = 0;
            q[0] = e;
            *ctr = (1ull << kCountShift) | (unsigned long long)deg;
        } else {
            *ctr = 0ull;
        }
    }
}

// Least and second-least (S, u) pairs in lexicographic order.
struct Top2 {
    unsigned long long s1 = ~0ull, s2 = ~0ull;
    int32_t u1 = 0x7FFFFFFF, u2 = 0x7FFFFFFF;
    __device__ __forceinline__ void insert(unsigned long long s, int32_t u) {
        if (s < s1 || (s == s1 && u < u1)) {
            s2 = s1; u2 = u1; s1 = s; u1 = u;
        } else if (s < s2 || (s == s2 && u < u2)) {
            s2 = s; u2 = u;
        }
    }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long a1 = __shfl_xor_sync(0xFFFFFFFFu, s1, off);
            const unsigned long long a2 = __shfl_xor_sync(0xFFFFFFFFu, s2, off);
            const int32_t b1 = __shfl_xor_sync(0xFFFFFFFFu, u1, off);
            const int32_t b2 = __shfl_xor_sync(0xFFFFFFFFu, u2, off);
            insert(a1, b1);
            insert(a2, b2);
        }
    }
};

constexpr int kGroupRows = 128;  // rows of a lazy-pick group record

__device__ __forceinline__ bool is_picked(const uint32_t* seed_bits, int64_t v) {
    return (__ldcg(seed_bits + (v >> 5)) >> (v & 31)) & 1u;
}

// The two least stored (S, u) of the unpicked rows of group g (warp-wide;
// every lane gets them), and their record in gsum (S1, S2, u1 | u2 << 32).
__device__ __forceinline__ Top2 group_top2(const PickArgs& a, int64_t g) {
    const int lane = (int)lane_id();
    const int64_t r0 = g * kGroupRows;
    Top2 t;
    for (int k = 0; k < kGroupRows / 32; ++k) {
        const int64_t v = r0 + k * 32 + lane;
        if (v < a.n && !is_picked(a.seed_bits, v)) t.insert(__ldcg(a.lb + v), (int32_t)v);
    }
    t.warp_reduce();
    if (lane == 0) {
        a.gsum[4 * g] = t.s1;
        a.gsum[4 * g + 1] = t.s2;
        a.gsum[4 * g + 2] = (unsigned long long)(uint32_t)t.u1 | ((unsigned long long)(uint32_t)t.u2 << 32);
    }
    return t;
}


// Block + grid reduction of the per-thread Top2 (last block by ticket), then
// the seed record: out_seed / out_S / out_est[k], the seed bit, the next
// lazy candidate, and (mark) the seed row visited + queued for the cover.
__device__ void pick_finish(const PickArgs& a, Top2 t) {
    __shared__ unsigned long long sS1[kWarpsPerBlock], sS2[kWarpsPerBlock];
    __shared__ int32_t sU1[kWarpsPerBlock], sU2[kWarpsPerBlock];
    __shared__ bool is_last;
    __shared__ unsigned long long fS;
    __shared__ int32_t fU;
    const int lane = (int)lane_id();
    const int wib = threadIdx.x >> 5;
    t.warp_reduce();
    if (lane == 0) { sS1[wib] = t.s1; sU1[wib] = t.u1; sS2[wib] = t.s2; sU2[wib] = t.u2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kWarpsPerBlock; ++w) { t.insert(sS1[w], sU1[w]); t.insert(sS2[w], sU2[w]); }
        a.part_S[blockIdx.x] = t.s1;
        a.part_u[blockIdx.x] = t.u1;
        if (a.part_S2) { a.part_S2[blockIdx.x] = t.s2; a.part_u2[blockIdx.x] = t.u2; }
        __threadfence();
        const unsigned tk = atomicAdd(a.ticket, 1u);
        is_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    // ---- last block: global top-2, seed record, cover seed ------------------
    __threadfence();
    Top2 g;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        g.insert(__ldcg(a.part_S + b), __ldcg(a.part_u + b));
        if (a.part_S2) g.insert(__ldcg(a.part_S2 + b), __ldcg(a.part_u2 + b));
    }
    g.warp_reduce();
    __syncthreads();  // the shared arrays are reused
    if (lane == 0) { sS1[wib] = g.s1; sU1[wib] = g.u1; sS2[wib] = g.s2; sU2[wib] = g.u2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kWarpsPerBlock; ++w) { g.insert(sS1[w], sU1[w]); g.insert(sS2[w], sU2[w]); }
        fS = g.s1;
        fU = g.u1;
        *a.ticket = 0u;
        if (a.cand) *a.cand = g.s2 == ~0ull ? -1 : g.u2;
        if (g.s1 == ~0ull) {
            a.out_seed[a.k] = -1;
            if (a.ctr_cover) *a.ctr_cover = 0ull;
        } else {
            a.out_seed[a.k] = g.u1;
            a.out_S[a.k] = g.s1;
            a.out_est[a.k] = ((double)a.J * 4294967296.0) / (0.77351 * (double)g.s1);
            a.seed_bits[g.u1 >> 5] |= 1u << (g.u1 & 31);
        }
    }
    __syncthreads();
    // lazy picks: the picked vertex's group is recorded again without it
    if (a.gsum && fS != ~0ull && threadIdx.x < 32) group_top2(a, (int64_t)fU / kGroupRows);
    if (fS == ~0ull || !a.mark) return;
    cover_seed_block(a.M, a.J, fU, a.rp_out, a.q_cover, a.ctr_cover, a.chg0, a.count, a.bk_end_out, a.chunks, a.nv);
}


// Full pick: S_u of every row (stored in lb when lazy picks follow).  Each
// lane sums up to `tile` (1, 2 or 4: the J-tile width, a schedule knob)
// consecutive 16-byte pieces of a row (LPR lanes a row, 32 / LPR rows a warp
// step) and a warp issues the loads of kPickSteps steps before summing any,
// so every warp keeps several KB of the stream in flight.
constexpr int kPickSteps = 2;
constexpr int kLazySteps = 4;
constexpr int kLazyRows = 4;  // stale rows a lazy-pick warp refreshes at once
__host__ __device__ __forceinline__ void pick_layout(int J, int tile, int& cpl, int& lpr, int& rpw) {
    const int cpr = J >> 4;
    // at most 32 lanes a row: a row of 64 pieces (J = 1024) takes 2 a lane at least
    const int least = (cpr + 31) >> 5;
    int tl = tile == 1 || tile == 2 ? tile : 4;
    if (tl < least) tl = least;
    cpl = cpr < tl ? cpr : tl;
    lpr = cpr / cpl;
    rpw = 32 / lpr;
}

__global__ void __launch_bounds__(kBlock) k_pick(PickArgs a) {
    const int J = a.J;
    int cpl, lpr, rpw;
    pick_layout(J, a.tile, cpl, lpr, rpw);
    const int lane = (int)lane_id();
    const int seg = lane / lpr, seg_lane = lane % lpr;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step_rows = (int64_t)rpw * kPickSteps;
    Top2 t;
    for (int64_t r0 = warp * step_rows; r0 < a.n; r0 += nwarps * step_rows) {
        uint4 q[kPickSteps][4];
#pragma unroll
        for (int u = 0; u < kPickSteps; ++u) {
            const int64_t row = r0 + (int64_t)u * rpw + seg;
            const uint4* p = reinterpret_cast<const uint4*>(a.M + (size_t)(row < a.n ? row : 0) * J) +
                             seg_lane * cpl;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                q[u][c] = (c < cpl && row < a.n) ? __ldcs(p + c) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kPickSteps; ++u) {
            const int64_t row = r0 + (int64_t)u * rpw + seg;
            unsigned long long sum = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < cpl) sum += row_terms16(q[u][c]);
            for (int off = lpr >> 1; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
            if (row < a.n && seg_lane == 0) {
                if (a.lb) a.lb[row] = sum;
                if (!is_picked(a.seed_bits, row)) t.insert(sum, (int32_t)row);
            }
        }
    }
    pick_finish(a, t);
}

// S of one row by a whole warp (every lane gets the sum).
__device__ __forceinline__ unsigned long long warp_row_sum(const uint8_t* __restrict__ M, int J,
                                                           int32_t row) {
    const int cpr = J >> 4;
    const uint4* p = reinterpret_cast<const uint4*>(M + (size_t)row * J);
    unsigned long long s = 0;
    for (int c = (int)lane_id(); c < cpr; c += 32) s += row_terms16(__ldcg(p + c));
    return warp_sum(s);
}

// Lazy pick (CELF-style, exact): S_u only grows during a selection (covers
// turn registers into visited = 2^32, rebuilds lower the ranks of what stays
// unvisited), so lb[v] <= S_v.  With S_c fresh for the candidate c, every
// unpicked v with (lb[v], v) < (S_c, c) is refreshed; then the least stored
// pair is the least current pair, the same vertex a full pick chooses.
// Refreshes the stale rows of rows r0 .. r0 + 31 (lv: this lane's stored sum,
// m: the stale lanes), kLazyRows of them at once with their loads in flight
// together (stale rows cluster: influential vertices sit together).
__device__ __forceinline__ void refresh_rows(const PickArgs& a, int64_t r0, unsigned int m) {
    const int lane = (int)lane_id();
    const int J = a.J, cpr = J >> 4;
    while (m) {
        int b[kLazyRows];
#pragma unroll
        for (int r = 0; r < kLazyRows; ++r) {
            b[r] = m ? __ffs(m) - 1 : -1;
            m &= m - 1;
        }
        unsigned long long s[kLazyRows];
#pragma unroll
        for (int r = 0; r < kLazyRows; ++r) s[r] = 0ull;
        // a row has at most 64 pieces: piece lane, then lane + 32
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            if (c >= cpr) break;  // lanes past the row's pieces (J < 512) sum nothing
            uint4 q[kLazyRows];
#pragma unroll
            for (int r = 0; r < kLazyRows; ++r)
                q[r] = b[r] >= 0 ? __ldcg(reinterpret_cast<const uint4*>(a.M + (size_t)(r0 + b[r]) * J) + c)
                                 : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int r = 0; r < kLazyRows; ++r) s[r] += row_terms16(q[r]);
        }
#pragma unroll
        for (int r = 0; r < kLazyRows; ++r) {
            if (b[r] < 0) continue;  // warp-uniform
            const unsigned long long sr = warp_sum(s[r]);
            if (lane == b[r]) a.lb[r0 + b[r]] = sr;
        }
    }
}

// Group records after a full pick (its stored sums and seed bit in place).
__global__ void __launch_bounds__(kBlock) k_group_summaries(PickArgs a) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = warp; g < a.ngroups; g += nwarps) group_top2(a, g);
}

// Lazy pick (CELF-style, exact): S_u only grows during a selection (covers
// turn registers into visited = 2^32, rebuilds lower the ranks of what stays
// unvisited), so lb[v] <= S_v.  With S_c fresh for the candidate c, every
// unpicked v with (lb[v], v) < (S_c, c) is refreshed; then the least stored
// pair is the least current pair, the same vertex a full pick chooses.  The
// rows are read through their groups' records: a group whose least stored
// pair is not below (S_c, c) holds no stale row and gives its two least pairs
// as they are; the few others are refreshed and re-recorded.  The picked
// vertex's group is re-recorded by the last block (pick_finish).
__global__ void __launch_bounds__(kBlock) k_pick_lazy(PickArgs a) {
    const int lane = (int)lane_id();
    const int32_t c = __ldcg(a.cand);
    unsigned long long Sc = 0;
    int32_t uc = -1;  // no candidate: nothing is refreshed
    if (c >= 0) {
        Sc = warp_row_sum(a.M, a.J, c);
        uc = c;
    }
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned refreshed = 0;  // rows refreshed by this warp
    Top2 t;
    // one group a lane; lane l of warp w takes group w + l * nwarps, so the
    // stale groups, which cluster after a rebuild (influential vertices sit
    // together), go to different warps
    for (int64_t base = warp; base < a.ngroups; base += nwarps * 32) {
        const int64_t g = base + (int64_t)lane * nwarps;
        unsigned long long s1 = ~0ull, s2 = ~0ull;
        int32_t u1 = 0x7FFFFFFF, u2 = 0x7FFFFFFF;
        if (g < a.ngroups) {
            s1 = __ldcg(a.gsum + 4 * g);
            s2 = __ldcg(a.gsum + 4 * g + 1);
            const unsigned long long pk = __ldcg(a.gsum + 4 * g + 2);
            u1 = (int32_t)(uint32_t)pk;
            u2 = (int32_t)(uint32_t)(pk >> 32);
        }
        const bool stale = g < a.ngroups && (s1 < Sc || (s1 == Sc && u1 < uc));
        if (!stale) {
            // no stale row: its two least pairs as recorded
            t.insert(s1, u1);
            t.insert(s2, u2);
        }
        unsigned int m = __ballot_sync(0xFFFFFFFFu, stale);
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int64_t gg = base + (int64_t)b * nwarps;
            for (int q = 0; q < kGroupRows / 32; ++q) {
                const int64_t r0 = gg * kGroupRows + q * 32;
                const int64_t v = r0 + lane;
                bool st = false;
                if (v < a.n && !is_picked(a.seed_bits, v)) {
                    const unsigned long long lv = __ldcg(a.lb + v);
                    st = lv < Sc || (lv == Sc && (int32_t)v < uc);
                }
                const unsigned int sm = __ballot_sync(0xFFFFFFFFu, st);
                refreshed += (unsigned)__popc(sm);
                refresh_rows(a, r0, sm);
            }
            const Top2 gt = group_top2(a, gg);
            if (lane == b) {
                t.insert(gt.s1, gt.u1);
                t.insert(gt.s2, gt.u2);
            }
        }
    }
    if (a.stats && lane == 0 && refreshed) atomicAdd(a.stats + kStPickRefreshed, (unsigned long long)refreshed);
    pick_finish(a, t);
}

int pick_grid(int32_t n, int J, int tile) {
    int cpl, lpr, rpw;
    pick_layout(J, tile, cpl, lpr, rpw);
    const int64_t rows_per_block = (int64_t)rpw * kPickSteps * kWarpsPerBlock;
    int64_t grid = (n + rows_per_block - 1) / rows_per_block;
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    return (int)grid;
}

cudaError_t launch_pick(const PickArgs& a, cudaStream_t st) {
    k_pick<<<pick_grid(a.n, a.J, a.tile), kBlock, 0, st>>>(a);
    return cudaGetLastError();
}

int pick_lazy_grid(int32_t n) {
    // one group a lane, and at least 2048 warps: the stale groups of a pick
    // (spread over the warps by the group-to-lane mapping) are refreshed by as
    // many warps as there are
    const int64_t groups = ((int64_t)n + kGroupRows - 1) / kGroupRows;
    int64_t warps = (groups + 31) / 32;
    if (warps < 2048) warps = 2048;
    int64_t grid = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (grid > 152 * 8) grid = 152 * 8;
    return (int)grid;
}

int pick_groups(int32_t n) { return (int)(((int64_t)n + kGroupRows - 1) / kGroupRows); }

cudaError_t launch_group_summaries(const PickArgs& a, cudaStream_t st) {
    int64_t grid = ((int64_t)a.ngroups + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (grid > 152 * 8) grid = 152 * 8;
    k_group_summaries<<<(int)(grid < 1 ? 1 : grid), kBlock, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pick_lazy(const PickArgs& a, cudaStream_t st) {
    k_pick_lazy<<<pick_lazy_grid(a.n), kBlock, 0, st>>>(a);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_cover_seed(uint8_t* M, int J, int32_t s,
                                                       const int32_t* rp_out, QEntry* q,
                                                       unsigned long long* ctr, uint32_t* chg0,
                                                       unsigned long long* count, const uint32_t* bk_end,
                                                       int C) {
    cover_seed_block(M, J, s, rp_out, q, ctr, chg0, count, bk_end, C);
}

cudaError_t launch_cover_seed(uint8_t* M, int J, int32_t s, const int32_t* rp_out, QEntry* q,
                              unsigned long long* ctr, uint32_t* chg0, unsigned long long* count,
                              const uint32_t* bk_end, int C, cudaStream_t st) {
    k_cover_seed<<<1, kBlock, 0, st>>>(M, J, s, rp_out, q, ctr, chg0, count, bk_end, C);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_sums(const uint8_t* __restrict__ M, int32_t n, int J,
                                                 unsigned long long* __restrict__ S) {
    const int cpr = J >> 4;
    const int lpr = cpr < 32 ? cpr : 32;
    const int cpl = cpr / lpr;
    const int rpw = 32 / lpr;
    const int lane = (int)lane_id();
    const int seg = lane / lpr, seg_lane = lane % lpr;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * rpw; r0 < n; r0 += nwarps * rpw) {
        const int64_t row = r0 + seg;
        const bool ok = row < n;
        const unsigned long long s = row_sum(M, J, ok ? (int32_t)row : 0, lpr, cpl, seg_lane);
        if (ok && seg_lane == 0) S[row] = s;
    }
}

cudaError_t launch_sums(const uint8_t* M, int32_t n, int J, unsigned long long* S, cudaStream_t st) {
    k_sums<<<pick_grid(n, J), kBlock, 0, st>>>(M, n, J, S);
    return cudaGetLastError();
}

__global__ void k_count_visited(const uint8_t* __restrict__ M, int64_t words16,
                                unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words16;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(M) + i);
        c += (__popc(visited_bytes(q.x)) + __popc(visited_bytes(q.y)) + __popc(visited_bytes(q.z)) +
              __popc(visited_bytes(q.w))) >> 3;
    }
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_count_visited(const uint8_t* M, int64_t bytes, unsigned long long* out,
                                 cudaStream_t st) {
    const int64_t w = bytes / 16;
    if (w == 0) return cudaSuccess;
    int64_t grid = (w + kBlock - 1) / kBlock;
    if (grid > 152 * 8) grid = 152 * 8;
    k_count_visited<<<(int)grid, kBlock, 0, st>>>(M, w, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Graph load: in-degrees, scan, reverse CSR, thresholds, the all-vertex queue.
// ---------------------------------------------------------------------------
__global__ void k_indegree(const int32_t* __restrict__ col, int64_t m, int32_t* cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[e], 1);
}

cudaError_t launch_indegree(const int32_t* col, int64_t m, int32_t* cnt, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_indegree<<<152 * 8, kBlock, 0, st>>>(col, m, cnt);
    return cudaGetLastError();
}

constexpr int kScanTile = 2048;  // elements per block (256 threads x 8)

__global__ void k_scan_tiles(const int32_t* __restrict__ in, int32_t n, int32_t* __restrict__ out,
                             int64_t* __restrict__ tile_sums) {
    __shared__ int64_t warp_tot[kWarpsPerBlock];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 8;
    int32_t v[8];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        local += v[i];
    }
    const int lane = (int)lane_id(), w = threadIdx.x >> 5;
    int64_t incl = local;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, s);
        if (lane >= s) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    int64_t wbase = 0;
    for (int i = 0; i < w; ++i) wbase += warp_tot[i];
    int64_t run = wbase + incl - local;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (base + i < n) out[base + i] = (int32_t)run;  // tile-local exclusive prefix
        run += v[i];
    }
    if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = wbase + incl;
}

// Exclusive scan of the tile sums in place (one block of kScanSumThreads:
// each thread scans a contiguous run of tiles), the 32-bit total into
// *out_total_slot and the exact 64-bit total into tile_sums[ntiles].
constexpr int kScanSumThreads = 1024;
__global__ void __launch_bounds__(kScanSumThreads) k_scan_sums(int64_t* tile_sums, int ntiles, int32_t* out_total_slot) {
    __shared__ int64_t part[kScanSumThreads];
    const int t = threadIdx.x;
    const int per = (ntiles + kScanSumThreads - 1) / kScanSumThreads;
    const int b = min(ntiles, t * per), e = min(ntiles, b + per);
    int64_t run = 0;
    for (int i = b; i < e; ++i) run += tile_sums[i];
    part[t] = run;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread totals
    for (int off = 1; off < kScanSumThreads; off <<= 1) {
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t acc = part[t] - run;  // exclusive prefix of this thread's run
    for (int i = b; i < e; ++i) {
        const int64_t x = tile_sums[i];
        tile_sums[i] = acc;
        acc += x;
    }
    if (t == kScanSumThreads - 1) {
        *out_total_slot = (int32_t)part[t];
        tile_sums[ntiles] = part[t];  // the exact 64-bit total
    }
}

__global__ void k_scan_add(int32_t* __restrict__ out, int32_t n, const int64_t* __restrict__ tile_sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += (int32_t)tile_sums[i / kScanTile];
}

size_t scan_tmp_bytes(int32_t n) {
    const int64_t tiles = ((int64_t)n + kScanTile - 1) / kScanTile;
    return (size_t)(tiles + 1) * sizeof(int64_t);
}

cudaError_t launch_exclusive_scan(const int32_t* cnt, int32_t n, int32_t* out, void* tmp,
                                  cudaStream_t st) {
    const int ntiles = (int)(((int64_t)n + kScanTile - 1) / kScanTile);
    int64_t* sums = static_cast<int64_t*>(tmp);
    if (ntiles > 0) k_scan_tiles<<<ntiles, kBlock, 0, st>>>(cnt, n, out, sums);
    k_scan_sums<<<1, kScanSumThreads, 0, st>>>(sums, ntiles, out + n);
    if (n > 0) k_scan_add<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(out, n, sums);
    return cudaGetLastError();
}

// Static queue of every vertex with in-edges (rp = the in-CSR) or out-edges
// (rp = the out-CSR), in vertex order (dense levels): entry k is the k-th such
// vertex, its flat-space offset is its row start; aux = thr_v (may be NULL).
__global__ void k_flag_in(const int32_t* __restrict__ rp_in, int32_t n, int32_t* flag) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flag[v] = rp_in[v + 1] > rp_in[v] ? 1 : 0;
}

__global__ void k_dense_queue(const int32_t* __restrict__ rp_in, int32_t n, const uint32_t* __restrict__ thr_v,
                              const int32_t* __restrict__ pos, QEntry* __restrict__ q) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t b = rp_in[v], e = rp_in[v + 1];
    if (e > b) {
        QEntry x;
        x.v = (int32_t)v; x.rp = b; x.off = b; x.aux = thr_v ? thr_v[v] : 0u;
        q[pos[v]] = x;
    }
}

cudaError_t launch_dense_queue(const int32_t* rp_in, int32_t n, const uint32_t* thr_v, int32_t* flag,
                               int32_t* pos, void* scan_tmp, QEntry* q, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_flag_in<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(rp_in, n, flag);
    cudaError_t e = launch_exclusive_scan(flag, n, pos, scan_tmp, st);
    if (e != cudaSuccess) return e;
    k_dense_queue<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(rp_in, n, thr_v, pos, q);
    return cudaGetLastError();
}

// Weighted cascade (Sec. 2.1): w = 1/indeg(v) rounded to fp32 (IEEE division),
// threshold floor(w * 2^31) computed exactly in fp64.
__device__ __forceinline__ uint32_t prob_threshold_dev(float w) {
    const double t = floor((double)w * 2147483648.0);
    if (!(t > 0.0)) return 0u;
    if (t >= 2147483648.0) return 2147483648u;
    return (uint32_t)t;
}

__global__ void k_thr_wc(const int32_t* __restrict__ rp_in, int32_t n, uint32_t* __restrict__ thr_v) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t d = rp_in[v + 1] - rp_in[v];
    thr_v[v] = d > 0 ? prob_threshold_dev(__fdiv_rn(1.0f, (float)d)) : 0u;
}

cudaError_t launch_thr_wc(const int32_t* rp_in, int32_t n, uint32_t* thr_v, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_thr_wc<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(rp_in, n, thr_v);
    return cudaGetLastError();
}

__global__ void k_thr_explicit(const float* __restrict__ w, int64_t m, uint32_t* __restrict__ thr) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        thr[e] = prob_threshold_dev(w[e]);
}

cudaError_t launch_thr_explicit(const float* w, int64_t m, uint32_t* thr, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_thr_explicit<<<152 * 8, kBlock, 0, st>>>(w, m, thr);
    return cudaGetLastError();
}

}  // namespace im

namespace im {

// ---------------------------------------------------------------------------
// Independent-cascade Monte-Carlo spread (the paper's independent quality
// oracle, Sec. 5.1, on the GPU).  In simulation r, out-edge e fires iff
// (SplitMix64 output r*m + e of the coin stream) >> 33 < thr[e]; an edge is
// tried once per simulation, when its source is first reached.  One frontier
// level walks the out-edges of the vertices newly reached at the previous
// level; lanes own 32-simulation words and flip coins only for simulations
// in which the source is new.
// ---------------------------------------------------------------------------
__global__ void k_mc_seed(McArgs a, const int32_t* __restrict__ seeds, int k, int valid,
                          const int32_t* __restrict__ rp_out) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int32_t s = seeds[i];
        for (int w = 0; w < a.words; ++w) {
            const int lo = w * 32;
            uint32_t mask = 0u;
            if (valid >= lo + 32) mask = 0xFFFFFFFFu;
            else if (valid > lo) mask = (1u << (valid - lo)) - 1u;
            a.vis[(size_t)s * a.words + w] = mask;
            a.f_next[(size_t)s * a.words + w] = mask;  // new bits of level 0
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int32_t s = seeds[i];
        if (atomicExch(a.gen + s, a.gen_next) == a.gen_next) continue;
        const int32_t rp = rp_out[s], deg = rp_out[s + 1] - rp;
        if (deg <= 0) continue;
        const unsigned long long base =
            atomicAdd(a.ctr_out, (1ull << kCountShift) | (unsigned long long)deg);
        QEntry e;
        e.v = s; e.rp = rp; e.off = (int32_t)(base & kEdgeMask); e.aux = 0;
        a.q_out[base >> kCountShift] = e;
    }
}

cudaError_t launch_mc_seed(const GraphDev& g, const McArgs& a, const int32_t* seeds, int k,
                           int valid, cudaStream_t st) {
    k_mc_seed<<<1, kBlock, 0, st>>>(a, seeds, k, valid, g.rp_out);
    return cudaGetLastError();
}

template <int KIND>
__global__ void __launch_bounds__(kBlock) k_mc_level(GraphDev g, McArgs a) {
    const int lane = (int)lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int words = a.words;
    // clear the new-bits of the level before the previous one (no one reads them now)
    if (a.q_prev) {
        const int32_t cp = (int32_t)(__ldcg(a.ctr_prev) >> kCountShift);
        for (int64_t i = warp; i < cp; i += nwarps) {
            const int32_t u = __ldcg(&a.q_prev[i].v);
            if (lane < words) a.f_prev[(size_t)u * words + lane] = 0u;
        }
    }
    const unsigned long long c = __ldcg(a.ctr_in);
    const int32_t count = (int32_t)(c >> kCountShift);
    const int64_t E = (int64_t)(c & kEdgeMask);
    if (E == 0) return;
    const int64_t nb = (E + 31) >> 5;
    const int64_t per = (nb + nwarps - 1) / nwarps;
    const int64_t b0 = warp * per;
    const int64_t b1 = min(nb, b0 + per);
    if (b0 >= b1) return;
    const int64_t fend = min(E, b1 << 5);
    int64_t f0 = b0 << 5;
    int32_t qi = find_covering(a.q_in, count, f0);
    for (; f0 < fend; f0 += 32) {
        const int32_t wi = qi + lane;
        const bool wvalid = wi < count;
        QEntry ent;
        if (wvalid) {
            const int4 raw = __ldcg(reinterpret_cast<const int4*>(a.q_in) + wi);
            ent.v = raw.x; ent.rp = raw.y; ent.off = raw.z; ent.aux = (uint32_t)raw.w;
        } else {
            ent.v = 0; ent.rp = 0; ent.off = 0x7FFFFFFF; ent.aux = 0;
        }
        const int64_t rel = (int64_t)ent.off - f0;
        const int c0 = __popc(__ballot_sync(0xFFFFFFFFu, wvalid && rel <= 0));
        const unsigned starts =
            __reduce_or_sync(0xFFFFFFFFu, (wvalid && rel >= 1 && rel <= 31) ? (1u << rel) : 0u);
        const int myw = c0 - 1 + __popc(starts & ((2u << lane) - 1u));
        const int32_t qv = __shfl_sync(0xFFFFFFFFu, ent.v, myw);
        const int32_t qrp = __shfl_sync(0xFFFFFFFFu, ent.rp, myw);
        const int32_t qoff = __shfl_sync(0xFFFFFFFFu, ent.off, myw);
        const int64_t f = f0 + lane;
        const int nact = (int)min((int64_t)32, fend - f0);
        int64_t e = 0;
        int32_t o = 0;
        uint32_t thr = 0;
        if (lane < nact) {
            e = (int64_t)qrp + (f - qoff);
            o = __ldg(g.col_out + e);
            thr = edge_threshold<KIND, false>(g, (uint32_t)qv, (uint32_t)o, e, 0u);
        }
        for (int i = 0; i < nact; ++i) {
            const int32_t u_i = __shfl_sync(0xFFFFFFFFu, qv, i);
            const int32_t o_i = __shfl_sync(0xFFFFFFFFu, o, i);
            const int64_t e_i = __shfl_sync(0xFFFFFFFFu, e, i);
            const uint32_t t_i = __shfl_sync(0xFFFFFFFFu, thr, i);
            bool changed = false;
            if (lane < words && t_i > 0u) {
                uint32_t bits = __ldcg(a.f_cur + (size_t)u_i * words + lane);
                uint32_t live = 0u;
                while (bits) {
                    const int b = __ffs((int)bits) - 1;
                    bits &= bits - 1u;
                    const uint64_t r = (uint64_t)a.r0 + (uint64_t)(lane * 32 + b);
                    const uint32_t coin = (uint32_t)(splitmix_at(a.seed, r * (uint64_t)a.m + (uint64_t)e_i) >> 33);
                    if (coin < t_i) live |= 1u << b;
                }
                if (live) {
                    uint32_t* vw = a.vis + (size_t)o_i * words + lane;
                    const uint32_t cand = live & ~__ldcg(vw);
                    if (cand) {
                        const uint32_t really = cand & ~atomicOr(vw, cand);
                        if (really) {
                            atomicOr(a.f_next + (size_t)o_i * words + lane, really);
                            changed = true;
                        }
                    }
                }
            }
            if (__ballot_sync(0xFFFFFFFFu, changed) && lane == 0) {
                if (atomicExch(a.gen + o_i, a.gen_next) != a.gen_next) {
                    const int32_t rp = __ldg(g.rp_out + o_i), deg = __ldg(g.rp_out + o_i + 1) - rp;
                    if (deg > 0) {
                        const unsigned long long base =
                            atomicAdd(a.ctr_out, (1ull << kCountShift) | (unsigned long long)deg);
                        QEntry x;
                        x.v = o_i; x.rp = rp; x.off = (int32_t)(base & kEdgeMask); x.aux = 0;
                        a.q_out[base >> kCountShift] = x;
                    }
                }
            }
        }
        const int n32 = __popc(__ballot_sync(0xFFFFFFFFu, wvalid && rel <= 32));
        int32_t qn = qi + n32 - 1;
        if (n32 == 32 && qi + 32 < count) {
            if ((int64_t)__ldcg(&a.q_in[qi + 32].off) <= f0 + 32) qn = qi + 32;
        }
        qi = qn;
    }
}

cudaError_t launch_mc_level(int kind, const GraphDev& g, const McArgs& a, int grid, cudaStream_t st) {
    switch (kind) {
        case kUniform: k_mc_level<kUniform><<<grid, kBlock, 0, st>>>(g, a); break;
        case kWC: k_mc_level<kWC><<<grid, kBlock, 0, st>>>(g, a); break;
        case kTrivalency: k_mc_level<kTrivalency><<<grid, kBlock, 0, st>>>(g, a); break;
        default: k_mc_level<kExplicit><<<grid, kBlock, 0, st>>>(g, a); break;
    }
    return cudaGetLastError();
}

// Per-simulation reach sizes: reach[32 w + b] += number of vertices with bit b of word w set.
__global__ void __launch_bounds__(kBlock) k_mc_count(const uint32_t* __restrict__ vis, int32_t n,
                                                     int words, unsigned long long* reach) {
    __shared__ unsigned int sh[kMaxJ];
    for (int i = threadIdx.x; i < words * 32; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const int w = threadIdx.x % words;
    const int rpb = blockDim.x / words;
    unsigned int cnt[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) cnt[b] = 0u;
    for (int64_t u = (int64_t)blockIdx.x * rpb + threadIdx.x / words; u < n; u += (int64_t)gridDim.x * rpb) {
        const uint32_t x = __ldg(vis + (size_t)u * words + w);
#pragma unroll
        for (int b = 0; b < 32; ++b) cnt[b] += (x >> b) & 1u;
    }
#pragma unroll
    for (int b = 0; b < 32; ++b)
        if (cnt[b]) atomicAdd(&sh[w * 32 + b], cnt[b]);
    __syncthreads();
    for (int i = threadIdx.x; i < words * 32; i += blockDim.x)
        if (sh[i]) atomicAdd(reach + i, (unsigned long long)sh[i]);
}

cudaError_t launch_mc_count(const uint32_t* vis, int32_t n, int words, unsigned long long* reach,
                            cudaStream_t st) {
    k_mc_count<<<152 * 4, kBlock, 0, st>>>(vis, n, words, reach);
    return cudaGetLastError();
}

__global__ void k_mc_reduce(const unsigned long long* __restrict__ reach, int valid,
                            unsigned long long* acc) {
    unsigned long long s = 0, q = 0;
    for (int r = threadIdx.x; r < valid; r += blockDim.x) {
        const unsigned long long x = reach[r];
        s += x;
        q += x * x;
    }
    s = warp_sum(s);
    q = warp_sum(q);
    if (lane_id() == 0) {
        atomicAdd(acc, s);
        atomicAdd(acc + 1, q);
    }
}

cudaError_t launch_mc_reduce(const unsigned long long* reach, int valid, unsigned long long* acc,
                             cudaStream_t st) {
    k_mc_reduce<<<1, kBlock, 0, st>>>(reach, valid, acc);
    return cudaGetLastError();
}

}  // namespace im

namespace im {

// ---------------------------------------------------------------------------
// Graph load: LSD radix sort (8-bit digits, stable) of 64-bit keys carrying a
// 32-bit payload.  Used once per graph to build the in-CSR sorted by
// (target, class, edge hash).
// ---------------------------------------------------------------------------
constexpr int kSortItems = 8;
constexpr int kSortTile = kBlock * kSortItems;  // 2048 keys per block (24 KB of them in shared memory)

__global__ void __launch_bounds__(kBlock) k_sort_hist(const unsigned long long* __restrict__ keys,
                                                      int64_t n, int shift, int nblocks,
                                                      int32_t* __restrict__ hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + (int64_t)r * kBlock + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = (int32_t)h[threadIdx.x];
}

// Scatter of one pass: the tile's keys are first ranked stably by digit
// (rounds of 256 keys in index order; inside a round, warps in order, lanes of
// a digit by __match_any_sync) and placed in shared memory in digit order,
// then written out from there: consecutive threads write a digit's keys to
// consecutive global positions (runs of about kSortTile / 256 keys instead of
// one key per store).
__global__ void __launch_bounds__(kBlock) k_sort_scatter(
    const unsigned long long* __restrict__ keys, const int32_t* __restrict__ vals, int64_t n, int shift,
    int nblocks, const int32_t* __restrict__ hist, const int32_t* __restrict__ offs,
    unsigned long long* __restrict__ keys_out, int32_t* __restrict__ vals_out) {
    __shared__ unsigned long long sk[kSortTile];
    __shared__ int32_t sv[kSortTile];
    __shared__ unsigned int wcount[kWarpsPerBlock][256];
    __shared__ unsigned int run[256];    // keys of the digit placed so far (tile order)
    __shared__ unsigned int start[256];  // first tile position of the digit
    __shared__ unsigned int gbase[256];  // global position of the tile's first key of the digit
    const int lane = (int)lane_id(), w = threadIdx.x >> 5;
    const int d0 = threadIdx.x;
    const unsigned cnt_d = (unsigned)hist[(int64_t)d0 * nblocks + blockIdx.x];
    gbase[d0] = (unsigned)offs[(int64_t)d0 * nblocks + blockIdx.x];
    run[d0] = 0u;
    // exclusive scan of the tile's digit counts (one digit a thread)
    start[d0] = cnt_d;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const unsigned x = d0 >= o ? start[d0 - o] : 0u;
        __syncthreads();
        start[d0] += x;
        __syncthreads();
    }
    start[d0] -= cnt_d;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        for (int d = lane; d < 256; d += 32) wcount[w][d] = 0u;
        __syncthreads();
        const int64_t i = base + (int64_t)r * kBlock + threadIdx.x;
        const bool ok = i < n;
        unsigned long long k = 0;
        int32_t v = 0;
        unsigned d = 256u + (unsigned)lane;  // distinct dummy digits for missing keys
        if (ok) {
            k = keys[i];
            v = vals[i];
            d = (unsigned)(k >> shift) & 0xFFu;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const unsigned rank_w = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank_w == 0) wcount[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            unsigned before = 0;
            for (int ww = 0; ww < w; ++ww) before += wcount[ww][d];
            const unsigned pos = start[d] + run[d] + before + rank_w;
            sk[pos] = k;
            sv[pos] = v;
        }
        __syncthreads();
        {
            unsigned tot = 0;
            for (int ww = 0; ww < kWarpsPerBlock; ++ww) tot += wcount[ww][threadIdx.x];
            run[threadIdx.x] += tot;
        }
        __syncthreads();
    }
    const int tile_n = (int)min((int64_t)kSortTile, n - base);
    for (int j = threadIdx.x; j < tile_n; j += kBlock) {
        const unsigned long long k = sk[j];
        const unsigned d = (unsigned)(k >> shift) & 0xFFu;
        const unsigned pos = gbase[d] + (unsigned)j - start[d];
        keys_out[pos] = k;
        vals_out[pos] = sv[j];
    }
}

size_t sort_tmp_bytes(int64_t n) {
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    const int64_t cnt = 256 * (nb > 0 ? nb : 1);
    return 2 * ((size_t)(cnt + 1) * 4 + 256) + scan_tmp_bytes((int32_t)cnt) + 256 +
           ((size_t)n * 8 + 256) + (size_t)n * 4 + 256;
}

// Sort keys of the in-CSR: (target << 33) | (class << 31) | hE(source, target),
// payload = out-edge index.  class = trivalency class (0 for other models).
// Edge-balanced over the out-CSR (a hub's row spreads over many warps, a run
// of small rows shares one warp).
__global__ void k_in_keys(const int32_t* __restrict__ rp_out, const int32_t* __restrict__ col_out,
                          int32_t n, int64_t m, int kind, uint32_t tri_seed, const int32_t* __restrict__ hkey,
                          unsigned long long* __restrict__ keys, int32_t* __restrict__ perm,
                          int32_t* __restrict__ src_out) {
    walk_rows(rp_out, n, m, [&](int64_t i, int32_t u) {
        const uint32_t v = (uint32_t)col_out[i];
        // hash keys: the vertex ids of the graph the edge belongs to
        const uint32_t ku = hkey ? (uint32_t)hkey[u] : (uint32_t)u;
        const uint32_t kv = hkey ? (uint32_t)hkey[v] : v;
        const uint32_t cls = kind == kTrivalency ? hash_pair(ku, kv, tri_seed) % 3u : 0u;
        keys[i] = ((unsigned long long)v << 33) | ((unsigned long long)cls << 31) | edge_hash(ku, kv);
        perm[i] = (int32_t)i;
        src_out[i] = u;
    });
}

// Out-edge hash and weighted-cascade threshold of every out-edge (out-CSR
// order), edge-balanced.
__global__ void k_out_edge_words(const int32_t* __restrict__ rp_out, const int32_t* __restrict__ col_out,
                                 int32_t n, int64_t m, const uint32_t* __restrict__ thr_v,
                                 const int32_t* __restrict__ hkey, uint32_t* __restrict__ h_out,
                                 uint32_t* __restrict__ thrw_out) {
    walk_rows(rp_out, n, m, [&](int64_t i, int32_t u) {
        const uint32_t v = (uint32_t)col_out[i];
        h_out[i] = hkey ? edge_hash((uint32_t)hkey[u], (uint32_t)hkey[v]) : edge_hash((uint32_t)u, v);
        thrw_out[i] = thr_v[v];
    });
}

// CSR validation on the device (graph load), before any kernel indexes by
// the ids: bad[0] = the lowest u with rowptr[u + 1] < rowptr[u]; bad[1] = the
// lowest row holding an id out of [0, n), a self-loop, or an id not above the
// previous one of its row.  Both start at kCsrOk (above any row: n < 2^26).
// The row walk needs a non-decreasing rowptr, so the second kernel returns at
// once after a bad one.
constexpr int32_t kCsrOk = 0x7F7F7F7F;  // the byte 0x7F in every byte (set by a memset)

__global__ void k_check_rowptr(const int32_t* __restrict__ rp, int32_t n, int32_t* __restrict__ bad) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        if (rp[u + 1] < rp[u]) atomicMin(bad, (int32_t)u);
}

__global__ void k_check_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n, int64_t m,
                             int32_t* __restrict__ bad) {
    if (*(volatile int32_t*)bad != kCsrOk) return;
    walk_rows(rp, n, m, [&](int64_t i, int32_t u) {
        const int32_t v = col[i];
        bool b = v < 0 || v >= n || v == u;
        if (!b && i > (int64_t)__ldg(rp + u)) b = col[i - 1] >= v;
        if (b) atomicMin(bad + 1, u);
    });
}

// Blocks of an edge-balanced walk over m positions (kLcmEdgesPerWarp a warp).
static int walk_grid(int64_t m) {
    const int64_t warps = (m + kLcmEdgesPerWarp - 1) / kLcmEdgesPerWarp;
    int64_t grid = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (grid > 152 * 16) grid = 152 * 16;
    return (int)(grid < 1 ? 1 : grid);
}

cudaError_t launch_check_csr(const int32_t* rp, const int32_t* col, int32_t n, int64_t m, int32_t* bad,
                             cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bad, 0x7F, 8, st);  // both words kCsrOk
    if (e != cudaSuccess) return e;
    k_check_rowptr<<<152 * 8, kBlock, 0, st>>>(rp, n, bad);
    if (m > 0) k_check_rows<<<walk_grid(m), kBlock, 0, st>>>(rp, col, n, m, bad);
    return cudaGetLastError();
}

cudaError_t launch_out_edge_words(const int32_t* rp_out, const int32_t* col_out, int32_t n, int64_t m,
                                  const uint32_t* thr_v, const int32_t* hkey, uint32_t* h_out,
                                  uint32_t* thrw_out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_out_edge_words<<<walk_grid(m), kBlock, 0, st>>>(rp_out, col_out, n, m, thr_v, hkey, h_out, thrw_out);
    return cudaGetLastError();
}

__global__ void k_in_gather(const unsigned long long* __restrict__ keys, const int32_t* __restrict__ perm,
                            int64_t m, const int32_t* __restrict__ src_out,
                            const uint32_t* __restrict__ thr_out, int32_t* __restrict__ src_in,
                            uint32_t* __restrict__ h_in, uint32_t* __restrict__ thr_in,
                            int32_t* __restrict__ out_to_in) {
    // four positions a thread per step, their random reads in flight together
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * st < m; i += 4 * st) {
        int32_t e[4], s4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = perm[i + k * st];
#pragma unroll
        for (int k = 0; k < 4; ++k) s4[k] = src_out[e[k]];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t ik = i + k * st;
            src_in[ik] = s4[k];
            h_in[ik] = (uint32_t)keys[ik] & 0x7FFFFFFFu;
            if (thr_in) thr_in[ik] = thr_out[e[k]];
            if (out_to_in) out_to_in[e[k]] = (int32_t)ik;
        }
    }
    for (; i < m; i += st) {
        const int32_t e = perm[i];
        src_in[i] = src_out[e];
        h_in[i] = (uint32_t)keys[i] & 0x7FFFFFFFu;
        if (thr_in) thr_in[i] = thr_out[e];
        if (out_to_in) out_to_in[e] = (int32_t)i;
    }
}

// dst[i] = src[idx[i]] (per-edge words from one CSR orientation to the other)
__global__ void k_gather_u32(const uint32_t* __restrict__ src, const int32_t* __restrict__ idx, int64_t m,
                             uint32_t* __restrict__ dst) {
    // four positions a thread per step, their random reads in flight together
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * st < m; i += 4 * st) {
        int32_t k4[4];
        uint32_t v4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) k4[k] = __ldg(idx + i + k * st);
#pragma unroll
        for (int k = 0; k < 4; ++k) v4[k] = __ldg(src + k4[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[i + k * st] = v4[k];
    }
    for (; i < m; i += st) dst[i] = __ldg(src + __ldg(idx + i));
}

cudaError_t launch_gather_u32(const uint32_t* src, const int32_t* idx, int64_t m, uint32_t* dst, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    // half the resident threads: the first fill runs next to it on the side stream
    k_gather_u32<<<152 * 4, kBlock, 0, st>>>(src, idx, m, dst);
    return cudaGetLastError();
}

// Trivalency class bounds of every in-row from the sorted keys: tri_b[v] =
// (first in-edge of class >= 1, first of class 2), the row end when absent.
__global__ void k_tri_init(const int32_t* __restrict__ rp_in, int32_t n, int2* __restrict__ tri_b) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) tri_b[v] = make_int2(rp_in[v + 1], rp_in[v + 1]);
}

__global__ void k_tri_bounds(const unsigned long long* __restrict__ keys, int64_t m, int2* __restrict__ tri_b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const int32_t v = (int32_t)(k >> 33);
        const int c = (int)((k >> 31) & 3u);
        int pc = -1;  // class of the previous edge of the row (none: row start)
        if (i > 0) {
            const unsigned long long kp = keys[i - 1];
            if ((int32_t)(kp >> 33) == v) pc = (int)((kp >> 31) & 3u);
        }
        // each class boundary of a row is crossed by exactly one edge
        if (pc < 1 && c >= 1) tri_b[v].x = (int32_t)i;
        if (pc < 2 && c >= 2) tri_b[v].y = (int32_t)i;
    }
}

cudaError_t launch_build_in_csr(const int32_t* rp_out, const int32_t* col_out, int32_t n, int64_t m,
                                int kind, uint32_t tri_seed, const int32_t* hkey, const uint32_t* thr_out,
                                int32_t* src_in, uint32_t* h_in,
                                uint32_t* thr_in, int32_t* out_to_in, const int32_t* rp_in, int2* tri_b,
                                void* tmp, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    char* p = static_cast<char*>(tmp);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(p);
    p += ((size_t)m * 8 + 255) & ~(size_t)255;
    int32_t* perm = reinterpret_cast<int32_t*>(p);
    p += ((size_t)m * 4 + 255) & ~(size_t)255;
    int32_t* src_out = reinterpret_cast<int32_t*>(p);
    p += ((size_t)m * 4 + 255) & ~(size_t)255;
    k_in_keys<<<walk_grid(m), kBlock, 0, st>>>(rp_out, col_out, n, m, kind, tri_seed, hkey, keys, perm, src_out);
    int bits = 33;
    while ((1ll << (bits - 33)) < n) ++bits;
    cudaError_t e = launch_radix_sort(keys, perm, m, bits, p, st);
    if (e != cudaSuccess) return e;
    k_in_gather<<<152 * 8, kBlock, 0, st>>>(keys, perm, m, src_out, thr_out, src_in, h_in, thr_in, out_to_in);
    if (kind == kTrivalency && tri_b) {
        k_tri_init<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(rp_in, n, tri_b);
        k_tri_bounds<<<152 * 8, kBlock, 0, st>>>(keys, m, tri_b);
    }
    return cudaGetLastError();
}

size_t build_in_csr_tmp_bytes(int64_t m) {
    return ((size_t)m * 8 + 256) + 2 * ((size_t)m * 4 + 256) + sort_tmp_bytes(m);
}

// Sorts (keys, vals) in place by the key bits [0, bits); tmp >= sort_tmp_bytes(n).
cudaError_t launch_radix_sort(unsigned long long* keys, int32_t* vals, int64_t n, int bits,
                              void* tmp, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    const int cnt = 256 * nb;
    char* p = static_cast<char*>(tmp);
    int32_t* hist = reinterpret_cast<int32_t*>(p);
    p += ((size_t)(cnt + 1) * 4 + 255) & ~(size_t)255;
    int32_t* offs = reinterpret_cast<int32_t*>(p);
    p += ((size_t)(cnt + 1) * 4 + 255) & ~(size_t)255;
    void* scan_tmp = p;
    p += (scan_tmp_bytes(cnt) + 255) & ~(size_t)255;
    unsigned long long* k2 = reinterpret_cast<unsigned long long*>(p);
    p += ((size_t)n * 8 + 255) & ~(size_t)255;
    int32_t* v2 = reinterpret_cast<int32_t*>(p);
    unsigned long long* ka = keys;
    unsigned long long* kb = k2;
    int32_t* va = vals;
    int32_t* vb = v2;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        k_sort_hist<<<nb, kBlock, 0, st>>>(ka, n, shift, nb, hist);
        cudaError_t e = launch_exclusive_scan(hist, cnt, offs, scan_tmp, st);
        if (e != cudaSuccess) return e;
        k_sort_scatter<<<nb, kBlock, 0, st>>>(ka, va, n, shift, nb, hist, offs, kb, vb);
        unsigned long long* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    if (passes & 1) {
        cudaError_t e = cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace im

namespace im {

// ---------------------------------------------------------------------------
// Batches: estimate + argmax of every active graph (Alg. 4 per graph).
// k_batch_tiles: per tile (row range inside one graph) the smallest (S_u, u)
// over rows not picked.  k_batch_graphs: one block per active graph reduces
// its tiles, records the seed and its estimate, marks its row visited (the
// graph's visited counter), and appends it to the cover's level-0 queue.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_batch_tiles(BatchPickArgs a) {
    __shared__ unsigned long long sS[kWarpsPerBlock];
    __shared__ int32_t sU[kWarpsPerBlock];
    const int J = a.J;
    const int cpr = J >> 4;
    const int lpr = cpr < 32 ? cpr : 32;
    const int cpl = cpr / lpr;
    const int rpw = 32 / lpr;
    const int lane = (int)lane_id();
    const int seg = lane / lpr, seg_lane = lane % lpr;
    const int wib = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 T = a.tiles[t];
        unsigned long long bestS = ~0ull;
        int32_t bestU = 0x7FFFFFFF;
        if (a.active[T.x]) {
            for (int64_t r0 = (int64_t)T.y + (int64_t)wib * rpw; r0 < T.z; r0 += (int64_t)kWarpsPerBlock * rpw) {
                const int64_t row = r0 + seg;
                const bool ok = row < T.z;
                const unsigned long long s = row_sum(a.M, J, ok ? (int32_t)row : T.y, lpr, cpl, seg_lane);
                if (ok && seg_lane == 0) {
                    const bool picked = (__ldcg(a.picked + (row >> 5)) >> (row & 31)) & 1u;
                    if (!picked) lex_min(bestS, bestU, s, (int32_t)row);
                }
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long oS = __shfl_xor_sync(0xFFFFFFFFu, bestS, off);
            const int32_t ou = __shfl_xor_sync(0xFFFFFFFFu, bestU, off);
            lex_min(bestS, bestU, oS, ou);
        }
        if (lane == 0) { sS[wib] = bestS; sU[wib] = bestU; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kWarpsPerBlock; ++w) lex_min(bestS, bestU, sS[w], sU[w]);
            a.part_S[t] = bestS;
            a.part_u[t] = bestU;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_batch_graphs(BatchPickArgs a) {
    __shared__ unsigned long long sS[kWarpsPerBlock];
    __shared__ int32_t sU[kWarpsPerBlock];
    __shared__ unsigned long long fS;
    __shared__ int32_t fU;
    __shared__ unsigned int newly_sh;
    const int g = blockIdx.x;
    if (g >= a.G || !a.active[g]) return;
    const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
    unsigned long long bS = ~0ull;
    int32_t bU = 0x7FFFFFFF;
    for (int t = a.tile_begin[g] + threadIdx.x; t < a.tile_end[g]; t += blockDim.x)
        lex_min(bS, bU, __ldcg(a.part_S + t), __ldcg(a.part_u + t));
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long oS = __shfl_xor_sync(0xFFFFFFFFu, bS, off);
        const int32_t ou = __shfl_xor_sync(0xFFFFFFFFu, bU, off);
        lex_min(bS, bU, oS, ou);
    }
    if (lane == 0) { sS[wib] = bS; sU[wib] = bU; }
    __syncthreads();
    const int slot = g * a.maxK + a.round;
    if (threadIdx.x == 0) {
        for (int w = 1; w < kWarpsPerBlock; ++w) lex_min(bS, bU, sS[w], sU[w]);
        fS = bS;
        fU = bU;
        newly_sh = 0u;
        if (bS == ~0ull) {
            a.out_seed[slot] = -1;
        } else {
            a.out_seed[slot] = bU;
            a.out_S[slot] = bS;
            a.out_est[slot] = ((double)a.J * 4294967296.0) / (0.77351 * (double)bS);
            atomicOr(a.picked + (bU >> 5), 1u << (bU & 31));
        }
    }
    __syncthreads();
    if (fS == ~0ull) return;
    // the cover's level 0: the seed's row becomes visited
    const int32_t s = fU;
    const int J = a.J;
    uint8_t* row = a.M + (size_t)s * J;
    const int Jr = (J + 31) & ~31;
    const int words = Jr >> 5;
    unsigned int newly = 0;
    for (int j = threadIdx.x; j < Jr; j += blockDim.x) {
        const bool fresh = j < J && row[j] != kVisited;
        if (fresh) { row[j] = (uint8_t)kVisited; ++newly; }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, fresh);
        if ((j & 31) == 0) a.chg0[(size_t)s * words + (j >> 5)] = bits;
    }
    newly = (unsigned)warp_sum(newly);
    if (lane == 0 && newly) atomicAdd(&newly_sh, newly);
    __syncthreads();
    if (threadIdx.x == 0 && a.bk_end_out) {
        const unsigned int nw = newly_sh;
        if (nw) atomicAdd(a.gcount + g, (unsigned long long)nw);
        if (nw) cover_seed_buckets(s, a.chg0 + (size_t)s * words, a.chunks, a.bk_end_out, a.q_cover, a.ctr_cover);
    } else if (threadIdx.x == 0) {
        const unsigned int nw = newly_sh;
        if (nw) atomicAdd(a.gcount + g, (unsigned long long)nw);
        const int32_t rp = a.rp_out[s];
        const int32_t deg = a.rp_out[s + 1] - rp;
        if (nw && deg > 0) {
            const unsigned long long base =
                atomicAdd(a.ctr_cover, (1ull << kCountShift) | (unsigned long long)deg);
            QEntry e;
            e.v = s; e.rp = rp; e.off = (int32_t)(base & kEdgeMask); e.aux = 0;
            a.q_cover[base >> kCountShift] = e;
        }
    }
}

cudaError_t launch_batch_pick(const BatchPickArgs& a, cudaStream_t st) {
    if (a.ntiles > 0) {
        const int grid = a.ntiles < 152 * 8 ? a.ntiles : 152 * 8;
        k_batch_tiles<<<grid, kBlock, 0, st>>>(a);
    }
    k_batch_graphs<<<a.G, kBlock, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace im
