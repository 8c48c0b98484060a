// Device-side building blocks of the sketch-based IM hot path (sm_103a).
//
// Hashes (Sec. 2.2 Eq. hash, Sec. 2.3 Eq. sketch-init), the fused-sampling
// live test (Eq. hash_prob), the per-simulation random draws (Sec. 2.2) and
// the byte-level register operations (Eq. sketch-merge with the visited
// marker of Sec. 3.1).  Written for this library from the published
// definitions of MurmurHash3_x86_32 and SplitMix64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace im {

constexpr uint32_t kVisited = 0xFFu;
constexpr int kMaxJ = 1024;
constexpr int kTabBits = 12;                   // range table resolution (top bits of X)
constexpr int kTabSize = (1 << kTabBits) + 1;  // 4097 entries
constexpr int kCountShift = 38;                // packed queue counter: count << 38 | edges
constexpr uint64_t kEdgeMask = (1ull << kCountShift) - 1;
constexpr int kMaxLevels = 16384;              // propagation sweeps / cover levels per phase
constexpr int kCasRetryLimit = 4096;

enum ModelKind : int { kUniform = 0, kWC = 1, kTrivalency = 2, kExplicit = 3,
                       kTargetModel = 4 /* per-target-vertex probability; runs as kWC */ };

// Error bits a kernel may raise (host turns them into IM_E_* codes).
enum : uint32_t { kErrCasLimit = 1u, kErrQueue = 2u, kErrBarrier = 4u, kErrLevels = 8u, kErrBounds = 16u };

// Index checks of the bounds-checked build (compiled with IM_BOUNDS_CHECK, a
// debug variant of the library): an index outside [0, hi) raises kErrBounds
// and is replaced by 0, an index every checked access may use, so the bad
// access is recorded and redirected instead of faulting; the host turns the
// bit into IM_E_STATE.  In the normal build a check is the index itself.
#ifdef IM_BOUNDS_CHECK
template <class T>
__device__ __forceinline__ T chk(T i, int64_t hi, uint32_t* err) {
    if ((int64_t)i < 0 || (int64_t)i >= hi) {
        if (err) atomicOr(err, kErrBounds);
        return (T)0;
    }
    return i;
}
#else
template <class T>
__device__ __forceinline__ T chk(T i, int64_t, uint32_t*) {
    return i;
}
#endif

// Device view of a loaded graph.
struct GraphDev {
    int32_t n;
    int64_t m;
    const int32_t* rp_out;   // n+1, out-CSR row pointers
    const int32_t* col_out;  // m, out-neighbours
    const int32_t* rp_in;    // n+1, in-CSR row pointers
    const int32_t* src_in;   // m, in-neighbours (sources of in-edges), rows sorted by (class, hash)
    const uint32_t* h_in;    // m, edge hash hE(source, target) of every in-edge
    const uint32_t* h_out;   // m, edge hash of every out-edge (out-CSR order)
    const uint32_t* thrw_out;// m, weighted-cascade threshold of every out-edge
    const uint32_t* thr_v;   // kWC: threshold of every edge into v
    const uint32_t* thr_out; // kExplicit: per out-edge threshold
    const uint32_t* thr_in;  // kExplicit: per in-edge threshold
    uint32_t thr_uniform;    // kUniform
    uint32_t tri_seed;       // kTrivalency class-hash seed
    uint32_t tri_thr[3];     // kTrivalency thresholds of the three classes
    // kTrivalency: in-rows are sorted by (class, hash), so the class of in-edge
    // e of row v is (e >= tri_b[v].x) + (e >= tri_b[v].y) (the first in-edges
    // of classes 1 and 2; the row end when a class is absent); used by the
    // once-per-sketch walk over every in-edge (the frontier levels hash: one
    // more load per row cost them more than the hash).  NULL when the rows were
    // sorted under another model than the sketch's.
    const int2* tri_b;
};

// Work-queue entry: a vertex, the start of its edge row in the CSR the phase
// walks, its offset in the phase's flat edge space, and a model word (the
// weighted-cascade threshold of its in-edges for propagation sweeps).  A
// bucket entry holds the bucket, its list start, its offset and a free word
// (the length, or the chunk's 16 bits in queues built at level 0).
struct __align__(16) QEntry {
    int32_t v;
    int32_t rp;
    int32_t off;
    uint32_t aux;
};

// ---------------------------------------------------------------------------
// MurmurHash3_x86_32 pieces (public-domain algorithm by A. Appleby).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rotl32(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

__device__ __forceinline__ uint32_t mm3_k(uint32_t k) {
    k *= 0xcc9e2d51u;
    k = rotl32(k, 15);
    return k * 0x1b873593u;
}

__device__ __forceinline__ uint32_t mm3_h(uint32_t h, uint32_t k) {
    h ^= k;
    h = rotl32(h, 13);
    return h * 5u + 0xe6546b64u;
}

__device__ __forceinline__ uint32_t mm3_final(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    return h ^ (h >> 16);
}

// Hash of the 8-byte key LE32(a) || LE32(b) (the GPU is little-endian, so a
// 4-byte block read of LE32(a) is a itself).
__device__ __forceinline__ uint32_t hash_pair(uint32_t a, uint32_t b, uint32_t seed) {
    return mm3_final(mm3_h(mm3_h(seed, mm3_k(a)), mm3_k(b)) ^ 8u);
}

// Eq. (hash): h(u,v) = Murmur3(u || v) mod 2^31.
__device__ __forceinline__ uint32_t edge_hash(uint32_t u, uint32_t v) {
    return hash_pair(u, v, 0u) & 0x7FFFFFFFu;
}

// Eq. (sketch-init): rank = clz(h_j(u)), h_j = Murmur3 of the 4-byte key u with
// seed salt_j.  `ku` = mm3_k(u), shared by all simulations of a vertex.
__device__ __forceinline__ uint32_t rank_of(uint32_t ku, uint32_t salt) {
    return (uint32_t)__clz((int)mm3_final(mm3_h(salt, ku) ^ 4u));
}

// SplitMix64 output number k (0-based) of the stream started at `seed`
// (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// Edge thresholds of the diffusion models (Sec. 2.1), fixed point of Eq. hash_prob.
// `e` is the edge's index in the CSR the caller walks (out- or in-CSR).
// ---------------------------------------------------------------------------
template <int KIND, bool IN_ORIENTATION>
__device__ __forceinline__ uint32_t edge_threshold(const GraphDev& g, uint32_t u, uint32_t v,
                                                   int64_t e, uint32_t aux) {
    if constexpr (KIND == kUniform) {
        return g.thr_uniform;
    } else if constexpr (KIND == kWC) {
        if constexpr (IN_ORIENTATION) return aux;  // threshold of the queue vertex's in-edges
        else return __ldg(g.thrw_out + e);
    } else if constexpr (KIND == kTrivalency) {
        const uint32_t cls = hash_pair(u, v, g.tri_seed) % 3u;
        return cls == 0u ? g.tri_thr[0] : (cls == 1u ? g.tri_thr[1] : g.tri_thr[2]);
    } else {
        if constexpr (IN_ORIENTATION) return __ldg(g.thr_in + e);
        else return __ldg(g.thr_out + e);
    }
}

// ---------------------------------------------------------------------------
// Candidate simulations of an edge.  With X sorted ascending (Sec. 4.1), the
// simulations in which an edge of hash h and threshold thr can be live form
// one contiguous index range: (X_j ^ h) < thr < 2^(t+1), t = msb(thr), forces
// X_j and h to agree on every bit above t, and the X_j with a given prefix
// are consecutive.  The range is a superset of the live simulations (at
// least half of it is live in expectation); the live test is still applied
// to every simulation in it.  sTab[b] = #{j : X_j < b << 19}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void candidate_range(uint32_t h, uint32_t thr, int J,
                                                const uint32_t* sX, const uint16_t* sTab,
                                                int& lo, int& hi) {
    if (thr == 0u) { lo = hi = 0; return; }
    if (thr >= 0x40000000u) { lo = 0; hi = J; return; }
    const int t = 31 - __clz((int)thr);  // 0..29
    const int L = 30 - t;                // prefix length in bits of a 31-bit value, 1..30
    const uint32_t p = h >> (t + 1);
    if (L <= kTabBits) {
        const int sh = kTabBits - L;
        lo = sTab[p << sh];
        hi = sTab[(p + 1u) << sh];
    } else {
        const uint32_t b = h >> (31 - kTabBits);
        int a = sTab[b];
        const int z = sTab[b + 1];
        while (a < z && (sX[a] >> (t + 1)) < p) ++a;
        int e = a;
        while (e < z && (sX[e] >> (t + 1)) == p) ++e;
        lo = a;
        hi = e;
    }
}

// Live mask of 4 consecutive simulations as bytes (0xFF = live): Eq. (hash_prob).
__device__ __forceinline__ uint32_t live4(uint4 x, uint32_t h, uint32_t thr) {
    return (((x.x ^ h) < thr) ? 0x000000FFu : 0u) | (((x.y ^ h) < thr) ? 0x0000FF00u : 0u) |
           (((x.z ^ h) < thr) ? 0x00FF0000u : 0u) | (((x.w ^ h) < thr) ? 0xFF000000u : 0u);
}

// 0xFF in every byte of x that is a visited register.  Register values are
// <= 32 < 0x80, so bit 7 of a byte marks the visited value 0xFF.
__device__ __forceinline__ uint32_t visited_bytes(uint32_t x) {
    return ((x & 0x80808080u) >> 7) * 0xFFu;
}

// Byte-wise max (Eq. sketch-merge) of a (bytes in [0,32] or 0xFF) and b (bytes
// in [0,32]); a visited byte of a stays 0xFF.  (a|0x80) - b never borrows
// across bytes because every byte of b is below 0x80.
__device__ __forceinline__ uint32_t byte_max(uint32_t a, uint32_t b) {
    const uint32_t ge = (((a | 0x80808080u) - b) & 0x80808080u) >> 7;
    const uint32_t m = ge * 0xFFu;
    return (a & m) | (b & ~m);
}

// 16-byte load that bypasses L1 (registers are updated in place by other SMs).
__device__ __forceinline__ uint4 ld_cg16(const uint8_t* p) {
    return __ldcg(reinterpret_cast<const uint4*>(p));
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Reductions whose result is not needed (change bits, visited marks, counters):
// sent as reductions, so nothing waits for a reply.
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v));
}
__device__ __forceinline__ void red_or64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.or.b64 [%0], %1;" ::"l"(p), "l"(v));
}
// The visited marks of a 16-byte register piece (8-byte aligned halves): two
// reductions at most, none for a half without marks.
__device__ __forceinline__ void red_or_piece(uint8_t* p, const uint32_t m[4]) {
    const unsigned long long lo = (unsigned long long)m[0] | ((unsigned long long)m[1] << 32);
    const unsigned long long hi = (unsigned long long)m[2] | ((unsigned long long)m[3] << 32);
    if (lo) red_or64(reinterpret_cast<unsigned long long*>(p), lo);
    if (hi) red_or64(reinterpret_cast<unsigned long long*>(p + 8), hi);
}
__device__ __forceinline__ void red_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v));
}

// ---------------------------------------------------------------------------
// Edge-balanced walks of a flat space split into rows (CSR edges, queue
// entries): a warp takes kLcmEdgesPerWarp consecutive positions, finds the
// row of the first by a 32-ary search of the row starts, then for each 32
// positions loads the starts of the next 32 rows and every lane picks its row
// among them (a lane whose position lies past those rows, after a run of
// empty rows, searches on its own).
// ---------------------------------------------------------------------------
constexpr int kLcmEdgesPerWarp = 512;

// Last row r in [lo, hi) with start(r) <= e (starts non-decreasing, start(lo) <= e), warp-wide.
template <class S>
__device__ __forceinline__ int32_t row_of_warp(S&& start, int32_t lo, int32_t hi, int64_t e) {
    const int lane = (int)lane_id();
    while (hi - lo > 1) {
        const int32_t step = (hi - lo + 31) >> 5;
        const int64_t idx = (int64_t)lo + (int64_t)step * (lane + 1);
        const bool le = idx < hi && start((int32_t)idx) <= e;
        const int c = __popc(__ballot_sync(0xFFFFFFFFu, le));
        const int32_t nlo = lo + step * c;
        const int32_t nhi = (c < 32) ? (int32_t)min((int64_t)hi, (int64_t)lo + (int64_t)step * (c + 1)) : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Same search by one thread (binary).
template <class S>
__device__ __forceinline__ int32_t row_of_thread(S&& start, int32_t lo, int32_t hi, int64_t e) {
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (start(mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Edge-balanced walk of a flat space [0, m) split into rows by the
// non-decreasing starts start(0..nrows) (start(0) = 0, start(nrows) = m), a
// warp taking kLcmEdgesPerWarp consecutive positions; ALL: every lane calls
// fn(f, row, valid) together, else fn(f, row) once per position.
template <bool ALL, class S, class F>
__device__ __forceinline__ void walk_rows_by(S&& start, int32_t nrows, int64_t m, F&& fn) {
    const int lane = (int)lane_id();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s0 = warp * kLcmEdgesPerWarp; s0 < m; s0 += nwarps * kLcmEdgesPerWarp) {
        const int64_t s1 = min(m, s0 + kLcmEdgesPerWarp);
        int32_t r0 = row_of_warp(start, 0, nrows, s0);
        for (int64_t f0 = s0; f0 < s1; f0 += 32) {
            const int64_t e = f0 + lane;
            // starts of rows r0 .. r0+31 (rows past nrows start after every position)
            const int64_t r = (int64_t)r0 + lane;
            const int64_t beg = r <= nrows ? start((int32_t)r) : INT64_MAX;
            int i = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int64_t b = __shfl_sync(0xFFFFFFFFu, beg, (i + s) & 31);
                if (i + s <= 31 && b <= e) i += s;
            }
            int32_t v = r0 + i;
            // past the 32 rows (a run of empty rows): own search
            if (e < s1 && i == 31 && r0 + 32 <= nrows && start(r0 + 32) <= e)
                v = row_of_thread(start, r0 + 31, nrows, e);
            // the next batch starts in the row of this batch's last position
            r0 = __shfl_sync(0xFFFFFFFFu, v, 31);
            if constexpr (ALL) {
                fn(e, v, e < s1);
            } else {
                if (e >= s1) continue;
                fn(e, v);
            }
        }
    }
}

// Edge-balanced walk of a flat space [0, m) split into rows by the
// non-decreasing starts rp[0..nrows] (rp[0] = 0, rp[nrows] = m): fn(f, row)
// once per position, a warp taking kLcmEdgesPerWarp consecutive positions.
template <class F>
__device__ __forceinline__ void walk_rows(const int32_t* __restrict__ rp, int32_t nrows, int64_t m, F&& fn) {
    walk_rows_by<false>([rp](int32_t r) -> int64_t { return (int64_t)__ldg(rp + r); }, nrows, m, fn);
}

// The same walk with the row starts given by start(r) (start(nrows) = m),
// fn(f, row, valid) called by every lane of the warp together (valid false
// past the end), so fn may use warp-wide operations.
template <class S, class F>
__device__ __forceinline__ void walk_rows_all(S&& start, int32_t nrows, int64_t m, F&& fn) {
    walk_rows_by<true>(start, nrows, m, fn);
}

}  // namespace im
