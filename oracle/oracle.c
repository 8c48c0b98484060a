/*
 * ORACLE — plain, slow CPU implementation of DiFuseR's sketch-based influence
 * maximization (Gokturk & Kaya, arXiv 2410.14047) under the independent
 * cascade model.  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA
 * library, shares no code with it, and only the test suite, the smoke check
 * and the CPU baseline of the benchmark may call it.
 *
 * Conventions (the paper leaves these open; the readings are listed with the
 * design notes of the repository):
 *   hE(u,v)   = MurmurHash3_x86_32(LE32(u) || LE32(v), seed 0) & 0x7FFFFFFF   (Sec. 2.2, Eq. hash)
 *   hV_j(u)   = MurmurHash3_x86_32(LE32(u), seed salt_j)                        (Sec. 2.3, Eq. sketch-init)
 *   r0(u,j)   = clz32(hV_j(u)), clz32(0) = 32                                   (Eq. sketch-init)
 *   thr(u,v)  = floor((double)w_fp32(u,v) * 2^31)                               (Eq. hash_prob, fixed point of Fig. 5)
 *   live(u,v,j) <=> (X_j XOR hE(u,v)) < thr(u,v)                                (Eq. hash_prob)
 *   M[u][j]   in [0,32], or 0xFF = u visited in simulation j                    (Sec. 3.1, Sec. 3.3)
 *   S_u       = sum_j f(M[u][j]), f(r) = 2^(32-r), f(0xFF) = 2^32               (Eq. gpu-sketch-int, exact)
 *   estimate  = J * 2^32 / (phi * S_u), phi = 0.77351                           (Eq. sketch-estimate, Sec. 3.1)
 *
 * Every function names the passage of the paper it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VISITED 0xFFu
#define PHI 0.77351

/* ------------------------------------------------------------------------- */
/* Hash and random-number primitives                                          */
/* ------------------------------------------------------------------------- */

static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

/* MurmurHash3_x86_32 (A. Appleby, public domain description): 4-byte blocks
 * mixed into h, then the 1-3 byte tail, then the length and the final
 * avalanche.  General length; little-endian block reads done byte by byte. */
uint32_t orc_murmur3_32(const uint8_t* key, int64_t len, uint32_t seed) {
    const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
    uint32_t h = seed;
    int64_t nblocks = len / 4;
    for (int64_t i = 0; i < nblocks; i++) {
        const uint8_t* p = key + 4 * i;
        uint32_t k = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                     ((uint32_t)p[3] << 24);
        k *= c1;
        k = rotl32(k, 15);
        k *= c2;
        h ^= k;
        h = rotl32(h, 13);
        h = h * 5u + 0xe6546b64u;
    }
    const uint8_t* tail = key + 4 * nblocks;
    uint32_t k = 0;
    switch (len & 3) {
        case 3: k ^= (uint32_t)tail[2] << 16; /* fall through */
        case 2: k ^= (uint32_t)tail[1] << 8;  /* fall through */
        case 1:
            k ^= (uint32_t)tail[0];
            k *= c1;
            k = rotl32(k, 15);
            k *= c2;
            h ^= k;
    }
    h ^= (uint32_t)len;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static void le32(uint8_t* p, uint32_t x) {
    p[0] = (uint8_t)x; p[1] = (uint8_t)(x >> 8); p[2] = (uint8_t)(x >> 16); p[3] = (uint8_t)(x >> 24);
}

/* Eq. (hash): h(u,v) = Murmur3(u||v) mod 2^31. */
uint32_t orc_edge_hash(int32_t u, int32_t v) {
    uint8_t key[8];
    le32(key, (uint32_t)u);
    le32(key + 4, (uint32_t)v);
    return orc_murmur3_32(key, 8, 0u) & 0x7FFFFFFFu;
}

static int clz32(uint32_t x) {
    if (x == 0) return 32;
    int n = 0;
    while (!(x & 0x80000000u)) { x <<= 1; n++; }
    return n;
}

/* Eq. (sketch-init): M_u[j] = clz(h_j(u)), h_j = Murmur3 of u salted by salt_j. */
int32_t orc_rank(int32_t u, uint32_t salt) {
    uint8_t key[4];
    le32(key, (uint32_t)u);
    return clz32(orc_murmur3_32(key, 4, salt));
}

/* SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden gamma,
 * the output is the state passed through the variant-13 mixer. */
uint64_t orc_splitmix64(uint64_t* state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sec. 2.2 (X_r uniform in [0, h_max]) and Sec. 4.1 (FASST sorts X):
 * draw J pairs (X_j, salt_j) from SplitMix64(seed), X = low 31 bits,
 * salt = high 32 bits, then stable-sort the pairs by X (insertion sort). */
void orc_draw_sims(uint64_t seed, int32_t J, uint32_t* X, uint32_t* salt) {
    uint64_t st = seed;
    for (int32_t j = 0; j < J; j++) {
        uint64_t z = orc_splitmix64(&st);
        X[j] = (uint32_t)(z & 0x7FFFFFFFu);
        salt[j] = (uint32_t)(z >> 32);
    }
    for (int32_t i = 1; i < J; i++) {
        uint32_t x = X[i], s = salt[i];
        int32_t k = i - 1;
        while (k >= 0 && X[k] > x) { X[k + 1] = X[k]; salt[k + 1] = salt[k]; k--; }
        X[k + 1] = x;
        salt[k + 1] = s;
    }
}

/* Fixed-point threshold of a float probability: floor(w * 2^31) clamped to [0, 2^31]. */
uint32_t orc_prob_threshold(float w) {
    double t = floor((double)w * 2147483648.0);
    if (!(t > 0.0)) return 0u;
    if (t >= 2147483648.0) return 2147483648u;
    return (uint32_t)t;
}

/* Sec. 2.1 diffusion models -> per-out-edge thresholds thr[e].
 * kind 0: uniform IC with probability p;
 * kind 1: weighted cascade, w(u,v) = 1/indeg(v) (fp32 division);
 * kind 2: trivalency, w(u,v) = {0.1, 0.01, 0.001}[Murmur3(u||v, seed32) mod 3];
 * kind 3: explicit per-edge probabilities w[e];
 * kind 4: per-target probabilities, w[v] for every edge into v.
 * Returns 0, or -1 on a bad kind. */
int orc_thresholds(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col, int32_t kind,
                   float p, uint64_t model_seed, const float* w, uint32_t* thr) {
    if (kind == 0) {
        uint32_t t = orc_prob_threshold(p);
        for (int64_t e = 0; e < m; e++) thr[e] = t;
        return 0;
    }
    if (kind == 1) {
        int64_t* indeg = (int64_t*)calloc((size_t)n, sizeof(int64_t));
        for (int64_t e = 0; e < m; e++) indeg[col[e]]++;
        for (int64_t e = 0; e < m; e++) thr[e] = orc_prob_threshold(1.0f / (float)indeg[col[e]]);
        free(indeg);
        return 0;
    }
    if (kind == 2) {
        static const float tri[3] = {0.1f, 0.01f, 0.001f};
        uint32_t s32 = (uint32_t)(model_seed ^ (model_seed >> 32));
        for (int32_t u = 0; u < n; u++)
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
                uint8_t key[8];
                le32(key, (uint32_t)u);
                le32(key + 4, (uint32_t)col[e]);
                thr[e] = orc_prob_threshold(tri[orc_murmur3_32(key, 8, s32) % 3u]);
            }
        return 0;
    }
    if (kind == 3) {
        for (int64_t e = 0; e < m; e++) thr[e] = orc_prob_threshold(w[e]);
        return 0;
    }
    if (kind == 4) {
        for (int64_t e = 0; e < m; e++) thr[e] = orc_prob_threshold(w[col[e]]);
        return 0;
    }
    return -1;
}

/* Eq. (hash_prob): edge live in simulation j iff (X_j XOR h) / h_max < w, in fixed point. */
static inline int live(uint32_t Xj, uint32_t h, uint32_t t) { return (Xj ^ h) < t; }

/* ------------------------------------------------------------------------- */
/* Graph helpers                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t n;
    int64_t m;
    const int32_t* rowptr;
    const int32_t* col;
    const uint32_t* thr;  /* per out-edge */
    uint32_t* hash;       /* per out-edge hE */
    int64_t* rrow;        /* reverse CSR: in-edges of each vertex */
    int32_t* rsrc;
    uint32_t* rhash;
    uint32_t* rthr;
} ograph;

static void og_init(ograph* g, int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                    const uint32_t* thr, int with_reverse) {
    g->n = n; g->m = m; g->rowptr = rowptr; g->col = col; g->thr = thr;
    g->hash = (uint32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    for (int32_t u = 0; u < n; u++)
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) g->hash[e] = orc_edge_hash(u, col[e]);
    g->rrow = NULL; g->rsrc = NULL; g->rhash = NULL; g->rthr = NULL;
    if (!with_reverse) return;
    g->rrow = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->rsrc = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    g->rhash = (uint32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    g->rthr = (uint32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    for (int64_t e = 0; e < m; e++) g->rrow[col[e] + 1]++;
    for (int32_t v = 0; v < n; v++) g->rrow[v + 1] += g->rrow[v];
    int64_t* fill = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    for (int32_t u = 0; u < n; u++)
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
            int32_t v = col[e];
            int64_t pos = g->rrow[v] + fill[v]++;
            g->rsrc[pos] = u;
            g->rhash[pos] = g->hash[e];
            g->rthr[pos] = thr[e];
        }
    free(fill);
}

static void og_free(ograph* g) {
    free(g->hash); free(g->rrow); free(g->rsrc); free(g->rhash); free(g->rthr);
}

/* ------------------------------------------------------------------------- */
/* Sketch build (Alg. 1 Fill-Sketches, Alg. 2 Simulate to a fixpoint)         */
/* ------------------------------------------------------------------------- */

/* Alg. 1: every non-visited register gets its vertex's own rank; visited
 * registers (0xFF) are left alone. */
void orc_fill(int32_t n, int32_t J, const uint32_t* salt, uint8_t* M) {
    #pragma omp parallel for schedule(static)
    for (int32_t u = 0; u < n; u++)
        for (int32_t j = 0; j < J; j++)
            if (M[(int64_t)u * J + j] != VISITED) M[(int64_t)u * J + j] = (uint8_t)orc_rank(u, salt[j]);
}

/* O1, brute force from the closed form of the fixpoint: M[u][j] is the
 * largest rank over R*_j(u), the vertices reachable from u along edges live
 * in simulation j without passing through vertices visited in j (u included).
 * One BFS per (u, j); tiny graphs only. */
void orc_build_bruteforce(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                          const uint32_t* thr, int32_t J, const uint32_t* X, const uint32_t* salt,
                          uint8_t* M) {
    ograph g;
    og_init(&g, n, m, rowptr, col, thr, 0);
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* mark = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    uint8_t* out = (uint8_t*)malloc((size_t)n * J);
    for (int32_t i = 0; i < n; i++) mark[i] = -1;
    int32_t stamp = 0;
    for (int32_t j = 0; j < J; j++) {
        for (int32_t u = 0; u < n; u++) {
            uint8_t* o = out + (int64_t)u * J + j;
            if (M[(int64_t)u * J + j] == VISITED) { *o = VISITED; continue; }
            stamp++;
            int32_t head = 0, tail = 0, best = 0;
            queue[tail++] = u;
            mark[u] = stamp;
            while (head < tail) {
                int32_t x = queue[head++];
                int32_t r = orc_rank(x, salt[j]);
                if (r > best) best = r;
                for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) {
                    int32_t y = col[e];
                    if (mark[y] == stamp || M[(int64_t)y * J + j] == VISITED) continue;
                    if (!live(X[j], g.hash[e], thr[e])) continue;
                    mark[y] = stamp;
                    queue[tail++] = y;
                }
            }
            *o = (uint8_t)best;
        }
    }
    memcpy(M, out, (size_t)n * J);
    free(out); free(queue); free(mark);
    og_free(&g);
}

/* O2, the paper's own iteration: Alg. 1 then Alg. 2 repeated until M no
 * longer changes (Alg. 4, "while M not converged").  Synchronous (Jacobi)
 * sweeps: every register pulls max(M_u[j], M_v[j]) from out-neighbours v over
 * edges live in j, reading the previous sweep's values; visited registers of
 * u are skipped and visited registers of v are ignored.  Returns the number
 * of sweeps, the last one changing nothing. */
int32_t orc_build_jacobi(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                         const uint32_t* thr, int32_t J, const uint32_t* X, const uint32_t* salt,
                         uint8_t* M) {
    ograph g;
    og_init(&g, n, m, rowptr, col, thr, 0);
    orc_fill(n, J, salt, M);
    uint8_t* old = (uint8_t*)malloc((size_t)n * J + 1);
    int32_t sweeps = 0;
    int changed = 1;
    while (changed) {
        memcpy(old, M, (size_t)n * J);
        sweeps++;
        changed = 0;
        #pragma omp parallel for schedule(dynamic, 64) reduction(| : changed)
        for (int32_t u = 0; u < n; u++) {
            uint8_t* Mu = M + (int64_t)u * J;
            const uint8_t* Ou = old + (int64_t)u * J;
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
                const uint8_t* Ov = old + (int64_t)col[e] * J;
                for (int32_t j = 0; j < J; j++) {
                    if (Ou[j] == VISITED || Ov[j] == VISITED) continue;
                    if (!live(X[j], g.hash[e], thr[e])) continue;
                    if (Ov[j] > Mu[j]) { Mu[j] = Ov[j]; changed = 1; }
                }
            }
        }
    }
    free(old);
    og_free(&g);
    return sweeps;
}

/* O3, the same closed form as O1 computed per simulation in O(n + m): for
 * r = 32 down to 0, every unassigned non-visited vertex of rank r starts a
 * reverse search over live in-edges through unassigned non-visited vertices,
 * and every vertex it reaches gets the value r.  A vertex first reached at
 * level r reaches a rank-r vertex and no vertex of higher rank (those were
 * all handled at earlier levels, and the assigned set is closed under
 * reverse reachability), so its value is the maximum rank over R*_j(u).
 * Simulations run in parallel (OpenMP), 64 at a time. */
static void reverse_search_sim(const ograph* g, uint32_t Xj, uint32_t saltj, uint8_t* colv,
                               int32_t* queue, int32_t* bucket_next, int32_t* head_of) {
    int32_t n = g->n;
    /* bucket non-visited vertices by rank (linked lists, ascending id) */
    for (int r = 0; r <= 32; r++) head_of[r] = -1;
    for (int32_t u = n - 1; u >= 0; u--) {
        if (colv[u] == VISITED) continue;
        int r = orc_rank(u, saltj);
        bucket_next[u] = head_of[r];
        head_of[r] = u;
        colv[u] = 0xFE; /* unassigned marker (never a valid register value) */
    }
    for (int r = 32; r >= 0; r--) {
        for (int32_t s = head_of[r]; s >= 0; s = bucket_next[s]) {
            if (colv[s] != 0xFE) continue;
            int32_t qh = 0, qt = 0;
            colv[s] = (uint8_t)r;
            queue[qt++] = s;
            while (qh < qt) {
                int32_t x = queue[qh++];
                for (int64_t e = g->rrow[x]; e < g->rrow[x + 1]; e++) {
                    int32_t y = g->rsrc[e];
                    if (colv[y] != 0xFE) continue; /* visited (0xFF) or assigned */
                    if (!live(Xj, g->rhash[e], g->rthr[e])) continue;
                    colv[y] = (uint8_t)r;
                    queue[qt++] = y;
                }
            }
        }
    }
}

void orc_build_reverse(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                       const uint32_t* thr, int32_t J, const uint32_t* X, const uint32_t* salt,
                       uint8_t* M) {
    ograph g;
    og_init(&g, n, m, rowptr, col, thr, 1);
    const int32_t G = 64;
    uint8_t* slab = (uint8_t*)malloc((size_t)G * (size_t)(n > 0 ? n : 1));
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    int32_t* work = (int32_t*)malloc((size_t)nthreads * (2 * (size_t)n + 33) * sizeof(int32_t) + 4);
    for (int32_t j0 = 0; j0 < J; j0 += G) {
        int32_t gs = (J - j0 < G) ? (J - j0) : G;
        for (int32_t u = 0; u < n; u++)
            for (int32_t jj = 0; jj < gs; jj++) slab[(int64_t)jj * n + u] = M[(int64_t)u * J + j0 + jj];
        #pragma omp parallel for schedule(dynamic, 1)
        for (int32_t jj = 0; jj < gs; jj++) {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            int32_t* w = work + (size_t)tid * (2 * (size_t)n + 33);
            reverse_search_sim(&g, X[j0 + jj], salt[j0 + jj], slab + (int64_t)jj * n, w, w + n,
                               w + 2 * (size_t)n);
        }
        for (int32_t u = 0; u < n; u++)
            for (int32_t jj = 0; jj < gs; jj++) M[(int64_t)u * J + j0 + jj] = slab[(int64_t)jj * n + u];
    }
    free(work);
    free(slab);
    og_free(&g);
}

/* ------------------------------------------------------------------------- */
/* Estimate, pick, cover, count (Alg. 3, Alg. 4)                              */
/* ------------------------------------------------------------------------- */

/* Eq. (gpu-sketch-int): the harmonic mean of 2^M[u][j] is J / sum_j 2^-M[u][j];
 * S_u = 2^32 * sum_j 2^-M[u][j] is that denominator in exact fixed point.
 * A visited register counts as 2^32 (the same as rank 0). */
void orc_sums(int32_t n, int32_t J, const uint8_t* M, uint64_t* S) {
    #pragma omp parallel for schedule(static)
    for (int32_t u = 0; u < n; u++) {
        uint64_t s = 0;
        for (int32_t j = 0; j < J; j++) {
            uint8_t r = M[(int64_t)u * J + j];
            s += (r == VISITED) ? (1ULL << 32) : (1ULL << (32 - r));
        }
        S[u] = s;
    }
}

/* Alg. 4 argmax of the estimate = smallest S_u among vertices not yet in the
 * seed set, lowest id on ties.  Returns -1 if every vertex is a seed. */
int32_t orc_pick(int32_t n, const uint64_t* S, const uint8_t* is_seed) {
    int32_t best = -1;
    for (int32_t u = 0; u < n; u++) {
        if (is_seed[u]) continue;
        if (best < 0 || S[u] < S[best]) best = u;
    }
    return best;
}

/* Estimated spread of a seed with denominator S (Eq. sketch-estimate with the
 * harmonic mean of Eq. gpu-sketch-int): J * 2^32 / (phi * S). */
double orc_estimate(int32_t J, uint64_t S) {
    return ((double)J * 4294967296.0) / (PHI * (double)S);
}

/* Alg. 3 / Alg. 4 influence cascade of a new seed s: s is marked visited in
 * every simulation, then each simulation j runs a BFS from s over edges live
 * in j, marking every reached non-visited vertex visited.  Already visited
 * vertices are not expanded: whatever they reach is visited already.
 * Returns the number of registers that became visited. */
uint64_t orc_cover(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                   const uint32_t* thr, int32_t J, const uint32_t* X, uint8_t* M, int32_t s) {
    ograph g;
    og_init(&g, n, m, rowptr, col, thr, 0);
    uint64_t newly = 0;
    #pragma omp parallel reduction(+ : newly)
    {
        int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        #pragma omp for schedule(dynamic, 1)
        for (int32_t j = 0; j < J; j++) {
            if (M[(int64_t)s * J + j] == VISITED) continue;
            M[(int64_t)s * J + j] = VISITED;
            newly++;
            int32_t head = 0, tail = 0;
            queue[tail++] = s;
            while (head < tail) {
                int32_t x = queue[head++];
                for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) {
                    if (!live(X[j], g.hash[e], thr[e])) continue;
                    uint8_t* my = M + (int64_t)col[e] * J + j;
                    if (*my == VISITED) continue;
                    *my = VISITED;
                    newly++;
                    queue[tail++] = col[e];
                }
            }
        }
        free(queue);
    }
    og_free(&g);
    return newly;
}

/* Count(M, -1) of Alg. 4: number of visited registers. */
uint64_t orc_count_visited(int64_t total, const uint8_t* M) {
    uint64_t c = 0;
    for (int64_t i = 0; i < total; i++) c += (M[i] == VISITED);
    return c;
}

/* Error-adaptive rebuild test of Alg. 4 in FP64: (score - oldscore) / score > e,
 * score = count / J.  A negative e disables rebuilds. */
int orc_rebuild_due(uint64_t count, uint64_t oldcount, int32_t J, double e) {
    if (e < 0.0) return 0;
    double score = (double)count / (double)J;
    double oldscore = (double)oldcount / (double)J;
    return (score - oldscore) / score > e;
}

/* Alg. 4 on one device (tau = 0, mu = 1): draw and sort the simulations,
 * build the sketches, then K times: estimate, pick, cover, count, and
 * rebuild when the error-adaptive test fires (never after the last seed).
 * build_mode: 0 = O2 (Jacobi), 1 = O3 (reverse search), 2 = O1 (brute force).
 * Outputs: seeds[K], score[K] (= count/J after each seed), est[K] (estimate of
 * each seed when picked), M (n*J final registers), *rebuilds.
 * Returns 0, or -1 if K > n. */
int orc_select_seeds(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                     const uint32_t* thr, int32_t J, int32_t K, uint64_t seed, double eps,
                     int32_t build_mode, int32_t* seeds, double* score, double* est, uint8_t* M,
                     int32_t* rebuilds) {
    if (K > n) return -1;
    uint32_t* X = (uint32_t*)malloc((size_t)J * sizeof(uint32_t));
    uint32_t* salt = (uint32_t*)malloc((size_t)J * sizeof(uint32_t));
    uint64_t* S = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
    uint8_t* is_seed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    orc_draw_sims(seed, J, X, salt);
    memset(M, 0, (size_t)n * J);
#define ORC_BUILD()                                                                     \
    do {                                                                                \
        if (build_mode == 0) orc_build_jacobi(n, m, rowptr, col, thr, J, X, salt, M);   \
        else {                                                                          \
            orc_fill(n, J, salt, M);                                                    \
            if (build_mode == 1) orc_build_reverse(n, m, rowptr, col, thr, J, X, salt, M); \
            else orc_build_bruteforce(n, m, rowptr, col, thr, J, X, salt, M);           \
        }                                                                               \
    } while (0)
    ORC_BUILD();
    uint64_t count = 0, oldcount = 0;
    int32_t nreb = 0;
    for (int32_t k = 0; k < K; k++) {
        orc_sums(n, J, M, S);
        int32_t s = orc_pick(n, S, is_seed);
        seeds[k] = s;
        est[k] = orc_estimate(J, S[s]);
        is_seed[s] = 1;
        count += orc_cover(n, m, rowptr, col, thr, J, X, M, s);
        score[k] = (double)count / (double)J;
        if (k + 1 < K && orc_rebuild_due(count, oldcount, J, eps)) {
            ORC_BUILD();
            oldcount = count;
            nreb++;
        }
    }
#undef ORC_BUILD
    if (rebuilds) *rebuilds = nreb;
    free(X); free(salt); free(S); free(is_seed);
    return 0;
}

/* Hash-sampled Monte-Carlo spread of a seed set (the influence score of
 * Sec. 5.1 computed with fused sampling): R simulations with X_r drawn from
 * SplitMix64(seed) (low 31 bits), each a BFS from all seeds over edges live
 * in r.  Returns sum_r |reach_r| and sum_r |reach_r|^2 (exact integers). */
void orc_spread_hash(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                     const uint32_t* thr, const int32_t* seeds, int32_t k, int64_t R,
                     uint64_t seed, uint64_t* sum_out, uint64_t* sumsq_out) {
    ograph g;
    og_init(&g, n, m, rowptr, col, thr, 0);
    uint64_t st = seed, sum = 0, sumsq = 0;
    int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    uint8_t* seen = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t r = 0; r < R; r++) {
        uint32_t Xr = (uint32_t)(orc_splitmix64(&st) & 0x7FFFFFFFu);
        memset(seen, 0, (size_t)n);
        int32_t head = 0, tail = 0;
        for (int32_t i = 0; i < k; i++)
            if (!seen[seeds[i]]) { seen[seeds[i]] = 1; queue[tail++] = seeds[i]; }
        while (head < tail) {
            int32_t x = queue[head++];
            for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) {
                int32_t y = col[e];
                if (seen[y] || !live(Xr, g.hash[e], thr[e])) continue;
                seen[y] = 1;
                queue[tail++] = y;
            }
        }
        sum += (uint64_t)tail;
        sumsq += (uint64_t)tail * (uint64_t)tail;
    }
    free(queue); free(seen);
    og_free(&g);
    *sum_out = sum;
    *sumsq_out = sumsq;
}

/* Independent-cascade Monte-Carlo spread of a seed set with independent
 * coins (the "standard RNG" oracle of Sec. 5.1, Sec. 2.1 IC definition):
 * in simulation r, out-edge e (CSR index) fires iff the 31-bit draw
 * c(r, e) = SplitMix64 output number r*m + e of the stream started at
 * `seed`, shifted right by 33, is below thr[e].  Each edge is tried at most
 * once per simulation (when its source first becomes active), so these are
 * exact IC semantics.  Returns sum_r |reach_r| and sum_r |reach_r|^2. */
static uint64_t sm64_at(uint64_t seed, uint64_t k) {
    uint64_t st = seed + k * 0x9E3779B97F4A7C15ULL;
    return orc_splitmix64(&st);
}

void orc_spread_ic(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                   const uint32_t* thr, const int32_t* seeds, int32_t k, int64_t R, uint64_t seed,
                   uint64_t* sum_out, uint64_t* sumsq_out) {
    uint64_t sum = 0, sumsq = 0;
    #pragma omp parallel reduction(+ : sum, sumsq)
    {
        int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        uint8_t* seen = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < R; r++) {
            memset(seen, 0, (size_t)n);
            int32_t head = 0, tail = 0;
            for (int32_t i = 0; i < k; i++)
                if (!seen[seeds[i]]) { seen[seeds[i]] = 1; queue[tail++] = seeds[i]; }
            while (head < tail) {
                int32_t x = queue[head++];
                for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) {
                    int32_t y = col[e];
                    if (seen[y]) continue;
                    uint32_t c = (uint32_t)(sm64_at(seed, (uint64_t)r * (uint64_t)m + (uint64_t)e) >> 33);
                    if (c >= thr[e]) continue;
                    seen[y] = 1;
                    queue[tail++] = y;
                }
            }
            sum += (uint64_t)tail;
            sumsq += (uint64_t)tail * (uint64_t)tail;
        }
        free(queue);
        free(seen);
    }
    *sum_out = sum;
    *sumsq_out = sumsq;
}

/* O1 for one register (full-size spot checks): the largest rank over
 * R*_j(u), by one BFS from u over edges live in simulation j that avoids
 * visited vertices (vis[v] != 0; vis may be NULL).  Returns 0xFF if u itself
 * is visited. */
int32_t orc_register_entry(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                           const uint32_t* thr, uint32_t Xj, uint32_t saltj, const uint8_t* vis,
                           int32_t u) {
    (void)m;
    if (vis && vis[u]) return VISITED;
    int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    int32_t head = 0, tail = 0, best = 0;
    queue[tail++] = u;
    seen[u] = 1;
    while (head < tail) {
        int32_t x = queue[head++];
        int32_t r = orc_rank(x, saltj);
        if (r > best) best = r;
        for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) {
            int32_t y = col[e];
            if (seen[y] || (vis && vis[y])) continue;
            if (!live(Xj, orc_edge_hash(x, y), thr[e])) continue;
            seen[y] = 1;
            queue[tail++] = y;
        }
    }
    free(queue);
    free(seen);
    return best;
}

/* Reach of a seed set in one simulation (Alg. 3 cascade written as a plain
 * BFS): mark[v] = 1 for every vertex reachable from the seeds along edges
 * live in simulation j.  Returns the number of marked vertices. */
int64_t orc_reach_mark(int32_t n, int64_t m, const int32_t* rowptr, const int32_t* col,
                       const uint32_t* thr, uint32_t Xj, const int32_t* seeds, int32_t k,
                       uint8_t* mark) {
    (void)m;
    memset(mark, 0, (size_t)n);
    int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t head = 0, tail = 0;
    for (int32_t i = 0; i < k; i++)
        if (!mark[seeds[i]]) { mark[seeds[i]] = 1; queue[tail++] = seeds[i]; }
    while (head < tail) {
        int32_t x = queue[head++];
        for (int64_t e = rowptr[x]; e < rowptr[x + 1]; e++) {
            int32_t y = col[e];
            if (mark[y] || !live(Xj, orc_edge_hash(x, y), thr[e])) continue;
            mark[y] = 1;
            queue[tail++] = y;
        }
    }
    free(queue);
    return tail;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
