/*
 * Seeded synthetic graph generators.
 *
 * Input generation only: nothing in this file computes any part of the
 * influence-maximization method (no edge hashes, thresholds, sketches or
 * simulations).  The generated CSR graphs stand in for the SNAP social
 * networks of the paper's evaluation (Sec. 5, Table 2), which are not
 * available here.  Every generator is driven by a counter-based SplitMix64
 * stream (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so its output depends only on the seed and the
 * parameters, never on the number of OpenMP threads.
 *
 * Output format of every generator: CSR of out-edges, rowptr[n+1] (int32),
 * col[m] (int32), rows sorted ascending, no duplicate edges, no self-loops.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define WL_GAMMA 0x9E3779B97F4A7C15ULL

/* k-th output (k >= 0) of the SplitMix64 sequence started from `seed`. */
static inline uint64_t wl_draw(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * WL_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double wl_unit(uint64_t seed, uint64_t k) {
    return (double)(wl_draw(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t* p, int64_t len) {
    if (len < 32) {
        for (int64_t i = 1; i < len; i++) {
            int32_t x = p[i];
            int64_t j = i - 1;
            while (j >= 0 && p[j] > x) { p[j + 1] = p[j]; j--; }
            p[j + 1] = x;
        }
    } else {
        qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Turn an edge list (src[e], dst[e]; dst < 0 = dropped) into a canonical CSR:
 * rows sorted, duplicates and self-loops removed.  Returns m, or -1 on
 * allocation failure.  `col` must hold at least E entries.
 */
static int64_t edges_to_csr(int32_t n, int64_t E, const int32_t* src, const int32_t* dst,
                            int32_t* rowptr, int32_t* col) {
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    if (!start || !fill) { free(start); free(fill); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; e++) {
        if (dst[e] < 0 || dst[e] == src[e]) continue;
        #pragma omp atomic
        start[src[e] + 1]++;
    }
    for (int32_t u = 0; u < n; u++) start[u + 1] += start[u];
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; e++) {
        if (dst[e] < 0 || dst[e] == src[e]) continue;
        int64_t pos;
        #pragma omp atomic capture
        pos = fill[src[e]]++;
        col[start[src[e]] + pos] = dst[e];
    }
    /* sort + dedup each row in place; fill[u] becomes the deduplicated length */
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t u = 0; u < n; u++) {
        int32_t* p = col + start[u];
        int64_t len = start[u + 1] - start[u];
        sort_row(p, len);
        int64_t k = 0;
        for (int64_t i = 0; i < len; i++)
            if (k == 0 || p[i] != p[k - 1]) p[k++] = p[i];
        fill[u] = k;
    }
    /* compact rows (serial: rows only move left) */
    int64_t out = 0;
    rowptr[0] = 0;
    for (int32_t u = 0; u < n; u++) {
        int64_t s = start[u], len = fill[u];
        if (out != s) memmove(col + out, col + s, (size_t)len * sizeof(int32_t));
        out += len;
        rowptr[u + 1] = (int32_t)out;
    }
    free(start);
    free(fill);
    return out;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with 2^scale vertices and
 * `draws` edge draws: each draw descends `scale` levels, choosing the
 * quadrant (src bit, dst bit) = (0,0) w.p. a, (0,1) w.p. b, (1,0) w.p. c,
 * (1,1) w.p. 1-a-b-c, most significant bit first.  No vertex permutation and
 * no noise.  Duplicates and self-loops are removed.  Returns m (< 2^31) or a
 * negative value on error.
 */
int64_t wl_rmat(int32_t scale, int64_t draws, double a, double b, double c, uint64_t seed,
                int32_t* rowptr, int32_t* col) {
    if (scale < 1 || scale > 30 || draws < 0 || draws > 2147483647LL) return -2;
    int32_t n = (int32_t)1 << scale;
    int32_t* src = (int32_t*)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < draws; e++) {
        uint32_t u = 0, v = 0;
        for (int32_t l = 0; l < scale; l++) {
            double r = wl_unit(seed, (uint64_t)e * (uint64_t)scale + (uint64_t)l);
            uint32_t ub = (r >= ab), vb = (r >= a && r < ab) || (r >= abc);
            u = (u << 1) | ub;
            v = (v << 1) | vb;
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
    int64_t m = edges_to_csr(n, draws, src, dst, rowptr, col);
    free(src);
    free(dst);
    return m;
}

/*
 * Directed Erdos-Renyi G(n, m): the first m distinct ordered pairs (u, v),
 * u != v, of a uniform pair stream.  Returns m or a negative value on error.
 */
int64_t wl_erdos_renyi(int32_t n, int64_t m, uint64_t seed, int32_t* rowptr, int32_t* col) {
    if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -2;
    uint64_t cap = 1;
    while (cap < (uint64_t)(2 * m + 16)) cap <<= 1;
    uint64_t* set = (uint64_t*)malloc(cap * sizeof(uint64_t));
    int32_t* src = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!set || !src || !dst) { free(set); free(src); free(dst); return -1; }
    memset(set, 0xFF, cap * sizeof(uint64_t));
    int64_t got = 0;
    for (uint64_t k = 0; got < m; k++) {
        uint64_t z = wl_draw(seed, k);
        uint32_t u = (uint32_t)(((z >> 32) * (uint64_t)n) >> 32);
        uint32_t v = (uint32_t)(((z & 0xFFFFFFFFULL) * (uint64_t)n) >> 32);
        if (u == v) continue;
        uint64_t key = ((uint64_t)u << 32) | v;
        uint64_t h = (key * WL_GAMMA) & (cap - 1);
        int dup = 0;
        while (set[h] != ~0ULL) {
            if (set[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        set[h] = key;
        src[got] = (int32_t)u;
        dst[got] = (int32_t)v;
        got++;
    }
    int64_t out = edges_to_csr(n, m, src, dst, rowptr, col);
    free(set);
    free(src);
    free(dst);
    return out;
}

/*
 * Directed Chung-Lu graph with power-law expected degrees: vertex i has
 * weight w_i = C (i + i0)^(-1/(gamma-1)), with C fixed so that
 * sum_i w_i = n * avg_deg and i0 chosen (with the power sum approximated by
 * its integral) so that w_0 is about sqrt(sum_i w_i).
 * Edge (u, v), u != v, appears independently with probability
 * min(1, w_u w_v / sum w).  Edges of a row are generated by geometric
 * skipping (Miller, Hagberg, "Efficient generation of networks with given
 * expected degrees", WAW 2011), one counter stream per source vertex.
 * Two passes (count, then write) keep the result thread-count independent.
 * Returns m, or a negative value on error (-3: more than cap edges).
 */
static double cl_weight_sum(int32_t n, double alpha, double i0) {
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += pow((double)i + i0, -alpha);
    return s;
}

static int64_t cl_row(int32_t u, int32_t n, const double* w, double S, uint64_t seed,
                      int32_t* out) {
    int64_t cnt = 0;
    uint64_t k = 0, base = (uint64_t)u << 32;
    int32_t v = 0;
    double p = fmin(w[u] * w[0] / S, 1.0);
    while (v < n && p > 0.0) {
        if (p < 1.0) {
            double r = wl_unit(seed, base + k++);
            double skip = floor(log1p(-r) / log1p(-p));
            if (skip >= (double)(n - v)) break;
            v += (int32_t)skip;
        }
        if (v >= n) break;
        double q = fmin(w[u] * w[v] / S, 1.0);
        double r = wl_unit(seed, base + k++);
        if (r < q / p && v != u) {
            if (out) out[cnt] = v;
            cnt++;
        }
        p = q;
        v++;
    }
    return cnt;
}

int64_t wl_chung_lu(int32_t n, double avg_deg, double gamma, uint64_t seed, int32_t* rowptr,
                    int32_t* col, int64_t cap) {
    if (n < 2 || avg_deg <= 0.0 || gamma <= 1.0) return -2;
    double alpha = 1.0 / (gamma - 1.0);
    double target = (double)n * avg_deg;
    /* bisection on i0 with sum_i (i+i0)^-alpha approximated by its integral
     * over [i0 - 1/2, n + i0 - 1/2]; C then comes from the exact sum */
    double lo = 1e-3, hi = (double)n * 4.0;
    for (int it = 0; it < 100; it++) {
        double mid = 0.5 * (lo + hi);
        double a0 = mid - 0.5 > 1e-9 ? mid - 0.5 : 1e-9;
        double sum = (pow((double)n + a0, 1.0 - alpha) - pow(a0, 1.0 - alpha)) / (1.0 - alpha);
        double C = target / sum;
        double w0 = C * pow(mid, -alpha);
        if (w0 * w0 > target) lo = mid; else hi = mid;
    }
    double i0 = hi;
    double C = target / cl_weight_sum(n, alpha, i0);
    double* w = (double*)malloc((size_t)n * sizeof(double));
    int64_t* cnt = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!w || !cnt) { free(w); free(cnt); return -1; }
    double S = 0.0;
    for (int32_t i = 0; i < n; i++) { w[i] = C * pow((double)i + i0, -alpha); S += w[i]; }
    #pragma omp parallel for schedule(dynamic, 256)
    for (int32_t u = 0; u < n; u++) cnt[u] = cl_row(u, n, w, S, seed, NULL);
    int64_t total = 0;
    rowptr[0] = 0;
    for (int32_t u = 0; u < n; u++) {
        total += cnt[u];
        if (total > cap || total > 2147483647LL) { free(w); free(cnt); return -3; }
        rowptr[u + 1] = (int32_t)total;
    }
    #pragma omp parallel for schedule(dynamic, 256)
    for (int32_t u = 0; u < n; u++) cl_row(u, n, w, S, seed, col + rowptr[u]);
    free(w);
    free(cnt);
    return total;
}

/*
 * Per-edge weights for the explicit-probability settings of the paper's
 * evaluation (Sec. 5): kind 0 = N(mean, sd) clipped to [0, 1] (Box-Muller),
 * kind 1 = U(lo, hi).  One counter stream per edge index.
 */
void wl_edge_weights(int64_t m, int32_t kind, double p0, double p1, uint64_t seed, float* w) {
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        double x;
        if (kind == 0) {
            double r1 = wl_unit(seed, 2 * (uint64_t)e), r2 = wl_unit(seed, 2 * (uint64_t)e + 1);
            double g = sqrt(-2.0 * log1p(-r1)) * cos(6.283185307179586 * r2);
            x = p0 + p1 * g;
        } else {
            x = p0 + (p1 - p0) * wl_unit(seed, (uint64_t)e);
        }
        if (x < 0.0) x = 0.0;
        if (x > 1.0) x = 1.0;
        w[e] = (float)x;
    }
}

/* SplitMix64 outputs, exposed so tests can pin the stream the generators use. */
void wl_splitmix_outputs(uint64_t seed, int64_t count, uint64_t* out) {
    for (int64_t k = 0; k < count; k++) out[k] = wl_draw(seed, (uint64_t)k);
}
