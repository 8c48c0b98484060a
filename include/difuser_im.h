/*
 * difuser_im.h — C ABI of the GB300 (sm_103a) implementation of the
 * single-GPU hot path of DiFuseR's sketch-based influence maximization
 * (Gokturk & Kaya, arXiv 2410.14047) under the independent cascade model.
 *
 * Everything here is plain C: host or device pointers and sizes, no C++ or
 * PyTorch types.  Every call returns an im_status; on error the outputs are
 * left untouched and im_last_error() describes the failure.  All device work
 * of a context runs on the CUDA stream given at im_ctx_create.  The library
 * never calls back into the caller except through the optional allocator.
 *
 * Conventions shared by every entry point (the paper leaves them open):
 *   edge hash      hE(u,v) = MurmurHash3_x86_32(LE32(u)||LE32(v), seed 0) & 0x7FFFFFFF   (Sec. 2.2, Eq. hash)
 *   vertex hash    hV_j(u) = MurmurHash3_x86_32(LE32(u), seed salt_j)                       (Sec. 2.3)
 *   rank           r0(u,j) = clz32(hV_j(u)) in [0,32]                                       (Eq. sketch-init)
 *   threshold      thr(u,v) = floor((double)w_fp32(u,v) * 2^31), w = 1 -> 2^31 (always live)
 *   live test      edge (u,v) live in simulation j iff (X_j XOR hE(u,v)) < thr(u,v)        (Eq. hash_prob)
 *   simulations    (X_j, salt_j), j < J, from SplitMix64(seed): z = next(), X = z & 0x7FFFFFFF,
 *                  salt = z >> 32, stable-sorted by X (Sec. 2.2, Sec. 4.1 FASST sort)
 *   registers      M[u][j] uint8, n x J row-major (a vertex's J registers contiguous, Sec. 3.1);
 *                  value in [0,32], or 0xFF = u visited in simulation j (Sec. 3.1, Sec. 3.3)
 *   estimate sum   S_u = sum_j f(M[u][j]), f(r) = 2^(32-r), f(0xFF) = 2^32, exact uint64
 *                  (harmonic mean of Eq. gpu-sketch-int: H_u = J * 2^32 / S_u)
 *   estimate       e_u = J * 2^32 / (phi * S_u), phi = 0.77351 (Eq. sketch-estimate)
 *
 * Limits: 1 <= n < 2^26, 0 <= m < 2^31, J in {16,32,64,128,256,512,1024}.
 */
#ifndef DIFUSER_IM_H
#define DIFUSER_IM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IM_API __attribute__((visibility("default")))
#else
#define IM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct im_ctx im_ctx;
typedef struct im_graph im_graph;
typedef struct im_sketch im_sketch;

typedef enum {
    IM_OK = 0,
    IM_E_INVAL = -1,   /* bad argument (NULL pointer, malformed CSR, unsupported J) */
    IM_E_RANGE = -2,   /* a size or id out of range (K > n, vertex id >= n, n too large) */
    IM_E_NOMEM = -3,   /* the allocation would exceed the context's HBM budget, or failed */
    IM_E_CUDA = -4,    /* a CUDA runtime call failed; im_last_error() has the CUDA message */
    IM_E_TIMEOUT = -5, /* an iteration bound was exceeded (a loop that should have converged) */
    IM_E_STATE = -6    /* call not valid in the current state (e.g. sketch of another graph) */
} im_status;

typedef enum {
    IM_IC_UNIFORM = 0,    /* every edge has probability p (Sec. 5 settings 0.005, 0.01, 0.1) */
    IM_IC_WC = 1,         /* weighted cascade, w(u,v) = 1 / indeg(v) in fp32 (Sec. 2.1, Fig. 1b) */
    IM_IC_TRIVALENCY = 2, /* w(u,v) = {0.1, 0.01, 0.001}[MurmurHash3_x86_32(LE32(u)||LE32(v),
                             (uint32)(seed ^ seed >> 32)) mod 3] */
    IM_IC_EXPLICIT = 3,   /* per-edge probabilities w[e] in out-CSR order (Sec. 5 N/U settings) */
    IM_IC_TARGET = 4      /* per-target-vertex probabilities w[v], n floats: every edge into v
                             fires with w[v] (weighted cascade is the case w[v] = 1/indeg(v)) */
} im_model_kind;

typedef struct {
    int32_t kind;     /* im_model_kind */
    float p;          /* IM_IC_UNIFORM: edge probability in [0, 1] */
    uint64_t seed;    /* IM_IC_TRIVALENCY: class-hash seed */
    const float* w;   /* IM_IC_EXPLICIT: m host floats in [0, 1], out-CSR order;
                         IM_IC_TARGET: n host floats in [0, 1]; copied */
} im_model;

/* Device memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes (256-byte aligned) usable on `stream`, or NULL; free releases it.
 * Passing NULL to im_ctx_create selects cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} im_allocator;

/* Per-call counters and phase times of the last im_select_seeds /
 * im_sketch_build on a context (device-side counters, CUDA-event times). */
typedef struct {
    double ms_total;          /* whole call, host wall clock */
    double ms_build;          /* sims + fill + propagation of the first build, host wall clock */
    double ms_rebuild;        /* all rebuilds, host wall clock */
    double ms_pick;           /* all pick + cover + score read-back steps, host wall clock */
    double ms_propagate;      /* CUDA-event time of all propagation sweep kernels (timing on) */
    double ms_cover_kernels;  /* CUDA-event time of all cover level kernels and affected-set
                                 searches of incremental rebuilds (timing on) */
    double ms_pick_kernels;   /* CUDA-event time of all estimate + argmax kernels (timing on) */
    double ms_fill_kernels;   /* CUDA-event time of all fill kernels, with the reset and pull of
                                 incremental rebuilds (timing on); a new sketch's first fill
                                 runs on a second stream next to the live chunk masks, so its
                                 time includes that overlap */
    int64_t launches;         /* kernels launched by the call */
    int64_t sweep_launches;   /* propagation sweep kernels launched (with or without work) */
    int64_t builds;           /* 1 + number of rebuilds */
    int64_t sweeps;           /* propagation sweep launches that had work */
    int64_t cover_levels;     /* cover level launches that had work */
    uint64_t sweep_vertices;  /* queue entries processed by all sweeps */
    uint64_t sweep_edges;     /* in-edges examined by all sweeps */
    uint64_t sweep_chunks;    /* (in-edge, 16-simulation chunk) pairs of vertex-format propagation
                                 levels with a simulation where the edge is live, the source
                                 changed and its register is not visited */
    uint64_t sweep_cas;       /* 16-register pieces written by 16-byte CAS (improvements) */
    uint64_t sweep_changed;   /* vertices whose registers a propagation level changed (vertex-format
                                 levels: the queued vertices of every level after the first) */
    uint64_t cover_edges;     /* out-edges examined by cover levels */
    uint64_t cover_chunks;    /* 16-simulation chunks examined by cover levels */
    uint64_t visited;         /* registers visited at the end (Count(M,-1)) */
    uint64_t alg_bytes_sweep; /* bytes the sweeps must move: per queued vertex 16 + J, per
                                 examined in-edge 4 (8 when J = 1024), per in-edge live in a
                                 changed chunk 8 (+4 explicit weights), per live chunk 32,
                                 per CAS 4 */
    uint64_t sweep_heavy;     /* hub vertices pushed by per-simulation hash search */
    uint64_t sweep_heavy_sims;/* (hub, changed simulation) searches */
    uint64_t sweep_batches;   /* 32-edge batches resolved by propagation levels */
    uint64_t sweep_dealt;     /* 16-simulation chunk items dealt (before the live test) */
    uint64_t sweep_edges_live;/* examined in-edges live in a chunk where the source changed */
    uint64_t sweep_buckets;   /* (vertex, chunk) buckets queued for propagation levels */
    uint64_t sweep_bucket_entries; /* bucket list entries processed by propagation levels */
    uint64_t affected;        /* registers recomputed by incremental rebuilds */
    uint64_t pull_buckets;    /* out-buckets queued by the pulls of incremental rebuilds */
    uint64_t pull_entries;    /* out-bucket entries walked by those pulls */
    uint64_t sweep_changed_buckets; /* (vertex, 16-simulation chunk) buckets whose registers a
                                 propagation level changed (bucket-format levels) */
    uint64_t pick_refreshed;  /* rows whose stored S_u lazy picks recomputed */
} im_stats;

/* Schedule knobs of the frontier kernels (chosen by the autotuner; results
 * do not depend on them).  heavy_indeg: in-degree above which a vertex whose
 * in-edges share one threshold below 2^26 (weighted cascade, small uniform p)
 * is pushed by per-simulation hash search instead of an in-edge scan;
 * light_batches: 32-edge batches a warp claims at once; grid_blocks: blocks
 * per frontier launch (0 = SM count x occupancy); check_every: frontier
 * launches between the host's first two emptiness checks (then doubling to 8);
 * persistent: 1 = all levels of a phase in one cooperative launch with grid
 * barriers between levels (per-level launches when tracing); dense_div: a
 * propagation level whose frontier exceeds (vertices with in-edges) /
 * dense_div walks every such vertex in vertex order (0 = never; the first
 * level of a build always does when dense_div > 0); lazy_pick: 1 = in
 * im_select_seeds, picks after the first recompute S_u only for the vertices
 * whose stored S_u (a lower bound: S_u never decreases during a selection)
 * could still beat the best candidate, 0 = every pick reads every row;
 * buckets: b > 0 = each sketch also groups the live (edge, 16-simulation
 * chunk) pairs of every vertex by chunk, with their live masks (at most 4
 * entries per edge, else edge scans only), and a level whose input work (edges
 * or entries) times b is below m queues the changed (vertex, chunk) groups, so
 * that the next level visits only the edges of changed chunks; 0 = edge scans
 * with live chunk masks throughout; incremental: 1 = im_select_seeds rebuilds
 * only the registers a rebuild can change (those of vertices that reach a
 * register visited since the last build) when the sketch has the bucketed
 * lists, 2 = also over edge scans, 0 = full rebuilds; chain: on a bucket
 * level of a propagation or affected-set search with at most one batch per
 * warp, a warp that raises a small bucket (<= 32 entries) queues it, then
 * also processes it at once, up to `chain` such continuations per warp and
 * level (0 = off): chains of small buckets advance several hops a level;
 * pick_tile: the J-tile width of a full estimate + argmax pass, the 16-byte
 * register pieces (16 simulations each) one lane sums per row: 1, 2 or 4
 * (0 = 4); fewer pieces a lane means more lanes per row; dense_out: 1 = a
 * propagation level that walks every vertex (dense_div) records what it raises
 * in the change bits only, without a queue, while the frontier stays large
 * (the next level walks every vertex again), 0 = every level builds a queue;
 * dense_all: bit 0 = such a walk pushes every live simulation of every vertex,
 * changed or not, so what a vertex raised earlier in the same walk moves on
 * at once (clear: only the simulations that changed at the previous level);
 * bit 1 = a cover level that walks every vertex pushes every visited
 * simulation, not only those visited at the previous level (values 0..3). */
typedef struct {
    int32_t heavy_indeg;
    int32_t light_batches;
    int32_t grid_blocks;
    int32_t check_every;
    int32_t persistent;
    int32_t dense_div;
    int32_t lazy_pick;
    int32_t buckets;
    int32_t incremental;
    int32_t chain;
    int32_t pick_tile;
    int32_t dense_out;
    int32_t dense_all;
} im_tuning;

/* One frontier launch of the last selection / build (tracing on). */
typedef struct {
    int32_t kind;    /* 0 = propagation sweep (Alg. 2), 1 = cover level (Alg. 3),
                        2 = affected-set search level (incremental rebuild) */
    int32_t level;   /* level index within its phase */
    int64_t count;   /* queued vertices the launch processed */
    int64_t edges;   /* edges of those vertices (in-edges for sweeps, out-edges for covers) */
    double ms;       /* duration of the level (see im_ctx_set_trace) */
} im_trace_rec;

/* ---- context ----------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream).  `hbm_budget_bytes` caps the device
 * memory the context may hold (0 = no cap).  `alloc` may be NULL.
 * Errors: IM_E_INVAL (out NULL), IM_E_CUDA (no such device). */
IM_API im_status im_ctx_create(int device, void* cuda_stream, uint64_t hbm_budget_bytes,
                        const im_allocator* alloc, im_ctx** out);
IM_API void im_ctx_destroy(im_ctx* ctx);
/* Bytes currently held / the high-water mark of a context. */
IM_API uint64_t im_ctx_bytes_in_use(const im_ctx* ctx);
IM_API uint64_t im_ctx_bytes_peak(const im_ctx* ctx);
/* Message of the last error on this context ("" if none); valid until the next call. */
IM_API const char* im_last_error(const im_ctx* ctx);
IM_API const char* im_status_str(im_status s);
/* Counters of the last selection / build (see im_stats). */
IM_API im_status im_last_stats(const im_ctx* ctx, im_stats* out);
/* enable != 0: bracket every kernel launch with CUDA events on the context's
 * stream and report per-kind kernel time in im_stats (adds two event records
 * per launch).  Off by default. */
IM_API im_status im_ctx_set_timing(im_ctx* ctx, int enable);
/* Sets (NULL = defaults {256, 4, 0, 2, 1, 0, 1, 2, 1, 8, 4, 1, 0}) or reads the schedule knobs. */
IM_API im_status im_ctx_set_tuning(im_ctx* ctx, const im_tuning* tuning);
IM_API im_status im_ctx_get_tuning(const im_ctx* ctx, im_tuning* tuning);
/* Bounds of the waits inside the device code, so that a loop that should end
 * but does not returns IM_E_TIMEOUT instead of holding the GPU:
 * barrier_wait_ns bounds every wait of a block at the grid barrier between
 * two levels of a phase (all levels of a build or a cover run in one
 * cooperative launch); a block that waits longer raises an abort word, every
 * block leaves the launch at its next barrier, and the call returns
 * IM_E_TIMEOUT (0: a block that has to wait at all gives up at once).
 * max_levels bounds the levels of one phase (propagation to the fixpoint,
 * one cover, one affected-set search): a frontier still non-empty after
 * max_levels levels ends the phase with IM_E_TIMEOUT.  Defaults: 2 s and
 * 16382 levels (the most a phase can record).  After IM_E_TIMEOUT the
 * context stays usable; the sketch of the failed call is released (or, for
 * step-level calls, must be rebuilt).  Errors: IM_E_INVAL (max_levels outside
 * [1, 16382]). */
IM_API im_status im_ctx_set_limits(im_ctx* ctx, uint64_t barrier_wait_ns, int32_t max_levels);
/* enable != 0: also keep one im_trace_rec per frontier level (implies timing):
 * its duration comes from CUDA events around the level's launch, or, when a
 * phase runs all its levels in one launch, from the device's global timer
 * read at every level boundary. */
IM_API im_status im_ctx_set_trace(im_ctx* ctx, int enable);
/* Copies up to `cap` trace records of the last selection / build into `out`
 * (may be NULL to query); returns the number of records available. */
IM_API int64_t im_last_trace(const im_ctx* ctx, im_trace_rec* out, int64_t cap);

/* ---- graph ------------------------------------------------------------- */

/* Copies a directed graph (CSR of out-edges: rowptr[n+1], col[m], host
 * int32, rows sorted ascending, no duplicate edges, no self-loops: parallel
 * edges must be merged beforehand, Sec. 2.1) and a diffusion model to the
 * device, builds the reverse CSR (in-edges) and the edge thresholds
 * (Sec. 2.1 models, Eq. hash_prob fixed point).  The caller keeps ownership of
 * every input.  The CSR is checked on the device right after the upload,
 * before any kernel uses its ids; an error names the lowest bad row (its first
 * bad edge).  Errors: IM_E_INVAL (malformed CSR or model: rowptr decreasing
 * or not from 0 to m, a self-loop, a row not strictly ascending), IM_E_RANGE
 * (n or m out of range, an id out of [0, n)), IM_E_NOMEM, IM_E_CUDA. */
IM_API im_status im_graph_load(im_ctx* ctx, int32_t n, int64_t m, const int32_t* rowptr,
                        const int32_t* col, const im_model* model, im_graph** out);
IM_API void im_graph_free(im_graph* g);
/* Size of a loaded graph: *n vertices, *m edges (either pointer may be NULL).
 * Errors: IM_E_INVAL (g NULL). */
IM_API im_status im_graph_info(const im_graph* g, int32_t* n, int64_t* m);

/* ---- sketches (the step-level interface of Alg. 4) ---------------------- */

/* Draws the J simulations (X_j, salt_j) from `seed` (Sec. 2.2, Sec. 4.1),
 * fills the registers with the vertices' own ranks (Alg. 1) and propagates
 * them to the fixpoint of Alg. 2: M[u][j] = max rank over the vertices
 * reachable from u along edges live in simulation j.  Errors: IM_E_INVAL
 * (unsupported J), IM_E_NOMEM, IM_E_CUDA, IM_E_TIMEOUT. */
IM_API im_status im_sketch_build(im_graph* g, int32_t J, uint64_t seed, im_sketch** out);
IM_API void im_sketch_free(im_sketch* sk);
/* Copies the n x J registers to host memory (n*J bytes, row-major). */
IM_API im_status im_sketch_registers(const im_sketch* sk, uint8_t* host_out);
/* Overwrites the registers from host memory (n*J bytes).  For tests: tie and
 * visited-mark injection.  The visited count is recomputed from the bytes. */
IM_API im_status im_sketch_set_registers(im_sketch* sk, const uint8_t* host_in);
/* Copies the sorted simulation parameters X[J], salt[J] to host memory. */
IM_API im_status im_sketch_sims(const im_sketch* sk, uint32_t* X_out, uint32_t* salt_out);
/* Sketchwise-Sum of Alg. 4: S_u for every vertex (exact uint64, host n). */
IM_API im_status im_sketch_sums(const im_sketch* sk, uint64_t* host_out);
/* Estimate + argmax of Alg. 4: the vertex s not yet picked on this sketch with
 * the smallest S_s (largest estimate), lowest id on ties; s becomes picked.
 * *S_out = S_s, *est_out = J * 2^32 / (phi * S_s).  IM_E_RANGE when every
 * vertex is already picked. */
IM_API im_status im_sketch_pick(im_sketch* sk, int32_t* s_out, uint64_t* S_out, double* est_out);
/* Cascade of Alg. 3 / Alg. 4 from vertex s: marks s and every vertex reachable
 * from s along live edges visited (0xFF) in each simulation.  *count_out =
 * Count(M,-1) after the cover.  s need not have been picked. */
IM_API im_status im_sketch_cover(im_sketch* sk, int32_t s, uint64_t* count_out);
/* Rebuild of Alg. 4: Fill-Sketches + Simulate to the fixpoint on the
 * non-visited registers; visited registers are kept. */
IM_API im_status im_sketch_rebuild(im_sketch* sk);

/* ---- the whole method --------------------------------------------------- */

/* Alg. 4 on one device: draws J simulations from `seed`, builds the sketches,
 * then K times picks the vertex of largest estimate (ties -> lowest id),
 * covers it and rebuilds when (score - oldscore) / score > rebuild_eps
 * (score = Count(M,-1)/J, FP64; never after the K-th seed; rebuild_eps < 0
 * disables rebuilds).  `model` = NULL uses the graph's model.
 * Outputs (host): seeds_out[K]; score_out[K] (score after each seed, may be
 * NULL); estimate_out[K] (estimate of each seed when picked, may be NULL);
 * sketch_out (may be NULL) receives the final sketch, which the caller frees.
 * Errors: IM_E_RANGE (K < 1 or K > n), IM_E_INVAL, IM_E_NOMEM, IM_E_CUDA,
 * IM_E_TIMEOUT. */
IM_API im_status im_select_seeds(im_graph* g, int32_t K, int32_t J, const im_model* model,
                          uint64_t seed, double rebuild_eps, int32_t* seeds_out,
                          double* score_out, double* estimate_out, im_sketch** sketch_out);

/* ---- batches: many graphs in one device union ---------------------------- */

typedef struct im_batch im_batch;

/* Loads G graphs (host CSRs, same rules as im_graph_load) as one device batch:
 * a disjoint union with vertex ids offset per graph, graph g under uniform IC
 * with probability p[g].  Errors: IM_E_INVAL, IM_E_RANGE (total vertices must
 * be < 2^26, total edges < 2^31), IM_E_NOMEM, IM_E_CUDA. */
IM_API im_status im_batch_load(im_ctx* ctx, int32_t G, const int32_t* n, const int64_t* m,
                               const int32_t* const* rowptr, const int32_t* const* col,
                               const float* p, im_batch** out);
IM_API void im_batch_free(im_batch* b);
/* Alg. 4 on every graph of the batch at once: graph g gets K[g] seeds with
 * J[g] simulations drawn from `seed` (all graphs share the draws of their J,
 * so each graph's result equals im_select_seeds on that graph alone with the
 * same seed, J, K and rebuild_eps).  Rounds pick one seed in every graph that
 * still needs one; covers of all graphs run as one frontier; rebuilds cover
 * the graphs whose rule fired.  Outputs concatenated in graph order (local
 * vertex ids): seeds_out[sum K], score_out[sum K] (may be NULL),
 * estimate_out[sum K] (may be NULL).  Errors: IM_E_RANGE (K[g] outside
 * [1, n_g]), IM_E_INVAL, IM_E_NOMEM, IM_E_CUDA, IM_E_TIMEOUT. */
IM_API im_status im_batch_select_seeds(im_batch* b, const int32_t* J, const int32_t* K, uint64_t seed,
                                       double rebuild_eps, int32_t* seeds_out, double* score_out,
                                       double* estimate_out);

/* Estimate + argmax without allocating (the paper has no counterpart: this is
 * a library entry point for callers that cannot allocate device memory, such
 * as code running inside a memory arena it does not own or a process whose
 * device memory is fully reserved up front, where a cudaMalloc would fail or
 * stall the device).  Same result as im_sketch_pick on the same registers:
 * the vertex s not marked in `picked` with the smallest S_s (largest
 * estimate), lowest id on ties; its bit in `picked` is set.
 *   M       device, n*J register bytes (row-major, as im_sketch_registers),
 *           16-byte aligned
 *   picked  device, ceil(n/32) uint32 words (4-byte aligned): bit v set =
 *           v excluded; in/out
 *   s_out   device int32 (4-byte aligned): the pick, -1 if every vertex is
 *           excluded
 *   S_out   device uint64 (8-byte aligned): S_s;  est_out: device double
 *           (8-byte aligned), J*2^32/(phi*S_s)
 * Work runs on `cuda_stream` (NULL = legacy default stream); results are
 * ready when the stream reaches them.  Scratch lives in one static device
 * array (at most 1216 blocks of partials, about 15 KB, held by every GPU that
 * loads the library until exit) shared by all calls: calls that overlap on
 * the GPU race and must be serialised by the caller.  The first call on each
 * device looks up the array's address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  Calls no cudaMalloc/cudaFree.
 * Errors (all found on the host, before any launch): IM_E_INVAL (NULL
 * pointer, a buffer below its alignment, unsupported J), IM_E_RANGE (n
 * outside [1, 2^26)), IM_E_CUDA. */
IM_API im_status im_argmax_noalloc(const uint8_t* M, int32_t n, int32_t J, uint32_t* picked,
                                   void* cuda_stream, int32_t* s_out, uint64_t* S_out,
                                   double* est_out);

/* Independent-cascade Monte-Carlo spread of a seed set (the independent
 * quality oracle of Sec. 5.1, run on the GPU): R simulations; in simulation r
 * out-edge e (out-CSR index) fires iff (SplitMix64 output number r*m + e of
 * the stream started at `seed`) >> 33 is below thr[e] — independent coins, each
 * edge tried once per simulation.  *mean_out = mean reach size, *stderr_out =
 * sample standard deviation / sqrt(R); sum_out / sumsq_out (may be NULL)
 * receive the exact sums of reach sizes and squares.  Seeds are host ids.
 * Errors: IM_E_RANGE (bad id, k < 1, R < 2), IM_E_NOMEM, IM_E_CUDA. */
IM_API im_status im_spread_mc(im_graph* g, const int32_t* seeds, int32_t k, int64_t R, uint64_t seed,
                       double* mean_out, double* stderr_out, uint64_t* sum_out,
                       uint64_t* sumsq_out);

/* ---- diagnostics ------------------------------------------------------- */

/* Warp fill rate of the live tests (Sec. 4.1, Table 6 analogue): with the J
 * simulations drawn from `seed` and the model (the graph's, or `model`: uniform
 * / weighted cascade / trivalency), over every in-edge:
 *   counts_out[0] = edges
 *   counts_out[1] = live (edge, simulation) pairs (Eq. hash_prob)
 *   counts_out[2] = 32-simulation warps, in draw order, holding a live pair:
 *                   what a kernel testing every simulation of an edge runs
 *   counts_out[3] = aligned 32-simulation warps, in sorted-X order, holding a
 *                   live pair: what a kernel over the candidate range runs
 *   counts_out[4] = candidate simulations (width of the sorted range)
 * Fill rate = live / (32 * warps).  Errors: IM_E_INVAL, IM_E_STATE (model fixed
 * at load), IM_E_NOMEM, IM_E_CUDA. */
IM_API im_status im_fill_rate(im_graph* g, int32_t J, uint64_t seed, const im_model* model,
                              uint64_t* counts_out);

/* ---- served form: concurrent queries on resident graphs ----------------- */

/* A query server (the paper has none: it serves one query per run).  It keeps
 * graphs resident and runs im_select_seeds queries that arrive at any time:
 * `slots` worker threads, each with its own CUDA stream and stream-ordered
 * memory pool, so the kernels of up to `slots` queries overlap on the device
 * (continuous batching: a query starts as soon as a slot and its device memory
 * are free, while others are running).  Admission control: the resident graphs
 * plus the device bytes reserved by running queries (im_server_query_bytes,
 * an exact upper bound of what a query allocates) never exceed the budget.
 * Pending queries start in arrival order; one that fits may start ahead of an
 * older one that does not, at most `max_bypass` times in a row for that older
 * query.  Each query's result is the one im_select_seeds gives for the same
 * graph and arguments: queries share only the read-only graph. */
typedef struct im_server im_server;

typedef struct {
    int32_t device;             /* CUDA device of the server and its graphs */
    int32_t slots;              /* concurrent queries, 1..64 */
    uint64_t hbm_budget_bytes;  /* resident graphs + running queries; 0 = no limit */
    int32_t max_bypass;         /* >= 0; see above */
} im_server_config;

typedef struct {
    int32_t graph;       /* id from im_server_add_graph */
    int32_t K;           /* seeds to select, 1..n */
    int32_t J;           /* simulations (registers per vertex) */
    im_model model;      /* uniform / weighted cascade / trivalency (w unused);
                            kind -1: the model the graph was loaded with */
    uint64_t seed;       /* simulation seed, as im_select_seeds */
    double rebuild_eps;  /* as im_select_seeds */
} im_query;

typedef struct {
    int64_t ticket;
    int32_t status;      /* im_status of the query */
    int32_t slot;        /* worker that ran it */
    double t_submit_ms;  /* im_server_clock_ms() at submission */
    double t_start_ms;   /* ... when a slot took it */
    double t_done_ms;    /* ... when its seeds were on the host */
    double ms_select;    /* host time of the selection itself */
    uint64_t bytes;      /* device bytes reserved for it */
    char error[160];     /* message when status != IM_OK */
} im_query_result;

typedef struct {
    int64_t submitted, completed, failed, bypassed;
    int32_t slots, running, running_peak, pending;
    uint64_t budget, graph_bytes, reserved, reserved_peak;
} im_server_stats;

/* Starts the worker threads.  Errors: IM_E_INVAL (NULL, slots outside
 * [1, 64], max_bypass < 0), IM_E_CUDA. */
IM_API im_status im_server_create(const im_server_config* cfg, im_server** out);
/* Runs every pending query to completion, then stops the workers and frees
 * the server (not the graphs). */
IM_API void im_server_destroy(im_server* srv);
/* Registers a loaded graph (any context on the server's device); the graph
 * must outlive the server and is only read.  Its device bytes count against
 * the budget.  Errors: IM_E_INVAL, IM_E_STATE (other device), IM_E_NOMEM
 * (graphs alone exceed the budget). */
IM_API im_status im_server_add_graph(im_server* srv, im_graph* g, int32_t* id_out);
/* Device bytes a query of J simulations and K seeds on graph `graph` reserves. */
IM_API im_status im_server_query_bytes(im_server* srv, int32_t graph, int32_t J, int32_t K,
                                       uint64_t* bytes_out);
/* Queues a query and returns at once.  seeds_out (K int32), score_out and
 * estimate_out (K doubles each, may be NULL) are host buffers the caller owns
 * and keeps valid until im_server_wait returns for this ticket; they are
 * written by the worker.  Errors (nothing queued): IM_E_INVAL, IM_E_RANGE
 * (graph id, K), IM_E_STATE (model fixed at load), IM_E_NOMEM (the query alone
 * exceeds what the budget leaves beside the graphs). */
IM_API im_status im_server_submit(im_server* srv, const im_query* q, int32_t* seeds_out,
                                  double* score_out, double* estimate_out, int64_t* ticket_out);
/* Waits up to timeout_ms (< 0: no limit) for the query to finish and fills
 * *out; the ticket is then released.  Returns IM_E_TIMEOUT if it is still
 * pending or running, IM_E_RANGE for an unknown ticket; otherwise IM_OK (the
 * query's own status is out->status). */
IM_API im_status im_server_wait(im_server* srv, int64_t ticket, double timeout_ms,
                                im_query_result* out);
IM_API im_status im_server_get_stats(im_server* srv, im_server_stats* out);
/* Monotonic clock of the result timestamps, in milliseconds. */
IM_API double im_server_clock_ms(void);

#ifdef __cplusplus
}
#endif
#endif /* DIFUSER_IM_H */
