// Host-side launch interface of the kernels in im_kernels.cu (internal to the
// library; the public C ABI is include/difuser_im.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "im_device.cuh"

namespace im {

// Indices of the device statistics block (unsigned long long each).
enum StatIndex : int {
    kStSweepVertices = 0,
    kStSweepEdges,
    kStSweepChunks,
    kStSweepCas,
    kStSweepChanged,
    kStCoverVertices,
    kStCoverEdges,
    kStCoverChunks,
    kStCoverNew,
    kStSweepLevels,
    kStCoverLevels,
    kStSweepHeavy,
    kStSweepHeavySims,
    kStSweepBatches,
    kStSweepDealt,
    kStSweepLiveEdges,  // examined in-edges live in a changed chunk (their ids and hashes are read)
    kStSweepBuckets,        // queued buckets walked by propagation levels
    kStSweepBucketEntries,  // bucket list entries processed (source chunk changed)
    kStAffected,            // registers recomputed by incremental rebuilds
    kStPullBuckets,         // out-buckets queued by the pulls of incremental rebuilds
    kStPullEntries,         // out-bucket entries walked by those pulls
    kStSweepChangedBuckets, // (vertex, chunk) buckets whose registers changed (bucket-format levels)
    kStPickRefreshed,       // rows whose stored S_u a lazy pick recomputed
    kStCount
};

// kAffect: the affected-set search of an incremental rebuild (in-edges, like
// propagation; marks bits instead of merging registers).
enum FrontierMode : int { kPush = 0, kCover = 1, kAffect = 2 };

// Formats of a level's queue: vertex entries, (vertex, chunk) bucket entries,
// or no queue at all (dense: the next level walks every vertex and reads the
// change bits; the counter's count field holds the raised items).
enum QueueFormat : int { kFmtVertex = 0, kFmtBucket = 1, kFmtDense = 2 };


// One frontier level (propagation sweep or cover level).  Queue t of a phase
// lives in buffer t % 3; counters pack count << 38 | edges.
struct LevelArgs {
    uint8_t* M;
    int J;
    int words;                           // J / 32 change-mask words per vertex
    const uint32_t* X;
    const uint16_t* tab;
    const QEntry* ql_in;                 // light queue (flat edge space)
    const unsigned long long* cl_in;
    const QEntry* qh_in;                 // heavy queue (propagation only; may be NULL)
    const unsigned long long* ch_in;
    QEntry* ql_out;
    unsigned long long* cl_out;
    QEntry* qh_out;
    unsigned long long* ch_out;
    const QEntry* ql_prev;               // queues of the previous level (change-bit clearing)
    const unsigned long long* cl_prev;
    const QEntry* qh_prev;
    const unsigned long long* ch_prev;
    const uint32_t* chg_cur;             // n * words: simulations changed at the previous level
    uint32_t* chg_next;
    uint32_t* chg_prev;                  // cleared for the previous level's queues (may be NULL)
    int all_changed;                     // level 0 of a build: every simulation counts as changed
    const QEntry* q_dense;               // every vertex with in-edges, vertex order (propagation)
    int32_t n_dense;
    int64_t e_dense;
    int32_t dense_div;                   // dense level when frontier > n_dense / dense_div (0: never)
    int32_t heavy_indeg;
    int light_batches;                   // 32-edge batches per claimed unit
    unsigned int* claim;                 // dynamic work counter of this level
    int32_t* gen;
    int32_t gen_next;
    unsigned long long* count;           // visited-register counter (cover)
    unsigned long long* stats;
    uint32_t* err;
    const int32_t* gid;                  // batches: graph of every vertex (NULL for one graph)
    unsigned long long* gcount;          // batches: visited-register counter per graph (cover)
    const uint8_t* gflag;                // batches: graphs whose vertices enter level 0 (build)
    // live chunk masks of the level's edge orientation (in-edges for
    // propagation, out-edges for covers): bit c of edge e = the edge is live
    // in a simulation of chunk c (16c .. 16c+15); chunks 32..63 in lcm_hi
    // (J = 1024, else NULL)
    const uint32_t* lcm_lo;
    const uint32_t* lcm_hi;
    // bucketed live lists of the level's orientation (NULL bk_end: edge scan).
    // Bucket b = v * chunks + c holds entries [start(b), end(b)), end(b) =
    // bk_end[b], start(b) = b ? bk_end[b - 1] : 0: the other endpoint of
    // every edge of v live in a simulation of chunk c, and its live mask over
    // the chunk's 16 simulations.  Queue entries are buckets (v = b).
    const uint32_t* bk_end;
    const int32_t* bk_other;
    const uint16_t* bk_mask;
    int32_t chunks;
    int64_t nbuckets;
    int32_t bq_cap;                      // bucket queue capacity; a fuller level walks every bucket
    // queue formats (hybrid mode): 0 = vertex entries, 1 = bucket entries.
    // fmt_in: format of this level's input queue; fmt_out: written by the
    // level with the format of its output queue; fmt_prev: the previous
    // level's input (change-bit clearing).  NULL: vertex format throughout.
    const uint8_t* fmt_in;
    uint8_t* fmt_out;
    const uint8_t* fmt_prev;
    int32_t bucket_div;                  // output in bucket format when input work * bucket_div < m
    int32_t bq_guard;                    // check the bucket queue's fill before each append (huge graphs)
    int32_t vq_cap;                      // vertex queue capacity (n)
    uint32_t* aff;                       // incremental rebuild: affected (vertex, simulation) bits
    uint32_t* awl;                       // affected-set search: words of aff that became nonzero
    unsigned int* awl_count;             //   (v * words + w each), their count (NULL: no list)
    uint32_t* nv;                        // covers: registers newly visited since the last build (may be NULL)
    int32_t chain;                       // continuation depth on small bucket levels (0 = none)
    int32_t dense_out;                   // dense walks of a propagation may output dense format
    int32_t dense_all;                   // dense walks of a propagation push every live simulation
};

// All levels of a phase in one cooperative launch (grid barrier between levels).
struct PhaseArgs {
    LevelArgs base;                      // fields that do not depend on the level
    QEntry* ql[3];
    QEntry* qh[3];
    ulonglong2* ctr;                     // per level: (light, heavy) packed counters
    unsigned int* claim;                 // per level work counters
    uint32_t* chg[3];
    int all_first;
    int max_levels;
    int32_t gen_base;                    // enqueue stamp of level t = gen_base + t
    unsigned int* bar_arrive;            // groups arrived
    unsigned int* bar_gen;
    unsigned int* abort_flag;
    unsigned long long limit_ns;         // bound on every barrier wait
    int* levels_out;                     // levels the phase ran
    unsigned long long* level_ns;        // tracing: global time at the start of level t (may be NULL)
    uint8_t* fmt;                        // per level queue format (hybrid mode; NULL otherwise)
};

int level_grid();
int phase_grid();  // 0 when cooperative launch is unavailable
cudaError_t launch_phase(int kind, int mode, const GraphDev& g, const PhaseArgs& p, int grid,
                         cudaStream_t st);
cudaError_t launch_level(int kind, int mode, const GraphDev& g, const LevelArgs& a, int grid,
                         cudaStream_t st);
cudaError_t launch_init_queues(int kind, const GraphDev& g, const LevelArgs& a, cudaStream_t st);
// Incremental rebuild steps: 0 level-0 queue of the affected-set search from
// the newly visited registers nv; 1 reset of the affected registers and the
// list of their vertices (out-degree, chunks of affected bits), in bucket mode
// also the pull queue of their affected chunks' out-buckets; 2 pull over the
// pull queue, or over the listed vertices' out-edges (loff: exclusive scan of
// their out-degrees, count + 1 entries, loff[count] the edges of the pull);
// 3 level-0 queue of the propagation from the list.  buckets: level-0 queues
// of (vertex, chunk) buckets.
struct IncrArgs {
    const uint32_t* nv;
    const uint32_t* salt;
    const int32_t* hkey;
    int32_t* list;
    int32_t* ldeg;
    const int32_t* loff;
    uint2* lmask;
    unsigned int* list_count;
    int32_t count;
    int buckets;
    // pull queue over the out-bucket lists (bucket mode): entries, packed
    // counter and overflow word; pull_buckets selects it for step 2
    QEntry* pq;
    unsigned long long* pctr;
    int pull_buckets;
    // the affected words listed by the search (bucket mode): steps 1 and 3
    // then walk only them (words_list)
    const uint32_t* awl;
    const unsigned int* awl_count;
    int words_list;
};
cudaError_t launch_incremental(int step, int kind, const GraphDev& g, const LevelArgs& a, const IncrArgs& x,
                               cudaStream_t st);

struct PickArgs {
    uint8_t* M;
    int J;
    int32_t n;
    uint32_t* seed_bits;          // n bits: vertices already picked
    unsigned long long* part_S;   // one per block
    int32_t* part_u;
    unsigned int* ticket;
    int32_t* out_seed;            // [k]
    unsigned long long* out_S;    // [k]
    double* out_est;              // [k]
    int k;
    const int32_t* rp_out;
    QEntry* q_cover;              // cover queue, level 0
    unsigned long long* ctr_cover;
    uint32_t* chg0;               // change mask of cover level 0 (n * J/32 words)
    unsigned long long* count;
    int mark;                     // 1: mark the seed's row visited and queue it for the cover
    // lazy picks (S_u never decreases during a selection, so a stored S_u is
    // a lower bound of the current one): lb[n] stored sums, cand = the vertex
    // of least stored (S, u) besides the pick, part_S2 / part_u2 = per-block
    // runner-up.  All null: plain full pick.
    unsigned long long* lb;
    int32_t* cand;
    unsigned long long* part_S2;
    int32_t* part_u2;
    // bucket mode: the cover's level-0 queue holds the seed's out-buckets
    // (chunks with newly visited simulations and live out-edges)
    const uint32_t* bk_end_out;
    int32_t chunks;
    uint32_t* nv;                 // registers newly visited since the last build (may be NULL)
    int tile;                     // J-tile width of a full pick: 16-byte pieces a lane sums (1, 2, 4)
    unsigned long long* stats;    // statistics block (rows refreshed by lazy picks; may be NULL)
    // lazy picks: per group of 128 rows the two least stored (S, u) of its
    // unpicked rows (4 words a group: S1, S2, u1 | u2 << 32, unused); NULL
    // for full picks that keep no records
    unsigned long long* gsum;
    int32_t ngroups;
};

// Blocks of a full pick: one row group per warp step, at most 152 * 8; tile
// = 16-byte pieces of a row a lane sums (1, 2 or 4; other values: 4).
int pick_grid(int32_t n, int J, int tile = 4);
int pick_lazy_grid(int32_t n);
int pick_groups(int32_t n);  // lazy-pick group records of n rows
// Group records of every group (after a full pick that stored every S_u).
cudaError_t launch_group_summaries(const PickArgs& a, cudaStream_t st);

cudaError_t launch_sims(uint64_t seed, int J, uint32_t* X, uint32_t* salt, uint16_t* tab,
                        cudaStream_t st);
cudaError_t launch_fill(uint8_t* M, int32_t n, int J, const uint32_t* salt, bool fresh, cudaStream_t st);
// Fill of the rows whose graph has gflag[gid[u]] != 0 (batches).
cudaError_t launch_fill_flagged(uint8_t* M, int32_t n, int J, const uint32_t* salt, const int32_t* gid,
                                const uint8_t* gflag, const int32_t* hkey, cudaStream_t st);

// Batches: estimate + argmax per graph.  Tiles are row ranges inside one
// graph: (graph, row begin, row end).
struct BatchPickArgs {
    uint8_t* M;
    int J;
    const int4* tiles;            // x = graph, y = row begin, z = row end
    int ntiles;
    const uint8_t* active;        // graph picks this round
    uint32_t* picked;             // picked bitmap over the union
    unsigned long long* part_S;   // per tile
    int32_t* part_u;
    const int32_t* tile_begin;    // per graph: first tile (tiles of a graph are consecutive)
    const int32_t* tile_end;
    int G;
    int round;
    int maxK;
    int32_t* out_seed;            // [G * maxK]: global vertex ids
    unsigned long long* out_S;
    double* out_est;
    const int32_t* rp_out;
    QEntry* q_cover;              // cover level-0 queue
    unsigned long long* ctr_cover;
    uint32_t* chg0;
    unsigned long long* gcount;
    uint32_t* err;
    const uint32_t* bk_end_out;   // bucket mode (see PickArgs)
    int32_t chunks;
};
cudaError_t launch_batch_pick(const BatchPickArgs& a, cudaStream_t st);
cudaError_t launch_pick(const PickArgs& a, cudaStream_t st);
// Live chunk masks of every in-edge (mode kPush) or out-edge (kCover) for the
// simulations X (sorted) of one sketch.
// Warp fill-rate counts of the live tests (see k_fill_rate); out[5] accumulates.
cudaError_t launch_fill_rate(int kind, const GraphDev& g, uint64_t seed, const uint32_t* X, const uint16_t* tab,
                             int J, unsigned long long* out, cudaStream_t st);
cudaError_t launch_live_chunks(int kind, int mode, const GraphDev& g, const uint32_t* X, const uint16_t* tab,
                               int J, uint32_t* lo, uint32_t* hi, cudaStream_t st);
// Bucketed live lists of one orientation (mode kPush: in-edges grouped by
// target, kCover: out-edges grouped by source).  Pass 0 counts bucket sizes
// into cnt[n * J/16] (zeroed by the caller) and non-empty buckets into
// *nonempty; after an exclusive scan of cnt into end[] (end[nb] = total),
// pass 1 fills other / mask and leaves end[b] = end of bucket b.
cudaError_t launch_buckets(int pass, int kind, int mode, const GraphDev& g, const uint32_t* X,
                           const uint16_t* tab, int J, uint32_t* cnt_or_end, unsigned long long* nonempty,
                           int32_t* other, uint16_t* mask, cudaStream_t st);
// Lazy pick: refreshes S_v of every unpicked v whose stored (lb[v], v) is
// below (S_cand, cand) with S_cand fresh, then takes the least stored pair.
cudaError_t launch_pick_lazy(const PickArgs& a, cudaStream_t st);
// Marks row s visited (adding the newly visited registers to *count) and
// queues s as level 0 of a cover.
cudaError_t launch_cover_seed(uint8_t* M, int J, int32_t s, const int32_t* rp_out, QEntry* q,
                              unsigned long long* ctr, uint32_t* chg0, unsigned long long* count,
                              const uint32_t* bk_end, int C, cudaStream_t st);
cudaError_t launch_sums(const uint8_t* M, int32_t n, int J, unsigned long long* S, cudaStream_t st);
cudaError_t launch_count_visited(const uint8_t* M, int64_t bytes, unsigned long long* out,
                                 cudaStream_t st);

// graph load
cudaError_t launch_indegree(const int32_t* col, int64_t m, int32_t* cnt, cudaStream_t st);
// exclusive scan of cnt[0..n) into out[0..n] (out[n] = total); `tmp` >= scan_tmp_bytes(n)
size_t scan_tmp_bytes(int32_t n);
cudaError_t launch_exclusive_scan(const int32_t* cnt, int32_t n, int32_t* out, void* tmp,
                                  cudaStream_t st);
// In-CSR sorted by (target, trivalency class, edge hash): src_in, h_in (edge
// hashes), thr_in (explicit models, may be NULL), in the order of the in-CSR
// row pointers built beforehand.  hkey (may be NULL = the vertex id itself) is
// the id each vertex hashes with (batches: its id inside its own graph).
size_t build_in_csr_tmp_bytes(int64_t m);
// out_to_in (may be NULL): in-CSR position of every out-edge; tri_b (trivalency,
// may be NULL): class bounds of every in-row (rp_in: the in-CSR row starts).
cudaError_t launch_build_in_csr(const int32_t* rp_out, const int32_t* col_out, int32_t n, int64_t m,
                                int kind, uint32_t tri_seed, const int32_t* hkey, const uint32_t* thr_out,
                                int32_t* src_in, uint32_t* h_in,
                                uint32_t* thr_in, int32_t* out_to_in, const int32_t* rp_in, int2* tri_b,
                                void* tmp, cudaStream_t st);
// dst[i] = src[idx[i]], i < m.
cudaError_t launch_gather_u32(const uint32_t* src, const int32_t* idx, int64_t m, uint32_t* dst, cudaStream_t st);
// CSR validation of an uploaded graph: bad[0] = the lowest u whose rowptr
// decreases, bad[1] = the lowest row with an id out of range, a self-loop or
// ids not strictly ascending; each >= n when there is none.
cudaError_t launch_check_csr(const int32_t* rp, const int32_t* col, int32_t n, int64_t m, int32_t* bad,
                             cudaStream_t st);
cudaError_t launch_out_edge_words(const int32_t* rp_out, const int32_t* col_out, int32_t n, int64_t m,
                                  const uint32_t* thr_v, const int32_t* hkey, uint32_t* h_out,
                                  uint32_t* thrw_out, cudaStream_t st);
cudaError_t launch_radix_sort(unsigned long long* keys, int32_t* vals, int64_t n, int bits,
                              void* tmp, cudaStream_t st);
size_t sort_tmp_bytes(int64_t n);
// Static queue of the vertices with in-edges in vertex order; pos[n] = count.
cudaError_t launch_dense_queue(const int32_t* rp_in, int32_t n, const uint32_t* thr_v, int32_t* flag,
                               int32_t* pos, void* scan_tmp, QEntry* q, cudaStream_t st);
cudaError_t launch_thr_wc(const int32_t* rp_in, int32_t n, uint32_t* thr_v, cudaStream_t st);
cudaError_t launch_thr_explicit(const float* w, int64_t m, uint32_t* thr, cudaStream_t st);

// Monte-Carlo spread (independent coins): simulations of a batch are bits of
// `words` 32-bit words per vertex.
struct McArgs {
    int32_t n;
    int64_t m;
    uint64_t seed;              // coin stream seed
    int64_t r0;                 // global index of the batch's first simulation
    int words;                  // words per vertex (batch size / 32, a power of two)
    uint32_t* vis;              // n * words: vertex reached in simulation
    const uint32_t* f_cur;      // n * words: newly reached at the previous level
    uint32_t* f_next;           // n * words: newly reached at this level
    uint32_t* f_prev;           // cleared for the entries of q_prev
    const QEntry* q_in;
    const unsigned long long* ctr_in;
    const QEntry* q_prev;       // may be NULL
    const unsigned long long* ctr_prev;
    QEntry* q_out;
    unsigned long long* ctr_out;
    int32_t* gen;
    int32_t gen_next;
};
cudaError_t launch_mc_level(int kind, const GraphDev& g, const McArgs& a, int grid,
                            cudaStream_t st);
cudaError_t launch_mc_seed(const GraphDev& g, const McArgs& a, const int32_t* seeds, int k,
                           int valid, cudaStream_t st);
cudaError_t launch_mc_count(const uint32_t* vis, int32_t n, int words, unsigned long long* reach,
                            cudaStream_t st);
cudaError_t launch_mc_reduce(const unsigned long long* reach, int valid, unsigned long long* acc,
                             cudaStream_t st);

}  // namespace im
