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
    kStCount
};

enum FrontierMode : int { kPush = 0, kCover = 1 };

struct FrontierArgs {
    uint8_t* M;
    int J;
    const uint32_t* X;     // J sorted draws
    const uint16_t* tab;   // kTabSize range table
    const QEntry* q_in;
    const unsigned long long* ctr_in;
    QEntry* q_out;
    unsigned long long* ctr_out;
    int32_t* gen;          // per-vertex enqueue stamps
    int32_t gen_next;
    unsigned long long* count;  // visited-register counter (cover)
    unsigned long long* stats;  // kStCount counters
    uint32_t* err;
};

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
    unsigned long long* count;
    int mark;                     // 1: mark the seed's row visited and queue it for the cover
};

int pick_grid(int32_t n, int J);

cudaError_t launch_sims(uint64_t seed, int J, uint32_t* X, uint32_t* salt, uint16_t* tab,
                        cudaStream_t st);
cudaError_t launch_fill(uint8_t* M, int32_t n, int J, const uint32_t* salt, cudaStream_t st);
cudaError_t launch_frontier(int kind, int mode, const GraphDev& g, const FrontierArgs& a,
                            int grid, cudaStream_t st);
int frontier_grid();
cudaError_t launch_pick(const PickArgs& a, cudaStream_t st);
// Marks row s visited (adding the newly visited registers to *count) and
// queues s as level 0 of a cover.
cudaError_t launch_cover_seed(uint8_t* M, int J, int32_t s, const int32_t* rp_out, QEntry* q,
                              unsigned long long* ctr, unsigned long long* count, cudaStream_t st);
cudaError_t launch_sums(const uint8_t* M, int32_t n, int J, unsigned long long* S, cudaStream_t st);
cudaError_t launch_count_visited(const uint8_t* M, int64_t bytes, unsigned long long* out,
                                 cudaStream_t st);

// graph load
cudaError_t launch_indegree(const int32_t* col, int64_t m, int32_t* cnt, cudaStream_t st);
// exclusive scan of cnt[0..n) into out[0..n] (out[n] = total); `tmp` >= scan_tmp_bytes(n)
size_t scan_tmp_bytes(int32_t n);
cudaError_t launch_exclusive_scan(const int32_t* cnt, int32_t n, int32_t* out, void* tmp,
                                  cudaStream_t st);
cudaError_t launch_scatter_in(const int32_t* rp_out, const int32_t* col_out, int32_t n,
                              const int32_t* rp_in, int32_t* fill, int32_t* src_in,
                              const uint32_t* thr_out, uint32_t* thr_in, cudaStream_t st);
cudaError_t launch_thr_wc(const int32_t* rp_in, int32_t n, uint32_t* thr_v, cudaStream_t st);
cudaError_t launch_thr_explicit(const float* w, int64_t m, uint32_t* thr, cudaStream_t st);
// queue of every vertex with in-degree > 0 (offsets = rp_in), count returned in *count_dev
cudaError_t launch_all_queue(const int32_t* rp_in, int32_t n, const uint32_t* thr_v,
                             const int32_t* pos, QEntry* q, cudaStream_t st);
cudaError_t launch_flag_nonzero_in(const int32_t* rp_in, int32_t n, int32_t* flag,
                                   cudaStream_t st);

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
