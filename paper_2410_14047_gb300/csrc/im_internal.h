// Library-internal entry points shared by the translation units of the shared
// library (hidden symbols: not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/difuser_im.h"

namespace imi {

// A context that runs on `stream`, allocates from `pool` (stream-ordered) and
// never uses the cooperative persistent launch (its kernels share the device
// with other contexts' kernels).
im_status ctx_create_worker(int device, cudaStream_t stream, cudaMemPool_t pool, im_ctx** out);
void ctx_set_budget(im_ctx* c, uint64_t bytes);
const char* ctx_error(const im_ctx* c);

// Alg. 4 of one query on context c, reading the resident graph g; the graph
// may belong to another context (same device) and is not modified.
im_status select_seeds_on(im_ctx* c, im_graph* g, int32_t K, int32_t J, const im_model* model,
                          uint64_t seed, double rebuild_eps, int32_t* seeds_out, double* score_out,
                          double* estimate_out);

// Device bytes one such query allocates (upper bound, allocator rounding included).
uint64_t query_bytes(const im_graph* g, int32_t J, int32_t K);
// Device bytes the graph holds; its vertex count; the device of its context.
uint64_t graph_bytes(const im_graph* g);
int32_t graph_n(const im_graph* g);
int graph_device(const im_graph* g);
// Validates a per-query model against the graph (uniform, WC, trivalency only
// when the graph was loaded with one of those).
im_status check_query_model(const im_graph* g, const im_model* model, char* msg, size_t cap);

}  // namespace imi
