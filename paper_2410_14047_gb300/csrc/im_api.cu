// Host implementation of the C ABI declared in include/difuser_im.h.
//
// Owns device memory (through the caller's allocator or cudaMallocAsync,
// charged against the context's HBM budget), validates inputs, and drives
// the kernels of im_kernels.cu through Alg. 4 of the paper: build
// (Alg. 1 + Alg. 2 to a fixpoint), then K times pick (Sketchwise-Sum +
// argmax), cover (Alg. 3 levels) and the error-adaptive rebuild.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/difuser_im.h"
#include "im_internal.h"
#include "im_launch.h"

using namespace im;

constexpr uint64_t kDefaultBarrierLimitNs = 2000000000ull;  // 2 s

struct im_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0;
    uint64_t in_use = 0;
    uint64_t peak = 0;
    bool custom_alloc = false;
    im_allocator alloc{};
    cudaMemPool_t pool = nullptr;  // stream-ordered pool of a server worker (else the device default)
    std::unordered_map<void*, size_t> sizes;
    std::string err;
    im_stats stats{};
    unsigned long long* pinned = nullptr;  // small pinned staging buffer (64 words)
    // kernel timing: event pairs recorded around launches, summed at sync points
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    std::vector<int64_t> ev_seq;     // launch sequence number of each recorded pair
    int ev_used = 0;
    int64_t seq = 0;                 // launches since the start of the call
    bool trace = false;
    std::vector<float> launch_ms;    // kernel time per launch sequence number (tracing)
    std::vector<im_trace_rec> recs;  // frontier launches of the last call
    im_tuning tuning{256, 4, 0, 2, 1, 0, 1, 2, 1, 8, 4, 1, 0};
    // bounds of the device-side waits (im_ctx_set_limits)
    uint64_t barrier_limit_ns = kDefaultBarrierLimitNs;
    int32_t max_levels = kMaxLevels - 2;
    // a second stream for work independent of the main stream's (the first
    // fill of a sketch next to its live chunk masks), forked and joined with
    // events; created on first use
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

im_status fail(im_ctx* c, im_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

im_status cuda_fail(im_ctx* c, cudaError_t e, const char* what) {
    return fail(c, IM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(ctx, call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

#define CKS(call)                        \
    do {                                 \
        im_status s_ = (call);           \
        if (s_ != IM_OK) return s_;      \
    } while (0)

size_t round_bytes(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    return bytes == 0 ? 256 : bytes;
}

im_status dalloc(im_ctx* c, size_t bytes, DBuf& out) {
    bytes = round_bytes(bytes);
    if (c->budget && c->in_use + bytes > c->budget)
        return fail(c, IM_E_NOMEM, "HBM budget exceeded: %llu + %llu > %llu bytes",
                    (unsigned long long)c->in_use, (unsigned long long)bytes,
                    (unsigned long long)c->budget);
    void* p = nullptr;
    if (c->custom_alloc) {
        p = c->alloc.alloc(bytes, c->stream, c->alloc.user);
        if (!p) return fail(c, IM_E_NOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = c->pool ? cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream)
                                : cudaMallocAsync(&p, bytes, c->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(c, IM_E_NOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    out.p = p;
    out.bytes = bytes;
    c->sizes[p] = bytes;
    c->in_use += bytes;
    if (c->in_use > c->peak) c->peak = c->in_use;
    return IM_OK;
}

void dfree(im_ctx* c, DBuf& b) {
    if (!b.p) return;
    if (c->custom_alloc) c->alloc.free(b.p, b.bytes, c->stream, c->alloc.user);
    else cudaFreeAsync(b.p, c->stream);
    c->sizes.erase(b.p);
    c->in_use -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

bool valid_J(int32_t J) {
    return J >= 16 && J <= kMaxJ && (J & (J - 1)) == 0;
}

uint32_t prob_threshold_host(float w) {
    const double t = std::floor((double)w * 2147483648.0);
    if (!(t > 0.0)) return 0u;
    if (t >= 2147483648.0) return 2147483648u;
    return (uint32_t)t;
}

// Alg. 4 rebuild test in FP64: (score - oldscore) / score > e, score = count/J.
bool rebuild_due(uint64_t count, uint64_t oldcount, int32_t J, double e) {
    if (e < 0.0) return false;
    const double score = (double)count / (double)J;
    const double oldscore = (double)oldcount / (double)J;
    return (score - oldscore) / score > e;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum TimeKind { kTPush = 0, kTCover = 1, kTPick = 2, kTFill = 3, kTOther = 4 };

// Adds the durations of the recorded event pairs (all complete: call after a
// stream synchronize) to the context's statistics.
void timing_collect(im_ctx* c) {
    for (int i = 0; i < c->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (c->trace) {
            const int64_t q = c->ev_seq[i];
            if ((int64_t)c->launch_ms.size() <= q) c->launch_ms.resize(q + 1024, 0.f);
            c->launch_ms[q] = ms;
        }
        switch (c->ev_kind[i]) {
            case kTPush: c->stats.ms_propagate += ms; break;
            case kTCover: c->stats.ms_cover_kernels += ms; break;
            case kTPick: c->stats.ms_pick_kernels += ms; break;
            case kTFill: c->stats.ms_fill_kernels += ms; break;
            default: break;
        }
    }
    c->ev_used = 0;
}

// Launch bracket: records a start event (timing on), runs the launch, records
// the stop event and counts the launch.
template <class F>
cudaError_t timed(im_ctx* c, int kind, F&& launch) {
    int slot = -1;
    if (c->timing) {
        if (c->ev_used * 2 + 2 > (int)c->ev.size()) {
            // (a pair recorded on the side stream must be complete as well)
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess && c->side) e = cudaStreamSynchronize(c->side);
            if (e != cudaSuccess) return e;
            timing_collect(c);
        }
        slot = c->ev_used++;
        c->ev_kind[slot] = kind;
        c->ev_seq[slot] = c->seq;
        cudaEventRecord(c->ev[2 * slot], c->stream);
    }
    cudaError_t e = launch();
    if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], c->stream);
    c->stats.launches++;
    c->seq++;
    if (kind == kTPush) c->stats.sweep_launches++;
    return e;
}

// The same bracket on another stream of the context.
template <class F>
cudaError_t timed_on(im_ctx* c, cudaStream_t st, int kind, F&& launch) {
    int slot = -1;
    if (c->timing) {
        if (c->ev_used * 2 + 2 > (int)c->ev.size()) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return e;
            timing_collect(c);
        }
        slot = c->ev_used++;
        c->ev_kind[slot] = kind;
        c->ev_seq[slot] = c->seq;
        cudaEventRecord(c->ev[2 * slot], st);
    }
    cudaError_t e = launch();
    if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], st);
    c->stats.launches++;
    c->seq++;
    return e;
}

// The context's second stream and its fork / join events (created once).
cudaError_t ensure_side(im_ctx* c) {
    if (c->side) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    return e;
}

// Stream synchronize followed by the collection of finished timings.
cudaError_t sync_collect(im_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && c->side) e = cudaStreamSynchronize(c->side);
    if (e == cudaSuccess && c->timing) timing_collect(c);
    return e;
}

}  // namespace

struct im_graph {
    im_ctx* ctx = nullptr;
    int32_t n = 0;
    int64_t m = 0;
    int kind = kUniform;       // kernel family (a per-target model runs as kWC)
    int load_kind = kUniform;  // model kind given at load
    DBuf rp_out, col_out, rp_in, src_in, h_in, h_out, thrw_out, thr_v, thr_out, thr_in, q_dense,
        hkey, q_dense_out, out_to_in, tri_b;
    int32_t n_dense = 0;      // vertices with in-edges (q_dense: their in-rows in vertex order)
    int32_t n_dense_out = 0;  // vertices with out-edges (q_dense_out: their out-rows)
    GraphDev dev{};
};

struct im_sketch {
    im_graph* g = nullptr;
    im_ctx* ctx = nullptr;  // execution context: allocator, stream, statistics
    int32_t J = 0;
    DBuf M, X, salt, tab, ql[3], qh[3], ctr, claim, chg[3], gen, seed_bits, count, part_S, part_u,
        ticket, stats, err, bar, lb, cand, part_S2, part_u2, lcm_in_lo, lcm_in_hi, lcm_out_lo, lcm_out_hi,
        level_ns, fmt, nv, aff, alist, acount, aldeg, aloff, almask, ascan, apctr, awl,
        awlc;
    bool incr = false;      // covers record newly visited registers; rebuilds are incremental
    // bucket mode: bucketed live lists per orientation (0: in-edges, 1:
    // out-edges); the light queues then hold buckets, bq_cap entries each
    DBuf bk_end[2], bk_other[2], bk_mask[2];
    // bucket mode keeps the cover's change masks apart from the
    // propagation's: a bucket that is empty in one orientation may keep stale
    // bits there (never read), which must not reach the other orientation
    DBuf chg_cov[3];
    bool buckets = false;
    int32_t bq_cap = 0;
    bool lazy = false;      // picks after the first refresh stored sums only (im_select_seeds)
    bool chg_dirty = true;  // change masks may hold bits (new sketch, or a phase that failed)
    // the registers were never written (a new sketch): the first fill writes
    // every register without reading it, so no zeroing pass precedes it
    bool fresh = true;
    // that first fill runs on the context's side stream next to the live
    // chunk masks; the main stream waits for it (ev_join) before its first use
    bool fill_pending = false;
    bool lb_ready = false;  // lb holds the sums of the last full pick or later refreshes
    // a selection in flight: phases and rebuilds queue without host reads;
    // their error word is read once at the end
    bool defer = false;
    bool pull_safe = false;  // the pull queue holds every out-bucket (it cannot overflow)
    DBuf out_seed, out_S, out_est;
    DBuf gsum;  // lazy-pick group records
    int32_t out_cap = 0;
    int32_t gen_counter = 0;
    int32_t picks = 0;
    // the graph's device view with this sketch's model words (a per-call model
    // override changes the copy, never the shared graph)
    GraphDev dev{};
    int kind = kUniform;
    // batches (several graphs in one union): graph of every vertex, visited
    // counter per graph, graphs whose rows a build covers
    const int32_t* gid = nullptr;
    unsigned long long* gcount = nullptr;
    const uint8_t* gflag = nullptr;
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" im_status im_ctx_create(int device, void* cuda_stream, uint64_t hbm_budget_bytes,
                                   const im_allocator* alloc, im_ctx** out) {
    if (!out) return IM_E_INVAL;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        (void)cudaGetLastError();
        return IM_E_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return IM_E_CUDA;
    im_ctx* c = new im_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->budget = hbm_budget_bytes;
    if (alloc && alloc->alloc && alloc->free) {
        c->custom_alloc = true;
        c->alloc = *alloc;
    }
    if (cudaMallocHost(&c->pinned, 64 * sizeof(unsigned long long)) != cudaSuccess) {
        delete c;
        return IM_E_CUDA;
    }
    *out = c;
    return IM_OK;
}

extern "C" void im_ctx_destroy(im_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
        cudaEventDestroy(c->ev_fork);
        cudaEventDestroy(c->ev_join);
    }
    if (c->pinned) cudaFreeHost(c->pinned);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
}

extern "C" im_status im_ctx_set_timing(im_ctx* c, int enable) {
    if (!c) return IM_E_INVAL;
    if (enable && c->ev.empty()) {
        c->ev.resize(256);
        c->ev_kind.resize(128);
        c->ev_seq.resize(128);
        for (auto& e : c->ev) CK(c, cudaEventCreate(&e));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    c->ev_used = 0;
    c->timing = enable != 0 || c->trace;
    return IM_OK;
}

extern "C" im_status im_ctx_set_tuning(im_ctx* c, const im_tuning* t) {
    if (!c) return IM_E_INVAL;
    if (!t) {
        c->tuning = im_tuning{256, 4, 0, 2, 1, 0, 1, 2, 1, 8, 4, 1, 0};
        return IM_OK;
    }
    if (t->heavy_indeg < 0 || t->light_batches < 1 || t->light_batches > 4096 || t->grid_blocks < 0 ||
        t->check_every < 1 || t->check_every > 64 || t->persistent < 0 || t->persistent > 1 ||
        t->dense_div < 0 || t->lazy_pick < 0 || t->lazy_pick > 1 || t->buckets < 0 || t->buckets > 1024 || t->incremental < 0 || t->incremental > 2 ||
        t->chain < 0 || t->chain > 64 ||
        !(t->pick_tile == 0 || t->pick_tile == 1 || t->pick_tile == 2 || t->pick_tile == 4) ||
        t->dense_out < 0 || t->dense_out > 1 || t->dense_all < 0 || t->dense_all > 3)
        return fail(c, IM_E_INVAL, "tuning out of range");
    c->tuning = *t;
    return IM_OK;
}

extern "C" im_status im_ctx_set_limits(im_ctx* c, uint64_t barrier_wait_ns, int32_t max_levels) {
    if (!c) return IM_E_INVAL;
    if (max_levels < 1 || max_levels > kMaxLevels - 2)
        return fail(c, IM_E_INVAL, "max_levels must be in [1, %d]", kMaxLevels - 2);
    c->barrier_limit_ns = barrier_wait_ns;
    c->max_levels = max_levels;
    return IM_OK;
}

extern "C" im_status im_ctx_get_tuning(const im_ctx* c, im_tuning* t) {
    if (!c || !t) return IM_E_INVAL;
    *t = c->tuning;
    return IM_OK;
}

extern "C" im_status im_ctx_set_trace(im_ctx* c, int enable) {
    if (!c) return IM_E_INVAL;
    c->trace = enable != 0;
    return im_ctx_set_timing(c, c->timing || c->trace);
}

extern "C" int64_t im_last_trace(const im_ctx* c, im_trace_rec* out, int64_t cap) {
    if (!c) return 0;
    const int64_t n = (int64_t)c->recs.size();
    if (out)
        for (int64_t i = 0; i < n && i < cap; ++i) out[i] = c->recs[i];
    return n;
}

extern "C" uint64_t im_ctx_bytes_in_use(const im_ctx* c) { return c ? c->in_use : 0; }
extern "C" uint64_t im_ctx_bytes_peak(const im_ctx* c) { return c ? c->peak : 0; }
extern "C" const char* im_last_error(const im_ctx* c) { return c ? c->err.c_str() : ""; }

extern "C" const char* im_status_str(im_status s) {
    switch (s) {
        case IM_OK: return "IM_OK";
        case IM_E_INVAL: return "IM_E_INVAL";
        case IM_E_RANGE: return "IM_E_RANGE";
        case IM_E_NOMEM: return "IM_E_NOMEM";
        case IM_E_CUDA: return "IM_E_CUDA";
        case IM_E_TIMEOUT: return "IM_E_TIMEOUT";
        case IM_E_STATE: return "IM_E_STATE";
    }
    return "IM_E_UNKNOWN";
}

extern "C" im_status im_last_stats(const im_ctx* c, im_stats* out) {
    if (!c || !out) return IM_E_INVAL;
    *out = c->stats;
    return IM_OK;
}

// ---------------------------------------------------------------------------
// graph
// ---------------------------------------------------------------------------
static im_status check_model(im_ctx* c, const im_model* mdl, int64_t m) {
    if (!mdl) return fail(c, IM_E_INVAL, "model is NULL");
    if (mdl->kind < kUniform || mdl->kind > kTargetModel)
        return fail(c, IM_E_INVAL, "unknown model kind %d", mdl->kind);
    if (mdl->kind == kTargetModel && !mdl->w)
        return fail(c, IM_E_INVAL, "per-target model needs w[n]");
    if (mdl->kind == kUniform && !(mdl->p >= 0.0f && mdl->p <= 1.0f))
        return fail(c, IM_E_INVAL, "uniform p must be in [0,1]");
    if (mdl->kind == kExplicit && m > 0 && !mdl->w)
        return fail(c, IM_E_INVAL, "explicit model needs w[m]");
    return IM_OK;
}

static void graph_release(im_graph* g) {
    im_ctx* c = g->ctx;
    for (DBuf* b : {&g->rp_out, &g->col_out, &g->rp_in, &g->src_in, &g->h_in, &g->h_out,
                    &g->thrw_out, &g->thr_v, &g->thr_out, &g->thr_in, &g->q_dense,
                    &g->hkey, &g->q_dense_out, &g->out_to_in, &g->tri_b})
        dfree(c, *b);
}

// Model words of a device view (uniform, weighted-cascade, trivalency: no
// per-edge data beyond what every graph holds).
static void model_words(GraphDev& dev, int& kind, const im_model* mdl) {
    kind = mdl->kind == kTargetModel ? kWC : mdl->kind;
    dev.thr_uniform = prob_threshold_host(mdl->p);
    dev.tri_seed = (uint32_t)(mdl->seed ^ (mdl->seed >> 32));
    dev.tri_thr[0] = prob_threshold_host(0.1f);
    dev.tri_thr[1] = prob_threshold_host(0.01f);
    dev.tri_thr[2] = prob_threshold_host(0.001f);
}

// The in-rows' trivalency class bounds hold for a device view only when its
// model is the trivalency model the rows were sorted under.
static void keep_class_bounds(GraphDev& dev, int kind, const im_graph* g) {
    if (kind != kTrivalency || g->kind != kTrivalency || dev.tri_seed != g->dev.tri_seed) dev.tri_b = nullptr;
}

// Sets the model part of the device view; allocates per-vertex / per-edge
// thresholds as the model needs.  thr_out / thr_in of an explicit model are
// filled by the caller (they need the reverse CSR).
static im_status set_model(im_graph* g, const im_model* mdl) {
    im_ctx* c = g->ctx;
    // a per-target-vertex model runs the weighted-cascade kernels (every
    // in-edge of v has v's threshold); its thresholds are set at load
    model_words(g->dev, g->kind, mdl);
    if (mdl->kind == kExplicit && g->m > 0) {
        DBuf w;
        CKS(dalloc(c, (size_t)g->m * sizeof(float), w));
        cudaError_t e = cudaMemcpyAsync(w.p, mdl->w, (size_t)g->m * sizeof(float),
                                        cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) {
            if (!g->thr_out.p) {
                im_status s = dalloc(c, (size_t)g->m * 4, g->thr_out);
                if (s != IM_OK) { dfree(c, w); return s; }
            }
            e = launch_thr_explicit(w.as<float>(), g->m, g->thr_out.as<uint32_t>(), c->stream);
        }
        dfree(c, w);
        if (e != cudaSuccess) return cuda_fail(c, e, "explicit thresholds");
    }
    return IM_OK;
}

// Validation of a host CSR: rows [r0, r1) ascending, ids in range, no
// self-loops, rows strictly ascending.  Returns the first bad row (r1 if
// none) and writes its error.  (The graph load validates on the device and
// runs this on the one row it reports, for the message.)
static int32_t check_rows(int32_t n, const int32_t* rowptr, const int32_t* col, int32_t r0, int32_t r1,
                          im_status* st, char* msg, size_t cap) {
    for (int32_t u = r0; u < r1; ++u) {
        const int32_t b = rowptr[u], e = rowptr[u + 1];
        if (e < b) { *st = IM_E_INVAL; snprintf(msg, cap, "rowptr decreases at %d", u); return u; }
        for (int32_t i = b; i < e; ++i) {
            const int32_t v = col[i];
            if (v < 0 || v >= n) { *st = IM_E_RANGE; snprintf(msg, cap, "col[%d] = %d out of range", i, v); return u; }
            if (v == u) { *st = IM_E_INVAL; snprintf(msg, cap, "self-loop at vertex %d", u); return u; }
            if (i > b && col[i - 1] >= v) {
                *st = IM_E_INVAL;
                snprintf(msg, cap, "row %d not strictly ascending (duplicate edge?)", u);
                return u;
            }
        }
    }
    return r1;
}

static im_status graph_load_impl(im_ctx* c, int32_t n, int64_t m, const int32_t* rowptr,
                                 const int32_t* col, const im_model* model, const int32_t* hkey_host,
                                 im_graph** out) {
    if (!c || !out || !rowptr || (m > 0 && !col)) return fail(c, IM_E_INVAL, "NULL argument");
    if (n < 1 || n >= (1 << 26)) return fail(c, IM_E_RANGE, "n must be in [1, 2^26)");
    if (m < 0 || m >= (1ll << 31)) return fail(c, IM_E_RANGE, "m must be in [0, 2^31)");
    CKS(check_model(c, model, m));
    if (rowptr[0] != 0 || rowptr[n] != m) return fail(c, IM_E_INVAL, "rowptr[0] != 0 or rowptr[n] != m");
    CK(c, cudaSetDevice(c->device));
    im_graph* g = new im_graph();
    g->ctx = c;
    g->n = n;
    g->m = m;
    auto bail = [&](im_status s) {
        graph_release(g);
        delete g;
        return s;
    };
    im_status s;
    const size_t rp_bytes = ((size_t)n + 1) * 4, e_bytes = (size_t)(m > 0 ? m : 1) * 4;
    if ((s = dalloc(c, rp_bytes, g->rp_out)) != IM_OK) return bail(s);
    if ((s = dalloc(c, e_bytes, g->col_out)) != IM_OK) return bail(s);
    if ((s = dalloc(c, rp_bytes, g->rp_in)) != IM_OK) return bail(s);
    if ((s = dalloc(c, e_bytes, g->src_in)) != IM_OK) return bail(s);
    if ((s = dalloc(c, e_bytes, g->h_in)) != IM_OK) return bail(s);
    if ((s = dalloc(c, e_bytes, g->h_out)) != IM_OK) return bail(s);
    if ((s = dalloc(c, e_bytes, g->thrw_out)) != IM_OK) return bail(s);
    if ((s = dalloc(c, e_bytes, g->out_to_in)) != IM_OK) return bail(s);
    if ((s = dalloc(c, (size_t)n * 4, g->thr_v)) != IM_OK) return bail(s);
    if ((s = dalloc(c, (size_t)n * sizeof(QEntry), g->q_dense)) != IM_OK) return bail(s);
    if ((s = dalloc(c, (size_t)n * sizeof(QEntry), g->q_dense_out)) != IM_OK) return bail(s);
    DBuf cnt, tmp;
    if ((s = dalloc(c, ((size_t)n + 1) * 4, cnt)) != IM_OK) return bail(s);
    const size_t tmp_bytes = std::max(scan_tmp_bytes(n), build_in_csr_tmp_bytes(m));
    if ((s = dalloc(c, tmp_bytes, tmp)) != IM_OK) { dfree(c, cnt); return bail(s); }
    auto release_tmp = [&]() { dfree(c, cnt); dfree(c, tmp); };
    auto st = c->stream;
    cudaError_t e = cudaMemcpyAsync(g->rp_out.p, rowptr, rp_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && m > 0)
        e = cudaMemcpyAsync(g->col_out.p, col, (size_t)m * 4, cudaMemcpyHostToDevice, st);
    // the CSR is validated on the device before any kernel indexes by its ids;
    // the message of a bad row comes from the host check of that row alone
    {
        int32_t bad[2] = {0, 0};
        if (e == cudaSuccess) e = launch_check_csr(g->rp_out.as<int32_t>(), g->col_out.as<int32_t>(), n, m,
                                                   cnt.as<int32_t>(), st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bad, cnt.p, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && (bad[0] < n || bad[1] < n)) {
            release_tmp();
            if (bad[0] < n) return bail(fail(c, IM_E_INVAL, "rowptr decreases at %d", bad[0]));
            im_status rs = IM_E_INVAL;
            char buf[256];
            snprintf(buf, sizeof buf, "invalid row %d", bad[1]);
            check_rows(n, rowptr, col, bad[1], bad[1] + 1, &rs, buf, sizeof buf);
            return bail(fail(c, rs, "%s", buf));
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, ((size_t)n + 1) * 4, st);
    if (e == cudaSuccess) e = launch_indegree(g->col_out.as<int32_t>(), m, cnt.as<int32_t>(), st);
    if (e == cudaSuccess) e = launch_exclusive_scan(cnt.as<int32_t>(), n, g->rp_in.as<int32_t>(), tmp.p, st);
    if (e == cudaSuccess) e = launch_thr_wc(g->rp_in.as<int32_t>(), n, g->thr_v.as<uint32_t>(), st);
    if (e == cudaSuccess && model->kind == kTargetModel) {
        // per-target probabilities replace the weighted-cascade thresholds
        DBuf w;
        if ((s = dalloc(c, (size_t)n * sizeof(float), w)) != IM_OK) { release_tmp(); return bail(s); }
        e = cudaMemcpyAsync(w.p, model->w, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_thr_explicit(w.as<float>(), n, g->thr_v.as<uint32_t>(), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        dfree(c, w);
    }
    if (e == cudaSuccess && hkey_host) {
        if ((s = dalloc(c, (size_t)n * 4, g->hkey)) != IM_OK) { release_tmp(); return bail(s); }
        e = cudaMemcpyAsync(g->hkey.p, hkey_host, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess)
        e = launch_out_edge_words(g->rp_out.as<int32_t>(), g->col_out.as<int32_t>(), n, m,
                                  g->thr_v.as<uint32_t>(), g->hkey.as<int32_t>(), g->h_out.as<uint32_t>(),
                                  g->thrw_out.as<uint32_t>(), st);
    if (e != cudaSuccess) { release_tmp(); return bail(cuda_fail(c, e, "graph load")); }
    if ((s = set_model(g, model)) != IM_OK) { release_tmp(); return bail(s); }
    g->load_kind = model->kind;
    if (g->kind == kExplicit && m > 0) {
        if ((s = dalloc(c, (size_t)m * 4, g->thr_in)) != IM_OK) { release_tmp(); return bail(s); }
    }
    if (g->kind == kTrivalency) {
        if ((s = dalloc(c, (size_t)n * sizeof(int2), g->tri_b)) != IM_OK) { release_tmp(); return bail(s); }
    }
    // in-CSR sorted by (target, class, edge hash): rows of equal-threshold in-edges in hash order
    e = launch_build_in_csr(g->rp_out.as<int32_t>(), g->col_out.as<int32_t>(), n, m, g->kind,
                            g->dev.tri_seed, g->hkey.as<int32_t>(), g->thr_out.as<uint32_t>(),
                            g->src_in.as<int32_t>(), g->h_in.as<uint32_t>(), g->thr_in.as<uint32_t>(),
                            g->out_to_in.as<int32_t>(), g->rp_in.as<int32_t>(), g->tri_b.as<int2>(), tmp.p, st);
    // static vertex-ordered queue for dense levels (cnt and tmp reused as scratch)
    DBuf pos;
    if (e == cudaSuccess && (s = dalloc(c, ((size_t)n + 1) * 4, pos)) != IM_OK) { release_tmp(); return bail(s); }
    if (e == cudaSuccess)
        e = launch_dense_queue(g->rp_in.as<int32_t>(), n, g->thr_v.as<uint32_t>(), cnt.as<int32_t>(),
                               pos.as<int32_t>(), tmp.p, g->q_dense.as<QEntry>(), st);
    int32_t nd = 0, ndo = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nd, pos.as<int32_t>() + n, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // the same over the out-rows (dense cover levels)
    if (e == cudaSuccess)
        e = launch_dense_queue(g->rp_out.as<int32_t>(), n, nullptr, cnt.as<int32_t>(), pos.as<int32_t>(), tmp.p,
                               g->q_dense_out.as<QEntry>(), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ndo, pos.as<int32_t>() + n, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(c, pos);
    release_tmp();
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "graph load"));
    g->n_dense = nd;
    g->n_dense_out = ndo;
    g->dev.n = n;
    g->dev.m = m;
    g->dev.rp_out = g->rp_out.as<int32_t>();
    g->dev.col_out = g->col_out.as<int32_t>();
    g->dev.rp_in = g->rp_in.as<int32_t>();
    g->dev.src_in = g->src_in.as<int32_t>();
    g->dev.h_in = g->h_in.as<uint32_t>();
    g->dev.h_out = g->h_out.as<uint32_t>();
    g->dev.thrw_out = g->thrw_out.as<uint32_t>();
    g->dev.thr_v = g->thr_v.as<uint32_t>();
    g->dev.thr_out = g->thr_out.as<uint32_t>();
    g->dev.thr_in = g->thr_in.as<uint32_t>();
    g->dev.tri_b = g->tri_b.as<int2>();
    *out = g;
    return IM_OK;
}

extern "C" im_status im_graph_load(im_ctx* c, int32_t n, int64_t m, const int32_t* rowptr,
                                   const int32_t* col, const im_model* model, im_graph** out) {
    return graph_load_impl(c, n, m, rowptr, col, model, nullptr, out);
}

extern "C" void im_graph_free(im_graph* g) {
    if (!g) return;
    graph_release(g);
    delete g;
}

extern "C" im_status im_graph_info(const im_graph* g, int32_t* n, int64_t* m) {
    if (!g) return IM_E_INVAL;
    if (n) *n = g->n;
    if (m) *m = g->m;
    return IM_OK;
}

// ---------------------------------------------------------------------------
// sketches
// ---------------------------------------------------------------------------
// Device buffers of a sketch of J simulations over n vertices, with their
// sizes; sketch_alloc allocates exactly this list and query_bytes sums it.
using BufPlan = std::vector<std::pair<DBuf*, size_t>>;
static void sketch_plan(im_sketch* sk, int32_t n, int64_t m_edges, int32_t J, BufPlan& plan) {
    // the partials of a full pick at any J-tile width, or of a lazy pick
    const int pg = std::max({pick_grid(n, J, 1), pick_grid(n, J, 2), pick_grid(n, J, 4), pick_lazy_grid(n)});
    auto A = [&](DBuf& b, size_t bytes) { plan.emplace_back(&b, bytes); };
    A(sk->M, (size_t)n * J);
    A(sk->X, (size_t)J * 4);
    A(sk->salt, (size_t)J * 4);
    A(sk->tab, (size_t)kTabSize * 2);
    A(sk->ctr, (size_t)(kMaxLevels + 2) * 16);
    A(sk->claim, (size_t)(kMaxLevels + 2) * 4);
    for (int i = 0; i < 3; ++i) A(sk->chg[i], (size_t)n * ((J + 31) / 32) * 4);
    A(sk->gen, (size_t)n * 4);
    A(sk->seed_bits, (((size_t)n + 31) / 32) * 4);
    A(sk->count, 8);
    A(sk->part_S, (size_t)pg * 8);
    A(sk->part_u, (size_t)pg * 4);
    A(sk->ticket, 4);
    A(sk->stats, (size_t)kStCount * 8);
    A(sk->err, 4);
    A(sk->bar, 256);  // barrier words: arrivals, abort, levels; generation from byte 128
    A(sk->level_ns, (size_t)(kMaxLevels + 2) * 8);
    A(sk->fmt, (size_t)(kMaxLevels + 2));
    // incremental rebuilds: newly visited and affected register bits, the
    // affected vertices
    A(sk->nv, (size_t)n * ((J + 31) / 32) * 4);
    A(sk->aff, (size_t)n * ((J + 31) / 32) * 4);
    A(sk->alist, (size_t)n * 4);
    A(sk->aldeg, (size_t)n * 4);
    A(sk->aloff, ((size_t)n + 1) * 4);
    A(sk->almask, (size_t)n * 8);
    A(sk->ascan, scan_tmp_bytes(n));
    A(sk->acount, 4);
    A(sk->apctr, 16);
    A(sk->awl, (size_t)n * ((J + 31) / 32) * 4);
    A(sk->awlc, 4);
    A(sk->lb, (size_t)n * 8);
    A(sk->gsum, (size_t)pick_groups(n) * 32);
    A(sk->cand, 4);
    A(sk->part_S2, (size_t)pg * 8);
    A(sk->part_u2, (size_t)pg * 4);
    (void)m_edges;
}

// Edge-scan mode buffers: vertex queues (light and heavy, n entries each) and
// the live chunk masks of every in-edge and out-edge (chunks 32..63: J = 1024).
static void scan_plan(im_sketch* sk, int32_t n, int64_t m_edges, int32_t J, BufPlan& plan) {
    auto A = [&](DBuf& b, size_t bytes) { plan.emplace_back(&b, bytes); };
    for (int i = 0; i < 3; ++i) A(sk->ql[i], (size_t)n * sizeof(QEntry));
    for (int i = 0; i < 3; ++i) A(sk->qh[i], (size_t)n * sizeof(QEntry));
    const size_t m = (size_t)m_edges;
    A(sk->lcm_in_lo, m * 4);
    A(sk->lcm_out_lo, m * 4);
    if (J > 512) {
        A(sk->lcm_in_hi, m * 4);
        A(sk->lcm_out_hi, m * 4);
    }
}

// Bucket mode limits: at most kBucketEntriesPerEdge entries per edge on
// average in each orientation (else the sketch uses edge scans), and the
// bucket queues hold bucket_queue_cap entries.
constexpr int64_t kBucketEntriesPerEdge = 4;
static int64_t bucket_queue_cap(int32_t n) {
    const int64_t cap = std::max<int64_t>(8 * (int64_t)n, 1 << 20);
    return std::min<int64_t>(cap, 1 << 25);
}
// Device bytes bucket mode may take beyond the fixed plan (upper bound).
static uint64_t bucket_reserve_bytes(int32_t n, int64_t m, int32_t J) {
    const uint64_t nb = (uint64_t)n * (uint64_t)(J / 16);
    const uint64_t ents = (uint64_t)(kBucketEntriesPerEdge * m);
    uint64_t r = 0;
    for (int o = 0; o < 2; ++o)
        r += round_bytes((nb + 1) * 4) + round_bytes(std::max<uint64_t>(ents, 1) * 4) +
             round_bytes(std::max<uint64_t>(ents, 1) * 2);
    r += 3 * round_bytes((uint64_t)std::min<int64_t>(bucket_queue_cap(n), (int64_t)std::max<uint64_t>(nb, 1)) *
                         sizeof(QEntry));
    r += round_bytes(scan_tmp_bytes((int32_t)std::min<uint64_t>(nb, 0x7FFFFFFF))) + 256;
    r += 3 * round_bytes((size_t)n * ((J + 31) / 32) * 4);  // the cover's change masks
    return r;
}

// Frees every buffer of the plans, the bucket lists and the output buffers
// (null ones are skipped).
static void sketch_release(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    if (sk->fill_pending) {
        cudaStreamWaitEvent(c->stream, c->ev_join, 0);
        sk->fill_pending = false;
    }
    BufPlan plan;
    sketch_plan(sk, sk->g->n, sk->g->m, sk->J, plan);
    scan_plan(sk, sk->g->n, sk->g->m, sk->J, plan);
    for (auto& pb : plan) dfree(c, *pb.first);
    for (int o = 0; o < 2; ++o)
        for (DBuf* b : {&sk->bk_end[o], &sk->bk_other[o], &sk->bk_mask[o]}) dfree(c, *b);
    for (int i = 0; i < 3; ++i) dfree(c, sk->chg_cov[i]);
    for (DBuf* b : {&sk->out_seed, &sk->out_S, &sk->out_est}) dfree(c, *b);
}

// Output buffers for K seeds (ensure_out_cap): seed ids, S and estimates.
static int32_t out_cap_for(int32_t K) { return K < 64 ? 64 : K; }

static im_status sketch_alloc(im_ctx* c, im_graph* g, int32_t J, im_sketch** out) {
    if (!valid_J(J)) return fail(c, IM_E_INVAL, "J must be a power of two in [16, 1024], got %d", J);
    im_sketch* sk = new im_sketch();
    sk->g = g;
    sk->ctx = c;
    sk->J = J;
    BufPlan plan;
    sketch_plan(sk, g->n, g->m, J, plan);
    im_status s = IM_OK;
    for (auto& [b, bytes] : plan)
        if (s == IM_OK) s = dalloc(c, bytes, *b);
    if (s != IM_OK) {
        sketch_release(sk);
        delete sk;
        return s;
    }
    auto st = c->stream;
    cudaError_t e = cudaMemsetAsync(sk->gen.p, 0, sk->gen.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->seed_bits.p, 0, sk->seed_bits.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->count.p, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->ticket.p, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->stats.p, 0, sk->stats.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->err.p, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->nv.p, 0, sk->nv.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sk->aff.p, 0, sk->aff.bytes, st);
    if (e != cudaSuccess) {
        sketch_release(sk);
        delete sk;
        return cuda_fail(c, e, "sketch init");
    }
    *out = sk;
    return IM_OK;
}

static im_status ensure_out_cap(im_sketch* sk, int32_t K) {
    if (K <= sk->out_cap) return IM_OK;
    im_ctx* c = sk->ctx;
    const int32_t cap = out_cap_for(K);
    DBuf a, b, d;
    CKS(dalloc(c, (size_t)cap * 4, a));
    im_status s = dalloc(c, (size_t)cap * 8, b);
    if (s == IM_OK) s = dalloc(c, (size_t)cap * 8, d);
    if (s != IM_OK) { dfree(c, a); dfree(c, b); return s; }
    dfree(c, sk->out_seed);
    dfree(c, sk->out_S);
    dfree(c, sk->out_est);
    sk->out_seed = a;
    sk->out_S = b;
    sk->out_est = d;
    sk->out_cap = cap;
    return IM_OK;
}

static LevelArgs level_args(im_sketch* sk) {
    LevelArgs a{};
    a.M = sk->M.as<uint8_t>();
    a.J = sk->J;
    a.words = (sk->J + 31) / 32;
    a.X = sk->X.as<uint32_t>();
    a.tab = sk->tab.as<uint16_t>();
    a.gen = sk->gen.as<int32_t>();
    a.count = sk->count.as<unsigned long long>();
    a.stats = sk->stats.as<unsigned long long>();
    a.err = sk->err.as<uint32_t>();
    const im_tuning& t = sk->ctx->tuning;
    // the heavy path reads 32 register bytes per lane: J >= 32 only
    a.heavy_indeg = sk->J >= 32 ? t.heavy_indeg : 0x7FFFFFFF;
    a.light_batches = t.light_batches > 0 ? t.light_batches : 4;
    a.q_dense = sk->g->q_dense.as<QEntry>();
    a.n_dense = sk->g->n_dense;
    a.e_dense = sk->g->m;
    a.dense_div = sk->gflag ? 0 : t.dense_div;  // a batch build covers only some graphs
    a.dense_out = t.dense_out;
    a.dense_all = t.dense_all;
    a.gid = sk->gid;
    a.gcount = sk->gcount;
    a.gflag = sk->gflag;
    return a;
}

// Change-mask buffer i of a phase of this mode.
static DBuf& chg_buf(im_sketch* sk, int mode, int i) {
    return (sk->buckets && mode == kCover) ? sk->chg_cov[i] : sk->chg[i];
}

// Live chunk masks of the phase's edge orientation.
// Incremental rebuilds walk the affected words the search lists (instead of
// every vertex) when the pull queue cannot overflow and word ids fit 32 bits.
static bool words_list_ok(const im_sketch* sk) {
    return sk->buckets && sk->pull_safe && (uint64_t)sk->g->n * (uint64_t)((sk->J + 31) / 32) < (1ull << 32);
}

static void set_lcm(LevelArgs& a, const im_sketch* sk, int mode) {
    const bool in = mode != kCover;
    a.aff = sk->aff.as<uint32_t>();
    // the affected-set search lists the words it makes nonzero (bucket mode;
    // a word is listed as v * words + w in 32 bits)
    const bool words = mode == kAffect && words_list_ok(sk);
    a.awl = words ? sk->awl.as<uint32_t>() : nullptr;
    a.awl_count = words ? sk->awlc.as<unsigned int>() : nullptr;
    a.nv = (mode == kCover && sk->incr) ? sk->nv.as<uint32_t>() : nullptr;
    a.lcm_lo = (in ? sk->lcm_in_lo : sk->lcm_out_lo).as<uint32_t>();
    if (mode == kCover) {
        // dense cover levels walk every vertex's out-row
        a.q_dense = sk->g->q_dense_out.as<QEntry>();
        a.n_dense = sk->g->n_dense_out;
        a.e_dense = sk->g->m;
    }
    a.lcm_hi = sk->J > 512 ? (in ? sk->lcm_in_hi : sk->lcm_out_hi).as<uint32_t>() : nullptr;
    a.chunks = sk->J / 16;
    a.nbuckets = (int64_t)sk->g->n * (sk->J / 16);
    a.bq_cap = sk->bq_cap;
    a.vq_cap = sk->g->n;
    // a level appends at most one bucket per processed entry (fewer than m):
    // below 2^26 - 2^22 edges the packed counter's count field cannot overflow
    a.bq_guard = sk->g->m >= (int64_t)((1 << 26) - (1 << 22)) ? 1 : 0;
    a.bucket_div = sk->buckets ? sk->ctx->tuning.buckets : 0;
    a.chain = sk->ctx->tuning.chain;
    if (sk->buckets) {
        const int o = in ? 0 : 1;
        a.bk_end = sk->bk_end[o].as<uint32_t>();
        a.bk_other = sk->bk_other[o].as<int32_t>();
        a.bk_mask = sk->bk_mask[o].as<uint16_t>();
    } else {
        a.bk_end = nullptr;
        a.bk_other = nullptr;
        a.bk_mask = nullptr;
    }
}

// Reads the device error word; converts raised bits to a status.
static im_status check_err(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    uint32_t err = 0;
    CK(c, cudaMemcpyAsync(&err, sk->err.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(c, sync_collect(c));
    if (err & kErrQueue) return fail(c, IM_E_STATE, "frontier queue overflow");
    if (err & kErrCasLimit) return fail(c, IM_E_TIMEOUT, "register CAS retry limit exceeded");
    if (err & kErrBarrier) return fail(c, IM_E_TIMEOUT, "grid barrier wait exceeded its time limit");
    if (err & kErrLevels) return fail(c, IM_E_TIMEOUT, "frontier did not empty within %d levels", c->max_levels);
    if (err & kErrBounds) return fail(c, IM_E_STATE, "device index out of bounds (bounds-checked build)");
    return IM_OK;
}

// Start of a propagation or cover phase: level counters and work counters
// back to zero.  A phase that completes leaves its change masks zero (the
// last level's bits are cleared by the phase itself); after a new sketch or a
// failed phase they are cleared here.
static im_status phase_begin(im_sketch* sk, int mode, int fmt0 = -1) {
    im_ctx* c = sk->ctx;
    auto st = c->stream;
    CK(c, cudaMemsetAsync(sk->ctr.p, 0, sk->ctr.bytes, st));
    // the level-0 queue: bucket entries (fmt0 = 1, or by default for a cover
    // in bucket mode: the seed kernel writes them), vertex entries otherwise
    if (fmt0 < 0) fmt0 = (mode == kCover && sk->buckets) ? 1 : 0;
    CK(c, cudaMemsetAsync(sk->fmt.p, fmt0, 1, st));
    CK(c, cudaMemsetAsync(sk->claim.p, 0, sk->claim.bytes, st));
    if (sk->chg_dirty) {
        for (int i = 0; i < 3; ++i) CK(c, cudaMemsetAsync(sk->chg[i].p, 0, sk->chg[i].bytes, st));
        for (int i = 0; i < 3; ++i)
            if (sk->chg_cov[i].p) CK(c, cudaMemsetAsync(sk->chg_cov[i].p, 0, sk->chg_cov[i].bytes, st));
        sk->chg_dirty = false;
    }
    CK(c, cudaMemsetAsync(sk->bar.p, 0, sk->bar.bytes, st));
    return IM_OK;
}

// All levels of a phase in one cooperative launch.  Inside a selection
// (sk->defer) nothing is read back: the host queues the next work at once and
// reads the error word at the end; otherwise (step-level calls, tracing) the
// host reads the level count and the error word after the launch.
static im_status run_phase_persistent(im_sketch* sk, int mode, bool all_first, int grid) {
    im_ctx* c = sk->ctx;
    auto st = c->stream;
    PhaseArgs p{};
    p.base = level_args(sk);
    set_lcm(p.base, sk, mode);
    for (int i = 0; i < 3; ++i) {
        p.ql[i] = sk->ql[i].as<QEntry>();
        p.qh[i] = sk->qh[i].as<QEntry>();
        p.chg[i] = chg_buf(sk, mode, i).as<uint32_t>();
    }
    p.ctr = sk->ctr.as<ulonglong2>();
    p.claim = sk->claim.as<unsigned int>();
    p.all_first = all_first ? 1 : 0;
    p.max_levels = c->max_levels;
    p.gen_base = sk->gen_counter + 1;
    unsigned int* bar = sk->bar.as<unsigned int>();
    // the generation word (polled by the waiting blocks) on its own 128-byte
    // line, away from the arrival counter
    p.bar_arrive = bar;
    p.abort_flag = bar + 2;
    p.levels_out = reinterpret_cast<int*>(bar + 3);
    p.bar_gen = bar + 32;
    p.limit_ns = c->barrier_limit_ns;
    p.level_ns = c->trace ? sk->level_ns.as<unsigned long long>() : nullptr;
    p.fmt = sk->fmt.as<uint8_t>();
    CK(c, timed(c, mode == kPush ? kTPush : kTCover,
                [&] { return launch_phase(sk->kind, mode, sk->dev, p, grid, st); }));
    // stamps gen_base .. gen_base + max_levels are this phase's
    sk->gen_counter += kMaxLevels;
    if (sk->gen_counter > (1 << 30)) {
        CK(c, cudaMemsetAsync(sk->gen.p, 0, sk->gen.bytes, st));
        sk->gen_counter = 0;
    }
    if (sk->defer && !c->trace) {
        sk->chg_dirty = false;  // a failed phase fails the whole selection
        return IM_OK;
    }
    CK(c, cudaMemcpyAsync(c->pinned, bar, 16, cudaMemcpyDeviceToHost, st));
    CK(c, sync_collect(c));
    const unsigned int* hb = reinterpret_cast<const unsigned int*>(c->pinned);
    const int levels = (int)hb[3];
    sk->chg_dirty = true;
    if (c->trace && levels > 0 && levels < p.max_levels) {
        // per-level records from the in-kernel clock (one launch for all levels)
        std::vector<ulonglong2> h((size_t)levels);
        std::vector<unsigned long long> ns((size_t)levels + 1);
        CK(c, cudaMemcpyAsync(h.data(), sk->ctr.p, (size_t)levels * 16, cudaMemcpyDeviceToHost, st));
        CK(c, cudaMemcpyAsync(ns.data(), sk->level_ns.p, ((size_t)levels + 1) * 8, cudaMemcpyDeviceToHost, st));
        CK(c, sync_collect(c));
        for (int l = 0; l < levels; ++l) {
            im_trace_rec r{};
            r.kind = mode;
            r.level = l;
            r.count = (int64_t)(h[l].x >> kCountShift) + (int64_t)(h[l].y >> kCountShift);
            r.edges = (int64_t)(h[l].x & kEdgeMask) + (int64_t)(h[l].y & kEdgeMask);
            r.ms = (double)(ns[l + 1] - ns[l]) * 1e-6;
            c->recs.push_back(r);
        }
    }
    if (levels >= p.max_levels)
        return fail(c, IM_E_TIMEOUT, "frontier did not empty within %d levels", p.max_levels);
    CKS(check_err(sk));
    sk->chg_dirty = false;
    return IM_OK;
}

// Runs frontier levels until both queues are empty.  Level t reads queue
// t % 3 with counters ctr[t], writes queue (t+1) % 3 with counters ctr[t+1],
// and clears the change bits of queue (t+2) % 3 (read by level t-1).  The host
// reads the newest counters every `check` levels; levels launched after the
// queues emptied see empty queues and return at once.
static im_status run_levels(im_sketch* sk, int mode, bool all_first) {
    im_ctx* c = sk->ctx;
    auto st = c->stream;
    if (c->tuning.persistent) {
        // one cooperative grid of every resident block (at most 2048)
        const int pgrid = std::min(phase_grid(), 64 * 32);
        if (pgrid > 0) return run_phase_persistent(sk, mode, all_first, pgrid);
    }
    ulonglong2* ctr = sk->ctr.as<ulonglong2>();
    unsigned int* claim = sk->claim.as<unsigned int>();
    LevelArgs a = level_args(sk);
    set_lcm(a, sk, mode);
    const int grid = c->tuning.grid_blocks > 0 ? c->tuning.grid_blocks : level_grid();
    int check = c->tuning.check_every > 0 ? c->tuning.check_every : 2;
    int64_t t = 0;
    const int64_t seq0 = c->seq;
    for (;;) {
        const int bi = (int)(t % 3), bo = (int)((t + 1) % 3), bp = (int)((t + 2) % 3);
        a.ql_in = sk->ql[bi].as<QEntry>();
        a.cl_in = &ctr[t].x;
        a.qh_in = sk->qh[bi].as<QEntry>();
        a.ch_in = &ctr[t].y;
        a.ql_out = sk->ql[bo].as<QEntry>();
        a.cl_out = &ctr[t + 1].x;
        a.qh_out = sk->qh[bo].as<QEntry>();
        a.ch_out = &ctr[t + 1].y;
        if (t >= 1) {
            a.ql_prev = sk->ql[bp].as<QEntry>();
            a.cl_prev = &ctr[t - 1].x;
            a.qh_prev = sk->qh[bp].as<QEntry>();
            a.ch_prev = &ctr[t - 1].y;
            a.chg_prev = chg_buf(sk, mode, bp).as<uint32_t>();
        } else {
            a.ql_prev = nullptr; a.cl_prev = nullptr; a.qh_prev = nullptr; a.ch_prev = nullptr;
            a.chg_prev = nullptr;
        }
        a.chg_cur = chg_buf(sk, mode, bi).as<uint32_t>();
        a.chg_next = chg_buf(sk, mode, bo).as<uint32_t>();
        a.all_changed = (t == 0 && all_first) ? 1 : 0;
        a.claim = claim + t;
        a.gen_next = ++sk->gen_counter;
        a.fmt_in = sk->fmt.as<uint8_t>() + t;
        a.fmt_out = sk->fmt.as<uint8_t>() + t + 1;
        a.fmt_prev = t >= 1 ? sk->fmt.as<uint8_t>() + t - 1 : nullptr;
        CK(c, timed(c, mode == kPush ? kTPush : kTCover,
                    [&] { return launch_level(sk->kind, mode, sk->dev, a, grid, st); }));
        ++t;
        if (t % check == 0) {
            CK(c, cudaMemcpyAsync(c->pinned, &ctr[t], 16, cudaMemcpyDeviceToHost, st));
            CK(c, sync_collect(c));
            if ((c->pinned[0] >> kCountShift) == 0 && (c->pinned[1] >> kCountShift) == 0) break;
            if (t >= c->max_levels || t + 16 >= kMaxLevels) {
                sk->chg_dirty = true;
                return fail(c, IM_E_TIMEOUT, "frontier did not empty within %d levels", (int)t);
            }
            if (check < 8) check *= 2;
        }
    }
    {
        // one more level on the empty queue t: it only clears the change bits
        // of queue t - 1, so the phase leaves every change mask zero
        const int bi = (int)(t % 3), bo = (int)((t + 1) % 3), bp = (int)((t + 2) % 3);
        a.ql_in = sk->ql[bi].as<QEntry>();
        a.cl_in = &ctr[t].x;
        a.qh_in = sk->qh[bi].as<QEntry>();
        a.ch_in = &ctr[t].y;
        a.ql_prev = sk->ql[bp].as<QEntry>();
        a.cl_prev = &ctr[t - 1].x;
        a.qh_prev = sk->qh[bp].as<QEntry>();
        a.ch_prev = &ctr[t - 1].y;
        a.chg_prev = chg_buf(sk, mode, bp).as<uint32_t>();
        a.chg_cur = chg_buf(sk, mode, bi).as<uint32_t>();
        a.chg_next = chg_buf(sk, mode, bo).as<uint32_t>();
        a.all_changed = 0;
        a.claim = claim + t;
        a.gen_next = ++sk->gen_counter;
        a.fmt_in = sk->fmt.as<uint8_t>() + t;
        a.fmt_out = sk->fmt.as<uint8_t>() + t + 1;
        a.fmt_prev = sk->fmt.as<uint8_t>() + t - 1;
        CK(c, timed(c, mode == kPush ? kTPush : kTCover,
                    [&] { return launch_level(sk->kind, mode, sk->dev, a, grid, st); }));
    }
    if (c->trace) {
        std::vector<ulonglong2> h((size_t)t);
        CK(c, cudaMemcpyAsync(h.data(), ctr, (size_t)t * 16, cudaMemcpyDeviceToHost, st));
        CK(c, sync_collect(c));
        for (int64_t l = 0; l < t; ++l) {
            im_trace_rec r{};
            r.kind = mode;
            r.level = (int32_t)l;
            r.count = (int64_t)(h[l].x >> kCountShift) + (int64_t)(h[l].y >> kCountShift);
            r.edges = (int64_t)(h[l].x & kEdgeMask) + (int64_t)(h[l].y & kEdgeMask);
            const int64_t q = seq0 + l;
            r.ms = q < (int64_t)c->launch_ms.size() ? c->launch_ms[q] : 0.0;
            c->recs.push_back(r);
        }
    }
    sk->chg_dirty = true;
    CKS(check_err(sk));
    sk->chg_dirty = false;
    return IM_OK;
}

static im_status propagate(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    CKS(phase_begin(sk, kPush));
    LevelArgs a = level_args(sk);
    ulonglong2* ctr = sk->ctr.as<ulonglong2>();
    a.ql_out = sk->ql[0].as<QEntry>();
    a.cl_out = &ctr[0].x;
    a.qh_out = sk->qh[0].as<QEntry>();
    a.ch_out = &ctr[0].y;
    CK(c, timed(c, kTOther, [&] { return launch_init_queues(sk->kind, sk->dev, a, c->stream); }));
    return run_levels(sk, kPush, true);
}

// Incremental rebuild (same registers as build_registers after covers):
// affected-set search from the registers visited since the last build, reset
// and pull of the affected registers, propagation from them.
static im_status incremental_rebuild(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    auto st = c->stream;
    ulonglong2* ctr = sk->ctr.as<ulonglong2>();
    IncrArgs x{};
    x.nv = sk->nv.as<uint32_t>();
    x.salt = sk->salt.as<uint32_t>();
    x.hkey = sk->g->hkey.as<int32_t>();
    x.list = sk->alist.as<int32_t>();
    x.ldeg = sk->aldeg.as<int32_t>();
    x.loff = sk->aloff.as<int32_t>();
    x.lmask = sk->almask.as<uint2>();
    x.list_count = sk->acount.as<unsigned int>();
    x.buckets = sk->buckets ? 1 : 0;
    // the pull queue: the third light queue, free between phases
    x.pq = sk->ql[2].as<QEntry>();
    x.pctr = sk->apctr.as<unsigned long long>();
    x.words_list = words_list_ok(sk) ? 1 : 0;
    x.awl = sk->awl.as<uint32_t>();
    x.awl_count = sk->awlc.as<unsigned int>();
    if (x.words_list) CK(c, cudaMemsetAsync(sk->awlc.p, 0, 4, st));
    // 1. the affected registers (level 0 in bucket format where the sketch
    // has bucketed lists)
    CKS(phase_begin(sk, kAffect, x.buckets));
    LevelArgs a = level_args(sk);
    set_lcm(a, sk, kAffect);
    a.ql_out = sk->ql[0].as<QEntry>();
    a.cl_out = &ctr[0].x;
    a.qh_out = sk->qh[0].as<QEntry>();
    a.ch_out = &ctr[0].y;
    a.chg_next = chg_buf(sk, kAffect, 0).as<uint32_t>();
    CK(c, timed(c, kTOther, [&] { return launch_incremental(0, sk->kind, sk->dev, a, x, st); }));
    CKS(run_levels(sk, kAffect, false));
    // 2. reset to the own ranks, list of affected vertices (and their
    // affected chunks' out-buckets); 3. pull over their out-edges
    LevelArgs b = level_args(sk);
    set_lcm(b, sk, kCover);
    CK(c, cudaMemsetAsync(x.list_count, 0, 4, st));
    CK(c, cudaMemsetAsync(x.pctr, 0, 16, st));
    CK(c, timed(c, kTFill, [&] { return launch_incremental(1, sk->kind, sk->dev, b, x, st); }));
    if (sk->buckets && sk->pull_safe) {
        // the pull reads its queue's counters on the device
        x.pull_buckets = 1;
    } else {
        CK(c, cudaMemcpyAsync(c->pinned, x.list_count, 4, cudaMemcpyDeviceToHost, st));
        CK(c, cudaMemcpyAsync(c->pinned + 1, x.pctr, 16, cudaMemcpyDeviceToHost, st));
        CK(c, sync_collect(c));
        x.count = (int32_t)(uint32_t)c->pinned[0];
        const int64_t npull = (int64_t)(c->pinned[1] >> kCountShift);
        x.pull_buckets = sk->buckets && c->pinned[2] == 0 && npull <= sk->bq_cap ? 1 : 0;
    }
    if (x.pull_buckets || x.count > 0) {
        // timed with the reset (both rebuild registers from their own ranks)
        CK(c, timed(c, kTFill, [&] {
            if (!x.pull_buckets) {
                cudaError_t e = launch_exclusive_scan(x.ldeg, x.count, sk->aloff.as<int32_t>(), sk->ascan.p, st);
                if (e != cudaSuccess) return e;
            }
            return launch_incremental(2, sk->kind, sk->dev, b, x, st);
        }));
    }
    // 4. propagation from the affected registers
    CKS(phase_begin(sk, kPush, x.buckets));
    LevelArgs p = level_args(sk);
    set_lcm(p, sk, kPush);
    p.ql_out = sk->ql[0].as<QEntry>();
    p.cl_out = &ctr[0].x;
    p.qh_out = sk->qh[0].as<QEntry>();
    p.ch_out = &ctr[0].y;
    p.chg_next = chg_buf(sk, kPush, 0).as<uint32_t>();
    CK(c, timed(c, kTOther, [&] { return launch_incremental(3, sk->kind, sk->dev, p, x, st); }));
    CKS(run_levels(sk, kPush, false));
    // 5. the next rebuild starts from what covers visit after this one
    CK(c, cudaMemsetAsync(sk->nv.p, 0, sk->nv.bytes, st));
    CK(c, cudaMemsetAsync(sk->aff.p, 0, sk->aff.bytes, st));
    return IM_OK;
}

// Fill (Alg. 1) of the non-visited registers, then Simulate to the fixpoint.
static im_status build_registers(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    if (sk->fill_pending) {
        // the first fill ran on the side stream (sketch_start)
        CK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        sk->fill_pending = false;
    } else {
        CK(c, timed(c, kTFill, [&] {
            return launch_fill(sk->M.as<uint8_t>(), sk->g->n, sk->J, sk->salt.as<uint32_t>(), sk->fresh, c->stream);
        }));
    }
    sk->fresh = false;
    // every stored S_u stays a lower bound, but after a full build every row
    // is stale for a lazy pick: the next pick reads every row in one pass
    sk->lb_ready = false;
    return propagate(sk);
}

static void stats_begin(im_ctx* c) {
    memset(&c->stats, 0, sizeof c->stats);
    c->ev_used = 0;
    c->seq = 0;
    c->recs.clear();
    c->launch_ms.clear();
}

static im_status stats_collect(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    unsigned long long h[kStCount];
    unsigned long long cnt = 0;
    CK(c, cudaMemcpyAsync(h, sk->stats.p, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&cnt, sk->count.p, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(c, sync_collect(c));
    im_stats& s = c->stats;
    s.sweeps = (int64_t)h[kStSweepLevels];
    s.cover_levels = (int64_t)h[kStCoverLevels];
    s.sweep_vertices = h[kStSweepVertices];
    s.sweep_edges = h[kStSweepEdges];
    s.sweep_chunks = h[kStSweepChunks];
    s.sweep_cas = h[kStSweepCas];
    s.sweep_changed = h[kStSweepChanged];
    s.cover_edges = h[kStCoverEdges];
    s.cover_chunks = h[kStCoverChunks];
    s.visited = cnt;
    s.sweep_heavy = h[kStSweepHeavy];
    s.sweep_heavy_sims = h[kStSweepHeavySims];
    s.sweep_batches = h[kStSweepBatches];
    s.sweep_dealt = h[kStSweepDealt];
    s.sweep_edges_live = h[kStSweepLiveEdges];
    s.sweep_buckets = h[kStSweepBuckets];
    s.sweep_bucket_entries = h[kStSweepBucketEntries];
    s.affected = h[kStAffected];
    s.pull_buckets = h[kStPullBuckets];
    s.pull_entries = h[kStPullEntries];
    s.sweep_changed_buckets = h[kStSweepChangedBuckets];
    s.pick_refreshed = h[kStPickRefreshed];
    // algorithmic bytes of the sweeps: queue entry (16 B) + the queued vertex's
    // register row (J B) per queued vertex; live chunk mask (4 B, 8 B when
    // J = 1024) per in-edge; source id + edge hash (8 B, + 4 B threshold for
    // explicit weights) per in-edge live in a changed chunk; source + target
    // 16-byte pieces per chunk with a live non-visited source register; one
    // 4-byte word per CAS write
    const uint64_t t = sk->kind == kExplicit ? 4 : 0;
    const uint64_t lw = sk->J > 512 ? 8 : 4;
    // levels on vertex queues, plus levels on bucket queues: per queued
    // bucket its 16-byte entry; per processed list entry its endpoint and
    // live mask (6 B) and the source and target 16-byte register pieces
    s.alg_bytes_sweep = s.sweep_vertices * (16 + (uint64_t)sk->J) + s.sweep_edges * lw +
                        s.sweep_edges_live * (8 + t) + s.sweep_chunks * 32 + s.sweep_cas * 4 +
                        s.sweep_buckets * 16 + s.sweep_bucket_entries * (6 + 32);
    return IM_OK;
}

// Edge-scan mode: vertex queues and the live chunk masks of every edge.
static im_status build_scan_mode(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    const int32_t J = sk->J;
    BufPlan plan;
    scan_plan(sk, sk->g->n, sk->g->m, J, plan);
    for (auto& [b, bytes] : plan) CKS(dalloc(c, bytes, *b));
    // an edge's live chunks are the same in both orientations: computed over
    // the in-edges (rows sorted by edge hash, so a warp's candidate ranges
    // agree), then gathered into out-CSR order
    CK(c, timed(c, kTOther, [&] {
        return launch_live_chunks(sk->kind, kPush, sk->dev, sk->X.as<uint32_t>(), sk->tab.as<uint16_t>(), J,
                                  sk->lcm_in_lo.as<uint32_t>(), J > 512 ? sk->lcm_in_hi.as<uint32_t>() : nullptr,
                                  c->stream);
    }));
    const int32_t* o2i = sk->g->out_to_in.as<int32_t>();
    CK(c, timed(c, kTOther, [&] {
        cudaError_t e = launch_gather_u32(sk->lcm_in_lo.as<uint32_t>(), o2i, sk->g->m, sk->lcm_out_lo.as<uint32_t>(),
                                          c->stream);
        if (e == cudaSuccess && J > 512)
            e = launch_gather_u32(sk->lcm_in_hi.as<uint32_t>(), o2i, sk->g->m, sk->lcm_out_hi.as<uint32_t>(), c->stream);
        return e;
    }));
    return IM_OK;
}

// Bucket mode: count bucket sizes, scan, place every live (edge, chunk)
// entry; bucket queues of bq_cap entries.  Leaves sk->buckets false (and
// nothing allocated) when the lists would exceed their memory bound.
static im_status build_buckets(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    auto st = c->stream;
    const int32_t n = sk->g->n, J = sk->J, C = J / 16;
    const int64_t m = sk->g->m;
    const int64_t nb = (int64_t)n * C;
    if (nb + 1 > 0x7FFFFFFF || m == 0) return IM_OK;
    DBuf tmp, ne;
    auto drop = [&]() {
        dfree(c, tmp);
        dfree(c, ne);
        for (int o = 0; o < 2; ++o)
            for (DBuf* b : {&sk->bk_end[o], &sk->bk_other[o], &sk->bk_mask[o]}) dfree(c, *b);
        (void)cudaGetLastError();
    };
    im_status s = IM_OK;
    for (int o = 0; o < 2 && s == IM_OK; ++o) s = dalloc(c, (size_t)(nb + 1) * 4, sk->bk_end[o]);
    if (s == IM_OK) s = dalloc(c, scan_tmp_bytes((int32_t)nb), tmp);
    if (s == IM_OK) s = dalloc(c, 16, ne);
    if (s != IM_OK) { drop(); return IM_OK; }  // no room: edge scans
    cudaError_t e = cudaMemsetAsync(ne.p, 0, 16, st);
    for (int o = 0; o < 2 && e == cudaSuccess; ++o) {
        e = cudaMemsetAsync(sk->bk_end[o].p, 0, sk->bk_end[o].bytes, st);
        if (e == cudaSuccess)
            e = timed(c, kTOther, [&] {
                return launch_buckets(0, sk->kind, o == 0 ? kPush : kCover, sk->dev, sk->X.as<uint32_t>(),
                                      sk->tab.as<uint16_t>(), J, sk->bk_end[o].as<uint32_t>(),
                                      ne.as<unsigned long long>() + o, nullptr, nullptr, st);
            });
    }
    int64_t total[2] = {0, 0};
    unsigned long long nonempty[2] = {0, 0};
    for (int o = 0; o < 2 && e == cudaSuccess; ++o) {
        int32_t* cnt = reinterpret_cast<int32_t*>(sk->bk_end[o].p);
        e = launch_exclusive_scan(cnt, (int32_t)nb, cnt, tmp.p, st);
        // the scan's 64-bit total is the last tile-sum slot
        const size_t slots = scan_tmp_bytes((int32_t)nb) / 8;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&total[o], tmp.as<int64_t>() + slots - 1, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(nonempty, ne.p, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { drop(); return cuda_fail(c, e, "bucket count"); }
    for (int o = 0; o < 2; ++o)
        if (total[o] > kBucketEntriesPerEdge * m || total[o] >= 0x7FFFFFFF) { drop(); return IM_OK; }
    for (int o = 0; o < 2 && s == IM_OK; ++o) {
        s = dalloc(c, (size_t)std::max<int64_t>(total[o], 1) * 4, sk->bk_other[o]);
        if (s == IM_OK) s = dalloc(c, (size_t)std::max<int64_t>(total[o], 1) * 2, sk->bk_mask[o]);
    }
    if (s != IM_OK) { drop(); return IM_OK; }
    for (int o = 0; o < 2 && e == cudaSuccess; ++o)
        e = timed(c, kTOther, [&] {
            return launch_buckets(1, sk->kind, o == 0 ? kPush : kCover, sk->dev, sk->X.as<uint32_t>(),
                                  sk->tab.as<uint16_t>(), J, sk->bk_end[o].as<uint32_t>(), nullptr,
                                  sk->bk_other[o].as<int32_t>(), sk->bk_mask[o].as<uint16_t>(), st);
        });
    if (e != cudaSuccess) { drop(); return cuda_fail(c, e, "bucket fill"); }
    dfree(c, tmp);
    dfree(c, ne);
    const int64_t most = (int64_t)std::max(nonempty[0], nonempty[1]);
    const int64_t cap = std::max<int64_t>(1, std::min(bucket_queue_cap(n), most));
    // the light queues hold vertex entries (n at most) or bucket entries
    DBuf nq[3];
    if (cap > n)
        for (int i = 0; i < 3 && s == IM_OK; ++i) s = dalloc(c, (size_t)cap * sizeof(QEntry), nq[i]);
    for (int i = 0; i < 3 && s == IM_OK; ++i) s = dalloc(c, sk->chg[i].bytes, sk->chg_cov[i]);
    if (s != IM_OK) {
        for (int i = 0; i < 3; ++i) { dfree(c, nq[i]); dfree(c, sk->chg_cov[i]); }
        drop();
        return IM_OK;
    }
    if (cap > n)
        for (int i = 0; i < 3; ++i) {
            dfree(c, sk->ql[i]);
            sk->ql[i] = nq[i];
        }
    sk->chg_dirty = true;  // the new buffers start zeroed by the next phase
    sk->bq_cap = (int32_t)cap;
    sk->pull_safe = cap >= (int64_t)nonempty[1];
    sk->buckets = true;
    return IM_OK;
}

// New sketch: buffers, the J simulations, the model words (the graph's, or
// `model` for this call) and the live chunk masks of every edge.
// prefill: the caller builds the registers next (im_sketch_build, a
// selection): the first fill is issued on the side stream right after the
// simulations are drawn, next to the live chunk masks, which do not read the
// registers.
static im_status sketch_start(im_ctx* c, im_graph* g, int32_t J, uint64_t seed, const im_model* model,
                              bool prefill, im_sketch** out) {
    CK(c, cudaSetDevice(c->device));
    im_sketch* sk = nullptr;
    CKS(sketch_alloc(c, g, J, &sk));
    sk->dev = g->dev;
    sk->kind = g->kind;
    if (model) model_words(sk->dev, sk->kind, model);  // this call's model, on the sketch's copy
    keep_class_bounds(sk->dev, sk->kind, g);
    cudaError_t e = timed(c, kTOther, [&] {
        return launch_sims(seed, J, sk->X.as<uint32_t>(), sk->salt.as<uint32_t>(),
                           sk->tab.as<uint16_t>(), c->stream);
    });
    if (e == cudaSuccess && prefill && sk->fresh) {
        e = ensure_side(c);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        if (e == cudaSuccess)
            e = timed_on(c, c->side, kTFill, [&] {
                return launch_fill(sk->M.as<uint8_t>(), g->n, J, sk->salt.as<uint32_t>(), true, c->side);
            });
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
        if (e == cudaSuccess) sk->fill_pending = true;
    }
    if (e != cudaSuccess) {
        sketch_release(sk);
        delete sk;
        return cuda_fail(c, e, "sketch setup");
    }
    im_status s = build_scan_mode(sk);
    if (s == IM_OK && c->tuning.buckets) s = build_buckets(sk);
    if (s != IM_OK) {
        sketch_release(sk);
        delete sk;
        return s;
    }
    *out = sk;
    return IM_OK;
}

extern "C" im_status im_sketch_build(im_graph* g, int32_t J, uint64_t seed, im_sketch** out) {
    if (!g || !out) return IM_E_INVAL;
    im_ctx* c = g->ctx;
    stats_begin(c);
    const double t0 = now_ms();
    im_sketch* sk = nullptr;
    CKS(sketch_start(c, g, J, seed, nullptr, true, &sk));
    im_status s = build_registers(sk);
    if (s == IM_OK) s = stats_collect(sk);
    if (s != IM_OK) {
        sketch_release(sk);
        delete sk;
        return s;
    }
    c->stats.builds = 1;
    c->stats.ms_build = c->stats.ms_total = now_ms() - t0;
    *out = sk;
    return IM_OK;
}

extern "C" void im_sketch_free(im_sketch* sk) {
    if (!sk) return;
    sketch_release(sk);
    delete sk;
}

extern "C" im_status im_sketch_registers(const im_sketch* sk, uint8_t* host_out) {
    if (!sk || !host_out) return IM_E_INVAL;
    im_ctx* c = sk->ctx;
    CK(c, cudaMemcpyAsync(host_out, sk->M.p, (size_t)sk->g->n * sk->J, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

extern "C" im_status im_sketch_set_registers(im_sketch* sk, const uint8_t* host_in) {
    if (!sk || !host_in) return IM_E_INVAL;
    im_ctx* c = sk->ctx;
    const size_t bytes = (size_t)sk->g->n * sk->J;
    for (size_t i = 0; i < bytes; ++i)
        if (host_in[i] > 32 && host_in[i] != 0xFF)
            return fail(c, IM_E_INVAL, "register byte %zu = %u is neither a rank nor 0xFF", i, host_in[i]);
    CK(c, cudaMemcpyAsync(sk->M.p, host_in, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemsetAsync(sk->count.p, 0, 8, c->stream));
    CK(c, launch_count_visited(sk->M.as<uint8_t>(), (int64_t)bytes, sk->count.as<unsigned long long>(), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

extern "C" im_status im_sketch_sims(const im_sketch* sk, uint32_t* X_out, uint32_t* salt_out) {
    if (!sk) return IM_E_INVAL;
    im_ctx* c = sk->ctx;
    if (X_out) CK(c, cudaMemcpyAsync(X_out, sk->X.p, (size_t)sk->J * 4, cudaMemcpyDeviceToHost, c->stream));
    if (salt_out) CK(c, cudaMemcpyAsync(salt_out, sk->salt.p, (size_t)sk->J * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return IM_OK;
}

extern "C" im_status im_sketch_sums(const im_sketch* sk, uint64_t* host_out) {
    if (!sk || !host_out) return IM_E_INVAL;
    im_ctx* c = sk->ctx;
    DBuf S;
    CKS(dalloc(c, (size_t)sk->g->n * 8, S));
    cudaError_t e = launch_sums(sk->M.as<uint8_t>(), sk->g->n, sk->J, S.as<unsigned long long>(), c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, S.p, (size_t)sk->g->n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, S);
    if (e != cudaSuccess) return cuda_fail(c, e, "sketch sums");
    return IM_OK;
}

static PickArgs pick_args(im_sketch* sk, int k) {
    PickArgs a{};
    a.M = sk->M.as<uint8_t>();
    a.J = sk->J;
    a.n = sk->g->n;
    a.seed_bits = sk->seed_bits.as<uint32_t>();
    a.part_S = sk->part_S.as<unsigned long long>();
    a.part_u = sk->part_u.as<int32_t>();
    a.ticket = sk->ticket.as<unsigned int>();
    a.out_seed = sk->out_seed.as<int32_t>();
    a.out_S = sk->out_S.as<unsigned long long>();
    a.out_est = sk->out_est.as<double>();
    a.k = k;
    a.rp_out = sk->g->rp_out.as<int32_t>();
    a.q_cover = sk->ql[0].as<QEntry>();
    a.ctr_cover = &sk->ctr.as<ulonglong2>()[0].x;
    a.chg0 = chg_buf(sk, kCover, 0).as<uint32_t>();
    a.count = sk->count.as<unsigned long long>();
    a.mark = 1;
    a.bk_end_out = sk->buckets ? sk->bk_end[1].as<uint32_t>() : nullptr;
    a.chunks = sk->J / 16;
    a.nv = sk->incr ? sk->nv.as<uint32_t>() : nullptr;
    a.tile = sk->ctx->tuning.pick_tile;
    a.stats = sk->stats.as<unsigned long long>();
    return a;
}

// Pick (estimate + argmax) followed by the cover of the picked vertex.  In
// a lazy sketch the first pick stores every S_u and later picks refresh only
// the stored sums that could beat the candidate.
static im_status pick_and_cover(im_sketch* sk, int k) {
    im_ctx* c = sk->ctx;
    CKS(phase_begin(sk, kCover));
    PickArgs a = pick_args(sk, k);
    if (sk->lazy) {
        a.lb = sk->lb.as<unsigned long long>();
        a.cand = sk->cand.as<int32_t>();
        a.part_S2 = sk->part_S2.as<unsigned long long>();
        a.part_u2 = sk->part_u2.as<int32_t>();
        a.gsum = sk->gsum.as<unsigned long long>();
        a.ngroups = pick_groups(sk->g->n);
    }
    const bool lazy_now = sk->lazy && sk->lb_ready;
    CK(c, timed(c, kTPick, [&] {
        if (lazy_now) return launch_pick_lazy(a, c->stream);
        // a full pick stores every S_u; the group records follow (the seed's
        // bit is set by then)
        PickArgs f = a;
        f.gsum = nullptr;
        cudaError_t e = launch_pick(f, c->stream);
        if (e == cudaSuccess && sk->lazy) e = launch_group_summaries(a, c->stream);
        return e;
    }));
    if (sk->lazy) sk->lb_ready = true;
    return run_levels(sk, kCover, false);
}

extern "C" im_status im_sketch_pick(im_sketch* sk, int32_t* s_out, uint64_t* S_out, double* est_out) {
    if (!sk) return IM_E_INVAL;
    im_ctx* c = sk->ctx;
    if (sk->picks >= sk->g->n) return fail(c, IM_E_RANGE, "every vertex is already picked");
    CKS(ensure_out_cap(sk, sk->picks + 1));
    PickArgs a = pick_args(sk, sk->picks);
    a.mark = 0;  // record the pick only; the caller covers with im_sketch_cover
    CK(c, launch_pick(a, c->stream));
    int32_t s = -1;
    unsigned long long S = 0;
    double est = 0;
    CK(c, cudaMemcpyAsync(&s, a.out_seed + a.k, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&S, a.out_S + a.k, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&est, a.out_est + a.k, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (s < 0) return fail(c, IM_E_RANGE, "no vertex left to pick");
    sk->picks++;
    if (s_out) *s_out = s;
    if (S_out) *S_out = S;
    if (est_out) *est_out = est;
    return IM_OK;
}

extern "C" im_status im_sketch_cover(im_sketch* sk, int32_t s, uint64_t* count_out) {
    if (!sk) return IM_E_INVAL;
    im_ctx* c = sk->ctx;
    if (s < 0 || s >= sk->g->n) return fail(c, IM_E_RANGE, "vertex %d out of range", s);
    CKS(phase_begin(sk, kCover));
    CK(c, launch_cover_seed(sk->M.as<uint8_t>(), sk->J, s, sk->g->rp_out.as<int32_t>(),
                            sk->ql[0].as<QEntry>(), &sk->ctr.as<ulonglong2>()[0].x,
                            chg_buf(sk, kCover, 0).as<uint32_t>(), sk->count.as<unsigned long long>(),
                            sk->buckets ? sk->bk_end[1].as<uint32_t>() : nullptr, sk->J / 16, c->stream));
    CKS(run_levels(sk, kCover, false));
    if (count_out) {
        unsigned long long cnt = 0;
        CK(c, cudaMemcpyAsync(&cnt, sk->count.p, 8, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        *count_out = cnt;
    }
    return IM_OK;
}

extern "C" im_status im_sketch_rebuild(im_sketch* sk) {
    if (!sk) return IM_E_INVAL;
    return build_registers(sk);
}

// ---------------------------------------------------------------------------
// Alg. 4
// ---------------------------------------------------------------------------
// Alg. 4 of one query, executed on context c (its allocator and stream); the
// graph is only read.
static im_status select_seeds_impl(im_ctx* c, im_graph* g, int32_t K, int32_t J, const im_model* model,
                                   uint64_t seed, double rebuild_eps, int32_t* seeds_out,
                                   double* score_out, double* estimate_out, im_sketch** sketch_out) {
    if (!c || !g || !seeds_out) return IM_E_INVAL;
    if (K < 1 || K > g->n) return fail(c, IM_E_RANGE, "K must be in [1, n], got %d", K);
    if (!valid_J(J)) return fail(c, IM_E_INVAL, "J must be a power of two in [16, 1024], got %d", J);
    if (model) {
        CKS(check_model(c, model, g->m));
        if (model->kind == kExplicit || model->kind == kTargetModel || g->load_kind == kExplicit ||
            g->load_kind == kTargetModel)
            return fail(c, IM_E_STATE, "explicit and per-target models are fixed at im_graph_load");
    }
    stats_begin(c);
    const double t0 = now_ms();
    im_sketch* sk = nullptr;
    CKS(sketch_start(c, g, J, seed, model, true, &sk));
    sk->lazy = c->tuning.lazy_pick != 0;
    sk->defer = true;
    // incremental rebuilds pay off with bucketed lists (sparse affected-set
    // searches); over edge scans a full rebuild is faster unless asked for (2)
    sk->incr = c->tuning.incremental == 2 || (c->tuning.incremental == 1 && sk->buckets);
    auto bail = [&](im_status s) {
        sketch_release(sk);
        delete sk;
        return s;
    };
    im_status s = ensure_out_cap(sk, K);
    if (s != IM_OK) return bail(s);
    if ((s = build_registers(sk)) != IM_OK) return bail(s);
    const double t_build = now_ms();
    c->stats.ms_build = t_build - t0;
    std::vector<double> score(K);
    uint64_t oldcount = 0;
    int64_t rebuilds = 0;
    double ms_rebuild = 0, ms_pc = 0;
    for (int32_t k = 0; k < K; ++k) {
        const double tk = now_ms();
        if ((s = pick_and_cover(sk, k)) != IM_OK) return bail(s);
        cudaError_t e = cudaMemcpyAsync(c->pinned, sk->count.p, 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = sync_collect(c);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "read count"));
        const uint64_t count = c->pinned[0];
        score[k] = (double)count / (double)J;
        const double tr = now_ms();
        ms_pc += tr - tk;
        if (k + 1 < K && rebuild_due(count, oldcount, J, rebuild_eps)) {
            if ((s = sk->incr ? incremental_rebuild(sk) : build_registers(sk)) != IM_OK) return bail(s);
            oldcount = count;
            ++rebuilds;
            ms_rebuild += now_ms() - tr;
        }
    }
    sk->picks = K;
    // the error word of every deferred phase and rebuild
    if ((s = check_err(sk)) != IM_OK) return bail(s);
    sk->defer = false;  // step-level calls on a returned sketch check each phase
    std::vector<int32_t> seeds(K);
    std::vector<double> est(K);
    cudaError_t e = cudaMemcpyAsync(seeds.data(), sk->out_seed.p, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(est.data(), sk->out_est.p, (size_t)K * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "read seeds"));
    if ((s = stats_collect(sk)) != IM_OK) return bail(s);
    c->stats.builds = 1 + rebuilds;
    c->stats.ms_rebuild = ms_rebuild;
    c->stats.ms_pick = ms_pc;
    c->stats.ms_total = now_ms() - t0;
    memcpy(seeds_out, seeds.data(), (size_t)K * 4);
    if (score_out) memcpy(score_out, score.data(), (size_t)K * 8);
    if (estimate_out) memcpy(estimate_out, est.data(), (size_t)K * 8);
    if (sketch_out) *sketch_out = sk;
    else bail(IM_OK);
    return IM_OK;
}

extern "C" im_status im_select_seeds(im_graph* g, int32_t K, int32_t J, const im_model* model,
                                     uint64_t seed, double rebuild_eps, int32_t* seeds_out,
                                     double* score_out, double* estimate_out, im_sketch** sketch_out) {
    if (!g) return IM_E_INVAL;
    return select_seeds_impl(g->ctx, g, K, J, model, seed, rebuild_eps, seeds_out, score_out,
                             estimate_out, sketch_out);
}

// ---------------------------------------------------------------------------
// warp fill-rate diagnostic (Table 6 analogue)
// ---------------------------------------------------------------------------
extern "C" im_status im_fill_rate(im_graph* g, int32_t J, uint64_t seed, const im_model* model,
                                  uint64_t* counts_out) {
    if (!g || !counts_out) return IM_E_INVAL;
    im_ctx* c = g->ctx;
    if (!valid_J(J)) return fail(c, IM_E_INVAL, "J must be a power of two in [16, 1024], got %d", J);
    if (model) {
        CKS(check_model(c, model, g->m));
        if (model->kind == kExplicit || model->kind == kTargetModel || g->load_kind == kExplicit ||
            g->load_kind == kTargetModel)
            return fail(c, IM_E_STATE, "explicit and per-target models are fixed at im_graph_load");
    }
    CK(c, cudaSetDevice(c->device));
    GraphDev dev = g->dev;
    int kind = g->kind;
    if (model) model_words(dev, kind, model);
    keep_class_bounds(dev, kind, g);
    DBuf X, salt, tab, cnt;
    im_status s = dalloc(c, (size_t)J * 4, X);
    if (s == IM_OK) s = dalloc(c, (size_t)J * 4, salt);
    if (s == IM_OK) s = dalloc(c, (size_t)kTabSize * 2, tab);
    if (s == IM_OK) s = dalloc(c, 5 * 8, cnt);
    auto release = [&]() { dfree(c, X); dfree(c, salt); dfree(c, tab); dfree(c, cnt); };
    if (s != IM_OK) { release(); return s; }
    auto st = c->stream;
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(cnt.p, 0, 5 * 8, st);
    if (e == cudaSuccess) e = launch_sims(seed, J, X.as<uint32_t>(), salt.as<uint32_t>(), tab.as<uint16_t>(), st);
    if (e == cudaSuccess)
        e = launch_fill_rate(kind, dev, seed, X.as<uint32_t>(), tab.as<uint16_t>(), J,
                             cnt.as<unsigned long long>(), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt.p, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(c, e, "fill rate");
    for (int i = 0; i < 5; ++i) counts_out[i] = h[i];
    return IM_OK;
}

// ---------------------------------------------------------------------------
// internal entry points of the query server
// ---------------------------------------------------------------------------
namespace imi {

im_status ctx_create_worker(int device, cudaStream_t stream, cudaMemPool_t pool, im_ctx** out) {
    im_ctx* c = nullptr;
    CKS(im_ctx_create(device, stream, 0, nullptr, &c));
    c->pool = pool;
    c->tuning.persistent = 0;
    *out = c;
    return IM_OK;
}

void ctx_set_budget(im_ctx* c, uint64_t bytes) { c->budget = bytes; }
const char* ctx_error(const im_ctx* c) { return c->err.c_str(); }

im_status select_seeds_on(im_ctx* c, im_graph* g, int32_t K, int32_t J, const im_model* model,
                          uint64_t seed, double rebuild_eps, int32_t* seeds_out, double* score_out,
                          double* estimate_out) {
    return select_seeds_impl(c, g, K, J, model, seed, rebuild_eps, seeds_out, score_out,
                             estimate_out, nullptr);
}

uint64_t query_bytes(const im_graph* g, int32_t J, int32_t K) {
    im_sketch probe;
    BufPlan plan;
    sketch_plan(&probe, g->n, g->m, J, plan);
    uint64_t total = 0;
    for (auto& pb : plan) total += round_bytes(pb.second);
    BufPlan scan;
    scan_plan(&probe, g->n, g->m, J, scan);
    uint64_t scan_bytes = 0;
    for (auto& pb : scan) scan_bytes += round_bytes(pb.second);
    total += scan_bytes + bucket_reserve_bytes(g->n, g->m, J);
    const size_t cap = (size_t)out_cap_for(K);
    total += round_bytes(cap * 4) + 2 * round_bytes(cap * 8);
    return total;
}

uint64_t graph_bytes(const im_graph* g) {
    uint64_t total = 0;
    for (const DBuf* b : {&g->rp_out, &g->col_out, &g->rp_in, &g->src_in, &g->h_in, &g->h_out,
                          &g->thrw_out, &g->thr_v, &g->thr_out, &g->thr_in,
                          &g->q_dense, &g->hkey, &g->q_dense_out, &g->out_to_in, &g->tri_b})
        total += b->bytes;
    return total;
}

int32_t graph_n(const im_graph* g) { return g->n; }
int graph_device(const im_graph* g) { return g->ctx->device; }

im_status check_query_model(const im_graph* g, const im_model* model, char* msg, size_t cap) {
    if (!model) return IM_OK;
    if (model->kind == kExplicit || model->kind == kTargetModel || g->load_kind == kExplicit ||
        g->load_kind == kTargetModel) {
        snprintf(msg, cap, "explicit and per-target models are fixed at im_graph_load");
        return IM_E_STATE;
    }
    if (model->kind < kUniform || model->kind > kTrivalency) {
        snprintf(msg, cap, "unknown model kind %d", model->kind);
        return IM_E_INVAL;
    }
    if (model->kind == kUniform && !(model->p >= 0.0f && model->p <= 1.0f)) {
        snprintf(msg, cap, "uniform p must be in [0,1]");
        return IM_E_INVAL;
    }
    return IM_OK;
}

}  // namespace imi

// ---------------------------------------------------------------------------
// Monte-Carlo spread with independent coins (Sec. 5.1 quality oracle)
// ---------------------------------------------------------------------------
extern "C" im_status im_spread_mc(im_graph* g, const int32_t* seeds, int32_t k, int64_t R,
                                  uint64_t seed, double* mean_out, double* stderr_out,
                                  uint64_t* sum_out, uint64_t* sumsq_out) {
    if (!g || !seeds) return IM_E_INVAL;
    im_ctx* c = g->ctx;
    if (k < 1) return fail(c, IM_E_RANGE, "k must be >= 1");
    if (R < 2) return fail(c, IM_E_RANGE, "R must be >= 2");
    for (int32_t i = 0; i < k; ++i)
        if (seeds[i] < 0 || seeds[i] >= g->n) return fail(c, IM_E_RANGE, "seed %d out of range", seeds[i]);
    CK(c, cudaSetDevice(c->device));
    const int32_t n = g->n;
    int B = 32;
    while (B < 1024 && B < R) B <<= 1;
    const int words = B / 32;
    DBuf vis, F[3], Q[3], ctr, gen, reach, acc, sd;
    std::vector<DBuf*> all = {&vis, &F[0], &F[1], &F[2], &Q[0], &Q[1], &Q[2], &ctr, &gen, &reach, &acc, &sd};
    auto release = [&]() {
        for (DBuf* b : all) dfree(c, *b);
    };
    im_status s = IM_OK;
    const size_t vbytes = (size_t)n * words * 4;
    for (DBuf* b : {&vis, &F[0], &F[1], &F[2]})
        if (s == IM_OK) s = dalloc(c, vbytes, *b);
    for (int i = 0; i < 3 && s == IM_OK; ++i) s = dalloc(c, (size_t)n * sizeof(QEntry), Q[i]);
    if (s == IM_OK) s = dalloc(c, (size_t)(kMaxLevels + 2) * 8, ctr);
    if (s == IM_OK) s = dalloc(c, (size_t)n * 4, gen);
    if (s == IM_OK) s = dalloc(c, (size_t)1024 * 8, reach);
    if (s == IM_OK) s = dalloc(c, 16, acc);
    if (s == IM_OK) s = dalloc(c, (size_t)k * 4, sd);
    if (s != IM_OK) { release(); return s; }
    auto st = c->stream;
    cudaError_t e = cudaMemcpyAsync(sd.p, seeds, (size_t)k * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(gen.p, 0, gen.bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc.p, 0, 16, st);
    if (e != cudaSuccess) { release(); return cuda_fail(c, e, "spread init"); }
    unsigned long long* cp = ctr.as<unsigned long long>();
    const int grid = level_grid();
    int32_t stamp = 0;
    for (int64_t r0 = 0; r0 < R; r0 += B) {
        const int valid = (int)std::min<int64_t>(B, R - r0);
        for (DBuf* b : {&vis, &F[0], &F[1], &F[2]})
            if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, vbytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(reach.p, 0, reach.bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(cp, 0, (size_t)(kMaxLevels + 2) * 8, st);
        McArgs a{};
        a.n = n;
        a.m = g->m;
        a.seed = seed;
        a.r0 = r0;
        a.words = words;
        a.vis = vis.as<uint32_t>();
        a.gen = gen.as<int32_t>();
        a.f_next = F[0].as<uint32_t>();
        a.q_out = Q[0].as<QEntry>();
        a.ctr_out = cp;
        a.gen_next = ++stamp;
        if (e == cudaSuccess) e = launch_mc_seed(g->dev, a, sd.as<int32_t>(), k, valid, st);
        int check = 2;
        for (int64_t l = 0; e == cudaSuccess; ) {
            a.f_cur = F[l % 3].as<uint32_t>();
            a.f_next = F[(l + 1) % 3].as<uint32_t>();
            a.f_prev = F[(l + 2) % 3].as<uint32_t>();
            a.q_in = Q[l % 3].as<QEntry>();
            a.ctr_in = cp + l;
            a.q_prev = l >= 1 ? Q[(l + 2) % 3].as<QEntry>() : nullptr;
            a.ctr_prev = l >= 1 ? cp + l - 1 : nullptr;
            a.q_out = Q[(l + 1) % 3].as<QEntry>();
            a.ctr_out = cp + l + 1;
            a.gen_next = ++stamp;
            e = launch_mc_level(g->kind, g->dev, a, grid, st);
            ++l;
            if (e == cudaSuccess && l % check == 0) {
                e = cudaMemcpyAsync(c->pinned, cp + l, 8, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) break;
                if ((c->pinned[0] >> kCountShift) == 0) break;
                if (l + 8 >= kMaxLevels) { release(); return fail(c, IM_E_TIMEOUT, "spread did not converge"); }
                if (check < 8) check *= 2;
            }
        }
        if (e == cudaSuccess) e = launch_mc_count(vis.as<uint32_t>(), n, words, reach.as<unsigned long long>(), st);
        if (e == cudaSuccess) e = launch_mc_reduce(reach.as<unsigned long long>(), valid, acc.as<unsigned long long>(), st);
        if (e != cudaSuccess) break;
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc.p, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(c, e, "spread");
    const double mean = (double)h[0] / (double)R;
    const long double var = ((long double)h[1] - (long double)h[0] * (long double)h[0] / (long double)R) /
                            (long double)(R - 1);
    if (mean_out) *mean_out = mean;
    if (stderr_out) *stderr_out = std::sqrt((double)(var > 0 ? var : 0) / (double)R);
    if (sum_out) *sum_out = h[0];
    if (sumsq_out) *sumsq_out = h[1];
    return IM_OK;
}


// ---------------------------------------------------------------------------
// Batches: many graphs as one disjoint union (vertex ids offset per graph),
// uniform IC probability per graph as a per-target model.  A selection runs
// Alg. 4 on every graph at once, one seed per graph per round; the graphs of
// one J share the simulation draws of the seed.
// ---------------------------------------------------------------------------
struct im_batch {
    im_ctx* ctx = nullptr;
    im_graph* g = nullptr;
    int32_t G = 0;
    std::vector<int32_t> voff;  // G + 1 vertex offsets
    DBuf gid;
};

extern "C" im_status im_batch_load(im_ctx* c, int32_t G, const int32_t* n, const int64_t* m,
                                   const int32_t* const* rowptr, const int32_t* const* col,
                                   const float* p, im_batch** out) {
    if (!c || !out || !n || !m || !rowptr || !col || !p) return fail(c, IM_E_INVAL, "NULL argument");
    if (G < 1) return fail(c, IM_E_RANGE, "G must be >= 1");
    int64_t N = 0, Mt = 0;
    for (int32_t g = 0; g < G; ++g) {
        if (n[g] < 1 || m[g] < 0 || !rowptr[g] || (m[g] > 0 && !col[g]))
            return fail(c, IM_E_INVAL, "graph %d: bad sizes or NULL arrays", g);
        if (!(p[g] >= 0.0f && p[g] <= 1.0f)) return fail(c, IM_E_INVAL, "graph %d: p outside [0,1]", g);
        if (rowptr[g][0] != 0 || rowptr[g][n[g]] != m[g]) return fail(c, IM_E_INVAL, "graph %d: bad rowptr", g);
        N += n[g];
        Mt += m[g];
    }
    if (N >= (1 << 26)) return fail(c, IM_E_RANGE, "total vertices must be < 2^26");
    if (Mt >= (1ll << 31)) return fail(c, IM_E_RANGE, "total edges must be < 2^31");
    std::vector<int32_t> rp((size_t)N + 1);
    std::vector<int32_t> cl((size_t)(Mt > 0 ? Mt : 1));
    std::vector<float> w((size_t)N);
    im_batch* b = new im_batch();
    b->ctx = c;
    b->G = G;
    b->voff.resize((size_t)G + 1);
    std::vector<int32_t> gid_h((size_t)N), key_h((size_t)N);
    int64_t vo = 0, eo = 0;
    for (int32_t g = 0; g < G; ++g) {
        b->voff[g] = (int32_t)vo;
        for (int32_t u = 0; u < n[g]; ++u) {
            rp[vo + u] = (int32_t)(eo + rowptr[g][u]);
            w[vo + u] = p[g];
            gid_h[vo + u] = g;
            key_h[vo + u] = u;  // hashes use the vertex id inside its own graph
        }
        for (int64_t e = 0; e < m[g]; ++e) cl[eo + e] = col[g][e] + (int32_t)vo;
        vo += n[g];
        eo += m[g];
    }
    b->voff[G] = (int32_t)vo;
    rp[N] = (int32_t)Mt;
    im_model md{};
    md.kind = kTargetModel;
    md.w = w.data();
    im_status s = graph_load_impl(c, (int32_t)N, Mt, rp.data(), cl.data(), &md, key_h.data(), &b->g);
    if (s != IM_OK) {
        delete b;
        return s;
    }
    if ((s = dalloc(c, (size_t)N * 4, b->gid)) != IM_OK) {
        im_graph_free(b->g);
        delete b;
        return s;
    }
    cudaError_t e = cudaMemcpyAsync(b->gid.p, gid_h.data(), (size_t)N * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dfree(c, b->gid);
        im_graph_free(b->g);
        delete b;
        return cuda_fail(c, e, "batch load");
    }
    *out = b;
    return IM_OK;
}

extern "C" void im_batch_free(im_batch* b) {
    if (!b) return;
    dfree(b->ctx, b->gid);
    im_graph_free(b->g);
    delete b;
}

// Fill of the flagged graphs' rows, then propagation from their vertices.
static im_status batch_build(im_sketch* sk) {
    im_ctx* c = sk->ctx;
    // the flagged fill keeps visited registers: a new sketch's are zeroed first
    if (sk->fresh) CK(c, cudaMemsetAsync(sk->M.p, 0, sk->M.bytes, c->stream));
    sk->fresh = false;
    CK(c, timed(c, kTFill, [&] {
        return launch_fill_flagged(sk->M.as<uint8_t>(), sk->g->n, sk->J, sk->salt.as<uint32_t>(),
                                   sk->gid, sk->gflag, sk->g->hkey.as<int32_t>(), c->stream);
    }));
    return propagate(sk);
}

extern "C" im_status im_batch_select_seeds(im_batch* b, const int32_t* J, const int32_t* K,
                                           uint64_t seed, double rebuild_eps, int32_t* seeds_out,
                                           double* score_out, double* estimate_out) {
    if (!b || !J || !K || !seeds_out) return IM_E_INVAL;
    im_ctx* c = b->ctx;
    const int32_t G = b->G;
    std::vector<int64_t> koff((size_t)G + 1, 0);
    for (int32_t g = 0; g < G; ++g) {
        const int32_t ng = b->voff[g + 1] - b->voff[g];
        if (K[g] < 1 || K[g] > ng) return fail(c, IM_E_RANGE, "graph %d: K must be in [1, n]", g);
        if (!valid_J(J[g])) return fail(c, IM_E_INVAL, "graph %d: unsupported J %d", g, J[g]);
        koff[g + 1] = koff[g] + K[g];
    }
    stats_begin(c);
    const double t0 = now_ms();
    auto st = c->stream;
    std::vector<int32_t> Js(J, J + G);
    std::sort(Js.begin(), Js.end());
    Js.erase(std::unique(Js.begin(), Js.end()), Js.end());
    int64_t builds = 0;
    for (int32_t Jg : Js) {
        std::vector<int32_t> members;
        int32_t maxK = 0;
        for (int32_t g = 0; g < G; ++g)
            if (J[g] == Jg) { members.push_back(g); maxK = std::max(maxK, K[g]); }
        // tiles: row ranges of at most 4096 rows inside one member graph
        std::vector<int4> tiles;
        std::vector<int32_t> tb((size_t)G, 0), te((size_t)G, 0);
        for (int32_t g : members) {
            tb[g] = (int32_t)tiles.size();
            for (int32_t r = b->voff[g]; r < b->voff[g + 1]; r += 4096)
                tiles.push_back(make_int4(g, r, std::min(r + 4096, b->voff[g + 1]), 0));
            te[g] = (int32_t)tiles.size();
        }
        im_sketch* sk = nullptr;
        CKS(sketch_start(c, b->g, Jg, seed, nullptr, false, &sk));
        DBuf tiles_d, tb_d, te_d, active_d, flag_d, gcount_d, pS, pU, oseed, oS, oest;
        std::vector<DBuf*> tmp = {&tiles_d, &tb_d, &te_d, &active_d, &flag_d, &gcount_d, &pS, &pU, &oseed, &oS, &oest};
        auto cleanup = [&]() {
            for (DBuf* x : tmp) dfree(c, *x);
            sketch_release(sk);
            delete sk;
        };
        im_status s = IM_OK;
        auto A = [&](DBuf& x, size_t bytes) { if (s == IM_OK) s = dalloc(c, bytes, x); };
        A(tiles_d, tiles.size() * sizeof(int4) + 16);
        A(tb_d, (size_t)G * 4);
        A(te_d, (size_t)G * 4);
        A(active_d, (size_t)G);
        A(flag_d, (size_t)G);
        A(gcount_d, (size_t)G * 8);
        A(pS, tiles.size() * 8 + 8);
        A(pU, tiles.size() * 4 + 4);
        A(oseed, (size_t)G * maxK * 4);
        A(oS, (size_t)G * maxK * 8);
        A(oest, (size_t)G * maxK * 8);
        if (s != IM_OK) { cleanup(); return s; }
        std::vector<uint8_t> active((size_t)G, 0), flag((size_t)G, 0);
        for (int32_t g : members) flag[g] = 1;
        cudaError_t e = cudaMemcpyAsync(tiles_d.p, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tb_d.p, tb.data(), (size_t)G * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(te_d.p, te.data(), (size_t)G * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(flag_d.p, flag.data(), (size_t)G, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gcount_d.p, 0, (size_t)G * 8, st);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch setup"); }
        sk->gid = b->gid.as<int32_t>();
        sk->gcount = gcount_d.as<unsigned long long>();
        sk->gflag = flag_d.as<uint8_t>();
        if ((s = batch_build(sk)) != IM_OK) { cleanup(); return s; }
        ++builds;
        std::vector<unsigned long long> count((size_t)G, 0), oldcount((size_t)G, 0);
        std::vector<std::vector<double>> score((size_t)G);
        for (int32_t r = 0; r < maxK; ++r) {
            for (int32_t g : members) active[g] = r < K[g] ? 1 : 0;
            e = cudaMemcpyAsync(active_d.p, active.data(), (size_t)G, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch round"); }
            if ((s = phase_begin(sk, kCover)) != IM_OK) { cleanup(); return s; }
            BatchPickArgs pa{};
            pa.M = sk->M.as<uint8_t>();
            pa.J = Jg;
            pa.tiles = tiles_d.as<int4>();
            pa.ntiles = (int)tiles.size();
            pa.active = active_d.as<uint8_t>();
            pa.picked = sk->seed_bits.as<uint32_t>();
            pa.part_S = pS.as<unsigned long long>();
            pa.part_u = pU.as<int32_t>();
            pa.tile_begin = tb_d.as<int32_t>();
            pa.tile_end = te_d.as<int32_t>();
            pa.G = G;
            pa.round = r;
            pa.maxK = maxK;
            pa.out_seed = oseed.as<int32_t>();
            pa.out_S = oS.as<unsigned long long>();
            pa.out_est = oest.as<double>();
            pa.rp_out = b->g->rp_out.as<int32_t>();
            pa.q_cover = sk->ql[0].as<QEntry>();
            pa.ctr_cover = &sk->ctr.as<ulonglong2>()[0].x;
            pa.chg0 = chg_buf(sk, kCover, 0).as<uint32_t>();
            pa.gcount = sk->gcount;
            pa.err = sk->err.as<uint32_t>();
            pa.bk_end_out = sk->buckets ? sk->bk_end[1].as<uint32_t>() : nullptr;
            pa.chunks = Jg / 16;
            e = timed(c, kTPick, [&] { return launch_batch_pick(pa, st); });
            if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch pick"); }
            if ((s = run_levels(sk, kCover, false)) != IM_OK) { cleanup(); return s; }
            e = cudaMemcpyAsync(count.data(), gcount_d.p, (size_t)G * 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = sync_collect(c);
            if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch counts"); }
            bool any = false;
            for (int32_t g : members) {
                flag[g] = 0;
                if (!active[g]) continue;
                score[g].push_back((double)count[g] / (double)Jg);
                if (r + 1 < K[g] && rebuild_due(count[g], oldcount[g], Jg, rebuild_eps)) {
                    flag[g] = 1;
                    oldcount[g] = count[g];
                    any = true;
                }
            }
            if (any) {
                e = cudaMemcpyAsync(flag_d.p, flag.data(), (size_t)G, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch flags"); }
                if ((s = batch_build(sk)) != IM_OK) { cleanup(); return s; }
                ++builds;
            }
        }
        std::vector<int32_t> hseed((size_t)G * maxK);
        std::vector<double> hest((size_t)G * maxK);
        e = cudaMemcpyAsync(hseed.data(), oseed.p, hseed.size() * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hest.data(), oest.p, hest.size() * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = sync_collect(c);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch results"); }
        for (int32_t g : members) {
            for (int32_t k = 0; k < K[g]; ++k) {
                const int32_t sg = hseed[(size_t)g * maxK + k];
                seeds_out[koff[g] + k] = sg >= 0 ? sg - b->voff[g] : -1;
                if (score_out) score_out[koff[g] + k] = score[g][k];
                if (estimate_out) estimate_out[koff[g] + k] = hest[(size_t)g * maxK + k];
            }
        }
        if ((s = stats_collect(sk)) != IM_OK) { cleanup(); return s; }
        cleanup();
    }
    c->stats.builds = builds;
    c->stats.ms_total = now_ms() - t0;
    return IM_OK;
}
