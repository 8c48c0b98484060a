// Query server: resident graphs, concurrent im_select_seeds queries on worker
// streams, admission under a device-memory budget.  Host-only code; every
// query runs the same kernels as a single im_select_seeds call, on the
// worker's own context (stream, memory pool, statistics).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/difuser_im.h"
#include "im_internal.h"

namespace {

double clock_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    int64_t ticket = 0;
    im_query q{};
    int32_t* seeds = nullptr;
    double* score = nullptr;
    double* est = nullptr;
    uint64_t bytes = 0;
    bool done = false;
    im_query_result res{};
};

}  // namespace

struct im_server {
    im_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work;  // a slot may be able to start a query
    std::condition_variable cv_done;  // a query finished
    std::deque<Job*> pending;         // arrival order
    std::unordered_map<int64_t, Job*> jobs;
    std::vector<im_graph*> graphs;
    uint64_t graph_bytes = 0;
    uint64_t reserved = 0, reserved_peak = 0;
    int32_t running = 0, running_peak = 0;
    int32_t head_bypassed = 0;  // queries started ahead of the current head
    int64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0, bypassed = 0;
    bool stop = false;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<im_ctx*> ctxs;
    std::vector<std::thread> workers;

    uint64_t capacity() const {
        if (cfg.hbm_budget_bytes == 0) return UINT64_MAX;
        return cfg.hbm_budget_bytes > graph_bytes ? cfg.hbm_budget_bytes - graph_bytes : 0;
    }
    bool fits(const Job* j) const { return reserved + j->bytes <= capacity(); }

    // The next pending query a free slot may start (caller holds mu), or null.
    Job* take() {
        for (size_t i = 0; i < pending.size(); ++i) {
            Job* j = pending[i];
            if (!fits(j)) {
                if (i == 0 && head_bypassed >= cfg.max_bypass) return nullptr;
                continue;
            }
            if (i == 0) head_bypassed = 0;
            else {
                ++head_bypassed;
                ++bypassed;
            }
            pending.erase(pending.begin() + (ptrdiff_t)i);
            return j;
        }
        return nullptr;
    }

    void worker(int slot) {
        cudaSetDevice(cfg.device);
        im_ctx* c = ctxs[slot];
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            Job* j = nullptr;
            cv_work.wait(lk, [&] { return (j = take()) != nullptr || (stop && pending.empty()); });
            if (!j) return;
            reserved += j->bytes;
            reserved_peak = std::max(reserved_peak, reserved);
            running_peak = std::max(running_peak, ++running);
            j->res.t_start_ms = clock_ms();
            j->res.slot = slot;
            lk.unlock();

            imi::ctx_set_budget(c, j->bytes);
            const double t0 = clock_ms();
            const im_model* mdl = j->q.model.kind < 0 ? nullptr : &j->q.model;
            const im_status s = imi::select_seeds_on(c, graphs[j->q.graph], j->q.K, j->q.J, mdl,
                                                     j->q.seed, j->q.rebuild_eps, j->seeds, j->score,
                                                     j->est);
            const double t1 = clock_ms();
            if (s != IM_OK) {
                snprintf(j->res.error, sizeof j->res.error, "%s", imi::ctx_error(c));
                // a failed query leaves its stream idle, with nothing allocated
                cudaStreamSynchronize(streams[slot]);
                (void)cudaGetLastError();
            }

            lk.lock();
            j->res.status = s;
            j->res.ms_select = t1 - t0;
            j->res.t_done_ms = t1;
            j->done = true;
            reserved -= j->bytes;
            --running;
            ++completed;
            if (s != IM_OK) ++failed;
            cv_done.notify_all();
            cv_work.notify_all();
        }
    }
};

extern "C" double im_server_clock_ms(void) { return clock_ms(); }

extern "C" im_status im_server_create(const im_server_config* cfg, im_server** out) {
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 64 || cfg->max_bypass < 0) return IM_E_INVAL;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        (void)cudaGetLastError();
        return IM_E_CUDA;
    }
    im_server* srv = new im_server();
    srv->cfg = *cfg;
    auto bail = [&]() {
        for (im_ctx* c : srv->ctxs) im_ctx_destroy(c);
        for (cudaStream_t st : srv->streams) cudaStreamDestroy(st);
        if (srv->pool) cudaMemPoolDestroy(srv->pool);
        delete srv;
        (void)cudaGetLastError();
        return IM_E_CUDA;
    };
    // one stream-ordered pool for all workers; freed blocks stay in the pool
    // (no unmapping between queries), so it holds at most the peak of what
    // running queries reserved
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = cfg->device;
    if (cudaMemPoolCreate(&srv->pool, &props) != cudaSuccess) return bail();
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
        return bail();
    for (int i = 0; i < cfg->slots; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return bail();
        srv->streams.push_back(st);
        im_ctx* c = nullptr;
        if (imi::ctx_create_worker(cfg->device, st, srv->pool, &c) != IM_OK) return bail();
        srv->ctxs.push_back(c);
    }
    for (int i = 0; i < cfg->slots; ++i) srv->workers.emplace_back([srv, i] { srv->worker(i); });
    *out = srv;
    return IM_OK;
}

extern "C" void im_server_destroy(im_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (std::thread& t : srv->workers) t.join();
    cudaSetDevice(srv->cfg.device);
    for (im_ctx* c : srv->ctxs) im_ctx_destroy(c);
    for (cudaStream_t st : srv->streams) cudaStreamDestroy(st);
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    for (auto& kv : srv->jobs) delete kv.second;
    delete srv;
}

extern "C" im_status im_server_add_graph(im_server* srv, im_graph* g, int32_t* id_out) {
    if (!srv || !g || !id_out) return IM_E_INVAL;
    if (imi::graph_device(g) != srv->cfg.device) return IM_E_STATE;
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t gb = imi::graph_bytes(g);
    if (srv->cfg.hbm_budget_bytes && srv->graph_bytes + gb > srv->cfg.hbm_budget_bytes) return IM_E_NOMEM;
    // the graph was loaded on another stream: make it visible to the workers
    if (cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return IM_E_CUDA;
    }
    srv->graph_bytes += gb;
    srv->graphs.push_back(g);
    *id_out = (int32_t)srv->graphs.size() - 1;
    return IM_OK;
}

extern "C" im_status im_server_query_bytes(im_server* srv, int32_t graph, int32_t J, int32_t K,
                                           uint64_t* bytes_out) {
    if (!srv || !bytes_out || J < 16 || J > 1024 || (J & (J - 1)) || K < 1) return IM_E_INVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (graph < 0 || graph >= (int32_t)srv->graphs.size()) return IM_E_RANGE;
    *bytes_out = imi::query_bytes(srv->graphs[graph], J, K);
    return IM_OK;
}

extern "C" im_status im_server_submit(im_server* srv, const im_query* q, int32_t* seeds_out,
                                      double* score_out, double* estimate_out, int64_t* ticket_out) {
    if (!srv || !q || !seeds_out || !ticket_out) return IM_E_INVAL;
    if (q->J < 16 || q->J > 1024 || (q->J & (q->J - 1))) return IM_E_INVAL;
    Job* j = new Job();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) { delete j; return IM_E_STATE; }
        if (q->graph < 0 || q->graph >= (int32_t)srv->graphs.size()) { delete j; return IM_E_RANGE; }
        im_graph* g = srv->graphs[q->graph];
        if (q->K < 1 || q->K > imi::graph_n(g)) { delete j; return IM_E_RANGE; }
        char msg[160];
        const im_status ms =
            imi::check_query_model(g, q->model.kind < 0 ? nullptr : &q->model, msg, sizeof msg);
        if (ms != IM_OK) { delete j; return ms; }
        j->bytes = imi::query_bytes(g, q->J, q->K);
        if (j->bytes > srv->capacity()) { delete j; return IM_E_NOMEM; }
        j->ticket = srv->next_ticket++;
        j->q = *q;
        j->q.model.w = nullptr;
        j->seeds = seeds_out;
        j->score = score_out;
        j->est = estimate_out;
        j->res.ticket = j->ticket;
        j->res.slot = -1;
        j->res.bytes = j->bytes;
        j->res.t_submit_ms = clock_ms();
        srv->jobs[j->ticket] = j;
        srv->pending.push_back(j);
        ++srv->submitted;
        *ticket_out = j->ticket;
    }
    srv->cv_work.notify_one();
    return IM_OK;
}

extern "C" im_status im_server_wait(im_server* srv, int64_t ticket, double timeout_ms,
                                    im_query_result* out) {
    if (!srv || !out) return IM_E_INVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return IM_E_RANGE;
    Job* j = it->second;
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, [&] { return j->done; });
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                      [&] { return j->done; })) {
        return IM_E_TIMEOUT;
    }
    *out = j->res;
    srv->jobs.erase(ticket);
    delete j;
    return IM_OK;
}

extern "C" im_status im_server_get_stats(im_server* srv, im_server_stats* out) {
    if (!srv || !out) return IM_E_INVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    out->bypassed = srv->bypassed;
    out->slots = srv->cfg.slots;
    out->running = srv->running;
    out->running_peak = srv->running_peak;
    out->pending = (int32_t)srv->pending.size();
    out->budget = srv->cfg.hbm_budget_bytes;
    out->graph_bytes = srv->graph_bytes;
    out->reserved = srv->reserved;
    out->reserved_peak = srv->reserved_peak;
    return IM_OK;
}
