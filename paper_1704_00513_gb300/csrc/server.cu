// server.cu -- a continuous-batching request server over resident graphs: BFS and frontier codec
// requests of mixed sizes, admitted by free slots and an HBM budget, executed concurrently on
// per-slot CUDA streams (fq_server_*).
//
// Each slot is a host worker thread with its own stream, its own codec workspace and its own BFS
// handle per resident graph (a handle serves one call at a time).  A request is admitted when a
// slot is idle and its device footprint fits in the budget next to the resident graphs and the
// requests already running; it then allocates its buffers stream-ordered, copies its input in,
// runs, copies its result out and frees.  Requests that arrive while others are on the GPU start as
// soon as a slot and memory free up, so their copies and kernels overlap with the running ones.
// The thesis has no serving layer; this is the serving form of its BFS + codec hot path.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "fq_common.cuh"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct GraphEntry {
    const int64_t *off;
    const uint32_t *cols;
    uint64_t n, m;
    std::vector<fq_graph *> per_slot;
};

}  // namespace

struct fq_server {
    uint64_t budget;
    uint64_t resident = 0;  // graphs' handles and the slots' workspaces
    uint64_t in_use = 0;    // running requests' buffers
    uint32_t nslots;
    int device = 0;
    uint64_t max_codec_ids;
    std::vector<cudaStream_t> streams;
    std::vector<void *> work;  // per-slot codec workspace
    std::vector<GraphEntry> graphs;
    std::deque<fq_request *> queue;
    std::vector<bool> busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> threads;
    bool stop = false;
    uint64_t completed = 0;
};

namespace {

uint64_t footprint(const fq_server *s, const fq_request *r)
{
    switch (r->kind) {
    case FQ_REQ_BFS: {
        if (r->graph >= s->graphs.size()) return 0;
        const uint64_t n = s->graphs[r->graph].n;
        return 8 * n + 4096;  // depth + parent
    }
    case FQ_REQ_ENCODE: return 4 * r->in_count + fq_queue_bound(r->in_count) + 4096;
    case FQ_REQ_DECODE: return r->in_count + r->out_cap + 4096;
    default: return 0;
    }
}

// CUDA calls of the request path note their failures (fq_last_cuda_error) before being tested.
cudaError_t noted(cudaError_t e, int line)
{
    if (e != cudaSuccess) fq::note_cuda_error(e, line);
    return e;
}
#define FQ_N(expr) noted((expr), __LINE__)

fq_status run_request(fq_server *s, uint32_t slot, fq_request *r)
{
    cudaStream_t st = s->streams[slot];
    switch (r->kind) {
    case FQ_REQ_BFS: {
        if (r->graph >= s->graphs.size()) return FQ_EINVAL;
        GraphEntry &g = s->graphs[r->graph];
        if (r->root >= g.n || r->out_cap < 4 * g.n) return FQ_EINVAL;
        int32_t *depth = nullptr;
        uint32_t *parent = nullptr;
        if (FQ_N(cudaMallocAsync(reinterpret_cast<void **>(&depth), 4 * g.n, st)) != cudaSuccess) return FQ_ENOMEM;
        if (FQ_N(cudaMallocAsync(reinterpret_cast<void **>(&parent), 4 * g.n, st)) != cudaSuccess) {
            cudaFreeAsync(depth, st);
            return FQ_ENOMEM;
        }
        fq_bfs_opts o{0, 0, r->flags, 0};
        fq_bfs_stats stats;
        fq_status rc = fq_bfs_run(g.per_slot[slot], r->root, depth, parent, &o, &stats, nullptr, 0, nullptr, 0, st);
        if (rc == FQ_OK && FQ_N(cudaMemcpyAsync(r->h_out, depth, 4 * g.n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            rc = FQ_ECUDA;
        if (rc == FQ_OK && r->h_out2 && r->out2_cap >= 4 * g.n &&
            FQ_N(cudaMemcpyAsync(r->h_out2, parent, 4 * g.n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            rc = FQ_ECUDA;
        cudaFreeAsync(depth, st);
        cudaFreeAsync(parent, st);
        if (FQ_N(cudaStreamSynchronize(st)) != cudaSuccess && rc == FQ_OK) rc = FQ_ECUDA;
        r->out_count = stats.reached;
        r->aux = stats.reached_edges;
        return rc;
    }
    case FQ_REQ_ENCODE: {
        const uint64_t n = r->in_count;
        if (n > s->max_codec_ids) return FQ_EINVAL;
        const uint64_t cap = fq_queue_bound(n);
        uint8_t *buf = nullptr;
        if (FQ_N(cudaMallocAsync(reinterpret_cast<void **>(&buf), fq::pad16(4 * n) + cap + 16, st)) != cudaSuccess)
            return FQ_ENOMEM;  // ids, the stream at a 16-byte boundary, then the 8-byte size
        uint32_t *ids = reinterpret_cast<uint32_t *>(buf);
        uint8_t *out = buf + fq::pad16(4 * n);
        uint64_t *nbytes = reinterpret_cast<uint64_t *>(out + cap);
        fq_status rc = FQ_OK;
        if (n && FQ_N(cudaMemcpyAsync(ids, r->h_in, 4 * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) rc = FQ_ECUDA;
        void *w = s->work[slot];
        const uint64_t wb = fq_workspace_bytes(s->max_codec_ids, 0);
        if (rc == FQ_OK) rc = fq_frontier_encode(ids, n, out, cap, nbytes, w, wb, st);
        uint64_t size = 0;
        if (rc == FQ_OK) rc = fq_work_status(w, st, nullptr);
        if (rc == FQ_OK && (FQ_N(cudaMemcpyAsync(&size, nbytes, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                            FQ_N(cudaStreamSynchronize(st)) != cudaSuccess))
            rc = FQ_ECUDA;
        if (rc == FQ_OK && size > r->out_cap) rc = FQ_ENOSPC;
        if (rc == FQ_OK && FQ_N(cudaMemcpyAsync(r->h_out, out, size, cudaMemcpyDeviceToHost, st)) != cudaSuccess) rc = FQ_ECUDA;
        cudaFreeAsync(buf, st);
        if (FQ_N(cudaStreamSynchronize(st)) != cudaSuccess && rc == FQ_OK) rc = FQ_ECUDA;
        r->out_count = size;
        return rc;
    }
    case FQ_REQ_DECODE: {
        const uint64_t bytes = r->in_count;
        const uint64_t cap_ids = r->out_cap / 4;
        if (cap_ids > s->max_codec_ids || bytes % 16 != 0) return FQ_EINVAL;
        uint8_t *buf = nullptr;
        if (FQ_N(cudaMallocAsync(reinterpret_cast<void **>(&buf), fq::pad16(bytes) + 4 * cap_ids + 32, st)) != cudaSuccess)
            return FQ_ENOMEM;
        uint8_t *in = buf;
        uint32_t *ids = reinterpret_cast<uint32_t *>(buf + fq::pad16(bytes));
        uint64_t *nout = reinterpret_cast<uint64_t *>(ids + cap_ids + (4 - cap_ids % 4) % 4);
        fq_status rc = FQ_OK;
        if (FQ_N(cudaMemcpyAsync(in, r->h_in, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) rc = FQ_ECUDA;
        void *w = s->work[slot];
        const uint64_t wb = fq_workspace_bytes(s->max_codec_ids, 0);
        if (rc == FQ_OK) rc = fq_frontier_decode(in, bytes, ids, cap_ids, nout, w, wb, st);
        uint64_t n = 0;
        if (rc == FQ_OK) rc = fq_work_status(w, st, nullptr);
        if (rc == FQ_OK && (FQ_N(cudaMemcpyAsync(&n, nout, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                            FQ_N(cudaStreamSynchronize(st)) != cudaSuccess))
            rc = FQ_ECUDA;
        if (rc == FQ_OK && n && FQ_N(cudaMemcpyAsync(r->h_out, ids, 4 * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            rc = FQ_ECUDA;
        cudaFreeAsync(buf, st);
        if (FQ_N(cudaStreamSynchronize(st)) != cudaSuccess && rc == FQ_OK) rc = FQ_ECUDA;
        r->out_count = n;
        return rc;
    }
    default: return FQ_EINVAL;
    }
}

void worker(fq_server *s, uint32_t slot)
{
    cudaSetDevice(s->device);
    for (;;) {
        fq_request *r = nullptr;
        uint64_t need = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admission: FIFO head, when it fits in the budget next to what is running
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->queue.empty()) return false;
                need = footprint(s, s->queue.front());
                return s->in_use + need + s->resident <= s->budget || s->in_use == 0;
            });
            if (s->stop && s->queue.empty()) return;
            r = s->queue.front();
            s->queue.pop_front();
            need = footprint(s, r);
            s->in_use += need;
            s->busy[slot] = true;
        }
        r->t_start = now_s();
        const fq_status rc = run_request(s, slot, r);
        r->t_end = now_s();
        if (rc == FQ_ECUDA) {
            int line = 0;
            const int e = fq_last_cuda_error(&line);
            r->aux = ((uint64_t)(uint32_t)e << 32) | (uint32_t)line;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= need;
            s->busy[slot] = false;
            r->status = rc;
            r->done = 1;
            s->completed++;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

fq_status fq_server_create(uint64_t hbm_budget_bytes, uint32_t slots, uint64_t max_codec_ids, fq_server **out)
{
    if (!out || slots == 0 || slots > 256) return FQ_EINVAL;
    *out = nullptr;
    fq_server *s = new (std::nothrow) fq_server();
    if (!s) return FQ_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->nslots = slots;
    s->max_codec_ids = max_codec_ids;
    cudaGetDevice(&s->device);
    const uint64_t wb = fq_workspace_bytes(max_codec_ids, 0);
    for (uint32_t i = 0; i < slots; i++) {
        cudaStream_t st;
        void *w = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaMalloc(&w, wb) != cudaSuccess) {
            cudaGetLastError();
            fq_server_destroy(s);
            return FQ_ENOMEM;
        }
        s->streams.push_back(st);
        s->work.push_back(w);
        s->resident += wb;
    }
    s->busy.assign(slots, false);
    for (uint32_t i = 0; i < slots; i++) s->threads.emplace_back(worker, s, i);
    *out = s;
    return FQ_OK;
}

fq_status fq_server_destroy(fq_server *s)
{
    if (!s) return FQ_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) t.join();
    cudaDeviceSynchronize();
    for (auto &g : s->graphs)
        for (fq_graph *h : g.per_slot)
            if (h) fq_graph_destroy(h);
    for (void *w : s->work) cudaFree(w);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return FQ_OK;
}

fq_status fq_server_add_graph(fq_server *s, const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, uint64_t m,
                              uint32_t *graph_id)
{
    if (!s || !graph_id) return FQ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);  // no request may run while handles are created
    for (bool b : s->busy)
        if (b) return FQ_EBUSY;
    GraphEntry e{d_offsets, d_cols, n, m, {}};
    size_t free0 = 0, free1 = 0, total = 0;
    cudaMemGetInfo(&free0, &total);
    for (uint32_t i = 0; i < s->nslots; i++) {
        fq_graph *h = nullptr;
        const fq_status rc = fq_graph_create(d_offsets, d_cols, n, m, &h);
        if (rc != FQ_OK) {
            for (fq_graph *x : e.per_slot) fq_graph_destroy(x);
            return rc;
        }
        e.per_slot.push_back(h);
    }
    cudaMemGetInfo(&free1, &total);
    s->resident += (free0 > free1 ? free0 - free1 : 0) + 8 * (n + 1) + 4 * m;  // handles + the CSR itself
    *graph_id = (uint32_t)s->graphs.size();
    s->graphs.push_back(std::move(e));
    return FQ_OK;
}

fq_status fq_server_submit(fq_server *s, fq_request *r)
{
    if (!s || !r) return FQ_EINVAL;
    if (r->kind != FQ_REQ_BFS && r->kind != FQ_REQ_ENCODE && r->kind != FQ_REQ_DECODE) return FQ_EINVAL;
    if (footprint(s, r) + s->resident > s->budget) return FQ_ENOMEM;  // could never be admitted
    r->done = 0;
    r->status = FQ_OK;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FQ_EBUSY;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    return FQ_OK;
}

fq_status fq_server_wait(fq_server *s, fq_request *r, double timeout_s)
{
    if (!s || !r) return FQ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done != 0; });
    return ok ? r->status : FQ_ETIMEOUT;
}

fq_status fq_server_info(fq_server *s, uint64_t *resident, uint64_t *in_use, uint64_t *queued, uint64_t *completed)
{
    if (!s) return FQ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (resident) *resident = s->resident;
    if (in_use) *in_use = s->in_use;
    if (queued) *queued = s->queue.size();
    if (completed) *completed = s->completed;
    return FQ_OK;
}

double fq_server_clock(void) { return now_s(); }

}  // extern "C"
