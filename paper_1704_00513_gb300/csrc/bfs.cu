// bfs.cu -- level-synchronous, direction-optimising BFS with the per-level frontier codec
// stage, and its C ABI (fq_graph_create / fq_graph_destroy / fq_bfs_run).
//
// One level d (the loop of Alg. "Our BFS algorithm with SpVM and compression", on one GPU):
//   1. encode F_d as Q_d (sorted queue, FQ) and B_d (bitmap, FB) [and the visited bitmap V_d]
//      -- the compress steps before the thesis' ALLGATHERV/ALLTOALLV; the byte counts are the
//      exchange volume;
//   2. choose the direction from (n_f, m_f, m_u): top-down -> bottom-up when m_f*alpha > m_u,
//      back when n_f*beta < n (direction optimisation, sec. 3.1);
//   3. decode the form that direction consumes (Q_d for top-down, B_d for bottom-up) -- the
//      decompress step;
//   4. expand: top-down over the decoded queue (t = A (x) f masked by the visited list) or
//      bottom-up against the decoded bitmap; depth/parent written by the discovering thread;
//   5. compact the next-frontier bitmap into the sorted queue F_{d+1} (popcount + prefix sum,
//      sec. 3.1 "Sparse vector with pop counting"), visited |= next, count n_f and m_f.
// The host reads one 512-byte counter record per level (termination test and direction).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "fq_common.cuh"

using namespace fq;

namespace {

constexpr uint32_t kHubDegree = 256;   // top-down: vertices of at least this degree are split
constexpr uint32_t kHubChunk = 2048;   //   into chunks of this many edges, one CTA each
constexpr uint32_t kThreads = 256;

struct HubItem {
    uint32_t v;
    uint32_t count;
    unsigned long long start;
};

// Device counters of one level (first 256 bytes of the handle's allocation).
struct Counters {
    unsigned long long n_f;       // |F_{d+1}| (compaction)
    unsigned long long m_f;       // degree sum over F_{d+1}
    unsigned long long examined;  // bottom-up adjacency entries read at this level
    unsigned long long hub_items; // top-down hub work items
    unsigned long long q_bytes, b_bytes, v_bytes, dec_n;
    unsigned long long pad[24];
};
static_assert(sizeof(Counters) == 256, "counter block is 256 bytes");

__device__ __forceinline__ void td_visit(uint32_t w, uint32_t src, const uint32_t *__restrict__ visited32,
                                         uint32_t *next32, int32_t *depth, uint32_t *parent, int32_t newdepth)
{
    const uint32_t bit = 1u << (w & 31u), wi = w >> 5;
    if (visited32[wi] & bit) return;
    if (next32[wi] & bit) return;
    const uint32_t old = atomicOr(&next32[wi], bit);
    if (!(old & bit)) {
        depth[w] = newdepth;
        if (parent) parent[w] = src;
    }
}

__global__ void bfs_init_kernel(const int64_t *off, uint32_t root, int32_t *depth, uint32_t *parent, uint32_t *q,
                                uint64_t *fbits, uint64_t *visited, Counters *ctr)
{
    depth[root] = 0;
    if (parent) parent[root] = root;
    q[0] = root;
    fbits[root >> 6] |= 1ull << (root & 63u);
    visited[root >> 6] |= 1ull << (root & 63u);
    ctr->n_f = 1;
    ctr->m_f = (unsigned long long)(off[root + 1] - off[root]);
}

// Top-down expansion of the decoded queue q[0..nf): each warp takes 32 frontier vertices,
// flattens their adjacency lists with a warp prefix sum of degrees and walks the edges 32 at a
// time (the owner of edge idx is found by a 5-step binary search over the lanes' prefix
// values).  Vertices of degree >= kHubDegree are split into kHubChunk-edge items instead and
// expanded by td_hub_kernel, so no warp walks a long list alone.
__global__ void __launch_bounds__(kThreads) td_expand_kernel(const uint32_t *__restrict__ q, uint64_t nf,
                                                             const int64_t *__restrict__ off,
                                                             const uint32_t *__restrict__ cols,
                                                             const uint32_t *__restrict__ visited32, uint32_t *next32,
                                                             int32_t *depth, uint32_t *parent, int32_t newdepth,
                                                             HubItem *items, unsigned long long *nitems,
                                                             unsigned long long items_cap, uint64_t n, Ctl *err)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = gw * 32u; base < nf; base += nw * 32u) {
        const uint64_t i = base + lane;
        uint32_t v = 0, deg = 0;
        long long s = 0;
        if (i < nf && q[i] >= n) set_error(err, FQ_ECORRUPT, kWhereBfs, i);  // defensive: ids come from our decoder
        if (i < nf && q[i] < n) {
            v = q[i];
            s = off[v];
            const long long d = off[v + 1] - s;
            if (d >= (long long)kHubDegree) {
                const unsigned long long chunks = ((unsigned long long)d + kHubChunk - 1) / kHubChunk;
                const unsigned long long at = atomicAdd(nitems, chunks);
                if (at + chunks > items_cap) {
                    set_error(err, FQ_ECORRUPT, kWhereBfs, i);  // only a frontier with repeated ids gets here
                } else {
                    for (unsigned long long c = 0; c < chunks; c++) {
                        HubItem it;
                        it.v = v;
                        it.start = (unsigned long long)s + c * kHubChunk;
                        it.count = (uint32_t)min((unsigned long long)kHubChunk, (unsigned long long)d - c * kHubChunk);
                        items[at + c] = it;
                    }
                }
            } else {
                deg = (uint32_t)d;
            }
        }
        const uint32_t incl = warp_incl_scan(deg);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t p = incl - deg;
        for (uint32_t c = 0; c < total; c += 32u) {
            const uint32_t idx = c + lane;
            uint32_t lo = 0;
#pragma unroll
            for (uint32_t step = 16; step > 0; step >>= 1) {
                const uint32_t cand = lo + step;
                const uint32_t pc = __shfl_sync(0xffffffffu, p, cand);
                if (pc <= idx) lo = cand;
            }
            const uint32_t src = __shfl_sync(0xffffffffu, v, lo);
            const long long ss = __shfl_sync(0xffffffffu, s, lo);
            const uint32_t ps = __shfl_sync(0xffffffffu, p, lo);
            if (idx < total) td_visit(cols[ss + (idx - ps)], src, visited32, next32, depth, parent, newdepth);
        }
    }
}

__global__ void __launch_bounds__(kThreads) td_hub_kernel(const HubItem *__restrict__ items,
                                                          const unsigned long long *nitems, unsigned long long items_cap,
                                                          const uint32_t *__restrict__ cols,
                                                          const uint32_t *__restrict__ visited32, uint32_t *next32,
                                                          int32_t *depth, uint32_t *parent, int32_t newdepth)
{
    const unsigned long long total = min(*nitems, items_cap);
    for (unsigned long long it = blockIdx.x; it < total; it += gridDim.x) {
        const HubItem h = items[it];
        for (uint32_t j = threadIdx.x; j < h.count; j += blockDim.x)
            td_visit(cols[h.start + j], h.v, visited32, next32, depth, parent, newdepth);
    }
}

// Bottom-up sweep: one thread per vertex; an unvisited vertex scans its adjacency in CSR order
// and stops at the first neighbour in the (decoded) frontier bitmap.  The 32 vertices of a warp
// share one 32-bit word of the next-frontier bitmap, written whole by lane 0 from a ballot, so
// the sweep needs no atomics.
__global__ void __launch_bounds__(kThreads) bu_sweep_kernel(const uint32_t *__restrict__ front32,
                                                            const uint32_t *__restrict__ visited32,
                                                            uint32_t *__restrict__ next32,
                                                            const int64_t *__restrict__ off,
                                                            const uint32_t *__restrict__ cols, int32_t *depth,
                                                            uint32_t *parent, int32_t newdepth, uint64_t n,
                                                            unsigned long long *examined)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cnt = 0;
    for (uint64_t word = gw; word * 32u < n; word += nw) {
        const uint32_t vis = visited32[word];
        if (vis == 0xffffffffu) continue;
        const uint64_t w = word * 32u + lane;
        bool found = false;
        uint32_t par = 0;
        if (w < n && !((vis >> lane) & 1u)) {
            const long long s = off[w], e = off[w + 1];
            for (long long j = s; j < e; j++) {
                const uint32_t u = cols[j];
                cnt++;
                if ((front32[u >> 5] >> (u & 31u)) & 1u) {
                    found = true;
                    par = u;
                    break;
                }
            }
        }
        if (found) {
            depth[w] = newdepth;
            if (parent) parent[w] = par;
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, found);
        if (lane == 0 && mask) next32[word] = mask;
    }
    cnt = warp_sum64(cnt);
    if (lane == 0 && cnt) atomicAdd(examined, cnt);
}

// ---- compaction: next bitmap -> sorted queue, n_f, m_f, visited |= next ----

__global__ void __launch_bounds__(kBitThreads) cmp_count_kernel(const uint64_t *__restrict__ next, uint64_t nwords,
                                                                uint32_t *tile_cnt)
{
    __shared__ uint32_t ws[kBitThreads / 32];
    const uint64_t w0 = (uint64_t)blockIdx.x * kTileWords + (uint64_t)threadIdx.x * kWordsPerThread;
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t j = 0; j < kWordsPerThread; j++)
        if (w0 + j < nwords) cnt += __popcll(next[w0 + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t i = 0; i < kBitThreads / 32; i++) t += ws[i];
        tile_cnt[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads) cmp_scan_kernel(const uint32_t *tile_cnt, uint32_t *tile_off,
                                                                uint64_t ntiles, Counters *ctr)
{
    __shared__ unsigned long long sm[33];
    const uint64_t chunk = (ntiles + kScanThreads - 1) / kScanThreads;
    const uint64_t t0 = (uint64_t)threadIdx.x * chunk, t1 = min(ntiles, t0 + chunk);
    unsigned long long local = 0, total = 0;
    for (uint64_t t = t0; t < t1; t++) local += tile_cnt[t];
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t t = t0; t < t1; t++) {
        tile_off[t] = (uint32_t)run;
        run += tile_cnt[t];
    }
    if (threadIdx.x == 0) {
        ctr->n_f = total;
        ctr->m_f = 0;
    }
}

__global__ void __launch_bounds__(kBitThreads) cmp_extract_kernel(const uint64_t *__restrict__ next, uint64_t nwords,
                                                                  const uint32_t *__restrict__ tile_off,
                                                                  uint64_t *visited, uint32_t *q,
                                                                  const int64_t *__restrict__ off, Counters *ctr)
{
    __shared__ unsigned long long sm[33];
    const uint64_t w0 = (uint64_t)blockIdx.x * kTileWords + (uint64_t)threadIdx.x * kWordsPerThread;
    uint64_t x[kWordsPerThread];
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t j = 0; j < kWordsPerThread; j++) {
        x[j] = (w0 + j < nwords) ? next[w0 + j] : 0ull;
        cnt += __popcll(x[j]);
        if (w0 + j < nwords && x[j]) visited[w0 + j] |= x[j];
    }
    unsigned long long total;
    unsigned long long pos = cta_excl_scan64<kBitThreads>(cnt, sm, &total) + tile_off[blockIdx.x];
    unsigned long long degsum = 0;
#pragma unroll
    for (uint32_t j = 0; j < kWordsPerThread; j++) {
        uint64_t y = x[j];
        while (y) {
            const uint32_t bit = __ffsll((long long)y) - 1;
            const uint32_t v = (uint32_t)((w0 + j) * 64u + bit);
            q[pos++] = v;
            degsum += (unsigned long long)(off[v + 1] - off[v]);
            y &= y - 1;
        }
    }
    degsum = warp_sum64(degsum);
    if ((threadIdx.x & 31u) == 0 && degsum) atomicAdd(&ctr->m_f, degsum);
}

}  // namespace

// ------------------------------------------------------------------ graph handle

struct fq_graph {
    const int64_t *off;
    const uint32_t *cols;
    uint64_t n, m, nwords;
    int device;
    uint8_t *mem;
    Counters *ctr;
    void *work;
    uint64_t work_bytes;
    Scratch sc;
    uint32_t *q, *q2;
    uint64_t *fbits, *fbits2, *next, *visited;
    uint8_t *qs, *bs, *vs;
    uint64_t qs_cap, bs_cap;
    HubItem *items;
    uint64_t items_cap;
    uint32_t *tile_cnt, *tile_off;
    uint64_t cmp_tiles;
    uint8_t *host;  // pinned: Counters + fq_device_status
    cudaEvent_t ev[2 * FQ_NUM_KCLASS];
};

namespace {

uint64_t al256(uint64_t x) { return (x + 255u) / 256u * 256u; }

struct Timer {
    fq_graph *g;
    cudaStream_t st;
    bool on;
    double *ms;
    uint64_t *launches;
    int open = -1;
    void begin(int k)
    {
        if (on) {
            cudaEventRecord(g->ev[2 * k], st);
            open = k;
        }
    }
    void end(int k, int nlaunch)
    {
        if (launches) launches[k] += nlaunch;
        if (on) cudaEventRecord(g->ev[2 * k + 1], st);
    }
    void collect(int k)
    {
        if (!on) return;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g->ev[2 * k], g->ev[2 * k + 1]) == cudaSuccess) ms[k] += t;
    }
};

}  // namespace

extern "C" {

fq_status fq_graph_create(const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, uint64_t m, fq_graph **out)
{
    if (!out || !d_offsets || (m && !d_cols) || n == 0 || n > 0xffffffffull) return FQ_EINVAL;
    *out = nullptr;
    fq_graph *g = new (std::nothrow) fq_graph();
    if (!g) return FQ_ENOMEM;
    g->off = d_offsets;
    g->cols = d_cols;
    g->n = n;
    g->m = m;
    g->nwords = cdiv(n, 64);
    cudaGetDevice(&g->device);

    const uint64_t nw = g->nwords + 2;  // +2: room for the 16-byte stream pads and u32 views
    g->work_bytes = workspace_bytes(n, n);
    g->qs_cap = fq_queue_bound(n);
    g->bs_cap = fq_bitmap_bound(n);
    g->items_cap = m / kHubChunk + m / kHubDegree + 16;  // every hub holds >= kHubDegree edges
    g->cmp_tiles = std::max<uint64_t>(1, cdiv(g->nwords, kTileWords));
    uint64_t o = 0;
    const uint64_t o_ctr = o; o = al256(o + sizeof(Counters));
    const uint64_t o_work = o; o = al256(o + g->work_bytes);
    const uint64_t o_q = o; o = al256(o + 4 * n);
    const uint64_t o_q2 = o; o = al256(o + 4 * n);
    const uint64_t o_fb = o; o = al256(o + 8 * nw);
    const uint64_t o_fb2 = o; o = al256(o + 8 * nw);
    const uint64_t o_next = o; o = al256(o + 8 * nw);
    const uint64_t o_vis = o; o = al256(o + 8 * nw);
    const uint64_t o_qs = o; o = al256(o + g->qs_cap);
    const uint64_t o_bs = o; o = al256(o + g->bs_cap);
    const uint64_t o_vs = o; o = al256(o + g->bs_cap);
    const uint64_t o_items = o; o = al256(o + sizeof(HubItem) * g->items_cap);
    const uint64_t o_tc = o; o = al256(o + 4 * g->cmp_tiles);
    const uint64_t o_to = o; o = al256(o + 4 * g->cmp_tiles);
    if (cudaMalloc(&g->mem, o) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return FQ_ENOMEM;
    }
    if (cudaMallocHost(&g->host, 512) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g->mem);
        delete g;
        return FQ_ENOMEM;
    }
    g->ctr = reinterpret_cast<Counters *>(g->mem + o_ctr);
    g->work = g->mem + o_work;
    g->sc = carve(g->work, n, n);
    g->q = reinterpret_cast<uint32_t *>(g->mem + o_q);
    g->q2 = reinterpret_cast<uint32_t *>(g->mem + o_q2);
    g->fbits = reinterpret_cast<uint64_t *>(g->mem + o_fb);
    g->fbits2 = reinterpret_cast<uint64_t *>(g->mem + o_fb2);
    g->next = reinterpret_cast<uint64_t *>(g->mem + o_next);
    g->visited = reinterpret_cast<uint64_t *>(g->mem + o_vis);
    g->qs = g->mem + o_qs;
    g->bs = g->mem + o_bs;
    g->vs = g->mem + o_vs;
    g->items = reinterpret_cast<HubItem *>(g->mem + o_items);
    g->tile_cnt = reinterpret_cast<uint32_t *>(g->mem + o_tc);
    g->tile_off = reinterpret_cast<uint32_t *>(g->mem + o_to);
    for (int i = 0; i < 2 * FQ_NUM_KCLASS; i++) cudaEventCreate(&g->ev[i]);
    if (cudaMemset(g->mem, 0, o) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        fq_graph_destroy(g);
        return FQ_ECUDA;
    }
    *out = g;
    return FQ_OK;
}

fq_status fq_graph_destroy(fq_graph *g)
{
    if (!g) return FQ_EINVAL;
    cudaDeviceSynchronize();
    for (int i = 0; i < 2 * FQ_NUM_KCLASS; i++)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    if (g->host) cudaFreeHost(g->host);
    if (g->mem) cudaFree(g->mem);
    delete g;
    return FQ_OK;
}

fq_status fq_bfs_run(fq_graph *g, uint32_t root, int32_t *d_depth, uint32_t *d_parent, const fq_bfs_opts *opts,
                     fq_bfs_stats *h_stats, fq_level_record *h_levels, uint32_t max_levels, uint8_t *d_stream_log,
                     uint64_t stream_log_cap, void *stream)
{
    if (!g || !d_depth || root >= g->n) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t alpha = (opts && opts->alpha) ? opts->alpha : 14u;
    const uint32_t beta = (opts && opts->beta) ? opts->beta : 24u;
    const uint32_t flags = opts ? opts->flags : 0u;
    const bool want_visited = flags & FQ_BFS_VISITED_STREAM;
    const uint64_t n = g->n, nwords = g->nwords;
    const int sms = num_sms();

    fq_bfs_stats stats;
    memset(&stats, 0, sizeof(stats));
    Timer tm{g, st, (flags & FQ_BFS_TIMING) != 0, stats.kernel_ms, stats.kernel_launches};

#define FQ_TRY(expr)                                  \
    do {                                              \
        if ((expr) != cudaSuccess) return FQ_ECUDA;   \
    } while (0)

    // ---- level 0 set-up
    tm.begin(FQ_K_OTHER);
    FQ_TRY(cudaMemsetAsync(d_depth, 0xff, 4 * n, st));
    if (d_parent) FQ_TRY(cudaMemsetAsync(d_parent, 0xff, 4 * n, st));
    FQ_TRY(cudaMemsetAsync(g->fbits, 0, 8 * (nwords + 2), st));
    FQ_TRY(cudaMemsetAsync(g->next, 0, 8 * (nwords + 2), st));
    FQ_TRY(cudaMemsetAsync(g->visited, 0, 8 * (nwords + 2), st));
    FQ_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(Counters), st));
    bfs_init_kernel<<<1, 1, 0, st>>>(g->off, root, d_depth, d_parent, g->q, g->fbits, g->visited, g->ctr);
    FQ_TRY(cudaGetLastError());
    tm.end(FQ_K_OTHER, 1);
    FQ_TRY(cudaMemcpyAsync(g->host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    FQ_TRY(cudaStreamSynchronize(st));
    tm.collect(FQ_K_OTHER);

    const Counters *hc = reinterpret_cast<const Counters *>(g->host);
    const fq_device_status *hs = reinterpret_cast<const fq_device_status *>(g->host + sizeof(Counters));
    uint64_t n_f = hc->n_f, m_f = hc->m_f;
    uint64_t visited_count = n_f;
    uint64_t m_u = g->m - m_f;
    int dir = FQ_TOP_DOWN;
    uint64_t log_used = 0;
    fq_status result = FQ_OK;

    for (uint32_t d = 0;; d++) {
        // 1. encode F_d
        tm.begin(FQ_K_ENCODE);
        FQ_TRY(reset_status(g->sc, st));
        FQ_TRY(encode_fq(g->q, n_f, nullptr, n_f, g->qs, g->qs_cap, reinterpret_cast<uint64_t *>(&g->ctr->q_bytes),
                         g->sc, st));
        FQ_TRY(encode_fb(g->fbits, n, g->bs, g->bs_cap, reinterpret_cast<uint64_t *>(&g->ctr->b_bytes), g->sc, st));
        if (want_visited)
            FQ_TRY(encode_fb(g->visited, n, g->vs, g->bs_cap, reinterpret_cast<uint64_t *>(&g->ctr->v_bytes), g->sc, st));
        tm.end(FQ_K_ENCODE, 1 + 3 + 7 + (want_visited ? 7 : 0));

        // 2. direction
        if (flags & FQ_BFS_FORCE_TOP_DOWN) dir = FQ_TOP_DOWN;
        else if (flags & FQ_BFS_FORCE_BOTTOM_UP) dir = FQ_BOTTOM_UP;
        else if (dir == FQ_TOP_DOWN && (unsigned __int128)m_f * alpha > (unsigned __int128)m_u) dir = FQ_BOTTOM_UP;
        else if (dir == FQ_BOTTOM_UP && (unsigned __int128)n_f * beta < (unsigned __int128)n) dir = FQ_TOP_DOWN;
        const int32_t newdepth = (int32_t)d + 1;

        // 3 + 4. decode the consumed form, expand
        if (dir == FQ_TOP_DOWN) {
            tm.begin(FQ_K_DECODE);
            FQ_TRY(decode_fq(g->qs, 0, reinterpret_cast<const uint64_t *>(&g->ctr->q_bytes), g->q2, n_f,
                             reinterpret_cast<uint64_t *>(&g->ctr->dec_n), g->sc, st));
            tm.end(FQ_K_DECODE, 2);
            tm.begin(FQ_K_TOP_DOWN);
            // one warp per 32 frontier vertices
            const uint32_t grid = (uint32_t)std::min<uint64_t>(cdiv(std::max<uint64_t>(n_f, 1), kThreads), (uint64_t)sms * 8);
            td_expand_kernel<<<std::max<uint32_t>(grid, 1), kThreads, 0, st>>>(
                g->q2, n_f, g->off, g->cols, reinterpret_cast<const uint32_t *>(g->visited),
                reinterpret_cast<uint32_t *>(g->next), d_depth, d_parent, newdepth, g->items, &g->ctr->hub_items,
                g->items_cap, n, g->sc.ctl);
            td_hub_kernel<<<sms * 4, kThreads, 0, st>>>(g->items, &g->ctr->hub_items, g->items_cap, g->cols,
                                                        reinterpret_cast<const uint32_t *>(g->visited),
                                                        reinterpret_cast<uint32_t *>(g->next), d_depth, d_parent, newdepth);
            FQ_TRY(cudaGetLastError());
            tm.end(FQ_K_TOP_DOWN, 2);
        } else {
            tm.begin(FQ_K_DECODE);
            FQ_TRY(decode_fb(g->bs, 0, reinterpret_cast<const uint64_t *>(&g->ctr->b_bytes), g->fbits2, n, g->sc, st));
            tm.end(FQ_K_DECODE, 3);
            tm.begin(FQ_K_BOTTOM_UP);
            const uint64_t words32 = cdiv(n, 32);
            const uint32_t grid = (uint32_t)std::min<uint64_t>(cdiv(words32, kThreads / 32), (uint64_t)sms * 16);
            bu_sweep_kernel<<<std::max<uint32_t>(grid, 1), kThreads, 0, st>>>(
                reinterpret_cast<const uint32_t *>(g->fbits2), reinterpret_cast<const uint32_t *>(g->visited),
                reinterpret_cast<uint32_t *>(g->next), g->off, g->cols, d_depth, d_parent, newdepth, n,
                &g->ctr->examined);
            FQ_TRY(cudaGetLastError());
            tm.end(FQ_K_BOTTOM_UP, 1);
        }

        // 5. compaction
        tm.begin(FQ_K_COMPACT);
        cmp_count_kernel<<<(uint32_t)g->cmp_tiles, kBitThreads, 0, st>>>(g->next, nwords, g->tile_cnt);
        cmp_scan_kernel<<<1, kScanThreads, 0, st>>>(g->tile_cnt, g->tile_off, g->cmp_tiles, g->ctr);
        cmp_extract_kernel<<<(uint32_t)g->cmp_tiles, kBitThreads, 0, st>>>(g->next, nwords, g->tile_off, g->visited,
                                                                          g->q, g->off, g->ctr);
        FQ_TRY(cudaGetLastError());
        tm.end(FQ_K_COMPACT, 3);

        FQ_TRY(cudaMemcpyAsync(g->host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        FQ_TRY(cudaMemcpyAsync(g->host + sizeof(Counters), g->sc.ctl, sizeof(fq_device_status), cudaMemcpyDeviceToHost, st));
        FQ_TRY(cudaStreamSynchronize(st));
        tm.collect(FQ_K_ENCODE);
        tm.collect(FQ_K_DECODE);
        tm.collect(dir == FQ_TOP_DOWN ? FQ_K_TOP_DOWN : FQ_K_BOTTOM_UP);
        tm.collect(FQ_K_COMPACT);
        if (hs->code != FQ_OK) return hs->code;
        if (dir == FQ_TOP_DOWN && hc->dec_n != n_f) return FQ_ECORRUPT;

        const uint64_t examined = dir == FQ_TOP_DOWN ? m_f : hc->examined;
        const uint64_t nf_next = hc->n_f, mf_next = hc->m_f;
        const uint64_t qb = hc->q_bytes, bb = hc->b_bytes, vb = want_visited ? hc->v_bytes : 0;

        // algorithmic bytes of this level (design model)
        stats.kernel_bytes[FQ_K_ENCODE] += 4 * n_f + qb + (n + 7) / 8 + bb + (want_visited ? (n + 7) / 8 + vb : 0);
        if (dir == FQ_TOP_DOWN) {
            stats.kernel_bytes[FQ_K_DECODE] += qb + 4 * n_f;
            stats.kernel_bytes[FQ_K_TOP_DOWN] += 4 * examined + 20 * n_f + 8 * nf_next;
        } else {
            stats.kernel_bytes[FQ_K_DECODE] += bb + (n + 7) / 8;
            stats.kernel_bytes[FQ_K_BOTTOM_UP] += 3 * ((n + 7) / 8) + 16 * (n - visited_count) + 4 * examined + 8 * nf_next;
        }
        stats.kernel_bytes[FQ_K_COMPACT] += 3 * ((n + 7) / 8) + 20 * nf_next;

        uint64_t log_off = ~0ull;
        if (d_stream_log) {
            const uint64_t need = qb + bb + vb;
            if (log_used + need > stream_log_cap) {
                result = FQ_ENOSPC;
            } else {
                log_off = log_used;
                FQ_TRY(cudaMemcpyAsync(d_stream_log + log_used, g->qs, qb, cudaMemcpyDeviceToDevice, st));
                FQ_TRY(cudaMemcpyAsync(d_stream_log + log_used + qb, g->bs, bb, cudaMemcpyDeviceToDevice, st));
                if (vb) FQ_TRY(cudaMemcpyAsync(d_stream_log + log_used + qb + bb, g->vs, vb, cudaMemcpyDeviceToDevice, st));
                log_used += need;
            }
        }
        if (h_levels && d < max_levels) {
            fq_level_record &r = h_levels[d];
            r.level = d;
            r.direction = (uint32_t)dir;
            r.n_f = n_f;
            r.m_f = m_f;
            r.m_u = m_u;
            r.examined = examined;
            r.q_bytes = qb;
            r.b_bytes = bb;
            r.v_bytes = vb;
            r.log_offset = log_off;
        }
        stats.levels = d + 1;
        if (dir == FQ_BOTTOM_UP && d < 32) stats.directions |= 1u << d;
        stats.reached += n_f;
        stats.reached_edges += m_f;
        stats.edges_examined += examined;
        stats.raw_queue_bytes += 4 * n_f;
        stats.enc_queue_bytes += qb;
        stats.raw_bitmap_bytes += (n + 7) / 8;
        stats.enc_bitmap_bytes += bb;
        stats.enc_visited_bytes += vb;

        if (nf_next == 0) break;
        // next level: F_{d+1} is in q (queue) and next (bitmap); swap bitmaps and clear the new next
        std::swap(g->fbits, g->next);
        tm.begin(FQ_K_OTHER);
        FQ_TRY(cudaMemsetAsync(g->next, 0, 8 * (nwords + 2), st));
        FQ_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(Counters), st));
        tm.end(FQ_K_OTHER, 0);
        n_f = nf_next;
        m_f = mf_next;
        visited_count += n_f;
        m_u -= m_f;
        if ((uint64_t)d + 1 >= n) return FQ_ECORRUPT;  // every level discovers a vertex: at most n levels
    }
    FQ_TRY(cudaStreamSynchronize(st));
    tm.collect(FQ_K_OTHER);
    stats.reached_edges /= 2;
    if (h_stats) *h_stats = stats;
#undef FQ_TRY
    return result;
}

}  // extern "C"
