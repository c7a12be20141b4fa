// bfs.cu -- level-synchronous, direction-optimising BFS with the per-level frontier codec
// stage, and its C ABI (fq_graph_create / fq_graph_destroy / fq_bfs_run).
//
// One level d (the loop of Alg. "Our BFS algorithm with SpVM and compression", on one GPU):
//   1. encode F_d as Q_d (sorted queue, FQ) and B_d (bitmap, FB), and the visited bitmap as
//      V_d -- the compress steps before the thesis' ALLGATHERV/ALLTOALLV; the byte counts are
//      the exchange volume.  When 2|F_d| <= n the set positions of the frontier bitmap are the
//      queue itself, so one single-pass encode writes Q_d and B_d together; V_d's positions were
//      extracted by the previous level's compaction;
//   2. choose the direction from (n_f, m_f, m_u): top-down -> bottom-up when m_f*alpha > m_u,
//      back when n_f*beta < n (direction optimisation, sec. 3.1);
//   3. decode the form that direction consumes (Q_d for top-down, B_d for bottom-up) -- the
//      decompress step;
//   4. expand: top-down over the decoded queue (t = A (x) f masked by the visited list) or
//      bottom-up against the decoded bitmap; depth/parent written by the discovering thread;
//   5. compact the next-frontier bitmap into the sorted queue F_{d+1} (popcount + prefix sum,
//      sec. 3.1 "Sparse vector with pop counting"), visited |= next, count n_f and m_f, and
//      extract the positions V_{d+1} will code.
// The host reads one 256-byte counter record per level (termination test and direction).
#include <algorithm>
#include <cstring>
#include <new>

#include "fq_common.cuh"

using namespace fq;

namespace {

constexpr uint32_t kHubDegree = 256;   // top-down: vertices of at least this degree are split
constexpr uint32_t kHubChunk = 2048;   //   into chunks of this many edges, one CTA each
constexpr uint32_t kThreads = 256;
constexpr uint32_t kCmpWordsPerThread = 1;
constexpr uint32_t kCmpWords = kThreads * kCmpWordsPerThread;  // 256 words = 16384 vertices per tile

struct HubItem {
    uint32_t v;
    uint32_t count;
    unsigned long long start;
};

// Device counters (first 256 bytes of the handle's allocation).  "live" fields are updated
// during a level; cmp_scan_kernel copies the ones it clears into the r_* record the host reads.
struct Counters {
    unsigned long long n_f_next;   // |F_{d+1}|                         (cmp_scan)
    unsigned long long m_f_next;   // live: degree sum over F_{d+1}     (expansion kernels)
    unsigned long long examined;   // live: bottom-up adjacency reads
    unsigned long long hub_items;  // live: top-down hub work items
    unsigned long long q_bytes, b_bytes, v_bytes, dec_n;
    unsigned long long r_examined, r_hub_items, vis_count, v_count, r_m_f;
    int32_t r_err_q, r_err_v;
    uint32_t r_where_q, r_where_v;
    unsigned long long r_detail_q, r_detail_v;
    unsigned long long pad[15];
};
static_assert(sizeof(Counters) == 256, "counter block is 256 bytes");

// Top-down visit of edge (src, w): the thread whose atomicOr sets w's bit in the next-frontier
// bitmap discovers w, writes depth and parent, and returns deg(w) for the next level's m_f.
__device__ __forceinline__ unsigned long long td_visit(uint32_t w, uint32_t src, const uint32_t *__restrict__ visited32,
                                                       uint32_t *next32, int32_t *depth, uint32_t *parent,
                                                       int32_t newdepth, const int64_t *__restrict__ off)
{
    const uint32_t bit = 1u << (w & 31u), wi = w >> 5;
    if (visited32[wi] & bit) return 0;
    if (next32[wi] & bit) return 0;
    const uint32_t old = atomicOr(&next32[wi], bit);
    if (old & bit) return 0;
    depth[w] = newdepth;
    if (parent) parent[w] = src;
    return (unsigned long long)(off[w + 1] - off[w]);
}

// Level 0: the root, V_0's single position, cleared codec scratch.
__global__ void bfs_init_kernel(const int64_t *off, uint32_t root, uint64_t n, int32_t *depth, uint32_t *parent,
                                uint32_t *q, uint64_t *fbits, uint64_t *visited, uint32_t *vis_cnt, Counters *ctr,
                                Scratch sq, Scratch sv)
{
    reset_scratch_device(sq, 1, threadIdx.x, blockDim.x);
    reset_scratch_device(sv, 1, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x != 0) return;
    depth[root] = 0;
    if (parent) parent[root] = root;
    q[0] = root;
    fbits[root >> 6] |= 1ull << (root & 63u);
    visited[root >> 6] |= 1ull << (root & 63u);
    vis_cnt[root / (64u * kCmpWords)] = 1;
    ctr->n_f_next = 1;
    ctr->r_m_f = (unsigned long long)(off[root + 1] - off[root]);
    ctr->m_f_next = 0;
    ctr->vis_count = 1;
    // V_0 codes {root}: its position in SET mode, or no clear position when n == 1
    if (2u <= n) {
        sv.ctl->fb_mode = kFbSet;
        sv.ctl->n = 1;
        sv.positions[0] = root;
    } else {
        sv.ctl->fb_mode = kFbClear;
        sv.ctl->n = 0;
    }
}

// Bitmap of the zero-degree vertices: they are never reached, so the sweep treats them as done.
__global__ void iso_kernel(const int64_t *off, uint64_t n, uint32_t *iso32)
{
    const uint64_t nw = (n + 31) / 32;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0;
        for (uint32_t b = 0; b < 32; b++) {
            const uint64_t v = w * 32 + b;
            if (v < n && off[v + 1] == off[v]) m |= 1u << b;
        }
        iso32[w] = m;
    }
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
                                                             unsigned long long items_cap, uint64_t n, Ctl *err,
                                                             unsigned long long *m_f_next)
{
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long degsum = 0;
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
            if (idx < total) degsum += td_visit(cols[ss + (idx - ps)], src, visited32, next32, depth, parent, newdepth, off);
        }
    }
    degsum = warp_sum64(degsum);
    if (lane == 0 && degsum) atomicAdd(m_f_next, degsum);
}

__global__ void __launch_bounds__(kThreads) td_hub_kernel(const HubItem *__restrict__ items,
                                                          const unsigned long long *nitems, unsigned long long items_cap,
                                                          const uint32_t *__restrict__ cols,
                                                          const uint32_t *__restrict__ visited32, uint32_t *next32,
                                                          int32_t *depth, uint32_t *parent, int32_t newdepth,
                                                          const int64_t *__restrict__ off, unsigned long long *m_f_next)
{
    const unsigned long long total = min(*nitems, items_cap);
    unsigned long long degsum = 0;
    for (unsigned long long it = blockIdx.x; it < total; it += gridDim.x) {
        const HubItem h = items[it];
        for (uint32_t j = threadIdx.x; j < h.count; j += blockDim.x)
            degsum += td_visit(cols[h.start + j], h.v, visited32, next32, depth, parent, newdepth, off);
    }
    degsum = warp_sum64(degsum);
    if ((threadIdx.x & 31u) == 0 && degsum) atomicAdd(m_f_next, degsum);
}

// Bottom-up sweep: one thread per vertex; an unvisited vertex scans its adjacency in CSR order
// (two entries per step, for memory parallelism) and stops at the first neighbour in the
// (decoded) frontier bitmap.  The 32 vertices of a warp share one 32-bit word of the next-frontier
// bitmap, written whole by lane 0 from a ballot, so the sweep needs no atomics.  Words whose
// vertices are all visited or of degree 0 are skipped without touching the graph.
__global__ void __launch_bounds__(kThreads) bu_sweep_kernel(const uint32_t *__restrict__ front32,
                                                            const uint32_t *__restrict__ visited32,
                                                            const uint32_t *__restrict__ iso32,
                                                            uint32_t *__restrict__ next32,
                                                            const int64_t *__restrict__ off,
                                                            const uint32_t *__restrict__ cols, int32_t *depth,
                                                            uint32_t *parent, int32_t newdepth, uint64_t n,
                                                            unsigned long long *examined, unsigned long long *m_f_next)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cnt = 0, degsum = 0;
    for (uint64_t word = gw; word * 32u < n; word += nw) {
        const uint32_t done = visited32[word] | iso32[word];
        if (done == 0xffffffffu) continue;
        const uint64_t w = word * 32u + lane;
        bool found = false;
        uint32_t par = 0;
        if (w < n && !((done >> lane) & 1u)) {
            const long long s = off[w], e = off[w + 1];
            long long j = s;
            for (; j + 1 < e; j += 2) {
                const uint32_t u0 = cols[j], u1 = cols[j + 1];
                const bool h0 = (front32[u0 >> 5] >> (u0 & 31u)) & 1u;
                const bool h1 = (front32[u1 >> 5] >> (u1 & 31u)) & 1u;
                if (h0 || h1) {
                    found = true;
                    par = h0 ? u0 : u1;
                    j += h0 ? 1 : 2;
                    break;
                }
            }
            if (!found && j < e) {
                const uint32_t u0 = cols[j];
                j += 1;
                if ((front32[u0 >> 5] >> (u0 & 31u)) & 1u) {
                    found = true;
                    par = u0;
                }
            }
            cnt += (unsigned long long)(j - s);
            if (found) degsum += (unsigned long long)(e - s);
        }
        if (found) {
            depth[w] = newdepth;
            if (parent) parent[w] = par;
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, found);
        if (lane == 0 && mask) next32[word] = mask;
    }
    cnt = warp_sum64(cnt);
    degsum = warp_sum64(degsum);
    if (lane == 0 && cnt) atomicAdd(examined, cnt);
    if (lane == 0 && degsum) atomicAdd(m_f_next, degsum);
}

// ---- compaction: next bitmap -> sorted queue, n_f, m_f, visited |= next, V positions ----

__device__ __forceinline__ uint64_t bits_in_word(uint64_t w, uint64_t nwords, uint64_t n)
{
    if (w >= nwords) return 0;
    const uint32_t tail = (uint32_t)(n & 63u);
    return (w == nwords - 1 && tail) ? tail : 64u;
}

__global__ void __launch_bounds__(kThreads) cmp_count_kernel(const uint64_t *__restrict__ next, uint64_t *visited,
                                                             uint64_t nwords, uint32_t *tile_cnt, uint32_t *vis_cnt)
{
    __shared__ uint32_t ws[kThreads / 32];
    const uint64_t w0 = (uint64_t)blockIdx.x * kCmpWords + (uint64_t)threadIdx.x * kCmpWordsPerThread;
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t j = 0; j < kCmpWordsPerThread; j++) {
        if (w0 + j < nwords) {
            const uint64_t x = next[w0 + j];
            if (x) {
                visited[w0 + j] |= x;
                cnt += __popcll(x);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t i = 0; i < kThreads / 32; i++) t += ws[i];
        tile_cnt[blockIdx.x] = t;
        vis_cnt[blockIdx.x] += t;  // the next frontier is disjoint from the visited set
    }
}

// One CTA: offsets of the next-frontier positions and of V's positions (set or clear bits of the
// visited bitmap), the level record, and cleared codec scratch for the next level.
__global__ void __launch_bounds__(kScanThreads) cmp_scan_kernel(const uint32_t *tile_cnt, uint32_t *tile_off,
                                                                const uint32_t *vis_cnt, uint32_t *vtile_off,
                                                                uint64_t ntiles, uint64_t n, Counters *ctr,
                                                                Scratch sq, Scratch sv)
{
    __shared__ unsigned long long sm[33];
    __shared__ unsigned long long s_nf, s_vis;
    const uint64_t chunk = (ntiles + kScanThreads - 1) / kScanThreads;
    const uint64_t t0 = (uint64_t)threadIdx.x * chunk, t1 = min(ntiles, t0 + chunk);
    const uint64_t tile_bits = 64ull * kCmpWords;
    unsigned long long local = 0, total = 0;
    for (uint64_t t = t0; t < t1; t++) local += tile_cnt[t];
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t t = t0; t < t1; t++) {
        tile_off[t] = (uint32_t)run;
        run += tile_cnt[t];
    }
    if (threadIdx.x == 0) s_nf = total;
    local = 0;
    for (uint64_t t = t0; t < t1; t++) local += vis_cnt[t];
    cta_excl_scan64<kScanThreads>(local, sm, &total);
    if (threadIdx.x == 0) s_vis = total;
    __syncthreads();
    const bool set_mode = 2ull * s_vis <= n;
    local = 0;
    for (uint64_t t = t0; t < t1; t++) {
        const uint64_t bits = min(n, (t + 1) * tile_bits) - t * tile_bits;
        local += set_mode ? vis_cnt[t] : bits - vis_cnt[t];
    }
    run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t t = t0; t < t1; t++) {
        vtile_off[t] = (uint32_t)run;
        const uint64_t bits = min(n, (t + 1) * tile_bits) - t * tile_bits;
        run += set_mode ? vis_cnt[t] : bits - vis_cnt[t];
    }
    const unsigned long long vcount = total;
    // snapshot the level's live counters and codec status, then clear for the next level
    if (threadIdx.x == 0) {
        ctr->n_f_next = s_nf;
        ctr->r_m_f = ctr->m_f_next;  // summed by the expansion kernels
        ctr->m_f_next = 0;
        ctr->vis_count = s_vis;
        ctr->v_count = vcount;
        ctr->r_examined = ctr->examined;
        ctr->examined = 0;
        ctr->r_hub_items = ctr->hub_items;
        ctr->hub_items = 0;
        ctr->r_err_q = sq.ctl->code;
        ctr->r_where_q = sq.ctl->where;
        ctr->r_detail_q = sq.ctl->detail;
        ctr->r_err_v = sv.ctl->code;
        ctr->r_where_v = sv.ctl->where;
        ctr->r_detail_v = sv.ctl->detail;
    }
    __syncthreads();
    const uint64_t qtiles = min((uint64_t)sq.etiles_cap, (uint64_t)((s_nf + 8191) / 8192 + 1));
    const uint64_t vtiles = min((uint64_t)sv.etiles_cap, (uint64_t)((vcount + 8191) / 8192 + 1));
    reset_scratch_device(sq, qtiles, threadIdx.x, blockDim.x);
    reset_scratch_device(sv, vtiles, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        sv.ctl->n = vcount;
        sv.ctl->fb_mode = set_mode ? kFbSet : kFbClear;
    }
}

__global__ void __launch_bounds__(kThreads) cmp_extract_kernel(uint64_t *__restrict__ next, uint64_t *__restrict__ fbits,
                                                               const uint64_t *__restrict__ visited, uint64_t nwords,
                                                               uint64_t n, const uint32_t *__restrict__ tile_off,
                                                               const uint32_t *__restrict__ vtile_off, uint32_t *q,
                                                               Scratch sv)
{
    __shared__ unsigned long long sm[33];
    const uint64_t w0 = (uint64_t)blockIdx.x * kCmpWords + (uint64_t)threadIdx.x * kCmpWordsPerThread;
    const bool v_clear = sv.ctl->fb_mode == kFbClear;
    uint64_t x[kCmpWordsPerThread], y[kCmpWordsPerThread];
    uint32_t cnt = 0, vcnt = 0;
#pragma unroll
    for (uint32_t j = 0; j < kCmpWordsPerThread; j++) {
        const uint64_t w = w0 + j;
        x[j] = 0;
        y[j] = 0;
        if (w < nwords) {
            x[j] = next[w];
            fbits[w] = x[j];  // F_{d+1} as a bitmap for the next level's B encode
            if (x[j]) next[w] = 0;
            uint64_t vis = visited[w];
            if (v_clear) {
                const uint64_t nb = bits_in_word(w, nwords, n);
                vis = ~vis & (nb == 64 ? ~0ull : ((1ull << nb) - 1ull));
            }
            y[j] = vis;
        }
        cnt += __popcll(x[j]);
        vcnt += __popcll(y[j]);
    }
    unsigned long long total;
    unsigned long long pos = cta_excl_scan64<kThreads>(cnt, sm, &total) + tile_off[blockIdx.x];
    unsigned long long vpos = cta_excl_scan64<kThreads>(vcnt, sm, &total) + vtile_off[blockIdx.x];
#pragma unroll
    for (uint32_t j = 0; j < kCmpWordsPerThread; j++) {
        uint64_t a = x[j];
        while (a) {
            const uint32_t bit = __ffsll((long long)a) - 1;
            q[pos++] = (uint32_t)((w0 + j) * 64u + bit);
            a &= a - 1;
        }
        uint64_t b = y[j];
        while (b) {
            const uint32_t bit = __ffsll((long long)b) - 1;
            sv.positions[vpos++] = (uint32_t)((w0 + j) * 64u + bit);
            b &= b - 1;
        }
    }
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
    Scratch sq, sv;   // codec scratch: Q/B streams and decodes; V stream
    uint32_t *q, *q2;
    uint64_t *fbits, *fbits2, *next, *visited;
    uint32_t *iso32;
    uint8_t *qs, *bs, *vs;
    uint64_t qs_cap, bs_cap;
    HubItem *items;
    uint64_t items_cap;
    uint32_t *tile_cnt, *tile_off, *vis_cnt, *vtile_off;
    uint64_t cmp_tiles;
    uint8_t *host;  // pinned copy of Counters
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
    void begin(int k)
    {
        if (on) cudaEventRecord(g->ev[2 * k], st);
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
    const uint64_t work_q = workspace_bytes(n, n);
    const uint64_t work_v = workspace_bytes(0, n);
    g->qs_cap = fq_queue_bound(n);
    g->bs_cap = fq_bitmap_bound(n);
    g->items_cap = m / kHubChunk + m / kHubDegree + 16;  // every hub holds >= kHubDegree edges
    g->cmp_tiles = std::max<uint64_t>(1, cdiv(g->nwords, kCmpWords));
    uint64_t o = 0;
    const uint64_t o_ctr = o; o = al256(o + sizeof(Counters));
    const uint64_t o_wq = o; o = al256(o + work_q);
    const uint64_t o_wv = o; o = al256(o + work_v);
    const uint64_t o_q = o; o = al256(o + 4 * n);
    const uint64_t o_q2 = o; o = al256(o + 4 * n);
    const uint64_t o_fb = o; o = al256(o + 8 * nw);
    const uint64_t o_fb2 = o; o = al256(o + 8 * nw);
    const uint64_t o_next = o; o = al256(o + 8 * nw);
    const uint64_t o_vis = o; o = al256(o + 8 * nw);
    const uint64_t o_iso = o; o = al256(o + 8 * nw);
    const uint64_t o_qs = o; o = al256(o + g->qs_cap);
    const uint64_t o_bs = o; o = al256(o + g->bs_cap);
    const uint64_t o_vs = o; o = al256(o + g->bs_cap);
    const uint64_t o_items = o; o = al256(o + sizeof(HubItem) * g->items_cap);
    const uint64_t o_tc = o; o = al256(o + 4 * g->cmp_tiles);
    const uint64_t o_to = o; o = al256(o + 4 * g->cmp_tiles);
    const uint64_t o_vc = o; o = al256(o + 4 * g->cmp_tiles);
    const uint64_t o_vo = o; o = al256(o + 4 * g->cmp_tiles);
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
    g->sq = carve(g->mem + o_wq, n, n);
    g->sv = carve(g->mem + o_wv, 0, n);
    g->q = reinterpret_cast<uint32_t *>(g->mem + o_q);
    g->q2 = reinterpret_cast<uint32_t *>(g->mem + o_q2);
    g->fbits = reinterpret_cast<uint64_t *>(g->mem + o_fb);
    g->fbits2 = reinterpret_cast<uint64_t *>(g->mem + o_fb2);
    g->next = reinterpret_cast<uint64_t *>(g->mem + o_next);
    g->visited = reinterpret_cast<uint64_t *>(g->mem + o_vis);
    g->iso32 = reinterpret_cast<uint32_t *>(g->mem + o_iso);
    g->qs = g->mem + o_qs;
    g->bs = g->mem + o_bs;
    g->vs = g->mem + o_vs;
    g->items = reinterpret_cast<HubItem *>(g->mem + o_items);
    g->tile_cnt = reinterpret_cast<uint32_t *>(g->mem + o_tc);
    g->tile_off = reinterpret_cast<uint32_t *>(g->mem + o_to);
    g->vis_cnt = reinterpret_cast<uint32_t *>(g->mem + o_vc);
    g->vtile_off = reinterpret_cast<uint32_t *>(g->mem + o_vo);
    for (int i = 0; i < 2 * FQ_NUM_KCLASS; i++) cudaEventCreate(&g->ev[i]);
    if (cudaMemset(g->mem, 0, o) != cudaSuccess) {
        fq_graph_destroy(g);
        return FQ_ECUDA;
    }
    iso_kernel<<<(uint32_t)std::min<uint64_t>(cdiv(cdiv(n, 32), 256), 4096), 256>>>(d_offsets, n, g->iso32);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
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
    const bool codec = !(flags & FQ_BFS_NO_CODEC);
    const bool want_visited = codec && (flags & FQ_BFS_VISITED_STREAM);
    const uint64_t n = g->n, nwords = g->nwords;
    const int sms = num_sms();
    uint32_t *next32 = reinterpret_cast<uint32_t *>(g->next);
    const uint32_t *vis32 = reinterpret_cast<const uint32_t *>(g->visited);

    fq_bfs_stats stats;
    memset(&stats, 0, sizeof(stats));
    Timer tm{g, st, (flags & FQ_BFS_TIMING) != 0, stats.kernel_ms, stats.kernel_launches};

#define FQ_TRY(expr)                                  \
    do {                                              \
        const cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) {                      \
            note_cuda_error(_e, __LINE__);            \
            return FQ_ECUDA;                          \
        }                                             \
    } while (0)

    // ---- level 0 set-up
    tm.begin(FQ_K_OTHER);
    FQ_TRY(cudaMemsetAsync(d_depth, 0xff, 4 * n, st));
    if (d_parent) FQ_TRY(cudaMemsetAsync(d_parent, 0xff, 4 * n, st));
    FQ_TRY(cudaMemsetAsync(g->fbits, 0, 8 * (nwords + 2), st));
    FQ_TRY(cudaMemsetAsync(g->next, 0, 8 * (nwords + 2), st));
    FQ_TRY(cudaMemsetAsync(g->visited, 0, 8 * (nwords + 2), st));
    FQ_TRY(cudaMemsetAsync(g->vis_cnt, 0, 4 * g->cmp_tiles, st));
    FQ_TRY(cudaMemsetAsync(g->ctr, 0, sizeof(Counters), st));
    bfs_init_kernel<<<1, 256, 0, st>>>(g->off, root, n, d_depth, d_parent, g->q, g->fbits, g->visited, g->vis_cnt,
                                       g->ctr, g->sq, g->sv);
    FQ_TRY(cudaGetLastError());
    tm.end(FQ_K_OTHER, 1);
    FQ_TRY(cudaMemcpyAsync(g->host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    FQ_TRY(cudaStreamSynchronize(st));
    tm.collect(FQ_K_OTHER);

    const Counters *hc = reinterpret_cast<const Counters *>(g->host);
    uint64_t n_f = hc->n_f_next, m_f = hc->r_m_f;
    uint64_t visited_count = n_f;
    uint64_t m_u = g->m - m_f;
    int dir = FQ_TOP_DOWN;
    uint64_t log_used = 0;
    fq_status result = FQ_OK;
    unsigned long long *q_bytes = &g->ctr->q_bytes, *b_bytes = &g->ctr->b_bytes, *v_bytes = &g->ctr->v_bytes;

    for (uint32_t d = 0;; d++) {
        // 1. encode F_d (Q_d and B_d), and V_d
        tm.begin(FQ_K_ENCODE);
        int enc_launches = 2;
        if (!codec) {
            enc_launches = 0;
        } else if (2 * n_f <= n) {
            Mirror mb;
            mb.out = g->bs;
            mb.cap = g->bs_cap;
            mb.out_bytes = reinterpret_cast<uint64_t *>(b_bytes);
            mb.words = g->fbits;
            mb.nbits = n;
            FQ_TRY(encode_fq_mirror(g->q, n_f, nullptr, n_f, g->qs, g->qs_cap, reinterpret_cast<uint64_t *>(q_bytes),
                                    mb, g->sq, st));
        } else {  // a frontier denser than half the vertices: its bitmap codes the clear positions
            FQ_TRY(encode_fq(g->q, n_f, nullptr, n_f, g->qs, g->qs_cap, reinterpret_cast<uint64_t *>(q_bytes), g->sq, st));
            FQ_TRY(reset_status(g->sq, n / 2 + 1, st));
            FQ_TRY(encode_fb(g->fbits, n, g->bs, g->bs_cap, reinterpret_cast<uint64_t *>(b_bytes), g->sq, st));
            enc_launches += 6;
        }
        if (want_visited) {
            FQ_TRY(encode_fb_positions(g->visited, n, g->vs, g->bs_cap, reinterpret_cast<uint64_t *>(v_bytes), g->sv, st));
            enc_launches += 2;
        }
        tm.end(FQ_K_ENCODE, enc_launches);

        // 2. direction
        if (flags & FQ_BFS_FORCE_TOP_DOWN) dir = FQ_TOP_DOWN;
        else if (flags & FQ_BFS_FORCE_BOTTOM_UP) dir = FQ_BOTTOM_UP;
        else if (dir == FQ_TOP_DOWN && (unsigned __int128)m_f * alpha > (unsigned __int128)m_u) dir = FQ_BOTTOM_UP;
        else if (dir == FQ_BOTTOM_UP && (unsigned __int128)n_f * beta < (unsigned __int128)n) dir = FQ_TOP_DOWN;
        const int32_t newdepth = (int32_t)d + 1;

        // 3 + 4. decode the consumed form, expand
        if (dir == FQ_TOP_DOWN) {
            tm.begin(FQ_K_DECODE);
            if (codec)
                FQ_TRY(decode_fq(g->qs, 0, reinterpret_cast<const uint64_t *>(q_bytes), g->q2, n_f,
                                 reinterpret_cast<uint64_t *>(&g->ctr->dec_n), g->sq, st));
            tm.end(FQ_K_DECODE, codec ? 3 : 0);
            const uint32_t *qin = codec ? g->q2 : g->q;
            tm.begin(FQ_K_TOP_DOWN);
            const uint32_t grid = (uint32_t)std::min<uint64_t>(cdiv(std::max<uint64_t>(n_f, 1), kThreads), (uint64_t)sms * 8);
            td_expand_kernel<<<grid, kThreads, 0, st>>>(qin, n_f, g->off, g->cols, vis32, next32, d_depth, d_parent,
                                                        newdepth, g->items, &g->ctr->hub_items, g->items_cap, n,
                                                        g->sq.ctl, &g->ctr->m_f_next);
            td_hub_kernel<<<sms * 4, kThreads, 0, st>>>(g->items, &g->ctr->hub_items, g->items_cap, g->cols, vis32,
                                                        next32, d_depth, d_parent, newdepth, g->off, &g->ctr->m_f_next);
            FQ_TRY(cudaGetLastError());
            tm.end(FQ_K_TOP_DOWN, 2);
        } else {
            tm.begin(FQ_K_DECODE);
            if (codec) FQ_TRY(decode_fb(g->bs, 0, reinterpret_cast<const uint64_t *>(b_bytes), g->fbits2, n, g->sq, st));
            tm.end(FQ_K_DECODE, codec ? 4 : 0);
            const uint64_t *fin = codec ? g->fbits2 : g->fbits;
            tm.begin(FQ_K_BOTTOM_UP);
            const uint64_t words32 = cdiv(n, 32);
            const uint32_t grid = (uint32_t)std::min<uint64_t>(cdiv(words32, kThreads / 32), (uint64_t)sms * 16);
            bu_sweep_kernel<<<std::max<uint32_t>(grid, 1), kThreads, 0, st>>>(
                reinterpret_cast<const uint32_t *>(fin), vis32, g->iso32, next32, g->off, g->cols, d_depth,
                d_parent, newdepth, n, &g->ctr->examined, &g->ctr->m_f_next);
            FQ_TRY(cudaGetLastError());
            tm.end(FQ_K_BOTTOM_UP, 1);
        }

        // 5. compaction (+ V_{d+1} positions, cleared scratch for the next level)
        tm.begin(FQ_K_COMPACT);
        const uint32_t ct = (uint32_t)g->cmp_tiles;
        cmp_count_kernel<<<ct, kThreads, 0, st>>>(g->next, g->visited, nwords, g->tile_cnt, g->vis_cnt);
        cmp_scan_kernel<<<1, kScanThreads, 0, st>>>(g->tile_cnt, g->tile_off, g->vis_cnt, g->vtile_off, g->cmp_tiles, n,
                                                    g->ctr, g->sq, g->sv);
        cmp_extract_kernel<<<ct, kThreads, 0, st>>>(g->next, g->fbits, g->visited, nwords, n, g->tile_off, g->vtile_off,
                                                    g->q, g->sv);
        FQ_TRY(cudaGetLastError());
        tm.end(FQ_K_COMPACT, 3);

        FQ_TRY(cudaMemcpyAsync(g->host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        FQ_TRY(cudaStreamSynchronize(st));
        tm.collect(FQ_K_ENCODE);
        tm.collect(FQ_K_DECODE);
        tm.collect(dir == FQ_TOP_DOWN ? FQ_K_TOP_DOWN : FQ_K_BOTTOM_UP);
        tm.collect(FQ_K_COMPACT);
        if (hc->r_err_q != FQ_OK) return hc->r_err_q;
        if (hc->r_err_v != FQ_OK) return hc->r_err_v;
        if (codec && dir == FQ_TOP_DOWN && hc->dec_n != n_f) return FQ_ECORRUPT;

        const uint64_t examined = dir == FQ_TOP_DOWN ? m_f : hc->r_examined;
        const uint64_t nf_next = hc->n_f_next, mf_next = hc->r_m_f;
        const uint64_t qb = codec ? hc->q_bytes : 0, bb = codec ? hc->b_bytes : 0, vb = want_visited ? hc->v_bytes : 0;

        // algorithmic bytes of this level (design model)
        if (codec) stats.kernel_bytes[FQ_K_ENCODE] += 4 * n_f + qb + (n + 7) / 8 + bb + (want_visited ? (n + 7) / 8 + vb : 0);
        if (dir == FQ_TOP_DOWN) {
            if (codec) stats.kernel_bytes[FQ_K_DECODE] += qb + 4 * n_f;
            stats.kernel_bytes[FQ_K_TOP_DOWN] += 4 * examined + 20 * n_f + 8 * nf_next;
        } else {
            if (codec) stats.kernel_bytes[FQ_K_DECODE] += bb + (n + 7) / 8;
            stats.kernel_bytes[FQ_K_BOTTOM_UP] += 3 * ((n + 7) / 8) + 16 * (n - visited_count) + 4 * examined + 8 * nf_next;
        }
        stats.kernel_bytes[FQ_K_COMPACT] += 3 * ((n + 7) / 8) + 20 * nf_next;

        uint64_t log_off = ~0ull;
        if (d_stream_log && codec) {
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
        n_f = nf_next;
        m_f = mf_next;
        visited_count += n_f;
        m_u -= m_f;
        if ((uint64_t)d + 1 >= n || visited_count > n) return FQ_ECORRUPT;  // at most n levels, n vertices
    }
    FQ_TRY(cudaStreamSynchronize(st));
    stats.reached_edges /= 2;
    if (h_stats) *h_stats = stats;
#undef FQ_TRY
    return result;
}

}  // extern "C"
