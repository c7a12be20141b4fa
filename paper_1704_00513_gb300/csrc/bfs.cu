// bfs.cu -- level-synchronous, direction-optimising BFS with the per-level frontier codec
// stage, and its C ABI (fq_graph_create / fq_graph_destroy / fq_bfs_run).
//
// One level d (the loop of Algorithm 4, on one GPU):
//   1. encode F_d as Q_d (sorted queue, FQ) and B_d (bitmap, FB), and the visited bitmap as
//      V_d -- the compress steps before the thesis' ALLGATHERV/ALLTOALLV; the byte counts are
//      the exchange volume.  When 2|F_d| <= n the set positions of the frontier bitmap are the
//      queue itself, so one encode call writes Q_d and B_d together; V_d's positions are
//      extracted from the visited bitmap (on a parallel branch with the device-driven loop);
//   2. choose the direction from (n_f, m_f, m_u): top-down -> bottom-up when m_f*alpha > m_u,
//      back when n_f*beta < n (direction optimisation, sec. 3.1);
//   3. decode the form that direction consumes (Q_d for top-down, B_d for bottom-up) -- the
//      decompress step;
//   4. expand: top-down over the decoded queue (t = A (x) f masked by the visited list) or
//      bottom-up against the decoded bitmap; depth/parent written by the discovering thread;
//   5. compact the next-frontier bitmap into the sorted queue F_{d+1} (popcount + prefix sum,
//      the popcount-indexed sparse vector of sec. 3.1), visited |= next, count n_f, m_f and
//      the visited bits per tile that V_{d+1}'s extraction starts from.
// The host reads one 256-byte counter record per level (termination test and direction).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "fq_common.cuh"

using namespace fq;

namespace {

constexpr uint32_t kHubDegree = 256;   // top-down: vertices of at least this degree are split
constexpr uint32_t kHubChunk = 2048;   //   into chunks of this many edges, one CTA each
constexpr uint32_t kThreads = 256;
// Compaction tiles: a tile is `sub` sub-tiles of 256 words (16,384 vertices each, one word per
// thread), `sub` chosen per handle so that the tiles fit in one wave of the extract kernel.
constexpr uint32_t kCmpSubWords = kThreads;

struct HubItem {
    uint32_t v;
    uint32_t count;
    unsigned long long start;
};

// Device counters (first 256 bytes of the handle's allocation).  "live" fields are updated
// during a level; the compaction's extract kernel (its first CTA) copies the ones it clears into
// the r_* record the host reads.
struct Counters {
    unsigned long long n_f_next;   // |F_{d+1}|                         (cmp_extract, first CTA)
    unsigned long long m_f_next;   // live: degree sum over F_{d+1}     (expansion kernels)
    unsigned long long examined;   // live: bottom-up adjacency reads
    unsigned long long hub_items;  // live: top-down hub work items
    unsigned long long q_bytes, b_bytes, v_bytes, dec_n;
    unsigned long long r_examined, r_hub_items, vis_count, v_count, r_m_f;
    int32_t r_err_q, r_err_v;
    uint32_t r_where_q, r_where_v;
    unsigned long long r_detail_q, r_detail_v;
    unsigned long long n_iso;      // degree-0 vertices (counted by iso_kernel at handle creation)
    uint32_t pad32a, pad32;
    unsigned long long cols_read;  // live: bottom-up reads of the column array (entries past the head records)
    unsigned long long r_cols_read;
    unsigned long long pad[11];
};
static_assert(sizeof(Counters) == 256, "counter block is 256 bytes");

// State of the device-driven level loop (FQ_BFS_DEVICE_LOOP).  The host writes the parameters
// before each run; loop_init_kernel sets the rest; loop_end_kernel advances it once per level.
struct LoopParams {
    uint32_t root, alpha, beta, flags;
    uint32_t max_levels, min_codec_ids;
    unsigned long long log_cap;
};
struct LoopState {
    LoopParams p;
    unsigned long long n_f, m_f, m_u, visited;  // the level about to run
    unsigned long long log_used;
    uint32_t d, dir;
    int32_t status, soft_status;  // a hard error stops the loop; ENOSPC of the log does not
    uint32_t coded;               // this level runs the codec stage (the frontier reaches the threshold)
    uint32_t root_iso;            // the root has degree 0 (it is visited, and isolated)
    uint32_t small;               // this level's codec stage is the one-CTA form (codec_small)
    uint32_t pad_small;
    fq_bfs_stats stats;
};
constexpr uint32_t kMaxDeviceRecords = 4096;
// Level bodies of the device-driven loop: 2 * encode form + direction (0..5), and the top-down
// level whose small frontier takes the one-CTA codec stage.
constexpr uint32_t kCaseSmall = 6;
constexpr int kCases = 7;

// Top-down visits of the K edges (src[c], w[c]) one thread holds, of which seen[c] marks those whose
// target is already visited (or absent).  For each remaining target the thread whose atomicOr sets
// its bit in the next-frontier bitmap discovers it, writes depth and parent, and adds deg(w) to the
// next level's m_f.  The steps run edge-parallel -- every next-frontier load, then every claim,
// then every discovery's stores and degree loads -- so the K edges' round trips overlap instead of
// following each other.
template <int K>
__device__ __forceinline__ unsigned long long td_visit_batch(const uint32_t (&w)[K], const uint32_t (&src)[K],
                                                             const bool (&seen)[K], uint32_t *next32, int32_t *depth,
                                                             uint32_t *parent, int32_t newdepth,
                                                             const int64_t *__restrict__ off)
{
    uint32_t old[K];
#pragma unroll
    for (int c = 0; c < K; c++) old[c] = seen[c] ? ~0u : next32[w[c] >> 5];  // claimed already this level?
#pragma unroll
    for (int c = 0; c < K; c++) {
        const uint32_t bit = 1u << (w[c] & 31u);
        if (!(old[c] & bit)) old[c] = atomicOr(&next32[w[c] >> 5], bit);
    }
    long long lo[K], hi[K];
#pragma unroll
    for (int c = 0; c < K; c++) {
        lo[c] = hi[c] = 0;
        if (!(old[c] & (1u << (w[c] & 31u)))) {  // this thread's claim set the bit: it discovers w
            depth[w[c]] = newdepth;
            if (parent) parent[w[c]] = src[c];
            lo[c] = off[w[c]];
            hi[c] = off[w[c] + 1];
        }
    }
    unsigned long long degsum = 0;
#pragma unroll
    for (int c = 0; c < K; c++) degsum += (unsigned long long)(hi[c] - lo[c]);
    return degsum;
}

// Level 0: the root, V_0's single position, cleared codec scratch.
__global__ void bfs_init_kernel(const int64_t *off, uint32_t root, uint64_t n, int32_t *depth, uint32_t *parent,
                                uint32_t *q, uint64_t *fbits, uint64_t *visited, uint32_t *vis_cnt, uint64_t tile_bits,
                                uint32_t ntiles, uint32_t *last_set, uint32_t *last_clear, Counters *ctr, Scratch sq,
                                Scratch sv, const LoopState *ls)
{
    if (ls) root = ls->p.root;  // device-driven loop: the root is a run parameter
    // per compaction tile, 1 + its last set / clear vertex of the visited bitmap {root} (0: none)
    for (uint32_t t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint64_t last = min(n, (uint64_t)(t + 1) * tile_bits) - 1;  // the tile's last vertex
        last_set[t] = root / tile_bits == t ? root + 1u : 0u;
        last_clear[t] = last != root ? (uint32_t)(last + 1) : (last > (uint64_t)t * tile_bits ? (uint32_t)last : 0u);
    }
    if (threadIdx.x != 0) return;
    reset_scratch_device(sq);
    reset_scratch_device(sv);
    depth[root] = 0;
    if (parent) parent[root] = root;
    q[0] = root;
    fbits[root >> 6] |= 1ull << (root & 63u);
    visited[root >> 6] |= 1ull << (root & 63u);
    vis_cnt[root / tile_bits] = 1;  // the visited count of the root's compaction tile
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

// Bitmap of the zero-degree vertices (they are never reached, so the sweep treats them as done),
// and their number.
__global__ void iso_kernel(const int64_t *off, uint64_t n, uint32_t *iso32, unsigned long long *count)
{
    const uint64_t nw = (n + 31) / 32;
    unsigned long long c = 0;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0;
        for (uint32_t b = 0; b < 32; b++) {
            const uint64_t v = w * 32 + b;
            if (v < n && off[v + 1] == off[v]) m |= 1u << b;
        }
        iso32[w] = m;
        c += __popc(m);
    }
    c = warp_sum64(c);
    if ((threadIdx.x & 31u) == 0 && c) atomicAdd(count, c);
}

// The design model of one level's algorithmic bytes per kernel class (fq_bfs_level_bytes, which
// documents each term), added into out[].  Shared by both level-loop drivers and the host-side
// entry point, so the bench's roofline numerator can be recomputed from the level records.
struct LevelIn {
    uint64_t n, n_iso, visited, n_f, examined, cols_read, n_f_next, qb, bb, vb;
    uint32_t dir, root_iso;
    bool coded, want_v;
};

__host__ __device__ inline void level_bytes(const LevelIn &x, uint64_t *out)
{
    const uint64_t nbytes = (x.n + 7) / 8;
    if (x.coded) out[FQ_K_ENCODE] += 4 * x.n_f + x.qb + nbytes + x.bb;
    if (x.want_v) out[FQ_K_ENCODE] += nbytes + x.vb;
    if (x.dir == FQ_TOP_DOWN) {
        if (x.coded) out[FQ_K_DECODE] += x.qb + 4 * x.n_f;
        out[FQ_K_TOP_DOWN] += 4 * x.examined + 20 * x.n_f + 8 * x.n_f_next;
    } else {
        if (x.coded) out[FQ_K_DECODE] += x.bb + nbytes;
        // the sweep reads 16 bytes (the offsets pair, or the head record) of every vertex that is
        // neither visited nor isolated, and the column entries its records do not hold; isolated
        // vertices other than an isolated root are never visited
        const uint64_t iso_unvisited = x.n_iso - (x.root_iso && x.n_iso ? 1u : 0u);
        const uint64_t swept = x.n > x.visited + iso_unvisited ? x.n - x.visited - iso_unvisited : 0u;
        out[FQ_K_BOTTOM_UP] += 4 * nbytes + 16 * swept + 4 * x.cols_read + 8 * x.n_f_next;
    }
    out[FQ_K_COMPACT] += 3 * nbytes + 20 * x.n_f_next;
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
                                                             unsigned long long *m_f_next, const LoopState *ls)
{
    if (ls) {  // device-driven loop: the level's size and depth come from the loop state
        nf = ls->n_f;
        newdepth = (int32_t)ls->d + 1;
    }
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long degsum = 0;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // frontier vertices per warp: 32 when the frontier fills the grid, fewer (down to one) when it
    // is small, so that a short frontier with long lists still spreads over every warp
    uint32_t vpw = 32;
    while (vpw > 1 && (uint64_t)(vpw / 2) * nw >= nf) vpw /= 2;
    for (uint64_t base = gw * vpw; base < nf; base += nw * vpw) {
        const uint64_t i = base + lane;
        const bool mine = lane < vpw && i < nf;
        uint32_t v = 0, deg = 0;
        long long s = 0;
        if (mine && q[i] >= n) set_error(err, FQ_ECORRUPT, kWhereBfs, i);  // defensive: ids come from our decoder
        if (mine && q[i] < n) {
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
        constexpr uint32_t kU = 4;  // edge slots per lane per round: their loads are all in flight at once
        for (uint32_t c = 0; c < total; c += 32u * kU) {
            uint32_t src[kU], w[kU];
#pragma unroll
            for (uint32_t r = 0; r < kU; r++) {
                const uint32_t idx = c + 32u * r + lane;
                uint32_t lo = 0;
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1) {
                    const uint32_t cand = lo + step;
                    const uint32_t pc = __shfl_sync(0xffffffffu, p, cand);
                    if (pc <= idx) lo = cand;
                }
                src[r] = __shfl_sync(0xffffffffu, v, lo);
                const long long ss = __shfl_sync(0xffffffffu, s, lo);
                const uint32_t ps = __shfl_sync(0xffffffffu, p, lo);
                w[r] = idx < total ? cols[ss + (idx - ps)] : 0xffffffffu;
            }
            bool seen[kU];
#pragma unroll
            for (uint32_t r = 0; r < kU; r++)
                seen[r] = w[r] == 0xffffffffu || ((visited32[w[r] >> 5] >> (w[r] & 31u)) & 1u);
            degsum += td_visit_batch<kU>(w, src, seen, next32, depth, parent, newdepth, off);
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
                                                          const int64_t *__restrict__ off, unsigned long long *m_f_next,
                                                          const LoopState *ls)
{
    if (ls) newdepth = (int32_t)ls->d + 1;
    const unsigned long long total = min(*nitems, items_cap);
    unsigned long long degsum = 0;
    constexpr uint32_t kPer = kHubChunk / kThreads;  // entries per thread per item
    for (unsigned long long it = blockIdx.x; it < total; it += gridDim.x) {
        const HubItem h = items[it];
        uint32_t w[kPer];
#pragma unroll
        for (uint32_t c = 0; c < kPer; c++) {  // the item's columns first, all loads in flight ...
            const uint32_t j = threadIdx.x + c * kThreads;
            w[c] = j < h.count ? cols[h.start + j] : 0xffffffffu;
        }
        bool seen[kPer];
        uint32_t src[kPer];
#pragma unroll
        for (uint32_t c = 0; c < kPer; c++) {  // ... then their visited bits ...
            seen[c] = w[c] == 0xffffffffu || ((visited32[w[c] >> 5] >> (w[c] & 31u)) & 1u);
            src[c] = h.v;
        }
        degsum += td_visit_batch<(int)kPer>(w, src, seen, next32, depth, parent, newdepth, off);  // ... then the claims
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
                                                            unsigned long long *examined, unsigned long long *m_f_next,
                                                            unsigned long long *cols_read, const LoopState *ls)
{
    if (ls) newdepth = (int32_t)ls->d + 1;
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
    if (lane == 0 && cnt) {
        atomicAdd(examined, cnt);
        atomicAdd(cols_read, cnt);  // every entry this sweep examines comes from cols
    }
    if (lane == 0 && degsum) atomicAdd(m_f_next, degsum);
}

// Head records of the bottom-up sweep (graphs with fewer than 2^32 adjacency entries): per vertex
// its adjacency start, its degree and its first two neighbours (UINT32_MAX where absent), so that a
// vertex whose parent is among its first two neighbours is settled from one coalesced 16-byte load,
// without the dependent random read of its adjacency list.
__global__ void head_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ cols, uint64_t n,
                            uint4 *__restrict__ hc)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const long long s = off[v], d = off[v + 1] - s;
        hc[v] = make_uint4((uint32_t)s, (uint32_t)d, d > 0 ? cols[s] : 0xffffffffu, d > 1 ? cols[s + 1] : 0xffffffffu);
    }
}

// The bottom-up sweep of bu_sweep_kernel over head records: the first two neighbours come with the
// record (their frontier bits are tested together), the rest of the list is scanned as there.  A
// warp takes 32 words (1,024 vertices) at a time: one coalesced load of their done masks (visited |
// isolated), a ballot of the words that still hold unvisited vertices, and only those words are
// swept -- late levels, where almost every word is done, cost one load per 32 words instead of a
// dependent load per word.
__global__ void __launch_bounds__(kThreads) bu_sweep_head_kernel(const uint32_t *__restrict__ front32,
                                                                 const uint32_t *__restrict__ visited32,
                                                                 const uint32_t *__restrict__ iso32,
                                                                 uint32_t *__restrict__ next32,
                                                                 const uint4 *__restrict__ hc,
                                                                 const uint32_t *__restrict__ cols, int32_t *depth,
                                                                 uint32_t *parent, int32_t newdepth, uint64_t n,
                                                                 unsigned long long *examined,
                                                                 unsigned long long *m_f_next,
                                                                 unsigned long long *cols_read, const LoopState *ls)
{
    if (ls) newdepth = (int32_t)ls->d + 1;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nwords = (n + 31) / 32;
    unsigned long long cnt = 0, degsum = 0, tail = 0;
    for (uint64_t chunk = gw; chunk * 32u < nwords; chunk += nw) {
        const uint64_t my_word = chunk * 32u + lane;
        const uint32_t my_done = my_word < nwords ? (visited32[my_word] | iso32[my_word]) : 0xffffffffu;
        uint32_t pending = __ballot_sync(0xffffffffu, my_done != 0xffffffffu);
        while (pending) {
            const uint32_t src = (uint32_t)__ffs(pending) - 1u;
            pending &= pending - 1u;
            const uint32_t done = __shfl_sync(0xffffffffu, my_done, src);
            const uint64_t word = chunk * 32u + src;
            const uint64_t w = word * 32u + lane;
            bool found = false;
            uint32_t par = 0;
            if (w < n && !((done >> lane) & 1u)) {
                const uint4 h = hc[w];
                const uint32_t deg = h.y;
                const bool h0 = deg > 0 && ((front32[h.z >> 5] >> (h.z & 31u)) & 1u);
                const bool h1 = deg > 1 && ((front32[h.w >> 5] >> (h.w & 31u)) & 1u);
                uint32_t j;  // entries examined
                if (h0 || h1) {
                    found = true;
                    par = h0 ? h.z : h.w;
                    j = h0 ? 1u : 2u;
                } else {
                    j = min(deg, 2u);
                    const uint32_t *row = cols + h.x;
                    for (; j + 1 < deg; j += 2) {
                        const uint32_t u0 = row[j], u1 = row[j + 1];
                        const bool f0 = (front32[u0 >> 5] >> (u0 & 31u)) & 1u;
                        const bool f1 = (front32[u1 >> 5] >> (u1 & 31u)) & 1u;
                        if (f0 || f1) {
                            found = true;
                            par = f0 ? u0 : u1;
                            j += f0 ? 1u : 2u;
                            break;
                        }
                    }
                    if (!found && j < deg) {
                        const uint32_t u0 = row[j];
                        j += 1;
                        if ((front32[u0 >> 5] >> (u0 & 31u)) & 1u) {
                            found = true;
                            par = u0;
                        }
                    }
                }
                cnt += j;
                tail += j - min(j, min(deg, 2u));  // entries past the record's two came from cols
                if (found) degsum += deg;
            }
            if (found) {
                depth[w] = newdepth;
                if (parent) parent[w] = par;
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, found);
            if (lane == 0 && mask) next32[word] = mask;
        }
    }
    cnt = warp_sum64(cnt);
    degsum = warp_sum64(degsum);
    tail = warp_sum64(tail);
    if (lane == 0 && cnt) atomicAdd(examined, cnt);
    if (lane == 0 && degsum) atomicAdd(m_f_next, degsum);
    if (lane == 0 && tail) atomicAdd(cols_read, tail);
}

// ---- compaction: next bitmap -> sorted queue, n_f, m_f, visited |= next, V positions ----
// Two launches per level and no one-CTA step: the count kernel writes each tile's counts, and
// every CTA of the extract kernel sums the counts of the tiles before its own (a few hundred
// words from L2) for its output offsets and the level's totals.

// Per tile: the next frontier's count, visited |= next, and (when V_{d+1} is coded) the tile's
// visited count after the update.  Every sub-tile's loads are issued before any is used.
__global__ void __launch_bounds__(kThreads) cmp_count_kernel(const uint64_t *__restrict__ next, uint64_t *visited,
                                                             uint64_t nwords, uint64_t n, uint32_t sub,
                                                             uint32_t *tile_cnt, uint32_t *vis_cnt, uint32_t *last_set,
                                                             uint32_t *last_clear, int want_v)
{
    __shared__ uint32_t ws[kThreads / 32], wv[kThreads / 32], wls[kThreads / 32], wlc[kThreads / 32];
    constexpr uint32_t kAhead = 4;  // sub-tiles whose words are in flight together
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t w0 = (uint64_t)blockIdx.x * sub * kCmpSubWords + threadIdx.x;
    uint32_t cnt = 0, vc = 0;
    uint32_t ls = 0, lc = 0;  // 1 + the last set / clear vertex of the updated visited bitmap (0: none)
    for (uint32_t s0 = 0; s0 < sub; s0 += kAhead) {
        uint64_t x[kAhead], v[kAhead];
#pragma unroll
        for (uint32_t j = 0; j < kAhead; j++) {
            const uint64_t w = w0 + (uint64_t)(s0 + j) * kCmpSubWords;
            const bool in = s0 + j < sub && w < nwords;
            x[j] = in ? next[w] : 0ull;
            v[j] = (in && want_v) ? visited[w] : 0ull;
        }
#pragma unroll
        for (uint32_t j = 0; j < kAhead; j++) {
            const uint64_t w = w0 + (uint64_t)(s0 + j) * kCmpSubWords;
            if (x[j]) {
                if (want_v) visited[w] = v[j] | x[j];
                else visited[w] |= x[j];
            }
            cnt += (uint32_t)__popcll(x[j]);
            const uint64_t nv = v[j] | x[j];
            vc += (uint32_t)__popcll(nv);  // the next frontier is disjoint from the visited set
            if (want_v && s0 + j < sub && w < nwords) {
                const uint32_t tail = (uint32_t)(n & 63u);
                const uint64_t in_n = (w == nwords - 1 && tail) ? (1ull << tail) - 1ull : ~0ull;
                const uint64_t clr = ~nv & in_n;
                if (nv) ls = max(ls, (uint32_t)(w * 64u + 64u - (uint32_t)__clzll((long long)nv)));
                if (clr) lc = max(lc, (uint32_t)(w * 64u + 64u - (uint32_t)__clzll((long long)clr)));
            }
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    vc = __reduce_add_sync(0xffffffffu, vc);
    ls = __reduce_max_sync(0xffffffffu, ls);
    lc = __reduce_max_sync(0xffffffffu, lc);
    if (lane == 0) {
        ws[warp] = cnt;
        wv[warp] = vc;
        wls[warp] = ls;
        wlc[warp] = lc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0, tv = 0, tls = 0, tlc = 0;
        for (uint32_t i = 0; i < kThreads / 32; i++) {
            t += ws[i];
            tv += wv[i];
            tls = max(tls, wls[i]);
            tlc = max(tlc, wlc[i]);
        }
        tile_cnt[blockIdx.x] = t;
        vis_cnt[blockIdx.x] = tv;
        if (want_v) {
            last_set[blockIdx.x] = tls;
            last_clear[blockIdx.x] = tlc;
        }
    }
}

// The level record and cleared codec scratch (first thread of the extract kernel's first CTA):
// the level's live counters and codec status are snapshot into the r_* fields and cleared for the
// next level, and V_{d+1}'s control block gets its count and mode.  Every load comes first: the
// stores could alias them, and this thread's round trips are on the kernel's critical path.
__device__ __forceinline__ void cmp_snapshot(Counters *ctr, const Scratch &sq, const Scratch &sv,
                                             unsigned long long nf, unsigned long long vis,
                                             unsigned long long vcount, bool set_mode)
{
    const unsigned long long m_f = ctr->m_f_next, ex = ctr->examined, hub = ctr->hub_items, cr = ctr->cols_read;
    const int32_t cq = sq.ctl->code, cv = sv.ctl->code;
    const uint32_t wq = sq.ctl->where, wv = sv.ctl->where;
    const unsigned long long dq = sq.ctl->detail, dv = sv.ctl->detail;
    ctr->n_f_next = nf;
    ctr->r_m_f = m_f;  // summed by the expansion kernels
    ctr->m_f_next = 0;
    ctr->vis_count = vis;
    ctr->v_count = vcount;
    ctr->r_examined = ex;
    ctr->examined = 0;
    ctr->r_cols_read = cr;
    ctr->cols_read = 0;
    ctr->r_hub_items = hub;
    ctr->hub_items = 0;
    ctr->r_err_q = cq;
    ctr->r_where_q = wq;
    ctr->r_detail_q = dq;
    ctr->r_err_v = cv;
    ctr->r_where_v = wv;
    ctr->r_detail_v = dv;
    reset_scratch_device(sq);
    reset_scratch_device(sv);
    sv.ctl->n = vcount;
    sv.ctl->fb_mode = set_mode ? kFbSet : kFbClear;
}

// Positions of the set bits of the warp's 32 words (lane L holds word wbase + L) written to
// out[pos ...] in increasing order: each lane writes its word's positions into the warp's
// shared-memory stage at its prefix offset, then the warp copies the stage out with coalesced
// stores (2,048 positions at most: 32 words x 64 bits).
__device__ __forceinline__ void extract_words(uint64_t x, uint64_t wbase, unsigned long long pos, uint32_t *out,
                                              uint32_t lane, uint32_t *stage)
{
    const uint32_t c = (uint32_t)__popcll(x);
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    uint32_t o = incl - c;
    const uint32_t p0 = (uint32_t)((wbase + lane) * 64u);
    while (x) {
        stage[o++] = p0 + (uint32_t)(__ffsll((long long)x) - 1);
        x &= x - 1ull;
    }
    __syncwarp();
    for (uint32_t i = lane; i < total; i += 32u) out[pos + i] = stage[i];
    __syncwarp();
}

constexpr size_t kCmpStage = 2048 * sizeof(uint32_t);               // one warp's stage
constexpr size_t kCmpSmem = (kThreads / 32) * kCmpStage;            // 64 KB per CTA

// Sums over the compaction tiles' counts, by every CTA: the counts of the tiles before its own
// (its output offset) and of all tiles.  cnt2 may be null (its sums are then 0).
struct TileSums {
    unsigned long long before, total, before2, total2;
};

__device__ __forceinline__ TileSums cta_tile_sums(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ cnt2,
                                                  uint32_t ntiles, unsigned long long (*red)[kThreads / 32])
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long b = 0, t = 0, b2 = 0, t2 = 0;
    for (uint32_t i = threadIdx.x; i < ntiles; i += kThreads) {
        const uint32_t c = cnt[i], c2 = cnt2 ? cnt2[i] : 0u;
        t += c;
        t2 += c2;
        if (i < blockIdx.x) {
            b += c;
            b2 += c2;
        }
    }
    b = warp_sum64(b);
    t = warp_sum64(t);
    b2 = warp_sum64(b2);
    t2 = warp_sum64(t2);
    if (lane == 0) {
        red[0][warp] = b;
        red[1][warp] = t;
        red[2][warp] = b2;
        red[3][warp] = t2;
    }
    __syncthreads();
    TileSums r{0, 0, 0, 0};
    for (uint32_t i = 0; i < kThreads / 32; i++) {
        r.before += red[0][i];
        r.total += red[1][i];
        r.before2 += red[2][i];
        r.total2 += red[3][i];
    }
    return r;
}

// Sub-tiles of a compaction tile whose words one thread holds at once (their loads in flight
// together); tiles of more sub-tiles are taken in rounds of this many.
constexpr uint32_t kCmpAhead = 4;

// The positions of a tile's sub-tiles [s0, s0 + kCmpAhead) from the words x[] the threads hold
// (thread i: word i of each sub-tile), written from out[o] on in increasing order; o advances by
// the count.  Within a sub-tile each warp's offset is a prefix of warp counts.
__device__ __forceinline__ void cmp_extract_round(const uint64_t (&x)[kCmpAhead], uint64_t tile_w0, uint32_t s0,
                                                  uint32_t sub, unsigned long long &o, uint32_t *out, uint32_t *stage,
                                                  uint32_t *wc)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (uint32_t j = 0; j < kCmpAhead; j++) {
        if (s0 + j >= sub) break;  // uniform over the CTA
        const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popcll(x[j]));
        if (lane == 0) wc[warp] = c;
        __syncthreads();
        unsigned long long p = o;
        for (uint32_t i = 0; i < kThreads / 32; i++) {
            if (i < warp) p += wc[i];
            o += wc[i];
        }
        extract_words(x[j], tile_w0 + (uint64_t)(s0 + j) * kCmpSubWords + warp * 32u, p, out, lane, stage);
        __syncthreads();  // the warp counts are rewritten by the next sub-tile
    }
}

// The next frontier F_{d+1} as a sorted queue (and as the bitmap the next level's B encode reads),
// next cleared, and the level record (first CTA).  Each CTA's offset and the level's totals come
// from the tile counts (cta_tile_sums); the visited counts give V_{d+1}'s size and mode.
__global__ void __launch_bounds__(kThreads) cmp_extract_kernel(uint64_t *__restrict__ next, uint64_t *__restrict__ fbits,
                                                               uint64_t nwords, uint64_t n, uint32_t sub, uint32_t ntiles,
                                                               const uint32_t *__restrict__ tile_cnt,
                                                               const uint32_t *__restrict__ vis_cnt, uint32_t *q,
                                                               Counters *ctr, Scratch sq, Scratch sv, int want_v)
{
    extern __shared__ __align__(16) uint32_t cstage[];  // [warps][2048]
    __shared__ uint32_t wc[kThreads / 32];
    __shared__ unsigned long long red[4][kThreads / 32];
    const uint64_t tile_w0 = (uint64_t)blockIdx.x * sub * kCmpSubWords;
    uint64_t x[kCmpAhead];
#pragma unroll
    for (uint32_t j = 0; j < kCmpAhead; j++) {  // the first round's words, in flight with the sums
        const uint64_t w = tile_w0 + (uint64_t)j * kCmpSubWords + threadIdx.x;
        x[j] = (j < sub && w < nwords) ? next[w] : 0ull;
    }
    const TileSums ts = cta_tile_sums(tile_cnt, want_v ? vis_cnt : nullptr, ntiles, red);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const bool set_mode = 2ull * ts.total2 <= n;
        cmp_snapshot(ctr, sq, sv, ts.total, ts.total2, set_mode ? ts.total2 : (unsigned long long)n - ts.total2,
                     set_mode);
    }
    uint32_t *stage = cstage + (threadIdx.x >> 5) * 2048u;
    unsigned long long o = ts.before;
    for (uint32_t s0 = 0; s0 < sub; s0 += kCmpAhead) {
        if (s0) {
#pragma unroll
            for (uint32_t j = 0; j < kCmpAhead; j++) {
                const uint64_t w = tile_w0 + (uint64_t)(s0 + j) * kCmpSubWords + threadIdx.x;
                x[j] = (s0 + j < sub && w < nwords) ? next[w] : 0ull;
            }
        }
#pragma unroll
        for (uint32_t j = 0; j < kCmpAhead; j++) {
            const uint64_t w = tile_w0 + (uint64_t)(s0 + j) * kCmpSubWords + threadIdx.x;
            if (s0 + j < sub && w < nwords) {
                fbits[w] = x[j];  // F_{d+1} as a bitmap for the next level's B encode
                if (x[j]) next[w] = 0;
            }
        }
        cmp_extract_round(x, tile_w0, s0, sub, o, q, stage, wc);
    }
}

// V_d's positions (step 1 of a level, before V_d's encode): the set bits of the visited bitmap when
// at most half are set, else the clear ones (bits past n excluded), from the per-tile visited
// counts the last compaction wrote (level 0: the root's tile holds 1).  The visited bitmap does not
// change until the level's compaction, so this runs beside the level's other work.
__global__ void __launch_bounds__(kThreads) v_extract_kernel(const uint64_t *__restrict__ visited, uint64_t nwords,
                                                             uint64_t n, uint32_t sub, uint32_t ntiles,
                                                             const uint32_t *__restrict__ vis_cnt, Scratch sv)
{
    extern __shared__ __align__(16) uint32_t cstage[];  // [warps][2048]
    __shared__ uint32_t wc[kThreads / 32];
    __shared__ unsigned long long red[4][kThreads / 32];
    if (sv.ctl->skip_pos) return;  // V_d is coded as raw words (fbw_kernel decided it from the bitmap)
    const uint64_t tile_w0 = (uint64_t)blockIdx.x * sub * kCmpSubWords;
    const uint32_t tail = (uint32_t)(n & 63u);
    uint64_t y[kCmpAhead];
#pragma unroll
    for (uint32_t j = 0; j < kCmpAhead; j++) {
        const uint64_t w = tile_w0 + (uint64_t)j * kCmpSubWords + threadIdx.x;
        y[j] = (j < sub && w < nwords) ? visited[w] : 0ull;
    }
    const TileSums ts = cta_tile_sums(vis_cnt, nullptr, ntiles, red);
    const bool set_mode = 2ull * ts.total <= n;
    // clear mode: the clear bits before this tile are its bits before it minus the set ones
    unsigned long long o = set_mode ? ts.before : min((unsigned long long)n, 64ull * tile_w0) - ts.before;
    uint32_t *stage = cstage + (threadIdx.x >> 5) * 2048u;
    for (uint32_t s0 = 0; s0 < sub; s0 += kCmpAhead) {
#pragma unroll
        for (uint32_t j = 0; j < kCmpAhead; j++) {
            const uint64_t w = tile_w0 + (uint64_t)(s0 + j) * kCmpSubWords + threadIdx.x;
            const bool in = s0 + j < sub && w < nwords;
            if (s0) y[j] = in ? visited[w] : 0ull;
            if (in && !set_mode) {
                const uint64_t nb = (w == nwords - 1 && tail) ? tail : 64u;
                y[j] = ~y[j] & (nb == 64 ? ~0ull : ((1ull << nb) - 1ull));
            }
        }
        cmp_extract_round(y, tile_w0, s0, sub, o, sv.positions, stage, wc);
    }
}

// ---- V_d's block widths from the visited bitmap ----
// V_d codes the positions of the members -- the set bits of the visited bitmap when at most half
// are set, else its clear bits below n -- as blocks of 128 positions (sec. 5.1), whose width b is
// the bit length of the largest gap (p - p_prev - 1) inside the block; the container is the raw
// bitmap unless the coded positions are strictly smaller.  Once the visited set is dense, raw is
// the usual outcome, and the stream's size -- so the decision -- needs only the sum of the
// widths, which this kernel takes from the bitmap without writing any position: member
// ranks come from the per-tile counts, each member's predecessor from the per-tile last members,
// and the gaps inside a word from zero-run tests on its bits.  When the sum says raw, the positions
// extraction and the widths pass are skipped (Ctl::skip_pos) and the pack kernel copies the words.

// Position of the j-th (0-based) set bit of x (j < popcount(x)).
__device__ __forceinline__ uint32_t select64(uint64_t x, uint32_t j)
{
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t s = 32; s >= 1; s >>= 1) {
        const uint32_t c = (uint32_t)__popcll(x & ((1ull << s) - 1ull));
        if (j >= c) {
            j -= c;
            x >>= s;
            pos += s;
        }
    }
    return pos;
}

// Bit length of the largest gap between consecutive set bits of y at or between bit lo and bit hi
// (both set): the longest zero run strictly inside (lo, hi), found by doubling -- r_L marks the bits
// that start L zeros -- so the answer is the number of L in 1, 2, 4, .., 32 with a run of L zeros.
__device__ __forceinline__ uint32_t inner_gap_bits(uint64_t y, uint32_t lo, uint32_t hi)
{
    if (hi <= lo + 1u) return 0u;
    const uint64_t between = ((1ull << hi) - 1ull) & ~((2ull << lo) - 1ull);
    uint64_t r = ~y & between;
    uint32_t b = 0;
#pragma unroll
    for (uint32_t L = 1; L <= 32; L <<= 1) {
        if (!r) break;
        b++;
        r &= r >> L;
    }
    return b;
}

// One CTA per sub-tile of 256 words, one word per thread.  The members before the sub-tile, and
// the last of them, come from the per-tile counts and last members of the tiles before its own and
// from the earlier sub-tiles of its tile (whose words it reads).  Each word's members and their
// block segments (at most two: a block start falls in a word at most once) give each segment's
// largest-gap bit length, combined per block in shared memory; the blocks that start and end in the
// sub-tile add their widths to the sub-tile's sum (wpart[]), the others go through wb[] (atomicMax;
// the sub-tile holding a block's first member names it in span[]).  The last CTA to finish adds the
// sums and the named blocks' widths (clearing wb[] for the next call) and takes the container's
// decision.  No counter is shared by all CTAs but the finishing ticket.  Sparse member sets (below
// n/16) are left to the positions path: there the positions are few and a scan of every word would
// cost more.
constexpr uint32_t kSubBlocks = 64u * kCmpSubWords / kBlock + 2u;  // blocks one sub-tile's members touch

__device__ __forceinline__ uint64_t member_word(const uint64_t *__restrict__ visited, uint64_t w, uint64_t nwords,
                                                uint32_t tail, bool set_mode)
{
    if (w >= nwords) return 0ull;
    const uint64_t y = visited[w];
    return set_mode ? y : ~y & ((w == nwords - 1 && tail) ? (1ull << tail) - 1ull : ~0ull);
}

__global__ void __launch_bounds__(kThreads, 6) fbw_kernel(const uint64_t *__restrict__ visited, uint64_t nwords, uint64_t n,
                                                          uint32_t sub, uint32_t ntiles,
                                                          const uint32_t *__restrict__ vis_cnt,
                                                          const uint32_t *__restrict__ last_set,
                                                          const uint32_t *__restrict__ last_clear, uint32_t *wb,
                                                          uint32_t *span, uint32_t *wpart, Scratch sv)
{
    // Counts and positions fit 32 bits (n < 2^32); a position p is carried as p + 1, 0 for none.
    __shared__ uint32_t red[8][kThreads / 32];
    __shared__ uint32_t wcnt[kThreads / 32], wlast[kThreads / 32];
    __shared__ uint32_t smax[kSubBlocks];
    __shared__ bool s_last;
    {  // a sparse member set (its count and mode were set by the last compaction) is left to the
       // positions path before anything else is read
        const unsigned long long m0 = sv.ctl->n;
        if (m0 == 0 || 16ull * m0 < n) return;
    }
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t tile = blockIdx.x / sub, s = blockIdx.x % sub;
    const uint32_t tail = (uint32_t)(n & 63u);
    const uint64_t tile_w0 = (uint64_t)tile * sub * kCmpSubWords;
    const uint64_t w = tile_w0 + (uint64_t)s * kCmpSubWords + threadIdx.x;
    const uint64_t in_n_last = tail ? (1ull << tail) - 1ull : ~0ull;  // the last word's bits below n
    // every load of the prologue first: this word, the tile's earlier sub-tiles' words (both modes'
    // members are counted, the mode is known only after the sums), the earlier tiles' records
    const uint64_t y_raw = w < nwords ? visited[w] : 0ull;
    uint64_t ye[kCmpAhead];
#pragma unroll
    for (uint32_t e = 0; e < kCmpAhead; e++) {
        const uint64_t we = tile_w0 + (uint64_t)e * kCmpSubWords + threadIdx.x;
        ye[e] = (e < s && we < nwords) ? visited[we] : 0ull;
    }
    for (uint32_t i = threadIdx.x; i < kSubBlocks; i += kThreads) smax[i] = 0u;
    uint32_t vb = 0, vt = 0, ls = 0, lc = 0;  // visited before / in all tiles, last set / clear + 1 before the tile
    for (uint32_t i = threadIdx.x; i < ntiles; i += kThreads) {
        const uint32_t c = vis_cnt[i];
        vt += c;
        if (i < tile) {
            vb += c;
            ls = max(ls, last_set[i]);
            lc = max(lc, last_clear[i]);
        }
    }
    uint32_t es = 0, ec = 0, els = 0, elc = 0;  // the earlier sub-tiles: set, clear, last set + 1, last clear + 1
    auto earlier = [&](uint32_t e, uint64_t y1) {
        const uint64_t we = tile_w0 + (uint64_t)e * kCmpSubWords + threadIdx.x;
        if (e >= s || we >= nwords) return;
        const uint64_t y0 = ~y1 & (we == nwords - 1 ? in_n_last : ~0ull);
        es += (uint32_t)__popcll(y1);
        ec += (uint32_t)__popcll(y0);
        if (y1) els = max(els, (uint32_t)(we * 64u + 64u - (uint32_t)__clzll((long long)y1)));
        if (y0) elc = max(elc, (uint32_t)(we * 64u + 64u - (uint32_t)__clzll((long long)y0)));
    };
#pragma unroll
    for (uint32_t e = 0; e < kCmpAhead; e++) earlier(e, ye[e]);
    for (uint32_t e = kCmpAhead; e < s; e++) {  // tiles of more sub-tiles (graphs above 29.9M vertices)
        const uint64_t we = tile_w0 + (uint64_t)e * kCmpSubWords + threadIdx.x;
        earlier(e, we < nwords ? visited[we] : 0ull);
    }
    vb = __reduce_add_sync(0xffffffffu, vb);
    vt = __reduce_add_sync(0xffffffffu, vt);
    ls = __reduce_max_sync(0xffffffffu, ls);
    lc = __reduce_max_sync(0xffffffffu, lc);
    es = __reduce_add_sync(0xffffffffu, es);
    ec = __reduce_add_sync(0xffffffffu, ec);
    els = __reduce_max_sync(0xffffffffu, els);
    elc = __reduce_max_sync(0xffffffffu, elc);
    if (lane == 0) {
        red[0][warp] = vb;
        red[1][warp] = vt;
        red[2][warp] = ls;
        red[3][warp] = lc;
        red[4][warp] = es;
        red[5][warp] = ec;
        red[6][warp] = els;
        red[7][warp] = elc;
    }
    __syncthreads();
    vb = vt = ls = lc = es = ec = els = elc = 0;
    for (uint32_t i = 0; i < kThreads / 32; i++) {
        vb += red[0][i];
        vt += red[1][i];
        ls = max(ls, red[2][i]);
        lc = max(lc, red[3][i]);
        es += red[4][i];
        ec += red[5][i];
        els = max(els, red[6][i]);
        elc = max(elc, red[7][i]);
    }
    const bool set_mode = 2ull * vt <= n;
    const uint32_t members = set_mode ? vt : (uint32_t)(n - vt);
    if (members == 0 || 16ull * members < n) return;  // (as tested on entry; the same in every CTA)
    // members before this sub-tile, and the last of them + 1 (0: none)
    const uint32_t R = set_mode ? vb + es : (uint32_t)min((unsigned long long)n, 64ull * tile_w0) - vb + ec;
    const uint32_t P1 = set_mode ? max(ls, els) : max(lc, elc);
    const uint64_t y = (w < nwords && !set_mode) ? ~y_raw & (w == nwords - 1 ? in_n_last : ~0ull) : y_raw;
    const uint32_t c = (uint32_t)__popcll(y);
    const uint32_t last1 = c ? (uint32_t)(w * 64u + 64u - (uint32_t)__clzll((long long)y)) : 0u;
    // count and last member + 1 over this sub-tile's words up to this one (inclusive)
    uint32_t incl = c, lmax = last1;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t yc = __shfl_up_sync(0xffffffffu, incl, o);
        const uint32_t yl = __shfl_up_sync(0xffffffffu, lmax, o);
        if (lane >= o) {
            incl += yc;
            lmax = max(lmax, yl);
        }
    }
    if (lane == 31) {
        wcnt[warp] = incl;
        wlast[warp] = lmax;
    }
    __syncthreads();
    uint32_t Rw = R + incl - c;  // members before this word
    uint32_t Pw1 = P1;           // the last of them + 1
    const uint32_t lprev = __shfl_up_sync(0xffffffffu, lmax, 1);
    if (lane > 0) Pw1 = max(Pw1, lprev);
    uint32_t tot = 0;
    for (uint32_t i = 0; i < kThreads / 32; i++) {
        if (i < warp) {
            Rw += wcnt[i];
            Pw1 = max(Pw1, wlast[i]);
        }
        tot += wcnt[i];
    }
    const uint32_t kfirst = R / kBlock;  // the first block this sub-tile's members touch
    if (c) {
        const uint32_t lo = (uint32_t)__ffsll((long long)y) - 1u;
        const uint32_t hi = 63u - (uint32_t)__clzll((long long)y);
        const uint32_t j0 = (kBlock - Rw % kBlock) % kBlock;  // in-word index of a block start
        const uint32_t loB = j0 < c ? select64(y, j0) : 64u;
        if (j0 > 0) {  // members [0, min(j0, c)) close block Rw / 128; member 0's gap is inside it
            const uint32_t hiA = j0 >= c ? hi : 63u - (uint32_t)__clzll((long long)(y & ((1ull << loB) - 1ull)));
            uint32_t v = inner_gap_bits(y, lo, hiA);
            const uint32_t g = (uint32_t)(w * 64u + lo) - Pw1;  // Rw > 0, so Pw1 >= 1: the gap p - p_prev - 1
            v = max(v, g ? 32u - (uint32_t)__clz(g) : 0u);
            if (v) atomicMax(&smax[Rw / kBlock - kfirst], v);
        }
        if (j0 < c) {  // members [j0, c) open block (Rw + j0) / 128; member j0's gap is outside it
            const uint32_t v = inner_gap_bits(y, loB, hi);
            if (v) atomicMax(&smax[(Rw + j0) / kBlock - kfirst], v);
        }
    }
    if (threadIdx.x == 0) span[blockIdx.x] = 0xffffffffu;
    __syncthreads();
    uint32_t local = 0;  // widths of the blocks that start and end in this sub-tile
    if (tot) {
        const uint32_t end = R + tot;  // members before the next sub-tile
        const uint32_t nloc = (end - 1) / kBlock - kfirst + 1;
        for (uint32_t j = threadIdx.x; j < nloc; j += kThreads) {
            const uint32_t k = kfirst + j;
            const bool owned = (uint64_t)k * kBlock >= R;  // its first member is in this sub-tile
            const bool complete = min((uint64_t)k * kBlock + kBlock, (uint64_t)members) <= end;
            if (owned && complete) {
                local += smax[j];
            } else {
                if (smax[j]) atomicMax(&wb[k], smax[j]);
                if (owned) span[blockIdx.x] = k;  // at most one: the sub-tile's last block
            }
        }
    }
    local = __reduce_add_sync(0xffffffffu, local);
    if (lane == 0) wcnt[warp] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t i = 0; i < kThreads / 32; i++) t += wcnt[i];
        wpart[blockIdx.x] = t;
    }
    // the last CTA: the sub-tiles' sums and the listed blocks' widths, the container's decision,
    // wb[] cleared
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&sv.ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long sum = 0;
    constexpr uint32_t kPer = 8;  // entries per thread whose loads are in flight together
    for (uint32_t i0 = 0; i0 < gridDim.x; i0 += kThreads * kPer) {
        uint32_t kk[kPer], wv[kPer];
#pragma unroll
        for (uint32_t j = 0; j < kPer; j++) {
            const uint32_t i = i0 + j * kThreads + threadIdx.x;
            kk[j] = i < gridDim.x ? __ldcg(span + i) : 0xffffffffu;
            sum += i < gridDim.x ? __ldcg(wpart + i) : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < kPer; j++) wv[j] = kk[j] != 0xffffffffu ? __ldcg(wb + kk[j]) : 0u;
#pragma unroll
        for (uint32_t j = 0; j < kPer; j++) {
            if (kk[j] != 0xffffffffu) {
                sum += wv[j];
                wb[kk[j]] = 0u;
            }
        }
    }
    sum = warp_sum64(sum);
    __syncthreads();
    if (lane == 0) red[0][warp] = (uint32_t)sum;  // at most 32 per block and under 2^25 blocks
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long total = 0;
        for (uint32_t i = 0; i < kThreads / 32; i++) total += red[0][i];
        // the FB container's rule: raw words unless the header plus the FQ stream (packed, or raw ids
        // when packing does not pay) is smaller
        const unsigned long long nb = ((unsigned long long)members + kBlock - 1) / kBlock;
        const unsigned long long packed = 16ull + (5ull * nb + 15ull) / 16ull * 16ull + 16ull * total;
        const unsigned long long rawq = 16ull + (4ull * members + 15ull) / 16ull * 16ull;
        const unsigned long long fq = packed < rawq ? packed : rawq;
        const unsigned long long fbr = 16ull + (8ull * ((n + 63) / 64) + 15ull) / 16ull * 16ull;
        if (16ull + fq >= fbr) {
            sv.ctl->total_b = total;
            sv.ctl->skip_pos = 1u;
        }
        sv.ctl->ticket = 0u;
    }
}

// ---- round-trip check of the overlapped codec stage (FQ_BFS_OVERLAP) ----
// With the overlap the expansion consumes the raw frontier, so the decoded form is not consumed;
// these kernels verify it instead: the decoded queue must equal the raw queue (and hold n_f ids),
// the decoded bitmap the raw bitmap.  A difference is reported as FQ_ECORRUPT in the codec status
// (detail: the first differing index), which the compaction's snapshot hands to the loop.

__global__ void rt_check_queue_kernel(const uint32_t *__restrict__ q, const uint32_t *__restrict__ q2, uint64_t nf,
                                      const unsigned long long *dec_n, Ctl *err, const LoopState *ls)
{
    if (ls) nf = ls->n_f;
    const unsigned long long got = *dec_n;
    if (got != nf) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_error(err, FQ_ECORRUPT, kWhereBfs, got < nf ? got : nf);
        return;
    }
    const uint64_t nv = nf / 4;  // both queues start 256-byte aligned: 128-bit compares, then the tail
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        const uint4 a = reinterpret_cast<const uint4 *>(q)[i], b = reinterpret_cast<const uint4 *>(q2)[i];
        if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w) set_error(err, FQ_ECORRUPT, kWhereBfs, 4 * i);
    }
    const uint64_t t = 4 * nv + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf && q[t] != q2[t]) set_error(err, FQ_ECORRUPT, kWhereBfs, t);
}

__global__ void rt_check_bitmap_kernel(const uint64_t *__restrict__ a, const uint64_t *__restrict__ b, uint64_t nwords,
                                       Ctl *err)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += stride)
        if (a[i] != b[i]) set_error(err, FQ_ECORRUPT, kWhereBfs, i);
}

// ---- the device-driven level loop (FQ_BFS_DEVICE_LOOP) ----
// The same level as the host-driven loop, with the host's per-level decisions taken by two
// one-thread kernels: loop_begin_kernel before the level (encode form, direction) and
// loop_end_kernel after it (records, statistics, termination), which set the graph's
// conditional handles.

__global__ void loop_init_kernel(LoopState *ls, const Counters *ctr, uint64_t m, uint64_t n_iso)
{
    ls->n_f = ctr->n_f_next;
    ls->m_f = ctr->r_m_f;
    ls->visited = ls->n_f;
    ls->m_u = m - ls->m_f;
    ls->log_used = 0;
    ls->d = 0;
    ls->dir = FQ_TOP_DOWN;
    ls->status = FQ_OK;
    ls->soft_status = FQ_OK;
    ls->root_iso = ls->m_f == 0 ? 1u : 0u;
    memset(&ls->stats, 0, sizeof(ls->stats));
    ls->stats.isolated = n_iso;
    ls->stats.kernel_launches[FQ_K_OTHER] = 2;  // bfs_init_kernel, loop_init_kernel
}

// Direction rule of the host loop: m_f*alpha > m_u  <=>  m_f > floor(m_u/alpha), and
// n_f*beta < n  <=>  n_f < ceil(n/beta), so no product can overflow.
// The handle set here picks the level body: 2 * encode form (0 queue + mirrored bitmap, 1 queue +
// bitmap from the bitmap, 2 no codec stage) + direction (0 top-down, 1 bottom-up), or kCaseSmall for
// a mirrored top-down level of at most kSmallIds ids when the one-CTA codec stage applies.
__global__ void loop_begin_kernel(LoopState *ls, uint64_t n, int codec, int small_ok, cudaGraphConditionalHandle h_case)
{
    const uint32_t flags = ls->p.flags;
    const unsigned long long alpha = ls->p.alpha, beta = ls->p.beta;
    uint32_t dir = ls->dir;
    if (flags & FQ_BFS_FORCE_TOP_DOWN) dir = FQ_TOP_DOWN;
    else if (flags & FQ_BFS_FORCE_BOTTOM_UP) dir = FQ_BOTTOM_UP;
    else if (dir == FQ_TOP_DOWN && ls->m_f > ls->m_u / alpha) dir = FQ_BOTTOM_UP;
    else if (dir == FQ_BOTTOM_UP && ls->n_f < (n + beta - 1) / beta) dir = FQ_TOP_DOWN;
    ls->dir = dir;
    const bool coded = codec && ls->n_f >= ls->p.min_codec_ids;
    ls->coded = coded ? 1u : 0u;
    const uint32_t enc = !coded ? 2u : (2ull * ls->n_f > n ? 1u : 0u);
    const bool small = small_ok && enc == 0u && dir == FQ_TOP_DOWN && ls->n_f <= kSmallIds;
    ls->small = small ? 1u : 0u;
    cudaGraphSetConditional(h_case, small ? kCaseSmall : 2u * enc + (dir == FQ_TOP_DOWN ? 0u : 1u));
}

// Appends the level's Q_d, B_d [, V_d] to the stream log when they fit (the test loop_end_kernel
// repeats to advance the log).
__global__ void log_append_kernel(const LoopState *ls, const Counters *ctr, const uint8_t *qs, const uint8_t *bs,
                                  const uint8_t *vs, uint8_t *log, int want_v)
{
    const bool coded = ls->coded != 0u;
    const unsigned long long qb = coded ? ctr->q_bytes : 0ull, bb = coded ? ctr->b_bytes : 0ull;
    const unsigned long long vb = want_v ? ctr->v_bytes : 0ull;
    const unsigned long long used = ls->log_used;
    if (used + qb + bb + vb > ls->p.log_cap) return;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    const uint8_t *src[3] = {qs, bs, vs};
    const unsigned long long len[3] = {qb, bb, vb};
    unsigned long long at = used;
    for (int k = 0; k < 3; k++) {
        uint8_t *dst = log + at;
        const bool vec = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src[k]) | len[k]) & 15u) == 0;
        if (vec) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src[k]);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            for (uint64_t i = tid; i < len[k] / 16; i += stride) d4[i] = s4[i];
        } else {
            for (uint64_t i = tid; i < len[k]; i += stride) dst[i] = src[k][i];
        }
        at += len[k];
    }
}

__global__ void loop_end_kernel(LoopState *ls_out, const Counters *ctr_in, fq_level_record *recs, uint64_t n,
                                uint64_t n_iso, int codec, int want_v, int has_log, int overlap,
                                cudaGraphConditionalHandle h_while)
{
    // local copies: every load is issued up front, the state is written back once at the end
    LoopState lsv = *ls_out;
    const Counters cv = *ctr_in;
    LoopState *ls = &lsv;
    const Counters *ctr = &cv;
    uint32_t go = 0;
    const uint32_t d = ls->d, dir = ls->dir;
    const unsigned long long n_f = ls->n_f, m_f = ls->m_f;
    fq_bfs_stats &st = ls->stats;
    if (ctr->r_err_q != FQ_OK) ls->status = ctr->r_err_q;
    else if (ctr->r_err_v != FQ_OK) ls->status = ctr->r_err_v;
    else if (ls->coded && dir == FQ_TOP_DOWN && ctr->dec_n != n_f) ls->status = FQ_ECORRUPT;
    if (ls->status != FQ_OK) {
        ls_out->status = ls->status;
        cudaGraphSetConditional(h_while, 0u);
        return;
    }
    const unsigned long long examined = dir == FQ_TOP_DOWN ? m_f : ctr->r_examined;
    const unsigned long long nf_next = ctr->n_f_next, mf_next = ctr->r_m_f;
    const bool coded = ls->coded != 0u;
    const unsigned long long qb = coded ? ctr->q_bytes : 0, bb = coded ? ctr->b_bytes : 0;
    const unsigned long long vb = want_v ? ctr->v_bytes : 0;
    const unsigned long long nbytes = (n + 7) / 8;
    const bool dense = 2ull * n_f > n;

    const unsigned long long cols_read = dir == FQ_TOP_DOWN ? m_f : ctr->r_cols_read;
    const LevelIn lin{n, n_iso, ls->visited, n_f, examined, cols_read, nf_next, qb, bb, vb, dir, ls->root_iso, coded,
                      want_v != 0};
    level_bytes(lin, st.kernel_bytes);
    const bool small = ls->small != 0u;
    if (coded) st.kernel_launches[FQ_K_ENCODE] += small ? 1 : (dense ? 8 : 2);
    if (want_v) st.kernel_launches[FQ_K_ENCODE] += 4;  // width sum from the bitmap, positions, widths, pack
    if (dir == FQ_TOP_DOWN) {
        if (coded && !small) st.kernel_launches[FQ_K_DECODE] += 3 + (overlap ? 1 : 0);
        st.kernel_launches[FQ_K_TOP_DOWN] += 2;
    } else {
        if (coded) st.kernel_launches[FQ_K_DECODE] += 4 + (overlap ? 1 : 0);
        st.kernel_launches[FQ_K_BOTTOM_UP] += 1;
    }
    st.kernel_launches[FQ_K_COMPACT] += 2;
    st.kernel_launches[FQ_K_OTHER] += 2 + (has_log ? 1 : 0);  // loop_begin, loop_end [, log_append]

    unsigned long long log_off = ~0ull;
    if (has_log && codec && (coded || want_v)) {
        const unsigned long long need = qb + bb + vb;
        if (ls->log_used + need > ls->p.log_cap) {
            ls->soft_status = FQ_ENOSPC;
        } else {
            log_off = ls->log_used;
            ls->log_used += need;
        }
    }
    if (d < ls->p.max_levels) {
        fq_level_record &r = recs[d];
        r.level = d;
        r.direction = dir;
        r.n_f = n_f;
        r.m_f = m_f;
        r.m_u = ls->m_u;
        r.examined = examined;
        r.cols_read = cols_read;
        r.q_bytes = qb;
        r.b_bytes = bb;
        r.v_bytes = vb;
        r.log_offset = log_off;
        for (int k = 0; k < FQ_NUM_KCLASS; k++) r.kernel_ms[k] = 0.f;
    }
    st.levels = d + 1;
    if (dir == FQ_BOTTOM_UP && d < 32) st.directions |= 1u << d;
    st.reached += n_f;
    st.reached_edges += m_f;
    st.edges_examined += examined;
    st.raw_queue_bytes += 4 * n_f;
    st.enc_queue_bytes += qb;
    st.raw_bitmap_bytes += nbytes;
    st.enc_bitmap_bytes += bb;
    st.enc_visited_bytes += vb;

    if (nf_next != 0) {
        ls->n_f = nf_next;
        ls->m_f = mf_next;
        ls->visited += nf_next;
        ls->m_u -= mf_next;
        ls->d = d + 1;
        if ((uint64_t)d + 1 >= n || ls->visited > n) ls->status = FQ_ECORRUPT;  // at most n levels, n vertices
        else go = 1;
    }
    *ls_out = lsv;
    cudaGraphSetConditional(h_while, go);
}

}  // namespace

// ------------------------------------------------------------------ graph handle

struct fq_graph {
    const int64_t *off;
    const uint32_t *cols;
    uint64_t n, m, nwords;
    uint64_t n_iso;   // vertices of degree 0
    int device;
    uint8_t *mem;
    uint64_t mem_bytes;
    fq_allocator alloc;  // the allocator mem came from (alloc == NULL: cudaMalloc)
    Counters *ctr;
    Scratch sq, sv;   // codec scratch: Q/B streams and decodes; V stream
    uint32_t *q, *q2;
    uint64_t *fbits, *fbits2, *next, *visited;
    uint32_t *iso32;
    uint4 *hc;        // bottom-up head records (NULL when the graph has 2^32 or more adjacency entries)
    uint8_t *qs, *bs, *vs;
    uint64_t qs_cap, bs_cap;
    HubItem *items;
    uint64_t items_cap;
    uint32_t *tile_cnt, *vis_cnt;  // compaction: per-tile counts of the next frontier and of the visited set
    uint32_t *last_set, *last_clear;  // per tile: 1 + its last set / clear vertex of the visited bitmap (0: none)
    uint32_t *wb;                     // V_d's block widths from the bitmap (fbw_kernel; zero between calls)
    uint32_t *wspan;                  //   per sub-tile: the block it starts that runs past it (or none), then
                                      //   the widths of the blocks it holds whole
    uint32_t cmp_tiles, cmp_sub;    //   tiles, and 256-word sub-tiles per tile
    uint8_t *host;  // pinned: Counters copy, then LoopState and level records (device-driven loop)
    cudaEvent_t ev[2 * FQ_NUM_KCLASS];
    cudaStream_t ov_stream;  // FQ_BFS_OVERLAP, host-driven loop: the codec stage's stream
    cudaStream_t tm_stream;  // FQ_BFS_TIMING, host-driven loop: where each level is captured
    cudaEvent_t ov_ev[2];    //   fork (after the previous compaction) and join (before this one)
    // device-driven level loop: state, records and the cached executable graph with its key
    LoopState *ls;
    fq_level_record *recs;
    cudaGraph_t dl_graph;
    cudaGraphExec_t dl_exec;
    cudaStream_t dl_stream;
    cudaStream_t dl_side[2];  // capture-time side streams of the level bodies (V_d; the overlapped codec stage)
    cudaEvent_t dl_ev[3];     // their fork and join events
    const int32_t *dl_depth;
    const uint32_t *dl_parent;
    const uint8_t *dl_log;
    uint32_t dl_mode;
    uint32_t dl_tune;  // tuning-table generation the graph's grids were taken from
};

namespace {

uint64_t al256(uint64_t x) { return (x + 255u) / 256u * 256u; }
constexpr uint64_t kHostLs = 256;  // offset of the LoopState copy in the pinned host block

// NVTX range names of the kernel classes (FQ_K_*): the host-driven loop encloses each class's
// launches in one range, so profilers can select a class by name.
const char *const kClassRange[FQ_NUM_KCLASS] = {"fq:top_down", "fq:bottom_up", "fq:compact",
                                                "fq:encode", "fq:decode", "fq:other"};

struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

struct Timer {
    fq_graph *g;
    cudaStream_t st;
    bool on;
    double *ms;
    uint64_t *launches;
    cudaStream_t cls_st[FQ_NUM_KCLASS];  // the stream each class's launches go to (0: st)
    bool ext = false;                    // recording inside a stream capture: as event record nodes
    cudaStream_t of(int k) const { return cls_st[k] ? cls_st[k] : st; }
    void record(cudaEvent_t e, cudaStream_t s) const
    {
        if (ext) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    void begin(int k)
    {
        nvtxRangePushA(kClassRange[k]);
        if (on) record(g->ev[2 * k], of(k));
    }
    void end(int k, int nlaunch)
    {
        if (launches) launches[k] += nlaunch;
        if (on) record(g->ev[2 * k + 1], of(k));
        nvtxRangePop();
    }
    // Adds the class's elapsed time since begin() to ms[k] and returns it (0 when not timing).
    float collect(int k)
    {
        if (!on) return 0.f;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g->ev[2 * k], g->ev[2 * k + 1]) != cudaSuccess) return 0.f;
        ms[k] += t;
        return t;
    }
};

#define FQ_CU(expr)                                   \
    do {                                              \
        const cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) {                      \
            note_cuda_error(_e, __LINE__);            \
            return _e;                                \
        }                                             \
    } while (0)

// The steps of one level, shared by the host-driven loop (sizes from the host, ls == nullptr)
// and the device-driven one (sizes from the loop state: ls != nullptr, grids sized for the
// largest case).

// Level 0: cleared outputs and bitmaps, the root, V_0.
cudaError_t step_init(fq_graph *g, uint32_t root, int32_t *d_depth, uint32_t *d_parent, const LoopState *ls,
                      cudaStream_t st)
{
    const uint64_t n = g->n, nwords = g->nwords;
    FQ_CU(cudaMemsetAsync(d_depth, 0xff, 4 * n, st));
    if (d_parent) FQ_CU(cudaMemsetAsync(d_parent, 0xff, 4 * n, st));
    FQ_CU(cudaMemsetAsync(g->fbits, 0, 8 * (nwords + 2), st));
    FQ_CU(cudaMemsetAsync(g->next, 0, 8 * (nwords + 2), st));
    FQ_CU(cudaMemsetAsync(g->visited, 0, 8 * (nwords + 2), st));
    FQ_CU(cudaMemsetAsync(g->vis_cnt, 0, 4 * (uint64_t)g->cmp_tiles, st));
    FQ_CU(cudaMemsetAsync(g->ctr, 0, sizeof(Counters), st));
    bfs_init_kernel<<<1, 256, 0, st>>>(g->off, root, n, d_depth, d_parent, g->q, g->fbits, g->visited, g->vis_cnt,
                                       64ull * kCmpSubWords * g->cmp_sub, g->cmp_tiles, g->last_set, g->last_clear, g->ctr,
                                       g->sq, g->sv, ls);
    return cudaGetLastError();
}

// Step 1: Q_d, and B_d (mirrored from the queue when 2 n_f <= n, else from the bitmap).  With px,
// Q_d is an FQX stream (patched exceptions) and B_d always comes from the bitmap (its inner stream
// is FQ, so it cannot be mirrored from Q_d).
cudaError_t step_encode_q(fq_graph *g, bool dense, uint64_t n_f, const LoopState *ls, cudaStream_t st, bool px)
{
    const uint64_t n = g->n;
    const uint64_t *n_dev = ls ? reinterpret_cast<const uint64_t *>(&ls->n_f) : nullptr;
    const uint64_t n_max = ls ? n : n_f;
    uint64_t *q_bytes = reinterpret_cast<uint64_t *>(&g->ctr->q_bytes);
    uint64_t *b_bytes = reinterpret_cast<uint64_t *>(&g->ctr->b_bytes);
    if (px) {
        FQ_CU(encode_fq(g->q, n_f, n_dev, n_max, g->qs, g->qs_cap, q_bytes, g->sq, st, true));
        FQ_CU(reset_status(g->sq, n / 2 + 1, st));
        FQ_CU(encode_fb(g->fbits, n, g->bs, g->bs_cap, b_bytes, g->sq, st));
    } else if (!dense) {
        Mirror mb;
        mb.out = g->bs;
        mb.cap = g->bs_cap;
        mb.out_bytes = b_bytes;
        mb.words = g->fbits;
        mb.nbits = n;
        FQ_CU(encode_fq_mirror(g->q, n_f, n_dev, n_max, g->qs, g->qs_cap, q_bytes, mb, g->sq, st));
    } else {  // a frontier denser than half the vertices: its bitmap codes the clear positions
        FQ_CU(encode_fq(g->q, n_f, n_dev, n_max, g->qs, g->qs_cap, q_bytes, g->sq, st));
        FQ_CU(reset_status(g->sq, n / 2 + 1, st));
        FQ_CU(encode_fb(g->fbits, n, g->bs, g->bs_cap, b_bytes, g->sq, st));
    }
    return cudaSuccess;
}

// Step 1 (V_d): the width sum from the bitmap (a dense visited set usually ends as raw words, and
// then nothing more is computed), else the visited bitmap's positions (set or clear, by the mode
// the previous compaction chose) and their FB encode.
cudaError_t step_encode_v(fq_graph *g, cudaStream_t st)
{
    fbw_kernel<<<g->cmp_tiles * g->cmp_sub, kThreads, 0, st>>>(g->visited, g->nwords, g->n, g->cmp_sub, g->cmp_tiles, g->vis_cnt,
                                                 g->last_set, g->last_clear, g->wb, g->wspan, g->wspan + g->cmp_tiles * g->cmp_sub,
                                                 g->sv);
    static std::atomic<bool> smem_set[64];
    FQ_CU(allow_smem(v_extract_kernel, kCmpSmem, smem_set));
    v_extract_kernel<<<g->cmp_tiles, kThreads, kCmpSmem, st>>>(g->visited, g->nwords, g->n, g->cmp_sub, g->cmp_tiles,
                                                               g->vis_cnt, g->sv);
    FQ_CU(cudaGetLastError());
    return encode_fb_positions(g->visited, g->n, g->vs, g->bs_cap, reinterpret_cast<uint64_t *>(&g->ctr->v_bytes),
                               g->sv, st);
}

// Steps 1 and 3 of a small top-down level in one launch: Q_d with its mirrored B_d, and Q_d's decode.
cudaError_t step_codec_small(fq_graph *g, uint64_t n_f, const LoopState *ls, cudaStream_t st)
{
    Mirror mb;
    mb.out = g->bs;
    mb.cap = g->bs_cap;
    mb.out_bytes = reinterpret_cast<uint64_t *>(&g->ctr->b_bytes);
    mb.words = g->fbits;
    mb.nbits = g->n;
    const uint64_t *n_dev = ls ? reinterpret_cast<const uint64_t *>(&ls->n_f) : nullptr;
    return codec_small(g->q, n_f, n_dev, g->qs, g->qs_cap, reinterpret_cast<uint64_t *>(&g->ctr->q_bytes), mb, g->q2,
                       kSmallIds, reinterpret_cast<uint64_t *>(&g->ctr->dec_n), g->sq, st);
}

// Step 3, top-down: decode Q_d.
cudaError_t step_decode_q(fq_graph *g, uint64_t n_f, const LoopState *ls, cudaStream_t st)
{
    return decode_fq(g->qs, 0, reinterpret_cast<const uint64_t *>(&g->ctr->q_bytes), g->q2, ls ? g->n : n_f,
                     reinterpret_cast<uint64_t *>(&g->ctr->dec_n), g->sq, st);
}

// Step 4, top-down: expand the (decoded) queue.
cudaError_t step_top_down(fq_graph *g, bool codec, uint64_t n_f, int32_t newdepth, int32_t *d_depth,
                          uint32_t *d_parent, const LoopState *ls, cudaStream_t st)
{
    const int sms = num_sms();
    const uint32_t *qin = codec ? g->q2 : g->q;
    const uint32_t grid =
        ls ? (uint32_t)sms * 8 : (uint32_t)std::min<uint64_t>(cdiv(std::max<uint64_t>(n_f, 1), kThreads / 32), (uint64_t)sms * 8);
    uint32_t *next32 = reinterpret_cast<uint32_t *>(g->next);
    const uint32_t *vis32 = reinterpret_cast<const uint32_t *>(g->visited);
    td_expand_kernel<<<grid, kThreads, 0, st>>>(qin, n_f, g->off, g->cols, vis32, next32, d_depth, d_parent, newdepth,
                                                g->items, &g->ctr->hub_items, g->items_cap, g->n, g->sq.ctl,
                                                &g->ctr->m_f_next, ls);
    td_hub_kernel<<<tuned_grid(FQ_TUNE_TD_HUB, g->n, (uint64_t)sms * 6, (uint64_t)sms * 32), kThreads, 0, st>>>(g->items, &g->ctr->hub_items, g->items_cap, g->cols, vis32, next32,
                                                d_depth, d_parent, newdepth, g->off, &g->ctr->m_f_next, ls);
    return cudaGetLastError();
}

// Step 3, bottom-up: decode B_d.
cudaError_t step_decode_b(fq_graph *g, cudaStream_t st)
{
    return decode_fb(g->bs, 0, reinterpret_cast<const uint64_t *>(&g->ctr->b_bytes), g->fbits2, g->n, g->sq, st);
}

// Overlap: the decoded queue / bitmap compared with the raw one the expansion consumes.
cudaError_t step_check_q(fq_graph *g, uint64_t n_f, const LoopState *ls, cudaStream_t st)
{
    const uint64_t nmax = ls ? g->n : n_f;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, cdiv(nmax, 4 * 256)), 4 * (uint64_t)num_sms());
    rt_check_queue_kernel<<<grid, 256, 0, st>>>(g->q, g->q2, n_f, &g->ctr->dec_n, g->sq.ctl, ls);
    return cudaGetLastError();
}
cudaError_t step_check_b(fq_graph *g, cudaStream_t st)
{
    const uint32_t grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, cdiv(g->nwords, 256)), 4 * (uint64_t)num_sms());
    rt_check_bitmap_kernel<<<grid, 256, 0, st>>>(g->fbits, g->fbits2, g->nwords, g->sq.ctl);
    return cudaGetLastError();
}

// Step 4, bottom-up: sweep the unvisited vertices against the (decoded) frontier bitmap.
cudaError_t step_bottom_up(fq_graph *g, bool codec, int32_t newdepth, int32_t *d_depth, uint32_t *d_parent,
                           const LoopState *ls, cudaStream_t st)
{
    const int sms = num_sms();
    const uint64_t *fin = codec ? g->fbits2 : g->fbits;
    const uint64_t words32 = cdiv(g->n, 32);
    const uint32_t grid = tuned_grid(FQ_TUNE_BU_SWEEP, g->n, std::min<uint64_t>(cdiv(words32, kThreads / 32), (uint64_t)sms * 16),
                                     cdiv(words32, kThreads / 32));
    if (g->hc)  // one warp per 32 words at a time: no more warps than chunks of 32 words
        bu_sweep_head_kernel<<<std::max<uint32_t>((uint32_t)std::min<uint64_t>(grid, cdiv(cdiv(words32, 32), kThreads / 32)), 1),
                               kThreads, 0, st>>>(
            reinterpret_cast<const uint32_t *>(fin), reinterpret_cast<const uint32_t *>(g->visited), g->iso32,
            reinterpret_cast<uint32_t *>(g->next), g->hc, g->cols, d_depth, d_parent, newdepth, g->n,
            &g->ctr->examined, &g->ctr->m_f_next, &g->ctr->cols_read, ls);
    else
        bu_sweep_kernel<<<std::max<uint32_t>(grid, 1), kThreads, 0, st>>>(
            reinterpret_cast<const uint32_t *>(fin), reinterpret_cast<const uint32_t *>(g->visited), g->iso32,
            reinterpret_cast<uint32_t *>(g->next), g->off, g->cols, d_depth, d_parent, newdepth, g->n,
            &g->ctr->examined, &g->ctr->m_f_next, &g->ctr->cols_read, ls);
    return cudaGetLastError();
}

// Step 5: compaction (+ the visited counts V_{d+1}'s extraction starts from, cleared scratch for the
// next level).
cudaError_t step_compact(fq_graph *g, bool want_v, cudaStream_t st)
{
    const uint32_t ct = g->cmp_tiles;
    cmp_count_kernel<<<ct, kThreads, 0, st>>>(g->next, g->visited, g->nwords, g->n, g->cmp_sub, g->tile_cnt, g->vis_cnt,
                                              g->last_set, g->last_clear, want_v ? 1 : 0);
    static std::atomic<bool> smem_set[64];
    FQ_CU(allow_smem(cmp_extract_kernel, kCmpSmem, smem_set));
    cmp_extract_kernel<<<ct, kThreads, kCmpSmem, st>>>(g->next, g->fbits, g->nwords, g->n, g->cmp_sub, ct, g->tile_cnt,
                                                       g->vis_cnt, g->q, g->ctr, g->sq, g->sv, want_v ? 1 : 0);
    return cudaGetLastError();
}

// Handle creation and destruction synchronise the whole device and free memory, which would
// invalidate a stream capture running in another thread; the device-loop build (its captures and
// instantiation) and those calls therefore never overlap.
std::mutex g_capture_mu;

// The allocator fq_graph_create takes handle workspaces from (fq_set_allocator); alloc == NULL
// selects cudaMalloc.
std::mutex g_alloc_mu;
fq_allocator g_alloc = {nullptr, nullptr, nullptr};

cudaError_t capture_segment(cudaStream_t cs, cudaGraph_t *out, cudaError_t (*fn)(void *), void *ctx)
{
    *out = nullptr;
    FQ_CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    const cudaError_t e = fn(ctx);
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        note_cuda_error(e != cudaSuccess ? e : e2, __LINE__);
        return e != cudaSuccess ? e : e2;
    }
    *out = gr;
    return cudaSuccess;
}

struct LoopBuild {
    fq_graph *g;
    int32_t *depth;
    uint32_t *parent;
    uint8_t *log;
    bool codec, want_v, px, overlap;
    int enc, dir;  // the level case a segment is captured for (seg_level); enc 3: kCaseSmall
};

cudaError_t add_kernel_node(cudaGraphNode_t *node, cudaGraph_t gr, const cudaGraphNode_t *dep, void *func,
                            void **args)
{
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = dim3(1, 1, 1);
    kp.blockDim = dim3(1, 1, 1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, gr, dep, dep ? 1 : 0, &kp);
}

// A conditional node after `dep` in `gr` on handle h (type, size bodies); returns the bodies.
cudaError_t add_conditional(cudaGraphNode_t *node, cudaGraph_t gr, const cudaGraphNode_t *dep,
                            cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, unsigned size,
                            cudaGraph_t *bodies)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    FQ_CU(cudaGraphAddNode(node, gr, dep, nullptr, dep ? 1 : 0, &p));
    for (unsigned i = 0; i < size; i++) bodies[i] = p.conditional.phGraph_out[i];
    return cudaSuccess;
}

// Segments of the loop body, each captured into its own graph.
cudaError_t seg_init(void *p)
{
    const LoopBuild &c = *static_cast<const LoopBuild *>(p);
    const cudaError_t r = step_init(c.g, 0, c.depth, c.parent, c.g->ls, c.g->dl_stream);
    if (r != cudaSuccess) return r;
    loop_init_kernel<<<1, 1, 0, c.g->dl_stream>>>(c.g->ls, c.g->ctr, c.g->m, c.g->n_iso);
    return cudaGetLastError();
}

// One level's work before the compaction, for one (encode form, direction) case: the visited stream
// V_d on a side stream, and on the main stream the Q/B encode, the decode of the consumed form and
// the expansion of it -- or, with the overlap, the expansion of the raw frontier on the main stream
// while a second side stream encodes, decodes and compares.  The side streams fork from and join
// back into the main stream inside the segment, so the level is one child graph with its own
// parallel branches.
cudaError_t seg_level(void *p)
{
    const LoopBuild &c = *static_cast<const LoopBuild *>(p);
    fq_graph *g = c.g;
    cudaStream_t s0 = g->dl_stream;
    const bool small = c.enc == 3;  // kCaseSmall: a mirrored top-down level, one-CTA codec stage
    const bool coded = c.codec && c.enc != 2;
    const bool ovl = coded && c.overlap && !small;
    FQ_CU(cudaEventRecord(g->dl_ev[0], s0));
    if (c.want_v) {
        FQ_CU(cudaStreamWaitEvent(g->dl_side[0], g->dl_ev[0], 0));
        FQ_CU(step_encode_v(g, g->dl_side[0]));
        FQ_CU(cudaEventRecord(g->dl_ev[1], g->dl_side[0]));
    }
    cudaStream_t cst = s0;
    if (ovl) {
        FQ_CU(cudaStreamWaitEvent(g->dl_side[1], g->dl_ev[0], 0));
        cst = g->dl_side[1];
    }
    if (small) {
        FQ_CU(step_codec_small(g, 0, g->ls, cst));
    } else if (coded) {
        FQ_CU(step_encode_q(g, c.enc == 1, 0, g->ls, cst, c.px));
        FQ_CU(c.dir == FQ_TOP_DOWN ? step_decode_q(g, 0, g->ls, cst) : step_decode_b(g, cst));
        if (ovl) {
            FQ_CU(c.dir == FQ_TOP_DOWN ? step_check_q(g, 0, g->ls, cst) : step_check_b(g, cst));
            FQ_CU(cudaEventRecord(g->dl_ev[2], cst));
        }
    }
    const bool consume_decoded = coded && !ovl;
    if (c.dir == FQ_TOP_DOWN) FQ_CU(step_top_down(g, consume_decoded, 0, 0, c.depth, c.parent, g->ls, s0));
    else FQ_CU(step_bottom_up(g, consume_decoded, 0, c.depth, c.parent, g->ls, s0));
    if (c.want_v) FQ_CU(cudaStreamWaitEvent(s0, g->dl_ev[1], 0));
    if (ovl) FQ_CU(cudaStreamWaitEvent(s0, g->dl_ev[2], 0));
    return cudaSuccess;
}

cudaError_t seg_compact(void *p)
{
    const LoopBuild &c = *static_cast<const LoopBuild *>(p);
    const cudaError_t r = step_compact(c.g, c.want_v, c.g->dl_stream);
    if (r != cudaSuccess || !c.log) return r;
    log_append_kernel<<<4 * num_sms(), 256, 0, c.g->dl_stream>>>(c.g->ls, c.g->ctr, c.g->qs, c.g->bs, c.g->vs, c.log,
                                                                 c.want_v ? 1 : 0);
    return cudaGetLastError();
}

// Build the device-driven loop for these buffers and mode, as a linear chain inside the while node:
//   init -> while(h_while) { begin -> switch(h_case: 7 level bodies) -> compact [-> log] -> end }
// loop_begin picks the case = 2 * (encode form: 0 mirrored, 1 from the bitmap, 2 none) + direction,
// or kCaseSmall (a small mirrored top-down level: the one-CTA codec stage).
// Every parallel branch (V_d beside the level; with the overlap, the codec stage beside the
// expansion) forks and joins inside a case body, which is a plain child graph.  A node that joins
// a conditional node with another branch directly in the while body was, on rare launches, never
// started by the executor although every branch had completed, so the body keeps no such join.
cudaError_t build_device_loop(const LoopBuild &b, cudaGraph_t *out)
{
    fq_graph *g = b.g;
    cudaStream_t cs = g->dl_stream;
    cudaGraph_t sg_init = nullptr, sg_cmp = nullptr, top = nullptr;
    cudaGraph_t sg_case[kCases] = {};
    cudaError_t e = capture_segment(cs, &sg_init, seg_init, const_cast<LoopBuild *>(&b));
    for (int k = 0; k < kCases && e == cudaSuccess; k++) {
        LoopBuild ctx = b;
        ctx.enc = b.codec ? k / 2 : 2;  // without the codec stage every case is the raw level
        ctx.dir = k % 2;
        if (k == (int)kCaseSmall) {  // enc 3: the one-CTA codec stage (top-down, mirrored)
            ctx.enc = b.codec ? 3 : 2;
            ctx.dir = FQ_TOP_DOWN;
        }
        e = capture_segment(cs, &sg_case[k], seg_level, &ctx);
    }
    if (e == cudaSuccess) e = capture_segment(cs, &sg_cmp, seg_compact, const_cast<LoopBuild *>(&b));
    if (e == cudaSuccess) e = cudaGraphCreate(&top, 0);
    if (e != cudaSuccess) goto done;
    {
        cudaGraphNode_t n_init, n_while, n_begin, n_sw, n_cmp, n_end;
        cudaGraph_t body, cases[kCases];
        cudaGraphConditionalHandle h_while, h_case;
        if ((e = cudaGraphAddChildGraphNode(&n_init, top, nullptr, 0, sg_init)) != cudaSuccess) goto done;
        if ((e = cudaGraphConditionalHandleCreate(&h_while, top, 1, cudaGraphCondAssignDefault)) != cudaSuccess) goto done;
        if ((e = add_conditional(&n_while, top, &n_init, h_while, cudaGraphCondTypeWhile, 1, &body)) != cudaSuccess)
            goto done;
        if ((e = cudaGraphConditionalHandleCreate(&h_case, body, 0, 0)) != cudaSuccess) goto done;
        {
            LoopState *ls = g->ls;
            uint64_t n = g->n;
            int codec = b.codec ? 1 : 0;
            int small_ok = b.codec && !b.px && !b.overlap ? 1 : 0;
            void *args[] = {&ls, &n, &codec, &small_ok, &h_case};
            if ((e = add_kernel_node(&n_begin, body, nullptr, (void *)loop_begin_kernel, args)) != cudaSuccess) goto done;
        }
        if ((e = add_conditional(&n_sw, body, &n_begin, h_case, cudaGraphCondTypeSwitch, kCases, cases)) != cudaSuccess)
            goto done;
        for (int k = 0; k < kCases; k++) {
            cudaGraphNode_t c;
            if ((e = cudaGraphAddChildGraphNode(&c, cases[k], nullptr, 0, sg_case[k])) != cudaSuccess) goto done;
        }
        if ((e = cudaGraphAddChildGraphNode(&n_cmp, body, &n_sw, 1, sg_cmp)) != cudaSuccess) goto done;
        {
            LoopState *ls = g->ls;
            const Counters *ctr = g->ctr;
            fq_level_record *recs = g->recs;
            uint64_t n = g->n;
            uint64_t n_iso = g->n_iso;
            int codec = b.codec ? 1 : 0, want_v = b.want_v ? 1 : 0, has_log = b.log ? 1 : 0;
            int overlap = b.codec && b.overlap ? 1 : 0;
            void *args[] = {&ls, &ctr, &recs, &n, &n_iso, &codec, &want_v, &has_log, &overlap, &h_while};
            if ((e = add_kernel_node(&n_end, body, &n_cmp, (void *)loop_end_kernel, args)) != cudaSuccess) goto done;
        }
    }
done:
    if (sg_init) cudaGraphDestroy(sg_init);  // child-graph nodes hold their own copies
    if (sg_cmp) cudaGraphDestroy(sg_cmp);
    for (int k = 0; k < kCases; k++)
        if (sg_case[k]) cudaGraphDestroy(sg_case[k]);
    if (e != cudaSuccess) {
        note_cuda_error(e, __LINE__);
        if (top) cudaGraphDestroy(top);
        return e;
    }
    *out = top;
    return cudaSuccess;
}

// Frees a handle; the caller holds g_capture_mu.
void fq_graph_destroy_locked(fq_graph *g)
{
    cudaDeviceSynchronize();
    if (g->dl_exec) cudaGraphExecDestroy(g->dl_exec);
    if (g->dl_graph) cudaGraphDestroy(g->dl_graph);
    if (g->dl_stream) cudaStreamDestroy(g->dl_stream);
    for (int i = 0; i < 2; i++)
        if (g->dl_side[i]) cudaStreamDestroy(g->dl_side[i]);
    for (int i = 0; i < 3; i++)
        if (g->dl_ev[i]) cudaEventDestroy(g->dl_ev[i]);
    if (g->ov_stream) cudaStreamDestroy(g->ov_stream);
    if (g->tm_stream) cudaStreamDestroy(g->tm_stream);
    for (int i = 0; i < 2; i++)
        if (g->ov_ev[i]) cudaEventDestroy(g->ov_ev[i]);
    for (int i = 0; i < 2 * FQ_NUM_KCLASS; i++)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    if (g->host) cudaFreeHost(g->host);
    if (g->mem) {
        if (g->alloc.alloc) g->alloc.release(g->mem, g->mem_bytes, g->alloc.ctx);
        else cudaFree(g->mem);
    }
    delete g;
}

}  // namespace

extern "C" {

fq_status fq_set_allocator(const fq_allocator *a)
{
    if (a && (!a->alloc || !a->release)) return FQ_EINVAL;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc = a ? *a : fq_allocator{nullptr, nullptr, nullptr};
    return FQ_OK;
}

void fq_bfs_level_bytes(uint64_t n, uint64_t n_isolated, uint32_t root_isolated, const fq_level_record *rec,
                        uint64_t visited, uint64_t n_f_next, uint64_t *out)
{
    if (!rec || !out) return;
    for (int k = 0; k < FQ_NUM_KCLASS; k++) out[k] = 0;
    const LevelIn lin{n, n_isolated, visited, rec->n_f, rec->examined, rec->cols_read, n_f_next, rec->q_bytes,
                      rec->b_bytes, rec->v_bytes, rec->direction, root_isolated ? 1u : 0u, rec->q_bytes > 0,
                      rec->v_bytes > 0};
    level_bytes(lin, out);
}

fq_status fq_graph_create(const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, uint64_t m, fq_graph **out)
{
    if (!out || !d_offsets || (m && !d_cols) || n == 0 || n > 0xffffffffull) return FQ_EINVAL;
    *out = nullptr;
    std::lock_guard<std::mutex> lock(g_capture_mu);
    fq_graph *g = new (std::nothrow) fq_graph();
    if (!g) return FQ_ENOMEM;
    {
        std::lock_guard<std::mutex> alock(g_alloc_mu);
        g->alloc = g_alloc;
    }
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
    {  // compaction tiles: at most one wave of the extract kernel (3 CTAs of 64 KB shared memory per SM)
        const uint64_t subs = std::max<uint64_t>(1, cdiv(g->nwords, kCmpSubWords));
        g->cmp_sub = (uint32_t)cdiv(subs, 3 * (uint64_t)num_sms());
        g->cmp_tiles = (uint32_t)cdiv(subs, g->cmp_sub);
    }
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
    const bool with_hc = m < (1ull << 32);
    const uint64_t o_hc = o; o = al256(o + (with_hc ? 16 * n : 0));
    const uint64_t o_qs = o; o = al256(o + g->qs_cap);
    const uint64_t o_bs = o; o = al256(o + g->bs_cap);
    const uint64_t o_vs = o; o = al256(o + g->bs_cap);
    const uint64_t o_items = o; o = al256(o + sizeof(HubItem) * g->items_cap);
    const uint64_t o_tc = o; o = al256(o + 4 * (uint64_t)g->cmp_tiles);
    const uint64_t o_vc = o; o = al256(o + 4 * (uint64_t)g->cmp_tiles);
    const uint64_t o_ls_t = o; o = al256(o + 4 * (uint64_t)g->cmp_tiles);
    const uint64_t o_lc_t = o; o = al256(o + 4 * (uint64_t)g->cmp_tiles);
    const uint64_t o_wb = o; o = al256(o + 4 * (n / 128 + 2));
    const uint64_t o_span = o; o = al256(o + 8 * (uint64_t)g->cmp_tiles * g->cmp_sub);  // span[], then wpart[]
    const uint64_t o_ls = o; o = al256(o + sizeof(LoopState));
    const uint64_t o_recs = o; o = al256(o + sizeof(fq_level_record) * kMaxDeviceRecords);
    g->mem_bytes = o;
    if (g->alloc.alloc) {
        g->mem = static_cast<uint8_t *>(g->alloc.alloc(o, g->alloc.ctx));
        if (g->mem && (reinterpret_cast<uintptr_t>(g->mem) & 255u)) {  // the contract asks for 256-byte alignment
            g->alloc.release(g->mem, o, g->alloc.ctx);
            delete g;
            return FQ_EINVAL;
        }
    } else if (cudaMalloc(&g->mem, o) != cudaSuccess) {
        cudaGetLastError();
        g->mem = nullptr;
    }
    if (!g->mem) {
        delete g;
        return FQ_ENOMEM;
    }
    if (cudaMallocHost(&g->host, kHostLs + al256(sizeof(LoopState)) + sizeof(fq_level_record) * kMaxDeviceRecords) !=
        cudaSuccess) {
        cudaGetLastError();
        g->host = nullptr;
        if (g->alloc.alloc) g->alloc.release(g->mem, o, g->alloc.ctx);
        else cudaFree(g->mem);
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
    g->hc = with_hc ? reinterpret_cast<uint4 *>(g->mem + o_hc) : nullptr;
    g->qs = g->mem + o_qs;
    g->bs = g->mem + o_bs;
    g->vs = g->mem + o_vs;
    g->items = reinterpret_cast<HubItem *>(g->mem + o_items);
    g->tile_cnt = reinterpret_cast<uint32_t *>(g->mem + o_tc);
    g->vis_cnt = reinterpret_cast<uint32_t *>(g->mem + o_vc);
    g->last_set = reinterpret_cast<uint32_t *>(g->mem + o_ls_t);
    g->last_clear = reinterpret_cast<uint32_t *>(g->mem + o_lc_t);
    g->wb = reinterpret_cast<uint32_t *>(g->mem + o_wb);
    g->wspan = reinterpret_cast<uint32_t *>(g->mem + o_span);
    g->ls = reinterpret_cast<LoopState *>(g->mem + o_ls);
    g->recs = reinterpret_cast<fq_level_record *>(g->mem + o_recs);
    for (int i = 0; i < 2 * FQ_NUM_KCLASS; i++) cudaEventCreate(&g->ev[i]);
    if (cudaMemset(g->mem, 0, o) != cudaSuccess) {
        fq_graph_destroy_locked(g);
        return FQ_ECUDA;
    }
    iso_kernel<<<(uint32_t)std::min<uint64_t>(cdiv(cdiv(n, 32), 256), 4096), 256>>>(d_offsets, n, g->iso32,
                                                                                     &g->ctr->n_iso);
    if (g->hc) head_kernel<<<(uint32_t)std::min<uint64_t>(cdiv(n, 256), 8 * (uint64_t)num_sms()), 256>>>(d_offsets, d_cols, n, g->hc);
    unsigned long long n_iso = 0;
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&n_iso, &g->ctr->n_iso, sizeof(n_iso), cudaMemcpyDeviceToHost) != cudaSuccess) {
        fq_graph_destroy_locked(g);
        return FQ_ECUDA;
    }
    g->n_iso = n_iso;
    *out = g;
    return FQ_OK;
}

fq_status fq_graph_destroy(fq_graph *g)
{
    if (!g) return FQ_EINVAL;
    std::lock_guard<std::mutex> lock(g_capture_mu);
    fq_graph_destroy_locked(g);
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
    const uint32_t min_codec_ids = opts ? opts->min_codec_ids : 0u;
    const bool codec = !(flags & FQ_BFS_NO_CODEC);
    const bool want_visited = codec && (flags & FQ_BFS_VISITED_STREAM);
    const bool px = codec && (flags & FQ_BFS_PATCHED);
    const bool overlap = codec && (flags & FQ_BFS_OVERLAP);
    const uint64_t n = g->n;
    NvtxScope search_range((flags & FQ_BFS_DEVICE_LOOP) ? "fq_bfs_run:device_loop" : "fq_bfs_run:host_loop");

#define FQ_TRY(expr)                                  \
    do {                                              \
        const cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) {                      \
            note_cuda_error(_e, __LINE__);            \
            return FQ_ECUDA;                          \
        }                                             \
    } while (0)

    if (flags & FQ_BFS_DEVICE_LOOP) {
        // the whole search is one graph launch; the host reads the records once at the end
        const uint32_t mode = (codec ? 0u : FQ_BFS_NO_CODEC) | (want_visited ? FQ_BFS_VISITED_STREAM : 0u) |
                              (px ? FQ_BFS_PATCHED : 0u) | (overlap ? FQ_BFS_OVERLAP : 0u);
        if (!g->dl_exec || g->dl_depth != d_depth || g->dl_parent != d_parent || g->dl_log != d_stream_log ||
            g->dl_mode != mode || g->dl_tune != tune_generation()) {
            std::lock_guard<std::mutex> lock(g_capture_mu);
            if (g->dl_exec) cudaGraphExecDestroy(g->dl_exec);
            if (g->dl_graph) cudaGraphDestroy(g->dl_graph);
            g->dl_exec = nullptr;
            g->dl_graph = nullptr;
            if (!g->dl_stream) {
                FQ_TRY(cudaStreamCreateWithFlags(&g->dl_stream, cudaStreamNonBlocking));
                for (int i = 0; i < 2; i++) FQ_TRY(cudaStreamCreateWithFlags(&g->dl_side[i], cudaStreamNonBlocking));
                for (int i = 0; i < 3; i++) FQ_TRY(cudaEventCreateWithFlags(&g->dl_ev[i], cudaEventDisableTiming));
            }
            LoopBuild b{g, d_depth, d_parent, d_stream_log, codec, want_visited, px, overlap, 0, 0};
            FQ_TRY(build_device_loop(b, &g->dl_graph));
            FQ_TRY(cudaGraphInstantiate(&g->dl_exec, g->dl_graph, 0));
            g->dl_depth = d_depth;
            g->dl_parent = d_parent;
            g->dl_log = d_stream_log;
            g->dl_mode = mode;
            g->dl_tune = tune_generation();
        }
        LoopState *hls = reinterpret_cast<LoopState *>(g->host + kHostLs);
        fq_level_record *hrec = reinterpret_cast<fq_level_record *>(g->host + kHostLs + al256(sizeof(LoopState)));
        LoopParams prm{};
        prm.root = root;
        prm.alpha = alpha;
        prm.beta = beta;
        prm.flags = flags;
        prm.max_levels = h_levels ? std::min<uint32_t>(max_levels, kMaxDeviceRecords) : 0u;
        prm.min_codec_ids = min_codec_ids;
        prm.log_cap = d_stream_log ? stream_log_cap : 0ull;
        hls->p = prm;
        FQ_TRY(cudaMemcpyAsync(&g->ls->p, &hls->p, sizeof(LoopParams), cudaMemcpyHostToDevice, st));
        FQ_TRY(cudaGraphLaunch(g->dl_exec, st));
        FQ_TRY(cudaMemcpyAsync(hls, g->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, st));
        const uint32_t first = std::min<uint32_t>(prm.max_levels, 64u);  // most searches have fewer levels
        if (first) FQ_TRY(cudaMemcpyAsync(hrec, g->recs, sizeof(fq_level_record) * first, cudaMemcpyDeviceToHost, st));
        FQ_TRY(cudaStreamSynchronize(st));
        if (hls->status != FQ_OK) return (fq_status)hls->status;
        const uint32_t kept = std::min<uint32_t>(prm.max_levels, hls->stats.levels);
        if (kept > first) {
            FQ_TRY(cudaMemcpyAsync(hrec + first, g->recs + first, sizeof(fq_level_record) * (kept - first),
                                   cudaMemcpyDeviceToHost, st));
            FQ_TRY(cudaStreamSynchronize(st));
        }
        if (h_levels)
            for (uint32_t d = 0; d < kept; d++) h_levels[d] = hrec[d];
        fq_bfs_stats stats = hls->stats;
        stats.reached_edges /= 2;
        stats.isolated = g->n_iso;
        if (h_stats) *h_stats = stats;
        return (fq_status)hls->soft_status;
    }

    fq_bfs_stats stats;
    memset(&stats, 0, sizeof(stats));
    stats.isolated = g->n_iso;
    Timer tm{g, st, (flags & FQ_BFS_TIMING) != 0, stats.kernel_ms, stats.kernel_launches, {}};
    if (overlap && !g->ov_stream) {  // the codec stage's own stream, made on first use
        FQ_TRY(cudaStreamCreateWithFlags(&g->ov_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; i++) FQ_TRY(cudaEventCreateWithFlags(&g->ov_ev[i], cudaEventDisableTiming));
    }

    // ---- level 0 set-up
    tm.begin(FQ_K_OTHER);
    FQ_TRY(step_init(g, root, d_depth, d_parent, nullptr, st));
    tm.end(FQ_K_OTHER, 1);
    FQ_TRY(cudaMemcpyAsync(g->host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    FQ_TRY(cudaStreamSynchronize(st));
    tm.collect(FQ_K_OTHER);

    const Counters *hc = reinterpret_cast<const Counters *>(g->host);
    uint64_t n_f = hc->n_f_next, m_f = hc->r_m_f;
    uint64_t visited_count = n_f;
    uint64_t m_u = g->m - m_f;
    const uint32_t root_iso = m_f == 0 ? 1u : 0u;
    int dir = FQ_TOP_DOWN;
    uint64_t log_used = 0;
    fq_status result = FQ_OK;

    for (uint32_t d = 0;; d++) {
        const bool coded = codec && n_f >= min_codec_ids;  // below the threshold the frontier crosses raw
        // direction (host arithmetic: nothing waits for it)
        if (flags & FQ_BFS_FORCE_TOP_DOWN) dir = FQ_TOP_DOWN;
        else if (flags & FQ_BFS_FORCE_BOTTOM_UP) dir = FQ_BOTTOM_UP;
        else if (dir == FQ_TOP_DOWN && (unsigned __int128)m_f * alpha > (unsigned __int128)m_u) dir = FQ_BOTTOM_UP;
        else if (dir == FQ_BOTTOM_UP && (unsigned __int128)n_f * beta < (unsigned __int128)n) dir = FQ_TOP_DOWN;
        const int32_t newdepth = (int32_t)d + 1;
        // with the overlap the codec stage forks onto its own stream after the previous compaction
        // and joins before this level's compaction, while the expansion consumes the raw frontier
        const bool ovl = overlap && coded;
        // a small mirrored top-down level takes the one-CTA codec stage (encode and decode together)
        const bool small = coded && !px && !ovl && dir == FQ_TOP_DOWN && 2 * n_f <= n && n_f <= kSmallIds;
#define FQ_LV(expr)                                   \
    do {                                              \
        const cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return _e;             \
    } while (0)
        // the level's launches, on stream lst
        auto launch_level = [&](cudaStream_t lst) -> cudaError_t {
            cudaStream_t cst = lst;
            if (ovl) {
                FQ_LV(cudaEventRecord(g->ov_ev[0], lst));
                FQ_LV(cudaStreamWaitEvent(g->ov_stream, g->ov_ev[0], 0));
                cst = g->ov_stream;
            }
            tm.cls_st[FQ_K_ENCODE] = tm.cls_st[FQ_K_DECODE] = ovl ? cst : nullptr;
            // 1. encode F_d (Q_d and B_d), and V_d
            tm.begin(FQ_K_ENCODE);
            int enc_launches = 0;
            if (small) {
                FQ_LV(step_codec_small(g, n_f, nullptr, cst));
                enc_launches = 1;
            } else if (coded) {
                const bool dense = 2 * n_f > n;
                FQ_LV(step_encode_q(g, dense, n_f, nullptr, cst, px));
                enc_launches = dense ? 8 : 2;
            }
            if (want_visited) {
                FQ_LV(step_encode_v(g, cst));
                enc_launches += 4;
            }
            tm.end(FQ_K_ENCODE, enc_launches);
            // 3 + 4. decode the consumed form (overlap: decode and compare with the raw form), expand
            tm.begin(FQ_K_DECODE);
            if (coded && !small && dir == FQ_TOP_DOWN) FQ_LV(step_decode_q(g, n_f, nullptr, cst));
            if (coded && dir == FQ_BOTTOM_UP) FQ_LV(step_decode_b(g, cst));
            if (ovl) FQ_LV(dir == FQ_TOP_DOWN ? step_check_q(g, n_f, nullptr, cst) : step_check_b(g, cst));
            tm.end(FQ_K_DECODE, coded && !small ? (dir == FQ_TOP_DOWN ? 3 : 4) + (ovl ? 1 : 0) : 0);
            if (ovl) FQ_LV(cudaEventRecord(g->ov_ev[1], cst));
            const bool consume_decoded = coded && !ovl;
            if (dir == FQ_TOP_DOWN) {
                tm.begin(FQ_K_TOP_DOWN);
                FQ_LV(step_top_down(g, consume_decoded, n_f, newdepth, d_depth, d_parent, nullptr, lst));
                tm.end(FQ_K_TOP_DOWN, 2);
            } else {
                tm.begin(FQ_K_BOTTOM_UP);
                FQ_LV(step_bottom_up(g, consume_decoded, newdepth, d_depth, d_parent, nullptr, lst));
                tm.end(FQ_K_BOTTOM_UP, 1);
            }
            if (ovl) FQ_LV(cudaStreamWaitEvent(lst, g->ov_ev[1], 0));
            // 5. compaction (+ the visited counts per tile, cleared scratch for the next level)
            tm.begin(FQ_K_COMPACT);
            FQ_LV(step_compact(g, want_visited, lst));
            tm.end(FQ_K_COMPACT, 2);
            return cudaSuccess;
        };
#undef FQ_LV
        if (!tm.on) {
            FQ_TRY(launch_level(st));
        } else {
            // Timed: the level is captured as a graph and launched whole, so the class events measure
            // the kernels back to back as the device-driven loop runs them, not the host's submission
            // of each launch.  (The capture stream is the handle's own: the caller's may be the
            // legacy stream, which cannot capture.)
            std::lock_guard<std::mutex> lock(g_capture_mu);  // no handle is created or freed meanwhile
            if (!g->tm_stream) FQ_TRY(cudaStreamCreateWithFlags(&g->tm_stream, cudaStreamNonBlocking));
            FQ_TRY(cudaStreamBeginCapture(g->tm_stream, cudaStreamCaptureModeRelaxed));
            tm.st = g->tm_stream;
            tm.ext = true;
            const cudaError_t le = launch_level(g->tm_stream);
            tm.ext = false;
            tm.st = st;
            cudaGraph_t lg = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(g->tm_stream, &lg);
            cudaGraphExec_t lx = nullptr;
            cudaError_t xe = le != cudaSuccess ? le : ce;
            if (xe == cudaSuccess) xe = cudaGraphInstantiate(&lx, lg, 0);
            if (xe == cudaSuccess) xe = cudaGraphLaunch(lx, st);
            if (xe == cudaSuccess) xe = cudaStreamSynchronize(st);
            if (lx) cudaGraphExecDestroy(lx);
            if (lg) cudaGraphDestroy(lg);
            FQ_TRY(xe);
        }

        FQ_TRY(cudaMemcpyAsync(g->host, g->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        FQ_TRY(cudaStreamSynchronize(st));
        float lms[FQ_NUM_KCLASS] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        lms[FQ_K_ENCODE] = tm.collect(FQ_K_ENCODE);
        lms[FQ_K_DECODE] = tm.collect(FQ_K_DECODE);
        const int xk = dir == FQ_TOP_DOWN ? FQ_K_TOP_DOWN : FQ_K_BOTTOM_UP;
        lms[xk] = tm.collect(xk);
        lms[FQ_K_COMPACT] = tm.collect(FQ_K_COMPACT);
        if (hc->r_err_q != FQ_OK) return hc->r_err_q;
        if (hc->r_err_v != FQ_OK) return hc->r_err_v;
        if (coded && dir == FQ_TOP_DOWN && hc->dec_n != n_f) return FQ_ECORRUPT;

        const uint64_t examined = dir == FQ_TOP_DOWN ? m_f : hc->r_examined;
        const uint64_t nf_next = hc->n_f_next, mf_next = hc->r_m_f;
        const uint64_t qb = coded ? hc->q_bytes : 0, bb = coded ? hc->b_bytes : 0, vb = want_visited ? hc->v_bytes : 0;

        // algorithmic bytes of this level (design model)
        const uint64_t cols_read = dir == FQ_TOP_DOWN ? m_f : hc->r_cols_read;
        const LevelIn lin{n, g->n_iso, visited_count, n_f, examined, cols_read, nf_next, qb, bb, vb, (uint32_t)dir,
                          root_iso, coded, want_visited};
        level_bytes(lin, stats.kernel_bytes);

        uint64_t log_off = ~0ull;
        if (d_stream_log && codec && (coded || want_visited)) {
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
            r.cols_read = cols_read;
            r.q_bytes = qb;
            r.b_bytes = bb;
            r.v_bytes = vb;
            r.log_offset = log_off;
            for (int k = 0; k < FQ_NUM_KCLASS; k++) r.kernel_ms[k] = lms[k];
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
