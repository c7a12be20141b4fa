// msbfs.cu -- multi-source BFS: up to 64 roots traversed together, one bit per root in a 64-bit
// mask per vertex, all levels in one persistent (cooperative) kernel launch.
//
// A level-synchronous BFS (the thesis' frontier / visited-list recurrence, Algorithm 2) run for
// k roots at once, the sparse vectors becoming bit-sliced:
//   seen[v]     roots that reached v,      frontier[v]  roots that reached v at this level,
//   next[v]     roots arriving at the next level (OR of frontier[u] over the neighbours u, masked
//               by not-seen -- the SpMV t = A (x) f with the element-wise mask of the thesis).
// Per level, three phases separated by grid barriers:
//   U  every vertex: new = next & ~seen; seen |= new; frontier = new; depth[i][v] = level for the
//      bits i of new; flag v when new != 0 (and v has edges); per-CTA counts;
//   Q  every CTA: its queue offset from all CTAs' counts; writes its flagged vertices and the
//      running degree prefix (stops everything when the queue is empty);
//   P  edge-balanced push: each warp takes an equal share of the frontier's edges, 32 at a time,
//      finds each edge's source with a 5-step search over 32 staged prefix values, and ORs
//      frontier[src] & ~seen[dst] into next[dst] (64-bit atomicOr).
// The grid barriers spin with a bound; a barrier that gives up sets FQ_ETIMEOUT and every CTA
// leaves at its next barrier.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "fq_common.cuh"

namespace fq {
namespace {

constexpr uint32_t kMsThreads = 256;
constexpr uint32_t kMsWarps = kMsThreads / 32;
constexpr uint32_t kBarrierSpins = 1u << 24;

struct MsState {
    const int64_t *off;
    const uint32_t *cols;
    uint64_t n;
    const uint32_t *roots;
    uint32_t k;
    int32_t *depth;                  // [k][n]
    unsigned long long *seen, *frontier, *next;
    unsigned long long *flags;       // n/64 words
    uint32_t *queue;                 // [n]
    unsigned long long *degpre;      // [n + 1]
    unsigned long long *cta_cnt;     // [2 * grid]: flagged vertices, their degree sum
    unsigned int *bar;               // [2]: arrivals, generation
    unsigned int *abort_flag;
    unsigned long long *stats;       // [8]: levels, edges examined, reached pairs, reached edges x2
    Ctl *err;
    uint32_t max_levels;
    uint32_t bar_extra;   // test hook: arrivals a barrier waits for beyond the grid (0 normally)
    uint32_t spin_limit;  // polls before a barrier wait gives up
};

// fq_msbfs_barrier_test settings, read at each launch.
std::atomic<uint32_t> g_bar_extra{0}, g_bar_spins{0};

constexpr uint64_t kBarrierLimitNs = 2ull * 1000ull * 1000ull * 1000ull;  // a barrier wait gives up after 2 s

__device__ __forceinline__ uint64_t barrier_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_sync(const MsState &s, int *s_abort)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = s.bar + 1;
        const unsigned int my_gen = *gen;
        __threadfence();
        if (atomicAdd(s.bar, 1u) == gridDim.x - 1 + s.bar_extra) {
            s.bar[0] = 0;
            __threadfence();
            atomicAdd(s.bar + 1, 1u);
        } else {
            uint32_t spins = 0;
            const uint64_t t0 = barrier_ns();
            while (*gen == my_gen) {
                if (++spins > s.spin_limit || barrier_ns() - t0 > kBarrierLimitNs ||
                    *reinterpret_cast<volatile unsigned int *>(s.abort_flag)) {
                    if (atomicExch(s.abort_flag, 1u) == 0u) set_error(s.err, FQ_ETIMEOUT, kWhereBfs, 0);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        *s_abort = *reinterpret_cast<volatile unsigned int *>(s.abort_flag) != 0u;
    }
    __syncthreads();
    return *s_abort == 0;
}

__global__ void __launch_bounds__(kMsThreads) msbfs_kernel(MsState s)
{
    __shared__ unsigned long long sm[33];
    __shared__ unsigned long long s_red[2 * kMsWarps];
    __shared__ unsigned long long s_q0, s_e0, s_Q, s_E;
    __shared__ int s_abort;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t G = gridDim.x;
    const uint64_t nwords = (s.n + 63) / 64;
    // static vertex ownership in whole 64-vertex words: CTA b owns words [wb0, wb1)
    const uint64_t words_per = (nwords + G - 1) / G;
    const uint64_t wb0 = min(nwords, blockIdx.x * words_per), wb1 = min(nwords, wb0 + words_per);

    // level "-1": the roots arrive
    if (blockIdx.x == 0)
        for (uint32_t i = threadIdx.x; i < s.k; i += blockDim.x)
            if (s.roots[i] < s.n) atomicOr(&s.next[s.roots[i]], 1ull << i);
    if (!grid_sync(s, &s_abort)) return;

    for (uint32_t level = 0; level < s.max_levels; level++) {
        // ---- U: fold next into seen/frontier, depths, flags, per-CTA counts (one vertex per thread)
        unsigned long long cnt = 0, dsum = 0, pairs = 0, redges = 0;
        uint32_t *flags32 = reinterpret_cast<uint32_t *>(s.flags);
        const uint64_t v_end = min(wb1 * 64, s.n);
        for (uint64_t base = wb0 * 64; base < wb1 * 64; base += blockDim.x) {
            const uint64_t v = base + threadIdx.x;
            unsigned long long nw = 0, deg = 0;
            if (v < v_end) {
                const unsigned long long x = s.next[v];
                if (x) {
                    const unsigned long long sv = s.seen[v];
                    nw = x & ~sv;
                    s.seen[v] = sv | nw;
                    s.next[v] = 0ull;
                }
                if (nw || s.frontier[v]) s.frontier[v] = nw;
                if (nw) {
                    deg = (unsigned long long)(s.off[v + 1] - s.off[v]);
                    for (unsigned long long m = nw; m; m &= m - 1)
                        s.depth[(uint64_t)(__ffsll((long long)m) - 1) * s.n + v] = (int32_t)level;
                    pairs += __popcll(nw);
                    redges += (unsigned long long)__popcll(nw) * deg;
                }
            }
            const bool fl = nw && deg;
            const uint32_t m = __ballot_sync(0xffffffffu, fl);
            if (lane == 0 && base + 32u * warp < wb1 * 64) flags32[(base >> 5) + warp] = m;  // own words only
            if (fl) {
                cnt++;
                dsum += deg;
            }
        }
        cnt = warp_sum64(cnt);
        dsum = warp_sum64(dsum);
        pairs = warp_sum64(pairs);
        redges = warp_sum64(redges);
        if (lane == 0) {
            s_red[warp] = cnt;
            s_red[kMsWarps + warp] = dsum;
            if (pairs) {
                atomicAdd(&s.stats[2], pairs);
                atomicMax(&s.stats[0], (unsigned long long)level + 1);  // levels = deepest level + 1
            }
            if (redges) atomicAdd(&s.stats[3], redges);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long c = 0, d = 0;
            for (uint32_t i = 0; i < kMsWarps; i++) {
                c += s_red[i];
                d += s_red[kMsWarps + i];
            }
            s.cta_cnt[2 * blockIdx.x] = c;
            s.cta_cnt[2 * blockIdx.x + 1] = d;
        }
        if (!grid_sync(s, &s_abort)) return;

        // ---- Q: queue offsets from all CTAs' counts; write own flagged vertices + degree prefix
        if (warp == 0) {
            unsigned long long q0 = 0, e0 = 0, Q = 0, E = 0;
            for (uint64_t b = lane; b < G; b += 32) {
                const unsigned long long c = s.cta_cnt[2 * b], d = s.cta_cnt[2 * b + 1];
                if (b < blockIdx.x) {
                    q0 += c;
                    e0 += d;
                }
                Q += c;
                E += d;
            }
            q0 = warp_sum64(q0);
            e0 = warp_sum64(e0);
            Q = warp_sum64(Q);
            E = warp_sum64(E);
            if (lane == 0) {
                s_q0 = q0;
                s_e0 = e0;
                s_Q = Q;
                s_E = E;
            }
        }
        __syncthreads();
        const unsigned long long Q = s_Q, E = s_E;
        if (Q == 0) break;  // every CTA sees the same totals
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            s.stats[1] += E;
            s.degpre[Q] = E;
        }
        {
            unsigned long long qpos = s_q0, epos = s_e0;
            for (uint64_t c0 = wb0; c0 < wb1; c0 += blockDim.x) {
                const uint64_t w = c0 + threadIdx.x;
                const unsigned long long fl = w < wb1 ? s.flags[w] : 0ull;
                unsigned long long my_c = __popcll(fl), my_d = 0;
                for (unsigned long long m = fl; m; m &= m - 1) {
                    const uint64_t v = w * 64 + (__ffsll((long long)m) - 1);
                    my_d += (unsigned long long)(s.off[v + 1] - s.off[v]);
                }
                unsigned long long tc, td;
                const unsigned long long pc = cta_excl_scan64<kMsThreads>(my_c, sm, &tc);
                const unsigned long long pd = cta_excl_scan64<kMsThreads>(my_d, sm, &td);
                unsigned long long q = qpos + pc, e = epos + pd;
                for (unsigned long long m = fl; m; m &= m - 1) {
                    const uint64_t v = w * 64 + (__ffsll((long long)m) - 1);
                    s.queue[q] = (uint32_t)v;
                    s.degpre[q] = e;
                    q++;
                    e += (unsigned long long)(s.off[v + 1] - s.off[v]);
                }
                qpos += tc;
                epos += td;
            }
        }
        if (!grid_sync(s, &s_abort)) return;

        // ---- P: edge-balanced push over E edges
        {
            const uint64_t W = G * kMsWarps;
            const uint64_t gw = (uint64_t)blockIdx.x * kMsWarps + warp;
            const uint64_t e_lo = E * gw / W, e_hi = E * (gw + 1) / W;
            if (e_lo < e_hi) {
                // vertex of the first edge: largest j with degpre[j] <= e_lo (binary search)
                uint64_t lo = 0, hi = Q;
                while (hi - lo > 1) {
                    const uint64_t mid = (lo + hi) / 2;
                    if (s.degpre[mid] <= e_lo) lo = mid;
                    else hi = mid;
                }
                uint64_t j0 = lo;
                for (uint64_t e0 = e_lo; e0 < e_hi; e0 += 32) {
                    // stage 32 queue entries starting at j0 (each has >= 1 edge, so 32 edges
                    // starting at e0 fall inside them)
                    const uint64_t j = j0 + lane;
                    unsigned long long dp = ~0ull, fr = 0;
                    long long st = 0;
                    if (j < Q) {
                        dp = s.degpre[j];
                        const uint32_t v = s.queue[j];
                        st = s.off[v];
                        fr = s.frontier[v];
                    }
                    const uint64_t e = e0 + lane;
                    uint32_t J = 0;
#pragma unroll
                    for (uint32_t step = 16; step > 0; step >>= 1) {
                        const unsigned long long pc = __shfl_sync(0xffffffffu, dp, J + step);
                        if (pc <= e) J += step;
                    }
                    const unsigned long long dJ = __shfl_sync(0xffffffffu, dp, J);
                    const long long sJ = __shfl_sync(0xffffffffu, st, J);
                    const unsigned long long fJ = __shfl_sync(0xffffffffu, fr, J);
                    if (e < e_hi) {
                        const uint32_t w = s.cols[sJ + (long long)(e - dJ)];
                        const unsigned long long bits = fJ & ~s.seen[w];
                        if (bits) atomicOr(&s.next[w], bits);
                    }
                    // the next chunk starts at the vertex of edge e0 + 32
                    const uint32_t Jl = __shfl_sync(0xffffffffu, J, 31);
                    uint64_t nj = j0 + Jl;
                    if (nj + 1 < Q && s.degpre[nj + 1] <= e0 + 32) nj++;
                    j0 = nj;
                }
            }
        }
        if (!grid_sync(s, &s_abort)) return;
    }
}

}  // namespace
}  // namespace fq

using namespace fq;

namespace {
uint64_t al256m(uint64_t x) { return (x + 255u) / 256u * 256u; }
}  // namespace

extern "C" {

fq_status fq_msbfs_barrier_test(uint32_t extra_arrivals, uint32_t spin_limit)
{
    if (extra_arrivals > 1024u) return FQ_EINVAL;
    g_bar_extra.store(extra_arrivals);
    g_bar_spins.store(spin_limit);
    return FQ_OK;
}

uint64_t fq_msbfs_scratch_bytes(uint64_t n)
{
    const uint64_t G = 4096;  // upper bound on the cooperative grid
    uint64_t o = 256;         // Ctl
    o = al256m(o + 3 * 8 * n);          // seen, frontier, next
    o = al256m(o + 8 * ((n + 63) / 64));  // flags
    o = al256m(o + 4 * n);              // queue
    o = al256m(o + 8 * (n + 1));        // degree prefix
    o = al256m(o + 16 * G);             // per-CTA counts
    o = al256m(o + 64);                 // barrier + abort
    o = al256m(o + 64 * 4);             // roots
    o = al256m(o + 8 * 8);              // stats
    return o;
}

fq_status fq_bfs_run_multi(const int64_t *d_offsets, const uint32_t *d_cols, uint64_t n, const uint32_t *h_roots,
                               uint32_t k, int32_t *d_depth, void *d_scratch, uint64_t scratch_bytes,
                               fq_bfs_stats *h_stats, void *stream)
{
    if (!d_offsets || !d_cols || !h_roots || !d_depth || !d_scratch || k == 0 || k > 64 || n == 0 ||
        n > 0xffffffffull)
        return FQ_EINVAL;
    if (scratch_bytes < fq_msbfs_scratch_bytes(n)) return FQ_EINVAL;
    for (uint32_t i = 0; i < k; i++)
        if (h_roots[i] >= n) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *p = static_cast<uint8_t *>(d_scratch);
    MsState s{};
    uint64_t o = 0;
    s.err = reinterpret_cast<Ctl *>(p + o); o = 256;
    s.seen = reinterpret_cast<unsigned long long *>(p + o);
    s.frontier = s.seen + n;
    s.next = s.frontier + n;
    o = al256m(o + 3 * 8 * n);
    s.flags = reinterpret_cast<unsigned long long *>(p + o); o = al256m(o + 8 * ((n + 63) / 64));
    s.queue = reinterpret_cast<uint32_t *>(p + o); o = al256m(o + 4 * n);
    s.degpre = reinterpret_cast<unsigned long long *>(p + o); o = al256m(o + 8 * (n + 1));
    s.cta_cnt = reinterpret_cast<unsigned long long *>(p + o); o = al256m(o + 16 * 4096);
    s.bar = reinterpret_cast<unsigned int *>(p + o);
    s.abort_flag = s.bar + 2;
    o = al256m(o + 64);
    uint32_t *roots_d = reinterpret_cast<uint32_t *>(p + o); o = al256m(o + 64 * 4);
    s.stats = reinterpret_cast<unsigned long long *>(p + o); o = al256m(o + 64);
    s.off = d_offsets;
    s.cols = d_cols;
    s.n = n;
    s.roots = roots_d;
    s.k = k;
    s.depth = d_depth;
    s.max_levels = (uint32_t)std::min<uint64_t>(n + 1, 0x7fffffffu);
    s.bar_extra = g_bar_extra.load();
    const uint32_t spins = g_bar_spins.load();
    s.spin_limit = spins ? spins : kBarrierSpins;

    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FQ_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return FQ_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, msbfs_kernel, kMsThreads, 0) != cudaSuccess || per_sm <= 0)
        return FQ_ECUDA;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)sms * (uint64_t)per_sm, 4096);

    if (cudaMemsetAsync(p, 0, 256, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaMemsetAsync(s.seen, 0, 3 * 8 * n, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaMemsetAsync(s.bar, 0, 64, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaMemsetAsync(s.stats, 0, 64, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaMemsetAsync(d_depth, 0xff, 4ull * k * n, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaMemcpyAsync(roots_d, h_roots, 4ull * k, cudaMemcpyHostToDevice, st) != cudaSuccess) return FQ_ECUDA;
    // the status record must start at FQ_OK with an empty detail
    fq_device_status init{FQ_OK, 0, ~0ull};
    if (cudaMemcpyAsync(p, &init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess) return FQ_ECUDA;
    void *args[] = {&s};
    if (cudaLaunchCooperativeKernel((const void *)msbfs_kernel, grid, kMsThreads, args, 0, st) != cudaSuccess)
        return FQ_ECUDA;
    unsigned long long hs[8];
    fq_device_status rec;
    if (cudaMemcpyAsync(hs, s.stats, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaMemcpyAsync(&rec, p, sizeof(rec), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FQ_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FQ_ECUDA;
    if (h_stats) {
        memset(h_stats, 0, sizeof(*h_stats));
        h_stats->levels = (uint32_t)hs[0];
        h_stats->edges_examined = hs[1];
        h_stats->reached = hs[2];
        h_stats->reached_edges = hs[3] / 2;
        h_stats->kernel_launches[FQ_K_OTHER] = 1;
    }
    return rec.code;
}

}  // extern "C"
