// pred.cu -- the predecessor list of a finished BFS as one compressed container and back
// (fq_pred_encode / fq_pred_decode).
//
// The thesis reduces its predecessor list once per BFS, uncompressed (sec. 6.5, predecessor
// reduction), and its results chapter finds that this one exchange moves more bytes than all the
// compressed frontier exchanges of the run together.  Here the list is written as the level sets
// F_0 .. F_{L-1} (FQ streams: delta + binary packing in blocks of 128, sec. 5.2-5.3), followed by,
// for every level d >= 1, the index of each vertex's parent inside F_{d-1} (FR streams: frame of
// reference without differencing, Eq. 5-6).  An index needs at most bitlen(|F_{d-1}| - 1) bits,
// and a level set of dense ids packs to a few bits per id.
//
// Encode (7 launches for up to 256 levels, 3 more per further 8-bit digit of the level count):
//   pe_init     status record, level counters
//   pe_hist     per tile of 4096 vertices: digit counts of the level (the first pass also
//               validates depth and the root)
//   pe_plan     one CTA: scan of the tile counts, level offsets, stream sizes in blocks
//   pe_scatter  stable scatter by digit; the last pass records (level, index in level) per vertex
//   pe_widths   one warp per 128-value block: width and base; rank blocks first look up each
//               parent's index (and check that the parent is one level up)
//   pe_layout   one CTA: width scan, stream sizes, container header and offset table
//   pe_pack     one warp per block: stream headers, base and width tables, packed payloads
// Decode: pd_plan (header, table, stream headers), pd_widths, pd_scan, pd_unpack, pd_fill,
// pd_scatter (depth and parent of every reached vertex, duplicate and order checks).
#include <algorithm>

#include "codec_dev.cuh"
#include "fq_common.cuh"

namespace fq {
namespace {

constexpr uint32_t kPT = 256;                 // CTA size of the tile and block kernels
constexpr uint32_t kPWarps = kPT / 32;
constexpr uint32_t kSortItems = 4096;         // vertices (or positions) per sort tile
constexpr uint32_t kWarpItems = kSortItems / kPWarps;  // 512: 16 chunks of 32 per warp
constexpr uint32_t kRadix = 256;
constexpr uint32_t kMagicPl = 0x314C5046u;    // "FPL1"
constexpr uint32_t kMagicForP = 0x31505246u;  // "FRP1"
constexpr uint32_t kMagicForR = 0x31525246u;  // "FRR1"
constexpr uint32_t kWherePredEnc = 7, kWherePredDec = 8;
constexpr unsigned long long kNoPos = ~0ull;

struct PStream {
    unsigned long long off;   // byte offset of the stream in the container
    unsigned long long size;  // bytes
    uint32_t n;               // values
    uint32_t nb;              // 128-value blocks
    uint32_t blk0;            // first global block index
    uint32_t mode;            // kModePacked / kModeRaw
    uint32_t words;           // decode: payload words announced by the header
    uint32_t pad_;
};

struct PWork {
    Ctl *ctl;
    uint32_t *lo;              // [L + 1] level offsets into S (level counts first when L > 256)
    PStream *st;               // [2L]
    uint32_t *S;               // [n] reached vertices ordered by (level, id)
    uint32_t *S2;              // [n] radix ping-pong; decode: bitmap of vertices seen
    unsigned long long *lvpos; // [n] encode: level << 32 | index in level (kNoPos if unreached)
    uint32_t *R;               // [n] at a child's position in S: its parent's index in the level above
    uint32_t *hist;            // [256 * tiles] digit counts per tile, scanned in place
    uint32_t *bw;              // [nb_max + 1] block widths, scanned in place into payload prefixes
    uint32_t *bbase;           // [nb_max] block bases
    uint64_t n, L, tiles, nb_max;
};

uint64_t al256(uint64_t x) { return (x + 255u) / 256u * 256u; }

uint64_t nb_max_of(uint64_t n, uint64_t L) { return 2u * cdiv(n, kBlock) + 2u * L; }

uint64_t pred_layout(uint64_t n, uint64_t L, PWork *w, void *base)
{
    const uint64_t tiles = cdiv(n, kSortItems), nbm = nb_max_of(n, L);
    uint64_t o = 256;
    const uint64_t o_lo = o; o = al256(o + 4 * (L + 1));
    const uint64_t o_st = o; o = al256(o + sizeof(PStream) * 2 * L);
    const uint64_t o_s = o; o = al256(o + 4 * n);
    const uint64_t o_s2 = o; o = al256(o + 4 * n);
    const uint64_t o_lv = o; o = al256(o + 8 * n);
    const uint64_t o_r = o; o = al256(o + 4 * n);
    const uint64_t o_h = o; o = al256(o + 4 * kRadix * tiles);
    const uint64_t o_bw = o; o = al256(o + 4 * (nbm + 1));
    const uint64_t o_bb = o; o = al256(o + 4 * nbm);
    if (w && base) {
        uint8_t *p = static_cast<uint8_t *>(base);
        w->ctl = reinterpret_cast<Ctl *>(p);
        w->lo = reinterpret_cast<uint32_t *>(p + o_lo);
        w->st = reinterpret_cast<PStream *>(p + o_st);
        w->S = reinterpret_cast<uint32_t *>(p + o_s);
        w->S2 = reinterpret_cast<uint32_t *>(p + o_s2);
        w->lvpos = reinterpret_cast<unsigned long long *>(p + o_lv);
        w->R = reinterpret_cast<uint32_t *>(p + o_r);
        w->hist = reinterpret_cast<uint32_t *>(p + o_h);
        w->bw = reinterpret_cast<uint32_t *>(p + o_bw);
        w->bbase = reinterpret_cast<uint32_t *>(p + o_bb);
        w->n = n;
        w->L = L;
        w->tiles = tiles;
        w->nb_max = nbm;
    }
    return o;
}

uint32_t radix_passes(uint64_t L)
{
    uint32_t bits = 0;
    for (uint64_t x = L - 1; x; x >>= 1) bits++;
    return bits <= 8 ? 1u : (bits + 7u) / 8u;
}

uint32_t digits_of_pass(uint64_t L, uint32_t p) { return (uint32_t)std::min<uint64_t>(kRadix, ((L - 1) >> (8 * p)) + 1); }

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ void reset_ctl(Ctl *c)
{
    c->code = FQ_OK;
    c->where = 0;
    c->detail = ~0ull;
    c->mode = c->mode2 = kModeNone;
    c->fb_mode = kFbRaw;
    c->n = c->nb = c->popcount = c->total_b = c->out_bytes = c->fq_offset = c->out2_bytes = c->total_e = 0;
    c->tile_ticket = 0;
}

// Exclusive scan by one CTA of kScanThreads over f(0) .. f(count-1); g(i, prefix) sees each
// item's exclusive prefix.  Returns the total to every thread.
template <typename F, typename G>
__device__ unsigned long long cta_scan_fn(uint64_t count, F f, G g, unsigned long long *sm)
{
    const uint64_t chunk = (count + kScanThreads - 1) / kScanThreads;
    const uint64_t i0 = (uint64_t)threadIdx.x * chunk, i1 = min(count, i0 + chunk);
    unsigned long long local = 0, total = 0;
    for (uint64_t i = i0; i < i1; i++) local += f(i);
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t i = i0; i < i1; i++) {
        const unsigned long long x = f(i);
        g(i, run);
        run += x;
    }
    return total;
}

// Stream holding global block gb: the largest k < K with st[k].blk0 <= gb.
__device__ __forceinline__ uint32_t stream_of_block(const PStream *st, uint32_t K, uint32_t gb)
{
    uint32_t lo = 0, hi = K;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (st[mid].blk0 <= gb) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31u)) - 1u; }

// ---------------------------------------------------------------- encode

__global__ void pe_init(PWork w, uint32_t zero_counts)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_ctl(w.ctl);
    if (zero_counts)
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= w.L; i += (uint64_t)gridDim.x * blockDim.x)
            w.lo[i] = 0;
}

// Key of item i of a sort pass: the first pass walks vertex ids 0 .. n-1 (unreached ones drop
// out), later passes walk the previous pass's output.  Returns the level, or -1 for no item.
template <bool kFirst>
__device__ __forceinline__ int64_t sort_item(const PWork &w, const int32_t *depth, const uint32_t *in, uint64_t i,
                                             uint64_t items, uint32_t *v)
{
    if (i >= items) return -1;
    if (kFirst) {
        *v = (uint32_t)i;
        return depth[i];
    }
    *v = in[i];
    return depth[*v];
}

template <bool kFirst>
__global__ void __launch_bounds__(kPT) pe_hist(PWork w, const int32_t *depth, const uint32_t *parent, const uint32_t *in,
                                                 uint32_t shift, uint32_t digits, uint32_t count_levels)
{
    __shared__ uint32_t cnt[kRadix];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = !kFirst && w.ctl->code != FQ_OK;
    for (uint32_t i = threadIdx.x; i < kRadix; i += kPT) cnt[i] = 0;
    __syncthreads();
    if (s_abort) return;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t items = kFirst ? w.n : w.lo[w.L];
    const uint64_t base = (uint64_t)blockIdx.x * kSortItems + (uint64_t)warp * kWarpItems;
    for (uint32_t c = 0; c < kWarpItems / 32u; c++) {
        const uint64_t i = base + 32u * c + lane;
        uint32_t v = 0;
        int64_t d = sort_item<kFirst>(w, depth, in, i, items, &v);
        if (kFirst && i < items) {
            if (d < -1 || d >= (int64_t)w.L) {
                set_error(w.ctl, FQ_EINVAL, kWherePredEnc, i);
                d = -1;
            } else if (d == 0 && parent[i] != (uint32_t)i) {
                set_error(w.ctl, FQ_EINVAL, kWherePredEnc, i);
            }
        }
        const bool valid = d >= 0;
        const uint32_t act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint32_t dig = ((uint32_t)d >> shift) & (kRadix - 1u);
            const uint32_t peers = __match_any_sync(act, dig);
            if (lane == (uint32_t)__ffs(peers) - 1u) atomicAdd(&cnt[dig], (uint32_t)__popc(peers));
            if (kFirst && count_levels) {
                const uint32_t pl = __match_any_sync(act, (uint32_t)d);
                if (lane == (uint32_t)__ffs(pl) - 1u) atomicAdd(&w.lo[d], (uint32_t)__popc(pl));
            }
        }
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < digits; r += kPT) w.hist[(uint64_t)r * w.tiles + blockIdx.x] = cnt[r];
}

// Exclusive scan of the digit counts of a later pass.
__global__ void __launch_bounds__(kScanThreads) pe_scan(PWork w, uint32_t digits)
{
    __shared__ unsigned long long sm[33];
    if (w.ctl->code != FQ_OK) return;  // uniform: nothing else writes the record during this kernel
    cta_chunk_scan_u32<kScanThreads>(w.hist, w.hist, (uint64_t)digits * w.tiles, sm);
}

// First-pass scan, level offsets, checks, and the stream table's counts and block offsets.
__global__ void __launch_bounds__(kScanThreads) pe_plan(PWork w, uint32_t digits, uint32_t from_counts)
{
    __shared__ unsigned long long sm[33];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = w.ctl->code != FQ_OK;
    __syncthreads();
    if (s_abort) return;
    const uint64_t L = w.L;
    const unsigned long long reached = cta_chunk_scan_u32<kScanThreads>(w.hist, w.hist, (uint64_t)digits * w.tiles, sm);
    __syncthreads();
    if (from_counts) {
        cta_chunk_scan_u32<kScanThreads>(w.lo, w.lo, L, sm);
    } else {
        for (uint64_t d = threadIdx.x; d < L; d += kScanThreads) w.lo[d] = w.hist[d * w.tiles];
    }
    if (threadIdx.x == 0) w.lo[L] = (uint32_t)reached;
    __syncthreads();
    for (uint64_t d = threadIdx.x; d < L; d += kScanThreads) {
        const uint32_t c = w.lo[d + 1] - w.lo[d];
        if (c == 0 || (d == 0 && c != 1)) set_error(w.ctl, FQ_EINVAL, kWherePredEnc, d);
    }
    const uint64_t K = 2 * L - 1;
    auto count_of = [&](uint64_t k) -> uint32_t {
        const uint64_t d = k < L ? k : k - L + 1;
        return w.lo[d + 1] - w.lo[d];
    };
    const unsigned long long nb = cta_scan_fn(
        K, [&](uint64_t k) { return (unsigned long long)((count_of(k) + kBlock - 1) / kBlock); },
        [&](uint64_t k, unsigned long long pre) {
            PStream s{};
            s.n = count_of(k);
            s.nb = (s.n + kBlock - 1) / kBlock;
            s.blk0 = (uint32_t)pre;
            w.st[k] = s;
        },
        sm);
    if (threadIdx.x == 0) {
        w.ctl->n = reached;
        w.ctl->nb = nb;
    }
}

template <bool kFirst>
__global__ void __launch_bounds__(kPT) pe_scatter(PWork w, const int32_t *depth, const uint32_t *in, uint32_t *out,
                                                    uint32_t shift, uint32_t digits, uint32_t last)
{
    __shared__ uint32_t wc[kPWarps][kRadix];
    __shared__ int32_t s_key[kSortItems];
    __shared__ uint32_t s_v[kFirst ? 1 : kSortItems];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = w.ctl->code != FQ_OK;
    for (uint32_t i = threadIdx.x; i < kPWarps * kRadix; i += kPT) (&wc[0][0])[i] = 0;
    __syncthreads();
    if (s_abort) return;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t items = kFirst ? w.n : w.lo[w.L];
    const uint64_t tbase = (uint64_t)blockIdx.x * kSortItems;
    const uint32_t wofs = warp * kWarpItems;
    for (uint32_t c = 0; c < kWarpItems / 32u; c++) {  // the warp's digit counts, keys kept in shared memory
        const uint32_t li = wofs + 32u * c + lane;
        uint32_t v = 0;
        const int64_t d = sort_item<kFirst>(w, depth, in, tbase + li, items, &v);
        s_key[li] = (int32_t)(d >= 0 ? d : -1);
        if (!kFirst) s_v[li] = v;
        const bool valid = d >= 0;
        const uint32_t act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint32_t dig = ((uint32_t)d >> shift) & (kRadix - 1u);
            const uint32_t peers = __match_any_sync(act, dig);
            if (lane == (uint32_t)__ffs(peers) - 1u) wc[warp][dig] += (uint32_t)__popc(peers);
        }
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < digits; r += kPT) {  // warp bases: tile base + earlier warps of the tile
        uint32_t run = w.hist[(uint64_t)r * w.tiles + blockIdx.x];
        for (uint32_t q = 0; q < kPWarps; q++) {
            const uint32_t x = wc[q][r];
            wc[q][r] = run;
            run += x;
        }
    }
    __syncthreads();
    for (uint32_t c = 0; c < kWarpItems / 32u; c++) {
        const uint32_t li = wofs + 32u * c + lane;
        const int32_t d = s_key[li];
        const uint32_t v = kFirst ? (uint32_t)(tbase + li) : s_v[li];
        const bool valid = d >= 0;
        const uint32_t act = __ballot_sync(0xffffffffu, valid);
        uint32_t dig = 0, peers = 0, pos = 0;
        if (valid) {
            dig = ((uint32_t)d >> shift) & (kRadix - 1u);
            peers = __match_any_sync(act, dig);
            pos = wc[warp][dig] + (uint32_t)__popc(peers & lanemask_lt());
        }
        __syncwarp();
        if (valid && lane == (uint32_t)__ffs(peers) - 1u) wc[warp][dig] += (uint32_t)__popc(peers);
        __syncwarp();
        if (valid) {
            out[pos] = v;
            if (last) w.lvpos[v] = ((unsigned long long)(uint32_t)d << 32) | (pos - w.lo[d]);
        } else if (kFirst && tbase + li < items) {
            w.lvpos[tbase + li] = kNoPos;
        }
    }
}

// Block gb's values, 4 per lane (slots 4*lane .. 4*lane+3): level-set ids, or parent indices
// (looked up and written to R when `lookup`).  Returns the stream index; *cnt = valid slots.
__device__ __forceinline__ uint32_t block_values(const PWork &w, const uint32_t *parent, uint32_t gb, uint32_t lane,
                                                 bool lookup, uint32_t v[4], uint32_t *cnt, bool *is_rank)
{
    const uint32_t K = (uint32_t)(2 * w.L - 1);
    const uint32_t k = stream_of_block(w.st, K, gb);
    const PStream s = w.st[k];
    const uint32_t j = gb - s.blk0;
    const bool isR = k >= w.L;
    const uint32_t d = isR ? k - (uint32_t)w.L + 1u : k;
    const uint64_t g0 = (uint64_t)w.lo[d] + (uint64_t)kBlock * j;
    const uint32_t c = min(kBlock, s.n - kBlock * j);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint32_t i = 4u * lane + q;
        v[q] = 0;
        if (i >= c) continue;
        if (!isR) {
            v[q] = w.S[g0 + i];
        } else if (lookup) {
            const uint32_t child = w.S[g0 + i];
            const uint32_t p = parent[child];
            const unsigned long long x = p < w.n ? w.lvpos[p] : kNoPos;
            uint32_t r = 0;
            if (x == kNoPos || (uint32_t)(x >> 32) != d - 1u) set_error(w.ctl, FQ_EINVAL, kWherePredEnc, child);
            else r = (uint32_t)x;
            w.R[g0 + i] = r;
            v[q] = r;
        } else {
            v[q] = w.R[g0 + i];
        }
    }
    *cnt = c;
    *is_rank = isR;
    return k;
}

// Gaps of a level-set block (slot 0 and padding slots 0); ids are strictly increasing by construction.
__device__ __forceinline__ void block_gaps(const uint32_t v[4], uint32_t cnt, uint32_t lane, uint32_t g[4])
{
    const uint32_t prev = __shfl_up_sync(0xffffffffu, v[3], 1);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint32_t i = 4u * lane + q;
        const uint32_t p = q ? v[q - 1] : prev;
        g[q] = (i > 0 && i < cnt) ? v[q] - p - 1u : 0u;
    }
}

__global__ void __launch_bounds__(kPT) pe_widths(PWork w, const uint32_t *parent)
{
    if (w.ctl->code != FQ_OK) return;  // warp-level work only: no CTA barrier below
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t NB = w.ctl->nb;
    for (uint64_t gb = ((uint64_t)blockIdx.x * kPT + threadIdx.x) / 32u; gb < NB; gb += (uint64_t)gridDim.x * kPWarps) {
        uint32_t v[4], cnt;
        bool isR;
        block_values(w, parent, (uint32_t)gb, lane, true, v, &cnt, &isR);
        uint32_t width, base;
        if (!isR) {
            uint32_t g[4];
            block_gaps(v, cnt, lane, g);
            width = bitlen32(__reduce_max_sync(0xffffffffu, max(max(g[0], g[1]), max(g[2], g[3]))));
            base = __shfl_sync(0xffffffffu, v[0], 0);
        } else {
            uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (4u * lane + q < cnt) {
                    mn = min(mn, v[q]);
                    mx = max(mx, v[q]);
                }
            mn = __reduce_min_sync(0xffffffffu, mn);
            mx = __reduce_max_sync(0xffffffffu, mx);
            width = bitlen32(mx - mn);
            base = mn;
        }
        if (lane == 0) {
            w.bw[gb] = width;
            w.bbase[gb] = base;
        }
    }
}

__device__ __forceinline__ unsigned long long stream_bytes(const PStream &s, const uint32_t *P, uint32_t *mode)
{
    const unsigned long long sumb = P[s.blk0 + s.nb] - P[s.blk0];
    const unsigned long long packed = 16u + dpad16(5ull * s.nb) + 16u * sumb;
    const unsigned long long raw = 16u + dpad16(4ull * s.n);
    const bool is_packed = s.n > 0 && packed < raw;
    *mode = is_packed ? kModePacked : kModeRaw;
    return is_packed ? packed : raw;
}

__global__ void __launch_bounds__(kScanThreads) pe_layout(PWork w, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    __shared__ unsigned long long sm[33];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = w.ctl->code != FQ_OK;
    __syncthreads();
    if (s_abort) {
        if (threadIdx.x == 0) *out_bytes = 0;
        return;
    }
    const uint64_t NB = w.ctl->nb, L = w.L, K = 2 * L - 1;
    const unsigned long long sumb = cta_chunk_scan_u32<kScanThreads>(w.bw, w.bw, NB, sm);
    if (threadIdx.x == 0) w.bw[NB] = (uint32_t)sumb;
    __syncthreads();
    const unsigned long long head = 16u + 16u * L;
    const unsigned long long body = cta_scan_fn(
        K, [&](uint64_t k) { uint32_t m; return stream_bytes(w.st[k], w.bw, &m); },
        [&](uint64_t k, unsigned long long pre) {
            PStream s = w.st[k];
            s.size = stream_bytes(s, w.bw, &s.mode);
            s.off = head + pre;
            w.st[k] = s;
        },
        sm);
    const unsigned long long total = head + body;
    __syncthreads();
    if (threadIdx.x == 0) *out_bytes = total;
    if (total > cap) {
        if (threadIdx.x == 0) set_error(w.ctl, FQ_ENOSPC, kWherePredEnc, total);
        return;
    }
    if (threadIdx.x == 0) {
        uint32_t *h = reinterpret_cast<uint32_t *>(out);
        h[0] = kMagicPl;
        h[1] = (uint32_t)w.n;
        h[2] = (uint32_t)L;
        h[3] = (uint32_t)w.ctl->n;
    }
    unsigned long long *tab = reinterpret_cast<unsigned long long *>(out + 16);
    for (uint64_t k = threadIdx.x; k <= K; k += kScanThreads) tab[k] = k < K ? w.st[k].off : total;
}

__global__ void __launch_bounds__(kPT) pe_pack(PWork w, const uint32_t *parent, uint8_t *out)
{
    __shared__ uint32_t rows[kPWarps][4 * 32 + 4];
    if (w.ctl->code != FQ_OK) return;  // warp-level work only
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t NB = w.ctl->nb;
    for (uint64_t gb = ((uint64_t)blockIdx.x * kPT + threadIdx.x) / 32u; gb < NB; gb += (uint64_t)gridDim.x * kPWarps) {
        uint32_t v[4], cnt;
        bool isR;
        const uint32_t k = block_values(w, parent, (uint32_t)gb, lane, false, v, &cnt, &isR);
        const PStream s = w.st[k];
        const uint32_t j = (uint32_t)gb - s.blk0;
        uint8_t *dst = out + s.off;
        uint32_t *dw = reinterpret_cast<uint32_t *>(dst);
        if (s.mode == kModeRaw) {
            if (j == 0 && lane == 0) {
                dw[0] = isR ? kMagicForR : kMagicRaw;
                dw[1] = s.n;
                dw[2] = 0u;
                dw[3] = s.n;
            }
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (4u * lane + q < cnt) dw[4u + kBlock * j + 4u * lane + q] = v[q];
            if (j + 1 == s.nb) {  // zero words up to the 16-byte boundary
                const uint32_t padw = (uint32_t)((dpad16(4ull * s.n) - 4ull * s.n) / 4u);
                if (lane < padw) dw[4u + s.n + lane] = 0u;
            }
            continue;
        }
        const uint32_t nb = s.nb;
        if (j == 0) {
            if (lane == 0) {
                dw[0] = isR ? kMagicForP : kMagicPacked;
                dw[1] = s.n;
                dw[2] = nb;
                dw[3] = 4u * (w.bw[s.blk0 + nb] - w.bw[s.blk0]);
            }
            const uint32_t t0 = 16u + 5u * nb, t1 = (uint32_t)(16u + dpad16(5ull * nb));
            if (t0 + lane < t1) dst[t0 + lane] = 0u;
        }
        const uint32_t b = w.bw[gb + 1] - w.bw[gb];
        const uint32_t base = w.bbase[gb];
        if (lane == 0) {
            dw[4u + j] = base;
            dst[16u + 4u * nb + j] = (uint8_t)b;
        }
        uint32_t g[4];
        if (!isR) {
            block_gaps(v, cnt, lane, g);
        } else {
#pragma unroll
            for (int q = 0; q < 4; q++) g[q] = (4u * lane + q < cnt) ? v[q] - base : 0u;
        }
        uint32_t words[4];
        pack_block_words(g, b, rows[warp], lane, words);
        uint8_t *pk = dst + 16u + dpad16(5ull * nb) + 16ull * (w.bw[gb] - w.bw[s.blk0]);
        store_block_words(pk, words, b, lane, 0ull, ~0ull);
    }
}

// ---------------------------------------------------------------- decode

__device__ __forceinline__ unsigned long long ld_u64(const uint8_t *p) { return *reinterpret_cast<const unsigned long long *>(p); }

// Header, offset table and stream headers; level offsets and block offsets.
__global__ void __launch_bounds__(kScanThreads) pd_plan(PWork w, const uint8_t *in, uint64_t in_bytes)
{
    __shared__ unsigned long long sm[33];
    __shared__ int s_bad;
    __shared__ uint32_t s_L, s_reached;
    Ctl *c = w.ctl;
    if (threadIdx.x == 0) {
        reset_ctl(c);
        s_bad = 0;
        uint32_t magic = 0, n = 0, L = 0, reached = 0;
        if (in_bytes >= 16u) {
            magic = ld_u32(in);
            n = ld_u32(in + 4);
            L = ld_u32(in + 8);
            reached = ld_u32(in + 12);
        }
        if (in_bytes < 16u || magic != kMagicPl || n != w.n || L == 0 || reached > n || reached == 0 ||
            in_bytes < 16ull + 16ull * L) {
            set_error(c, FQ_ECORRUPT, kWherePredDec, 0);
            s_bad = 1;
        } else if (L > w.L) {
            set_error(c, FQ_ENOSPC, kWherePredDec, L);
            s_bad = 1;
        }
        s_L = L;
        s_reached = reached;
    }
    __syncthreads();
    if (s_bad) return;
    const uint64_t L = s_L, K = 2 * L - 1;
    const uint8_t *tab = in + 16;
    for (uint64_t k = threadIdx.x; k < K; k += kScanThreads) {
        const unsigned long long o0 = ld_u64(tab + 8 * k), o1 = ld_u64(tab + 8 * (k + 1));
        bool ok = (o0 & 15u) == 0 && o1 >= o0 + 16u && o1 <= in_bytes;
        if (k == 0) ok = ok && o0 == 16u + 16u * L;
        if (k + 1 == K) ok = ok && o1 == in_bytes;
        if (ok) {
            const uint8_t *h = in + o0;
            const uint32_t magic = ld_u32(h), n = ld_u32(h + 4), nb = ld_u32(h + 8), words = ld_u32(h + 12);
            const bool isR = k >= L;
            const unsigned long long size = o1 - o0;
            PStream s{};
            s.off = o0;
            s.size = size;
            s.n = n;
            s.nb = (uint32_t)(((unsigned long long)n + kBlock - 1) / kBlock);
            s.words = words;
            if (n == 0) {
                ok = false;
            } else if (magic == (isR ? kMagicForP : kMagicPacked)) {
                s.mode = kModePacked;
                ok = nb == s.nb && (words & 3u) == 0 && size == 16ull + dpad16(5ull * nb) + 4ull * words;
            } else if (magic == (isR ? kMagicForR : kMagicRaw)) {
                s.mode = kModeRaw;
                ok = nb == 0 && words == n && size == 16ull + dpad16(4ull * n);
            } else {
                ok = false;
            }
            w.st[k] = s;
        }
        if (!ok) {
            set_error(c, FQ_ECORRUPT, kWherePredDec, k);
            s_bad = 1;
        }
    }
    __syncthreads();
    if (s_bad) return;
    for (uint64_t d = 1 + threadIdx.x; d < L; d += kScanThreads)
        if (w.st[L + d - 1].n != w.st[d].n) {
            set_error(c, FQ_ECORRUPT, kWherePredDec, L + d - 1);
            s_bad = 1;
        }
    if (threadIdx.x == 0 && w.st[0].n != 1) {
        set_error(c, FQ_ECORRUPT, kWherePredDec, 0);
        s_bad = 1;
    }
    const unsigned long long reached = cta_scan_fn(
        L, [&](uint64_t d) { return (unsigned long long)w.st[d].n; },
        [&](uint64_t d, unsigned long long pre) { w.lo[d] = (uint32_t)pre; }, sm);
    if (reached != s_reached) {
        if (threadIdx.x == 0) set_error(c, FQ_ECORRUPT, kWherePredDec, 0);
        return;  // uniform: every thread sees the same total
    }
    __syncthreads();
    if (s_bad) return;
    const unsigned long long nb = cta_scan_fn(
        K, [&](uint64_t k) { return (unsigned long long)w.st[k].nb; },
        [&](uint64_t k, unsigned long long pre) { w.st[k].blk0 = (uint32_t)pre; }, sm);
    if (threadIdx.x == 0) {
        w.lo[L] = (uint32_t)reached;
        c->n = reached;
        c->nb = nb;
        c->mode = (uint32_t)L;  // the container's level count, for the later kernels
    }
}

__global__ void __launch_bounds__(kPT) pd_widths(PWork w, const uint8_t *in)
{
    if (w.ctl->code != FQ_OK) return;
    const uint32_t K = 2u * w.ctl->mode - 1u;
    const uint64_t NB = w.ctl->nb;
    for (uint64_t gb = (uint64_t)blockIdx.x * kPT + threadIdx.x; gb < NB; gb += (uint64_t)gridDim.x * kPT) {
        const uint32_t k = stream_of_block(w.st, K, (uint32_t)gb);
        const PStream s = w.st[k];
        uint32_t b = 0;
        if (s.mode == kModePacked) {
            b = in[s.off + 16u + 4ull * s.nb + (gb - s.blk0)];
            if (b > 32u) {
                set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, k);
                b = 0;
            }
        }
        w.bw[gb] = b;
    }
}

__global__ void __launch_bounds__(kScanThreads) pd_scan(PWork w)
{
    __shared__ unsigned long long sm[33];
    if (w.ctl->code != FQ_OK) return;  // uniform: pd_widths has finished
    const uint64_t NB = w.ctl->nb, K = 2u * w.ctl->mode - 1u;
    const unsigned long long total = cta_chunk_scan_u32<kScanThreads>(w.bw, w.bw, NB, sm);
    if (threadIdx.x == 0) w.bw[NB] = (uint32_t)total;
    __syncthreads();
    for (uint64_t k = threadIdx.x; k < K; k += kScanThreads) {
        const PStream s = w.st[k];
        if (s.mode == kModePacked && 4ull * (w.bw[s.blk0 + s.nb] - w.bw[s.blk0]) != s.words)
            set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, k);
    }
}

__global__ void __launch_bounds__(kPT) pd_unpack(PWork w, const uint8_t *in)
{
    __shared__ uint32_t rows[kPWarps][4 * 32 + 4];
    if (w.ctl->code != FQ_OK) return;  // warp-level work only
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t L = w.ctl->mode, K = 2u * L - 1u;
    const uint64_t NB = w.ctl->nb;
    uint32_t *row = rows[warp];
    for (uint64_t gb = ((uint64_t)blockIdx.x * kPT + threadIdx.x) / 32u; gb < NB; gb += (uint64_t)gridDim.x * kPWarps) {
        const uint32_t k = stream_of_block(w.st, K, (uint32_t)gb);
        const PStream s = w.st[k];
        const uint32_t j = (uint32_t)gb - s.blk0;
        const bool isR = k >= L;
        const uint32_t d = isR ? k - L + 1u : k;
        const uint64_t g0 = (uint64_t)w.lo[d] + (uint64_t)kBlock * j;
        const uint32_t cnt = min(kBlock, s.n - kBlock * j);
        const uint32_t above = isR ? w.lo[d] - w.lo[d - 1] : 0u;  // size of level d - 1
        uint32_t *dstv = isR ? w.R : w.S;
        const uint8_t *src = in + s.off;
        bool ok = true;
        uint32_t out[4];
        if (s.mode == kModeRaw) {
            const uint32_t *vw = reinterpret_cast<const uint32_t *>(src + 16) + (uint64_t)kBlock * j;
#pragma unroll
            for (int q = 0; q < 4; q++) out[q] = (4u * lane + q < cnt) ? vw[4u * lane + q] : 0u;
            if (j + 1 == s.nb) {
                const uint32_t padw = (uint32_t)((dpad16(4ull * s.n) - 4ull * s.n) / 4u);
                if (lane < padw && reinterpret_cast<const uint32_t *>(src + 16)[s.n + lane] != 0u) ok = false;
            }
        } else {
            const uint32_t nb = s.nb;
            if (j == 0) {
                const uint32_t t0 = 16u + 5u * nb, t1 = (uint32_t)(16u + dpad16(5ull * nb));
                if (t0 + lane < t1 && src[t0 + lane] != 0u) ok = false;
            }
            const uint32_t b = w.bw[gb + 1] - w.bw[gb];
            const uint32_t base = ld_u32(src + 16u + 4u * j);
            const uint32_t *pk = reinterpret_cast<const uint32_t *>(src + 16u + dpad16(5ull * nb) +
                                                                   16ull * (w.bw[gb] - w.bw[s.blk0]));
            // stage the block's 4b words, then three zero words past them for the slot reader
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                const uint32_t i = lane + 32u * q;
                row[i] = i < 4u * b ? pk[i] : 0u;
            }
            if (lane < 4u) row[128u + lane] = 0u;
            __syncwarp();
            uint32_t g[4];
            extract_slots(row, b, lane, g);
            __syncwarp();
            if (!isR) {
                unsigned long long last;
                ok = scan_slots(g, base, j, s.n, lane, out, &last) && ok;
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const bool valid = 4u * lane + q < cnt;
                    const unsigned long long x = (unsigned long long)base + g[q];
                    if ((!valid && g[q] != 0u) || (valid && x > 0xffffffffull)) ok = false;
                    out[q] = (uint32_t)x;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = 4u * lane + q;
            if (i < cnt) {
                if (isR && out[q] >= above) ok = false;
                dstv[g0 + i] = out[q];
            }
        }
        if (!ok) set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, k);
    }
}

__global__ void __launch_bounds__(kPT) pd_fill(PWork w, int32_t *depth, uint32_t *parent)
{
    if (w.ctl->code != FQ_OK) return;  // a stream that failed validation leaves the outputs untouched
    const uint64_t stride = (uint64_t)gridDim.x * kPT;
    for (uint64_t v = (uint64_t)blockIdx.x * kPT + threadIdx.x; v < w.n; v += stride) {
        depth[v] = -1;
        parent[v] = 0xffffffffu;
    }
    for (uint64_t i = (uint64_t)blockIdx.x * kPT + threadIdx.x; i < (w.n + 31) / 32; i += stride) w.S2[i] = 0u;
}

__global__ void __launch_bounds__(kPT) pd_scatter(PWork w, int32_t *depth, uint32_t *parent)
{
    if (w.ctl->code != FQ_OK) return;
    const uint32_t L = w.ctl->mode;
    const uint64_t reached = w.ctl->n;
    for (uint64_t g = (uint64_t)blockIdx.x * kPT + threadIdx.x; g < reached; g += (uint64_t)gridDim.x * kPT) {
        uint32_t lo = 0, hi = L;  // level: largest d with lo[d] <= g
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (w.lo[mid] <= g) lo = mid;
            else hi = mid;
        }
        const uint32_t d = lo;
        const uint32_t v = w.S[g];
        if (v >= w.n || (g > w.lo[d] && w.S[g - 1] >= v)) {
            set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, g);
            continue;
        }
        const uint32_t bit = 1u << (v & 31u);
        if (atomicOr(&w.S2[v >> 5], bit) & bit) {  // the vertex already appeared at some level
            set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, g);
            continue;
        }
        depth[v] = (int32_t)d;
        parent[v] = d == 0 ? v : w.S[w.lo[d - 1] + w.R[g]];
    }
}

uint32_t grid_for(uint64_t items, uint64_t per_cta)
{
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(cdiv(items, per_cta), (uint64_t)16 * num_sms()));
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

}  // namespace
}  // namespace fq

using namespace fq;

extern "C" {

uint64_t fq_pred_bound(uint64_t n, uint32_t levels) { return 16u + 72ull * levels + 8ull * n; }

uint64_t fq_pred_workspace_bytes(uint64_t n, uint32_t levels) { return pred_layout(n, levels ? levels : 1, nullptr, nullptr); }

fq_status fq_pred_encode(const int32_t *d_depth, const uint32_t *d_parent, uint64_t n, uint32_t levels, uint8_t *d_out,
                         uint64_t cap, uint64_t *d_out_bytes, void *d_work, uint64_t work_bytes, void *stream)
{
    if (!d_depth || !d_parent || !d_out || !d_out_bytes || !d_work) return FQ_EINVAL;
    if (n == 0 || n > 0xffffffffull || levels == 0 || levels > n) return FQ_EINVAL;
    if (!aligned16(d_out) || !aligned16(d_work) || !aligned4(d_depth) || !aligned4(d_parent)) return FQ_EINVAL;
    if (work_bytes < fq_pred_workspace_bytes(n, levels)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PWork w{};
    pred_layout(n, levels, &w, d_work);
    const uint32_t P = radix_passes(levels);
    const uint32_t tiles = (uint32_t)w.tiles;
    const uint32_t multi = levels > kRadix;
    pe_init<<<grid_for((uint64_t)levels + 1, kPT), kPT, 0, st>>>(w, multi);
    const uint32_t D0 = digits_of_pass(levels, 0);
    pe_hist<true><<<tiles, kPT, 0, st>>>(w, d_depth, d_parent, nullptr, 0u, D0, multi);
    pe_plan<<<1, kScanThreads, 0, st>>>(w, D0, multi);
    // pass p writes S when P - 1 - p is even, so that the last pass lands in S
    uint32_t *bufs[2] = {w.S, w.S2};
    const uint32_t *prev = nullptr;
    for (uint32_t p = 0; p < P; p++) {
        uint32_t *dst = bufs[(P - 1 - p) & 1u];
        const uint32_t D = digits_of_pass(levels, p), last = p + 1 == P;
        if (p == 0) {
            pe_scatter<true><<<tiles, kPT, 0, st>>>(w, d_depth, nullptr, dst, 0u, D, last);
        } else {
            pe_hist<false><<<tiles, kPT, 0, st>>>(w, d_depth, nullptr, prev, 8u * p, D, 0u);
            pe_scan<<<1, kScanThreads, 0, st>>>(w, D);
            pe_scatter<false><<<tiles, kPT, 0, st>>>(w, d_depth, prev, dst, 8u * p, D, last);
        }
        prev = dst;
    }
    const uint32_t gridb = grid_for(w.nb_max, kPWarps);
    pe_widths<<<gridb, kPT, 0, st>>>(w, d_parent);
    pe_layout<<<1, kScanThreads, 0, st>>>(w, d_out, cap, d_out_bytes);
    pe_pack<<<gridb, kPT, 0, st>>>(w, d_parent, d_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e, __LINE__);
        return FQ_ECUDA;
    }
    return FQ_OK;
}

fq_status fq_pred_decode(const uint8_t *d_in, uint64_t in_bytes, int32_t *d_depth, uint32_t *d_parent, uint64_t n,
                         uint32_t max_levels, void *d_work, uint64_t work_bytes, void *stream)
{
    if (!d_in || !d_depth || !d_parent || !d_work) return FQ_EINVAL;
    if (n == 0 || n > 0xffffffffull || max_levels == 0) return FQ_EINVAL;
    if (!aligned16(d_in) || !aligned16(d_work) || !aligned4(d_depth) || !aligned4(d_parent)) return FQ_EINVAL;
    if (work_bytes < fq_pred_workspace_bytes(n, max_levels)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PWork w{};
    pred_layout(n, max_levels, &w, d_work);
    const uint32_t gridb = grid_for(w.nb_max, kPWarps);
    pd_plan<<<1, kScanThreads, 0, st>>>(w, d_in, in_bytes);
    pd_widths<<<grid_for(w.nb_max, kPT), kPT, 0, st>>>(w, d_in);
    pd_scan<<<1, kScanThreads, 0, st>>>(w);
    pd_unpack<<<gridb, kPT, 0, st>>>(w, d_in);
    pd_fill<<<grid_for(n, kPT), kPT, 0, st>>>(w, d_depth, d_parent);
    pd_scatter<<<grid_for(n, kPT), kPT, 0, st>>>(w, d_depth, d_parent);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e, __LINE__);
        return FQ_ECUDA;
    }
    return FQ_OK;
}

}  // extern "C"
