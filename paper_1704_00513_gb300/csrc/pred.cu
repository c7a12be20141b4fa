// pred.cu -- the predecessor list of a finished BFS as one compressed container and back
// (fq_pred_encode / fq_pred_decode).
//
// The thesis reduces its predecessor list once per BFS, uncompressed (sec. 4.1.4, the
// predecessor list bitmap), and its results chapter finds that this one exchange moves more
// bytes than all the compressed frontier exchanges of the run together.  Here the list is
// written as the level sets
// F_0 .. F_{L-1} (FQ streams: delta + binary packing in blocks of 128, sec. 5.1, 5.3), followed by,
// for every level d >= 1, the index of each vertex's parent inside F_{d-1} (FR streams: frame of
// reference without differencing, Eq. 5-6).  An index needs at most bitlen(|F_{d-1}| - 1) bits,
// and a level set of dense ids packs to a few bits per id.
//
// Encode (8 launches for up to 256 levels, 4 more per further 8-bit digit of the level count):
//   pe_init     status record, level counters
//   pe_hist     per tile of 4096 vertices: digit counts of the level (the first pass also
//               validates depth and the root)
//   pe_rowscan  one CTA per digit: that digit's tile counts scanned
//   pe_plan     one CTA: digit bases, level offsets, checks, stream sizes in blocks
//   pe_scatter  stable scatter by digit; the last pass records (level, index in level) per vertex
//   pe_widths   tiles of 64 blocks, 8 per warp: width and base of each block and in-tile
//               prefixes; rank blocks first look up each parent's index (and check that the
//               parent is one level up)
//   pe_layout   one CTA: tile prefixes, stream sizes, container header and offset table
//   pe_pack     8 blocks per warp: stream headers, base and width tables, packed payloads
// Decode: pd_plan (header, table, stream headers), pd_widths, pd_scan (tile prefixes, payload
// sizes), pd_unpack; then, for a workspace of at most 128 levels, pd_chunks (where each level
// enters each chunk of 4096 ids) and pd_build (each chunk's depth and parent assembled in shared
// memory and written once, with the order and duplicate checks); for more levels pd_fill,
// pd_scatter (depth and parent of every reached vertex) and pd_verify (ids increasing within a
// level, no vertex at two levels).
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
constexpr uint32_t kBW = 8;                   // 128-value blocks per warp per tile
constexpr uint32_t kBT = kPWarps * kBW;       // 64 blocks per tile
constexpr uint32_t kPosPerThread = 8;         // positions per thread in the decode scatter and check
constexpr uint32_t kPosTile = kPT * kPosPerThread;
constexpr uint32_t kVmIds = 4096;             // vertex ids per chunk of the vertex-ordered decode
constexpr uint32_t kVmLevels = 128;           // most levels the vertex-ordered decode takes
constexpr uint32_t kMagicPl = 0x314C5046u;    // "FPL1"
constexpr uint32_t kMagicForP = 0x31505246u;  // "FRP1"
constexpr uint32_t kMagicForR = 0x31525246u;  // "FRR1"
constexpr uint32_t kWherePredEnc = 7, kWherePredDec = 8;
constexpr uint32_t kNoPos = 0xffffffffu;  // position of an unreached vertex

struct PStream {
    unsigned long long off;   // byte offset of the stream in the container
    unsigned long long size;  // bytes
    uint32_t n;               // values
    uint32_t nb;              // 128-value blocks
    uint32_t blk0;            // first global block index
    uint32_t mode;            // kModePacked / kModeRaw
    uint32_t words;           // decode: payload words announced by the header
    uint32_t pstart;          // payload units (16 bytes) of all blocks before the stream's first one
};

struct PWork {
    Ctl *ctl;
    uint32_t *lo;              // [L + 1] level offsets into S (level counts first when L > 256)
    PStream *st;               // [2L]
    uint32_t *S;               // [n] reached vertices ordered by (level, id)
    uint32_t *S2;              // [n] radix ping-pong; decode: bitmap of vertices seen
    uint32_t *gpos;            // [n] encode: the vertex's position in S (kNoPos if unreached); its level
                               // is the d with lo[d] <= position < lo[d+1], its index position - lo[d]
    uint32_t *R;               // [n] at a child's position in S: its parent's index in the level above
    uint32_t *hist;            // [256 * tiles] digit counts per tile; each digit's row scanned in place
    uint32_t *rsum;            // [256] digit totals
    uint32_t *dbase;           // [256] first position of each digit
    uint32_t *bw;              // [nb_max] block widths (payload units of 16 bytes)
    uint32_t *lpre;            // [nb_max] payload units before the block within its tile of 64 blocks
    uint32_t *tsum;            // [nt_max + 1] tile totals, scanned in place into tile prefixes
    uint32_t *bbase;           // [nb_max] block bases
    uint32_t *cstart;          // decode, L <= kVmLevels: [L][nch + 1] first position of each id chunk per level
    uint64_t n, L, tiles, nb_max, nch;
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
    const uint64_t o_lv = o; o = al256(o + 4 * n);
    const uint64_t o_r = o; o = al256(o + 4 * n);
    const uint64_t o_h = o; o = al256(o + 4 * kRadix * tiles);
    const uint64_t o_rs = o; o = al256(o + 4 * kRadix);
    const uint64_t o_db = o; o = al256(o + 4 * kRadix);
    const uint64_t o_bw = o; o = al256(o + 4 * nbm);
    const uint64_t o_lp = o; o = al256(o + 4 * nbm);
    const uint64_t o_ts = o; o = al256(o + 4 * (cdiv(nbm, kBT) + 1));
    const uint64_t o_bb = o; o = al256(o + 4 * nbm);
    const uint64_t nch = cdiv(n, kVmIds);
    const uint64_t o_cs = o; o = al256(o + (L <= kVmLevels ? 4 * L * (nch + 1) : 0));
    if (w && base) {
        uint8_t *p = static_cast<uint8_t *>(base);
        w->ctl = reinterpret_cast<Ctl *>(p);
        w->lo = reinterpret_cast<uint32_t *>(p + o_lo);
        w->st = reinterpret_cast<PStream *>(p + o_st);
        w->S = reinterpret_cast<uint32_t *>(p + o_s);
        w->S2 = reinterpret_cast<uint32_t *>(p + o_s2);
        w->gpos = reinterpret_cast<uint32_t *>(p + o_lv);
        w->R = reinterpret_cast<uint32_t *>(p + o_r);
        w->hist = reinterpret_cast<uint32_t *>(p + o_h);
        w->rsum = reinterpret_cast<uint32_t *>(p + o_rs);
        w->dbase = reinterpret_cast<uint32_t *>(p + o_db);
        w->bw = reinterpret_cast<uint32_t *>(p + o_bw);
        w->lpre = reinterpret_cast<uint32_t *>(p + o_lp);
        w->tsum = reinterpret_cast<uint32_t *>(p + o_ts);
        w->bbase = reinterpret_cast<uint32_t *>(p + o_bb);
        w->cstart = reinterpret_cast<uint32_t *>(p + o_cs);
        w->nch = nch;
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

// Keys of a warp's kWarpItems sort items, all loads issued first: the first pass walks vertex
// ids 0 .. n-1 (unreached ones drop out), later passes the previous pass's output.  key = level,
// or -1 for no item; v = the vertex.
constexpr uint32_t kChunks = kWarpItems / 32u;

template <bool kFirst>
__device__ __forceinline__ void load_keys(const int32_t *depth, const uint32_t *in, uint64_t base, uint64_t items,
                                          uint32_t lane, int32_t key[kChunks], uint32_t v[kChunks])
{
#pragma unroll
    for (uint32_t c = 0; c < kChunks; c++) {
        const uint64_t i = base + 32u * c + lane;
        v[c] = kFirst ? (uint32_t)i : (i < items ? in[i] : 0u);
    }
#pragma unroll
    for (uint32_t c = 0; c < kChunks; c++) {
        const uint64_t i = base + 32u * c + lane;
        key[c] = i < items ? depth[kFirst ? i : (uint64_t)v[c]] : -1;
    }
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
    int32_t key[kChunks];
    uint32_t vv[kChunks];
    load_keys<kFirst>(depth, in, base, items, lane, key, vv);
#pragma unroll
    for (uint32_t c = 0; c < kChunks; c++) {
        const uint64_t i = base + 32u * c + lane;
        int32_t d = key[c];
        if (kFirst && i < items) {
            if (d < -1 || (int64_t)d >= (int64_t)w.L) {
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

// One CTA per digit: that digit's counts over all tiles, scanned in place; the digit's total.
__global__ void __launch_bounds__(kScanThreads) pe_rowscan(PWork w)
{
    __shared__ unsigned long long sm[33];
    if (w.ctl->code != FQ_OK) return;  // uniform: nothing writes the record during this kernel
    const unsigned long long total =
        cta_chunk_scan_u32<kScanThreads>(w.hist + (uint64_t)blockIdx.x * w.tiles, w.hist + (uint64_t)blockIdx.x * w.tiles,
                                         w.tiles, sm);
    if (threadIdx.x == 0) w.rsum[blockIdx.x] = (uint32_t)total;
}

// Digit bases of a later pass.
__global__ void __launch_bounds__(kScanThreads) pe_dscan(PWork w, uint32_t digits)
{
    __shared__ unsigned long long sm[33];
    if (w.ctl->code != FQ_OK) return;
    cta_chunk_scan_u32<kScanThreads>(w.rsum, w.dbase, digits, sm);
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
    const unsigned long long reached = cta_chunk_scan_u32<kScanThreads>(w.rsum, w.dbase, digits, sm);
    __syncthreads();
    if (from_counts) {
        cta_chunk_scan_u32<kScanThreads>(w.lo, w.lo, L, sm);
    } else {
        for (uint64_t d = threadIdx.x; d < L; d += kScanThreads) w.lo[d] = w.dbase[d];
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
    int32_t key[kChunks];
    uint32_t vv[kChunks];
    load_keys<kFirst>(depth, in, tbase + wofs, items, lane, key, vv);
#pragma unroll
    for (uint32_t c = 0; c < kChunks; c++) {  // the warp's digit counts, keys kept in shared memory
        const uint32_t li = wofs + 32u * c + lane;
        const int32_t d = key[c] >= 0 ? key[c] : -1;
        s_key[li] = d;
        if (!kFirst) s_v[li] = vv[c];
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
        uint32_t run = w.dbase[r] + w.hist[(uint64_t)r * w.tiles + blockIdx.x];
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
            if (last) w.gpos[v] = pos;
        } else if (kFirst && tbase + li < items) {
            w.gpos[tbase + li] = kNoPos;
        }
    }
}

// One 128-value block of a tile, as seen by a warp: lane i < kBW computes the record of block
// gb0 + i; bcast() hands record i to every lane.
struct BInfo {
    unsigned long long g0;  // position of the block's first value in S (level sets) or R (ranks)
    uint32_t cnt;           // values in the block; 0 = no block
    uint32_t k;             // stream
    uint32_t d;             // level
    uint32_t isR;           // rank (FR) stream
};

__device__ __forceinline__ BInfo lane_block_info(const PWork &w, uint32_t L, uint64_t gb0, uint64_t NB, uint32_t lane)
{
    BInfo b{};
    const uint64_t gb = gb0 + lane;
    if (lane < kBW && gb < NB) {
        const uint32_t k = stream_of_block(w.st, 2u * L - 1u, (uint32_t)gb);
        const uint32_t n = w.st[k].n, j = (uint32_t)gb - w.st[k].blk0;
        b.isR = k >= L;
        b.d = b.isR ? k - L + 1u : k;
        b.g0 = (unsigned long long)w.lo[b.d] + (unsigned long long)kBlock * j;
        b.cnt = min(kBlock, n - kBlock * j);
        b.k = k;
    }
    return b;
}

__device__ __forceinline__ BInfo bcast(const BInfo &b, uint32_t i)
{
    BInfo r;
    r.g0 = __shfl_sync(0xffffffffu, b.g0, i);
    r.cnt = __shfl_sync(0xffffffffu, b.cnt, i);
    r.k = __shfl_sync(0xffffffffu, b.k, i);
    r.d = __shfl_sync(0xffffffffu, b.d, i);
    r.isR = __shfl_sync(0xffffffffu, b.isR, i);
    return r;
}

// Payload units (16 bytes) of all blocks before global block x: tile prefix + in-tile prefix.
__device__ __forceinline__ uint32_t prefix_at(const PWork &w, uint64_t x, uint64_t NB, uint64_t NT)
{
    return x < NB ? w.tsum[x / kBT] + w.lpre[x] : w.tsum[NT];
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

// In-tile exclusive prefix of the tile's 64 widths (s_w) by warp 0, and the tile's total.
__device__ __forceinline__ void tile_prefix(const PWork &w, const uint32_t *s_w, uint64_t t, uint64_t NB, uint32_t lane)
{
    const uint32_t a = s_w[2u * lane], b = s_w[2u * lane + 1u];
    const uint32_t incl = warp_incl_scan(a + b), ex = incl - a - b;
    const uint64_t gb = t * kBT + 2u * lane;
    if (gb < NB) w.lpre[gb] = ex;
    if (gb + 1 < NB) w.lpre[gb + 1] = ex + a;
    if (lane == 31) w.tsum[t] = incl;
}

// Widths and bases of all blocks, tile by tile (64 blocks, 8 per warp with all their loads in
// flight together).  Rank blocks first look up each child's parent and its (level, index) record,
// check that the parent is one level up, and store the index in R.
__global__ void __launch_bounds__(kPT, 3) pe_widths(PWork w, const uint32_t *parent)
{
    __shared__ uint32_t s_w[kBT];
    __shared__ int s_abort;
    __shared__ unsigned long long s_nb;
    if (threadIdx.x == 0) {
        s_abort = w.ctl->code != FQ_OK;
        s_nb = w.ctl->nb;
    }
    __syncthreads();
    if (s_abort) return;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t NB = s_nb, NT = dcdiv(NB, kBT);
    const uint32_t L = (uint32_t)w.L;
    for (uint64_t t = blockIdx.x; t < NT; t += gridDim.x) {
        const uint64_t gb0 = t * kBT + (uint64_t)warp * kBW;
        const BInfo mine = lane_block_info(w, L, gb0, NB, lane);
        uint32_t myw = 0, myb = 0;
        constexpr uint32_t H = kBW / 2;  // blocks per round: all their loads in flight together
#pragma unroll 1
        for (uint32_t h = 0; h < kBW; h += H) {
            BInfo bi[H];
#pragma unroll
            for (uint32_t i = 0; i < H; i++) bi[i] = bcast(mine, h + i);
            uint32_t v[H][4], p[H][4];
#pragma unroll
            for (uint32_t i = 0; i < H; i++)
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t slot = 4u * lane + q;
                    v[i][q] = slot < bi[i].cnt ? w.S[bi[i].g0 + slot] : 0u;
                }
            // rank blocks: each child's parent, then the parent's (level, index) record
#pragma unroll
            for (uint32_t i = 0; i < H; i++)
#pragma unroll
                for (uint32_t q = 0; q < 4; q++)
                    p[i][q] = (bi[i].isR && 4u * lane + q < bi[i].cnt) ? parent[v[i][q]] : 0u;
            uint32_t x[H][4];
#pragma unroll
            for (uint32_t i = 0; i < H; i++)
#pragma unroll
                for (uint32_t q = 0; q < 4; q++)
                    x[i][q] = (bi[i].isR && 4u * lane + q < bi[i].cnt && p[i][q] < w.n) ? w.gpos[p[i][q]] : kNoPos;
#pragma unroll
            for (uint32_t i = 0; i < H; i++) {
                if (!bi[i].isR) continue;  // uniform over the warp
                const uint32_t up0 = w.lo[bi[i].d - 1], up1 = w.lo[bi[i].d];  // level d - 1 in S
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t slot = 4u * lane + q;
                    if (slot >= bi[i].cnt) continue;
                    uint32_t r = 0;
                    if (x[i][q] == kNoPos || x[i][q] < up0 || x[i][q] >= up1)
                        set_error(w.ctl, FQ_EINVAL, kWherePredEnc, v[i][q]);
                    else
                        r = x[i][q] - up0;
                    w.R[bi[i].g0 + slot] = r;
                    v[i][q] = r;
                }
            }
#pragma unroll
            for (uint32_t i = 0; i < H; i++) {
                uint32_t width = 0, base = 0;
                if (!bi[i].isR) {
                    uint32_t g[4];
                    block_gaps(v[i], bi[i].cnt, lane, g);
                    width = bitlen32(__reduce_max_sync(0xffffffffu, max(max(g[0], g[1]), max(g[2], g[3]))));
                    base = __shfl_sync(0xffffffffu, v[i][0], 0);
                } else {
                    uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
                    for (uint32_t q = 0; q < 4; q++)
                        if (4u * lane + q < bi[i].cnt) {
                            mn = min(mn, v[i][q]);
                            mx = max(mx, v[i][q]);
                        }
                    mn = __reduce_min_sync(0xffffffffu, mn);
                    mx = __reduce_max_sync(0xffffffffu, mx);
                    width = bitlen32(mx - mn);
                    base = mn;
                }
                if (lane == h + i) {
                    myw = bi[i].cnt ? width : 0u;
                    myb = base;
                }
            }
        }
        if (lane < kBW) {
            if (gb0 + lane < NB) {
                w.bw[gb0 + lane] = myw;
                w.bbase[gb0 + lane] = myb;
            }
            s_w[warp * kBW + lane] = myw;
        }
        __syncthreads();
        if (warp == 0) tile_prefix(w, s_w, t, NB, lane);
        __syncthreads();
    }
}

__device__ __forceinline__ unsigned long long stream_bytes(const PStream &s, unsigned long long sumb, uint32_t *mode)
{
    const unsigned long long packed = 16u + dpad16(5ull * s.nb) + 16u * sumb;
    const unsigned long long raw = 16u + dpad16(4ull * s.n);
    const bool is_packed = s.n > 0 && packed < raw;
    *mode = is_packed ? kModePacked : kModeRaw;
    return is_packed ? packed : raw;
}

// Tile prefixes, each stream's payload start, sizes and offsets, the container header and table.
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
    const uint64_t NB = w.ctl->nb, NT = dcdiv(NB, kBT), L = w.L, K = 2 * L - 1;
    const unsigned long long sumb = cta_chunk_scan_u32<kScanThreads>(w.tsum, w.tsum, NT, sm);
    if (threadIdx.x == 0) w.tsum[NT] = (uint32_t)sumb;
    __syncthreads();
    for (uint64_t k = threadIdx.x; k < K; k += kScanThreads) w.st[k].pstart = prefix_at(w, w.st[k].blk0, NB, NT);
    __syncthreads();
    auto sumb_of = [&](uint64_t k) -> unsigned long long {
        return (k + 1 < K ? w.st[k + 1].pstart : w.tsum[NT]) - w.st[k].pstart;
    };
    const unsigned long long head = 16u + 16u * L;
    const unsigned long long body = cta_scan_fn(
        K, [&](uint64_t k) { uint32_t m; return stream_bytes(w.st[k], sumb_of(k), &m); },
        [&](uint64_t k, unsigned long long pre) {
            uint32_t m;
            w.st[k].size = stream_bytes(w.st[k], sumb_of(k), &m);
            w.st[k].mode = m;
            w.st[k].off = head + pre;
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

// Stream headers, base and width tables, payloads (packed) or values (raw); 8 blocks per warp.
__global__ void __launch_bounds__(kPT) pe_pack(PWork w, uint8_t *out)
{
    __shared__ uint32_t s_val[kPWarps][kBW][kBlock];
    __shared__ uint32_t rows[kPWarps][4 * 32 + 4];
    if (w.ctl->code != FQ_OK) return;  // warp-level work only
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t NB = w.ctl->nb, NT = dcdiv(NB, kBT);
    const uint32_t L = (uint32_t)w.L;
    for (uint64_t t = blockIdx.x; t < NT; t += gridDim.x) {
        const uint64_t gb0 = t * kBT + (uint64_t)warp * kBW;
        const BInfo mine = lane_block_info(w, L, gb0, NB, lane);
        uint32_t mw = 0, mb = 0, mp = 0;  // lane i: block i's width, base, payload units before it in its stream
        if (mine.cnt) {
            const uint64_t gb = gb0 + lane;
            mw = w.bw[gb];
            mb = w.bbase[gb];
            mp = prefix_at(w, gb, NB, NT) - w.st[mine.k].pstart;
        }
        {  // the 8 blocks' values, all loads in flight, staged in shared memory
            uint32_t v[kBW][4];
#pragma unroll
            for (uint32_t i = 0; i < kBW; i++) {
                const BInfo bi = bcast(mine, i);
                const uint32_t *src = bi.isR ? w.R : w.S;
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t slot = 4u * lane + q;
                    v[i][q] = slot < bi.cnt ? src[bi.g0 + slot] : 0u;
                }
            }
#pragma unroll
            for (uint32_t i = 0; i < kBW; i++)
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) s_val[warp][i][4u * lane + q] = v[i][q];
        }
        __syncwarp();
#pragma unroll 1
        for (uint32_t i = 0; i < kBW; i++) {
            const BInfo bi = bcast(mine, i);
            const uint32_t b = __shfl_sync(0xffffffffu, mw, i), base = __shfl_sync(0xffffffffu, mb, i);
            const uint32_t poff = __shfl_sync(0xffffffffu, mp, i);
            if (!bi.cnt) continue;  // uniform over the warp
            uint32_t v[4];
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) v[q] = s_val[warp][i][4u * lane + q];
            const PStream s = w.st[bi.k];
            const uint32_t j = (uint32_t)(gb0 + i) - s.blk0;
            const bool isR = bi.isR;
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
                for (uint32_t q = 0; q < 4; q++)
                    if (4u * lane + q < bi.cnt) dw[4u + kBlock * j + 4u * lane + q] = v[q];
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
                    dw[3] = (uint32_t)((s.size - 16u - dpad16(5ull * nb)) / 4u);
                }
                const uint32_t t0 = 16u + 5u * nb, t1 = (uint32_t)(16u + dpad16(5ull * nb));
                if (t0 + lane < t1) dst[t0 + lane] = 0u;
            }
            if (lane == 0) {
                dw[4u + j] = base;
                dst[16u + 4u * nb + j] = (uint8_t)b;
            }
            uint32_t g[4];
            if (!isR) {
                block_gaps(v, bi.cnt, lane, g);
            } else {
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) g[q] = (4u * lane + q < bi.cnt) ? v[q] - base : 0u;
            }
            uint32_t words[4];
            pack_block_words(g, b, rows[warp], lane, words);
            store_block_words(dst + 16u + dpad16(5ull * nb) + 16ull * poff, words, b, lane, 0ull, ~0ull);
        }
        __syncwarp();
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

// Widths of every block from the streams' width tables (0 for raw streams), tile prefixes.
__global__ void __launch_bounds__(kPT) pd_widths(PWork w, const uint8_t *in)
{
    __shared__ uint32_t s_w[kBT];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = w.ctl->code != FQ_OK;
    __syncthreads();
    if (s_abort) return;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t K = 2u * w.ctl->mode - 1u;
    const uint64_t NB = w.ctl->nb, NT = dcdiv(NB, kBT);
    for (uint64_t t = blockIdx.x; t < NT; t += gridDim.x) {
        if (threadIdx.x < kBT) {
            const uint64_t gb = t * kBT + threadIdx.x;
            uint32_t b = 0;
            if (gb < NB) {
                const uint32_t k = stream_of_block(w.st, K, (uint32_t)gb);
                const PStream s = w.st[k];
                if (s.mode == kModePacked) {
                    b = in[s.off + 16u + 4ull * s.nb + (gb - s.blk0)];
                    if (b > 32u) {
                        set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, k);
                        b = 0;
                    }
                }
                w.bw[gb] = b;
            }
            s_w[threadIdx.x] = b;
        }
        __syncthreads();
        if (warp == 0) tile_prefix(w, s_w, t, NB, lane);
        __syncthreads();
    }
}

// Tile prefixes, each stream's payload start; every packed stream's widths must add up to its
// announced payload.
__global__ void __launch_bounds__(kScanThreads) pd_scan(PWork w)
{
    __shared__ unsigned long long sm[33];
    if (w.ctl->code != FQ_OK) return;  // uniform: pd_widths has finished
    const uint64_t NB = w.ctl->nb, NT = dcdiv(NB, kBT), K = 2u * w.ctl->mode - 1u;
    const unsigned long long total = cta_chunk_scan_u32<kScanThreads>(w.tsum, w.tsum, NT, sm);
    if (threadIdx.x == 0) w.tsum[NT] = (uint32_t)total;
    __syncthreads();
    for (uint64_t k = threadIdx.x; k < K; k += kScanThreads) w.st[k].pstart = prefix_at(w, w.st[k].blk0, NB, NT);
    __syncthreads();
    for (uint64_t k = threadIdx.x; k < K; k += kScanThreads) {
        const PStream s = w.st[k];
        const uint32_t next = k + 1 < K ? w.st[k + 1].pstart : w.tsum[NT];
        if (s.mode == kModePacked && 4ull * (next - s.pstart) != s.words) set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, k);
    }
}

// Level-set ids into S and parent indices into R, 8 blocks per warp: the payload words of all 8
// are staged in shared memory before any is decoded.
__global__ void __launch_bounds__(kPT) pd_unpack(PWork w, const uint8_t *in)
{
    __shared__ uint32_t rows[kPWarps][kBW][4 * 32 + 4];
    if (w.ctl->code != FQ_OK) return;  // warp-level work only
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t L = w.ctl->mode;
    const uint64_t NB = w.ctl->nb, NT = dcdiv(NB, kBT);
    for (uint64_t t = blockIdx.x; t < NT; t += gridDim.x) {
        const uint64_t gb0 = t * kBT + (uint64_t)warp * kBW;
        const BInfo mine = lane_block_info(w, L, gb0, NB, lane);
        uint32_t mw = 0, mp = 0, mmode = 0, mj = 0;
        unsigned long long moff = 0;
        if (mine.cnt) {
            const uint64_t gb = gb0 + lane;
            const PStream s = w.st[mine.k];
            mw = w.bw[gb];
            mp = prefix_at(w, gb, NB, NT) - s.pstart;
            mmode = s.mode;
            mj = (uint32_t)gb - s.blk0;
            moff = s.off + 16u + (s.mode == kModeRaw ? 4ull * kBlock * mj : dpad16(5ull * s.nb) + 16ull * mp);
        }
        {  // stage the 8 blocks: payload words (packed) or values (raw), all loads in flight
            uint32_t x[kBW][4];
#pragma unroll
            for (uint32_t i = 0; i < kBW; i++) {
                const uint32_t cnt = __shfl_sync(0xffffffffu, mine.cnt, i), b = __shfl_sync(0xffffffffu, mw, i);
                const uint32_t mode = __shfl_sync(0xffffffffu, mmode, i);
                const unsigned long long o = __shfl_sync(0xffffffffu, moff, i);
                const uint32_t *src = reinterpret_cast<const uint32_t *>(in + o);
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t idx = mode == kModeRaw ? 4u * lane + q : lane + 32u * q;
                    const bool live = cnt && (mode == kModeRaw ? idx < cnt : idx < 4u * b);
                    x[i][q] = live ? src[idx] : 0u;
                }
            }
#pragma unroll
            for (uint32_t i = 0; i < kBW; i++) {
                const uint32_t mode = __shfl_sync(0xffffffffu, mmode, i);
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) rows[warp][i][mode == kModeRaw ? 4u * lane + q : lane + 32u * q] = x[i][q];
                if (lane < 4u) rows[warp][i][128u + lane] = 0u;
            }
        }
        __syncwarp();
#pragma unroll 1
        for (uint32_t i = 0; i < kBW; i++) {
            const BInfo bi = bcast(mine, i);
            const uint32_t b = __shfl_sync(0xffffffffu, mw, i);
            if (!bi.cnt) continue;  // uniform
            const PStream s = w.st[bi.k];
            const uint32_t j = (uint32_t)(gb0 + i) - s.blk0;
            const uint8_t *src = in + s.off;
            const bool isR = bi.isR;
            const uint32_t cnt = bi.cnt, d = bi.d;
            const uint32_t above = isR ? w.lo[d] - w.lo[d - 1] : 0u;  // size of level d - 1
            bool ok = true;
            uint32_t out[4];
            if (s.mode == kModeRaw) {
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) out[q] = rows[warp][i][4u * lane + q];
                if (j + 1 == s.nb) {
                    const uint32_t padw = (uint32_t)((dpad16(4ull * s.n) - 4ull * s.n) / 4u);
                    if (lane < padw && reinterpret_cast<const uint32_t *>(src + 16)[s.n + lane] != 0u) ok = false;
                }
            } else {
                if (j == 0) {
                    const uint32_t t0 = 16u + 5u * s.nb, t1 = (uint32_t)(16u + dpad16(5ull * s.nb));
                    if (t0 + lane < t1 && src[t0 + lane] != 0u) ok = false;
                }
                const uint32_t base = ld_u32(src + 16u + 4u * j);
                if (!isR && cnt == kBlock && b <= 16u) {  // full narrow block: 32-bit extraction and scan
                    uint32_t last;
                    ok = unpack_full_narrow(rows[warp][i], b, base, lane, out, &last) && ok;
                } else {
                    uint32_t g[4];
                    extract_slots(rows[warp][i], b, lane, g);
                    if (!isR) {
                        unsigned long long last;
                        ok = scan_slots(g, base, j, s.n, lane, out, &last) && ok;
                    } else {
#pragma unroll
                        for (uint32_t q = 0; q < 4; q++) {
                            const bool valid = 4u * lane + q < cnt;
                            const unsigned long long x = (unsigned long long)base + g[q];
                            if ((!valid && g[q] != 0u) || (valid && x > 0xffffffffull)) ok = false;
                            out[q] = (uint32_t)x;
                        }
                    }
                }
            }
            uint32_t *dstv = isR ? w.R : w.S;
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                const uint32_t slot = 4u * lane + q;
                if (slot < cnt) {
                    if (isR && out[q] >= above) ok = false;
                    dstv[bi.g0 + slot] = out[q];
                }
            }
            if (!ok) set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, bi.k);
        }
        __syncwarp();
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
}

// Level of position g: the largest d < L with lo[d] <= g.
__device__ __forceinline__ uint32_t level_of(const uint32_t *lo, uint32_t L, uint64_t g)
{
    uint32_t a = 0, b = L;
    while (b - a > 1) {
        const uint32_t mid = (a + b) / 2;
        if (lo[mid] <= g) a = mid;
        else b = mid;
    }
    return a;
}

// depth and parent of every reached vertex; kPosPerThread positions per thread, loads batched.
__global__ void __launch_bounds__(kPT) pd_scatter(PWork w, int32_t *depth, uint32_t *parent)
{
    if (w.ctl->code != FQ_OK) return;
    const uint32_t L = w.ctl->mode;
    const uint64_t reached = w.ctl->n;
    for (uint64_t base = (uint64_t)blockIdx.x * kPosTile; base < reached; base += (uint64_t)gridDim.x * kPosTile) {
        uint32_t v[kPosPerThread], d[kPosPerThread], r[kPosPerThread], pv[kPosPerThread];
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            v[i] = g < reached ? w.S[g] : 0u;
            d[i] = g < reached ? level_of(w.lo, L, g) : 0u;
        }
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            r[i] = (g < reached && d[i] > 0) ? w.R[g] : 0u;
        }
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            pv[i] = (g < reached && d[i] > 0) ? w.S[w.lo[d[i] - 1] + r[i]] : v[i];
        }
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            if (g >= reached) continue;
            if (v[i] >= w.n) {
                set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, g);
                continue;
            }
            depth[v[i]] = (int32_t)d[i];
            parent[v[i]] = pv[i];
        }
    }
}

// After the scatter: ids strictly increasing within each level, and every vertex holding the
// level it was listed at (a vertex listed at two levels fails at one of them).
__global__ void __launch_bounds__(kPT) pd_verify(PWork w, const int32_t *depth)
{
    if (w.ctl->code != FQ_OK) return;
    const uint32_t L = w.ctl->mode;
    const uint64_t reached = w.ctl->n;
    for (uint64_t base = (uint64_t)blockIdx.x * kPosTile; base < reached; base += (uint64_t)gridDim.x * kPosTile) {
        uint32_t v[kPosPerThread], pv[kPosPerThread], d[kPosPerThread];
        int32_t got[kPosPerThread];
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            v[i] = g < reached ? w.S[g] : 0u;
            pv[i] = (g < reached && g > 0) ? w.S[g - 1] : 0u;
            d[i] = g < reached ? level_of(w.lo, L, g) : 0u;
        }
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            got[i] = (g < reached && v[i] < w.n) ? depth[v[i]] : (int32_t)d[i];
        }
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            if (g >= reached) continue;
            const bool first = g == w.lo[d[i]];
            if (v[i] >= w.n || (!first && pv[i] >= v[i]) || got[i] != (int32_t)d[i])
                set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, g);
        }
    }
}

// ---- vertex-ordered decode (at most kVmLevels levels): chunks of kVmIds ids built in shared memory

// For every level d and id chunk c: the first position of level d whose id lies in chunk c or later
// (cstart[d][nch] = end of the level).  Written only at chunk changes; an unsorted level leaves
// entries that pd_build's checks reject.
__global__ void __launch_bounds__(kPT) pd_chunks(PWork w)
{
    if (w.ctl->code != FQ_OK) return;
    const uint32_t L = w.ctl->mode;
    const uint64_t reached = w.ctl->n, nch = w.nch;
    for (uint64_t base = (uint64_t)blockIdx.x * kPosTile; base < reached; base += (uint64_t)gridDim.x * kPosTile) {
        uint32_t v[kPosPerThread], pv[kPosPerThread], d[kPosPerThread];
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            v[i] = g < reached ? w.S[g] : 0u;
            pv[i] = (g < reached && g > 0) ? w.S[g - 1] : 0u;
            d[i] = g < reached ? level_of(w.lo, L, g) : 0u;
        }
#pragma unroll
        for (uint32_t i = 0; i < kPosPerThread; i++) {
            const uint64_t g = base + threadIdx.x + (uint64_t)kPT * i;
            if (g >= reached) continue;
            uint32_t *row = w.cstart + (uint64_t)d[i] * (nch + 1);
            const uint64_t c = min((uint64_t)(v[i] / kVmIds), nch);
            const int64_t cp = g > w.lo[d[i]] ? (int64_t)min((uint64_t)(pv[i] / kVmIds), nch) : -1;
            for (int64_t x = cp + 1; x <= (int64_t)c; x++) row[x] = (uint32_t)g;
            if (g + 1 == w.lo[d[i] + 1])
                for (uint64_t x = c + 1; x <= nch; x++) row[x] = w.lo[d[i] + 1];
        }
    }
}

// One CTA per chunk: every level's positions with ids in the chunk (checked: ids inside the chunk,
// increasing within the level, no vertex at two levels), depth and parent built in shared memory,
// then the chunk written out whole.
__global__ void __launch_bounds__(kPT) pd_build(PWork w, int32_t *depth, uint32_t *parent)
{
    __shared__ int32_t s_d[kVmIds];
    __shared__ uint32_t s_p[kVmIds];
    __shared__ uint32_t s_x0[kVmLevels], s_pre[kVmLevels + 1];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = w.ctl->code != FQ_OK;
    __syncthreads();
    if (s_abort) return;
    const uint32_t L = w.ctl->mode, lane = threadIdx.x & 31u;
    const uint64_t nch = w.nch;
    for (uint64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint64_t a = c * kVmIds;
        const uint32_t m = (uint32_t)min((uint64_t)kVmIds, w.n - a);
        for (uint32_t i = threadIdx.x; i < kVmIds; i += kPT) {
            s_d[i] = -1;
            s_p[i] = 0xffffffffu;
        }
        if (threadIdx.x < 32) {  // each level's positions in this chunk, and their prefix
            uint32_t cnt[kVmLevels / 32];
#pragma unroll
            for (uint32_t q = 0; q < kVmLevels / 32; q++) {
                const uint32_t d = lane * (kVmLevels / 32) + q;
                cnt[q] = 0;
                if (d >= L) continue;
                const uint32_t lo = w.lo[d], hi = w.lo[d + 1];
                const uint32_t *row = w.cstart + (uint64_t)d * (nch + 1);
                uint32_t x0 = row[c], x1 = row[c + 1];
                const bool ok = lo <= x0 && x0 <= x1 && x1 <= hi && (c > 0 || x0 == lo) && (c + 1 < nch || x1 == hi);
                if (!ok) {
                    set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, (unsigned long long)lo);
                    x0 = x1 = lo;
                }
                s_x0[d] = x0;
                cnt[q] = x1 - x0;
            }
            uint32_t sum = 0;
#pragma unroll
            for (uint32_t q = 0; q < kVmLevels / 32; q++) sum += cnt[q];
            uint32_t run = warp_incl_scan(sum) - sum;
#pragma unroll
            for (uint32_t q = 0; q < kVmLevels / 32; q++) {
                s_pre[lane * (kVmLevels / 32) + q] = run;
                run += cnt[q];
            }
            if (lane == 31) s_pre[kVmLevels] = run;
        }
        __syncthreads();
        const uint32_t total = s_pre[kVmLevels];
        for (uint32_t it0 = 0; it0 < total; it0 += 4u * kPT) {
            uint32_t d[4], v[4], r[4], pv[4];
            uint64_t g[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) {
                const uint32_t it = it0 + threadIdx.x + u * kPT;
                d[u] = 0;
                g[u] = 0;
                if (it < total) {
                    uint32_t lo = 0, hi = L;  // the level: largest d with s_pre[d] <= it
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) / 2;
                        if (s_pre[mid] <= it) lo = mid;
                        else hi = mid;
                    }
                    d[u] = lo;
                    g[u] = (uint64_t)s_x0[lo] + (it - s_pre[lo]);
                }
                v[u] = it < total ? w.S[g[u]] : 0u;
                pv[u] = (it < total && g[u] > s_x0[d[u]]) ? w.S[g[u] - 1] : 0u;
                r[u] = (it < total && d[u] > 0) ? __ldcs(w.R + g[u]) : 0u;
            }
            uint32_t par[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) {
                const uint32_t it = it0 + threadIdx.x + u * kPT;
                par[u] = (it < total && d[u] > 0) ? w.S[w.lo[d[u] - 1] + r[u]] : v[u];
            }
#pragma unroll
            for (uint32_t u = 0; u < 4; u++) {
                const uint32_t it = it0 + threadIdx.x + u * kPT;
                if (it >= total) continue;
                if (v[u] < a || v[u] - a >= m || (g[u] > s_x0[d[u]] && pv[u] >= v[u])) {
                    set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, g[u]);
                    continue;
                }
                if (atomicCAS(&s_d[v[u] - a], -1, (int32_t)d[u]) != -1) {  // the vertex is at another level too
                    set_error(w.ctl, FQ_ECORRUPT, kWherePredDec, g[u]);
                    continue;
                }
                s_p[v[u] - a] = par[u];
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += kPT) {  // streaming stores: keep S resident in L2 for the lookups
            __stcs(depth + a + i, s_d[i]);
            __stcs(parent + a + i, s_p[i]);
        }
        __syncthreads();
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
    pe_rowscan<<<D0, kScanThreads, 0, st>>>(w);
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
            pe_rowscan<<<D, kScanThreads, 0, st>>>(w);
            pe_dscan<<<1, kScanThreads, 0, st>>>(w, D);
            pe_scatter<false><<<tiles, kPT, 0, st>>>(w, d_depth, prev, dst, 8u * p, D, last);
        }
        prev = dst;
    }
    const uint32_t gridt = grid_for(cdiv(w.nb_max, kBT), 1);
    pe_widths<<<gridt, kPT, 0, st>>>(w, d_parent);
    pe_layout<<<1, kScanThreads, 0, st>>>(w, d_out, cap, d_out_bytes);
    pe_pack<<<gridt, kPT, 0, st>>>(w, d_out);
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
    const uint32_t gridt = grid_for(cdiv(w.nb_max, kBT), 1);
    const uint32_t gridp = grid_for(n, kPosTile);
    pd_plan<<<1, kScanThreads, 0, st>>>(w, d_in, in_bytes);
    pd_widths<<<gridt, kPT, 0, st>>>(w, d_in);
    pd_scan<<<1, kScanThreads, 0, st>>>(w);
    pd_unpack<<<gridt, kPT, 0, st>>>(w, d_in);
    if (max_levels <= kVmLevels) {
        pd_chunks<<<gridp, kPT, 0, st>>>(w);
        pd_build<<<grid_for(w.nch, 1), kPT, 0, st>>>(w, d_depth, d_parent);
    } else {
        pd_fill<<<grid_for(n, kPT), kPT, 0, st>>>(w, d_depth, d_parent);
        pd_scatter<<<gridp, kPT, 0, st>>>(w, d_depth, d_parent);
        pd_verify<<<gridp, kPT, 0, st>>>(w, d_depth);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e, __LINE__);
        return FQ_ECUDA;
    }
    return FQ_OK;
}

}  // extern "C"
