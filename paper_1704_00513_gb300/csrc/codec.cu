// codec.cu -- GPU kernels of the frontier codec (FQ queue streams, FB bitmap streams) and its
// C ABI.  Delta coding + frame-of-reference binary packing in blocks of 128 ids, the integer
// codec the thesis wraps around its per-level exchanges (binary packing and delta coding, sec.
// 5.1; S4-BP128 chosen in sec. 5.3; width = bit length, Eq. 6-7).  The byte layout is
// this library's own (documented in include/fqbfs.h), designed for warp-per-block GPU decoding:
// every block's payload is 16*b_k bytes, so it starts on a 16-byte boundary and a warp moves
// it with b_k 128-bit accesses.
//
// Encode = 2 launches: widths (one warp per 8 blocks: gaps, widths, bases, sortedness, per-tile
// width sums) and pack (packed/raw decision, headers, offsets, bits assembled with warp shuffles,
// vector stores -- or the raw body).  Decode = 3 launches: per-tile width sums, plan (one CTA:
// header and size validation, scan of the tile sums), unpack (one warp per 8 blocks: the group's
// payload staged in shared memory by one TMA bulk copy, slot extraction, warp prefix sum of the
// gaps, 128-bit stores).
#include <algorithm>
#include <cstdio>

#include "fq_common.cuh"
#include "codec_dev.cuh"

namespace fq {

// ------------------------------------------------------------------ workspace layout

namespace {
struct Layout {
    uint64_t widths, bases, block_off, tile_sum, tile_off, btile_cnt, btile_off, positions, ex, tile_ex, tile_exoff, total;
    uint64_t ids_cap, nb_cap, etiles_cap, btiles_cap, pos_cap;
};

uint64_t align256(uint64_t x) { return (x + 255u) / 256u * 256u; }

Layout layout(uint64_t max_ids, uint64_t max_nbits)
{
    Layout L{};
    L.pos_cap = max_nbits ? max_nbits / 2 + 1 : 0;  // FB codes the minority bit value: <= N/2
    L.ids_cap = std::max(max_ids, max_nbits);       // a decoded FB stream may hold up to N positions
    L.nb_cap = std::max<uint64_t>(1, cdiv(L.ids_cap, kBlock));
    L.etiles_cap = std::max<uint64_t>(1, cdiv(L.nb_cap, kTileBlocks));
    L.btiles_cap = std::max<uint64_t>(1, cdiv(cdiv(max_nbits, 64), kTileWords));
    uint64_t o = 256;  // Ctl
    L.widths = o;    o = align256(o + L.nb_cap);
    L.bases = o;     o = align256(o + 4 * L.nb_cap);
    L.block_off = o; o = align256(o + 4 * L.nb_cap);
    L.tile_sum = o;  o = align256(o + 4 * L.etiles_cap);
    L.tile_off = o;  o = align256(o + 4 * L.etiles_cap);
    L.btile_cnt = o; o = align256(o + 4 * L.btiles_cap);
    L.btile_off = o; o = align256(o + 4 * L.btiles_cap);
    L.positions = o; o = align256(o + 4 * L.pos_cap);
    L.ex = o;        o = align256(o + L.nb_cap);
    L.tile_ex = o;   o = align256(o + 4 * L.etiles_cap);
    L.tile_exoff = o; o = align256(o + 4 * L.etiles_cap);
    L.total = o;
    return L;
}
}  // namespace

uint64_t workspace_bytes(uint64_t max_ids, uint64_t max_nbits) { return layout(max_ids, max_nbits).total; }

bool workspace_fits(uint64_t bytes, uint64_t ids, uint64_t nbits) { return bytes >= workspace_bytes(ids, nbits); }

Scratch carve(void *base, uint64_t max_ids, uint64_t max_nbits)
{
    Layout L = layout(max_ids, max_nbits);
    uint8_t *b = static_cast<uint8_t *>(base);
    Scratch s;
    s.ctl = reinterpret_cast<Ctl *>(b);
    s.widths = b + L.widths;
    s.bases = reinterpret_cast<uint32_t *>(b + L.bases);
    s.block_off = reinterpret_cast<uint32_t *>(b + L.block_off);
    s.tile_sum = reinterpret_cast<uint32_t *>(b + L.tile_sum);
    s.tile_off = reinterpret_cast<uint32_t *>(b + L.tile_off);
    s.btile_cnt = reinterpret_cast<uint32_t *>(b + L.btile_cnt);
    s.btile_off = reinterpret_cast<uint32_t *>(b + L.btile_off);
    s.positions = reinterpret_cast<uint32_t *>(b + L.positions);
    s.ex = b + L.ex;
    s.tile_ex = reinterpret_cast<uint32_t *>(b + L.tile_ex);
    s.tile_exoff = reinterpret_cast<uint32_t *>(b + L.tile_exoff);
    s.ids_cap = L.ids_cap;
    s.nbits_cap = max_nbits;
    s.nb_cap = L.nb_cap;
    s.etiles_cap = L.etiles_cap;
    s.btiles_cap = L.btiles_cap;
    s.pos_cap = L.pos_cap;
    return s;
}

namespace {
thread_local int g_last_cuda_error = 0;
thread_local int g_last_cuda_line = 0;
}  // namespace

void note_cuda_error(cudaError_t e, int line)
{
    g_last_cuda_error = (int)e;
    g_last_cuda_line = line;
}

// Autotuned CTAs per SM by launch site and size class (0: the built-in grid).
// The tuning table and its generation are set from any host thread (fq_tune_set) and read at
// every launch, hence atomics.
static std::atomic<uint8_t> g_tune[FQ_TUNE_NUM_SITES][FQ_TUNE_MAX_CLASS + 1];
static std::atomic<uint32_t> g_tune_generation{0};  // bumped by every change: cached graphs that baked a grid rebuild

uint32_t tune_generation() { return g_tune_generation.load(); }

uint32_t tuned_grid(uint32_t site, uint64_t items, uint64_t default_grid, uint64_t max_grid)
{
    uint32_t cls = 0;
    for (uint64_t x = items; x > 1; x >>= 1) cls++;
    const uint32_t per_sm = (site < FQ_TUNE_NUM_SITES && cls <= FQ_TUNE_MAX_CLASS) ? g_tune[site][cls].load(std::memory_order_relaxed) : 0u;
    uint64_t g = per_sm ? (uint64_t)per_sm * (uint64_t)num_sms() : default_grid;
    g = std::min<uint64_t>(g, std::max<uint64_t>(max_grid, 1));
    return (uint32_t)std::max<uint64_t>(g, 1);
}

int num_sms()
{
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (!v) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// ------------------------------------------------------------------ kernels

namespace {

struct EncArgs {
    const uint32_t *ids;
    uint64_t n_host;
    const uint64_t *n_dev;  // when set, the id count is read here (e.g. from the bitmap plan)
    uint8_t *out;
    uint64_t cap;
    uint64_t *out_bytes;
    int fb;                 // container is an FB stream (inner FQ at out + 16)
    uint64_t nbits;
    const uint64_t *fb_words;
    Scratch s;
    // optional mirror: the same ids also written as an FB (SET) stream at m_out
    uint8_t *m_out;
    uint64_t m_cap;
    uint64_t *m_out_bytes;
    const uint64_t *m_words;
    uint64_t m_nbits;
    int px;                 // patched codec (exceptions); plain FQ containers only
};

struct DecArgs {
    const uint8_t *in;
    uint64_t in_bytes_host;
    const uint64_t *in_bytes_dev;
    uint32_t *ids;          // FQ output
    uint64_t cap;
    uint64_t *n_out;        // FQ: decoded count (device)
    int fb;
    uint64_t *words;        // FB output
    uint64_t nbits;
    Scratch s;
};

__device__ __forceinline__ uint64_t enc_count(const EncArgs &a) { return a.n_dev ? *a.n_dev : a.n_host; }
// ---- encode: widths kernel + pack kernel ----
//
// W (one warp per group of 8 blocks, one CTA per 64-block tile): gaps, block widths and bases,
// the sortedness check, per-tile width sums, and the grand width sum (one atomic per tile).
// P: every CTA takes the packed/raw decision from the grand sum on its own (the same pure
// function the header writer uses), then packs the tiles it owns -- a tile's payload offset is
// the sum of the earlier tiles' width sums, added up incrementally by the CTA -- or copies the
// raw body.  The id count may live in device memory (n_dev), so the launches need no host sync.

__device__ __forceinline__ uint64_t fb_raw_size(uint64_t nbits) { return 16u + dpad16(8u * dcdiv(nbits, 64)); }

// Modes and sizes of the output (and of its mirror) from the id count and the width sum.  A pure
// function of its inputs, so every CTA of the pack kernel takes the same decision on its own.
struct EncPlan {
    uint32_t mode, mode2;
    uint64_t size, size2;
    int32_t err;          // FQ_OK, or the error the header writer records
    uint64_t err_detail;
    bool fatal;           // the main output is not written at all
};

// Bytes of a packed patched stream: header, u32 bases + u8 widths + u8 exception counts, payload,
// u8 exception slots, u32 high parts, every section padded to 16.
__device__ __forceinline__ uint64_t px_bytes(uint64_t nb, uint64_t sum_b, uint64_t e)
{
    return kPxHeader + dpad16(6u * nb) + 16u * sum_b + dpad16(e) + dpad16(4u * e);
}

__device__ EncPlan enc_decide(const EncArgs &a, uint64_t n, uint64_t nb, unsigned long long total,
                              unsigned long long total_e, int32_t code)
{
    EncPlan p{kModeNone, kModeNone, 0, 0, FQ_OK, 0, false};
    if (code != FQ_OK) {
        p.fatal = true;
        return p;
    }
    const uint64_t packed = a.px ? px_bytes(nb, total, total_e) : 16u + dpad16(5u * nb) + 16u * total;
    const uint64_t raw = 16u + dpad16(4u * n);
    const bool is_packed = n > 0 && packed < raw;
    const uint64_t fq_size = is_packed ? packed : raw;
    const uint32_t fq_mode = is_packed ? (a.px ? kModePatched : kModePacked) : kModeRaw;
    p.mode = fq_mode;
    p.size = fq_size;
    if (a.fb) {
        const uint64_t fbr = fb_raw_size(a.nbits);
        if (16u + fq_size >= fbr) {
            p.mode = kModeFbRaw;
            p.size = fbr;
        } else {
            p.size = 16u + fq_size;
        }
    }
    if (a.m_out) {
        const uint64_t fbr = fb_raw_size(a.m_nbits);
        if (2u * n > a.m_nbits) {
            p.err = FQ_EINVAL;  // the mirror is only defined for SET mode
            p.err_detail = n;
        } else if (16u + fq_size >= fbr) {
            p.mode2 = kModeFbRaw;
            p.size2 = fbr;
        } else {
            p.mode2 = fq_mode;
            p.size2 = 16u + fq_size;
        }
        if (p.size2 > a.m_cap) {
            p.err = FQ_ENOSPC;
            p.err_detail = p.size2;
            p.mode2 = kModeNone;
        }
    }
    if (p.size > a.cap) {
        p.err = FQ_ENOSPC;
        p.err_detail = p.size;
        p.mode = p.mode2 = kModeNone;
        p.fatal = true;
    }
    return p;
}

// Record the decision, write the headers and sizes.  One thread, after every widths-kernel write.
__device__ void enc_finalize(const EncArgs &a, uint64_t n, uint64_t nb, unsigned long long total,
                             unsigned long long total_e, const EncPlan &p)
{
    Ctl *c = a.s.ctl;
    c->n = n;
    c->nb = nb;
    c->total_b = total;
    c->fq_offset = a.fb ? 16u : 0u;
    if (p.err != FQ_OK) set_error(c, p.err, kWhereEncPlan, p.err_detail);
    if (p.fatal) {
        c->mode = kModeNone;
        c->mode2 = kModeNone;
        *a.out_bytes = p.err == FQ_ENOSPC ? p.size : 0;
        if (a.m_out) *a.m_out_bytes = 0;
        return;
    }
    // headers (+ the zero pad between the width bytes and the payload of a packed stream)
    for (int which = 0; which < 2; which++) {
        uint8_t *base = which == 0 ? a.out : a.m_out;
        const uint32_t md = which == 0 ? p.mode : p.mode2;
        if (!base || md == kModeNone) continue;
        uint32_t *h = reinterpret_cast<uint32_t *>(base);
        const bool fbc = which == 1 || a.fb;
        if (fbc) {
            const uint64_t nbits = which == 0 ? a.nbits : a.m_nbits;
            h[0] = kMagicBitmap;
            h[1] = (md == kModeFbRaw) ? kFbRaw : (which == 0 ? c->fb_mode : kFbSet);
            h[2] = (uint32_t)(nbits & 0xffffffffu);
            h[3] = (uint32_t)(nbits >> 32);
            h += 4;
        }
        if (md == kModePacked) {
            h[0] = kMagicPacked; h[1] = (uint32_t)n; h[2] = (uint32_t)nb; h[3] = (uint32_t)(4u * total);
            uint8_t *fq = reinterpret_cast<uint8_t *>(h);
            for (uint64_t q = 16u + 5u * nb; q < 16u + dpad16(5u * nb); q++) fq[q] = 0;
        } else if (md == kModePatched) {
            h[0] = kMagicPatched; h[1] = (uint32_t)n; h[2] = (uint32_t)nb; h[3] = (uint32_t)(4u * total);
            h[4] = (uint32_t)total_e; h[5] = h[6] = h[7] = 0u;
            uint8_t *fq = reinterpret_cast<uint8_t *>(h);
            const uint64_t meta = kPxHeader + dpad16(6u * nb), xpos = meta + 16u * total;
            const uint64_t xhigh = xpos + dpad16(total_e), end = xhigh + dpad16(4u * total_e);
            for (uint64_t q = kPxHeader + 6u * nb; q < meta; q++) fq[q] = 0;  // the zero pads
            for (uint64_t q = xpos + total_e; q < xhigh; q++) fq[q] = 0;
            for (uint64_t q = xhigh + 4u * total_e; q < end; q++) fq[q] = 0;
        } else if (md == kModeRaw) {
            h[0] = kMagicRaw; h[1] = (uint32_t)n; h[2] = 0u; h[3] = (uint32_t)n;
        }
    }
    c->mode = p.mode;
    c->mode2 = p.mode2;
    c->out_bytes = p.size;
    c->out2_bytes = p.size2;
    *a.out_bytes = p.size;
    if (a.m_out) *a.m_out_bytes = p.size2;
}

__device__ __forceinline__ void load_blocks8(const uint32_t *ids, uint64_t k0, uint64_t n, uint32_t lane,
                                             uint32_t v[kBlocksPerWarp][4])
{
#pragma unroll
    for (uint32_t i = 0; i < kBlocksPerWarp; i++) load4_guard(ids, (k0 + i) * kBlock + 4u * lane, n, v[i]);
}

// Patched codec: width and exception count of one block -- the b in 0..32 minimising the block's
// bytes 16*b + 5*e_b, e_b = number of gaps >= 2^b, ties to the larger b.  A per-warp histogram of
// the gaps' bit lengths gives every e_b at once: lane b sums the bins above b.  All 32 lanes call it.
__device__ __forceinline__ void px_width(const uint32_t g[4], uint32_t lane, uint32_t *hist, uint32_t *b_out,
                                         uint32_t *e_out)
{
    hist[lane] = 0u;
    if (lane == 0) hist[32] = 0u;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; j++) atomicAdd(&hist[bitlen32(g[j])], 1u);
    __syncwarp();
    uint32_t e = hist[lane + 1];  // gaps of bit length lane + 1
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {  // suffix sum: e = gaps of bit length > lane
        const uint32_t y = __shfl_down_sync(0xffffffffu, e, o);
        if (lane + o < 32u) e += y;
    }
    const uint32_t key = ((16u * lane + 5u * e) << 6) | (63u - lane);  // min cost, then max b
    const uint32_t best = min(__reduce_min_sync(0xffffffffu, key), ((16u * 32u) << 6) | (63u - 32u));
    const uint32_t b = 63u - (best & 63u);
    *b_out = b;
    *e_out = b == 32u ? 0u : __shfl_sync(0xffffffffu, e, b & 31u);
    __syncwarp();  // the histogram is reused for the next block
}

// W: every warp issues the loads of its eight blocks before using any of them.
// W for tile t (all threads of the CTA; ws, we, hist: the CTA's shared scratch).
template <bool kPx>
__device__ __forceinline__ void enc_widths_tile(const EncArgs &a, uint64_t n, uint64_t nb, uint64_t t, uint32_t *ws,
                                                uint32_t *we, uint32_t (*hist)[33])
{
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    {
        const uint64_t k0 = t * kTileBlocks + warp * kBlocksPerWarp;
        uint32_t v[kBlocksPerWarp][4];
        load_blocks8(a.ids, k0, n, lane, v);
        const uint32_t before = (lane == 0 && k0 > 0 && k0 < nb) ? a.ids[k0 * kBlock - 1] : 0u;
        unsigned long long bad = ~0ull;
        uint32_t sum = 0, sum_e = 0;
#pragma unroll
        for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
            const uint64_t k = k0 + i;
            const uint32_t prev_last = __shfl_sync(0xffffffffu, i > 0 ? v[i > 0 ? i - 1 : 0][3] : 0u, 31);
            if (k >= nb) continue;
            uint32_t g[4];
            gaps_of(v[i], i > 0 ? prev_last : before, k > 0, k, n, lane, g, &bad);
            uint32_t b, e = 0;
            if (kPx) px_width(g, lane, hist[kPx ? warp : 0], &b, &e);
            else b = bitlen32(__reduce_or_sync(0xffffffffu, g[0] | g[1] | g[2] | g[3]));
            if (lane == 0) {
                a.s.widths[k] = (uint8_t)b;
                a.s.bases[k] = v[i][0];
                if (kPx) a.s.ex[k] = (uint8_t)e;
            }
            sum += b;
            sum_e += e;
        }
        if (bad != ~0ull) set_error(a.s.ctl, FQ_EUNSORTED, kWhereEncWidths, bad);
        if (lane == 0) {
            ws[warp] = sum;
            we[warp] = sum_e;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tsum = 0, tex = 0;
            for (uint32_t w = 0; w < kEncWarps; w++) {
                tsum += ws[w];
                tex += we[w];
            }
            a.s.tile_sum[t] = tsum;
            if (tsum) atomicAdd(&a.s.ctl->total_b, (unsigned long long)tsum);
            if (kPx) {
                a.s.tile_ex[t] = tex;
                if (tex) atomicAdd(&a.s.ctl->total_e, (unsigned long long)tex);
            }
        }
        __syncthreads();
    }
}

template <bool kPx>
__global__ void __launch_bounds__(kEncThreads, 4) enc_widths_kernel(EncArgs a)
{
    __shared__ uint32_t ws[kEncWarps], we[kEncWarps];
    __shared__ uint32_t hist[kPx ? kEncWarps : 1][33];
    if (a.s.ctl->skip_pos) return;  // FB: the widths were summed from the bitmap, which is coded raw
    const uint64_t n = enc_count(a), nb = dcdiv(n, kBlock), ntiles = dcdiv(nb, kTileBlocks);
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) enc_widths_tile<kPx>(a, n, nb, t, ws, we, hist);
}

// Raw bodies (FQ raw ids, or FB raw words) for whichever output the decision chose them; every
// thread of the grid takes a strided share.
__device__ void enc_raw_bodies(const EncArgs &a, const EncPlan &p, uint64_t n, uint64_t tid, uint64_t stride)
{
    for (int which = 0; which < 2; which++) {
        const uint32_t md = which == 0 ? p.mode : p.mode2;
        uint8_t *base = which == 0 ? a.out : a.m_out;
        if (md == kModeRaw) {
            uint32_t *dst = reinterpret_cast<uint32_t *>(base + (which == 0 ? (a.fb ? 16u : 0u) : 16u) + 16u);
            const uint64_t padded = dcdiv(n, 4) * 4;
            for (uint64_t i = tid; i < padded; i += stride) dst[i] = i < n ? a.ids[i] : 0u;
        } else if (md == kModeFbRaw) {
            const uint64_t nbits = which == 0 ? a.nbits : a.m_nbits;
            const uint64_t *src = which == 0 ? a.fb_words : a.m_words;
            const uint64_t nwords = dcdiv(nbits, 64);
            const uint64_t padded = dcdiv(nwords, 2) * 2;
            const uint32_t tail = (uint32_t)(nbits & 63u);
            uint64_t *dst = reinterpret_cast<uint64_t *>(base + 16);
            for (uint64_t i = tid; i < padded; i += stride) {
                uint64_t w = 0;
                if (i < nwords) {
                    w = src[i];
                    if (i == nwords - 1 && tail) w &= (1ull << tail) - 1ull;
                }
                dst[i] = w;
            }
        }
    }
}

// P for tile t, whose blocks' payload starts at width sum `prefix` (exceptions: `prefix_e`) of the
// stream -- every warp of the CTA; pk: the CTA's per-warp staging rows.
template <bool kPx>
__device__ __forceinline__ void enc_pack_tile(const EncArgs &a, const EncPlan &p, uint64_t n, uint64_t nb,
                                              unsigned long long total, unsigned long long total_e, uint64_t t,
                                              unsigned long long prefix, unsigned long long prefix_e,
                                              uint32_t (*pk)[4 * 32 + 4])
{
    const uint32_t packed_mode = kPx ? kModePatched : kModePacked;
    const bool pk1 = p.mode == packed_mode, pk2 = p.mode2 == packed_mode;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t off1 = a.fb ? 16u : 0u, off2 = 16u;  // where each output's FQ stream starts
    const uint64_t hdr = kPx ? kPxHeader : 16u;
    const uint64_t payload = hdr + dpad16((kPx ? 6u : 5u) * nb);
    const uint64_t xpos = payload + 16u * total, xhigh = xpos + dpad16(total_e);  // patched: exception areas
    {
        const uint64_t k0 = t * kTileBlocks + warp * kBlocksPerWarp;
        if (k0 >= nb) return;
        uint32_t v[kBlocksPerWarp][4];
        load_blocks8(a.ids, k0, n, lane, v);
        const uint64_t kk = t * kTileBlocks + 2 * lane;
        const uint32_t x0 = kk < nb ? a.s.widths[kk] : 0u, x1 = kk + 1 < nb ? a.s.widths[kk + 1] : 0u;
        const uint32_t my_base = (lane < kBlocksPerWarp && k0 + lane < nb) ? a.s.bases[k0 + lane] : 0u;
        const uint32_t incl = warp_incl_scan(x0 + x1);
        // lane l describes blocks 2l and 2l+1 of the tile: exclusive width prefix | b(2l) << 16 | b(2l+1) << 24
        const uint32_t info = (incl - x0 - x1) | (x0 << 16) | (x1 << 24);
        uint32_t infoe = 0;  // the same for exception counts (a tile holds at most 64 * 127 exceptions)
        if (kPx) {
            const uint32_t e0 = kk < nb ? a.s.ex[kk] : 0u, e1 = kk + 1 < nb ? a.s.ex[kk + 1] : 0u;
            const uint32_t ie = warp_incl_scan(e0 + e1);
            infoe = (ie - e0 - e1) | (e0 << 16) | (e1 << 24);
        }
        const uint32_t src = (warp * kBlocksPerWarp + (lane & 7u)) >> 1;
        const uint32_t mine = __shfl_sync(0xffffffffu, info, src);
        const uint32_t mine_e = __shfl_sync(0xffffffffu, infoe, src);
        if (lane < kBlocksPerWarp && k0 + lane < nb) {
            const uint8_t wb = (uint8_t)((lane & 1u) ? (mine >> 24) : ((mine >> 16) & 0xffu));
            if (pk1) {
                reinterpret_cast<uint32_t *>(a.out + off1 + hdr)[k0 + lane] = my_base;
                a.out[off1 + hdr + 4 * nb + k0 + lane] = wb;
                if (kPx) a.out[off1 + hdr + 5 * nb + k0 + lane] = (uint8_t)((lane & 1u) ? (mine_e >> 24) : ((mine_e >> 16) & 0xffu));
            }
            if (pk2) {
                reinterpret_cast<uint32_t *>(a.m_out + off2 + hdr)[k0 + lane] = my_base;
                a.m_out[off2 + hdr + 4 * nb + k0 + lane] = wb;
            }
        }
#pragma unroll
        for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
            const uint64_t k = k0 + i;
            const uint32_t in = __shfl_sync(0xffffffffu, info, (warp * kBlocksPerWarp + i) >> 1);
            const uint32_t b = (i & 1u) ? (in >> 24) : ((in >> 16) & 0xffu);
            const uint32_t pre = (in & 0xffffu) + ((i & 1u) ? ((in >> 16) & 0xffu) : 0u);
            if (k >= nb) continue;
            uint32_t e = 0;
            uint32_t g[4];
            unsigned long long dummy = ~0ull;
            gaps_of(v[i], 0u, false, k, n, lane, g, &dummy);
            if (kPx) {
                const uint32_t ine = __shfl_sync(0xffffffffu, infoe, (warp * kBlocksPerWarp + i) >> 1);
                e = (i & 1u) ? (ine >> 24) : ((ine >> 16) & 0xffu);
                if (e) {  // exceptions: slot numbers and high parts, in slot order
                    const uint32_t pre_e = (ine & 0xffffu) + ((i & 1u) ? ((ine >> 16) & 0xffu) : 0u);
                    uint32_t cnt = 0;
#pragma unroll
                    for (int j = 0; j < 4; j++) cnt += (b < 32u && (g[j] >> b) != 0u) ? 1u : 0u;
                    const uint32_t ex_incl = warp_incl_scan(cnt);
                    uint64_t x = prefix_e + pre_e + (ex_incl - cnt);
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (b < 32u && (g[j] >> b) != 0u) {
                            a.out[off1 + xpos + x] = (uint8_t)(4u * lane + j);
                            reinterpret_cast<uint32_t *>(a.out + off1 + xhigh)[x] = g[j] >> b;
                            x++;
                        }
                    }
                }
            }
            if (b == 0) continue;
            if (kPx && e) {
#pragma unroll
                for (int j = 0; j < 4; j++) g[j] &= (b < 32u) ? ((1u << b) - 1u) : 0xffffffffu;  // low bits only
            }
            uint32_t w4[4];
            pack_block_words(g, b, pk[warp], lane, w4);
            const uint64_t rel = payload + 16u * (prefix + pre);
            if (pk1) store_block_words(a.out + off1 + rel, w4, b, lane, 0, ~0ull);
            if (pk2) store_block_words(a.m_out + off2 + rel, w4, b, lane, 0, ~0ull);
        }
    }
}

// P: decision, headers (CTA 0), then the packed body tile by tile -- one warp per group of
// kBlocksPerWarp blocks, offsets from the tile's width bytes (two per lane, one warp scan) -- or
// the raw bodies.  Packed words go to the output and, identical, to the mirror's inner stream.
template <bool kPx>
__global__ void __launch_bounds__(kEncThreads, 3) enc_pack_kernel(EncArgs a)
{
    __shared__ uint32_t pk[kEncWarps][4 * 32 + 4];
    __shared__ unsigned long long s_part[kEncWarps], s_parte[kEncWarps];
    const Ctl *c = a.s.ctl;
    const uint64_t n = enc_count(a), nb = dcdiv(n, kBlock), ntiles = dcdiv(nb, kTileBlocks);
    const unsigned long long total = c->total_b, total_e = kPx ? c->total_e : 0ull;
    const EncPlan p = enc_decide(a, n, nb, total, total_e, *reinterpret_cast<const volatile int32_t *>(&c->code));
    if (blockIdx.x == 0 && threadIdx.x == 0) enc_finalize(a, n, nb, total, total_e, p);
    if (p.fatal) return;
    enc_raw_bodies(a, p, n, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
    const uint32_t packed_mode = kPx ? kModePatched : kModePacked;
    if (p.mode != packed_mode && p.mode2 != packed_mode) return;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    unsigned long long prefix = 0, prefix_e = 0;  // width and exception sums of tiles [0, done)
    uint64_t done = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // add the width (and exception) sums of tiles [done, t)
        unsigned long long part = 0, parte = 0;
        for (uint64_t i = done + threadIdx.x; i < t; i += blockDim.x) {
            part += a.s.tile_sum[i];
            if (kPx) parte += a.s.tile_ex[i];
        }
        part = warp_sum64(part);
        if (kPx) parte = warp_sum64(parte);
        if (lane == 0) {
            s_part[warp] = part;
            s_parte[warp] = parte;
        }
        __syncthreads();
        for (uint32_t w = 0; w < kEncWarps; w++) {
            prefix += s_part[w];
            if (kPx) prefix_e += s_parte[w];
        }
        __syncthreads();
        done = t;
        enc_pack_tile<kPx>(a, p, n, nb, total, total_e, t, prefix, prefix_e, pk);
    }
}

// ---- bitmap -> positions (FB encode) ----

__device__ __forceinline__ uint64_t masked_word(const uint64_t *words, uint64_t w, uint64_t nbits, bool invert)
{
    const uint64_t nwords = dcdiv(nbits, 64);
    if (w >= nwords) return 0;
    uint64_t x = words[w];
    if (invert) x = ~x;
    const uint32_t tail = (uint32_t)(nbits & 63u);
    if (w == nwords - 1 && tail) x &= (1ull << tail) - 1ull;
    return x;
}

__global__ void __launch_bounds__(kBitThreads) bits_count_kernel(const uint64_t *words, uint64_t nbits, uint32_t *tile_cnt)
{
    __shared__ uint32_t ws[kBitThreads / 32];
    const uint64_t w0 = (uint64_t)blockIdx.x * kTileWords + (uint64_t)threadIdx.x * kWordsPerThread;
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t j = 0; j < kWordsPerThread; j++) cnt += __popcll(masked_word(words, w0 + j, nbits, false));
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

// One CTA: popcount P, SET/CLEAR choice, exclusive scan of the chosen per-tile counts.
__global__ void __launch_bounds__(kScanThreads) fb_plan_kernel(uint64_t nbits, Scratch s)
{
    __shared__ unsigned long long sm[33];
    __shared__ unsigned long long sP;
    const uint64_t nwords = dcdiv(nbits, 64);
    const uint64_t ntiles = dcdiv(nwords, kTileWords);
    const uint64_t chunk = dcdiv(ntiles, kScanThreads);
    const uint64_t t0 = (uint64_t)threadIdx.x * chunk, t1 = min(ntiles, t0 + chunk);
    unsigned long long local = 0, total = 0;
    for (uint64_t t = t0; t < t1; t++) local += s.btile_cnt[t];
    cta_excl_scan64<kScanThreads>(local, sm, &total);
    if (threadIdx.x == 0) sP = total;
    __syncthreads();
    const unsigned long long P = sP;
    const bool set_mode = 2ull * P <= nbits;
    local = 0;
    const uint64_t tile_bits = (uint64_t)kTileWords * 64u;
    for (uint64_t t = t0; t < t1; t++) {
        const uint64_t bits_in = min(nbits, (t + 1) * tile_bits) - t * tile_bits;
        local += set_mode ? s.btile_cnt[t] : bits_in - s.btile_cnt[t];
    }
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t t = t0; t < t1; t++) {
        s.btile_off[t] = (uint32_t)run;
        const uint64_t bits_in = min(nbits, (t + 1) * tile_bits) - t * tile_bits;
        run += set_mode ? s.btile_cnt[t] : bits_in - s.btile_cnt[t];
    }
    if (threadIdx.x == 0) {
        s.ctl->popcount = P;
        s.ctl->fb_mode = set_mode ? kFbSet : kFbClear;
        s.ctl->n = total;  // positions to code
    }
}

__global__ void __launch_bounds__(kBitThreads) bits_extract_kernel(const uint64_t *words, uint64_t nbits, Scratch s)
{
    __shared__ unsigned long long sm[33];
    const bool invert = s.ctl->fb_mode == kFbClear;
    const uint64_t w0 = (uint64_t)blockIdx.x * kTileWords + (uint64_t)threadIdx.x * kWordsPerThread;
    uint64_t x[kWordsPerThread];
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t j = 0; j < kWordsPerThread; j++) {
        x[j] = masked_word(words, w0 + j, nbits, invert);
        cnt += __popcll(x[j]);
    }
    unsigned long long total;
    unsigned long long off = cta_excl_scan64<kBitThreads>(cnt, sm, &total) + s.btile_off[blockIdx.x];
#pragma unroll
    for (uint32_t j = 0; j < kWordsPerThread; j++) {
        uint64_t y = x[j];
        while (y) {
            const uint32_t bit = __ffsll((long long)y) - 1;
            s.positions[off++] = (uint32_t)((w0 + j) * 64u + bit);
            y &= y - 1;
        }
    }
}

// ---- decode ----

// ---- decode ----
//
// D0 (many CTAs): per tile of 64 blocks, the sum of the block widths (widths > 32 flagged).
// D1 (one CTA):   header validation, scan of the tile sums into tile offsets, size checks.
// D2 (many CTAs): per tile, block offsets from the tile offset + a local scan; one warp per block
//                 unpacks, prefix-sums the gaps, validates and writes the ids (or bits).
// Every check that bounds a read or a write happens before that access: no output is written
// unless the header, the widths and the sizes are consistent with in_bytes and the capacity.

struct FqHeader {
    bool ok;          // container and FQ header readable and self-consistent (sizes not yet summed)
    bool over;        // n above the output capacity
    uint32_t mode;    // kModePacked / kModeRaw / kModeFbRaw
    uint32_t fb_mode;
    uint64_t fq_off, fq_bytes, n, nb, words;
    uint64_t hdr, meta;  // packed forms: header bytes (16, patched 32) and metadata bytes per block (5, 6)
    uint64_t e_total;    // patched: exceptions announced by the header
};

__device__ FqHeader parse_header(const DecArgs &a, uint64_t in_bytes)
{
    FqHeader h{};
    h.ok = true;
    h.over = false;
    h.mode = kModeNone;
    h.fb_mode = kFbRaw;
    h.fq_off = 0;
    h.fq_bytes = in_bytes;
    const uint64_t limit = a.fb ? a.nbits : a.cap;
    if (a.fb) {
        if (in_bytes < 16 || ld_u32(a.in) != kMagicBitmap ||
            ((uint64_t)ld_u32(a.in + 8) | ((uint64_t)ld_u32(a.in + 12) << 32)) != a.nbits) {
            h.ok = false;
            return h;
        }
        const uint32_t m = ld_u32(a.in + 4);
        if (m == kFbRaw) {
            h.ok = in_bytes == 16u + dpad16(8u * dcdiv(a.nbits, 64));
            h.mode = kModeFbRaw;
            return h;
        }
        if (m != kFbSet && m != kFbClear) {
            h.ok = false;
            return h;
        }
        h.fb_mode = m;
        h.fq_off = 16;
        h.fq_bytes = in_bytes - 16u;
    }
    const uint8_t *fq = a.in + h.fq_off;
    if (h.fq_bytes < 16) {
        h.ok = false;
        return h;
    }
    const uint32_t magic = ld_u32(fq);
    h.n = ld_u32(fq + 4);
    h.nb = ld_u32(fq + 8);
    h.words = ld_u32(fq + 12);
    if (h.n > limit) {  // more ids than the output (or the scratch) holds: nothing is written
        h.ok = false;
        h.over = true;
        return h;
    }
    h.hdr = 16;
    h.meta = 5;
    h.e_total = 0;
    if (magic == kMagicRaw) {
        h.mode = kModeRaw;
        h.ok = h.nb == 0 && h.words == h.n && h.fq_bytes == 16u + dpad16(4u * h.n);
    } else if (magic == kMagicPacked) {
        h.mode = kModePacked;
        h.ok = h.nb == dcdiv(h.n, kBlock) && h.n > 0 && h.fq_bytes >= 16u + dpad16(5u * h.nb);
    } else if (magic == kMagicPatched && !a.fb && h.fq_bytes >= kPxHeader) {
        h.mode = kModePatched;
        h.hdr = kPxHeader;
        h.meta = 6;
        h.e_total = ld_u32(fq + 16);
        h.ok = h.nb == dcdiv(h.n, kBlock) && h.n > 0 && h.fq_bytes >= kPxHeader + dpad16(6u * h.nb) &&
               ld_u32(fq + 20) == 0u && ld_u32(fq + 24) == 0u && ld_u32(fq + 28) == 0u;
    } else {
        h.ok = false;
    }
    return h;
}

__device__ __forceinline__ uint64_t dec_in_bytes(const DecArgs &a)
{
    return a.in_bytes_dev ? *a.in_bytes_dev : a.in_bytes_host;
}

template <uint32_t NT>
__device__ void dec_plan_body(const DecArgs &a);

// The per-tile width (and exception) sums of a packed stream: a CTA takes kEncThreads / kTileBlocks
// tiles at a time (one thread per block), tile groups strided over the grid.
__device__ void dec_tile_sums(const DecArgs &a)
{
    constexpr uint32_t kTilesPerPass = kEncThreads / kTileBlocks;  // 4
    constexpr uint32_t kWarpsPerTile = kTileBlocks / 32u;          // 2
    __shared__ uint32_t ws[kEncWarps], we[kEncWarps];
    const FqHeader h = parse_header(a, dec_in_bytes(a));
    if (!h.ok || (h.mode != kModePacked && h.mode != kModePatched)) return;
    const bool px = h.mode == kModePatched;
    const uint8_t *wd = a.in + h.fq_off + h.hdr + 4 * h.nb;
    const uint64_t ntiles = dcdiv(h.nb, kTileBlocks);
    const uint32_t warp = threadIdx.x >> 5;
    for (uint64_t t0 = (uint64_t)blockIdx.x * kTilesPerPass; t0 < ntiles; t0 += (uint64_t)gridDim.x * kTilesPerPass) {
        const uint64_t k = t0 * kTileBlocks + threadIdx.x;  // tile t0 + threadIdx.x / 64, its block threadIdx.x % 64
        uint32_t b = 0, e = 0;
        if (k < h.nb) {
            b = wd[k];
            if (b > 32u) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecPlan, h.fq_off + h.hdr + 4 * h.nb + k);
            if (px) {  // exception count: at most 127 (slot 0 never), none at width 32
                e = wd[h.nb + k];
                if (e > 127u || (b == 32u && e)) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecPlan, h.hdr + 5 * h.nb + k);
            }
        }
        b = __reduce_add_sync(0xffffffffu, b);
        e = __reduce_add_sync(0xffffffffu, e);
        if ((threadIdx.x & 31u) == 0) {
            ws[warp] = b;
            we[warp] = e;
        }
        __syncthreads();
        if (threadIdx.x < kTilesPerPass && t0 + threadIdx.x < ntiles) {
            uint32_t sum = 0, sume = 0;
            for (uint32_t i = 0; i < kWarpsPerTile; i++) {
                sum += ws[threadIdx.x * kWarpsPerTile + i];
                sume += we[threadIdx.x * kWarpsPerTile + i];
            }
            a.s.tile_sum[t0 + threadIdx.x] = sum;
            if (px) a.s.tile_ex[t0 + threadIdx.x] = sume;
        }
        __syncthreads();
    }
}

// D0, and D1 in the last CTA to finish: per-tile width sums (widths > 32 flagged); then, once every
// CTA has taken its ticket after a fence (so all tile sums are visible), the last one validates the
// header and sizes and scans the tile sums (dec_plan_body).
__global__ void __launch_bounds__(kEncThreads) dec_tiles_kernel(DecArgs a)
{
    __shared__ bool s_last;
    dec_tile_sums(a);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&a.s.ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    dec_plan_body<kEncThreads>(a);
    if (threadIdx.x == 0) a.s.ctl->ticket = 0u;
}

// D1 (one CTA of NT threads): header validation, scan of the tile sums into tile offsets, size checks.
template <uint32_t NT>
__device__ void dec_plan_body(const DecArgs &a)
{
    __shared__ unsigned long long sm[33];
    Ctl *c = a.s.ctl;
    const FqHeader h = parse_header(a, dec_in_bytes(a));
    bool ok = h.ok;
    if (ok && h.mode == kModeRaw && threadIdx.x == 0) {
        const uint8_t *fq = a.in + h.fq_off;
        for (uint64_t i = 16u + 4u * h.n; i < h.fq_bytes; i++)
            if (fq[i]) ok = false;
    }
    if (ok && h.mode == kModePacked) {
        const uint8_t *fq = a.in + h.fq_off;
        const uint64_t ntiles = dcdiv(h.nb, kTileBlocks);
        const unsigned long long total = cta_chunk_scan_u32<NT>(a.s.tile_sum, a.s.tile_off, ntiles, sm);
        if (threadIdx.x == 0) {
            c->total_b = total;
            if (h.words != 4u * total || h.fq_bytes != 16u + dpad16(5u * h.nb) + 16u * total) ok = false;
            for (uint64_t i = 16u + 5u * h.nb; i < 16u + dpad16(5u * h.nb); i++)
                if (fq[i]) ok = false;
        }
    }
    if (ok && h.mode == kModePatched) {
        const uint8_t *fq = a.in + h.fq_off;
        const uint64_t ntiles = dcdiv(h.nb, kTileBlocks);
        const unsigned long long total = cta_chunk_scan_u32<NT>(a.s.tile_sum, a.s.tile_off, ntiles, sm);
        const unsigned long long tex = cta_chunk_scan_u32<NT>(a.s.tile_ex, a.s.tile_exoff, ntiles, sm);
        if (threadIdx.x == 0) {
            c->total_b = total;
            c->total_e = tex;
            const uint64_t meta = kPxHeader + dpad16(6u * h.nb), xpos = meta + 16u * total;
            const uint64_t xhigh = xpos + dpad16(tex), end = xhigh + dpad16(4u * tex);
            if (h.words != 4u * total || h.e_total != tex || h.fq_bytes != end) ok = false;
            for (uint64_t i = kPxHeader + 6u * h.nb; ok && i < meta; i++)  // the zero pads
                if (fq[i]) ok = false;
            for (uint64_t i = xpos + tex; ok && i < xhigh; i++)
                if (fq[i]) ok = false;
            for (uint64_t i = xhigh + 4u * tex; ok && i < end; i++)
                if (fq[i]) ok = false;
        }
    }
    if (threadIdx.x != 0) return;
    c->fq_offset = h.fq_off;
    c->fb_mode = h.fb_mode;
    c->n = h.n;
    c->nb = h.nb;
    if (h.over) {
        set_error(c, a.fb ? FQ_ECORRUPT : FQ_ENOSPC, kWhereDecPlan, h.n);
        c->mode = kModeNone;
        if (a.n_out) *a.n_out = h.n;
        return;
    }
    if (!ok || __ldcg(&c->code) != FQ_OK) {  // D0 may have flagged a width > 32
        set_error(c, FQ_ECORRUPT, kWhereDecPlan, 0ull);
        c->mode = kModeNone;
        if (a.n_out) *a.n_out = 0;
        return;
    }
    c->mode = h.mode;
    if (a.n_out) *a.n_out = h.n;
}

// FB decode, before the scatter: clear (SET) or fill (CLEAR) the words, or copy raw words.
__global__ void fb_init_kernel(DecArgs a)
{
    const Ctl *c = a.s.ctl;
    const uint32_t mode = c->mode;
    if (mode == kModeNone) return;
    const uint64_t nwords = dcdiv(a.nbits, 64);
    const uint32_t tail = (uint32_t)(a.nbits & 63u);
    const uint64_t tail_mask = tail ? (1ull << tail) - 1ull : ~0ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += stride) {
        uint64_t w;
        if (mode == kModeFbRaw) {
            w = reinterpret_cast<const uint64_t *>(a.in + 16)[i];
            if (i == nwords - 1 && (w & ~tail_mask)) set_error(a.s.ctl, FQ_ECORRUPT, kWhereFbDecode, 16 + 8 * i);
            if (i == nwords - 1) w &= tail_mask;
        } else {
            w = (c->fb_mode == kFbClear) ? ~0ull : 0ull;
            if (i == nwords - 1) w &= tail_mask;
        }
        a.words[i] = w;
    }
    if (mode == kModeFbRaw && blockIdx.x == 0 && threadIdx.x == 0 && (nwords & 1u)) {
        if (reinterpret_cast<const uint64_t *>(a.in + 16)[nwords] != 0ull)
            set_error(a.s.ctl, FQ_ECORRUPT, kWhereFbDecode, 16 + 8 * nwords);
    }
}

__device__ __forceinline__ void emit_id(const DecArgs &a, uint32_t clear_mode, uint64_t i, uint32_t v)
{
    if (!a.fb) {
        a.ids[i] = v;
        return;
    }
    if ((uint64_t)v >= a.nbits) {
        set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecUnpack, i);
        return;
    }
    uint32_t *w32 = reinterpret_cast<uint32_t *>(a.words);
    if (clear_mode) atomicAnd(&w32[v >> 5], ~(1u << (v & 31u)));
    else atomicOr(&w32[v >> 5], 1u << (v & 31u));
}

// A group's largest payload (kBlocksPerWarp blocks of width 32) + slack for the 3-word windows.
constexpr uint32_t kDecStage = kBlocksPerWarp * 32u * 16u + 16u;
constexpr size_t kDecSmem = (size_t)kEncWarps * 2 * kDecStage;

// Where one group of kBlocksPerWarp blocks (never straddling a tile) sits: lane l describes tile
// blocks 2l, 2l+1 in `info` (exclusive width prefix | b(2l) << 16 | b(2l+1) << 24), lane i <= 8
// holds the base of the group's block i in `base` (i = 8: the next group's first, for the bound
// check), and the payload range is [off, off + bytes) of the payload area.
struct GroupMeta {
    uint32_t info, base, pre;
    uint64_t off;
    uint32_t bytes;
    uint32_t infoe;  // patched: like info, for the exception counts (in-tile prefix | e(2l) << 16 | e(2l+1) << 24)
    uint64_t exoff;  // patched: the tile's first exception
};

__device__ __forceinline__ GroupMeta group_meta(const DecArgs &a, const uint8_t *wd, const uint32_t *bases,
                                                const uint8_t *exn, uint64_t nb, uint64_t grp, uint32_t lane)
{
    constexpr uint32_t kGroupsPerTile = kTileBlocks / kBlocksPerWarp;
    const uint64_t t = grp / kGroupsPerTile, k0 = grp * kBlocksPerWarp;
    const uint32_t git = (uint32_t)(grp % kGroupsPerTile);
    const uint64_t kk = t * kTileBlocks + 2 * lane;
    const uint32_t x0 = kk < nb ? wd[kk] : 0u, x1 = kk + 1 < nb ? wd[kk + 1] : 0u;
    const uint32_t tile_base = a.s.tile_off[t];
    GroupMeta m;
    m.base = (lane <= kBlocksPerWarp && k0 + lane < nb) ? bases[k0 + lane] : 0u;
    const uint32_t incl = warp_incl_scan(x0 + x1);
    m.info = (incl - x0 - x1) | (x0 << 16) | (x1 << 24);
    const uint32_t lead = git * (kBlocksPerWarp / 2);  // the lane describing the group's first block
    m.pre = __shfl_sync(0xffffffffu, incl - x0 - x1, lead);
    const uint32_t end = __shfl_sync(0xffffffffu, incl, lead + kBlocksPerWarp / 2 - 1);
    m.off = 16ull * ((uint64_t)tile_base + m.pre);
    m.bytes = 16u * (end - m.pre);
    m.infoe = 0;
    m.exoff = 0;
    if (exn) {
        const uint32_t e0 = kk < nb ? exn[kk] : 0u, e1 = kk + 1 < nb ? exn[kk + 1] : 0u;
        const uint32_t ie = warp_incl_scan(e0 + e1);
        m.infoe = (ie - e0 - e1) | (e0 << 16) | (e1 << 24);
        m.exoff = a.s.tile_exoff[t];
    }
    return m;
}

// D2: one warp per group of kBlocksPerWarp blocks, groups assigned round-robin over all warps, no
// CTA barrier.  A group's payload is one contiguous range: lane 0 stages it into the warp's own
// shared-memory buffer with one TMA bulk copy while the warp decodes the previous group from the
// other buffer (extract, prefix-sum the gaps, validate, 128-bit stores).
// dbuf: [kEncWarps][2][kDecStage] bytes (128-byte aligned); bars, patch: the CTA's shared scratch.
__device__ __forceinline__ void dec_unpack_body(const DecArgs &a, uint8_t *dbuf, unsigned long long (*bars)[2],
                                                uint32_t (*patch)[kBlock])
{
    const Ctl *c = a.s.ctl;
    const uint32_t mode = c->mode;
    if (mode != kModePacked && mode != kModeRaw && mode != kModePatched) return;
    const uint64_t n = c->n, nb = c->nb;
    const uint8_t *fq = a.in + c->fq_offset;
    const uint32_t clear_mode = (a.fb && c->fb_mode == kFbClear) ? 1u : 0u;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;

    if (mode == kModeRaw) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(fq + 16);
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const uint32_t v = src[i];
            if (i > 0 && src[i - 1] >= v) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecUnpack, 16 + 4 * i);
            emit_id(a, clear_mode, i, v);
        }
        return;
    }

    const bool px = mode == kModePatched;
    const uint64_t hdr = px ? kPxHeader : 16u;
    const uint8_t *wd = fq + hdr + 4 * nb;
    const uint32_t *bases = reinterpret_cast<const uint32_t *>(fq + hdr);
    const uint8_t *exn = px ? fq + hdr + 5 * nb : nullptr;  // patched: exceptions per block
    const uint8_t *payload = fq + hdr + dpad16((px ? 6u : 5u) * nb);
    const uint8_t *xslot = payload + 16u * c->total_b;    // patched: exception slots, then high parts
    const uint32_t *xhigh = reinterpret_cast<const uint32_t *>(xslot + dpad16(c->total_e));
    const uint64_t ngroups = dcdiv(nb, kBlocksPerWarp);
    const uint64_t nwarps = (uint64_t)gridDim.x * kEncWarps;
    uint64_t grp = (uint64_t)blockIdx.x * kEncWarps + warp;
    if (grp >= ngroups) return;
    uint8_t *buf = dbuf + (size_t)warp * 2 * kDecStage;
    unsigned long long *bar = bars[warp];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncwarp();
    GroupMeta cur = group_meta(a, wd, bases, exn, nb, grp, lane);
    if (lane == 0 && cur.bytes) bulk_load(buf, payload + cur.off, cur.bytes, &bar[0]);
    uint32_t phase0 = 0u, phase1 = 0u;
    for (uint32_t it = 0;; it++) {
        const uint32_t stage = it & 1u;
        const uint64_t gn = grp + nwarps;
        GroupMeta nxt{};
        if (gn < ngroups) nxt = group_meta(a, wd, bases, exn, nb, gn, lane);
        __syncwarp();  // every lane is done with the other buffer (read in the previous iteration)
        if (gn < ngroups && lane == 0 && nxt.bytes)
            bulk_load(buf + (stage ^ 1u) * kDecStage, payload + nxt.off, nxt.bytes, &bar[stage ^ 1u]);
        if (cur.bytes) {
            // Bounded wait for the group's payload.  A copy still missing after it is reported;
            // lane 0 then lets the warp's copies in flight land (bounded again), and the warp leaves.
            if (!__all_sync(0xffffffffu, mbar_wait(&bar[stage], stage ? phase1 : phase0))) {
                if (lane == 0) {
                    set_error(a.s.ctl, FQ_ETIMEOUT, kWhereDecUnpack, grp);
                    mbar_wait(&bar[stage], stage ? phase1 : phase0);
                    if (gn < ngroups && nxt.bytes) mbar_wait(&bar[stage ^ 1u], stage ? phase0 : phase1);
                }
                return;
            }
            if (stage) phase1 ^= 1u;
            else phase0 ^= 1u;
        }
        const uint32_t *sp = reinterpret_cast<const uint32_t *>(buf + stage * kDecStage);
        const uint32_t git = (uint32_t)(grp % (kTileBlocks / kBlocksPerWarp));
        const uint64_t k0 = grp * kBlocksPerWarp;
        // One block of the group (any width, patched or not).
        auto one_block = [&](uint32_t i) {
            const uint64_t k = k0 + i;
            const uint32_t in = __shfl_sync(0xffffffffu, cur.info, git * (kBlocksPerWarp / 2) + (i >> 1));
            const uint32_t base = __shfl_sync(0xffffffffu, cur.base, i);
            const uint32_t next = __shfl_sync(0xffffffffu, cur.base, i + 1);
            if (k >= nb) return;
            const uint32_t b = (i & 1u) ? (in >> 24) : ((in >> 16) & 0xffu);
            const uint32_t pre = (in & 0xffffu) + ((i & 1u) ? ((in >> 16) & 0xffu) : 0u) - cur.pre;
            const uint32_t *pk = sp + 4u * pre;
            const uint64_t i0 = k * kBlock + 4u * lane;
            uint32_t out[4];
            bool good;
            uint32_t e = 0, pre_e = 0;
            if (px) {
                const uint32_t ine = __shfl_sync(0xffffffffu, cur.infoe, git * (kBlocksPerWarp / 2) + (i >> 1));
                e = (i & 1u) ? (ine >> 24) : ((ine >> 16) & 0xffu);
                pre_e = (ine & 0xffffu) + ((i & 1u) ? ((ine >> 16) & 0xffu) : 0u);
            }
            if (e) {  // patched block: low bits, plus each exception's high part above them
                uint32_t g[4];
                if (b <= 16u) extract_narrow(pk, b, lane, g);
                else extract_slots(pk, b, lane, g);
                uint32_t *pt = patch[warp];
                const uint64_t x0 = cur.exoff + pre_e;
                bool okx = true;
                uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0, hor = 0;  // 128-bit mask of exception slots
                for (uint32_t q0 = 0; q0 < e; q0 += 32u) {
                    const uint32_t q = q0 + lane;
                    uint32_t slot = 0, bit = 0;
                    if (q < e) {
                        slot = xslot[x0 + q];
                        const uint32_t prev = q ? xslot[x0 + q - 1] : 0u, high = xhigh[x0 + q];
                        // slots 1..127, increasing, inside the id range; a nonzero high part that fits above b
                        if (slot == 0u || slot >= kBlock || slot <= prev || k * kBlock + slot >= n || high == 0u ||
                            ((uint64_t)high >> (32u - b)) != 0ull) {
                            okx = false;
                        } else {
                            pt[slot] = high;
                            bit = 1u << (slot & 31u);
                            hor |= high;
                        }
                    }
                    m0 |= __reduce_or_sync(0xffffffffu, (slot >> 5) == 0u ? bit : 0u);
                    m1 |= __reduce_or_sync(0xffffffffu, (slot >> 5) == 1u ? bit : 0u);
                    m2 |= __reduce_or_sync(0xffffffffu, (slot >> 5) == 2u ? bit : 0u);
                    m3 |= __reduce_or_sync(0xffffffffu, (slot >> 5) == 3u ? bit : 0u);
                }
                __syncwarp();
                const uint32_t mw = (lane < 8u) ? m0 : (lane < 16u) ? m1 : (lane < 24u) ? m2 : m3;
                const uint32_t mine4 = (mw >> ((4u * lane) & 31u)) & 0xfu;  // my four slots
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if ((mine4 >> j) & 1u) g[j] |= pt[4 * lane + j] << b;  // b < 32: width 32 has no exceptions
                __syncwarp();  // the stage is rewritten by the next patched block
                const uint32_t widest = b + bitlen32(__reduce_or_sync(0xffffffffu, hor));
                // every lane runs the scan (it shuffles across the warp); then the exception checks count
                if (k + 1 < nb && widest <= 16u) {  // increments still sum below 2^32: the 32-bit scan
                    uint32_t lastv;
                    good = scan_full32(g, base, lane, out, &lastv);
                    if (lane == 31 && lastv >= next) good = false;
                } else {
                    unsigned long long lastv;
                    good = scan_slots(g, base, k, n, lane, out, &lastv);
                    if (k + 1 < nb && lane == 31 && lastv >= (unsigned long long)next) good = false;
                }
                good = good && okx;
            } else if (k + 1 < nb && b <= 16u) {  // full narrow block: the lean 32-bit path
                uint32_t lastv;
                good = unpack_full_narrow(pk, b, base, lane, out, &lastv);
                if (lane == 31 && lastv >= next) good = false;
            } else {
                unsigned long long lastv;
                good = unpack_block(pk, b, base, k, n, lane, out, &lastv);
                // a full block (k + 1 < nb) ends in lane 31's last slot: it must stay below the next base
                if (k + 1 < nb && lane == 31 && lastv >= (unsigned long long)next) good = false;
            }
            if (!good) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecUnpack, k * kBlock);
            if (!a.fb && i0 + 3 < n) {
                *reinterpret_cast<uint4 *>(a.ids + i0) = make_uint4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (i0 + j < n) emit_id(a, clear_mode, i0 + j, out[j]);
            }
        };
        // Blocks in pairs: two full unpatched blocks of width <= 8 (and a block after them, whose
        // base bounds the second) share one warp scan -- each block's increments sum below 2^15,
        // so the two prefix sums ride in the halves of one 32-bit scan without a carry between them.
        for (uint32_t i = 0; i < kBlocksPerWarp; i += 2) {
            const uint64_t kA = k0 + i;
            const uint32_t in = __shfl_sync(0xffffffffu, cur.info, git * (kBlocksPerWarp / 2) + (i >> 1));
            const uint32_t ine = px ? __shfl_sync(0xffffffffu, cur.infoe, git * (kBlocksPerWarp / 2) + (i >> 1)) : 0u;
            const uint32_t baseA = __shfl_sync(0xffffffffu, cur.base, i), baseB = __shfl_sync(0xffffffffu, cur.base, i + 1);
            const uint32_t nextB = __shfl_sync(0xffffffffu, cur.base, i + 2);
            if (kA >= nb) break;
            const uint32_t bA = (in >> 16) & 0xffu, bB = in >> 24;
            if (!(kA + 2 < nb && bA <= 8u && bB <= 8u && (ine >> 16) == 0u)) {  // uniform over the warp
                one_block(i);
                one_block(i + 1);
                continue;
            }
            const uint32_t preA = (in & 0xffffu) - cur.pre, preB = preA + bA;
            uint32_t oA[4], oB[4];
            bool goodA, goodB;
            unpack_pair_narrow(sp + 4u * preA, bA, baseA, sp + 4u * preB, bB, baseB, nextB, lane, oA, oB, &goodA,
                               &goodB);
            if (!goodA) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecUnpack, kA * kBlock);
            if (!goodB) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecUnpack, (kA + 1) * kBlock);
            const uint64_t iA = kA * kBlock + 4u * lane, iB = iA + kBlock;
            if (!a.fb) {  // full blocks: every slot holds an id
                *reinterpret_cast<uint4 *>(a.ids + iA) = make_uint4(oA[0], oA[1], oA[2], oA[3]);
                *reinterpret_cast<uint4 *>(a.ids + iB) = make_uint4(oB[0], oB[1], oB[2], oB[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    emit_id(a, clear_mode, iA + j, oA[j]);
                    emit_id(a, clear_mode, iB + j, oB[j]);
                }
            }
        }
        if (gn >= ngroups) break;
        grp = gn;
        cur = nxt;
    }
}

__global__ void __launch_bounds__(kEncThreads, 3) dec_unpack_kernel(DecArgs a)
{
    extern __shared__ __align__(128) uint8_t dbuf[];  // [kEncWarps][2][kDecStage]
    __shared__ __align__(8) unsigned long long bars[kEncWarps][2];
    __shared__ uint32_t patch[kEncWarps][kBlock];  // patched: one block's high parts by slot
    dec_unpack_body(a, dbuf, bars, patch);
}

// A small frontier's whole codec stage in one CTA (at most kSmallTiles tiles of ids): W and P of
// the FQ encode with its FB mirror, then D0, D1 and D2 of the decode -- the same steps as the five
// launches of the general path, each starting after the previous one's writes (CTA barriers), the
// decode reading only the stream bytes just written.  For a frontier this small the general path
// is bound by its launches and their grid-wide handoffs, not by its work.
__global__ void __launch_bounds__(kEncThreads, 1) small_codec_kernel(EncArgs ea, DecArgs da)
{
    extern __shared__ __align__(128) uint8_t dbuf[];  // [kEncWarps][2][kDecStage]
    __shared__ __align__(8) unsigned long long bars[kEncWarps][2];
    __shared__ uint32_t patch[kEncWarps][kBlock];
    __shared__ uint32_t ws[kEncWarps], we[kEncWarps];
    __shared__ uint32_t hist[1][33];
    __shared__ uint32_t pk[kEncWarps][4 * 32 + 4];
    Ctl *c = ea.s.ctl;
    const uint64_t n = enc_count(ea), nb = dcdiv(n, kBlock), ntiles = dcdiv(nb, kTileBlocks);
    if (ntiles > kSmallTiles) {  // the caller picks this path only for small frontiers
        if (threadIdx.x == 0) set_error(c, FQ_EINVAL, kWhereEncWidths, n);
        return;
    }
    for (uint64_t t = 0; t < ntiles; t++) enc_widths_tile<false>(ea, n, nb, t, ws, we, hist);  // ends in a barrier
    unsigned long long total = 0;
    for (uint64_t t = 0; t < ntiles; t++) total += ea.s.tile_sum[t];
    const EncPlan p = enc_decide(ea, n, nb, total, 0ull, *reinterpret_cast<const volatile int32_t *>(&c->code));
    if (threadIdx.x == 0) enc_finalize(ea, n, nb, total, 0ull, p);
    if (!p.fatal) {
        enc_raw_bodies(ea, p, n, threadIdx.x, blockDim.x);
        if (p.mode == kModePacked || p.mode2 == kModePacked) {
            unsigned long long prefix = 0;
            for (uint64_t t = 0; t < ntiles; t++) {
                enc_pack_tile<false>(ea, p, n, nb, total, 0ull, t, prefix, 0ull, pk);
                prefix += ea.s.tile_sum[t];
            }
        }
    }
    __syncthreads();  // the stream and its size are written
    if (p.fatal || p.err != FQ_OK) return;  // the encode's error is the stage's status
    dec_tile_sums(da);
    __syncthreads();
    dec_plan_body<kEncThreads>(da);
    __syncthreads();
    dec_unpack_body(da, dbuf, bars, patch);
}

__global__ void reset_status_kernel(Scratch s) { reset_scratch_device(s); }

uint32_t grid_for(uint64_t items, uint32_t per_cta, uint32_t max_ctas)
{
    uint64_t g = cdiv(std::max<uint64_t>(items, 1), per_cta);
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(g, 1), max_ctas);
}

uint64_t enc_tiles(uint64_t n) { return cdiv(cdiv(n, kBlock), kTileBlocks); }

// CTAs of `kernel` (static shared memory only) resident on the whole GPU at once, cached per device
// in `cache`: a grid-stride kernel launched with exactly this many CTAs runs in a single wave.
template <typename K>
uint64_t resident_grid(K kernel, int threads, std::atomic<int> *cache)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return (uint64_t)num_sms();
    int per_sm = cache[dev].load(std::memory_order_relaxed);
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm <= 0)
            per_sm = 1;
        cache[dev].store(per_sm, std::memory_order_relaxed);
    }
    return (uint64_t)per_sm * num_sms();
}

cudaError_t prepare_unpack()
{
    static std::atomic<bool> done[64];
    return allow_smem(dec_unpack_kernel, kDecSmem, done);
}

// W then P, with grids of at most one resident wave (both kernels stride over their tiles).
cudaError_t launch_encode(EncArgs a, uint64_t n_max, cudaStream_t st)
{
    static std::atomic<int> occ_w[64], occ_p[64];
    const uint64_t tiles = std::max<uint64_t>(1, enc_tiles(n_max));
    uint64_t raw_items = cdiv(n_max, 4) * 4;  // the raw bodies P may have to copy instead
    if (a.fb) raw_items = std::max<uint64_t>(raw_items, cdiv(a.nbits, 64));
    if (a.m_out) raw_items = std::max<uint64_t>(raw_items, cdiv(a.m_nbits, 64));
    static std::atomic<int> occ_wx[64], occ_px[64];
    const uint64_t pack_items = std::max<uint64_t>(tiles, cdiv(raw_items, kEncThreads));
    if (a.px) {
        const uint32_t gw = tuned_grid(FQ_TUNE_ENC_WIDTHS, n_max, resident_grid(enc_widths_kernel<true>, kEncThreads, occ_wx), tiles);
        const uint32_t gp = tuned_grid(FQ_TUNE_ENC_PACK, n_max, resident_grid(enc_pack_kernel<true>, kEncThreads, occ_px), pack_items);
        enc_widths_kernel<true><<<gw, kEncThreads, 0, st>>>(a);
        enc_pack_kernel<true><<<gp, kEncThreads, 0, st>>>(a);
        return cudaGetLastError();
    }
    const uint32_t gw = tuned_grid(FQ_TUNE_ENC_WIDTHS, n_max, resident_grid(enc_widths_kernel<false>, kEncThreads, occ_w), tiles);
    const uint32_t gp = tuned_grid(FQ_TUNE_ENC_PACK, n_max, resident_grid(enc_pack_kernel<false>, kEncThreads, occ_p), pack_items);
    enc_widths_kernel<false><<<gw, kEncThreads, 0, st>>>(a);
    enc_pack_kernel<false><<<gp, kEncThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------ internal launches

cudaError_t reset_status(const Scratch &s, uint64_t max_ids, cudaStream_t st)
{
    (void)max_ids;
    reset_status_kernel<<<1, 1, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t encode_fq(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint64_t n_max, uint8_t *out,
                      uint64_t cap, uint64_t *out_bytes, const Scratch &s, cudaStream_t st, bool px)
{
    EncArgs a{ids, n_host, n_dev, out, cap, out_bytes, 0, 0, nullptr, s, nullptr, 0, nullptr, nullptr, 0, px ? 1 : 0};
    return launch_encode(a, n_dev ? n_max : n_host, st);
}

cudaError_t encode_fq_mirror(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint64_t n_max,
                             uint8_t *out, uint64_t cap, uint64_t *out_bytes, const Mirror &m, const Scratch &s,
                             cudaStream_t st)
{
    EncArgs a{ids, n_host, n_dev, out, cap, out_bytes, 0, 0, nullptr, s, m.out, m.cap, m.out_bytes, m.words, m.nbits, 0};
    return launch_encode(a, n_dev ? n_max : n_host, st);
}

cudaError_t codec_small(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint8_t *out, uint64_t cap,
                        uint64_t *out_bytes, const Mirror &m, uint32_t *ids_out, uint64_t dec_cap, uint64_t *n_out,
                        const Scratch &s, cudaStream_t st)
{
    static std::atomic<bool> done[64];
    FQ_CUDA_TRY(allow_smem(small_codec_kernel, kDecSmem, done));
    const EncArgs ea{ids, n_host, n_dev, out, cap, out_bytes, 0, 0, nullptr, s, m.out, m.cap, m.out_bytes, m.words,
                     m.nbits, 0};
    const DecArgs da{out, 0, out_bytes, ids_out, dec_cap, n_out, 0, nullptr, 0, s};
    small_codec_kernel<<<1, kEncThreads, kDecSmem, st>>>(ea, da);
    return cudaGetLastError();
}

cudaError_t encode_fb_positions(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap,
                                uint64_t *out_bytes, const Scratch &s, cudaStream_t st)
{
    EncArgs a{s.positions, 0, reinterpret_cast<const uint64_t *>(&s.ctl->n), out, cap, out_bytes, 1, nbits, words, s,
              nullptr, 0, nullptr, nullptr, 0, 0};
    return launch_encode(a, nbits / 2 + 1, st);
}

cudaError_t encode_fb(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap, uint64_t *out_bytes,
                      const Scratch &s, cudaStream_t st)
{
    const uint64_t nwords = cdiv(nbits, 64);
    const uint32_t btiles = (uint32_t)std::max<uint64_t>(1, cdiv(nwords, kTileWords));
    bits_count_kernel<<<btiles, kBitThreads, 0, st>>>(words, nbits, s.btile_cnt);
    fb_plan_kernel<<<1, kScanThreads, 0, st>>>(nbits, s);
    bits_extract_kernel<<<btiles, kBitThreads, 0, st>>>(words, nbits, s);
    return encode_fb_positions(words, nbits, out, cap, out_bytes, s, st);
}

// The tile-sum kernel's grid: four tiles per CTA per pass, at most two CTAs per SM (its last CTA's
// ticket is one atomic per CTA on a single counter, and small streams need few CTAs).
static uint32_t dec_tiles_grid(uint64_t tiles)
{
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(cdiv(tiles, kEncThreads / kTileBlocks), 2 * (uint64_t)num_sms()));
}

cudaError_t decode_fq(const uint8_t *in, uint64_t in_bytes_host, const uint64_t *in_bytes_dev, uint32_t *ids,
                      uint64_t cap, uint64_t *n_out, const Scratch &s, cudaStream_t st)
{
    DecArgs a{in, in_bytes_host, in_bytes_dev, ids, cap, n_out, 0, nullptr, 0, s};
    const uint64_t tiles = std::max<uint64_t>(1, enc_tiles(cap));
    dec_tiles_kernel<<<dec_tiles_grid(tiles), kEncThreads, 0, st>>>(a);
    FQ_CUDA_TRY(prepare_unpack());
    dec_unpack_kernel<<<tuned_grid(FQ_TUNE_DEC_UNPACK, cap, grid_for(std::max(tiles * kEncThreads, cap), kEncThreads, 3 * num_sms()),
                                   cdiv(std::max(tiles * kEncThreads, cap), kEncThreads)), kEncThreads, kDecSmem,
                        st>>>(a);
    return cudaGetLastError();
}

cudaError_t decode_fb(const uint8_t *in, uint64_t in_bytes_host, const uint64_t *in_bytes_dev, uint64_t *words,
                      uint64_t nbits, const Scratch &s, cudaStream_t st)
{
    DecArgs a{in, in_bytes_host, in_bytes_dev, nullptr, nbits, nullptr, 1, words, nbits, s};
    const uint64_t tiles = std::max<uint64_t>(1, enc_tiles(nbits));
    dec_tiles_kernel<<<dec_tiles_grid(tiles), kEncThreads, 0, st>>>(a);
    const uint64_t nwords = cdiv(nbits, 64);
    fb_init_kernel<<<grid_for(nwords, 256, 4 * num_sms()), 256, 0, st>>>(a);
    FQ_CUDA_TRY(prepare_unpack());
    dec_unpack_kernel<<<grid_for(std::max(tiles * kEncThreads, nbits), kEncThreads, 3 * num_sms()), kEncThreads,
                        kDecSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fq

// ------------------------------------------------------------------ C ABI

using namespace fq;

namespace {
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
fq_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return FQ_OK;
    note_cuda_error(e, __LINE__);
    return FQ_ECUDA;
}
}  // namespace

extern "C" {

const char *fq_status_string(fq_status s)
{
    switch (s) {
    case FQ_OK: return "FQ_OK";
    case FQ_EINVAL: return "FQ_EINVAL";
    case FQ_ENOMEM: return "FQ_ENOMEM";
    case FQ_ENOSPC: return "FQ_ENOSPC";
    case FQ_ECORRUPT: return "FQ_ECORRUPT";
    case FQ_EUNSORTED: return "FQ_EUNSORTED";
    case FQ_ETIMEOUT: return "FQ_ETIMEOUT";
    case FQ_ECUDA: return "FQ_ECUDA";
    case FQ_EBUSY: return "FQ_EBUSY";
    default: return "FQ_UNKNOWN";
    }
}

int fq_last_cuda_error(int *line)
{
    if (line) *line = g_last_cuda_line;
    return g_last_cuda_error;
}

uint64_t fq_queue_bound(uint64_t n) { return 16u + pad16(4u * n); }

uint64_t fq_bitmap_bound(uint64_t nbits) { return 16u + pad16(8u * cdiv(nbits, 64)); }

uint64_t fq_workspace_bytes(uint64_t max_ids, uint64_t max_nbits) { return workspace_bytes(max_ids, max_nbits); }

fq_status fq_work_status(const void *d_work, void *stream, uint64_t *h_detail)
{
    if (!d_work) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return FQ_ECUDA;
    fq_device_status rec;
    if (cudaMemcpy(&rec, d_work, sizeof(rec), cudaMemcpyDeviceToHost) != cudaSuccess) return FQ_ECUDA;
    if (h_detail) *h_detail = rec.code == FQ_OK ? 0u : rec.detail;
    return rec.code;
}

fq_status fq_frontier_encode(const uint32_t *d_ids, uint64_t n, uint8_t *d_out, uint64_t cap, uint64_t *d_out_bytes,
                             void *d_work, uint64_t work_bytes, void *stream)
{
    if ((n && !d_ids) || !d_out || !d_out_bytes || !d_work) return FQ_EINVAL;
    if (n > 0xffffffffull || !aligned16(d_ids) || !aligned16(d_out) || !aligned16(d_work)) return FQ_EINVAL;
    if (!workspace_fits(work_bytes, n, 0)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch s = carve(d_work, n, 0);
    cudaError_t e = reset_status(s, n, st);
    if (e == cudaSuccess) e = encode_fq(d_ids, n, nullptr, n, d_out, cap, d_out_bytes, s, st);
    return cuda_status(e);
}

fq_status fq_tune_set(uint32_t site, uint32_t size_class, uint32_t ctas_per_sm)
{
    if (site >= FQ_TUNE_NUM_SITES || size_class > FQ_TUNE_MAX_CLASS || ctas_per_sm > 32u) return FQ_EINVAL;
    if (g_tune[site][size_class].exchange((uint8_t)ctas_per_sm) != (uint8_t)ctas_per_sm) g_tune_generation++;
    return FQ_OK;
}

uint32_t fq_tune_get(uint32_t site, uint32_t size_class)
{
    if (site >= FQ_TUNE_NUM_SITES || size_class > FQ_TUNE_MAX_CLASS) return 0u;
    return g_tune[site][size_class].load();
}

fq_status fq_frontier_encode_px(const uint32_t *d_ids, uint64_t n, uint8_t *d_out, uint64_t cap,
                                uint64_t *d_out_bytes, void *d_work, uint64_t work_bytes, void *stream)
{
    if ((n && !d_ids) || !d_out || !d_out_bytes || !d_work) return FQ_EINVAL;
    if (n > 0xffffffffull || !aligned16(d_ids) || !aligned16(d_out) || !aligned16(d_work)) return FQ_EINVAL;
    if (!workspace_fits(work_bytes, n, 0)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch s = carve(d_work, n, 0);
    EncArgs a{d_ids, n, nullptr, d_out, cap, d_out_bytes, 0, 0, nullptr, s, nullptr, 0, nullptr, nullptr, 0, 1};
    cudaError_t e = reset_status(s, n, st);
    if (e == cudaSuccess) e = launch_encode(a, n, st);
    return cuda_status(e);
}

fq_status fq_frontier_decode(const uint8_t *d_in, uint64_t in_bytes, uint32_t *d_ids, uint64_t cap, uint64_t *d_n,
                             void *d_work, uint64_t work_bytes, void *stream)
{
    if (!d_in || (cap && !d_ids) || !d_n || !d_work) return FQ_EINVAL;
    if (!aligned16(d_in) || !aligned16(d_ids) || !aligned16(d_work) || cap > 0xffffffffull) return FQ_EINVAL;
    if (!workspace_fits(work_bytes, cap, 0)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch s = carve(d_work, cap, 0);
    cudaError_t e = reset_status(s, 0, st);
    if (e == cudaSuccess) e = decode_fq(d_in, in_bytes, nullptr, d_ids, cap, d_n, s, st);
    return cuda_status(e);
}

fq_status fq_bitmap_encode(const uint64_t *d_words, uint64_t nbits, uint8_t *d_out, uint64_t cap, uint64_t *d_out_bytes,
                           void *d_work, uint64_t work_bytes, void *stream)
{
    if ((nbits && !d_words) || !d_out || !d_out_bytes || !d_work) return FQ_EINVAL;
    if (nbits > 0x100000000ull || !aligned16(d_words) || !aligned16(d_out) || !aligned16(d_work)) return FQ_EINVAL;
    if (!workspace_fits(work_bytes, 0, nbits)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch s = carve(d_work, 0, nbits);
    cudaError_t e = reset_status(s, nbits / 2 + 1, st);
    if (e == cudaSuccess) e = encode_fb(d_words, nbits, d_out, cap, d_out_bytes, s, st);
    return cuda_status(e);
}

fq_status fq_bitmap_decode(const uint8_t *d_in, uint64_t in_bytes, uint64_t *d_words, uint64_t nbits, void *d_work,
                           uint64_t work_bytes, void *stream)
{
    if (!d_in || (nbits && !d_words) || !d_work) return FQ_EINVAL;
    if (nbits > 0x100000000ull || !aligned16(d_in) || !aligned16(d_words) || !aligned16(d_work)) return FQ_EINVAL;
    if (!workspace_fits(work_bytes, 0, nbits)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch s = carve(d_work, 0, nbits);
    cudaError_t e = reset_status(s, 0, st);
    if (e == cudaSuccess) e = decode_fb(d_in, in_bytes, nullptr, d_words, nbits, s, st);
    return cuda_status(e);
}

}  // extern "C"
