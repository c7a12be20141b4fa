// codec.cu -- GPU kernels of the frontier codec (FQ queue streams, FB bitmap streams) and its
// C ABI.  Delta coding + frame-of-reference binary packing in blocks of 128 ids, the integer
// codec the thesis wraps around its per-level exchanges (sec. 5.2 "Binary packing" and "Delta
// compression"; S4-BP128 chosen in sec. 5.3; width = bit length, Eq. 6-7).  The byte layout is
// this library's own (documented in include/fqbfs.h), designed for warp-per-block GPU decoding:
// every block's payload is 16*b_k bytes, so it starts on a 16-byte boundary and a warp moves
// it with b_k 128-bit accesses.
//
// Encode = 3 launches: widths (one warp per 128-id block: gaps, max, bit length, sortedness),
// plan (one CTA: scan of per-tile width sums, packed/raw choice, headers), pack (one warp per
// block: bits OR-ed into a shared-memory staging row, then b_k vector stores).
// Decode = 2 launches: plan (one CTA: header and size validation, scan of widths into per-block
// payload offsets), unpack (one warp per block: b_k vector loads, slot extraction, warp prefix
// sum of the gaps, 128-bit stores).
#include <algorithm>
#include <cstdio>

#include "fq_common.cuh"

namespace fq {

// ------------------------------------------------------------------ workspace layout

namespace {
struct Layout {
    uint64_t widths, bases, block_off, tile_sum, tile_off, btile_cnt, btile_off, positions, total;
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
    s.ids_cap = L.ids_cap;
    s.nbits_cap = max_nbits;
    s.nb_cap = L.nb_cap;
    s.etiles_cap = L.etiles_cap;
    s.btiles_cap = L.btiles_cap;
    s.pos_cap = L.pos_cap;
    return s;
}

int num_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
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
__device__ __forceinline__ uint64_t dpad16(uint64_t b) { return (b + 15u) & ~uint64_t(15); }
__device__ __forceinline__ uint64_t dcdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint32_t ld_u32(const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Four consecutive ids starting at i (a multiple of 4); ids past n are flagged invalid.
__device__ __forceinline__ void load4(const uint32_t *ids, uint64_t i, uint64_t n, uint32_t v[4], bool valid[4])
{
    if (i + 3 < n) {
        uint4 q = *reinterpret_cast<const uint4 *>(ids + i);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        valid[0] = valid[1] = valid[2] = valid[3] = true;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            valid[j] = (i + j) < n;
            v[j] = valid[j] ? ids[i + j] : 0u;
        }
    }
}

// Gaps of the four slots lane*4 .. lane*4+3 of block k: slot 0 of the block is 0; slot j >= 1
// is v[j] - v[j-1] - 1; slots past n are 0.  Also reports the first unsorted index.
__device__ __forceinline__ void block_gaps(const uint32_t *ids, uint64_t k, uint64_t n, uint32_t lane, uint32_t v[4],
                                           uint32_t g[4], unsigned long long *bad)
{
    bool valid[4];
    const uint64_t i0 = k * kBlock + lane * 4u;
    load4(ids, i0, n, v, valid);
    uint32_t prev = __shfl_up_sync(0xffffffffu, v[3], 1);
    bool has_prev = lane > 0;
    if (lane == 0 && k > 0) {
        prev = ids[k * kBlock - 1];
        has_prev = true;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        g[j] = 0;
        if (!valid[j]) continue;
        const uint32_t p = (j == 0) ? prev : v[j - 1];
        const bool hp = (j == 0) ? has_prev : true;
        if (hp) {
            if (v[j] <= p) {
                *bad = min(*bad, (unsigned long long)(i0 + j));
            } else if (!(lane == 0 && j == 0)) {
                g[j] = v[j] - p - 1u;
            }
        }
    }
}

// E1: one warp per block -- width b_k, base_k, per-tile width sums.
__global__ void __launch_bounds__(kEncThreads) enc_widths_kernel(EncArgs a)
{
    const uint64_t n = enc_count(a);
    const uint64_t nb = dcdiv(n, kBlock);
    const uint32_t tile = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    if ((uint64_t)tile * kTileBlocks >= nb) return;
    __shared__ uint32_t wsum[kEncWarps];
    uint32_t sum = 0;
    unsigned long long bad = ~0ull;
    for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
        const uint64_t k = (uint64_t)tile * kTileBlocks + warp * kBlocksPerWarp + i;
        if (k >= nb) break;
        uint32_t v[4], g[4];
        block_gaps(a.ids, k, n, lane, v, g, &bad);
        const uint32_t mg = warp_max(max(max(g[0], g[1]), max(g[2], g[3])));
        const uint32_t b = bitlen32(mg);
        if (lane == 0) {
            a.s.widths[k] = (uint8_t)b;
            a.s.bases[k] = v[0];
        }
        sum += b;
    }
    if (lane == 0) wsum[warp] = sum;
    if (bad != ~0ull) set_error(a.s.ctl, FQ_EUNSORTED, kWhereEncWidths, bad);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < kEncWarps; w++) t += wsum[w];
        a.s.tile_sum[tile] = t;
    }
}

// E2: one CTA -- exclusive scan of the tile width sums, packed/raw (and FB raw) decision,
// capacity check, headers.
__global__ void __launch_bounds__(kScanThreads) enc_plan_kernel(EncArgs a)
{
    __shared__ unsigned long long sm[33];
    const uint64_t n = enc_count(a);
    const uint64_t nb = dcdiv(n, kBlock);
    const uint64_t ntiles = dcdiv(nb, kTileBlocks);
    const uint64_t chunk = dcdiv(ntiles, kScanThreads);
    const uint64_t t0 = (uint64_t)threadIdx.x * chunk, t1 = min(ntiles, t0 + chunk);
    unsigned long long local = 0, total = 0;
    for (uint64_t t = t0; t < t1; t++) local += a.s.tile_sum[t];
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t t = t0; t < t1; t++) {
        a.s.tile_off[t] = (uint32_t)run;
        run += a.s.tile_sum[t];
    }
    if (threadIdx.x != 0) return;
    Ctl *c = a.s.ctl;
    c->n = n;
    c->nb = nb;
    c->total_b = total;
    c->fq_offset = a.fb ? 16u : 0u;
    if (c->code != FQ_OK) {
        c->mode = kModeNone;
        *a.out_bytes = 0;
        return;
    }
    const uint64_t packed = 16u + dpad16(5u * nb) + 16u * total;
    const uint64_t raw = 16u + dpad16(4u * n);
    const bool is_packed = n > 0 && packed < raw;
    const uint64_t fq_size = is_packed ? packed : raw;
    uint32_t mode = is_packed ? kModePacked : kModeRaw;
    uint64_t size = fq_size;
    if (a.fb) {
        const uint64_t fb_raw = 16u + dpad16(8u * dcdiv(a.nbits, 64));
        if (16u + fq_size >= fb_raw) {
            mode = kModeFbRaw;
            size = fb_raw;
        } else {
            size = 16u + fq_size;
        }
    }
    if (size > a.cap) {
        set_error(c, FQ_ENOSPC, kWhereEncPlan, size);
        c->mode = kModeNone;
        *a.out_bytes = size;
        return;
    }
    uint32_t *h = reinterpret_cast<uint32_t *>(a.out);
    if (a.fb) {
        h[0] = kMagicBitmap;
        h[1] = (mode == kModeFbRaw) ? kFbRaw : c->fb_mode;
        h[2] = (uint32_t)(a.nbits & 0xffffffffu);
        h[3] = (uint32_t)(a.nbits >> 32);
        h += 4;
    }
    if (mode == kModePacked) {
        h[0] = kMagicPacked; h[1] = (uint32_t)n; h[2] = (uint32_t)nb; h[3] = (uint32_t)(4u * total);
    } else if (mode == kModeRaw) {
        h[0] = kMagicRaw; h[1] = (uint32_t)n; h[2] = 0u; h[3] = (uint32_t)n;
    }
    c->mode = mode;
    c->out_bytes = size;
    *a.out_bytes = size;
}

// E3: one warp per block -- pack the gaps of block k into 4*b_k words.
__global__ void __launch_bounds__(kEncThreads) enc_pack_kernel(EncArgs a)
{
    const Ctl *c = a.s.ctl;
    const uint32_t mode = c->mode;
    if (mode != kModePacked && mode != kModeRaw) return;
    const uint64_t n = c->n, nb = c->nb;
    uint8_t *fq = a.out + c->fq_offset;
    const uint32_t tile = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;

    if (mode == kModeRaw) {
        const uint64_t per_tile = (uint64_t)kTileBlocks * kBlock;
        const uint64_t i0 = (uint64_t)tile * per_tile, i1 = min(n, i0 + per_tile);
        uint32_t *dst = reinterpret_cast<uint32_t *>(fq + 16);
        for (uint64_t i = i0 + 4u * threadIdx.x; i < i1; i += 4u * kEncThreads) {
            if (i + 3 < n) {
                *reinterpret_cast<uint4 *>(dst + i) = *reinterpret_cast<const uint4 *>(a.ids + i);
            } else {
                for (uint64_t j = i; j < n; j++) dst[j] = a.ids[j];
            }
        }
        // zero the pad [16 + 4n, 16 + pad16(4n)) -- owned by the tile holding id n-1 (tile 0 if n == 0)
        const uint64_t last_tile = n ? (n - 1) / per_tile : 0;
        if (tile == last_tile && threadIdx.x == 0)
            for (uint64_t j = n; j < dcdiv(n, 4) * 4; j++) dst[j] = 0u;
        return;
    }

    const uint64_t ntiles = dcdiv(nb, kTileBlocks);
    if (tile >= ntiles) return;
    __shared__ uint32_t sb[kTileBlocks];     // exclusive prefix of widths inside the tile
    __shared__ uint8_t swidth[kTileBlocks];
    __shared__ uint32_t pk[kEncWarps][4 * 32 + 4];
    if (threadIdx.x < kTileBlocks) {
        const uint64_t k = (uint64_t)tile * kTileBlocks + threadIdx.x;
        const uint32_t b = (k < nb) ? a.s.widths[k] : 0u;
        swidth[threadIdx.x] = (uint8_t)b;
        if (k < nb) {
            reinterpret_cast<uint32_t *>(fq + 16)[k] = a.s.bases[k];
            fq[16 + 4 * nb + k] = (uint8_t)b;
        }
    }
    if (tile == 0 && threadIdx.x >= kTileBlocks && threadIdx.x < kTileBlocks + 16) {
        const uint64_t p = 16u + 5u * nb + (threadIdx.x - kTileBlocks);
        if (p < 16u + dpad16(5u * nb)) fq[p] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r = 0;
        for (uint32_t i = 0; i < kTileBlocks; i++) {
            sb[i] = r;
            r += swidth[i];
        }
    }
    __syncthreads();
    const uint64_t payload = 16u + dpad16(5u * nb);
    const uint64_t tile_base = a.s.tile_off[tile];
    unsigned long long bad = ~0ull;
    for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
        const uint32_t local = warp * kBlocksPerWarp + i;
        const uint64_t k = (uint64_t)tile * kTileBlocks + local;
        if (k >= nb) break;
        const uint32_t b = swidth[local];
        if (b == 0) continue;
        uint32_t v[4], g[4];
        block_gaps(a.ids, k, n, lane, v, g, &bad);
#pragma unroll
        for (int j = 0; j < 4; j++) pk[warp][4 * lane + j] = 0u;
        if (lane == 0) pk[warp][128] = 0u;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (g[j] == 0u) continue;
            const uint32_t pos = (4u * lane + j) * b;
            const uint32_t w0 = pos >> 5, sh = pos & 31u;
            atomicOr(&pk[warp][w0], g[j] << sh);
            if (sh + b > 32u) atomicOr(&pk[warp][w0 + 1], g[j] >> (32u - sh));
        }
        __syncwarp();
        if (lane < b) {
            uint4 q = make_uint4(pk[warp][4 * lane], pk[warp][4 * lane + 1], pk[warp][4 * lane + 2], pk[warp][4 * lane + 3]);
            *reinterpret_cast<uint4 *>(fq + payload + 16u * (tile_base + sb[local] + lane)) = q;
        }
        __syncwarp();
    }
}

// FB raw container: copy the words (tail bits cleared) behind the 16-byte header.
__global__ void fb_raw_kernel(EncArgs a)
{
    if (a.s.ctl->mode != kModeFbRaw) return;
    const uint64_t nwords = dcdiv(a.nbits, 64);
    uint64_t *dst = reinterpret_cast<uint64_t *>(a.out + 16);
    const uint64_t padded = dcdiv(nwords, 2) * 2;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < padded; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t w = 0;
        if (i < nwords) {
            w = a.fb_words[i];
            const uint32_t tail = (uint32_t)(a.nbits & 63u);
            if (i == nwords - 1 && tail) w &= (1ull << tail) - 1ull;
        }
        dst[i] = w;
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

// D1: one CTA -- validate the container and FQ header, scan widths into block offsets.
__global__ void __launch_bounds__(kScanThreads) dec_plan_kernel(DecArgs a)
{
    __shared__ unsigned long long sm[33];
    __shared__ int s_ok;
    __shared__ uint32_t s_mode, s_fbmode;
    __shared__ unsigned long long s_n, s_nb, s_words, s_fq_bytes, s_fq_off, s_bad;
    __shared__ int s_over;
    Ctl *c = a.s.ctl;
    const uint64_t in_bytes = a.in_bytes_dev ? *a.in_bytes_dev : a.in_bytes_host;
    const uint64_t limit = a.fb ? a.nbits : a.cap;
    if (threadIdx.x == 0) {
        s_ok = 1;
        s_over = 0;
        s_bad = ~0ull;
        s_mode = kModeNone;
        s_fbmode = kFbRaw;
        s_fq_off = 0;
        s_fq_bytes = in_bytes;
        s_n = s_nb = s_words = 0;
        if (a.fb) {
            if (in_bytes < 16 || ld_u32(a.in) != kMagicBitmap ||
                ((uint64_t)ld_u32(a.in + 8) | ((uint64_t)ld_u32(a.in + 12) << 32)) != a.nbits) {
                s_ok = 0;
            } else {
                const uint32_t m = ld_u32(a.in + 4);
                if (m == kFbRaw) {
                    if (in_bytes != 16u + dpad16(8u * dcdiv(a.nbits, 64))) s_ok = 0;
                    else s_mode = kModeFbRaw;
                } else if (m == kFbSet || m == kFbClear) {
                    s_fbmode = m;
                    s_fq_off = 16;
                    s_fq_bytes = in_bytes - 16u;
                } else {
                    s_ok = 0;
                }
            }
        }
        if (s_ok && s_mode != kModeFbRaw) {
            const uint8_t *fq = a.in + s_fq_off;
            const uint64_t fqb = s_fq_bytes;
            if (fqb < 16) {
                s_ok = 0;
            } else {
                const uint32_t magic = ld_u32(fq);
                const uint64_t n = ld_u32(fq + 4), nb = ld_u32(fq + 8), words = ld_u32(fq + 12);
                s_n = n; s_nb = nb; s_words = words;
                if (n > limit) {
                    s_ok = 0;  // more ids than the output (or the scratch) holds: nothing is written
                    s_over = 1;
                } else if (magic == kMagicRaw) {
                    if (nb != 0 || words != n || fqb != 16u + dpad16(4u * n)) s_ok = 0;
                    else {
                        for (uint64_t i = 16u + 4u * n; i < fqb; i++)
                            if (fq[i]) s_ok = 0;
                        s_mode = kModeRaw;
                    }
                } else if (magic == kMagicPacked) {
                    if (nb != dcdiv(n, kBlock) || n == 0 || fqb < 16u + dpad16(5u * nb)) s_ok = 0;
                    else {
                        for (uint64_t i = 16u + 5u * nb; i < 16u + dpad16(5u * nb); i++)
                            if (fq[i]) s_ok = 0;
                        s_mode = kModePacked;
                    }
                } else {
                    s_ok = 0;
                }
            }
        }
    }
    __syncthreads();
    if (s_ok && s_mode == kModePacked) {
        const uint8_t *fq = a.in + s_fq_off;
        const uint64_t nb = s_nb;
        const uint8_t *wd = fq + 16 + 4 * nb;
        const uint64_t chunk = dcdiv(nb, kScanThreads);
        const uint64_t k0 = (uint64_t)threadIdx.x * chunk, k1 = min(nb, k0 + chunk);
        unsigned long long local = 0, total = 0;
        for (uint64_t k = k0; k < k1; k++) {
            const uint32_t b = wd[k];
            if (b > 32u) atomicMin(&s_bad, (unsigned long long)(16 + 4 * nb + k));
            local += b;
        }
        unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
        for (uint64_t k = k0; k < k1; k++) {
            a.s.block_off[k] = (uint32_t)run;
            run += wd[k];
        }
        if (threadIdx.x == 0) {
            if (s_bad != ~0ull || s_words != 4u * total || s_fq_bytes != 16u + dpad16(5u * nb) + 16u * total)
                s_ok = 0;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    c->fq_offset = s_fq_off;
    c->fb_mode = s_fbmode;
    c->n = s_n;
    c->nb = s_nb;
    if (s_over) {
        set_error(c, a.fb ? FQ_ECORRUPT : FQ_ENOSPC, kWhereDecPlan, s_n);
        c->mode = kModeNone;
        if (a.n_out) *a.n_out = s_n;
        return;
    }
    if (!s_ok) {
        set_error(c, FQ_ECORRUPT, kWhereDecPlan, s_bad != ~0ull ? s_bad : 0ull);
        c->mode = kModeNone;
        if (a.n_out) *a.n_out = 0;
        return;
    }
    c->mode = s_mode;
    if (a.n_out) *a.n_out = s_n;
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

// D2: one warp per block -- unpack, prefix-sum the gaps, validate, write ids (or bits).
__global__ void __launch_bounds__(kEncThreads) dec_unpack_kernel(DecArgs a)
{
    const Ctl *c = a.s.ctl;
    const uint32_t mode = c->mode;
    if (mode != kModePacked && mode != kModeRaw) return;
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

    __shared__ uint32_t pk[kEncWarps][4 * 32 + 4];
    const uint8_t *wd = fq + 16 + 4 * nb;
    const uint32_t *bases = reinterpret_cast<const uint32_t *>(fq + 16);
    const uint8_t *payload = fq + 16 + dpad16(5u * nb);
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t k = gwarp; k < nb; k += nwarps) {
        const uint32_t b = wd[k];
        const uint64_t base = bases[k];
        if (lane < b) {
            const uint4 q = *reinterpret_cast<const uint4 *>(payload + 16u * ((uint64_t)a.s.block_off[k] + lane));
            pk[warp][4 * lane] = q.x; pk[warp][4 * lane + 1] = q.y; pk[warp][4 * lane + 2] = q.z; pk[warp][4 * lane + 3] = q.w;
        }
        if (lane == 0) pk[warp][4 * b] = 0u;
        __syncwarp();
        const uint32_t mask = (b == 32u) ? 0xffffffffu : ((1u << b) - 1u);
        unsigned long long inc[4];
        unsigned long long lsum = 0;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t slot = 4u * lane + j;
            uint32_t g = 0;
            if (b) {
                const uint32_t pos = slot * b, w0 = pos >> 5, sh = pos & 31u;
                const uint64_t two = ((uint64_t)pk[warp][w0 + 1] << 32) | pk[warp][w0];
                g = (uint32_t)(two >> sh) & mask;
            }
            const uint64_t i = k * kBlock + slot;
            if (slot == 0 || i >= n) {
                if (g) bad = true;
                inc[j] = 0;
            } else {
                inc[j] = (unsigned long long)g + 1ull;
            }
            lsum += inc[j];
        }
        const unsigned long long excl = warp_incl_scan64(lsum) - lsum;
        unsigned long long v = base + excl;
        const uint64_t i0 = k * kBlock + 4u * lane;
        uint32_t out[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            v += inc[j];
            out[j] = (uint32_t)v;
            if (i0 + j < n && v > 0xffffffffull) bad = true;
        }
        // a full block (k + 1 < nb) ends in lane 31's last slot: it must stay below the next base
        if (k + 1 < nb && lane == 31 && v >= (unsigned long long)bases[k + 1]) bad = true;
        if (bad) set_error(a.s.ctl, FQ_ECORRUPT, kWhereDecUnpack, k * kBlock);
        if (!a.fb && i0 + 3 < n) {
            *reinterpret_cast<uint4 *>(a.ids + i0) = make_uint4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (i0 + j < n) emit_id(a, clear_mode, i0 + j, out[j]);
        }
        __syncwarp();
    }
}

__global__ void reset_status_kernel(Ctl *c)
{
    c->code = FQ_OK;
    c->where = 0;
    c->detail = ~0ull;
    c->mode = kModeNone;
    c->fb_mode = kFbRaw;
    c->n = c->nb = c->popcount = c->total_b = c->out_bytes = c->fq_offset = 0;
}

uint32_t grid_for(uint64_t items, uint32_t per_cta, uint32_t max_ctas)
{
    uint64_t g = cdiv(std::max<uint64_t>(items, 1), per_cta);
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(g, 1), max_ctas);
}

}  // namespace

// ------------------------------------------------------------------ internal launches

cudaError_t reset_status(const Scratch &s, cudaStream_t st)
{
    reset_status_kernel<<<1, 1, 0, st>>>(s.ctl);
    return cudaGetLastError();
}

cudaError_t encode_fq(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint64_t n_max, uint8_t *out,
                      uint64_t cap, uint64_t *out_bytes, const Scratch &s, cudaStream_t st)
{
    EncArgs a{ids, n_host, n_dev, out, cap, out_bytes, 0, 0, nullptr, s};
    const uint64_t nmax = n_dev ? n_max : n_host;
    const uint32_t tiles = (uint32_t)std::max<uint64_t>(1, cdiv(cdiv(nmax, kBlock), kTileBlocks));
    enc_widths_kernel<<<tiles, kEncThreads, 0, st>>>(a);
    enc_plan_kernel<<<1, kScanThreads, 0, st>>>(a);
    enc_pack_kernel<<<tiles, kEncThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t encode_fb(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap, uint64_t *out_bytes,
                      const Scratch &s, cudaStream_t st)
{
    const uint64_t nwords = cdiv(nbits, 64);
    const uint32_t btiles = (uint32_t)std::max<uint64_t>(1, cdiv(nwords, kTileWords));
    bits_count_kernel<<<btiles, kBitThreads, 0, st>>>(words, nbits, s.btile_cnt);
    fb_plan_kernel<<<1, kScanThreads, 0, st>>>(nbits, s);
    bits_extract_kernel<<<btiles, kBitThreads, 0, st>>>(words, nbits, s);
    EncArgs a{s.positions, 0, reinterpret_cast<const uint64_t *>(&s.ctl->n), out, cap, out_bytes, 1, nbits, words, s};
    const uint64_t nmax = nbits / 2 + 1;
    const uint32_t tiles = (uint32_t)std::max<uint64_t>(1, cdiv(cdiv(nmax, kBlock), kTileBlocks));
    enc_widths_kernel<<<tiles, kEncThreads, 0, st>>>(a);
    enc_plan_kernel<<<1, kScanThreads, 0, st>>>(a);
    enc_pack_kernel<<<tiles, kEncThreads, 0, st>>>(a);
    fb_raw_kernel<<<grid_for(nwords, 256, 4 * num_sms()), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t decode_fq(const uint8_t *in, uint64_t in_bytes_host, const uint64_t *in_bytes_dev, uint32_t *ids,
                      uint64_t cap, uint64_t *n_out, const Scratch &s, cudaStream_t st)
{
    DecArgs a{in, in_bytes_host, in_bytes_dev, ids, cap, n_out, 0, nullptr, 0, s};
    dec_plan_kernel<<<1, kScanThreads, 0, st>>>(a);
    const uint64_t nb = cdiv(cap, kBlock);
    dec_unpack_kernel<<<grid_for(std::max(nb * 32, cap), kEncThreads, 8 * num_sms()), kEncThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t decode_fb(const uint8_t *in, uint64_t in_bytes_host, const uint64_t *in_bytes_dev, uint64_t *words,
                      uint64_t nbits, const Scratch &s, cudaStream_t st)
{
    DecArgs a{in, in_bytes_host, in_bytes_dev, nullptr, nbits, nullptr, 1, words, nbits, s};
    dec_plan_kernel<<<1, kScanThreads, 0, st>>>(a);
    const uint64_t nwords = cdiv(nbits, 64);
    fb_init_kernel<<<grid_for(nwords, 256, 4 * num_sms()), 256, 0, st>>>(a);
    const uint64_t nmax = nbits / 2 + 1;
    dec_unpack_kernel<<<grid_for(std::max(cdiv(nmax, kBlock) * 32, nmax), kEncThreads, 8 * num_sms()), kEncThreads, 0,
                        st>>>(a);
    return cudaGetLastError();
}

}  // namespace fq

// ------------------------------------------------------------------ C ABI

using namespace fq;

namespace {
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
fq_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FQ_OK : FQ_ECUDA; }
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
    cudaError_t e = reset_status(s, st);
    if (e == cudaSuccess) e = encode_fq(d_ids, n, nullptr, n, d_out, cap, d_out_bytes, s, st);
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
    cudaError_t e = reset_status(s, st);
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
    cudaError_t e = reset_status(s, st);
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
    cudaError_t e = reset_status(s, st);
    if (e == cudaSuccess) e = decode_fb(d_in, in_bytes, nullptr, d_words, nbits, s, st);
    return cuda_status(e);
}

}  // extern "C"
