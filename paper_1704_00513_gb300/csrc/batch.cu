// batch.cu -- the frontier codec over many independent segments in a fixed number of launches
// (fq_frontier_encode_batch / fq_frontier_decode_batch).
//
// The thesis groups many small transfers into one (custom MPI datatypes, sec. 6.5) and exchanges
// one compressed frontier per processor pair; here S sorted id segments of any lengths become S
// independent FQ streams (each exactly what fq_frontier_encode writes for that segment).  The ids
// of all segments are cut into tiles of 8192 (a segment's last tile may be short).  Encode: a plan
// (segment tiles, empty-segment headers, the tile -> segment map), a widths pass (each tile's sum
// of block widths), one scan of the tile sums, and a pack pass in which every tile finds its
// payload offset and its segment's packed/raw decision from the scan and writes its blocks, its
// table entries, and (first tile) the header -- 4 launches for any S, with no inter-CTA waiting.
// Decoding runs the inverse over all tiles of all streams (4 launches).
#include <algorithm>

#include "codec_dev.cuh"
#include "fq_common.cuh"

namespace fq {
namespace {

constexpr uint32_t kBTileIds = kTileBlocks * kBlock;  // 8192 ids per tile
constexpr uint32_t kDecStageB = kTileBlocks * 32u * 16u + 16u;
constexpr size_t kBatchDecSmem = 2 * (size_t)kDecStageB;

struct SegInfo {
    unsigned long long n;       // ids in the segment (decode: announced by the stream header)
    unsigned long long nb;      // 128-id blocks
    unsigned long long total_b; // sum of widths
    uint32_t mode;              // kMode* (kModeNone: nothing to write / invalid)
    uint32_t ok;
};

struct BatchScratch {
    Ctl *ctl;
    unsigned long long *tile_base;  // [S + 1] first global tile of each segment
    SegInfo *seg;                   // [S]
    unsigned long long *status;     // [T + 1] encode: exclusive prefix of the tile width sums
    uint32_t *tile_sum;             // [T] decode
    uint32_t *tile_off;             // [T] decode: segment-local payload offset (16-byte units)
    uint32_t *tile_seg;             // [T] the segment of each global tile (written by the plan kernels)
    uint64_t tiles_cap;
};

uint64_t batch_tiles_cap(uint64_t total_ids, uint64_t S) { return total_ids / kBTileIds + S + 1; }

uint64_t al256(uint64_t x) { return (x + 255u) / 256u * 256u; }

uint64_t batch_layout(uint64_t total_ids, uint64_t S, BatchScratch *b, void *base)
{
    const uint64_t T = batch_tiles_cap(total_ids, S);
    uint64_t o = 256;
    const uint64_t o_tb = o; o = al256(o + 8 * (S + 1));
    const uint64_t o_seg = o; o = al256(o + sizeof(SegInfo) * (S ? S : 1));
    const uint64_t o_st = o; o = al256(o + 8 * (T + 1));
    const uint64_t o_ts = o; o = al256(o + 4 * T);
    const uint64_t o_to = o; o = al256(o + 4 * T);
    const uint64_t o_sg = o; o = al256(o + 4 * T);
    if (b && base) {
        uint8_t *p = static_cast<uint8_t *>(base);
        b->ctl = reinterpret_cast<Ctl *>(p);
        b->tile_base = reinterpret_cast<unsigned long long *>(p + o_tb);
        b->seg = reinterpret_cast<SegInfo *>(p + o_seg);
        b->status = reinterpret_cast<unsigned long long *>(p + o_st);
        b->tile_sum = reinterpret_cast<uint32_t *>(p + o_ts);
        b->tile_off = reinterpret_cast<uint32_t *>(p + o_to);
        b->tile_seg = reinterpret_cast<uint32_t *>(p + o_sg);
        b->tiles_cap = T;
    }
    return o;
}



__device__ __forceinline__ void reset_ctl(Ctl *c)
{
    c->code = FQ_OK;
    c->where = 0;
    c->detail = ~0ull;
    c->mode = c->mode2 = kModeNone;
    c->fb_mode = kFbRaw;
    c->n = c->nb = c->popcount = c->total_b = c->out_bytes = c->fq_offset = c->out2_bytes = 0;
}

struct BEnc {
    const uint32_t *ids;
    const uint64_t *seg_off;
    uint32_t S;
    uint8_t *out;
    const uint64_t *out_off;
    uint64_t *out_bytes;
    BatchScratch b;
};

// ---- encode ----

// One CTA: segment sizes, tiles per segment and their prefix, the tile -> segment map, headers
// of empty segments.
__global__ void __launch_bounds__(kScanThreads) bat_plan_kernel(BEnc a)
{
    __shared__ unsigned long long sm[33];
    if (threadIdx.x == 0) reset_ctl(a.b.ctl);
    __syncthreads();
    const uint64_t S = a.S;
    const uint64_t chunk = dcdiv(S, kScanThreads);
    const uint64_t s0 = (uint64_t)threadIdx.x * chunk, s1 = min(S, s0 + chunk);
    unsigned long long local = 0, total = 0;
    for (uint64_t s = s0; s < s1; s++) {
        const uint64_t lo = a.seg_off[s], hi = a.seg_off[s + 1];
        if (hi < lo || hi - lo > 0xffffffffull) {
            set_error(a.b.ctl, FQ_EINVAL, kWhereEncPlan, s);
            continue;
        }
        local += dcdiv(dcdiv(hi - lo, kBlock), kTileBlocks);
    }
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t s = s0; s < s1; s++) {
        a.b.tile_base[s] = run;
        const uint64_t lo = a.seg_off[s], hi = a.seg_off[s + 1];
        const uint64_t n = hi >= lo ? hi - lo : 0;
        const uint64_t nt = dcdiv(dcdiv(n, kBlock), kTileBlocks);
        if (hi >= lo && n <= 0xffffffffull)
            for (uint64_t g = run; g < run + nt && g < a.b.tiles_cap; g++) a.b.tile_seg[g] = (uint32_t)s;
        run += hi >= lo && n <= 0xffffffffull ? nt : 0;
        SegInfo si{};
        si.n = n;
        si.nb = dcdiv(n, kBlock);
        si.mode = kModeNone;
        a.b.seg[s] = si;
        if (n == 0 && hi >= lo) {  // the empty stream is a bare raw header
            const uint64_t cap = a.out_off[s + 1] - a.out_off[s];
            if (cap < 16) {
                set_error(a.b.ctl, FQ_ENOSPC, kWhereEncPlan, s);
                a.out_bytes[s] = 16;
            } else {
                uint32_t *h = reinterpret_cast<uint32_t *>(a.out + a.out_off[s]);
                h[0] = kMagicRaw; h[1] = 0; h[2] = 0; h[3] = 0;
                a.out_bytes[s] = 16;
            }
        }
    }
    if (threadIdx.x == 0) {
        a.b.tile_base[S] = total;
        if (total > a.b.tiles_cap) set_error(a.b.ctl, FQ_EINVAL, kWhereEncPlan, total);
    }
}

// Ids i .. i+3 of a segment (zeros past n); a segment may start anywhere, so the 128-bit load is
// taken only where the address allows it (the same for every lane of a warp).
__device__ __forceinline__ void load4_any(const uint32_t *ids, uint64_t i, uint64_t n, uint32_t v[4])
{
    if (i + 3 < n && (reinterpret_cast<uintptr_t>(ids + i) & 15u) == 0) {
        const uint4 q = *reinterpret_cast<const uint4 *>(ids + i);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] = (i + j < n) ? ids[i + j] : 0u;
    }
}

// The tile's 64 blocks, 8 per warp with all loads in flight: lane's ids and gaps of each; the
// widths (warp-uniform); the first unsorted position (segment-local) in *bad.
__device__ __forceinline__ void tile_gaps(const uint32_t *ids, uint64_t n, uint64_t t, uint32_t warp, uint32_t lane,
                                          bool check, uint32_t v[kBlocksPerWarp][4], uint32_t gp[kBlocksPerWarp][4],
                                          uint32_t b[kBlocksPerWarp], unsigned long long *bad)
{
    const uint64_t nb = dcdiv(n, kBlock);
    uint32_t prev[kBlocksPerWarp];
#pragma unroll
    for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
        const uint64_t k = t * kTileBlocks + warp * kBlocksPerWarp + i;
        prev[i] = 0u;
        if (k < nb) {
            load4_any(ids, k * kBlock + 4u * lane, n, v[i]);
            if (check && lane == 0 && k > 0) prev[i] = ids[k * kBlock - 1];
        } else {
            v[i][0] = v[i][1] = v[i][2] = v[i][3] = 0u;
        }
    }
#pragma unroll
    for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
        const uint64_t k = t * kTileBlocks + warp * kBlocksPerWarp + i;
        b[i] = 0u;
        gp[i][0] = gp[i][1] = gp[i][2] = gp[i][3] = 0u;
        if (k < nb) {  // uniform over the warp
            unsigned long long dummy = ~0ull;
            gaps_of(v[i], prev[i], check && k > 0, k, n, lane, gp[i], check ? bad : &dummy);
            b[i] = bitlen32(__reduce_or_sync(0xffffffffu, gp[i][0] | gp[i][1] | gp[i][2] | gp[i][3]));
        }
    }
}

// Pass 1: each tile's sum of block widths (and the sortedness check).
__global__ void __launch_bounds__(kEncThreads) bat_widths_kernel(BEnc a)
{
    __shared__ uint32_t s_sum[kEncWarps];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = a.b.ctl->code != FQ_OK;  // the plan rejected the segment table
    __syncthreads();
    if (s_abort) return;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t T = a.b.tile_base[a.S];
    for (uint64_t g = blockIdx.x; g < T; g += gridDim.x) {
        const uint32_t s = a.b.tile_seg[g];
        const uint32_t *ids = a.ids + a.seg_off[s];
        const uint64_t n = a.seg_off[s + 1] - a.seg_off[s];
        const uint64_t t = g - a.b.tile_base[s];
        uint32_t v[kBlocksPerWarp][4], gp[kBlocksPerWarp][4], b[kBlocksPerWarp];
        unsigned long long bad = ~0ull;
        tile_gaps(ids, n, t, warp, lane, true, v, gp, b, &bad);
        if (bad != ~0ull) set_error(a.b.ctl, FQ_EUNSORTED, kWhereEncWidths, a.seg_off[s] + bad);
        uint32_t sum = 0;
#pragma unroll
        for (uint32_t i = 0; i < kBlocksPerWarp; i++) sum += b[i];
        if (lane == 0) s_sum[warp] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (uint32_t q = 0; q < kEncWarps; q++) tot += s_sum[q];
            a.b.tile_sum[g] = tot;
        }
        __syncthreads();
    }
}

// Pass 2 (one CTA): exclusive prefix of all tile sums, in coalesced rounds of 4,096 tiles.
__global__ void __launch_bounds__(kScanThreads) bat_escan_kernel(BEnc a)
{
    __shared__ unsigned long long sm[33];
    if (a.b.ctl->code != FQ_OK) return;  // uniform: the widths pass has finished
    const uint64_t T = a.b.tile_base[a.S];
    unsigned long long carry = 0;
    for (uint64_t base = 0; base < T; base += 4u * kScanThreads) {
        const uint64_t i0 = base + 4u * threadIdx.x;
        uint32_t x[4];
#pragma unroll
        for (uint32_t j = 0; j < 4; j++) x[j] = i0 + j < T ? a.b.tile_sum[i0 + j] : 0u;
        unsigned long long tot = 0;
        unsigned long long run = carry + cta_excl_scan64<kScanThreads>((unsigned long long)x[0] + x[1] + x[2] + x[3], sm, &tot);
#pragma unroll
        for (uint32_t j = 0; j < 4; j++) {
            if (i0 + j < T) a.b.status[i0 + j] = run;
            run += x[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) a.b.status[T] = carry;
}

// Pass 3: per tile, its segment's decision (packed only when smaller than raw) and payload
// offset from the scan; the tile's blocks packed (or its ids copied raw), its base and width
// table entries; the first tile of a segment writes the header and the stream size.
__global__ void __launch_bounds__(kEncThreads) bat_pack_kernel(BEnc a)
{
    __shared__ uint32_t sw[kTileBlocks], spre[kTileBlocks];
    __shared__ uint32_t pk[kEncWarps][4 * 32 + 4];
    __shared__ int s_abort;
    Ctl *c = a.b.ctl;
    if (threadIdx.x == 0) s_abort = c->code != FQ_OK;
    __syncthreads();
    if (s_abort) return;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t T = a.b.tile_base[a.S];
    const unsigned long long *pre = a.b.status;
    for (uint64_t g = blockIdx.x; g < T; g += gridDim.x) {
        const uint32_t s = a.b.tile_seg[g];
        const uint32_t *ids = a.ids + a.seg_off[s];
        const uint64_t n = a.seg_off[s + 1] - a.seg_off[s];
        const uint64_t g0 = a.b.tile_base[s], t = g - g0;
        const uint64_t nb = dcdiv(n, kBlock), ntiles_s = a.b.tile_base[s + 1] - g0;
        const unsigned long long excl = pre[g] - pre[g0], total = pre[g0 + ntiles_s] - pre[g0];
        uint8_t *out = a.out + a.out_off[s];
        const uint64_t cap = a.out_off[s + 1] - a.out_off[s];
        const uint64_t packed = 16u + dpad16(5u * nb) + 16u * total;
        const uint64_t raw = 16u + dpad16(4u * n);
        const bool is_packed = packed < raw;  // n > 0: the segment has a tile
        const uint64_t size = is_packed ? packed : raw;
        if (size > cap) {  // uniform over the CTA
            if (t == 0 && threadIdx.x == 0) {
                set_error(c, FQ_ENOSPC, kWhereEncPlan, s);
                a.out_bytes[s] = size;
            }
            continue;
        }
        uint32_t *h = reinterpret_cast<uint32_t *>(out);
        if (t == 0 && threadIdx.x == 0) {
            if (is_packed) {
                h[0] = kMagicPacked; h[1] = (uint32_t)n; h[2] = (uint32_t)nb; h[3] = (uint32_t)(4u * total);
            } else {
                h[0] = kMagicRaw; h[1] = (uint32_t)n; h[2] = 0u; h[3] = (uint32_t)n;
            }
            a.out_bytes[s] = size;
        }
        if (!is_packed) {  // raw body: this tile's ids, and the zero words to 16 bytes after the last
            for (uint32_t i = threadIdx.x; i < kBTileIds; i += kEncThreads) {
                const uint64_t gi = t * kBTileIds + i;
                if (gi < n) h[4u + gi] = ids[gi];
            }
            if (t + 1 == ntiles_s) {
                const uint32_t padw = (uint32_t)((dpad16(4u * n) - 4u * n) / 4u);
                if (threadIdx.x < padw) h[4u + n + threadIdx.x] = 0u;
            }
            continue;
        }
        if (t == 0) {  // zero bytes after the width table, to 16 bytes
            const uint64_t p = 16u + 5u * nb + threadIdx.x;
            if (p < 16u + dpad16(5u * nb)) out[p] = 0u;
        }
        uint32_t v[kBlocksPerWarp][4], gp[kBlocksPerWarp][4], b[kBlocksPerWarp];
        tile_gaps(ids, n, t, warp, lane, false, v, gp, b, nullptr);
#pragma unroll
        for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
            const uint32_t lb = warp * kBlocksPerWarp + i;
            const uint64_t k = t * kTileBlocks + lb;
            if (lane == 0) {
                sw[lb] = b[i];
                if (k < nb) {
                    h[4u + k] = v[i][0];
                    out[16u + 4u * nb + k] = (uint8_t)b[i];
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t x0 = sw[2 * lane], x1 = sw[2 * lane + 1];
            const uint32_t incl = warp_incl_scan(x0 + x1);
            spre[2 * lane] = incl - x0 - x1;
            spre[2 * lane + 1] = incl - x1;
        }
        __syncthreads();
        const uint64_t payload = 16u + dpad16(5u * nb);
#pragma unroll
        for (uint32_t i = 0; i < kBlocksPerWarp; i++) {
            const uint32_t lb = warp * kBlocksPerWarp + i;
            const uint64_t k = t * kTileBlocks + lb;
            if (k >= nb || b[i] == 0) continue;  // uniform over the warp
            uint32_t w4[4];
            pack_block_words(gp[i], b[i], pk[warp], lane, w4);
            store_block_words(out + payload + 16u * (excl + spre[lb]), w4, b[i], lane, 0ull, ~0ull);
        }
        __syncthreads();
    }
}

// ---- decode ----

struct BDec {
    const uint8_t *in;
    const uint64_t *in_off;
    const uint64_t *in_bytes;
    uint32_t S;
    uint32_t *ids;
    const uint64_t *seg_off;  // output positions; capacity of segment s = seg_off[s+1] - seg_off[s]
    uint64_t *n_out;
    BatchScratch b;
};

// One CTA: parse every stream header, tiles per stream and their prefix.
__global__ void __launch_bounds__(kScanThreads) bat_dplan_kernel(BDec a)
{
    __shared__ unsigned long long sm[33];
    if (threadIdx.x == 0) reset_ctl(a.b.ctl);
    __syncthreads();
    const uint64_t S = a.S;
    const uint64_t chunk = dcdiv(S, kScanThreads);
    const uint64_t s0 = (uint64_t)threadIdx.x * chunk, s1 = min(S, s0 + chunk);
    unsigned long long local = 0, total = 0;
    for (uint64_t s = s0; s < s1; s++) {
        const uint8_t *fq = a.in + a.in_off[s];
        const uint64_t bytes = a.in_bytes[s];
        const uint64_t cap = a.seg_off[s + 1] - a.seg_off[s];
        SegInfo si{};
        si.mode = kModeNone;
        si.ok = 0;
        if (bytes >= 16 && (reinterpret_cast<uintptr_t>(fq) & 15u) == 0) {
            const uint32_t magic = ld_u32(fq);
            const uint64_t n = ld_u32(fq + 4), nb = ld_u32(fq + 8), words = ld_u32(fq + 12);
            si.n = n;
            si.nb = nb;
            if (n > cap) {
                set_error(a.b.ctl, FQ_ENOSPC, kWhereDecPlan, s);
            } else if (magic == kMagicRaw && nb == 0 && words == n && bytes == 16u + dpad16(4u * n)) {
                si.mode = kModeRaw;
                si.ok = 1;
                for (uint64_t i = 16u + 4u * n; i < bytes; i++)
                    if (fq[i]) si.ok = 0;
            } else if (magic == kMagicPacked && n > 0 && nb == dcdiv(n, kBlock) && bytes >= 16u + dpad16(5u * nb)) {
                si.mode = kModePacked;
                si.ok = 1;
                for (uint64_t i = 16u + 5u * nb; i < 16u + dpad16(5u * nb); i++)
                    if (fq[i]) si.ok = 0;
            }
        }
        if (!si.ok) {
            if (si.n <= cap) set_error(a.b.ctl, FQ_ECORRUPT, kWhereDecPlan, s);
            si.mode = kModeNone;
        }
        a.b.seg[s] = si;
        local += si.mode == kModePacked ? dcdiv(si.nb, kTileBlocks) : si.mode == kModeRaw ? dcdiv(si.n, kBTileIds) : 0;
    }
    unsigned long long run = cta_excl_scan64<kScanThreads>(local, sm, &total);
    for (uint64_t s = s0; s < s1; s++) {
        a.b.tile_base[s] = run;
        const SegInfo si = a.b.seg[s];
        const uint64_t nt = si.mode == kModePacked ? dcdiv(si.nb, kTileBlocks) : si.mode == kModeRaw ? dcdiv(si.n, kBTileIds) : 0;
        for (uint64_t g = run; g < run + nt && g < a.b.tiles_cap; g++) a.b.tile_seg[g] = (uint32_t)s;
        run += nt;
        a.n_out[s] = si.mode == kModeNone ? 0 : si.n;
    }
    if (threadIdx.x == 0) {
        a.b.tile_base[S] = total;
        if (total > a.b.tiles_cap) set_error(a.b.ctl, FQ_EINVAL, kWhereDecPlan, total);
    }
}

__global__ void __launch_bounds__(kEncThreads) bat_dtiles_kernel(BDec a)
{
    __shared__ uint32_t ws[kEncWarps];
    const uint64_t T = min((uint64_t)a.b.tile_base[a.S], a.b.tiles_cap);
    for (uint64_t g = blockIdx.x; g < T; g += gridDim.x) {
        const uint32_t s = a.b.tile_seg[g];
        const SegInfo si = a.b.seg[s];
        if (si.mode != kModePacked) continue;  // uniform per CTA
        const uint64_t t = g - a.b.tile_base[s];
        const uint8_t *wd = a.in + a.in_off[s] + 16 + 4 * si.nb;
        uint32_t b = 0;
        if (threadIdx.x < kTileBlocks) {
            const uint64_t k = t * kTileBlocks + threadIdx.x;
            if (k < si.nb) {
                b = wd[k];
                if (b > 32u) set_error(a.b.ctl, FQ_ECORRUPT, kWhereDecPlan, s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t sum = 0;
            for (uint32_t i = 0; i < kEncWarps; i++) sum += ws[i];
            a.b.tile_sum[g] = sum;
        }
        __syncthreads();
    }
}

// One CTA per stream (round robin): scan its tile sums, check its total against its header.
__global__ void __launch_bounds__(kEncThreads) bat_dscan_kernel(BDec a)
{
    __shared__ unsigned long long sm[33];
    for (uint64_t s = blockIdx.x; s < a.S; s += gridDim.x) {
        SegInfo si = a.b.seg[s];
        if (si.mode != kModePacked) continue;
        const uint64_t base = a.b.tile_base[s];
        const uint64_t nt = dcdiv(si.nb, kTileBlocks);
        const uint64_t chunk = dcdiv(nt, kEncThreads);
        const uint64_t t0 = (uint64_t)threadIdx.x * chunk, t1 = min(nt, t0 + chunk);
        unsigned long long local = 0, total = 0;
        for (uint64_t t = t0; t < t1; t++) local += a.b.tile_sum[base + t];
        unsigned long long run = cta_excl_scan64<kEncThreads>(local, sm, &total);
        for (uint64_t t = t0; t < t1; t++) {
            a.b.tile_off[base + t] = (uint32_t)run;
            run += a.b.tile_sum[base + t];
        }
        if (threadIdx.x == 0) {
            const uint8_t *fq = a.in + a.in_off[s];
            const uint64_t words = ld_u32(fq + 12);
            si.total_b = total;
            if (words != 4u * total || a.in_bytes[s] != 16u + dpad16(5u * si.nb) + 16u * total) {
                set_error(a.b.ctl, FQ_ECORRUPT, kWhereDecPlan, s);
                si.mode = kModeNone;
                a.n_out[s] = 0;
            }
            a.b.seg[s] = si;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kEncThreads, 3) bat_dunpack_kernel(BDec a)
{
    extern __shared__ __align__(128) uint8_t dbuf[];  // [2][kDecStageB]
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ uint32_t spre[kTileBlocks];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = a.b.ctl->code == FQ_EINVAL;  // tile table larger than the workspace
    __syncthreads();
    if (s_abort) return;
    const uint64_t T = min((uint64_t)a.b.tile_base[a.S], a.b.tiles_cap);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    // payload bytes of a packed tile, or 0 (raw tiles and empty tiles are read directly)
    auto tile_bytes = [&](uint64_t g, uint32_t s, const SegInfo &si) -> uint32_t {
        if (si.mode != kModePacked) return 0;
        const uint64_t t = g - a.b.tile_base[s];
        const uint64_t nt = dcdiv(si.nb, kTileBlocks);
        const uint64_t end = (t + 1 < nt) ? a.b.tile_off[g + 1] : si.total_b;
        return (uint32_t)(16u * (end - a.b.tile_off[g]));
    };
    auto payload_at = [&](uint64_t g, uint32_t s, const SegInfo &si) -> const uint8_t * {
        return a.in + a.in_off[s] + 16 + dpad16(5u * si.nb) + 16u * (uint64_t)a.b.tile_off[g];
    };
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
        const uint64_t g0 = blockIdx.x;
        if (g0 < T) {
            const uint32_t s = a.b.tile_seg[g0];
            const SegInfo si = a.b.seg[s];
            const uint32_t by = tile_bytes(g0, s, si);
            if (by) bulk_load(dbuf, payload_at(g0, s, si), by, &bars[0]);
        }
    }
    __syncthreads();
    uint32_t phase0 = 0u, phase1 = 0u;
    for (uint64_t i = 0;; i++) {
        const uint64_t g = blockIdx.x + i * gridDim.x;
        if (g >= T) break;
        const uint32_t stage = (uint32_t)(i & 1u);
        const uint32_t s = a.b.tile_seg[g];
        const SegInfo si = a.b.seg[s];
        const uint64_t gn = g + gridDim.x;
        uint32_t pf_by = 0;  // thread 0: bytes of the next tile's copy issued into the other stage
        if (threadIdx.x == 0 && gn < T) {
            const uint32_t s2 = a.b.tile_seg[gn];
            const SegInfo si2 = a.b.seg[s2];
            pf_by = tile_bytes(gn, s2, si2);
            if (pf_by) bulk_load(dbuf + (stage ^ 1u) * kDecStageB, payload_at(gn, s2, si2), pf_by, &bars[stage ^ 1u]);
        }
        const uint64_t t = g - a.b.tile_base[s];
        const uint8_t *fq = a.in + a.in_off[s];
        uint32_t *ids = a.ids + a.seg_off[s];
        const bool vec_ok = (reinterpret_cast<uintptr_t>(ids) & 15u) == 0;
        const uint32_t by = tile_bytes(g, s, si);
        if (si.mode == kModeRaw) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(fq + 16);
            const uint64_t i0 = t * kBTileIds, i1 = min((uint64_t)si.n, (uint64_t)(i0 + kBTileIds));
            for (uint64_t j = i0 + threadIdx.x; j < i1; j += kEncThreads) {
                const uint32_t v = src[j];
                if (j > 0 && src[j - 1] >= v) set_error(a.b.ctl, FQ_ECORRUPT, kWhereDecUnpack, s);
                ids[j] = v;
            }
        } else if (si.mode == kModePacked) {
            const uint64_t nb = si.nb, n = si.n;
            const uint8_t *wd = fq + 16 + 4 * nb;
            const uint32_t *bases = reinterpret_cast<const uint32_t *>(fq + 16);
            if (warp == 0) {
                const uint64_t k0 = t * kTileBlocks + 2 * lane;
                const uint32_t x0 = k0 < nb ? wd[k0] : 0u, x1 = k0 + 1 < nb ? wd[k0 + 1] : 0u;
                const uint32_t incl = warp_incl_scan(x0 + x1);
                spre[2 * lane] = incl - x0 - x1;
                spre[2 * lane + 1] = incl - x1;
            }
            // Bounded wait for the tile's payload (the barrier also publishes spre).  A copy still
            // missing after it is reported; thread 0 then lets the CTA's copies in flight land
            // (bounded again) before the shared memory is released, and the CTA leaves.
            if (!__syncthreads_and(by == 0u || mbar_wait(&bars[stage], stage ? phase1 : phase0))) {
                if (threadIdx.x == 0) {
                    set_error(a.b.ctl, FQ_ETIMEOUT, kWhereDecUnpack, g);
                    mbar_wait(&bars[stage], stage ? phase1 : phase0);
                    if (pf_by) mbar_wait(&bars[stage ^ 1u], stage ? phase0 : phase1);
                }
                return;
            }
            if (by) {
                if (stage) phase1 ^= 1u;
                else phase0 ^= 1u;
            }
            const uint32_t *sp = reinterpret_cast<const uint32_t *>(dbuf + stage * kDecStageB);
            auto store4 = [&](uint64_t k, const uint32_t out[4]) {
                const uint64_t i0 = k * kBlock + 4u * lane;
                if (vec_ok && i0 + 3 < n) {
                    *reinterpret_cast<uint4 *>(ids + i0) = make_uint4(out[0], out[1], out[2], out[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (i0 + j < n) ids[i0 + j] = out[j];
                }
            };
            auto one_block = [&](uint32_t bi) {
                const uint32_t local = warp * kBlocksPerWarp + bi;
                const uint64_t k = t * kTileBlocks + local;
                if (k >= nb) return;
                uint32_t out[4];
                const uint32_t b = wd[k];
                bool good;
                if (k + 1 < nb && b <= 16u) {  // full narrow block: the lean 32-bit path
                    uint32_t last;
                    good = unpack_full_narrow(sp + 4u * spre[local], b, bases[k], lane, out, &last);
                    if (lane == 31 && last >= bases[k + 1]) good = false;
                } else {
                    unsigned long long last;
                    good = unpack_block(sp + 4u * spre[local], b, bases[k], k, n, lane, out, &last);
                    if (k + 1 < nb && lane == 31 && last >= (unsigned long long)bases[k + 1]) good = false;
                }
                if (!good) set_error(a.b.ctl, FQ_ECORRUPT, kWhereDecUnpack, s);
                store4(k, out);
            };
            for (uint32_t bi = 0; bi < kBlocksPerWarp; bi += 2) {  // full narrow blocks in pairs, one scan each
                const uint32_t local = warp * kBlocksPerWarp + bi;
                const uint64_t k = t * kTileBlocks + local;
                if (k >= nb) break;
                const uint32_t bA = wd[k], bB = k + 1 < nb ? wd[k + 1] : 0u;
                if (!(k + 2 < nb && bA <= 8u && bB <= 8u)) {  // uniform over the warp
                    one_block(bi);
                    one_block(bi + 1);
                    continue;
                }
                uint32_t oA[4], oB[4];
                bool goodA, goodB;
                unpack_pair_narrow(sp + 4u * spre[local], bA, bases[k], sp + 4u * spre[local + 1], bB, bases[k + 1],
                                   bases[k + 2], lane, oA, oB, &goodA, &goodB);
                if (!goodA || !goodB) set_error(a.b.ctl, FQ_ECORRUPT, kWhereDecUnpack, s);
                store4(k, oA);
                store4(k + 1, oB);
            }
        }
        __syncthreads();
    }
}


}  // namespace
}  // namespace fq

using namespace fq;

extern "C" {

uint64_t fq_batch_workspace_bytes(uint64_t total_ids, uint32_t S) { return batch_layout(total_ids, S, nullptr, nullptr); }

fq_status fq_frontier_encode_batch(const uint32_t *d_ids, const uint64_t *d_seg_off, uint32_t S, uint64_t total_ids,
                                   uint8_t *d_out, const uint64_t *d_out_off, uint64_t *d_out_bytes, void *d_work,
                                   uint64_t work_bytes, void *stream)
{
    if (S == 0) return FQ_OK;
    if (!d_seg_off || !d_out || !d_out_off || !d_out_bytes || !d_work || (total_ids && !d_ids)) return FQ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_out) & 15u) || (reinterpret_cast<uintptr_t>(d_work) & 15u)) return FQ_EINVAL;
    if (work_bytes < fq_batch_workspace_bytes(total_ids, S)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BEnc a{d_ids, d_seg_off, S, d_out, d_out_off, d_out_bytes, {}};
    batch_layout(total_ids, S, &a.b, d_work);
    bat_plan_kernel<<<1, kScanThreads, 0, st>>>(a);
    const uint32_t grid = tuned_grid(FQ_TUNE_BAT_ENCODE, total_ids, (uint64_t)4 * num_sms(), a.b.tiles_cap);
    bat_widths_kernel<<<grid, kEncThreads, 0, st>>>(a);
    bat_escan_kernel<<<1, kScanThreads, 0, st>>>(a);
    bat_pack_kernel<<<grid, kEncThreads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? FQ_OK : FQ_ECUDA;
}

fq_status fq_frontier_decode_batch(const uint8_t *d_in, const uint64_t *d_in_off, const uint64_t *d_in_bytes, uint32_t S,
                                   uint32_t *d_ids, const uint64_t *d_seg_off, uint64_t total_ids, uint64_t *d_n,
                                   void *d_work, uint64_t work_bytes, void *stream)
{
    if (S == 0) return FQ_OK;
    if (!d_in || !d_in_off || !d_in_bytes || !d_seg_off || !d_n || !d_work || (total_ids && !d_ids)) return FQ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_in) & 15u) || (reinterpret_cast<uintptr_t>(d_work) & 15u)) return FQ_EINVAL;
    if (work_bytes < fq_batch_workspace_bytes(total_ids, S)) return FQ_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BDec a{d_in, d_in_off, d_in_bytes, S, d_ids, d_seg_off, d_n, {}};
    batch_layout(total_ids, S, &a.b, d_work);
    static std::atomic<bool> done[64];
    if (allow_smem(bat_dunpack_kernel, kBatchDecSmem, done) != cudaSuccess) return FQ_ECUDA;
    bat_dplan_kernel<<<1, kScanThreads, 0, st>>>(a);
    const uint32_t grid = (uint32_t)std::min<uint64_t>(a.b.tiles_cap, (uint64_t)8 * num_sms());
    bat_dtiles_kernel<<<grid, kEncThreads, 0, st>>>(a);
    bat_dscan_kernel<<<(uint32_t)std::min<uint64_t>(S, (uint64_t)8 * num_sms()), kEncThreads, 0, st>>>(a);
    bat_dunpack_kernel<<<tuned_grid(FQ_TUNE_BAT_DUNPACK, total_ids, (uint64_t)3 * num_sms(), a.b.tiles_cap), kEncThreads,
                         kBatchDecSmem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? FQ_OK : FQ_ECUDA;
}

}  // extern "C"
