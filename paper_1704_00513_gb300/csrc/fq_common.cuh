// fq_common.cuh -- shared device helpers and the internal (C++) interface between the codec
// (codec.cu) and the BFS level loop (bfs.cu) of libfqbfs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/fqbfs.h"

namespace fq {

constexpr uint32_t kBlock = 128;          // B: ids per packed block (sec. 5.1, S4-BP128 in sec. 5.3)
constexpr uint32_t kEncThreads = 256;     // CTA size of the block-parallel codec kernels
constexpr uint32_t kEncWarps = kEncThreads / 32;
constexpr uint32_t kBlocksPerWarp = 8;    // 128-id blocks one warp handles per tile
constexpr uint32_t kTileBlocks = kEncWarps * kBlocksPerWarp;  // 64 blocks = 8192 ids per tile
constexpr uint32_t kBitThreads = 256;     // CTA size of the bitmap kernels
constexpr uint32_t kWordsPerThread = 8;   // uint64 words per thread in the bitmap kernels
constexpr uint32_t kTileWords = kBitThreads * kWordsPerThread;  // 2048 words = 131072 bits
constexpr uint32_t kScanThreads = 1024;   // single-CTA plan/scan kernels

// stream magics: ASCII 'F','Q','P','1' etc. read as little-endian u32
constexpr uint32_t kMagicPacked = 0x31505146u;  // "FQP1"
constexpr uint32_t kMagicRaw = 0x31525146u;     // "FQR1"
constexpr uint32_t kMagicBitmap = 0x314D4246u;  // "FBM1"
constexpr uint32_t kMagicPatched = 0x31585146u; // "FQX1": binary packing with exceptions
constexpr uint32_t kPxHeader = 32;              // bytes of the patched stream's header

enum : uint32_t { kFbRaw = 0, kFbSet = 1, kFbClear = 2 };

// result of a plan kernel
enum : uint32_t {
    kModeNone = 0,      // error: write nothing
    kModePacked = 1,    // FQ packed
    kModeRaw = 2,       // FQ raw
    kModeFbRaw = 3,     // FB raw words
    kModePatched = 4,   // FQX packed (exceptions)
};

// internal stage ids recorded in fq_device_status.where
enum : uint32_t {
    kWhereEncWidths = 1, kWhereEncPlan = 2, kWhereDecPlan = 3, kWhereDecUnpack = 4,
    kWhereFbDecode = 5, kWhereBfs = 6,
};

// Control block at the start of every codec workspace.  The first 16 bytes are the public
// fq_device_status record.
struct Ctl {
    int32_t code;
    uint32_t where;
    unsigned long long detail;
    uint32_t mode;        // kMode*
    uint32_t fb_mode;     // kFb* chosen by the bitmap plan
    unsigned long long n; // ids being encoded (FB: positions count) or decoded
    unsigned long long nb;
    unsigned long long popcount;
    unsigned long long total_b;
    unsigned long long out_bytes;
    unsigned long long fq_offset;  // byte offset of the FQ stream inside the container
    uint32_t ticket;               // CTAs of a launch done with their part (a last-CTA step; 0 between launches)
    uint32_t mode2;                // mode of the mirrored FB stream (kMode*), kModeNone if absent
    unsigned long long out2_bytes;
    unsigned long long total_e;    // patched codec: exceptions over all blocks
    uint32_t skip_pos;             // FB: the width sum (total_b) came from the bitmap and the stream is raw
                                   // words, so no positions are extracted and no widths pass runs
    uint32_t pad0;
};
static_assert(sizeof(Ctl) <= 256, "control block must fit its slot");

// Pointers into one codec workspace (computed on the host from its base and capacities).
struct Scratch {
    Ctl *ctl;
    uint8_t *widths;      // [nb_cap]
    uint32_t *bases;      // [nb_cap]
    uint32_t *block_off;  // [nb_cap] decode: payload word offset of each block
    uint32_t *tile_sum;   // [etiles_cap]
    uint32_t *tile_off;   // [etiles_cap]
    uint32_t *btile_cnt;  // [btiles_cap]
    uint32_t *btile_off;  // [btiles_cap]
    uint32_t *positions;  // [pos_cap]  bitmap positions (FB)
    uint8_t *ex;          // [nb_cap] patched codec: exceptions per block
    uint32_t *tile_ex;    // [etiles_cap] patched codec: exceptions per tile
    uint32_t *tile_exoff; // [etiles_cap] patched codec: exception offset of each tile
    uint64_t ids_cap;     // largest id count an encode/decode may see
    uint64_t nbits_cap;
    uint64_t nb_cap, etiles_cap, btiles_cap, pos_cap;
};

uint64_t workspace_bytes(uint64_t max_ids, uint64_t max_nbits);
Scratch carve(void *base, uint64_t max_ids, uint64_t max_nbits);
// Largest (max_ids, max_nbits) a workspace of `bytes` serves, with max_nbits fixed by caller.
bool workspace_fits(uint64_t bytes, uint64_t ids, uint64_t nbits);

inline uint64_t pad16(uint64_t b) { return (b + 15u) / 16u * 16u; }
inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------ internal launches
// Every launch helper enqueues on `st` and returns cudaGetLastError().

// FQ-encode ids[0..n) (FQX, patched exceptions, with px).  n is *n_dev when n_dev != nullptr
// (device-resident count, then n_max bounds it for the grid), else n_host.  Container: FQ stream at out (fb == false) or an
// FB stream whose inner FQ starts at out + 16 (fb == true; positions come from the bitmap plan).
cudaError_t encode_fq(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint64_t n_max, uint8_t *out,
                      uint64_t cap, uint64_t *out_bytes, const Scratch &s, cudaStream_t st, bool px = false);
cudaError_t encode_fb(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap, uint64_t *out_bytes,
                      const Scratch &s, cudaStream_t st);
// Decode: in_bytes is in_bytes_host unless in_bytes_dev != nullptr.
cudaError_t decode_fq(const uint8_t *in, uint64_t in_bytes_host, const uint64_t *in_bytes_dev, uint32_t *ids,
                      uint64_t cap, uint64_t *n_out, const Scratch &s, cudaStream_t st);
cudaError_t decode_fb(const uint8_t *in, uint64_t in_bytes_host, const uint64_t *in_bytes_dev, uint64_t *words,
                      uint64_t nbits, const Scratch &s, cudaStream_t st);
// Reset the status record to FQ_OK (max_ids: the largest call the scratch serves).
cudaError_t reset_status(const Scratch &s, uint64_t max_ids, cudaStream_t st);

// Optional mirror of an FQ encode: the same ids written a second time as an FB stream in SET
// mode (header + the FQ stream, or the raw words when that is not smaller).  Valid when the
// ids are exactly the set bits of `words` (nbits bits) and 2 * n <= nbits.
struct Mirror {
    uint8_t *out = nullptr;
    uint64_t cap = 0;
    uint64_t *out_bytes = nullptr;
    const uint64_t *words = nullptr;
    uint64_t nbits = 0;
};
cudaError_t encode_fq_mirror(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint64_t n_max,
                             uint8_t *out, uint64_t cap, uint64_t *out_bytes, const Mirror &mirror,
                             const Scratch &s, cudaStream_t st);
// Frontiers of at most kSmallIds ids: the mirrored encode (as encode_fq_mirror) and the decode of
// the FQ stream it wrote (as decode_fq, into ids_out) in one launch of one CTA.
constexpr uint32_t kSmallTiles = 1;
constexpr uint64_t kSmallIds = (uint64_t)kSmallTiles * kTileBlocks * kBlock;  // 8,192
cudaError_t codec_small(const uint32_t *ids, uint64_t n_host, const uint64_t *n_dev, uint8_t *out, uint64_t cap,
                        uint64_t *out_bytes, const Mirror &mirror, uint32_t *ids_out, uint64_t dec_cap,
                        uint64_t *n_out, const Scratch &s, cudaStream_t st);
// FB encode when the positions to code are already in s.positions with count and mode set in
// s.ctl (n, fb_mode), e.g. by the BFS compaction.
cudaError_t encode_fb_positions(const uint64_t *words, uint64_t nbits, uint8_t *out, uint64_t cap,
                                uint64_t *out_bytes, const Scratch &s, cudaStream_t st);

// Bitmap -> sorted positions, shared with the BFS compaction: tile counts then extraction.
int num_sms();

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ uint32_t bitlen32(uint32_t x) { return 32u - __clz(x); }

__device__ __forceinline__ void set_error(Ctl *c, int32_t code, uint32_t where, unsigned long long detail)
{
    // first error wins; detail keeps the smallest index reported for that code
    int32_t prev = atomicCAS(&c->code, 0, code);
    if (prev == 0 || prev == code) {
        if (prev == 0) c->where = where;
        atomicMin(&c->detail, detail);
    }
}

// Clear a Scratch's control block (status OK, no mode); called by one thread.
__device__ __forceinline__ void reset_scratch_device(const Scratch &s)
{
    Ctl *c = s.ctl;
    c->code = FQ_OK;
    c->where = 0;
    c->detail = ~0ull;
    c->mode = kModeNone;
    c->mode2 = kModeNone;
    c->fb_mode = kFbRaw;
    c->n = c->nb = c->popcount = c->total_b = c->out_bytes = c->fq_offset = c->out2_bytes = c->total_e = 0;
    c->ticket = 0;
    c->skip_pos = 0;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long x)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Exclusive scan over a CTA of NT threads (NT multiple of 32, <= 1024) of one u64 per thread.
// Returns the thread's exclusive prefix; *total receives the CTA total.  Uses `sm` (32 u64).
template <int NT>
__device__ __forceinline__ unsigned long long cta_excl_scan64(unsigned long long x, unsigned long long *sm,
                                                              unsigned long long *total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long incl = warp_incl_scan64(x);
    if (lane == 31) sm[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = (lane < NT / 32) ? sm[lane] : 0ull;
        unsigned long long wi = warp_incl_scan64(w);
        sm[lane] = wi - w;
        if (lane == 31) sm[32] = wi;
    }
    __syncthreads();
    unsigned long long r = sm[warp] + incl - x;
    *total = sm[32];
    __syncthreads();
    return r;
}

// Exclusive scan (from 0) of the u32 values in[0..count) into out[0..count) by one CTA of NT
// threads; out may equal in.  Returns the 64-bit total to every thread.  Thread i owns a
// contiguous chunk and reads it kScanWin values at a time with all of a window's loads issued
// before any is used, so a chunk of a few dozen values costs one memory latency, not one each.
// The loads bypass L1 (ld.global.cg): the values may have been written by other CTAs of the same
// launch (a last-CTA scan).
constexpr uint32_t kScanWin = 16;
template <uint32_t NT>
__device__ unsigned long long cta_chunk_scan_u32(const uint32_t *in, uint32_t *out, uint64_t count,
                                                 unsigned long long *sm)
{
    const uint64_t chunk = (count + NT - 1) / NT;
    const uint64_t t0 = (uint64_t)threadIdx.x * chunk, t1 = t0 + chunk < count ? t0 + chunk : count;
    unsigned long long local = 0, total = 0;
    for (uint64_t w = t0; w < t1; w += kScanWin) {
        uint32_t x[kScanWin];
#pragma unroll
        for (uint32_t i = 0; i < kScanWin; i++) x[i] = (w + i < t1) ? __ldcg(in + w + i) : 0u;
#pragma unroll
        for (uint32_t i = 0; i < kScanWin; i++) local += x[i];
    }
    unsigned long long run = cta_excl_scan64<NT>(local, sm, &total);
    for (uint64_t w = t0; w < t1; w += kScanWin) {
        uint32_t x[kScanWin];
#pragma unroll
        for (uint32_t i = 0; i < kScanWin; i++) x[i] = (w + i < t1) ? __ldcg(in + w + i) : 0u;
#pragma unroll
        for (uint32_t i = 0; i < kScanWin; i++) {
            if (w + i < t1) out[w + i] = (uint32_t)run;
            run += x[i];
        }
    }
    return total;
}

}  // namespace fq

namespace fq {
// The last CUDA error the library saw in this thread (reported by fq_last_cuda_error()).
void note_cuda_error(cudaError_t e, int line);
// Grid of a tunable launch site for `items` work items: the autotuned CTAs per SM (fq_tune_set)
// times the SM count when one is set for the items' size class, else default_grid; at most
// max_grid, at least 1.
uint32_t tuned_grid(uint32_t site, uint64_t items, uint64_t default_grid, uint64_t max_grid);
// Changes whenever the tuning table does (a graph that captured grids must then be rebuilt).
uint32_t tune_generation();
}

#define FQ_CUDA_TRY(expr)                                \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) {                         \
            fq::note_cuda_error(_e, __LINE__);           \
            return _e;                                   \
        }                                                \
    } while (0)

namespace fq {
// Kernels with more than 48 KB of dynamic shared memory opt in once per device; done[dev] records
// it.  Host threads may race here: the attribute call is idempotent, and the flag is atomic.
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes, std::atomic<bool> *done)
{
    int dev = 0;
    FQ_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev].load(std::memory_order_acquire)) {
        FQ_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        done[dev].store(true, std::memory_order_release);
    }
    return cudaSuccess;
}
}  // namespace fq
