// codec_dev.cuh -- device building blocks shared by the single-stream codec (codec.cu) and the
// batched codec (batch.cu): byte helpers, TMA bulk staging, gap extraction and block
// packing/unpacking.
#pragma once

#include "fq_common.cuh"

namespace fq {

__device__ __forceinline__ uint64_t dpad16(uint64_t b) { return (b + 15u) & ~uint64_t(15); }
__device__ __forceinline__ uint64_t dcdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint32_t ld_u32(const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); }


constexpr uint32_t kSpinLimit = 1u << 22;  // polls before a bounded wait gives up ...
constexpr uint64_t kWaitLimitNs = 200ull * 1000ull * 1000ull;  // ... or this much time, whichever comes first
constexpr uint32_t kTryWaitHintNs = 20000;  // longest a single poll may suspend the thread

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- TMA staging helpers (1-D bulk copies into shared memory, completion on an mbarrier) ----

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issue a bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) global -> shared,
// arriving on `bar` with the byte count as its transaction.
__device__ __forceinline__ void bulk_load(void *sdst, const void *gsrc, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Wait until phase `parity` of `bar` completes; bounded in time: a poll suspends the thread for at
// most kTryWaitHintNs, and the wait gives up after kWaitLimitNs of global time (or kSpinLimit polls).
// A bound on polls alone is not one on time: how long an unsatisfied try_wait suspends is up to the
// hardware unless the hint caps it.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kSpinLimit; i++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity), "r"(kTryWaitHintNs)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}


// Gaps of the four slots lane*4 .. lane*4+3 of block k from its four ids v; prev is the id
// before the block (used only for the sortedness check of slot 0).
__device__ __forceinline__ void gaps_of(const uint32_t v[4], uint32_t prev_block_last, bool has_prev_block, uint64_t k,
                                        uint64_t n, uint32_t lane, uint32_t g[4], unsigned long long *bad)
{
    uint32_t prev = __shfl_up_sync(0xffffffffu, v[3], 1);
    bool has_prev = lane > 0;
    if (lane == 0) {
        prev = prev_block_last;
        has_prev = has_prev_block;
    }
    if ((k + 1) * kBlock <= n) {  // full block: 32-bit gaps and one sortedness test per lane
        g[0] = lane ? v[0] - prev - 1u : 0u;
        g[1] = v[1] - v[0] - 1u;
        g[2] = v[2] - v[1] - 1u;
        g[3] = v[3] - v[2] - 1u;
        const bool unsorted = (has_prev && v[0] <= prev) | (v[1] <= v[0]) | (v[2] <= v[1]) | (v[3] <= v[2]);
        if (!unsorted) return;  // otherwise the general path below finds the first bad index
    }
    const uint64_t i0 = k * kBlock + 4u * lane;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        g[j] = 0;
        if (i0 + j >= n) continue;
        const uint32_t p = (j == 0) ? prev : v[j - 1];
        const bool hp = (j == 0) ? has_prev : true;
        if (hp) {
            if (v[j] <= p) *bad = min(*bad, (unsigned long long)(i0 + j));
            else if (!(lane == 0 && j == 0)) g[j] = v[j] - p - 1u;
        }
    }
}

__device__ __forceinline__ void load4_guard(const uint32_t *ids, uint64_t i, uint64_t n, uint32_t v[4])
{
    if (i + 3 < n) {
        const uint4 q = *reinterpret_cast<const uint4 *>(ids + i);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] = (i + j < n) ? ids[i + j] : 0u;
    }
}


// floor(x / b) == (x * kRecip16[b]) >> 16 for 1 <= b <= 32 and 0 <= x < 2048 (kRecip16[b] is
// ceil(2^16 / b)); used where a width divides a small bit count, instead of an integer division.
static __constant__ uint32_t kRecip16[33] = {
    0u,     65536u, 32768u, 21846u, 16384u, 13108u, 10923u, 9363u, 8192u, 7282u, 6554u,
    5958u,  5462u,  5042u,  4682u,  4370u,  4096u,  3856u,  3641u, 3450u, 3277u, 3121u,
    2979u,  2850u,  2731u,  2622u,  2521u,  2428u,  2341u,  2260u, 2185u, 2115u, 2048u};

// Pack the 128 gaps of one block (4 per lane, slot 4*lane + j at bits [slot*b, slot*b + b)) into
// its 4*b payload words.  Lane L returns words L, L+32, L+64, L+96 in w[0..3] (those below 4*b are
// meaningful).  For b <= 16 each lane first forms its 4*b-bit segment; while segments are shorter
// than a word, pairs of neighbouring segments are merged by shuffles (after k merges the segment of
// lane 2^k * i covers S = 4*b*2^k bits, 32 <= S < 64), so that each output word overlaps at most two
// segments and takes three shuffles.  Wider blocks OR the slots into a shared-memory row (129+
// words).  All 32 lanes must call it.
__device__ __forceinline__ void pack_block_words(const uint32_t g[4], uint32_t b, uint32_t *row, uint32_t lane,
                                                 uint32_t w[4])
{
    w[0] = w[1] = w[2] = w[3] = 0u;
    if (b == 0u) return;  // no payload words
    if (b <= 16u) {
        uint32_t lo = g[0] | (g[1] << b), hi = 0u;  // 2b <= 32: slot 1 never spills
        const uint32_t s2 = 2u * b, s3 = 3u * b;
        if (s2 < 32u) {
            lo |= g[2] << s2;
            hi |= __funnelshift_l(g[2], 0u, s2);
        } else {
            hi |= g[2] << (s2 - 32u);
        }
        if (s3 < 32u) {
            lo |= g[3] << s3;
            hi |= __funnelshift_l(g[3], 0u, s3);
        } else {
            hi |= g[3] << (s3 - 32u);
        }
        uint32_t S = 4u * b, k = 0;
        while (S < 32u) {  // segments here fit in S < 32 bits, so hi is still 0
            const uint32_t p = __shfl_down_sync(0xffffffffu, lo, 1u << k);
            hi = __funnelshift_l(p, 0u, S);
            lo |= p << S;
            S <<= 1;
            k++;
        }
        const uint32_t m = kRecip16[b];
        const uint32_t nw = b <= 8u ? 1u : 2u;
        for (uint32_t i = 0; i < nw; i++) {
            const uint32_t word = lane + 32u * i;
            const uint32_t first = ((8u * word * m) >> 16) >> k;  // segment holding the word's first bit
            const uint32_t sL = __shfl_sync(0xffffffffu, lo, min(first << k, 31u));
            const uint32_t sH = __shfl_sync(0xffffffffu, hi, min(first << k, 31u));
            const uint32_t nL = __shfl_sync(0xffffffffu, lo, min((first + 1u) << k, 31u));
            const uint32_t r = 32u * word - first * S;  // bit of that segment where the word starts
            uint32_t v = r < 32u ? __funnelshift_r(sL, sH, r) : (sH >> (r - 32u));
            if (S - r < 32u) v |= nL << (S - r);
            if (word < 4u * b) w[i] = v;
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) row[4 * lane + j] = 0u;
    if (lane == 0) row[128] = 0u;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (g[j] == 0u) continue;
        const uint32_t pos = (4u * lane + j) * b;
        const uint32_t w0 = pos >> 5, sh = pos & 31u;
        atomicOr(&row[w0], g[j] << sh);
        if (sh + b > 32u) atomicOr(&row[w0 + 1], g[j] >> (32u - sh));
    }
    __syncwarp();
#pragma unroll
    for (uint32_t i = 0; i < 4; i++) w[i] = row[lane + 32u * i];
    __syncwarp();
}

// Store the words of pack_block_words at dst (the block's payload, 16-byte aligned), keeping only
// those below `limit` bytes of dst's buffer position `pos0` (speculative writes stop at the bound).
__device__ __forceinline__ void store_block_words(uint8_t *dst, const uint32_t w[4], uint32_t b, uint32_t lane,
                                                  uint64_t pos0, uint64_t limit)
{
    const uint64_t room = limit > pos0 ? limit - pos0 : 0ull;
    const uint32_t room32 = room > 0xffffffffull ? 0xffffffffu : (uint32_t)room;
    const uint32_t nwords = min(4u * b, room32 >> 2);
#pragma unroll
    for (uint32_t i = 0; i < 4; i++) {
        const uint32_t word = lane + 32u * i;
        if (word < nwords) reinterpret_cast<uint32_t *>(dst)[word] = w[i];
    }
}

// Pack the 128 gaps of one block into 4*b words staged in row, then return lane's 4 consecutive
// output words as one 128-bit value (meaningful for lane < b).  All 32 lanes must call it.
__device__ __forceinline__ uint4 pack_block(const uint32_t g[4], uint32_t b, uint32_t *row, uint32_t lane)
{
    uint32_t w[4];
    pack_block_words(g, b, row, lane, w);
    __syncwarp();
#pragma unroll
    for (uint32_t i = 0; i < 4; i++) row[lane + 32u * i] = w[i];
    __syncwarp();
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (lane < b) q = make_uint4(row[4 * lane], row[4 * lane + 1], row[4 * lane + 2], row[4 * lane + 3]);
    __syncwarp();
    return q;
}

// The slots of a block of width 0 <= b <= 16 with 32-bit arithmetic only: a lane's four slots are
// the 4*b bits at 4*lane*b, read as a funnel-shifted 64-bit window of three staged words.
__device__ __forceinline__ void extract_narrow(const uint32_t *pk, uint32_t b, uint32_t lane, uint32_t g[4])
{
    const uint32_t bit0 = 4u * lane * b, ws = bit0 >> 5, sh = bit0 & 31u;
    const uint32_t w0 = pk[ws], w1 = pk[ws + 1], w2 = pk[ws + 2];
    const uint32_t lo = __funnelshift_r(w0, w1, sh), hi = __funnelshift_r(w1, w2, sh);
    const uint32_t mask = (1u << b) - 1u;
    g[0] = lo & mask;
    g[1] = __funnelshift_r(lo, hi, b) & mask;  // b < 32
    const uint32_t s2 = 2u * b, s3 = 3u * b;
    g[2] = (s2 < 32u ? __funnelshift_r(lo, hi, s2) : (hi >> (s2 - 32u))) & mask;
    g[3] = (s3 < 32u ? __funnelshift_r(lo, hi, s3) : (hi >> (s3 - 32u))) & mask;
}

// Ids of a FULL block (all 128 slots hold ids) whose increments g + 1 sum to less than 2^32 (true
// for any block of width <= 16: at most 128 * 2^16): a 32-bit warp scan.  The only checks a full
// block needs: slot 0 holds 0, and the last id does not pass 2^32 - 1 (lane 31 tests it in 64
// bits).  Returns false if either fails.
__device__ __forceinline__ bool scan_full32(const uint32_t g[4], uint32_t base, uint32_t lane, uint32_t out[4],
                                            uint32_t *last)
{
    const uint32_t first = (lane == 0) ? 0u : g[0] + 1u;  // slot 0 of the block is the base itself
    const uint32_t lsum = first + g[1] + g[2] + g[3] + 3u;
    const uint32_t excl = warp_incl_scan(lsum) - lsum;
    uint32_t v = base + excl + first;
    out[0] = v;
    v += g[1] + 1u;
    out[1] = v;
    v += g[2] + 1u;
    out[2] = v;
    v += g[3] + 1u;
    out[3] = v;
    *last = v;
    bool ok = !(lane == 0 && g[0] != 0u);
    if (lane == 31) ok = ok && ((unsigned long long)base + excl + lsum <= 0xffffffffull);
    return ok;
}

// Unpack a FULL block of width 0 <= b <= 16 with 32-bit arithmetic only.
__device__ __forceinline__ bool unpack_full_narrow(const uint32_t *pk, uint32_t b, uint32_t base, uint32_t lane,
                                                   uint32_t out[4], uint32_t *last)
{
    uint32_t g[4];
    extract_narrow(pk, b, lane, g);
    return scan_full32(g, base, lane, out, last);
}

// Two FULL consecutive blocks A, B of width <= 8 with one warp scan: each block's increments
// g + 1 sum below 2^15 (127 slots of at most 256), so the two prefix sums ride in the halves of one
// 32-bit word without a carry between them.  nextB is the base of the block after B.  good*
// report, per block, slot 0 holding 0 and the last id staying below the next block's base (no
// wrap: the bases are u32).  All 32 lanes must call it.
__device__ __forceinline__ void unpack_pair_narrow(const uint32_t *pkA, uint32_t bA, uint32_t baseA,
                                                   const uint32_t *pkB, uint32_t bB, uint32_t baseB, uint32_t nextB,
                                                   uint32_t lane, uint32_t oA[4], uint32_t oB[4], bool *goodA,
                                                   bool *goodB)
{
    uint32_t gA[4], gB[4];
    extract_narrow(pkA, bA, lane, gA);
    extract_narrow(pkB, bB, lane, gB);
    const uint32_t fA = lane ? gA[0] + 1u : 0u, fB = lane ? gB[0] + 1u : 0u;  // slot 0 is the base itself
    const uint32_t sA = fA + gA[1] + gA[2] + gA[3] + 3u, sB = fB + gB[1] + gB[2] + gB[3] + 3u;
    const uint32_t both = sA | (sB << 16);
    const uint32_t incl = warp_incl_scan(both), ex = incl - both;
    uint32_t vA = baseA + (ex & 0xffffu) + fA, vB = baseB + (ex >> 16) + fB;
    oA[0] = vA;
    oB[0] = vB;
#pragma unroll
    for (int j = 1; j < 4; j++) {
        vA += gA[j] + 1u;
        vB += gB[j] + 1u;
        oA[j] = vA;
        oB[j] = vB;
    }
    *goodA = !(lane == 0 && gA[0] != 0u);
    *goodB = !(lane == 0 && gB[0] != 0u);
    if (lane == 31) {
        *goodA = *goodA && (unsigned long long)baseA + (incl & 0xffffu) < baseB;
        *goodB = *goodB && (unsigned long long)baseB + (incl >> 16) < nextB;
    }
}

// The b-bit slot values of one block whose payload words start at pk (readable two words past
// the block): lane's slots 4*lane .. 4*lane+3 in g[].
__device__ __forceinline__ void extract_slots(const uint32_t *pk, uint32_t b, uint32_t lane, uint32_t g[4])
{
    const uint32_t mask = (b == 32u) ? 0xffffffffu : ((1u << b) - 1u);
    if (b <= 16u) {  // the lane's four slots lie in one 3-word window
        const uint32_t bit0 = 4u * lane * b, ws = bit0 >> 5, sh = bit0 & 31u;
        const unsigned long long x = ((unsigned long long)pk[ws + 1] << 32) | pk[ws];
        unsigned long long seg = x >> sh;
        if (sh) seg |= (unsigned long long)pk[ws + 2] << (64u - sh);
#pragma unroll
        for (int j = 0; j < 4; j++) g[j] = b ? (uint32_t)(seg >> (j * b)) & mask : 0u;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t pos = (4u * lane + j) * b, w0 = pos >> 5, sh = pos & 31u;
            const unsigned long long two = ((unsigned long long)pk[w0 + 1] << 32) | pk[w0];
            g[j] = (uint32_t)(two >> sh) & mask;
        }
    }
}

// Ids of block k from its gaps g[] (lane's slots) and base: a 64-bit warp prefix sum of gap + 1.
// Returns false if the block is inconsistent (non-zero slot 0 or padding slot, u32 overflow);
// `last` receives lane's last value.
__device__ __forceinline__ bool scan_slots(const uint32_t g[4], uint64_t base, uint64_t k, uint64_t n,
                                           uint32_t lane, uint32_t out[4], unsigned long long *last)
{
    const uint64_t i0 = k * kBlock + 4u * lane;
    bool bad = false;
    unsigned long long lsum64 = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const bool pad = (lane == 0 && j == 0) || i0 + j >= n;
        if (pad && g[j]) bad = true;
        lsum64 += pad ? 0ull : (unsigned long long)g[j] + 1ull;
    }
    unsigned long long v = base + (warp_incl_scan64(lsum64) - lsum64);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v += (i0 + j >= n || (lane == 0 && j == 0)) ? 0ull : (unsigned long long)g[j] + 1ull;
        out[j] = (uint32_t)v;
        if (i0 + j < n && v > 0xffffffffull) bad = true;
    }
    *last = v;
    return !bad;
}

// Unpack one block of width b (payload at pk, base = the block's first id): lane's four ids.
__device__ __forceinline__ bool unpack_block(const uint32_t *pk, uint32_t b, uint64_t base, uint64_t k, uint64_t n,
                                             uint32_t lane, uint32_t out[4], unsigned long long *last)
{
    uint32_t g[4];
    extract_slots(pk, b, lane, g);
    return scan_slots(g, base, k, n, lane, out, last);
}

}  // namespace fq
