// codec_dev.cuh -- device building blocks shared by the single-stream codec (codec.cu) and the
// batched codec (batch.cu): byte helpers, the decoupled look-back, TMA bulk staging, gap
// extraction and block packing/unpacking.
#pragma once

#include "fq_common.cuh"

namespace fq {

__device__ __forceinline__ uint64_t dpad16(uint64_t b) { return (b + 15u) & ~uint64_t(15); }
__device__ __forceinline__ uint64_t dcdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint32_t ld_u32(const uint8_t *p) { return *reinterpret_cast<const uint32_t *>(p); }


constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void publish(unsigned long long *status, uint64_t t, unsigned long long flag,
                                        unsigned long long value)
{
    __threadfence();
    atomicExch(status + t, flag | (value & kValueMask));
}

// CTA-wide: sum of the width sums of tiles 0 .. t-1 (t >= 1), by decoupled look-back.  Every
// thread polls one predecessor, so one round covers kEncThreads tiles: the running prefix moves
// that many tiles per L2 round trip.  All threads of the CTA must call it.
static __device__ unsigned long long lookback(unsigned long long *status, uint64_t t, Ctl *c, unsigned long long *red,
                                       uint32_t *s_first)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    unsigned long long excl = 0;
    long long base = (long long)t - 1;
    for (;;) {
        const long long idx = base - (long long)tid;
        unsigned long long w = kFlagPrefix;  // before tile 0: an empty prefix
        if (idx >= 0) {
            uint32_t spins = 0;
            w = ld_volatile_u64(status + idx);
            while ((w >> 62) == 0ull) {
                if (++spins > kSpinLimit) {
                    set_error(c, FQ_ETIMEOUT, kWhereEncWidths, (unsigned long long)idx);
                    w = kFlagPrefix;
                    break;
                }
                __nanosleep(32);
                w = ld_volatile_u64(status + idx);
            }
        }
        __threadfence();
        if (tid == 0) *s_first = kEncThreads;
        __syncthreads();
        if ((w >> 62) == 2ull) atomicMin(s_first, tid);  // nearest predecessor holding a full prefix
        __syncthreads();
        const uint32_t first = *s_first;
        unsigned long long val = (tid <= first) ? (w & kValueMask) : 0ull;
        val = warp_sum64(val);
        if (lane == 0) red[warp] = val;
        __syncthreads();
        unsigned long long sum = 0;
#pragma unroll
        for (uint32_t i = 0; i < kEncWarps; i++) sum += red[i];
        __syncthreads();
        excl += sum;
        if (first < kEncThreads) return excl;
        base -= kEncThreads;
    }
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

// Wait until phase `parity` of `bar` completes; bounded: gives up after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kSpinLimit; i++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
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


// Pack the 128 gaps of one block (4 per lane, slot 4*lane + j at bits [slot*b, slot*b + b)) into
// 4*b words staged in row (129+ words of shared memory), then return lane's 4 output words
// (meaningful for lane < b).  All 32 lanes must call it.
__device__ __forceinline__ uint4 pack_block(const uint32_t g[4], uint32_t b, uint32_t *row, uint32_t lane)
{
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
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (lane < b) q = make_uint4(row[4 * lane], row[4 * lane + 1], row[4 * lane + 2], row[4 * lane + 3]);
    __syncwarp();
    return q;
}

// Unpack one block of width b whose payload words start at pk (readable one word past the block),
// base = the block's first id.  Writes lane's four ids to out[] and returns false if the block is
// inconsistent (non-zero slot 0 or padding slot, u32 overflow); `last` receives lane's last value.
__device__ __forceinline__ bool unpack_block(const uint32_t *pk, uint32_t b, uint64_t base, uint64_t k, uint64_t n,
                                             uint32_t lane, uint32_t out[4], unsigned long long *last)
{
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
            const uint64_t two = ((uint64_t)pk[w0 + 1] << 32) | pk[w0];
            g = (uint32_t)(two >> sh) & mask;
        }
        const uint64_t idx = k * kBlock + slot;
        if (slot == 0 || idx >= n) {
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
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v += inc[j];
        out[j] = (uint32_t)v;
        if (i0 + j < n && v > 0xffffffffull) bad = true;
    }
    *last = v;
    return !bad;
}

}  // namespace fq
