// codec_static.cu -- fq_frontier_encode_static: the frontier encode without a caller workspace.
//
// Who needs it: code that runs where device allocation is off limits -- for example a plugin
// invoked inside another framework's memory pool (which must not see foreign cudaMalloc/cudaFree
// calls), or a real-time path that may not call into the allocator (cudaMalloc/cudaFree can
// synchronise the device and take unbounded time).  Such a caller still owns its input and output
// buffers but cannot provide scratch, so the encoder's scratch (per-block widths and bases,
// per-tile sums and offsets, the status record) lives in one fixed array in device memory
// declared below.  Every GPU that loads this library reserves that array until the process
// exits, which is why its size is kept modest (FQ_STATIC_MAX_IDS ids).
//
// The kernels are the ones fq_frontier_encode launches; only the scratch location differs.
#include <mutex>

#include "fq_common.cuh"

namespace {

// Scratch for encoding up to FQ_STATIC_MAX_IDS ids: the encoder's workspace layout for 2^24 ids
// takes 1,344,256 bytes (status record 256; per 128-id block a width byte, a u32 base, a u32
// block offset and an exception byte, 10 B x 131,072 blocks; per 8,192-id tile four u32 sums,
// 4 x 8 KiB; two bitmap-tile words, padded to 256 B each).  2 MiB are reserved, and every call
// checks its own layout against them.
constexpr size_t kStaticScratchBytes = 2u << 20;
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device.  In host code the array's name is
// only a host-side stand-in, so the address is asked from the runtime, once per device.
cudaError_t static_scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" fq_status fq_frontier_encode_static(const uint32_t *d_ids, uint64_t n, uint8_t *d_out, uint64_t cap,
                                               uint64_t *d_out_bytes, void *stream)
{
    if ((n && !d_ids) || !d_out || !d_out_bytes) return FQ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_ids) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u)) return FQ_EINVAL;
    if (n > FQ_STATIC_MAX_IDS) return FQ_EINVAL;  // beyond the fixed scratch: nothing is enqueued
    if (fq::workspace_bytes(n, 0) > kStaticScratchBytes) return FQ_EINVAL;
    void *scratch = nullptr;
    cudaError_t e = static_scratch_address(&scratch);
    if (e != cudaSuccess) {
        fq::note_cuda_error(e, __LINE__);
        return FQ_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fq::Scratch s = fq::carve(scratch, n, 0);
    // the status record must start cleared; the rest is rewritten by each call
    e = fq::reset_status(s, n, st);
    if (e == cudaSuccess) e = fq::encode_fq(d_ids, n, nullptr, n, d_out, cap, d_out_bytes, s, st);
    if (e != cudaSuccess) {
        fq::note_cuda_error(e, __LINE__);
        return FQ_ECUDA;
    }
    return FQ_OK;
}
