// svb_decode_noalloc: the reduce-then-decode decoder with its scratch in a
// fixed, file-scope device array instead of memory the library allocates.
//
// Who needs it: code that must not allocate device memory while it decodes,
// for instance a custom allocator or memory pool that decodes from inside its
// own bookkeeping (a nested cudaMalloc would re-enter or deadlock it), a
// framework that has reserved nearly all of HBM for its caching allocator (a
// stray cudaMalloc fails or fragments the pool), or a latency-bound serving
// path that cannot afford cudaMalloc/cudaFree, which may synchronize the
// device.  The regular synchronous calls allocate a workspace on first use
// and a pinned result buffer; this one never does.
//
// The scratch holds the workspace of one decode of up to SVB_NOALLOC_MAX_N
// integers (about 1.5 MB).  Every GPU that loads the library keeps it until
// the process exits.  All calls share it, so calls that overlap on the GPU
// race: order them on one stream or serialize them on the host.
#include <cuda_runtime.h>

#include <mutex>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"

namespace {

using svb::u64;

// Workspace bytes of one decode of SVB_NOALLOC_MAX_N integers, laid out as
// svb::ws_layout lays it out (header, sub-tile offsets and carries, records).
constexpr u64 kNoAllocBytes = svb::ws_layout(SVB_NOALLOC_MAX_N).total;

// Zero-initialised when the module loads; never freed.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code may not take the array's address: in host code its name stands
// for a host-side shadow.  The device address is looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

size_t noalloc_fail(int code)
{
    svb::set_last_error(code);
    return SVB_ERROR;
}

}  // namespace

extern "C" size_t svb_decode_noalloc(const uint8_t *in, size_t in_len, size_t n,
                                     uint32_t *out, uint32_t prev, int delta,
                                     svb_stream_t stream)
{
    if (n == 0) {
        svb::set_last_error(SVB_OK);
        return 0;
    }
    if (!in || !out)
        return noalloc_fail(SVB_EINVAL);
    if ((u64)n > (u64)SVB_NOALLOC_MAX_N)
        return noalloc_fail(SVB_EINVAL);  // beyond the fixed scratch
    if (in_len < ((u64)n + 3) / 4)
        return noalloc_fail(SVB_ETRUNCATED);
    if (svb::ws_layout(n).total > kNoAllocBytes)
        return noalloc_fail(SVB_EINVAL);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SVB_ECUDA);
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // First call on this device (it is current): find the array.
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return noalloc_fail(SVB_ECUDA);
            g_noalloc_ptr[dev] = p;
        }
        ws = g_noalloc_ptr[dev];
    }

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    svb::WsHeader *hdr = static_cast<svb::WsHeader *>(ws);
    // The counters and the error word must start at zero.  The epoch is left
    // as the last call left it: records of earlier calls carry older epochs
    // in their tags, and whatever else an earlier call of another size left
    // where this call's records lie never has a tag's mark bit (see
    // svb::TileStatus), so nothing stale reads as published.
    if (cudaMemsetAsync(&hdr->tile_counter, 0, 2 * sizeof(u64), s) != cudaSuccess ||
        cudaMemsetAsync(&hdr->error, 0, 4 * sizeof(u64), s) != cudaSuccess)
        return noalloc_fail(SVB_ECUDA);
    auto *res = reinterpret_cast<svb::DeviceResult *>(static_cast<char *>(ws) +
                                                      svb::kResultOffset);
    u64 limit = 1ull << 21;
    if (svb::launch_decode_tiled(in, in_len, n, out, prev, delta != 0, ws, res, s, limit) != 0)
        return noalloc_fail(SVB_ECUDA);
    svb_result h = {0, 0};  // pageable: no pinned buffer is allocated
    if (cudaMemcpyAsync(&h, res, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(SVB_ECUDA);
    if (h.status != SVB_OK)
        return noalloc_fail((int)h.status);
    svb::set_last_error(SVB_OK);
    return (size_t)h.bytes;
}
