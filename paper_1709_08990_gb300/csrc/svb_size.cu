// Compressed sizes without writing a stream: Stream VByte against VByte.
//
// Sec. 5 (Fig. 5b) reports how many more bits per integer Stream VByte needs
// than VByte on posting lists.  Both sizes are sums of per-value byte counts
// over the coded values (the integers, or their gaps to the previous one,
// Sec. 1 and Sec. 5):
//   Stream VByte  ceil(n/4) control bytes + L(v) = max(1, ceil(bits(v)/8))
//                 data bytes per value (Sec. 3-4);
//   VByte         max(1, ceil(bits(v)/7)) bytes per value: seven data bits
//                 and one continuation bit per byte (Sec. 2-3).
// One pass over the 4n input bytes: each thread takes whole quads with 16-byte
// loads (grid-stride, four loads in flight per thread), counts both lengths,
// and the block's totals go to two 64-bit counters.  Bound: HBM read bandwidth.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"

namespace svb {

constexpr int kSizeThreads = 256;

// Bytes of one value under Stream VByte: 1 + (v >= 2^8) + (v >= 2^16) + (v >= 2^24).
__device__ __forceinline__ uint32_t svb_bytes_of(uint32_t v)
{
    return 1u + (v >= (1u << 8)) + (v >= (1u << 16)) + (v >= (1u << 24));
}

// Bytes of one value under VByte: 1 + one per further 7-bit group.
__device__ __forceinline__ uint32_t vbyte_bytes_of(uint32_t v)
{
    return 1u + (v >= (1u << 7)) + (v >= (1u << 14)) + (v >= (1u << 21)) + (v >= (1u << 28));
}

struct SizeArgs {
    const uint32_t *in;
    u64 n;
    u64 *sums;   // [0] Stream VByte bytes, [1] VByte bytes; zero before the launch
    uint32_t prev;
    uint32_t delta;
    uint32_t aligned;   // in is 16-byte aligned
};

__global__ void __launch_bounds__(kSizeThreads) size_report_kernel(SizeArgs a)
{
    const u64 nq = a.n / 4;   // whole quads; the rest is the tail
    const u64 stride = (u64)gridDim.x * blockDim.x;
    u64 s_svb = 0, s_vb = 0;
    // kLoads quads per thread and round, their loads issued together.
    constexpr int kLoads = 4;
    for (u64 q0 = (u64)blockIdx.x * blockDim.x + threadIdx.x; q0 < nq; q0 += kLoads * stride) {
        uint32_t x[kLoads][4], before[kLoads];
#pragma unroll
        for (int k = 0; k < kLoads; k++) {
            const u64 q = q0 + k * stride;
            const bool in = q < nq;
            if (a.aligned) {
                const uint4 v = in ? ldg_stream128(a.in + 4 * q) : make_uint4(0, 0, 0, 0);
                x[k][0] = v.x;
                x[k][1] = v.y;
                x[k][2] = v.z;
                x[k][3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    x[k][j] = in ? __ldg(a.in + 4 * q + j) : 0u;
            }
            before[k] = a.delta && in ? (q ? __ldg(a.in + 4 * q - 1) : a.prev) : 0u;
        }
        uint32_t c_svb = 0, c_vb = 0;
#pragma unroll
        for (int k = 0; k < kLoads; k++) {
            if (q0 + k * stride >= nq)
                continue;
            uint32_t b = before[k];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t v = a.delta ? x[k][j] - b : x[k][j];
                b = x[k][j];
                c_svb += svb_bytes_of(v);
                c_vb += vbyte_bytes_of(v);
            }
        }
        s_svb += c_svb;
        s_vb += c_vb;
    }
    // The tail (n mod 4 values) and the control bytes, once.
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (u64 i = 4 * nq; i < a.n; i++) {
            const uint32_t x = __ldg(a.in + i);
            const uint32_t v = a.delta ? x - (i ? __ldg(a.in + i - 1) : a.prev) : x;
            s_svb += svb_bytes_of(v);
            s_vb += vbyte_bytes_of(v);
        }
        s_svb += (a.n + 3) / 4;
    }
    __shared__ u64 w_svb[kSizeThreads / 32], w_vb[kSizeThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_svb = warp_sum64(s_svb);
    s_vb = warp_sum64(s_vb);
    if (lane == 0) {
        w_svb[warp] = s_svb;
        w_vb[warp] = s_vb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t_svb = 0, t_vb = 0;
        for (int w = 0; w < kSizeThreads / 32; w++) {
            t_svb += w_svb[w];
            t_vb += w_vb[w];
        }
        atomicAdd(a.sums, t_svb);
        atomicAdd(a.sums + 1, t_vb);
    }
}

int launch_size_report(const uint32_t *in, u64 n, uint32_t prev, bool delta, u64 *d_sizes,
                       cudaStream_t stream)
{
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, size_report_kernel, kSizeThreads, 0);
        grid = (sms > 0 ? sms : 148) * (occ > 0 ? occ : 1);
    }
    if (cudaMemsetAsync(d_sizes, 0, 2 * sizeof(u64), stream) != cudaSuccess)
        return SVB_ECUDA;
    SizeArgs a;
    a.in = in;
    a.n = n;
    a.sums = d_sizes;
    a.prev = prev;
    a.delta = delta ? 1u : 0u;
    a.aligned = (((uintptr_t)in) & 15u) == 0;
    const u64 quads = n / 4;
    const u64 need = (quads + kSizeThreads - 1) / kSizeThreads;
    const unsigned g = (unsigned)std::max<u64>(1, std::min<u64>((u64)grid, need));
    prof_begin("size_report_kernel", stream);
    size_report_kernel<<<g, kSizeThreads, 0, stream>>>(a);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? SVB_OK : SVB_ECUDA;
}

}  // namespace svb

namespace {

// Two counters and their pinned host copy per device, for the sync form.
struct SizeCache {
    std::mutex mu;
    unsigned long long *d = nullptr;
    unsigned long long *h = nullptr;
};
constexpr int kMaxDevices = 64;
SizeCache g_size_cache[kMaxDevices];

}  // namespace

extern "C" int svb_size_report_async(const uint32_t *in, size_t n, uint32_t prev, int delta,
                                     uint64_t *d_sizes, svb_stream_t stream)
{
    if (!d_sizes || (n && !in)) {
        svb::set_last_error(SVB_EINVAL);
        return SVB_EINVAL;
    }
    int st = svb::launch_size_report(in, n, prev, delta != 0,
                                     reinterpret_cast<svb::u64 *>(d_sizes),
                                     reinterpret_cast<cudaStream_t>(stream));
    svb::set_last_error(st);
    return st;
}

extern "C" int svb_size_report(const uint32_t *in, size_t n, uint32_t prev, int delta,
                               uint64_t *sizes)
{
    if (!sizes || (n && !in)) {
        svb::set_last_error(SVB_EINVAL);
        return SVB_EINVAL;
    }
    if (n == 0) {
        sizes[0] = sizes[1] = 0;
        svb::set_last_error(SVB_OK);
        return SVB_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        svb::set_last_error(SVB_ECUDA);
        return SVB_ECUDA;
    }
    SizeCache &c = g_size_cache[dev];
    std::lock_guard<std::mutex> lock(c.mu);
    if (!c.d && cudaMalloc(&c.d, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        c.d = nullptr;
        svb::set_last_error(SVB_ENOMEM);
        return SVB_ENOMEM;
    }
    if (!c.h && cudaMallocHost(&c.h, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        c.h = nullptr;
        svb::set_last_error(SVB_ENOMEM);
        return SVB_ENOMEM;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(svb_get_stream());
    int st = svb::launch_size_report(in, n, prev, delta != 0, c.d, s);
    if (st == SVB_OK &&
        (cudaMemcpyAsync(c.h, c.d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
             cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        st = SVB_ECUDA;
    if (st == SVB_OK) {
        sizes[0] = c.h[0];
        sizes[1] = c.h[1];
    }
    svb::set_last_error(st);
    return st;
}
