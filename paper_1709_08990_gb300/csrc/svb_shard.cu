// The per-shard steps of coding one array split across several parties
// (GPUs, or shards on one GPU).
//
// Sec. 4 keeps the control bytes apart from the data so that where each
// integer's bytes start follows from the control bytes alone.  So a stream cut
// at control-byte boundaries needs only one small exchange: each shard sums
// the data bytes its control bytes cover (svb_control_range_bytes), an
// exclusive prefix over the shards' totals gives each shard's data offset,
// and the shard's control bytes followed by its data bytes are a stream of
// its own integers.  Differential streams (Sec. 2, Sec. 5) need a second
// exchange: each shard's sum of coded values (svb_gap_sum over that stream),
// whose exclusive prefix from prev is each shard's start value.
#include <cuda_runtime.h>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"

namespace svb {
namespace {

constexpr int kRangeThreads = 256;

// Data bytes covered by control byte c of quad qq (Sec. 4: 4 + the sum of
// its codes); quad nquads - 1 has last_nints integers and its pad fields
// count nothing.
__device__ __forceinline__ u64 quad_bytes(uint32_t c, u64 qq, u64 nquads, uint32_t last_nints)
{
    const uint32_t k = qq == nquads - 1 ? last_nints : 4u;
    if (k < 4)
        c &= (1u << (2 * k)) - 1u;
    return k + __popc(c & 0x55u) + 2u * __popc(c & 0xAAu);
}

// Grid-stride over the 16-byte-aligned chunks of addresses that meet
// [lo, hi) = [in + q0, in + q1): a chunk wholly inside by one 16-byte load,
// the ragged ends byte by byte (no byte outside [lo, hi) is read); one atomic
// add per CTA into *d_bytes (zeroed before the launch).
__global__ void __launch_bounds__(kRangeThreads) control_range_bytes_kernel(
    const uint8_t *in, u64 q0, u64 q1, u64 nquads, uint32_t last_nints,
    unsigned long long *d_bytes)
{
    const uintptr_t lo = (uintptr_t)(in + q0), hi = (uintptr_t)(in + q1);
    const uintptr_t a0 = lo & ~(uintptr_t)15;
    const u64 nchunks = (hi - a0 + 15) / 16;
    u64 t = 0;
    for (u64 c = blockIdx.x * (u64)blockDim.x + threadIdx.x; c < nchunks;
         c += (u64)gridDim.x * blockDim.x) {
        const uintptr_t addr = a0 + 16 * c;
        if (addr >= lo && addr + 16 <= hi) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(addr));
            const uint32_t x[4] = {v.x, v.y, v.z, v.w};
            const u64 q = (u64)(addr - (uintptr_t)in);
            if (q + 16 < nquads) {  // no last quad inside: every field counts
                t += 64;
#pragma unroll
                for (int i = 0; i < 4; i++)
                    t += __popc(x[i] & 0x55555555u) + 2u * __popc(x[i] & 0xAAAAAAAAu);
            } else {
#pragma unroll
                for (int b = 0; b < 16; b++)
                    t += quad_bytes((x[b >> 2] >> (8 * (b & 3))) & 0xffu, q + b, nquads,
                                    last_nints);
            }
        } else {
            for (int b = 0; b < 16; b++) {
                const uintptr_t ab = addr + b;
                if (ab >= lo && ab < hi)
                    t += quad_bytes(__ldg(reinterpret_cast<const uint8_t *>(ab)),
                                    (u64)(ab - (uintptr_t)in), nquads, last_nints);
            }
        }
    }
    t = warp_sum64(t);
    __shared__ u64 s_w[kRangeThreads / 32];
    if ((threadIdx.x & 31) == 0)
        s_w[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 s = 0;
        for (int i = 0; i < kRangeThreads / 32; i++)
            s += s_w[i];
        if (s)
            atomicAdd(d_bytes, (unsigned long long)s);
    }
}

}  // namespace
}  // namespace svb

extern "C" int svb_control_range_bytes(const uint8_t *in, size_t n, size_t q0, size_t q1,
                                       uint64_t *d_bytes, svb_stream_t stream)
{
    using svb::u64;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const u64 nquads = ((u64)n + 3) / 4;
    if (!d_bytes || q0 > q1 || q1 > nquads || (q1 > q0 && !in))
        return SVB_EINVAL;
    if (cudaMemsetAsync(d_bytes, 0, sizeof(uint64_t), s) != cudaSuccess)
        return SVB_ECUDA;
    if (q1 == q0)
        return SVB_OK;
    const uint32_t last_nints = (uint32_t)(n - 4 * (nquads - 1));
    const u64 chunks = (q1 - q0) / 16 + 2;
    const u64 blocks = (chunks + svb::kRangeThreads - 1) / svb::kRangeThreads;
    const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
    svb::prof_begin("control_range_bytes_kernel", s);
    svb::control_range_bytes_kernel<<<grid, svb::kRangeThreads, 0, s>>>(
        in, q0, q1, nquads, last_nints, reinterpret_cast<unsigned long long *>(d_bytes));
    svb::prof_end(s);
    return cudaGetLastError() == cudaSuccess ? SVB_OK : SVB_ECUDA;
}
