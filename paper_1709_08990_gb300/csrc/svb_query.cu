// Seek and select on compressed lists (the operations benchmarked at the end
// of Sec. 5, Fig. 6), many queries in one launch.
//
//   seek(target)  index of the first integer >= target in a list, and that
//                 integer (n and 0 when there is none);
//   select(i)     the integer at index i.
// Both work on the compressed bytes directly, as the paper's point is: one
// warp per query walks its list 32 quads (128 integers) at a time.  Each lane
// takes one quad: its control byte gives the quad's data bytes (Sec. 4), a
// warp scan gives every quad's data offset, the lane reads its integers
// little-endian (Sec. 4), and for differential coding quad sums, a warp scan
// and the carry of the chunks before turn gaps into integers (Sec. 2).  The
// walk stops at the chunk holding the answer.  A plain select only needs the
// control bytes before its quad, so it skips decoding those chunks.
//
// A list's stream must hold all its control bytes; data bytes past the
// stream's end are never read, and an answer whose integer they would hold
// is reported as SVB_ETRUNCATED (data offsets only grow, so every integer
// before an intact one is intact too).
#include <cuda_runtime.h>

#include <algorithm>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"

namespace svb {

constexpr int kQueryThreads = 256;

struct QueryArgs {
    const svb_list *lists;
    u64 num_lists;
    const uint8_t *in;
    const svb_query *queries;
    u64 num_queries;
    svb_answer *answers;
    uint32_t delta;
};

__device__ __forceinline__ void answer(svb_answer *a, u64 index, uint32_t value, uint32_t status)
{
    a->index = index;
    a->value = value;
    a->status = status;
}

__global__ void __launch_bounds__(kQueryThreads) query_kernel(QueryArgs a)
{
    const int lane = threadIdx.x & 31;
    const u64 warps = (u64)gridDim.x * (kQueryThreads / 32);
    for (u64 qi = ((u64)blockIdx.x * kQueryThreads + threadIdx.x) / 32; qi < a.num_queries;
         qi += warps) {
        const svb_query q = a.queries[qi];
        svb_answer *out = a.answers + qi;
        if (q.list >= a.num_lists || (q.op != SVB_SEEK && q.op != SVB_SELECT)) {
            if (lane == 0)
                answer(out, 0, 0, SVB_EINVAL);
            continue;
        }
        const svb_list L = a.lists[q.list];
        const u64 n = L.n, nq = (n + 3) / 4;
        const bool seek = q.op == SVB_SEEK;
        if (!seek && q.arg >= n) {
            if (lane == 0)
                answer(out, q.arg, 0, SVB_EINVAL);
            continue;
        }
        if (seek && n == 0) {
            if (lane == 0)
                answer(out, 0, 0, SVB_OK);
            continue;
        }
        if (L.in_len < nq) {   // every control byte is needed
            if (lane == 0)
                answer(out, seek ? 0 : q.arg, 0, SVB_ETRUNCATED);
            continue;
        }
        const uint8_t *ctrl = a.in + L.in_off;
        const uint8_t *data = ctrl + nq;
        const u64 dlen = L.in_len - nq;
        const uint32_t last_nints = (uint32_t)(n - 4 * (nq - 1));
        const uint32_t target = (uint32_t)q.arg;
        u64 base = 0;             // data offset of the chunk
        uint32_t carry = L.prev;  // differential: the integer before the chunk
        bool done = false;
        for (u64 c0 = 0; c0 < nq && !done; c0 += 32) {
            const u64 quad = c0 + lane;
            const bool valid = quad < nq;
            const uint32_t nints = !valid ? 0u : (quad == nq - 1 ? last_nints : 4u);
            uint32_t c = valid ? ctrl[quad] : 0u;
            if (nints < 4)
                c &= (1u << (2 * nints)) - 1u;
            const uint32_t bytes = nints ? quad_count(c, nints) : 0u;
            const uint32_t incl = warp_incl_scan(bytes);
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const u64 chunk_end = 4 * (c0 + 32);   // first integer after the chunk
            if (!seek && !a.delta && q.arg >= chunk_end) {
                base += total;    // plain select: this chunk only moves the offset
                continue;
            }
            // This lane's integers, and whether their bytes are all present.
            u64 p = base + incl - bytes;
            uint32_t v[4], cut = 0;   // bit j: integer j lies past the stream's end
#pragma unroll
            for (int j = 0; j < 4; j++) {
                v[j] = 0;
                if ((uint32_t)j < nints) {
                    const uint32_t len = ((c >> (2 * j)) & 3u) + 1;
                    if (p + len <= dlen) {
                        for (uint32_t b = 0; b < len; b++)
                            v[j] |= (uint32_t)data[p + b] << (8 * b);
                    } else {
                        cut |= 1u << j;
                    }
                    p += len;
                }
            }
            if (a.delta) {
                v[1] += v[0];
                v[2] += v[1];
                v[3] += v[2];
                const uint32_t qs = v[3];   // pad fields decode to 0
                const uint32_t qincl = warp_incl_scan(qs);
                const uint32_t add = carry + qincl - qs;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    v[j] += add;
                carry += __shfl_sync(0xffffffffu, qincl, 31);
            }
            // The deciding integer of this chunk, if any: for seek the first
            // that is >= target or cut off; for select integer q.arg.
            int hit = -1;
            if (seek) {
#pragma unroll
                for (int j = 3; j >= 0; j--)
                    if ((uint32_t)j < nints && (((cut >> j) & 1u) || v[j] >= target))
                        hit = j;
            } else if (q.arg >= 4 * c0 && q.arg < chunk_end && (q.arg - 4 * c0) / 4 == (u64)lane) {
                hit = (int)(q.arg & 3u);
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit >= 0);
            if (m) {
                const int src = __ffs(m) - 1;
                if (lane == src) {
                    const u64 idx = 4 * quad + hit;
                    uint32_t val = 0;
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        val = j == hit ? v[j] : val;
                    if ((cut >> hit) & 1u)
                        answer(out, idx, 0, SVB_ETRUNCATED);
                    else
                        answer(out, idx, val, SVB_OK);
                }
                done = true;
            }
            base += total;
        }
        if (!done && lane == 0)
            answer(out, n, 0, SVB_OK);   // seek: no integer >= target
    }
}

int launch_query(const svb_list *lists, u64 num_lists, const uint8_t *in, bool delta,
                 const svb_query *queries, u64 num_queries, svb_answer *answers,
                 cudaStream_t stream)
{
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, query_kernel, kQueryThreads, 0);
        grid = (sms > 0 ? sms : 148) * (occ > 0 ? occ : 1);
    }
    if (num_queries == 0)
        return SVB_OK;
    QueryArgs a;
    a.lists = lists;
    a.num_lists = num_lists;
    a.in = in;
    a.queries = queries;
    a.num_queries = num_queries;
    a.answers = answers;
    a.delta = delta ? 1u : 0u;
    const u64 need = (num_queries + kQueryThreads / 32 - 1) / (kQueryThreads / 32);
    const unsigned g = (unsigned)std::max<u64>(1, std::min<u64>((u64)grid, need));
    prof_begin("query_kernel", stream);
    query_kernel<<<g, kQueryThreads, 0, stream>>>(a);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? SVB_OK : SVB_ECUDA;
}

}  // namespace svb

extern "C" int svb_query_batch(const svb_list *d_lists, size_t num_lists, const uint8_t *in_base,
                               int delta, const svb_query *d_queries, size_t num_queries,
                               svb_answer *d_answers, svb_stream_t stream)
{
    if (num_queries && (!d_lists || !in_base || !d_queries || !d_answers)) {
        svb::set_last_error(SVB_EINVAL);
        return SVB_EINVAL;
    }
    int st = svb::launch_query(d_lists, num_lists, in_base, delta != 0, d_queries, num_queries,
                               d_answers, reinterpret_cast<cudaStream_t>(stream));
    svb::set_last_error(st);
    return st;
}
