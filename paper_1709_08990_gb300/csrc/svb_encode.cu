// Stream VByte encoding on sm_103a, plain and differential, in one pass.
//
// What is computed (arXiv 1709.08990): the paper prints no encoder; it is the
// inverse of the format.  Each coded value v (the integer itself, or its gap
// to the previous integer, the first gap taken from prev, Sec. 1 and Sec. 5)
// takes L(v) = ceil(log_256(v + 1)) bytes, at least one (Sec. 3); control
// byte q packs L - 1 of integers 4q..4q+3, first in the low bits (Fig. 3);
// the data stream follows the ceil(N/4) control bytes and holds each value's
// L low-order bytes, least significant first (Sec. 4).
//
// How (one CTA per tile of kEncQuads quads, tiles in atomic-counter order):
//   1. each lane loads one quad per round (16-byte loads), forms the gaps
//      (the neighbour quad's last value comes by shuffle or one extra load),
//      the lengths from count-leading-zeros, the control byte, and stores
//      the control byte;
//   2. block scan of the per-quad byte counts and a decoupled look-back over
//      the tiles' totals give every quad its byte offset in the data stream;
//   3. the tile's data bytes are assembled in shared memory, aligned like
//      their destination, and written with 16-byte stores (the partial
//      chunks at both ends byte by byte, so neighbouring tiles never write
//      the same byte).
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"

namespace svb {

constexpr int kEncQuads = 1024;
constexpr int kEncRounds = kEncQuads / kThreads;
constexpr int kEncDataMax = 16 * kEncQuads;
constexpr int kEncStage = kEncDataMax + 32;
constexpr int kEncChunks = (kEncDataMax + 16 + 15) / 16;
constexpr int kEncChunkIters = (kEncChunks + kThreads - 1) / kThreads;

struct EncodeArgs {
    const uint32_t *in;
    u64 n;
    uint8_t *out;
    u64 nquads;
    u64 ntiles;
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    uint32_t prev;
    uint32_t in_aligned;
    uint32_t delta;
};

// Sec. 3: bytes of v, 1..4 (zero takes one byte).
__device__ __forceinline__ uint32_t byte_len(uint32_t v)
{
    return max(1u, (39u - (uint32_t)__clz(v)) >> 3);
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads, 4) encode_kernel(EncodeArgs a)
{
    __shared__ __align__(16) uint8_t s_data[kEncStage];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ u64 s_tile, s_etag, s_base;
    __shared__ uint32_t s_skip;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_tile = atomicAdd(&a.hdr->tile_counter, 1ull);
        s_etag = epoch_tag(a.hdr);
        s_skip = (s_tile >= a.ntiles || error_raised(a.hdr)) ? 1u : 0u;
    }
    __syncthreads();
    const u64 tile = s_tile, etag = s_etag;
    if (s_skip) {
        finish_launch(a.hdr, a.result);
        return;
    }

    const u64 q0 = tile * kEncQuads;
    const uint32_t nq = (uint32_t)min((u64)kEncQuads, a.nquads - q0);
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));

    // ---- 1. values -> gaps -> lengths -> control bytes --------------------
    uint32_t d[kEncRounds][4];
    uint32_t ctrl[kEncRounds];
    uint32_t qexcl[kEncRounds];
    uint32_t wrun = 0;
#pragma unroll
    for (int r = 0; r < kEncRounds; r++) {
        const uint32_t lq = warp * (32 * kEncRounds) + r * 32 + lane;
        const bool valid = lq < nq;
        const u64 Q = q0 + lq;
        const uint32_t nints = !valid ? 0u : (Q == a.nquads - 1 ? last_nints : 4u);
        uint32_t x[4] = {0, 0, 0, 0};
        if (nints == 4 && a.in_aligned) {
            uint4 t = __ldg(reinterpret_cast<const uint4 *>(a.in) + Q);
            x[0] = t.x;
            x[1] = t.y;
            x[2] = t.z;
            x[3] = t.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if ((uint32_t)k < nints)
                    x[k] = __ldg(a.in + 4 * Q + k);
        }
        if (kDelta) {
            uint32_t before = __shfl_up_sync(0xffffffffu, x[3], 1);
            if (lane == 0 && valid)
                before = Q == 0 ? a.prev : __ldg(a.in + 4 * Q - 1);
            d[r][0] = x[0] - before;
            d[r][1] = x[1] - x[0];
            d[r][2] = x[2] - x[1];
            d[r][3] = x[3] - x[2];
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++)
                d[r][k] = x[k];
        }
        uint32_t c = 0, C = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if ((uint32_t)k < nints) {
                uint32_t L = byte_len(d[r][k]);
                c |= (L - 1) << (2 * k);
                C += L;
            }
        }
        ctrl[r] = c;
        if (valid)
            a.out[Q] = (uint8_t)c;
        uint32_t inc = warp_incl_scan(C);
        qexcl[r] = wrun + inc - C;
        wrun += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0)
        s_warp[warp] = wrun;
    __syncthreads();
    uint32_t bpre = 0, agg = 0;
#pragma unroll
    for (int k = 0; k < kWarps; k++) {
        uint32_t t = s_warp[k];
        bpre += k < warp ? t : 0u;
        agg += t;
    }

    // ---- 2. tile offset (look-back) ---------------------------------------
    if (warp == 0) {
        u64 base = 0;
        bool ok = true;
        TileStatus *me = &a.st[tile];
        if (tile == 0) {
            if (lane == 0)
                publish(&me->off_tag, &me->off_pre, agg, kFlagPrefix, etag);
        } else {
            if (lane == 0)
                publish(&me->off_tag, &me->off_agg, agg, kFlagAgg, etag);
            base = lookback<false>(a.st, tile, etag, a.spin_limit, a.hdr, ok);
            if (ok && lane == 0)
                publish(&me->off_tag, &me->off_pre, base + agg, kFlagPrefix, etag);
        }
        if (lane == 0) {
            if (!ok)
                raise_error(a.hdr, kErrTimeout);
            else if (tile == a.ntiles - 1)
                st_relaxed(&a.hdr->total, a.nquads + base + agg);
            s_base = base;
            s_skip = ok ? 0u : 1u;
        }
    }
    __syncthreads();
    if (s_skip) {
        finish_launch(a.hdr, a.result);
        return;
    }

    // ---- 3. assemble the tile's data bytes, then write them out -----------
    uint8_t *dst = a.out + a.nquads + s_base;
    const uint32_t h = (uint32_t)((uintptr_t)dst & 15u);
#pragma unroll
    for (int r = 0; r < kEncRounds; r++) {
        uint32_t p = h + bpre + qexcl[r];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            uint32_t code = (ctrl[r] >> (2 * k)) & 3u;
            const uint32_t lq = warp * (32 * kEncRounds) + r * 32 + lane;
            const uint32_t nints =
                lq >= nq ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
            if ((uint32_t)k < nints) {
                uint32_t val = d[r][k];
#pragma unroll
                for (uint32_t b = 0; b < 4; b++)
                    if (b <= code)
                        s_data[p + b] = (uint8_t)(val >> (8 * b));
                p += code + 1;
            }
        }
    }
    __syncthreads();
    uint8_t *adst = dst - h;
    const uint32_t nchunks = (h + agg + 15u) >> 4;
#pragma unroll
    for (int i = 0; i < kEncChunkIters; i++) {
        uint32_t k = tid + i * kThreads;
        if (k < nchunks) {
            if (16u * k >= h && 16u * k + 16u <= h + agg) {
                stg_stream128(adst + 16u * k, *reinterpret_cast<const uint4 *>(s_data + 16u * k));
            } else {
                for (uint32_t b = 0; b < 16; b++) {
                    uint32_t idx = 16u * k + b;
                    if (idx >= h && idx < h + agg)
                        adst[idx] = s_data[idx];
                }
            }
        }
    }
    finish_launch(a.hdr, a.result);
}

int launch_encode(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta, void *ws,
                  DeviceResult *result, cudaStream_t stream, u64 spin_limit)
{
    EncodeArgs a;
    a.in = in;
    a.n = n;
    a.out = out;
    a.nquads = (n + 3) / 4;
    a.ntiles = (a.nquads + kEncQuads - 1) / kEncQuads;
    a.hdr = reinterpret_cast<WsHeader *>(ws);
    a.st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + ws_layout(n).status);
    a.result = result;
    a.spin_limit = spin_limit;
    a.prev = prev;
    a.in_aligned = (((uintptr_t)in) & 15u) == 0;
    a.delta = delta;
    dim3 grid((unsigned)a.ntiles);
    prof_begin(delta ? "encode_kernel<delta>" : "encode_kernel<plain>", stream);
    if (delta)
        encode_kernel<true><<<grid, kThreads, 0, stream>>>(a);
    else
        encode_kernel<false><<<grid, kThreads, 0, stream>>>(a);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

u64 encode_tiles(u64 n)
{
    u64 nq = (n + 3) / 4;
    return (nq + kEncQuads - 1) / kEncQuads;
}

}  // namespace svb
