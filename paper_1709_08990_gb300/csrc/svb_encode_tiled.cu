// Stream VByte encoding of one array, chunked single pass over DRAM.
//
// What is computed is the inverse of the format (Sec. 3-4): each coded value
// v (the integer, or its gap to the previous one with the first gap taken from
// prev, Sec. 1 and Sec. 5) takes L(v) in {1,2,3,4} bytes (Sec. 3), control byte
// q packs L - 1 of integers 4q..4q+3 (first in the low bits, Fig. 3), and the
// data stream after the ceil(N/4) control bytes holds each value's L low-order
// bytes (Sec. 4).
//
// The only serial dependency is where each tile's data bytes go: the sum of
// all earlier lengths.  Persistent CTAs claim chunks of kChunkTiles tiles in
// order.  For each chunk the producer warp streams the values in twice with
// bulk copies (cp.async.bulk, mbarrier completion):
//   sizing pass   the consumers only sum the byte lengths of each tile;
//                 one decoupled look-back per chunk then gives the chunk's
//                 offset in the data stream;
//   writing pass  the consumers form gaps, lengths and control bytes, store the
//                 control bytes, assemble each tile's data bytes in shared
//                 memory aligned like their destination and store them with
//                 16-byte writes (ragged ends byte by byte).
// The second read of a chunk comes from L2 (the chunks in flight on the whole
// GPU take far less than its 129 MB), so DRAM sees each value once.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"

namespace svb {

constexpr int kEtQuads = 1024;                  // quads per tile (4096 values)
constexpr int kEtRounds = kEtQuads / kThreads;
constexpr int kChunkTiles = 8;                  // tiles per look-back unit
constexpr int kEtStages = 3;
constexpr int kEtStageBytes = 16 * kEtQuads + 16;
constexpr int kEtOutBytes = 16 * kEtQuads + 32;
constexpr int kEtBlock = kThreads + 32;
constexpr u64 kEtPolls = 1ull << 24;
constexpr uint32_t kEtNone = 0xffffffffu;

struct EncTiledArgs {
    const uint32_t *in;
    u64 n, nquads, ntiles, nchunks;
    uint8_t *out;
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    uint32_t prev;
    uint32_t delta;
};

struct EtPipe {
    uint8_t vals[kEtStages][kEtStageBytes];
    uint8_t outb[kEtOutBytes];
    uint64_t full[kEtStages];
    uint64_t empty[kEtStages];
    uint32_t tile[kEtStages];   // tile index, or kEtNone
    uint32_t pass[kEtStages];   // 0 sizing, 1 writing
    uint32_t hv[kEtStages];     // phase (mod 16) of the staged values
};

__device__ void et_produce(const EncTiledArgs &a, EtPipe &P, int lane)
{
    uint32_t issued = 0;
    uint32_t g = 0;
    bool stop = false;
    auto post = [&](uint32_t tile, uint32_t pass) -> bool {
        const int s = g % kEtStages;
        if (g >= (uint32_t)kEtStages) {
            bool ok = mbar_wait_bounded(&P.empty[s], ((g / kEtStages) - 1) & 1u, kEtPolls);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0)
                    raise_error(a.hdr, kErrTimeout);
                return false;
            }
        }
        if (tile == kEtNone) {
            if (lane == 0) {
                P.tile[s] = kEtNone;
                mbar_arrive_expect_tx(&P.full[s], 0);
            } else {
                mbar_arrive(&P.full[s]);
            }
        } else {
            const u64 i0 = (u64)tile * 4 * kEtQuads;
            const uint32_t cnt = (uint32_t)min((u64)4 * kEtQuads, a.n - i0);
            const uint8_t *gv = reinterpret_cast<const uint8_t *>(a.in + i0);
            range_edges(gv, 4 * cnt, P.vals[s], lane);
            if (lane == 0) {
                const uint8_t *av;
                uint32_t ov;
                uint32_t bv = range_interior(gv, 4 * cnt, av, ov);
                P.tile[s] = tile;
                P.pass[s] = pass;
                P.hv[s] = (uint32_t)((uintptr_t)gv & 15u);
                mbar_arrive_expect_tx(&P.full[s], bv);
                if (bv)
                    bulk_g2s(P.vals[s] + ov, av, bv, &P.full[s]);
            } else {
                mbar_arrive(&P.full[s]);
            }
        }
        g++;
        issued = g;
        return true;
    };
    for (;;) {
        u64 c = 0;
        if (lane == 0)
            c = atomicAdd(&a.hdr->tile_counter, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= a.nchunks) {
            post(kEtNone, 0);
            break;
        }
        const uint32_t t0 = (uint32_t)(c * kChunkTiles);
        const uint32_t t1 = (uint32_t)min((u64)t0 + kChunkTiles, a.ntiles);
        for (uint32_t t = t0; t < t1 && !stop; t++)
            stop = !post(t, 0);
        for (uint32_t t = t0; t < t1 && !stop; t++)
            stop = !post(t, 1);
        if (stop)
            break;
    }
    if (lane == 0) {
        for (int s = 0; s < kEtStages; s++)
            if (issued > (uint32_t)s) {
                uint32_t fills = (issued - 1 - s) / kEtStages + 1;
                mbar_wait_bounded(&P.full[s], (fills - 1) & 1u, kEtPolls);
            }
    }
    __syncwarp();
}

// Gaps (or values) of one quad from the staged tile; lq is the tile-local quad.
__device__ __forceinline__ void et_quad(const EncTiledArgs &a, const uint32_t *V, u64 q0,
                                        uint32_t lq, uint32_t nints, uint32_t (&d)[4])
{
    uint32_t x[4];
#pragma unroll
    for (int j = 0; j < 4; j++)
        x[j] = (uint32_t)j < nints ? V[4 * lq + j] : 0u;
    if (a.delta) {
        uint32_t pv;
        if (lq > 0)
            pv = V[4 * lq - 1];
        else
            pv = q0 == 0 ? a.prev : __ldg(a.in + 4 * q0 - 1);
        d[0] = x[0] - pv;
        d[1] = x[1] - x[0];
        d[2] = x[2] - x[1];
        d[3] = x[3] - x[2];
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            d[j] = x[j];
    }
}

__device__ void et_consume(const EncTiledArgs &a, EtPipe &P, uint32_t *s_warp,
                           uint32_t *s_tt, u64 *s_tb, u64 etag)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    uint32_t chunk_tiles = 0;  // sizing-pass tiles seen in the current chunk
    for (uint32_t g = 0;; g++) {
        const int s = g % kEtStages;
        if (!mbar_wait_bounded(&P.full[s], (g / kEtStages) & 1u, kEtPolls)) {
            raise_error(a.hdr, kErrTimeout);
            break;
        }
        const uint32_t tile = P.tile[s];
        if (tile == kEtNone)
            break;
        const uint32_t pass = P.pass[s];
        const u64 q0 = (u64)tile * kEtQuads;
        const uint32_t nq = (uint32_t)min((u64)kEtQuads, a.nquads - q0);
        const uint32_t *V = reinterpret_cast<const uint32_t *>(P.vals[s] + P.hv[s]);
        const uint32_t lq0 = warp * (32 * kEtRounds) + lane;

        if (pass == 0) {
            // ---- sizing: bytes of this tile's data ---------------------------
            uint32_t t = 0;
#pragma unroll
            for (int r = 0; r < kEtRounds; r++) {
                const uint32_t lq = lq0 + r * 32;
                const uint32_t nints = lq >= nq ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
                uint32_t d[4];
                et_quad(a, V, q0, lq, nints, d);
#pragma unroll
                for (int j = 0; j < 4; j++)
                    t += (uint32_t)j < nints ? byte_len(d[j]) : 0u;
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&P.empty[s]);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1)
                t += __shfl_xor_sync(0xffffffffu, t, d);
            if (lane == 0)
                s_warp[warp] = t;
            named_sync(1, kThreads);
            if (tid == 0) {
                uint32_t tt = 0;
#pragma unroll
                for (int j = 0; j < kWarps; j++)
                    tt += s_warp[j];
                s_tt[chunk_tiles] = tt;
            }
            chunk_tiles++;
            const u64 chunk = tile / kChunkTiles;
            const bool last_of_chunk = tile + 1 == a.ntiles || (tile + 1) % kChunkTiles == 0;
            named_sync(1, kThreads);
            if (last_of_chunk) {
                // ---- the chunk's offset: one look-back ------------------------
                if (warp == 0) {
                    uint32_t tt = lane < (int)chunk_tiles ? s_tt[lane] : 0u;
                    uint32_t inc = warp_incl_scan(tt);
                    const u64 agg = __shfl_sync(0xffffffffu, inc, 31);
                    TileStatus *me = &a.st[chunk];
                    u64 base = 0;
                    bool ok = true;
                    if (chunk == 0) {
                        if (lane == 0)
                            publish(&me->off_tag, &me->off_pre, agg, kFlagPrefix, etag);
                    } else {
                        if (lane == 0)
                            publish(&me->off_tag, &me->off_agg, agg, kFlagAgg, etag);
                        base = lookback<false>(a.st, chunk, etag, a.spin_limit, a.hdr, ok);
                        if (ok && lane == 0)
                            publish(&me->off_tag, &me->off_pre, base + agg, kFlagPrefix, etag);
                    }
                    if (!ok && lane == 0)
                        raise_error(a.hdr, kErrTimeout);
                    if (lane < (int)chunk_tiles)
                        s_tb[lane] = base + (inc - tt);
                    if (chunk + 1 == a.nchunks && lane == 0)
                        st_relaxed(&a.hdr->total, a.nquads + base + agg);
                }
                chunk_tiles = 0;
                named_sync(1, kThreads);
            }
            continue;
        }

        // ---- writing: control bytes and data bytes of this tile ---------------
        uint32_t d[kEtRounds][4], ctrl[kEtRounds], qexcl[kEtRounds], wrun = 0;
#pragma unroll
        for (int r = 0; r < kEtRounds; r++) {
            const uint32_t lq = lq0 + r * 32;
            const uint32_t nints = lq >= nq ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
            et_quad(a, V, q0, lq, nints, d[r]);
            uint32_t c = 0, C = 0;
#pragma unroll
            for (int j = 0; j < 4; j++)
                if ((uint32_t)j < nints) {
                    const uint32_t L = byte_len(d[r][j]);
                    c |= (L - 1) << (2 * j);
                    C += L;
                }
            ctrl[r] = c;
            if (nints)
                a.out[q0 + lq] = (uint8_t)c;
            const uint32_t inc = warp_incl_scan(C);
            qexcl[r] = wrun + inc - C;
            wrun += __shfl_sync(0xffffffffu, inc, 31);
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.empty[s]);
        if (lane == 0)
            s_warp[warp] = wrun;
        named_sync(1, kThreads);
        uint32_t bpre = 0, agg = 0;
#pragma unroll
        for (int j = 0; j < kWarps; j++) {
            const uint32_t t = s_warp[j];
            bpre += j < warp ? t : 0u;
            agg += t;
        }
        const u64 tbase = s_tb[tile % kChunkTiles];
        uint8_t *dst = a.out + a.nquads + tbase;
        const uint32_t h = (uint32_t)((uintptr_t)dst & 15u);
#pragma unroll
        for (int r = 0; r < kEtRounds; r++) {
            const uint32_t lq = lq0 + r * 32;
            const uint32_t nints = lq >= nq ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
            uint32_t p = h + bpre + qexcl[r];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if ((uint32_t)j < nints) {
                    const uint32_t code = (ctrl[r] >> (2 * j)) & 3u;
#pragma unroll
                    for (uint32_t b = 0; b < 4; b++)
                        if (b <= code)
                            P.outb[p + b] = (uint8_t)(d[r][j] >> (8 * b));
                    p += code + 1;
                }
            }
        }
        named_sync(1, kThreads);
        uint8_t *adst = dst - h;
        const uint32_t nchunks = (h + agg + 15u) >> 4;
        for (uint32_t c = tid; c < nchunks; c += kThreads) {
            if (16u * c >= h && 16u * c + 16u <= h + agg) {
                stg_stream128(adst + 16u * c, *reinterpret_cast<const uint4 *>(P.outb + 16u * c));
            } else {
                for (uint32_t b = 0; b < 16; b++) {
                    const uint32_t idx = 16u * c + b;
                    if (idx >= h && idx < h + agg)
                        adst[idx] = P.outb[idx];
                }
            }
        }
        named_sync(1, kThreads);  // P.outb and s_warp free again
    }
}

__global__ void __launch_bounds__(kEtBlock, 3) encode_tiled_kernel(EncTiledArgs a)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    EtPipe &P = *reinterpret_cast<EtPipe *>(dyn_smem);
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_tt[kChunkTiles];
    __shared__ u64 s_tb[kChunkTiles];
    __shared__ u64 s_etag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kEtStages; s++) {
            mbar_init(&P.full[s], 32);
            mbar_init(&P.empty[s], kWarps);
        }
        fence_mbar_init();
        s_etag = (ld_relaxed(&a.hdr->epoch) + 1) << 2;
    }
    __syncthreads();
    if (warp == kWarps)
        et_produce(a, P, lane);
    else
        et_consume(a, P, s_warp, s_tt, s_tb, s_etag);
    finish_launch(a.hdr, a.result);
}

int launch_encode_tiled(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta,
                        void *ws, DeviceResult *result, cudaStream_t stream, u64 spin_limit)
{
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(encode_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(EtPipe));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, encode_tiled_kernel, kEtBlock,
                                                      sizeof(EtPipe));
        grid = (sms > 0 ? sms : 148) * (occ > 0 ? occ : 1);
    }
    const WsLayout L = ws_layout(n);
    EncTiledArgs a;
    a.in = in;
    a.n = n;
    a.nquads = (n + 3) / 4;
    a.ntiles = (a.nquads + kEtQuads - 1) / kEtQuads;
    a.nchunks = (a.ntiles + kChunkTiles - 1) / kChunkTiles;
    a.out = out;
    a.hdr = reinterpret_cast<WsHeader *>(ws);
    a.st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + L.status);
    a.result = result;
    a.spin_limit = spin_limit;
    a.prev = prev;
    a.delta = delta ? 1u : 0u;
    u64 g = min((u64)grid, a.nchunks);
    prof_begin(delta ? "encode_tiled_kernel<delta>" : "encode_tiled_kernel<plain>", stream);
    encode_tiled_kernel<<<(unsigned)g, kEtBlock, sizeof(EtPipe), stream>>>(a);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // namespace svb
