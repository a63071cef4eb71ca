// Stream VByte encoding of one array, chunked single pass over DRAM.
//
// What is computed is the inverse of the format (Sec. 3-4): each coded value
// v (the integer, or its gap to the previous one with the first gap taken from
// prev, Sec. 1 and Sec. 5) takes L(v) in {1,2,3,4} bytes (Sec. 3), control byte
// q packs L - 1 of integers 4q..4q+3 (first in the low bits, Fig. 3), and the
// data stream after the ceil(N/4) control bytes holds each value's L low-order
// bytes (Sec. 4).
//
// The only serial dependency is where each sub-tile's data bytes go: the sum
// of all earlier lengths.  Persistent CTAs claim chunks of kChunkTiles tiles
// (64 sub-tiles of 512 values) in order, and the producer warp streams each
// chunk's values in twice with bulk copies (cp.async.bulk, mbarrier
// completion):
//   sizing pass   each consumer warp sums the byte lengths of its sub-tile;
//                 at the chunk's end warp 0 scans the 64 sizes and publishes
//                 the chunk's aggregate for a decoupled look-back;
//   writing pass  posted after the next chunk's sizing pass, so the look-back
//                 (warp 0, just before it) usually finds its predecessors
//                 done.  Each warp then forms its sub-tile's control bytes and
//                 data bytes alone - warp scans and shuffles, no barrier with
//                 the other warps - assembling the data word by word in its
//                 own shared slice, phased like the destination, and storing
//                 it with 16-byte writes (ragged ends byte by byte).
// Consumers meet at two bounded barriers per chunk.  The second read of a
// chunk comes from L2 (the chunks in flight on the whole GPU take far less
// than its 129 MB), so DRAM sees each value once.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"

namespace svb {

constexpr int kEtQuads = 1024;                  // quads per tile (4096 values)
constexpr int kEtSubs = kEtQuads / kSubQuads;   // sub-tiles per tile = consumer warps
constexpr int kEtRounds = kSubQuads / 32;       // quads per lane per sub-tile
constexpr int kChunkTiles = 8;                  // tiles per look-back unit
constexpr int kChunkSubs = kChunkTiles * kEtSubs;
constexpr int kEtStages = 3;
constexpr int kEtStageBytes = 16 * kEtQuads + 16;
constexpr int kEtSliceWords = (16 * kSubQuads + 32) / 4;   // one warp's data bytes + phase
constexpr int kEtBlock = kThreads + 32;
constexpr u64 kEtPolls = 1ull << 24;
constexpr uint32_t kEtNone = 0xffffffffu;
constexpr u64 kNoChunk = ~0ull;

static_assert(kEtSubs == kWarps, "one consumer warp per sub-tile");
static_assert(kChunkSubs == 64, "a chunk's sub-tile sizes are scanned two per lane");

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
    uint32_t slice[kWarps][kEtSliceWords];   // each warp's data bytes, phased like the output
    uint64_t full[kEtStages];
    uint64_t empty[kEtStages];
    uint64_t group;                          // consumer-warp barrier
    uint32_t tile[kEtStages];   // tile index, or kEtNone
    uint32_t pass[kEtStages];   // 0 sizing, 1 writing
    uint32_t hv[kEtStages];     // phase (mod 16) of the staged values
};

// Per-chunk bookkeeping, double-buffered by the CTA's own chunk count: chunk
// k is sized, then chunk k+1 is sized while chunk k's look-back result is
// still pending, then chunk k is written.
struct EtChunks {
    uint32_t size[2][kChunkSubs];   // data bytes of each sub-tile
    uint32_t excl[2][kChunkSubs];   // exclusive prefix inside the chunk
    uint32_t agg[2];
    u64 base[2];                    // the chunk's offset in the data stream
};

// The producer warp claims chunks in order and posts, for each, its sizing
// tiles; the writing tiles of a chunk follow the sizing tiles of the next one,
// so a chunk's look-back runs one chunk after its aggregate was published.
__device__ void et_produce(const EncTiledArgs &a, EtPipe &P, int lane)
{
    uint32_t g = 0;
    const uint8_t *lo = reinterpret_cast<const uint8_t *>(a.in);
    const uint8_t *hi = lo + 4 * a.n;
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
            const uint32_t len = 4u * (uint32_t)min((u64)4 * kEtQuads, a.n - i0);
            const uint8_t *gv = reinterpret_cast<const uint8_t *>(a.in + i0);
            const StagePlan pv = stage_plan(gv, len, lo, hi);
            if (pv.edges)
                range_edges(gv, len, P.vals[s], lane);
            if (lane == 0) {
                P.tile[s] = tile;
                P.pass[s] = pass;
                P.hv[s] = (uint32_t)((uintptr_t)gv & 15u);
                mbar_arrive_expect_tx(&P.full[s], pv.bytes);
                if (pv.bytes)
                    bulk_g2s(P.vals[s] + pv.dst_off, pv.src, pv.bytes, &P.full[s]);
            } else {
                mbar_arrive(&P.full[s]);
            }
        }
        g++;
        return true;
    };
    u64 pending = kNoChunk;
    for (;;) {
        u64 c = 0;
        if (lane == 0)
            c = atomicAdd(&a.hdr->tile_counter, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        bool ok = true;
        if (c < a.nchunks) {
            const uint32_t t0 = (uint32_t)(c * kChunkTiles);
            const uint32_t t1 = (uint32_t)min((u64)t0 + kChunkTiles, a.ntiles);
            for (uint32_t t = t0; t < t1 && ok; t++)
                ok = post(t, 0);
        }
        if (ok && pending != kNoChunk) {
            const uint32_t t0 = (uint32_t)(pending * kChunkTiles);
            const uint32_t t1 = (uint32_t)min((u64)t0 + kChunkTiles, a.ntiles);
            for (uint32_t t = t0; t < t1 && ok; t++)
                ok = post(t, 1);
        }
        if (!ok)
            break;
        if (c >= a.nchunks) {
            post(kEtNone, 0);
            break;
        }
        pending = c;
    }
    // Leave only once every posted copy has landed (stage s was filled
    // ceil((g - s) / kEtStages) times).
    if (lane == 0) {
        for (int s = 0; s < kEtStages; s++)
            if (g > (uint32_t)s) {
                uint32_t fills = (g - 1 - s) / kEtStages + 1;
                mbar_wait_bounded(&P.full[s], (fills - 1) & 1u, kEtPolls);
            }
    }
    __syncwarp();
}

// Barrier of the eight consumer warps, bounded.
__device__ __forceinline__ bool et_group_sync(EtPipe &P, uint32_t &phase)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0)
        mbar_arrive(&P.group);
    const bool ok = mbar_wait_bounded(&P.group, phase & 1u, kEtPolls);
    phase++;
    return __all_sync(0xffffffffu, ok);
}

// Integers of quad q (tile-local lq): 4, fewer for the stream's last quad, 0
// past the end.
__device__ __forceinline__ uint32_t et_nints(const EncTiledArgs &a, u64 q0, uint32_t lq,
                                             uint32_t nq, uint32_t last_nints)
{
    return lq >= nq ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
}

// The coded values of one warp's sub-tile: lane l holds quad sq0 + 32r + l in
// round r.  Gaps for differential coding (the first gap from prev, Sec. 5);
// 0 in every field past the end.
__device__ __forceinline__ void et_load(const EncTiledArgs &a, const uint32_t *V, bool aligned,
                                        u64 q0, uint32_t sq0, const uint32_t (&nints)[kEtRounds],
                                        uint32_t (&d)[kEtRounds][4])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < kEtRounds; r++) {
        const uint32_t lq = sq0 + 32 * r + lane;
        if (nints[r] == 4 && aligned) {
            const uint4 v = *reinterpret_cast<const uint4 *>(V + 4 * lq);
            d[r][0] = v.x;
            d[r][1] = v.y;
            d[r][2] = v.z;
            d[r][3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                d[r][j] = (uint32_t)j < nints[r] ? V[4 * lq + j] : 0u;
        }
    }
    if (a.delta) {
        uint32_t carry = 0;  // value before the lane's first one, in lane 0
        if (lane == 0 && nints[0])
            carry = sq0 ? V[4 * sq0 - 1] : (q0 == 0 ? a.prev : __ldg(a.in + 4 * q0 - 1));
#pragma unroll
        for (int r = 0; r < kEtRounds; r++) {
            uint32_t pv = __shfl_up_sync(0xffffffffu, d[r][3], 1);
            if (lane == 0)
                pv = carry;
            carry = __shfl_sync(0xffffffffu, d[r][3], 31);
            const uint32_t x0 = d[r][0], x1 = d[r][1], x2 = d[r][2];
            d[r][3] = nints[r] > 3 ? d[r][3] - x2 : 0u;
            d[r][2] = nints[r] > 2 ? x2 - x1 : 0u;
            d[r][1] = nints[r] > 1 ? x1 - x0 : 0u;
            d[r][0] = nints[r] > 0 ? x0 - pv : 0u;
        }
    }
}

// L(v) - 1 (Sec. 3) with 0 -> 0: the index of the highest set bit over 8.
__device__ __forceinline__ uint32_t extra_bytes(uint32_t v)
{
    return (31u - (uint32_t)__clz(v | 1u)) >> 3;
}

// 128-bit left shift of (s3:s2:s1:s0) by k in [0, 32] bits.
__device__ __forceinline__ void shl128(uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t &s3,
                                       uint32_t k)
{
    s3 = __funnelshift_lc(s2, s3, k);
    s2 = __funnelshift_lc(s1, s2, k);
    s1 = __funnelshift_lc(s0, s1, k);
    s0 = __funnelshift_lc(0u, s0, k);
}

// Warp 0 at the end of a chunk's sizing tiles: prefix of the sub-tile sizes
// and the chunk's aggregate, published for the look-back.
__device__ void et_chunk_scan(const EncTiledArgs &a, EtChunks &C, int b, u64 chunk, u64 etag)
{
    const int lane = threadIdx.x & 31;
    const u64 tiles = min((u64)kChunkTiles, a.ntiles - chunk * kChunkTiles);
    const uint32_t v0 = (u64)(2 * lane) / kEtSubs < tiles ? C.size[b][2 * lane] : 0u;
    const uint32_t v1 = (u64)(2 * lane + 1) / kEtSubs < tiles ? C.size[b][2 * lane + 1] : 0u;
    const uint32_t t = v0 + v1;
    const uint32_t inc = warp_incl_scan(t);
    C.excl[b][2 * lane] = inc - t;
    C.excl[b][2 * lane + 1] = inc - t + v0;
    const uint32_t agg = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 0) {
        C.agg[b] = agg;
        TileStatus *me = &a.st[chunk];
        if (chunk == 0)
            publish(&me->off_tag, &me->off_pre, agg, kFlagPrefix, etag);
        else
            publish(&me->off_tag, &me->off_agg, agg, kFlagAgg, etag);
    }
}

// Warp 0 before a chunk's writing tiles: the chunk's offset in the data stream.
__device__ void et_chunk_base(const EncTiledArgs &a, EtChunks &C, int b, u64 chunk, u64 etag)
{
    const int lane = threadIdx.x & 31;
    u64 base = 0;
    bool ok = true;
    const u64 agg = C.agg[b];
    if (chunk > 0) {
        base = lookback<false>(a.st, chunk, etag, a.spin_limit, a.hdr, ok);
        if (ok && lane == 0)
            publish(&a.st[chunk].off_tag, &a.st[chunk].off_pre, base + agg, kFlagPrefix, etag);
    }
    if (lane == 0) {
        if (!ok)
            raise_error(a.hdr, kErrTimeout);
        C.base[b] = base;
        if (chunk + 1 == a.nchunks)
            st_relaxed(&a.hdr->total, a.nquads + base + agg);
    }
}

// One warp writes its sub-tile: control bytes straight to global memory; the
// data bytes are laid end to end in the warp's shared slice at the phase of
// their destination (word by word: each lane shifts its quad's 4..16 bytes to
// their byte position and writes the words it completes, taking the partial
// first word from the previous lane), then copied out with 16-byte stores.
__device__ __forceinline__ void et_write(const EncTiledArgs &a, uint32_t *slice, uint8_t *dst,
                                         u64 q0, uint32_t sq0, uint32_t nvq,
                                         const uint32_t (&nints)[kEtRounds],
                                         const uint32_t (&ctrl)[kEtRounds],
                                         const uint32_t (&cb)[kEtRounds],
                                         const uint32_t (&d)[kEtRounds][4])
{
    const int lane = threadIdx.x & 31;
    const uint32_t h = (uint32_t)((uintptr_t)dst & 15u);
    uint32_t run = 0, carry = 0, fidx = kEtNone, fword = 0;
#pragma unroll
    for (int r = 0; r < kEtRounds; r++) {
        if (32u * r >= nvq)
            break;
        const uint32_t lq = sq0 + 32 * r + lane;
        const uint32_t C = cb[r];
        uint32_t L[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            L[j] = (uint32_t)j < nints[r] ? ((ctrl[r] >> (2 * j)) & 3u) + 1 : 0u;
        if (nints[r])
            a.out[q0 + lq] = (uint8_t)ctrl[r];
        const uint32_t inc = warp_incl_scan(C);
        const uint32_t pos = h + run + inc - C;
        run += __shfl_sync(0xffffffffu, inc, 31);
        // The quad's bytes end to end (Fig. 3's data layout), then moved to
        // their phase inside a word.
        uint32_t s0 = d[r][3], s1 = 0, s2 = 0, s3 = 0;
        shl128(s0, s1, s2, s3, 8 * L[2]);
        s0 |= d[r][2];
        shl128(s0, s1, s2, s3, 8 * L[1]);
        s0 |= d[r][1];
        shl128(s0, s1, s2, s3, 8 * L[0]);
        s0 |= d[r][0];
        const uint32_t sh = 8 * (pos & 3);
        const uint32_t t4 = __funnelshift_l(s3, 0u, sh);
        const uint32_t t3 = __funnelshift_l(s2, s3, sh);
        const uint32_t t2 = __funnelshift_l(s1, s2, sh);
        const uint32_t t1 = __funnelshift_l(s0, s1, sh);
        const uint32_t t0 = s0 << sh;
        const uint32_t nfull = ((pos & 3) + C) >> 2;   // words this lane completes
        const uint32_t tail = nfull == 0 ? t0 : nfull == 1 ? t1 : nfull == 2 ? t2
                                                : nfull == 3 ? t3 : t4;
        uint32_t pt = __shfl_up_sync(0xffffffffu, tail, 1);
        if (lane == 0)
            pt = carry;
        carry = __shfl_sync(0xffffffffu, tail, 31);
        const uint32_t w0 = t0 | pt;
        uint32_t *wp = slice + (pos >> 2);
        if (nfull > 0)
            wp[0] = w0;
        if (nfull > 1)
            wp[1] = t1;
        if (nfull > 2)
            wp[2] = t2;
        if (nfull > 3)
            wp[3] = t3;
        if (lq + 1 == sq0 + nvq && ((pos + C) & 3u)) {   // the sub-tile's last, partial word
            fidx = (pos + C) >> 2;
            fword = nfull ? tail : w0;
        }
    }
    if (fidx != kEtNone)
        slice[fidx] = fword;
    __syncwarp();
    const uint8_t *sb = reinterpret_cast<const uint8_t *>(slice);
    uint8_t *adst = dst - h;
    const uint32_t end = h + run;
    const uint32_t c0 = (h + 15) >> 4, c1 = end >> 4;   // whole 16-byte chunks [c0, c1)
    for (uint32_t c = c0 + lane; c < c1; c += 32)
        stg_stream128(adst + 16 * c, *reinterpret_cast<const uint4 *>(sb + 16 * c));
    if (lane < 16) {
        const uint32_t i = h + lane;
        if (i < min(16 * c0, end))
            adst[i] = sb[i];
    } else {
        const uint32_t i = 16 * c1 + (lane - 16);
        if (c1 >= c0 && i < end)
            adst[i] = sb[i];
    }
    __syncwarp();
}

__device__ void et_consume(const EncTiledArgs &a, EtPipe &P, EtChunks &C, u64 etag)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    const uint32_t sq0 = warp * kSubQuads;
    uint32_t sized = 0, written = 0, phase = 0;   // chunks this CTA has sized / written
    for (uint32_t g = 0;; g++) {
        const int s = g % kEtStages;
        if (!mbar_wait_bounded(&P.full[s], (g / kEtStages) & 1u, kEtPolls)) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            break;
        }
        const uint32_t tile = P.tile[s];
        if (tile == kEtNone)
            break;
        const uint32_t pass = P.pass[s];
        const u64 q0 = (u64)tile * kEtQuads;
        const uint32_t nq = (uint32_t)min((u64)kEtQuads, a.nquads - q0);
        const uint32_t nvq = nq > sq0 ? min(nq - sq0, (uint32_t)kSubQuads) : 0u;
        const uint32_t *V = reinterpret_cast<const uint32_t *>(P.vals[s] + P.hv[s]);
        uint32_t nints[kEtRounds], d[kEtRounds][4], ctrl[kEtRounds], cb[kEtRounds];
#pragma unroll
        for (int r = 0; r < kEtRounds; r++)
            nints[r] = et_nints(a, q0, sq0 + 32 * r + lane, nq, last_nints);
        et_load(a, V, P.hv[s] == 0, q0, sq0, nints, d);
        // Control byte and data bytes of each quad (fields past the end are 0
        // and add nothing); they use every staged value this warp loaded.
#pragma unroll
        for (int r = 0; r < kEtRounds; r++) {
            uint32_t c = 0, C = nints[r];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t e = extra_bytes(d[r][j]);
                c |= e << (2 * j);
                C += e;
            }
            ctrl[r] = c;
            cb[r] = C;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.empty[s]);
        const uint32_t ti = tile % kChunkTiles;
        const u64 chunk = tile / kChunkTiles;

        if (pass == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int r = 0; r < kEtRounds; r++)
                t += cb[r];
#pragma unroll
            for (int k = 16; k >= 1; k >>= 1)
                t += __shfl_xor_sync(0xffffffffu, t, k);
            const int b = sized & 1;
            if (lane == 0)
                C.size[b][ti * kEtSubs + warp] = t;
            if (ti + 1 == kChunkTiles || tile + 1 == a.ntiles) {
                sized++;
                if (!et_group_sync(P, phase)) {
                    if (lane == 0)
                        raise_error(a.hdr, kErrTimeout);
                    break;
                }
                if (warp == 0)
                    et_chunk_scan(a, C, b, chunk, etag);
            }
            continue;
        }

        if (ti == 0)
            written++;
        const int b = (written - 1) & 1;   // the same buffer for all tiles of the chunk
        if (ti == 0) {
            if (warp == 0)
                et_chunk_base(a, C, b, chunk, etag);
            if (!et_group_sync(P, phase)) {
                if (lane == 0)
                    raise_error(a.hdr, kErrTimeout);
                break;
            }
        }
        uint8_t *dst = a.out + a.nquads + C.base[b] + C.excl[b][ti * kEtSubs + warp];
        et_write(a, P.slice[warp], dst, q0, sq0, nvq, nints, ctrl, cb, d);
    }
}

__global__ void __launch_bounds__(kEtBlock, 3) encode_tiled_kernel(EncTiledArgs a)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    EtPipe &P = *reinterpret_cast<EtPipe *>(dyn_smem);
    __shared__ EtChunks s_chunks;
    __shared__ u64 s_etag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kEtStages; s++) {
            mbar_init(&P.full[s], 32);
            mbar_init(&P.empty[s], kWarps);
        }
        mbar_init(&P.group, kWarps);
        fence_mbar_init();
        s_etag = (ld_relaxed(&a.hdr->epoch) + 1) << 2;
    }
    __syncthreads();
    if (warp == kWarps)
        et_produce(a, P, lane);
    else
        et_consume(a, P, s_chunks, s_etag);
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
