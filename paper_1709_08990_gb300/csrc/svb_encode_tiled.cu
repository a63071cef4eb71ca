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
// (32 sub-tiles of 512 values) in order, and the producer warp streams each
// chunk's values in twice with bulk copies (cp.async.bulk, mbarrier
// completion):
//   sizing pass   each consumer warp sums the byte lengths of its sub-tile;
//                 the chunk warp then scans the chunk's sub-tile sizes,
//                 publishes its aggregate and finds its offset by decoupled
//                 look-back, while the consumers size the next chunk;
//   writing pass  each warp forms its sub-tile's control bytes and data bytes
//                 alone - warp scans and shuffles, no barrier with the other
//                 warps - assembling the data word by word in its own shared
//                 slice, phased like the destination, and storing it with
//                 16-byte writes (ragged ends byte by byte).
// Consumers and the chunk warp hand chunks over through two mbarriers; the
// chunk warp writes no output, so its release stores and fences do not wait
// on data stores in flight.  The sizing read asks L2 to keep the values and
// the writing read, one chunk later, takes them from there, so DRAM sees each
// value once.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"
#include "svb_subenc.cuh"

namespace svb {

constexpr int kEtQuads = 1024;                  // quads per tile (4096 values)
constexpr int kEtSubs = kEtQuads / kSubQuads;   // sub-tiles per tile = consumer warps
constexpr int kChunkTiles = 4;                  // tiles per look-back unit
constexpr int kChunkSubs = kChunkTiles * kEtSubs;
constexpr int kEtStages = 3;
constexpr int kEtStageBytes = 16 * kEtQuads + 16;
constexpr int kEtBlock = kThreads + 64;          // 8 consumer warps, producer, chunk warp
constexpr u64 kEtPolls = 1ull << 24;            // bound on a busy-polled wait
constexpr u64 kEtSuspends = 1ull << 18;         // bound on a suspending wait ...
constexpr uint32_t kEtSuspendNs = 10000;        // ... of up to 10 us per poll (2.6 s in all)
constexpr uint32_t kEtNone = 0xffffffffu;
constexpr u64 kNoChunk = ~0ull;

static_assert(kEtSubs == kWarps, "one consumer warp per sub-tile");
static_assert(kChunkSubs <= 32, "a chunk's sub-tile sizes are scanned one per lane");

struct EncTiledArgs {
    const uint32_t *in;
    u64 n, nquads, ntiles, nchunks;
    uint8_t *out;             // control bytes (and, unless data is set, the data after them)
    uint8_t *data;            // where data byte 0 goes, minus *data_back; null: out + nquads
    const u64 *data_back;     // device value subtracted from data (null: 0)
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    uint32_t prev;
    uint32_t delta;
};

struct EtPipe {
    uint8_t vals[kEtStages][kEtStageBytes];
    uint32_t slice[kWarps][kEncSliceWords];   // each warp's data bytes, phased like the output
    uint64_t full[kEtStages];
    uint64_t empty[kEtStages];
    uint64_t sizes_ready[2];    // consumers -> chunk warp: a chunk's sub-tile sizes are in
    uint64_t base_ready[2];     // chunk warp -> consumers: the chunk's offsets are known
    uint32_t tile[kEtStages];   // tile index, or kEtNone
    uint32_t pass[kEtStages];   // 0 sizing, 1 writing
    uint32_t hv[kEtStages];     // phase (mod 16) of the staged values
};

// Per-chunk bookkeeping, double-buffered by the CTA's own chunk count (the
// k-th chunk uses buffer k & 1): chunk k is sized, then chunk k+1 is sized
// while the chunk warp finds chunk k's offset, then chunk k is written.
struct EtChunks {
    uint32_t size[2][kChunkSubs];   // data bytes of each sub-tile
    uint32_t excl[2][kChunkSubs];   // exclusive prefix inside the chunk
    uint32_t agg[2];
    u64 base[2];                    // the chunk's offset in the data stream
    u64 chunk[2];                   // the chunk's index, kNoChunk once the work is out
};

// The producer warp claims chunks in order and posts, for each, its sizing
// tiles; the writing tiles of a chunk follow the sizing tiles of the next one,
// so a chunk's look-back runs one chunk after its aggregate was published.
__device__ void et_produce(const EncTiledArgs &a, EtPipe &P, int lane)
{
    uint32_t g = 0;
    const uint64_t keep = l2_policy_evict_last(), keep_not = l2_policy_evict_first();
    const uint8_t *lo = reinterpret_cast<const uint8_t *>(a.in);
    const uint8_t *hi = lo + 4 * a.n;
    auto post = [&](uint32_t tile, uint32_t pass) -> bool {
        const int s = g % kEtStages;
        if (g >= (uint32_t)kEtStages) {
            bool ok = mbar_wait_suspend(&P.empty[s], ((g / kEtStages) - 1) & 1u, kEtSuspends,
                                        kEtSuspendNs);
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
                // The sizing read asks L2 to keep the lines for the writing
                // read, which marks them first to go.
                if (pv.bytes)
                    bulk_g2s_hint(P.vals[s] + pv.dst_off, pv.src, pv.bytes, &P.full[s],
                                  pass ? keep_not : keep);
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

// Chunk warp, once a chunk's sizing tiles are done: prefix of the sub-tile
// sizes and the chunk's aggregate, published for the look-back.
__device__ void et_chunk_scan(const EncTiledArgs &a, EtChunks &C, int b, u64 chunk, u64 etag)
{
    const int lane = threadIdx.x & 31;
    const u64 tiles = min((u64)kChunkTiles, a.ntiles - chunk * kChunkTiles);
    const uint32_t t = lane < kChunkSubs && (u64)lane / kEtSubs < tiles ? C.size[b][lane] : 0u;
    const uint32_t inc = warp_incl_scan(t);
    if (lane < kChunkSubs)
        C.excl[b][lane] = inc - t;
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

// Chunk warp, right after: the chunk's offset in the data stream, by
// decoupled look-back over the chunks claimed before it.
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

// The chunk warp: for each chunk of this CTA, in order, once the consumers
// have sized it: scan, publish, look back, hand the offsets to the
// consumers.  It writes no output, so its release stores and fences wait on
// nothing but its own status records.
__device__ void et_chunk_warp(const EncTiledArgs &a, EtPipe &P, EtChunks &C, u64 etag)
{
    const int lane = threadIdx.x & 31;
    for (uint32_t k = 0;; k++) {
        const int b = k & 1;
        if (!mbar_wait_suspend(&P.sizes_ready[b], (k >> 1) & 1u, kEtSuspends, kEtSuspendNs)) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            break;
        }
        const u64 chunk = C.chunk[b];
        if (chunk == kNoChunk)
            break;
        et_chunk_scan(a, C, b, chunk, etag);
        __syncwarp();
        et_chunk_base(a, C, b, chunk, etag);
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.base_ready[b]);
    }
}

__device__ void et_consume(const EncTiledArgs &a, EtPipe &P, EtChunks &C, u64 etag)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *const data_base =
        a.data ? a.data - (a.data_back ? *a.data_back : 0ull) : a.out + a.nquads;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    const uint32_t sq0 = warp * kSubQuads;
    uint32_t sized = 0, written = 0;   // chunks this CTA has sized / started writing
    for (uint32_t g = 0;; g++) {
        const int s = g % kEtStages;
        if (!mbar_wait_suspend(&P.full[s], (g / kEtStages) & 1u, kEtSuspends, kEtSuspendNs)) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            break;
        }
        const uint32_t tile = P.tile[s];
        if (tile == kEtNone) {
            // Tell the chunk warp that no chunk follows.
            const int b = sized & 1;
            if (warp == 0 && lane == 0)
                C.chunk[b] = kNoChunk;
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&P.sizes_ready[b]);
            break;
        }
        const uint32_t pass = P.pass[s];
        const u64 q0 = (u64)tile * kEtQuads;
        const uint32_t nq = (uint32_t)min((u64)kEtQuads, a.nquads - q0);
        const uint32_t nvq = nq > sq0 ? min(nq - sq0, (uint32_t)kSubQuads) : 0u;
        const uint32_t *V = reinterpret_cast<const uint32_t *>(P.vals[s] + P.hv[s]);
        // Whole sub-tile of 512 integers, staged 16-byte aligned: no per-quad
        // end checks.
        const bool fast = P.hv[s] == 0 && 4 * (q0 + sq0 + kSubQuads) <= a.n;
        uint32_t nints[kEncRounds], d[kEncRounds][4], ctrl[kEncRounds], cb[kEncRounds];
        const uint32_t tail = q0 + nq == a.nquads ? last_nints : 4u;
        auto before = [&]() { return q0 == 0 ? a.prev : __ldg(a.in + 4 * q0 - 1); };
        const bool sizing = P.pass[s] == 0;
        // A whole sub-tile of one-byte values (the common case of sorted
        // lists with small gaps) needs no lengths: 512 data bytes, control 0.
        bool small = false;
        if (fast) {
            subenc_values<true>(V, sq0, nq, tail, a.delta, before, nints, d);
            small = subenc_all_small(d);
            if (!small && sizing)
                subenc_lengths<true>(nints, d, ctrl, cb);
            else if (!small)
                subenc_lengths<false>(nints, d, ctrl, cb);
        } else {
            subenc_load<false>(V, sq0, nq, tail, a.delta, before, nints, d, ctrl, cb);
        }
        // The control bytes use every staged value this warp loaded, so its
        // loads are complete; the fence orders them before the refill.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.empty[s]);
        const uint32_t ti = tile % kChunkTiles;
        const u64 chunk = tile / kChunkTiles;

        if (pass == 0) {
            const uint32_t t = small ? 4u * kSubQuads : subenc_bytes(cb);
            const int b = sized & 1;
            if (lane == 0) {
                C.size[b][ti * kEtSubs + warp] = t;
                if (warp == 0 && ti == 0)
                    C.chunk[b] = chunk;
            }
            if (ti + 1 == kChunkTiles || tile + 1 == a.ntiles) {
                sized++;
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&P.sizes_ready[b]);
            }
            continue;
        }

        if (ti == 0)
            written++;
        const uint32_t k = written - 1;   // this CTA's chunk count: buffer k & 1
        const int b = k & 1;
        if (ti == 0 &&
            !mbar_wait_suspend(&P.base_ready[b], (k >> 1) & 1u, kEtSuspends, kEtSuspendNs)) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            break;
        }
        uint8_t *dst = data_base + C.base[b] + C.excl[b][ti * kEtSubs + warp];
        if (small)
            subenc_write_small(P.slice[warp], a.out + q0 + sq0, dst, d);
        else if (fast)
            subenc_write<true>(P.slice[warp], a.out + q0 + sq0, dst, nvq, nints, ctrl, cb, d);
        else
            subenc_write<false>(P.slice[warp], a.out + q0 + sq0, dst, nvq, nints, ctrl, cb, d);
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
        for (int b = 0; b < 2; b++) {
            mbar_init(&P.sizes_ready[b], kWarps);
            mbar_init(&P.base_ready[b], 1);
        }
        fence_mbar_init();
        s_etag = epoch_tag(a.hdr);
    }
    __syncthreads();
    if (warp == kWarps)
        et_produce(a, P, lane);
    else if (warp == kWarps + 1)
        et_chunk_warp(a, P, s_chunks, s_etag);
    else
        et_consume(a, P, s_chunks, s_etag);
    finish_launch(a.hdr, a.result);
}

int launch_encode_tiled(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta,
                        void *ws, DeviceResult *result, cudaStream_t stream, u64 spin_limit,
                        uint8_t *data, const u64 *data_back)
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
    a.data = data;
    a.data_back = data_back;
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
