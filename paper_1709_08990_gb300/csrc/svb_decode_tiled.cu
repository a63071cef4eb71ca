// Stream VByte decoding, reduce-then-decode form: two kernels, no waits for
// plain streams.
//
// The decoder's only serial dependency is where each quad's data bytes start:
// the data pointer advances by C in [4,16] per control byte (Sec. 4, Fig. 4),
// the same chain that in varint-GB also hides the next control byte (Sec. 4).
// With the control stream apart, those positions depend on the control bytes
// alone, so:
//   offsets_kernel   reads only the control stream (2 bits per integer) and
//                    writes, for every tile of kTileQuads quads, its byte
//                    offset in the data stream.  Persistent CTAs each sum a
//                    contiguous range of tiles, chain the range totals with
//                    one decoupled look-back, then add their base.  It also
//                    writes the stream's size and checks it against in_len.
//   decode_tiled     persistent CTAs with one producer warp and eight
//                    consumer warps.  The producer claims tiles, reads their
//                    offsets and has the TMA engine copy each tile's control
//                    and data bytes into one of kStages shared-memory stages
//                    (cp.async.bulk completing on the stage's "full"
//                    mbarrier); consumers decode a full stage and release it
//                    on its "empty" mbarrier.  Plain streams never wait on
//                    another CTA; loads for later tiles are always in flight.
// Differential streams need each tile's carry-in, prev plus the sum of all
// earlier gaps (Sec. 2's prefix sum continued across tiles).  A sums pass runs
// the same pipeline without stores: persistent CTAs take contiguous tile
// ranges, sum each tile's gaps, and chain the range totals with one look-back
// per CTA into per-tile carries.  The decode pass then adds a known carry and
// never waits on another CTA.  For streams that fit in L2 (129 MB) the second
// read of the stream is served by L2.
//
// Bytes outside the stream are never read: each tile's range is copied as its
// 16-byte-aligned interior by the bulk engine plus a ragged head and tail of
// at most 15 bytes each by plain loads.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"

namespace svb {

constexpr int kTileQuads = 1024;                    // quads per tile (4096 integers)
constexpr int kTileRounds = kTileQuads / kThreads;  // quads per lane per tile
constexpr int kTileData = 16 * kTileQuads;          // data bytes per tile, at most
constexpr int kStageData = kTileData + 64;          // + 16-byte phase + 2-word read slack
constexpr int kStageCtrl = kTileQuads + 32;
constexpr int kStages = 4;
constexpr int kDecBlock = kThreads + 32;            // 8 consumer warps + 1 producer warp
constexpr u64 kBarrierPolls = 1ull << 24;           // bound on one mbarrier wait
constexpr u64 kNoTile = ~0ull;

// ---------------------------------------------------------------------------
// Pass 1: tile offsets from the control stream.

constexpr int kOffGroup = 16;                       // tiles summed per CTA iteration

struct OffsetsArgs {
    const uint8_t *in;
    u64 in_len;
    u64 n, nquads, ntiles;
    u64 groups;      // ceil(ntiles / kOffGroup)
    u64 per_cta;     // groups per CTA
    u64 *offs;       // ntiles + 1 entries
    WsHeader *hdr;
    TileStatus *st;
    u64 spin_limit;
    uint32_t in_aligned;
};

// Data bytes covered by the control bytes of quads [q, q + 16) taken from
// the 16-byte chunk v; quads at or beyond nquads count nothing, and the pad
// fields of the last quad count nothing.
__device__ __forceinline__ uint32_t chunk_bytes(uint4 v, u64 q, u64 nquads, uint32_t last_nints)
{
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
    if (q + 16 < nquads) {  // no last quad inside: the common case
        uint32_t t = 64;
#pragma unroll
        for (int i = 0; i < 4; i++)
            t += __popc(w[i] & 0x55555555u) + 2u * __popc(w[i] & 0xAAAAAAAAu);
        return t;
    }
    uint32_t t = 0;
#pragma unroll
    for (int b = 0; b < 16; b++) {
        u64 qq = q + b;
        uint32_t c = (w[b >> 2] >> (8 * (b & 3))) & 0xffu;
        uint32_t k = qq < nquads - 1 ? 4u : (qq == nquads - 1 ? last_nints : 0u);
        if (k < 4)
            c &= (1u << (2 * k)) - 1u;
        t += k ? k + __popc(c & 0x55u) + 2u * __popc(c & 0xAAu) : 0u;
    }
    return t;
}

// Sum of the data bytes of 64 quads starting at q (one thread's share).
__device__ __forceinline__ uint32_t sum64(const OffsetsArgs &a, u64 q, uint32_t last_nints)
{
    uint32_t sum = 0;
    if (q >= a.nquads)
        return 0;
    if (a.in_aligned && q + 64 <= a.nquads) {
        const uint4 *p = reinterpret_cast<const uint4 *>(a.in + q);
        uint4 v[4];
#pragma unroll
        for (int i = 0; i < 4; i++)
            v[i] = __ldg(p + i);
#pragma unroll
        for (int i = 0; i < 4; i++)
            sum += chunk_bytes(v[i], q + 16 * i, a.nquads, last_nints);
    } else {
        for (int i = 0; i < 4; i++) {
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int b = 0; b < 16; b++) {
                u64 qq = q + 16 * i + b;
                if (qq < a.nquads)
                    w[b >> 2] |= (uint32_t)__ldg(a.in + qq) << (8 * (b & 3));
            }
            sum += chunk_bytes(make_uint4(w[0], w[1], w[2], w[3]), q + 16 * i, a.nquads,
                               last_nints);
        }
    }
    return sum;
}

__global__ void __launch_bounds__(kThreads) offsets_kernel(OffsetsArgs a)
{
    __shared__ uint32_t s_tsum[2][kOffGroup];
    __shared__ u64 s_cta, s_etag, s_base;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_cta = atomicAdd(&a.hdr->a_counter, 1ull);
        s_etag = (ld_relaxed(&a.hdr->epoch) + 1) << 2;
    }
    __syncthreads();
    const u64 cta = s_cta, etag = s_etag;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    const u64 g0 = cta * a.per_cta;
    const u64 g1 = min(g0 + a.per_cta, a.groups);

    // Local offsets: each group of 16 tiles is 16 KB of control bytes, 64 per
    // thread and 16 threads per tile; warp 0 keeps the running total.
    u64 running = 0;  // meaningful in warp 0
    int buf = 0;
    for (u64 g = g0; g < g1; g++, buf ^= 1) {
        const u64 q = g * (u64)(kOffGroup * kTileQuads) + 64u * tid;
        uint32_t sum = sum64(a, q, last_nints);
#pragma unroll
        for (int d = 8; d >= 1; d >>= 1)
            sum += __shfl_xor_sync(0xffffffffu, sum, d);
        if ((tid & 15) == 0)
            s_tsum[buf][tid >> 4] = sum;
        __syncthreads();
        if (warp == 0) {
            uint32_t ts = lane < kOffGroup ? s_tsum[buf][lane] : 0u;
            uint32_t inc = warp_incl_scan(ts);
            u64 tile = g * kOffGroup + lane;
            if (lane < kOffGroup && tile < a.ntiles)
                a.offs[tile] = running + (inc - ts);
            running += __shfl_sync(0xffffffffu, inc, 31);
        }
        // s_tsum is double-buffered: the next iteration writes the other half,
        // and the barrier of that iteration orders this read before reuse.
    }

    // Chain the CTA totals, then add this CTA's base to its tiles.
    if (warp == 0) {
        TileStatus *me = &a.st[cta];
        u64 base = 0;
        bool ok = true;
        if (cta == 0) {
            if (lane == 0)
                publish(&me->off_tag, &me->off_pre, running, kFlagPrefix, etag);
        } else {
            if (lane == 0)
                publish(&me->off_tag, &me->off_agg, running, kFlagAgg, etag);
            base = lookback<false>(a.st, cta, etag, a.spin_limit, a.hdr, ok);
            if (ok && lane == 0)
                publish(&me->off_tag, &me->off_pre, base + running, kFlagPrefix, etag);
        }
        if (lane == 0) {
            if (!ok)
                raise_error(a.hdr, kErrTimeout);
            if (ok && g1 == a.groups && g0 < g1) {  // the CTA holding the last tile
                u64 stream = a.nquads + base + running;
                a.offs[a.ntiles] = base + running;
                st_relaxed(&a.hdr->total, stream);
                if (stream > a.in_len)
                    raise_error(a.hdr, kErrTruncated);
            }
            s_base = base;
        }
    }
    __syncthreads();
    const u64 base = s_base;
    if (base) {
        const u64 t0 = g0 * kOffGroup, t1 = min(g1 * kOffGroup, a.ntiles);
        for (u64 t = t0 + tid; t < t1; t += kThreads)
            a.offs[t] += base;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        u64 done = atomicAdd(&a.hdr->a_done, 1ull);
        if (done == (u64)gridDim.x - 1) {
            st_relaxed(&a.hdr->a_counter, 0);
            st_relaxed(&a.hdr->a_done, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// Pass 2: persistent decode, producer warp + consumer warps.

enum TiledMode : int {
    kPlain = 0,  // decode and store
    kDelta = 1,  // decode, running sums plus the tile's precomputed carry, store
    kSums = 2,   // decode, sum the tile's gaps; write per-tile carries (no stores)
};

struct TiledArgs {
    const uint8_t *in;
    u64 n, nquads, ntiles;
    uint32_t *out;
    const u64 *offs;
    uint32_t *carries;  // per tile: written by kSums, read by kDelta
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    u64 per_cta;        // kSums: tiles per CTA (contiguous ranges)
    uint32_t prev;
    uint32_t out_aligned;
};

struct Pipe {
    uint8_t data[kStages][kStageData];
    uint8_t ctrl[kStages][kStageCtrl];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    u64 tile[kStages];
    uint32_t hd[kStages], hc[kStages];  // address phase (mod 16) of the data / control range
    uint32_t carry[kStages];            // kDelta: the tile's carry-in
};

// The k-th tile this CTA handles: round-robin for decoding, a contiguous
// range for the sums pass (whose look-back chains ranges in order).
template <int kMode>
__device__ __forceinline__ u64 tile_of(const TiledArgs &a, u64 first, uint32_t k)
{
    if (kMode == kSums) {
        const u64 end = min(first + a.per_cta, a.ntiles);
        return first + k < end ? first + k : a.ntiles;
    }
    return first + (u64)k * gridDim.x;
}

// Producer warp: fill stages with tiles until none is left, then post one
// stage marked kNoTile.  Returns normally or after a bounded wait gave up.
template <int kMode>
__device__ void produce(const TiledArgs &a, Pipe &P, u64 first, int lane)
{
    uint32_t issued = 0;  // stage fills posted (iteration k fills stage k % kStages)
    u64 next = tile_of<kMode>(a, first, 0);
    u64 nd0 = 0, nd1 = 0;
    if (next < a.ntiles) {
        nd0 = a.offs[next];
        nd1 = a.offs[next + 1];
    }
    for (uint32_t k = 0;; k++) {
        const int s = k % kStages;
        if (k >= (uint32_t)kStages) {
            bool ok = mbar_wait_bounded(&P.empty[s], ((k / kStages) - 1) & 1u, kBarrierPolls);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0)
                    raise_error(a.hdr, kErrTimeout);
                break;
            }
        }
        const u64 t = next;
        const u64 d0 = nd0, d1 = nd1;
        if (t >= a.ntiles) {
            if (lane == 0) {
                P.tile[s] = kNoTile;
                mbar_arrive_expect_tx(&P.full[s], 0);
            } else {
                mbar_arrive(&P.full[s]);
            }
            issued = k + 1;
            break;
        }
        // Read the next tile's offsets now so that the load overlaps this one.
        next = tile_of<kMode>(a, first, k + 1);
        if (next < a.ntiles) {
            nd0 = a.offs[next];
            nd1 = a.offs[next + 1];
        }
        const u64 q0 = t * kTileQuads;
        const uint32_t clen = (uint32_t)min((u64)kTileQuads, a.nquads - q0);
        const uint8_t *gc = a.in + q0;
        const uint8_t *gd = a.in + a.nquads + d0;
        const uint32_t dlen = (uint32_t)(d1 - d0);
        range_edges(gc, clen, P.ctrl[s], lane);
        range_edges(gd, dlen, P.data[s], lane);
        if (lane == 0) {
            const uint8_t *ac, *ad;
            uint32_t oc, od;
            uint32_t bc = range_interior(gc, clen, ac, oc);
            uint32_t bd = range_interior(gd, dlen, ad, od);
            P.tile[s] = t;
            P.hc[s] = (uint32_t)((uintptr_t)gc & 15u);
            P.hd[s] = (uint32_t)((uintptr_t)gd & 15u);
            if (kMode == kDelta)
                P.carry[s] = a.carries[t];
            mbar_arrive_expect_tx(&P.full[s], bc + bd);
            if (bc)
                bulk_g2s(P.ctrl[s] + oc, ac, bc, &P.full[s]);
            if (bd)
                bulk_g2s(P.data[s] + od, ad, bd, &P.full[s]);
        } else {
            mbar_arrive(&P.full[s]);
        }
        issued = k + 1;
    }
    // Let every copy this warp started land before the CTA can exit: stage s
    // was filled (issued - 1 - s) / kStages + 1 times; wait for the last fill.
    if (lane == 0) {
        for (int s = 0; s < kStages; s++)
            if (issued > (uint32_t)s) {
                uint32_t fills = (issued - 1 - s) / kStages + 1;
                mbar_wait_bounded(&P.full[s], (fills - 1) & 1u, kBarrierPolls);
            }
    }
    __syncwarp();
}

// Consumer warps (8, synchronised among themselves by named barrier 1).
template <int kMode>
__device__ void consume(const TiledArgs &a, Pipe &P, uint16_t *s_qoff, uint32_t *s_warp,
                        u64 first, u64 etag)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    uint32_t running = 0;  // kSums: gap sum of this CTA's tiles so far (thread 0)
    for (uint32_t k = 0;; k++) {
        const int s = k % kStages;
        bool ok = mbar_wait_bounded(&P.full[s], (k / kStages) & 1u, kBarrierPolls);
        if (!ok) {  // cannot happen unless a copy is lost; give up quietly
            raise_error(a.hdr, kErrTimeout);
            break;
        }
        const u64 tile = P.tile[s];
        if (tile == kNoTile)
            break;

        // ---- control bytes -> staged position of every quad -----------------
        const u64 q0 = tile * kTileQuads;
        const uint32_t nq = (uint32_t)min((u64)kTileQuads, a.nquads - q0);
        // Every tile but possibly the last holds kTileQuads quads of four.
        const bool full = nq == kTileQuads && (tile + 1 < a.ntiles || last_nints == 4);
        const uint8_t *C = P.ctrl[s] + P.hc[s];
        const uint8_t *D = P.data[s];
        const uint32_t h = P.hd[s];
        const uint32_t carry_in = kMode == kDelta ? P.carry[s] : 0u;
        uint32_t w = 0;
        if (P.hc[s] == 0 && 4u * tid + 4u <= nq) {
            w = reinterpret_cast<const uint32_t *>(C)[tid];
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (4u * tid + j < nq)
                    w |= (uint32_t)C[4 * tid + j] << (8 * j);
        }
        uint32_t o1, o2, o3, tsum;
        if (full) {
            // Byte j of cs = sum of the four codes of quad j; the multiply turns
            // the four bytes into their running sums (at most 48, no carries).
            uint32_t cs = (w & 0x33333333u) + ((w >> 2) & 0x33333333u);
            cs = (cs & 0x0F0F0F0Fu) + ((cs >> 4) & 0x0F0F0F0Fu);
            const uint32_t run = cs * 0x01010101u;
            o1 = 4u + (run & 0xffu);
            o2 = 8u + ((run >> 8) & 0xffu);
            o3 = 12u + ((run >> 16) & 0xffu);
            tsum = 16u + (run >> 24);
        } else {
            uint32_t cnt[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                uint32_t lq = 4u * tid + j;
                uint32_t c = (w >> (8 * j)) & 0xffu;
                uint32_t nints = 4;
                if (q0 + lq == a.nquads - 1 && last_nints < 4) {
                    nints = last_nints;
                    c &= (1u << (2 * nints)) - 1u;
                }
                cnt[j] = lq < nq ? quad_count(c, nints) : 0u;
            }
            o1 = cnt[0];
            o2 = o1 + cnt[1];
            o3 = o2 + cnt[2];
            tsum = o3 + cnt[3];
        }
        uint32_t incl = warp_incl_scan(tsum);
        if (lane == 31)
            s_warp[warp] = incl;
        named_sync(1, kThreads);
        uint32_t wpre = 0;
#pragma unroll
        for (int j = 0; j < kWarps; j++)
            wpre += j < warp ? s_warp[j] : 0u;
        {
            const uint32_t o0 = h + wpre + incl - tsum;  // staged position of the thread's data
            reinterpret_cast<uint2 *>(s_qoff)[tid] =
                make_uint2(o0 | ((o0 + o1) << 16), (o0 + o2) | ((o0 + o3) << 16));
        }
        named_sync(1, kThreads);

        // ---- gather: one quad per lane per round ----------------------------
        const uint32_t lq0 = warp * (32 * kTileRounds) + lane;
        const uint8_t *Cl = C + lq0;
        const uint16_t *Ql = s_qoff + lq0;
        uint32_t *op = a.out + 4 * (q0 + lq0);
        uint32_t v[kTileRounds][4];
        if (full) {
#pragma unroll
            for (int r = 0; r < kTileRounds; r++) {
                const uint32_t c = Cl[32 * r];
                const uint32_t p = Ql[32 * r];
                uint4 x;
                if (__all_sync(0xffffffffu, c == 0))
                    x = widen_quad(D, p);
                else
                    x = decode_quad(D, p, c);
                v[r][0] = x.x;
                v[r][1] = x.y;
                v[r][2] = x.z;
                v[r][3] = x.w;
                if (kMode == kPlain) {
                    if (a.out_aligned) {
                        stg_stream128(op + 128 * r, x);
                    } else {
                        op[128 * r + 0] = x.x;
                        op[128 * r + 1] = x.y;
                        op[128 * r + 2] = x.z;
                        op[128 * r + 3] = x.w;
                    }
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < kTileRounds; r++) {
                const uint32_t lq = lq0 + r * 32;
                const bool valid = lq < nq;
                uint32_t c = valid ? C[lq] : 0u;
                const uint32_t nints = !valid ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
                if (nints < 4)
                    c &= (1u << (2 * nints)) - 1u;
                const uint32_t p = valid ? s_qoff[lq] : h;
                uint4 x = decode_quad(D, p, c);
                v[r][0] = nints > 0 ? x.x : 0u;
                v[r][1] = nints > 1 ? x.y : 0u;
                v[r][2] = nints > 2 ? x.z : 0u;
                v[r][3] = nints > 3 ? x.w : 0u;
                if (kMode == kPlain && valid) {
                    op[128 * r] = x.x;
                    if (nints > 1)
                        op[128 * r + 1] = x.y;
                    if (nints > 2)
                        op[128 * r + 2] = x.z;
                    if (nints > 3)
                        op[128 * r + 3] = x.w;
                }
            }
        }
        // This warp no longer reads stage s.
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.empty[s]);

        if (kMode == kSums) {
            // ---- the tile's gap sum; thread 0 keeps the CTA's running total --
            uint32_t t = 0;
#pragma unroll
            for (int r = 0; r < kTileRounds; r++)
                t += v[r][0] + v[r][1] + v[r][2] + v[r][3];
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1)
                t += __shfl_xor_sync(0xffffffffu, t, d);
            named_sync(1, kThreads);  // every warp has read s_warp (offsets) above
            if (lane == 0)
                s_warp[warp] = t;
            named_sync(1, kThreads);
            if (tid == 0) {
                uint32_t vagg = 0;
#pragma unroll
                for (int j = 0; j < kWarps; j++)
                    vagg += s_warp[j];
                a.carries[tile] = running;  // carry relative to the CTA's first tile
                running += vagg;
            }
        }
        if (kMode == kDelta) {
            // ---- running sums: quad, warp, block, plus the carry-in -----------
            uint32_t qexcl[kTileRounds], wrun = 0;
#pragma unroll
            for (int r = 0; r < kTileRounds; r++) {
                v[r][1] += v[r][0];
                v[r][2] += v[r][1];
                v[r][3] += v[r][2];
                uint32_t qs = v[r][3];
                uint32_t inc = warp_incl_scan(qs);
                qexcl[r] = wrun + inc - qs;
                wrun += __shfl_sync(0xffffffffu, inc, 31);
            }
            named_sync(1, kThreads);  // every warp has read s_warp (offsets) above
            if (lane == 0)
                s_warp[warp] = wrun;
            named_sync(1, kThreads);
            uint32_t bpre = carry_in;
#pragma unroll
            for (int j = 0; j < kWarps; j++)
                bpre += j < warp ? s_warp[j] : 0u;
#pragma unroll
            for (int r = 0; r < kTileRounds; r++) {
                const uint32_t lq = lq0 + r * 32;
                if (lq >= nq)
                    continue;
                const uint32_t nints = full ? 4u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
                const uint32_t add = bpre + qexcl[r];
                uint32_t *dst = op + 128 * r;
                uint4 y = make_uint4(v[r][0] + add, v[r][1] + add, v[r][2] + add, v[r][3] + add);
                if (nints == 4 && a.out_aligned) {
                    stg_stream128(dst, y);
                } else {
                    dst[0] = y.x;
                    if (nints > 1)
                        dst[1] = y.y;
                    if (nints > 2)
                        dst[2] = y.z;
                    if (nints > 3)
                        dst[3] = y.w;
                }
            }
        }
    }

    if (kMode == kSums) {
        // Chain this CTA's range total with the ranges before it, then turn
        // the range-relative carries into absolute ones (prev included).
        __shared__ uint32_t s_base;
        if (warp == 0) {
            u64 range_total = __shfl_sync(0xffffffffu, running, 0);
            TileStatus *me = &a.st[first / (a.per_cta ? a.per_cta : 1)];
            const u64 cta = first / (a.per_cta ? a.per_cta : 1);
            u64 base = a.prev;
            bool ok = true;
            if (cta == 0) {
                if (lane == 0)
                    publish(&me->val_tag, &me->val_pre, (uint32_t)(a.prev + range_total),
                            kFlagPrefix, etag);
            } else {
                if (lane == 0)
                    publish(&me->val_tag, &me->val_agg, (uint32_t)range_total, kFlagAgg, etag);
                base = lookback<true>(a.st, cta, etag, a.spin_limit, a.hdr, ok);
                if (ok && lane == 0)
                    publish(&me->val_tag, &me->val_pre, (uint32_t)(base + range_total),
                            kFlagPrefix, etag);
            }
            if (lane == 0) {
                if (!ok)
                    raise_error(a.hdr, kErrTimeout);
                s_base = (uint32_t)base;
            }
        }
        named_sync(1, kThreads);
        const uint32_t base = s_base;
        const u64 end = min(first + a.per_cta, a.ntiles);
        for (u64 t = first + tid; t < end; t += kThreads)
            a.carries[t] += base;
    }
}

template <int kMode>
__global__ void __launch_bounds__(kDecBlock, 3) decode_tiled_kernel(TiledArgs a)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    Pipe &P = *reinterpret_cast<Pipe *>(dyn_smem);
    __shared__ __align__(16) uint16_t s_qoff[kTileQuads];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ u64 s_etag, s_first;
    __shared__ uint32_t s_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&P.full[s], 32);        // the 32 producer lanes arrive
            mbar_init(&P.empty[s], kWarps);   // one arrival per consumer warp
        }
        fence_mbar_init();
        s_etag = (ld_relaxed(&a.hdr->epoch) + 1) << 2;
        s_flag = error_raised(a.hdr) ? 1u : 0u;
        // The sums pass takes ranges in claim order, so every range before
        // this one belongs to a CTA that is running or done.
        s_first = kMode == kSums ? atomicAdd(&a.hdr->tile_counter, 1ull) * a.per_cta
                                 : (u64)blockIdx.x;
    }
    __syncthreads();
    if (!s_flag) {  // else the offsets pass failed (truncated stream)
        if (warp == kWarps)
            produce<kMode>(a, P, s_first, lane);
        else
            consume<kMode>(a, P, s_qoff, s_warp, s_first, s_etag);
    }
    if (kMode == kSums) {
        // The decode pass that follows owns the result and the counters; only
        // reset the claim counter for it.
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            u64 done = atomicAdd(&a.hdr->done_counter, 1ull);
            if (done == (u64)gridDim.x - 1) {
                st_relaxed(&a.hdr->tile_counter, 0);
                st_relaxed(&a.hdr->done_counter, 0);
            }
        }
    } else {
        finish_launch(a.hdr, a.result);
    }
}

// ---------------------------------------------------------------------------

static int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 148;
    }
    return sms;
}

template <int kMode>
static int tiled_grid()
{
    static int g = 0;
    if (!g) {
        cudaFuncSetAttribute(decode_tiled_kernel<kMode>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Pipe));
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_tiled_kernel<kMode>, kDecBlock,
                                                      sizeof(Pipe));
        g = sm_count() * (occ > 0 ? occ : 1);
    }
    return g;
}

static int offsets_grid()
{
    static int g = 0;
    if (!g) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, offsets_kernel, kThreads, 0);
        g = sm_count() * (occ > 0 ? occ : 1);
    }
    return g;
}

int launch_decode_tiled(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                        bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                        u64 spin_limit)
{
    const WsLayout L = ws_layout(n);
    const u64 nquads = (n + 3) / 4;
    const u64 ntiles = (nquads + kTileQuads - 1) / kTileQuads;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    u64 *offs = reinterpret_cast<u64 *>(static_cast<char *>(ws) + L.offs);
    uint32_t *carries = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + L.carries);
    TileStatus *st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + L.status);

    OffsetsArgs o;
    o.in = in;
    o.in_len = in_len;
    o.n = n;
    o.nquads = nquads;
    o.ntiles = ntiles;
    o.groups = (ntiles + kOffGroup - 1) / kOffGroup;
    u64 ogrid = min((u64)offsets_grid(), o.groups);
    o.per_cta = (o.groups + ogrid - 1) / ogrid;
    ogrid = (o.groups + o.per_cta - 1) / o.per_cta;  // no CTA without groups
    o.offs = offs;
    o.hdr = hdr;
    o.st = st;
    o.spin_limit = spin_limit;
    o.in_aligned = (((uintptr_t)in) & 15u) == 0;
    prof_begin("offsets_kernel", stream);
    offsets_kernel<<<(unsigned)ogrid, kThreads, 0, stream>>>(o);
    prof_end(stream);

    TiledArgs t;
    t.in = in;
    t.n = n;
    t.nquads = nquads;
    t.ntiles = ntiles;
    t.out = out;
    t.offs = offs;
    t.carries = carries;
    t.hdr = hdr;
    t.st = st;
    t.result = result;
    t.spin_limit = spin_limit;
    t.per_cta = 0;
    t.prev = prev;
    t.out_aligned = (((uintptr_t)out) & 15u) == 0;
    if (delta) {
        // Sums pass over contiguous ranges, then the decode with carries.
        u64 sgrid = min((u64)tiled_grid<kSums>(), ntiles);
        t.per_cta = (ntiles + sgrid - 1) / sgrid;
        sgrid = (ntiles + t.per_cta - 1) / t.per_cta;
        prof_begin("decode_tiled_kernel<sums>", stream);
        decode_tiled_kernel<kSums><<<(unsigned)sgrid, kDecBlock, sizeof(Pipe), stream>>>(t);
        prof_end(stream);
        t.per_cta = 0;
        u64 grid = min((u64)tiled_grid<kDelta>(), ntiles);
        prof_begin("decode_tiled_kernel<delta>", stream);
        decode_tiled_kernel<kDelta><<<(unsigned)grid, kDecBlock, sizeof(Pipe), stream>>>(t);
        prof_end(stream);
    } else {
        u64 grid = min((u64)tiled_grid<kPlain>(), ntiles);
        prof_begin("decode_tiled_kernel<plain>", stream);
        decode_tiled_kernel<kPlain><<<(unsigned)grid, kDecBlock, sizeof(Pipe), stream>>>(t);
        prof_end(stream);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // namespace svb
