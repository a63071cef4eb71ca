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
//                    offset in the data stream (a prefix sum of the per-quad
//                    counts C, chained across CTAs by a decoupled look-back),
//                    plus the stream's total size and the truncation check;
//   decode_tiled     persistent CTAs claim tiles in order; the TMA engine
//                    copies the next tile's control and data bytes into one
//                    of two shared-memory stages (cp.async.bulk, completion on
//                    an mbarrier) while the current tile is decoded, so every
//                    SM keeps loads in flight without waiting on other CTAs.
// Differential streams add one look-back over the tiles' gap sums (the carry
// of Sec. 2's prefix sum across tiles) before a tile's values are stored.
//
// Bytes outside the stream are never read: each tile's range is copied as its
// 16-byte-aligned interior by the bulk engine plus a ragged head and tail of
// at most 15 bytes each by plain loads.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"

namespace svb {

constexpr int kTileQuads = 1024;                    // quads per tile (4096 integers)
constexpr int kTileRounds = kTileQuads / kThreads;  // quads per lane per tile
constexpr int kTileData = 16 * kTileQuads;          // data bytes per tile, at most
constexpr int kStageData = kTileData + 64;          // + 16-byte phase + 2-word read slack
constexpr int kStageCtrl = kTileQuads + 32;
constexpr int kOffTiles = 16;                       // tiles per CTA of the offsets pass
constexpr u64 kBarrierPolls = 1ull << 24;           // bound on one mbarrier wait

// ---------------------------------------------------------------------------
// Pass 1: tile offsets from the control stream.

struct OffsetsArgs {
    const uint8_t *in;
    u64 in_len;
    u64 n, nquads, ntiles, nctas;
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
    if (q + 16 < nquads) {  // no last quad inside: the common case
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t t = 64;
#pragma unroll
        for (int i = 0; i < 4; i++)
            t += __popc(w[i] & 0x55555555u) + 2u * __popc(w[i] & 0xAAAAAAAAu);
        return t;
    }
    uint32_t w[4] = {v.x, v.y, v.z, v.w}, t = 0;
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

__global__ void __launch_bounds__(kThreads) offsets_kernel(OffsetsArgs a)
{
    __shared__ uint32_t s_tsum[kOffTiles];
    __shared__ u64 s_cta, s_etag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_cta = atomicAdd(&a.hdr->a_counter, 1ull);
        s_etag = (ld_relaxed(&a.hdr->epoch) + 1) << 2;
    }
    __syncthreads();
    const u64 cta = s_cta, etag = s_etag;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));

    // Thread t sums control bytes [64t, 64t + 64) of this CTA's 16 tiles:
    // 16 threads per tile.
    const u64 q = cta * (u64)(kOffTiles * kTileQuads) + 64u * tid;
    uint32_t sum = 0;
    if (q < a.nquads) {
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
    }
#pragma unroll
    for (int d = 8; d >= 1; d >>= 1)
        sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if ((tid & 15) == 0)
        s_tsum[tid >> 4] = sum;
    __syncthreads();

    if (warp == 0) {
        uint32_t ts = lane < kOffTiles ? s_tsum[lane] : 0u;
        uint32_t inc = warp_incl_scan(ts);
        uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        TileStatus *me = &a.st[cta];
        u64 base = 0;
        bool ok = true;
        if (cta == 0) {
            if (lane == 0)
                publish(&me->off_tag, &me->off_pre, total, kFlagPrefix, etag);
        } else {
            if (lane == 0)
                publish(&me->off_tag, &me->off_agg, total, kFlagAgg, etag);
            base = lookback<false>(a.st, cta, etag, a.spin_limit, a.hdr, ok);
            if (ok && lane == 0)
                publish(&me->off_tag, &me->off_pre, base + total, kFlagPrefix, etag);
        }
        if (!ok) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
        } else {
            u64 tile = cta * kOffTiles + lane;
            if (lane < kOffTiles && tile < a.ntiles)
                a.offs[tile] = base + (inc - ts);
            if (cta == a.nctas - 1 && lane == 0) {
                u64 stream = a.nquads + base + total;
                a.offs[a.ntiles] = base + total;
                st_relaxed(&a.hdr->total, stream);
                if (stream > a.in_len)
                    raise_error(a.hdr, kErrTruncated);
            }
        }
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
// Pass 2: persistent decode with double-buffered bulk staging.

struct TiledArgs {
    const uint8_t *in;
    u64 n, nquads, ntiles;
    uint32_t *out;
    const u64 *offs;
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    uint32_t prev;
    uint32_t out_aligned;
};

struct Stages {
    uint8_t data[2][kStageData];
    uint8_t ctrl[2][kStageCtrl];
    uint64_t bar[2];
    u64 tile[2];
    uint32_t hd[2], hc[2];  // address phase (mod 16) of the data and control ranges
};

// Copy global [g, g + len) to smem base + (g mod 16) .. : interior by one
// bulk copy (lane 0 issues it), head and tail bytes by the warp's lanes.
// Returns the bulk byte count.
__device__ __forceinline__ uint32_t range_interior(const uint8_t *g, uint32_t len,
                                                   const uint8_t *&a0, uint32_t &off0)
{
    uintptr_t s = (uintptr_t)g, e = s + len;
    uintptr_t c0 = (s + 15) & ~(uintptr_t)15, c1 = e & ~(uintptr_t)15;
    a0 = reinterpret_cast<const uint8_t *>(c0);
    off0 = (uint32_t)(c0 - (s & ~(uintptr_t)15));
    return c1 > c0 ? (uint32_t)(c1 - c0) : 0u;
}

__device__ __forceinline__ void range_edges(const uint8_t *g, uint32_t len, uint8_t *base,
                                            int lane)
{
    uintptr_t s = (uintptr_t)g, e = s + len;
    uintptr_t c0 = (s + 15) & ~(uintptr_t)15, c1 = e & ~(uintptr_t)15;
    uint32_t h = (uint32_t)(s & 15u);
    uint32_t head = (uint32_t)((c0 < e ? c0 : e) - s);                 // bytes [0, head)
    uint32_t tail0 = (uint32_t)((c1 > c0 ? c1 : (c0 < e ? c0 : e)) - s);  // bytes [tail0, len)
    for (uint32_t i = lane; i < head; i += 32)
        base[h + i] = __ldg(g + i);
    for (uint32_t i = tail0 + lane; i < len; i += 32)
        base[h + i] = __ldg(g + i);
}

// Warp 0: claim the next tile and start its copies into stage ns.
__device__ __forceinline__ void claim_and_issue(const TiledArgs &a, Stages &S, int ns, int lane)
{
    u64 t = 0;
    if (lane == 0)
        t = atomicAdd(&a.hdr->tile_counter, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (lane == 0)
        S.tile[ns] = t;
    if (t >= a.ntiles)
        return;
    const u64 q0 = t * kTileQuads;
    const uint32_t clen = (uint32_t)min((u64)kTileQuads, a.nquads - q0);
    const uint8_t *gc = a.in + q0;
    const u64 d0 = a.offs[t], d1 = a.offs[t + 1];
    const uint8_t *gd = a.in + a.nquads + d0;
    const uint32_t dlen = (uint32_t)(d1 - d0);
    const uint8_t *ac, *ad;
    uint32_t oc, od;
    uint32_t bc = range_interior(gc, clen, ac, oc);
    uint32_t bd = range_interior(gd, dlen, ad, od);
    if (lane == 0) {
        S.hc[ns] = (uint32_t)((uintptr_t)gc & 15u);
        S.hd[ns] = (uint32_t)((uintptr_t)gd & 15u);
        mbar_arrive_expect_tx(&S.bar[ns], bc + bd);
        if (bc)
            bulk_g2s(S.ctrl[ns] + oc, ac, bc, &S.bar[ns]);
        if (bd)
            bulk_g2s(S.data[ns] + od, ad, bd, &S.bar[ns]);
    }
    range_edges(gc, clen, S.ctrl[ns], lane);
    range_edges(gd, dlen, S.data[ns], lane);
}

__device__ __forceinline__ uint32_t quad_count(uint32_t c, uint32_t nints)
{
    return nints + __popc(c & 0x55u) + 2u * __popc(c & 0xAAu);
}

__device__ __forceinline__ uint32_t value_at(const uint32_t *s32, uint32_t p, uint32_t code)
{
    uint32_t v = __funnelshift_r(s32[p >> 2], s32[(p >> 2) + 1], (p & 3u) * 8u);
    return v & (0xffffffffu >> (24u - 8u * code));
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads, 3) decode_tiled_kernel(TiledArgs a)
{
    __shared__ __align__(16) Stages S;
    __shared__ __align__(16) uint16_t s_qoff[kTileQuads];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ u64 s_etag;
    __shared__ uint32_t s_flag, s_carry;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        s_etag = (ld_relaxed(&a.hdr->epoch) + 1) << 2;
        s_flag = error_raised(a.hdr) ? 1u : 0u;
    }
    __syncthreads();
    if (s_flag) {  // the offsets pass failed (truncated stream)
        finish_launch(a.hdr, a.result);
        return;
    }
    const u64 etag = s_etag;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    if (warp == 0)
        claim_and_issue(a, S, 0, lane);
    __syncthreads();

    // Stage s is used for iterations it = s, s + 2, ...; its k-th fill
    // completes phase k of its barrier, so iteration it waits on parity
    // (it >> 1) & 1.
    int exit_reason = 0;  // 0 done, 1 a copy never completed, 2 carry look-back failed
    uint32_t it = 0;
    for (;; it++) {
        const int s = it & 1;
        const u64 tile = S.tile[s];
        if (tile >= a.ntiles)
            break;
        if (warp == 0)
            claim_and_issue(a, S, s ^ 1, lane);
        bool ok = mbar_wait_bounded(&S.bar[s], (it >> 1) & 1u, kBarrierPolls);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                raise_error(a.hdr, kErrTimeout);
            exit_reason = 1;
            break;
        }

        // ---- control bytes -> quad offsets inside the tile ------------------
        const u64 q0 = tile * kTileQuads;
        const uint32_t nq = (uint32_t)min((u64)kTileQuads, a.nquads - q0);
        const uint8_t *C = S.ctrl[s] + S.hc[s];
        const uint8_t *D = S.data[s];
        const uint32_t h = S.hd[s];
        uint32_t w = 0;
        if (S.hc[s] == 0 && 4u * tid + 4u <= nq) {
            w = reinterpret_cast<const uint32_t *>(C)[tid];
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (4u * tid + j < nq)
                    w |= (uint32_t)C[4 * tid + j] << (8 * j);
        }
        uint32_t cnt[4], tsum = 0;
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
            tsum += cnt[j];
        }
        uint32_t incl = warp_incl_scan(tsum);
        if (lane == 31)
            s_warp[warp] = incl;
        __syncthreads();
        uint32_t wpre = 0;
#pragma unroll
        for (int k = 0; k < kWarps; k++)
            wpre += k < warp ? s_warp[k] : 0u;
        {
            uint32_t o0 = wpre + incl - tsum, o1 = o0 + cnt[0], o2 = o1 + cnt[1], o3 = o2 + cnt[2];
            reinterpret_cast<uint2 *>(s_qoff)[tid] = make_uint2(o0 | (o1 << 16), o2 | (o3 << 16));
        }
        __syncthreads();

        // ---- gather: one quad per lane per round ----------------------------
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(D);
        uint32_t v[kTileRounds][4];
#pragma unroll
        for (int r = 0; r < kTileRounds; r++) {
            const uint32_t lq = warp * (32 * kTileRounds) + r * 32 + lane;
            const bool valid = lq < nq;
            uint32_t c = valid ? C[lq] : 0u;
            const uint32_t nints = !valid ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
            if (nints < 4)
                c &= (1u << (2 * nints)) - 1u;
            const uint32_t p = h + (valid ? s_qoff[lq] : 0u);
            if (__all_sync(0xffffffffu, c == 0)) {
                uint32_t d = __funnelshift_r(s32[p >> 2], s32[(p >> 2) + 1], (p & 3u) * 8u);
                v[r][0] = __byte_perm(d, 0, 0x4440);
                v[r][1] = __byte_perm(d, 0, 0x4441);
                v[r][2] = __byte_perm(d, 0, 0x4442);
                v[r][3] = __byte_perm(d, 0, 0x4443);
            } else {
                uint32_t pp = p;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    uint32_t code = (c >> (2 * k)) & 3u;
                    v[r][k] = value_at(s32, pp, code);
                    pp += code + 1;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                if ((uint32_t)k >= nints)
                    v[r][k] = 0;
            if (!kDelta && valid) {
                uint32_t *dst = a.out + 4 * (q0 + lq);
                if (nints == 4 && a.out_aligned) {
                    stg_stream128(dst, make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]));
                } else {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if ((uint32_t)k < nints)
                            dst[k] = v[r][k];
                }
            }
        }

        if (kDelta) {
            // ---- running sums: quad, warp, block, then across tiles ----------
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
            __syncthreads();  // everyone has read s_warp (offsets) above
            if (lane == 0)
                s_warp[warp] = wrun;
            __syncthreads();
            uint32_t bpre = 0, vagg = 0;
#pragma unroll
            for (int k = 0; k < kWarps; k++) {
                uint32_t t = s_warp[k];
                bpre += k < warp ? t : 0u;
                vagg += t;
            }
            if (warp == 0) {
                TileStatus *me = &a.st[tile];
                u64 carry = a.prev;
                bool lok = true;
                if (tile == 0) {
                    if (lane == 0)
                        publish(&me->val_tag, &me->val_pre, (uint32_t)(a.prev + vagg),
                                kFlagPrefix, etag);
                } else {
                    if (lane == 0)
                        publish(&me->val_tag, &me->val_agg, vagg, kFlagAgg, etag);
                    carry = lookback<true>(a.st, tile, etag, a.spin_limit, a.hdr, lok);
                    if (lok && lane == 0)
                        publish(&me->val_tag, &me->val_pre, (uint32_t)(carry + vagg),
                                kFlagPrefix, etag);
                }
                if (lane == 0) {
                    if (!lok)
                        raise_error(a.hdr, kErrTimeout);
                    s_carry = (uint32_t)carry;
                    s_flag = lok ? 0u : 1u;
                }
            }
            __syncthreads();
            if (s_flag) {
                exit_reason = 2;
                break;
            }
            const uint32_t base = s_carry + bpre;
#pragma unroll
            for (int r = 0; r < kTileRounds; r++) {
                const uint32_t lq = warp * (32 * kTileRounds) + r * 32 + lane;
                if (lq >= nq)
                    continue;
                const uint32_t nints = q0 + lq == a.nquads - 1 ? last_nints : 4u;
                const uint32_t add = base + qexcl[r];
                uint32_t *dst = a.out + 4 * (q0 + lq);
                uint4 x = make_uint4(v[r][0] + add, v[r][1] + add, v[r][2] + add, v[r][3] + add);
                if (nints == 4 && a.out_aligned) {
                    stg_stream128(dst, x);
                } else {
                    dst[0] = x.x;
                    if (nints > 1)
                        dst[1] = x.y;
                    if (nints > 2)
                        dst[2] = x.z;
                    if (nints > 3)
                        dst[3] = x.w;
                }
            }
        }
        __syncthreads();  // stage s, s_qoff and s_warp are free again
    }

    // After an early exit, let the copies still in flight land before the
    // CTA's shared memory goes away (bounded like every other wait).
    if (exit_reason != 0 && tid == 0) {
        const int s = it & 1;
        if (exit_reason == 1)
            mbar_wait_bounded(&S.bar[s], (it >> 1) & 1u, kBarrierPolls);
        if (S.tile[s ^ 1] < a.ntiles)
            mbar_wait_bounded(&S.bar[s ^ 1], ((it + 1) >> 1) & 1u, kBarrierPolls);
    }
    finish_launch(a.hdr, a.result);
}

// ---------------------------------------------------------------------------

static int tiled_grid(bool delta)
{
    static int cached[2] = {0, 0};
    int &g = cached[delta ? 1 : 0];
    if (!g) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (delta)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_tiled_kernel<true>,
                                                          kThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_tiled_kernel<false>,
                                                          kThreads, 0);
        g = (sms > 0 ? sms : 148) * (occ > 0 ? occ : 1);
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
    TileStatus *st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + L.status);

    OffsetsArgs o;
    o.in = in;
    o.in_len = in_len;
    o.n = n;
    o.nquads = nquads;
    o.ntiles = ntiles;
    o.nctas = (ntiles + kOffTiles - 1) / kOffTiles;
    o.offs = offs;
    o.hdr = hdr;
    o.st = st;
    o.spin_limit = spin_limit;
    o.in_aligned = (((uintptr_t)in) & 15u) == 0;
    offsets_kernel<<<(unsigned)o.nctas, kThreads, 0, stream>>>(o);

    TiledArgs t;
    t.in = in;
    t.n = n;
    t.nquads = nquads;
    t.ntiles = ntiles;
    t.out = out;
    t.offs = offs;
    t.hdr = hdr;
    t.st = st;
    t.result = result;
    t.spin_limit = spin_limit;
    t.prev = prev;
    t.out_aligned = (((uintptr_t)out) & 15u) == 0;
    u64 grid = min((u64)tiled_grid(delta), ntiles);
    if (delta)
        decode_tiled_kernel<true><<<(unsigned)grid, kThreads, 0, stream>>>(t);
    else
        decode_tiled_kernel<false><<<(unsigned)grid, kThreads, 0, stream>>>(t);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // namespace svb
