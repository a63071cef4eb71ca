// Batched Stream VByte codec: many independent streams (posting lists, the
// paper's use case in Sec. 5) of very uneven lengths in one persistent launch.
//
// Each list is its own stream (ceil(n/4) control bytes, then data, Sec. 4)
// with its own start value for differential coding (Sec. 2, Sec. 5).  Lists
// are independent, so no list ever waits on another:
//   * big lists (n >= the plan's threshold, longest first) are each taken by
//     one CTA and processed tile by tile through the same producer/consumer
//     pipeline as the single-stream decoder.  The producer sums each tile's
//     control bytes to find where the next tile's data starts, so it needs no
//     separate offsets pass; consumers carry the running differential sum of
//     the list from tile to tile in registers.
//   * small lists are taken one at a time by single warps once the big lists
//     are handed out; every warp of the CTA (the producer included) takes
//     part, which also evens out the end of the launch.
// The plan (built on the host from the list lengths) holds the two id lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"
#include "svb_subtile.cuh"
#include "svb_subenc.cuh"

namespace svb {

constexpr int kBQuads = 1024;                // quads per tile of 4096 integers
constexpr int kBBlock = kThreads + 32;       // 8 consumer warps + 1 producer warp
constexpr u64 kBPolls = 1ull << 24;
constexpr uint32_t kNoList = 0xffffffffu;
constexpr uint32_t kDefaultBigThreshold = 8192;
constexpr u64 kErrInvalid = 1;   // SVB_EINVAL: a plan made for another decode tile
constexpr int kBSubs = kBQuads / kSubQuads;   // sub-tiles per tile = consumer warps
static_assert(kBSubs == kWarps, "one consumer warp per sub-tile");

// Plan layout in device memory: header, big ids, small ids; then, when the
// plan has units (nunits > 0), a units header, the units and one record per
// unit.  A unit is a run of tiles of one big list; a list longer than the
// split length is cut into several units so that several CTAs decode it at
// once.  The split lists' units come first (units [0, nsplit)); a batch
// decode first runs batch_prep_kernel over them to find each unit's data
// offset and carry-in within its list, then decodes units as it would lists.
// Plans without units (nunits = 0) decode each big list whole.
// tile_quads is the decode tile (kBQuads times 1 or 2) the plan's units and
// split decisions were made for; a decode built for another tile refuses it.
struct PlanHeader {
    uint32_t nbig, nsmall, threshold, nunits;
    uint32_t tile_quads, pad[3];
};

struct PlanUnit {
    uint32_t list, t0, nt;   // tiles [t0, t0 + nt) of list `list`
    uint32_t seg;            // the unit's index among its list's units
    u64 d0;                  // data offset of tile t0 within the list's data (prep)
    uint32_t c0;             // carry-in: the list's integer before tile t0 (prep)
    uint32_t first;          // index of the list's first unit
};

constexpr uint32_t kSegTiles = 16;          // default tiles per unit of a split list
constexpr size_t kExtraUnits = 32768;       // units a plan may add beyond one per list

// ---------------------------------------------------------------------------
// Decode

struct BatchDecArgs {
    const svb_list *lists;
    const PlanHeader *plan;
    const uint8_t *in;
    uint32_t *out;
    WsHeader *hdr;
    DeviceResult *result;
    uint32_t delta;
};

// Control bytes travel ahead of the data: tile g's control bytes sit in ring
// slot g % kCRing and are fetched kCAhead tiles before its data, so the
// producer never waits a round trip to learn where a tile's data start.  Slot
// (g + kCAhead) % kCRing was last used by tile g - S, whose stage the
// producer has seen released before it refills the slot.
constexpr int kCAhead = 2;

// Staging depth S (stages of tile data) and tile size (K * 4096 integers:
// each consumer warp decodes K sub-tiles of a tile, 16 K integers a lane)
// are compile-time parameters of the decode kernel: the autotuner picks
// among the instantiations.
template <int S, int K>
struct BPipe {
    static constexpr int kCRing = S + kCAhead;
    static constexpr int kTQ = K * kBQuads;   // quads per tile
    uint8_t data[S][16 * kTQ + 64];
    uint8_t ctrl[kCRing][kTQ + 32];
    uint64_t full[S];   // control and data landed (consumers wait)
    uint64_t cfull[kCRing];    // control landed (the producer waits)
    uint64_t empty[S];  // consumers done with the stage
    uint32_t list[S];   // list id, or kNoList
    uint32_t tile[S];   // tile index within the list
    uint32_t skip[S];   // the list is truncated: decode nothing
    uint32_t hd[S], hc[S];
    uint32_t clist[kCRing], ctile[kCRing], chc[kCRing];   // what each ring slot holds
    uint32_t cfirst[kCRing], cc0[kCRing];   // first tile of a unit; the unit's carry-in
    u64 cd0[kCRing];                        // and its data offset within the list
    uint32_t soff[S][K * kBSubs];   // each sub-tile's data offset inside the tile
    u64 out_off[S];             // the tile's list: where its integers go,
    uint32_t n[S], prev[S];   // how many, and the unit's carry-in
    uint32_t first[S];               // the stage holds a unit's first tile
};

__device__ __forceinline__ const uint32_t *plan_big(const PlanHeader *p)
{
    return reinterpret_cast<const uint32_t *>(p + 1);
}

__device__ __forceinline__ const uint32_t *plan_small(const PlanHeader *p)
{
    return plan_big(p) + p->nbig;
}

// Byte offsets within the plan of its units header (one u32: nsplit), its
// units and its records, for a plan of `ids` big + small ids and up to
// `units` units.
__host__ __device__ __forceinline__ size_t plan_units_off(size_t ids)
{
    return (sizeof(PlanHeader) + 4 * ids + 15) / 16 * 16;
}

__host__ __device__ __forceinline__ size_t plan_recs_off(size_t ids, size_t units)
{
    return (plan_units_off(ids) + 16 + sizeof(PlanUnit) * units + 63) / 64 * 64;
}

__device__ __forceinline__ uint32_t plan_nsplit(const PlanHeader *p)
{
    if (p->nunits == 0)
        return 0;
    const size_t ids = (size_t)p->nbig + p->nsmall;
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(p) +
                                               plan_units_off(ids));
}

__device__ __forceinline__ PlanUnit *plan_units(const PlanHeader *p)
{
    const size_t ids = (size_t)p->nbig + p->nsmall;
    return reinterpret_cast<PlanUnit *>(
        const_cast<char *>(reinterpret_cast<const char *>(p)) + plan_units_off(ids) + 16);
}

__device__ __forceinline__ TileStatus *plan_recs(const PlanHeader *p)
{
    const size_t ids = (size_t)p->nbig + p->nsmall;
    return reinterpret_cast<TileStatus *>(const_cast<char *>(reinterpret_cast<const char *>(p)) +
                                          plan_recs_off(ids, p->nunits));
}

// Data bytes of the quads of one tile, from its staged control bytes
// (pad fields of the list's last quad count nothing).
// Data bytes before each sub-tile of one tile, from its staged control bytes
// (C, 16-byte phase h in the stage): lane i < kBSubs gets the offset of
// sub-tile i, every lane the tile's total.  A whole tile is read a word (four
// control bytes) at a time: word lane + 32i lies in sub-tile i, and a word of
// codes covers 16 + the sum of its codes bytes (Sec. 4).
__device__ __forceinline__ uint32_t tile_sub_offsets(const uint8_t *stage, uint32_t h, uint32_t nq,
                                                     bool last_tile, uint32_t last_nints,
                                                     int lane, uint32_t &total)
{
    uint32_t acc[kBSubs];
    if (nq == (uint32_t)kBQuads && !(last_tile && last_nints < 4)) {
        const uint32_t *W = reinterpret_cast<const uint32_t *>(stage) + (h >> 2);
        const uint32_t sh = 8 * (h & 3u);
#pragma unroll
        for (int i = 0; i < kBSubs; i++) {
            const uint32_t w = __funnelshift_r(W[lane + 32 * i], W[lane + 32 * i + 1], sh);
            acc[i] = 16u + __popc(w & 0x55555555u) + 2u * __popc(w & 0xAAAAAAAAu);
        }
    } else {
        const uint8_t *C = stage + h;
#pragma unroll
        for (int i = 0; i < kBSubs; i++) {
            acc[i] = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t q = 4 * (lane + 32 * i) + j;
                if (q < nq) {
                    uint32_t c = C[q];
                    const uint32_t k = (last_tile && q == nq - 1) ? last_nints : 4u;
                    if (k < 4)
                        c &= (1u << (2 * k)) - 1u;
                    acc[i] += quad_count(c, k);
                }
            }
        }
    }
    // Reduce-scatter over the warp: after the exchanges across lane bits 4, 3
    // and 2 each lane holds one sub-tile's sum over 8 lanes (sub-tile
    // lane >> 2), and two more finish it over all 32.
    const bool hi4 = lane & 16, hi3 = lane & 8, hi2 = lane & 4;
    uint32_t b[4], c[2];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t keep = hi4 ? acc[4 + j] : acc[j];
        const uint32_t give = hi4 ? acc[j] : acc[4 + j];
        b[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const uint32_t keep = hi3 ? b[2 + j] : b[j];
        const uint32_t give = hi3 ? b[j] : b[2 + j];
        c[j] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    uint32_t x = (hi2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, hi2 ? c[0] : c[1], 4);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    // Inclusive prefix over the sub-tiles, held by lanes 0, 4, .., 28.
    uint32_t inc = x;
#pragma unroll
    for (int d = 4; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d)
            inc += y;
    }
    total = __shfl_sync(0xffffffffu, inc, 28);
    const uint32_t excl = __shfl_sync(0xffffffffu, inc - x, (4 * lane) & 31);
    return lane < kBSubs ? excl : 0u;
}

__device__ __forceinline__ uint32_t tile_data_bytes(const uint8_t *C, uint32_t nq, bool last_tile,
                                                    uint32_t last_nints, int lane)
{
    uint32_t t = 0;
    for (uint32_t q = lane; q < nq; q += 32) {
        uint32_t c = C[q];
        uint32_t k = (last_tile && q == nq - 1) ? last_nints : 4u;
        if (k < 4)
            c &= (1u << (2 * k)) - 1u;
        t += quad_count(c, k);
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        t += __shfl_xor_sync(0xffffffffu, t, d);
    return t;
}

// Producer warp of the big-list phase.  Two cursors walk the big lists in
// claim order: the look-ahead cursor fetches control bytes kCAhead tiles
// ahead (claiming the next list as soon as it needs one), the data cursor
// sums each tile's staged control bytes to find where its data start and
// copies the data.  Every tile whose control bytes were fetched gets one stage
// (a skipped one if its list's data are cut short), so stage g always pairs
// with ring slot g % kCRing.
template <int S, int K>
__device__ void bdec_produce(const BatchDecArgs &a, BPipe<S, K> &P, int lane)
{
    constexpr int kCRing = BPipe<S, K>::kCRing;
    constexpr uint32_t kTQ = BPipe<S, K>::kTQ;
    const PlanHeader *plan = a.plan;
    const uint32_t *big = plan_big(plan);
    uint32_t issued = 0;   // stages posted

    // Look-ahead cursor.  With units, it claims units (a list's tiles
    // [t0, t0 + nt), starting at data offset d0 with carry-in c0, both from
    // batch_prep_kernel for the units of split lists); without, whole lists.
    const uint32_t nunits = plan->nunits;
    const PlanUnit *units = nunits ? plan_units(plan) : nullptr;
    uint32_t la_li = kNoList, la_k = 0, la_end = 0, la_nql = 0, la_c0 = 0;
    u64 la_off = 0, la_len = 0, la_d0 = 0;
    bool la_have = false, la_first = false;
    auto la_claim = [&]() {
        for (;;) {
            uint32_t j = 0;
            if (lane == 0)
                j = (uint32_t)atomicAdd(&a.hdr->tile_counter, 1ull);
            j = __shfl_sync(0xffffffffu, j, 0);
            if (j >= (nunits ? nunits : plan->nbig)) {
                la_have = false;
                return;
            }
            uint32_t li, t0 = 0, nt = 0, c0 = 0;
            u64 d0 = 0;
            bool seg = false;
            if (nunits) {
                const PlanUnit U = units[j];
                li = U.list;
                t0 = U.t0;
                nt = U.nt;
                seg = U.seg != 0;
                d0 = U.d0;
                c0 = U.c0;
            } else {
                li = big[j];
            }
            const svb_list L = a.lists[li];
            const uint32_t nql = (L.n + 3) / 4;
            if (nql > L.in_len) {   // its control bytes do not fit: reported, skipped
                if (lane == 0)
                    raise_error(a.hdr, kErrTruncated);
                continue;
            }
            const uint32_t ntl = (nql + kTQ - 1) / kTQ;
            la_li = li;
            la_nql = nql;
            la_off = L.in_off;
            la_len = L.in_len;
            la_k = nunits ? t0 : 0u;
            la_end = nunits ? min(t0 + nt, ntl) : ntl;
            la_d0 = seg ? d0 : 0;
            la_c0 = seg ? c0 : L.prev;
            la_first = true;
            la_have = la_k < la_end;
            if (la_have)
                return;
        }
    };
    uint32_t c_issued = 0;   // tiles whose control bytes were fetched
    auto fetch_ctrl = [&]() {
        if (!la_have)
            return;
        const int slot = c_issued % kCRing;
        const uint8_t *lo = a.in + la_off;
        const uint8_t *gc = lo + (u64)la_k * kTQ;
        const uint32_t clen = min(kTQ, la_nql - la_k * kTQ);
        const StagePlan pc = stage_plan(gc, clen, lo, lo + la_len);
        if (pc.edges)
            range_edges(gc, clen, P.ctrl[slot], lane);
        if (lane == 0) {
            P.clist[slot] = la_li;
            P.ctile[slot] = la_k;
            P.cfirst[slot] = la_first ? 1u : 0u;
            P.cd0[slot] = la_d0;
            P.cc0[slot] = la_c0;
            P.chc[slot] = (uint32_t)((uintptr_t)gc & 15u);
            mbar_arrive_expect_tx(&P.cfull[slot], pc.bytes);
            if (pc.bytes)
                bulk_g2s(P.ctrl[slot] + pc.dst_off, pc.src, pc.bytes, &P.cfull[slot]);
        } else {
            mbar_arrive(&P.cfull[slot]);
        }
        c_issued++;
        la_first = false;
        if (++la_k == la_end)
            la_claim();
    };
    auto wait_empty = [&](uint32_t g) -> bool {
        if (g < (uint32_t)S)
            return true;
        bool ok = mbar_wait_bounded(&P.empty[g % S], ((g / S) - 1) & 1u, kBPolls);
        return __all_sync(0xffffffffu, ok);
    };

    la_claim();
    for (int j = 0; j < kCAhead; j++)
        fetch_ctrl();

    // Data cursor.
    uint32_t li = kNoList, nql = 0, ntl = 0, last_nints = 4;
    u64 running = 0;
    svb_list L = {};
    bool cut = false;
    uint32_t c0 = 0;
    uint32_t g = 0;
    bool failed = false;
    for (; g < c_issued; g++) {
        const int slot = g % kCRing, s = g % S;
        if (!mbar_wait_bounded(&P.cfull[slot], (g / kCRing) & 1u, kBPolls)) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
        }
        __syncwarp();
        const uint32_t tli = P.clist[slot], tk = P.ctile[slot];
        const bool first = P.cfirst[slot] != 0;
        if (first) {   // a new unit (or list)
            li = tli;
            L = a.lists[li];
            nql = (L.n + 3) / 4;
            ntl = (nql + kTQ - 1) / kTQ;
            last_nints = L.n - 4 * (nql - 1);
            running = P.cd0[slot];
            c0 = P.cc0[slot];
            cut = false;
        }
        if (!wait_empty(g)) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            failed = true;
            break;
        }
        const bool last_tile = tk + 1 == ntl;
        const uint32_t nq = min(kTQ, nql - tk * kTQ);
        uint32_t dsize = 0, soff[K];
        if (!cut) {
            // The tile's 1024-quad pieces in turn: offsets within a piece,
            // plus the data bytes of the pieces before it.
#pragma unroll
            for (int k = 0; k < K; k++) {
                const uint32_t q0 = (uint32_t)k * kBQuads;
                soff[k] = dsize;
                if (q0 < nq) {
                    const uint32_t hq = min((uint32_t)kBQuads, nq - q0);
                    uint32_t part = 0;
                    soff[k] += tile_sub_offsets(P.ctrl[slot] + q0, P.chc[slot], hq,
                                                last_tile && q0 + hq == nq, last_nints, lane, part);
                    dsize += part;
                }
            }
            if (nql + running + dsize > L.in_len) {
                cut = true;
                if (lane == 0)
                    raise_error(a.hdr, kErrTruncated);
            }
        }
        fence_proxy_async_smem();  // these reads come before the slot's next fill
        const uint8_t *lo = a.in + L.in_off;
        const uint8_t *gd = lo + nql + running;
        const uint32_t dlen = cut ? 0u : dsize;
        const StagePlan pd = stage_plan(gd, dlen, lo, lo + L.in_len);
        if (pd.edges)
            range_edges(gd, dlen, P.data[s], lane);
        if (lane < kBSubs && !cut)
#pragma unroll
            for (int k = 0; k < K; k++)
                P.soff[s][k * kBSubs + lane] = soff[k];
        if (lane == 0) {
            P.list[s] = li;
            P.tile[s] = tk;
            P.out_off[s] = L.out_off;
            P.n[s] = L.n;
            P.prev[s] = c0;
            P.first[s] = first ? 1u : 0u;
            P.skip[s] = cut ? 1u : 0u;
            P.hd[s] = (uint32_t)((uintptr_t)gd & 15u);
            P.hc[s] = P.chc[slot];
            mbar_arrive_expect_tx(&P.full[s], pd.bytes);
            if (pd.bytes)
                bulk_g2s(P.data[s] + pd.dst_off, pd.src, pd.bytes, &P.full[s]);
        } else {
            mbar_arrive(&P.full[s]);
        }
        if (!cut) {
            running += dsize;
            if (last_tile && lane == 0)
                atomicAdd(&a.hdr->total, (u64)nql + running);
        }
        issued = g + 1;
        fetch_ctrl();   // the control bytes of tile g + kCAhead
    }
    if (!failed) {
        // No tile left: one stage marked kNoList ends the big-list phase.
        if (wait_empty(g)) {
            const int s = g % S;
            if (lane == 0) {
                P.list[s] = kNoList;
                mbar_arrive_expect_tx(&P.full[s], 0);
            } else {
                mbar_arrive(&P.full[s]);
            }
            issued = g + 1;
        } else if (lane == 0) {
            raise_error(a.hdr, kErrTimeout);
        }
    }
    // Let every copy this warp started land before the CTA can exit.
    if (lane == 0) {
        for (int s = 0; s < S; s++)
            if (issued > (uint32_t)s) {
                uint32_t fills = (issued - 1 - s) / S + 1;
                mbar_wait_bounded(&P.full[s], (fills - 1) & 1u, kBPolls);
            }
        for (int r = 0; r < kCRing; r++)
            if (c_issued > (uint32_t)r) {
                uint32_t fills = (c_issued - 1 - r) / kCRing + 1;
                mbar_wait_bounded(&P.cfull[r], (fills - 1) & 1u, kBPolls);
            }
    }
    __syncwarp();
}

// A full sub-tile's 512 integers (lane l holds quad 32r + l in v[r]) stored
// to dst, which is 4-byte aligned with M = (dst / 4) mod 4 in {1, 2, 3},
// with 16-byte writes.  The aligned chunk that ends with the first 4 - M
// integers of quad Q starts with the last M of quad Q - 1: lane l - 1's of
// the same round, or, for lane 0, lane 31's of the round before, which the
// rotated shuffle of that round already delivered to lane 0.  Only the
// sub-tile's first 4 - M integers and its last M go out one by one.
template <int M>
__device__ __forceinline__ void store_full_realigned(uint32_t *dst,
                                                     const uint32_t (&v)[kSubRounds][4])
{
    const int lane = threadIdx.x & 31;
    const int src = (lane + 31) & 31;
    uint32_t *chunk = dst + 4 * lane - M;   // 16-byte aligned
    uint32_t w1 = 0, w2 = 0, w3 = 0;        // lane 0: lane 31's last three of the round before
#pragma unroll
    for (int r = 0; r < kSubRounds; r++) {
        const uint32_t p1 = __shfl_sync(0xffffffffu, v[r][1], src);
        const uint32_t p2 = __shfl_sync(0xffffffffu, v[r][2], src);
        const uint32_t p3 = __shfl_sync(0xffffffffu, v[r][3], src);
        const uint32_t a1 = lane ? p1 : w1, a2 = lane ? p2 : w2, a3 = lane ? p3 : w3;
        uint4 c;
        if (M == 1)
            c = make_uint4(a3, v[r][0], v[r][1], v[r][2]);
        else if (M == 2)
            c = make_uint4(a2, a3, v[r][0], v[r][1]);
        else
            c = make_uint4(a1, a2, a3, v[r][0]);
        if (r > 0 || lane > 0)   // the chunk before quad 0 is not the sub-tile's
            stg_stream128(chunk + 128 * r, c);
        w1 = p1;
        w2 = p2;
        w3 = p3;
    }
    if (lane == 0) {
        dst[0] = v[0][0];
        if (M < 3)
            dst[1] = v[0][1];
        if (M < 2)
            dst[2] = v[0][2];
    }
    if (lane == 31) {
        uint32_t *q = dst + 4 * (kSubQuads - 1);
        q[3] = v[kSubRounds - 1][3];
        if (M > 1)
            q[2] = v[kSubRounds - 1][2];
        if (M > 2)
            q[1] = v[kSubRounds - 1][1];
    }
}

// A full sub-tile's integers to dst (4-byte aligned): 16-byte writes,
// realigned unless dst is 16-byte aligned.
__device__ __forceinline__ void store_full_subtile(uint32_t *dst,
                                                   const uint32_t (&v)[kSubRounds][4])
{
    const int lane = threadIdx.x & 31;
    const uint32_t m = (uint32_t)((uintptr_t)dst >> 2) & 3u;
    if (m == 0) {
#pragma unroll
        for (int r = 0; r < kSubRounds; r++)
            stg_stream128(dst + 128 * r + 4 * lane, make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]));
    } else if (m == 1) {
        store_full_realigned<1>(dst, v);
    } else if (m == 2) {
        store_full_realigned<2>(dst, v);
    } else {
        store_full_realigned<3>(dst, v);
    }
}

// Consumer warps of the big-list phase: warp w decodes sub-tiles w, w + 8,
// .. of every tile on its own (the same sub-tile decode as the
// single-stream decoder), one group of eight sub-tiles after another.  For
// differential lists the eight warps trade their sub-tile gap sums once per
// group (one barrier), and each keeps the list's running sum itself.
template <int S, int K>
__device__ void bdec_consume(const BatchDecArgs &a, BPipe<S, K> &P, uint16_t *s_pos,
                             uint32_t (*s_sum)[kWarps])
{
    constexpr int kCRing = BPipe<S, K>::kCRing;
    constexpr uint32_t kTQ = BPipe<S, K>::kTQ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *pos = s_pos + warp * kSubQuads;
    uint32_t carry = 0;  // the list's integer before the current group
    uint32_t ex = 0;     // gap-sum exchanges so far (selects the s_sum buffer)
    for (uint32_t g = 0;; g++) {
        const int s = g % S;
        if (!mbar_wait_bounded(&P.full[s], (g / S) & 1u, kBPolls)) {
            raise_error(a.hdr, kErrTimeout);
            break;
        }
        const uint32_t li = P.list[s];
        if (li == kNoList)
            break;
        const uint32_t n = P.n[s];
        const u64 out_off = P.out_off[s];
        const uint32_t k = P.tile[s];
        const uint32_t nql = (n + 3) / 4;
        const uint32_t last_nints = n - 4 * (nql - 1);
        const bool skip = P.skip[s] != 0;
        if (P.first[s])
            carry = P.prev[s];
        const bool aligned = ((uintptr_t)(a.out + out_off) & 15u) == 0;
#pragma unroll 1
        for (int j = 0; j < K; j++) {
            const uint32_t sub = (uint32_t)(j * kBSubs + warp);   // sub-tile within the tile
            const uint32_t q0 = k * kTQ + sub * kSubQuads;        // its first quad
            const bool have = !skip && q0 < nql;
            uint32_t v[kSubRounds][4] = {};
            SubTile t;
            t.nq = have ? min((uint32_t)kSubQuads, nql - q0) : 0u;
            if (have) {
                t.C = P.ctrl[g % kCRing] + P.hc[s] + sub * kSubQuads;
                t.D = P.data[s];
                t.base = P.hd[s] + P.soff[s][sub];
                t.tail = q0 + t.nq == nql ? last_nints : 4u;
                const uint32_t w = subtile_ctrl_word(t);
                __syncwarp();   // the previous group's gather has read pos
                subtile_positions(t, w, pos);
                __syncwarp();
                subtile_gather(t, pos, v);
            }
            if (j == K - 1) {   // the stage's last reads are done
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&P.empty[s]);
            }

            if (a.delta) {
                uint32_t run = 0;   // this sub-tile's gaps so far
#pragma unroll
                for (int r = 0; r < kSubRounds; r++) {
                    v[r][1] += v[r][0];
                    v[r][2] += v[r][1];
                    v[r][3] += v[r][2];
                    const uint32_t qs = v[r][3];
                    const uint32_t inc = warp_incl_scan(qs);
                    const uint32_t add = run + inc - qs;
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        v[r][i] += add;
                    run += __shfl_sync(0xffffffffu, inc, 31);
                }
                uint32_t *sums = s_sum[ex++ & 1];   // double-buffered: the next group's
                if (lane == 0)                      // barrier orders these reads before
                    sums[warp] = run;               // the reuse
                named_sync(1, kThreads);
                uint32_t before = carry, all = 0;
#pragma unroll
                for (int i = 0; i < kWarps; i++) {
                    const uint32_t x = sums[i];
                    before += i < warp ? x : 0u;
                    all += x;
                }
                carry += all;
#pragma unroll
                for (int r = 0; r < kSubRounds; r++)
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        v[r][i] += before;
            }
            if (!have)
                continue;
            uint32_t *base = a.out + out_off + 4 * (u64)q0;
            if (t.full()) {
                store_full_subtile(base, v);
                continue;
            }
            uint32_t *op = base + 4 * lane;
            const uint32_t m = (uint32_t)((uintptr_t)base >> 2) & 3u;
#pragma unroll
            for (int r = 0; r < kSubRounds; r++) {
                // Most lists start at an integer that is not 16-byte aligned: a
                // whole round of 32 quads still goes out in 16-byte writes.
                if (!aligned && subtile_nints(t, 32u * r + 31u) == 4u) {
                    stg_round_realigned(base + 128 * r,
                                        make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]), m);
                    continue;
                }
                const uint32_t lq = r * 32 + lane;
                const uint32_t nints = subtile_nints(t, lq);
                if (!nints)
                    continue;
                uint32_t *dst = op + 128 * r;
                if (nints == 4 && aligned) {
                    stg_stream128(dst, make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]));
                } else {
                    dst[0] = v[r][0];
                    if (nints > 1)
                        dst[1] = v[r][1];
                    if (nints > 2)
                        dst[2] = v[r][2];
                    if (nints > 3)
                        dst[3] = v[r][3];
                }
            }
        }
    }
}

// Data bytes of a sub-tile from its control word w (every lane): four quads
// per lane (Sec. 4: a control byte covers 4 + the sum of its codes bytes;
// the pad fields of the last quad cover none).
__device__ __forceinline__ uint32_t subtile_bytes(const SubTile &t, uint32_t w)
{
    const int lane = threadIdx.x & 31;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t nints = subtile_nints(t, 4u * lane + j);
        uint32_t b = (w >> (8 * j)) & 0xffu;
        if (nints < 4)
            b &= (1u << (2 * nints)) - 1u;
        c += nints ? quad_count(b, nints) : 0u;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        c += __shfl_xor_sync(0xffffffffu, c, d);
    return c;
}

// Shared memory one warp uses for a small list: a staged sub-tile's data
// bytes (16-byte phase, 2048 bytes, round-up and read slack) and its quad
// positions.
constexpr int kSmallData = 16 * kSubQuads + 48;
constexpr int kSmallSlot = kSmallData + 2 * kSubQuads;

// One small list, decoded by one warp, 128 quads (512 integers) at a time:
// the piece's data bytes are staged into the warp's slot by cp.async (bytes
// of the list's stream only), decoded with the sub-tile code and stored
// with 16-byte writes (realigned where the list starts off a 16-byte
// boundary); differential lists keep a running carry.
__device__ void bdec_small(const BatchDecArgs &a, uint32_t li, int lane, uint8_t *slot)
{
    const svb_list L = a.lists[li];
    const uint32_t n = L.n, nq = (n + 3) / 4;
    const uint8_t *base = a.in + L.in_off;
    if (nq > L.in_len) {
        if (lane == 0)
            raise_error(a.hdr, kErrTruncated);
        return;
    }
    const uint8_t *data = base + nq;
    const u64 dcap = L.in_len - nq;  // data bytes the stream may use
    const uintptr_t lo = (uintptr_t)base, hi = (uintptr_t)(base + L.in_len);
    const uint32_t last_nints = n - 4 * (nq - 1);
    uint32_t *out = a.out + L.out_off;
    const bool aligned = ((uintptr_t)out & 15u) == 0;
    const uint32_t m = (uint32_t)((uintptr_t)out >> 2) & 3u;
    const uint64_t policy = l2_policy_evict_first();
    uint16_t *pos = reinterpret_cast<uint16_t *>(slot + kSmallData);
    u64 running = 0;
    uint32_t carry = L.prev;
    for (uint32_t q0 = 0; q0 < nq; q0 += kSubQuads) {
        SubTile t;
        t.C = base + q0;   // read in place (global memory)
        t.D = slot;
        t.nq = min((uint32_t)kSubQuads, nq - q0);
        t.tail = q0 + t.nq == nq ? last_nints : 4u;
        const uint32_t w = subtile_ctrl_word(t);
        const uint32_t total = subtile_bytes(t, w);
        if (running + total > dcap) {
            if (lane == 0)
                raise_error(a.hdr, kErrTruncated);
            return;
        }
        const uint8_t *g = data + running;
        t.base = (uint32_t)((uintptr_t)g & 15u);
        warp_stage(g, total, slot, lo, hi, policy);
        cp_async_commit();
        subtile_positions(t, w, pos);
        cp_async_wait<0>();
        __syncwarp();
        uint32_t v[kSubRounds][4];
        subtile_gather(t, pos, v);
        if (a.delta) {
#pragma unroll
            for (int r = 0; r < kSubRounds; r++) {
                v[r][1] += v[r][0];
                v[r][2] += v[r][1];
                v[r][3] += v[r][2];
                const uint32_t qs = v[r][3];
                const uint32_t inc = warp_incl_scan(qs);
                const uint32_t add = carry + inc - qs;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    v[r][j] += add;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        __syncwarp();  // the slot and pos are read before the next piece is staged
        uint32_t *op = out + 4 * q0;
        if (t.full()) {
            store_full_subtile(op, v);
            running += total;
            continue;
        }
#pragma unroll
        for (int r = 0; r < kSubRounds; r++) {
            const bool whole = subtile_nints(t, 32u * r + 31u) == 4u;
            const uint4 x = make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]);
            if (whole && aligned) {
                stg_stream128(op + 128 * r + 4 * lane, x);
            } else if (whole) {
                stg_round_realigned(op + 128 * r, x, m);
            } else {
                const uint32_t nints = subtile_nints(t, 32u * r + lane);
                uint32_t *dst = op + 128 * r + 4 * lane;
                if (nints > 0)
                    dst[0] = x.x;
                if (nints > 1)
                    dst[1] = x.y;
                if (nints > 2)
                    dst[2] = x.z;
                if (nints > 3)
                    dst[3] = x.w;
            }
        }
        running += total;
    }
    if (lane == 0)
        atomicAdd(&a.hdr->total, (u64)nq + running);
}

// ---------------------------------------------------------------------------
// Units of split lists: each one's data offset and carry-in within its list.
//
// One CTA per unit at a time, units claimed in order (a list's units are
// consecutive), so every earlier unit of the list belongs to a CTA that is
// running or done.  For unit u of list L:
//   A  each sub-tile's data bytes from its control bytes (Sec. 4), scanned
//      into offsets within the unit, and the unit's total B_u;
//   B  d0 = the data bytes of L's earlier units: B_u is published and the
//      prefix found by a look-back over L's units (prefix 0 at unit 0);
//   C  each sub-tile's gap sum: a full sub-tile with 512 data bytes has only
//      zero codes, so its sum is a byte sum (read straight from memory, in
//      coalesced byte loads); any other sub-tile is staged and decoded;
//   D  c0 = L.prev plus the gaps of L's earlier units, by a second
//      look-back; d0 and c0 go into the unit for the decode launch.
// The list's last unit skips A and C and publishes nothing: no later unit
// reads its totals, so it only looks back for d0 and c0.
// A list whose stream is cut short publishes zeros (the decode reports it).

constexpr int kBPrepCtrl = 144;                      // 15-byte phase + 128 control bytes
constexpr int kBPrepData = 16 * kSubQuads + 48;      // phase + 2048 + read slack
constexpr uint32_t kMaxSegTiles = 32;   // the most 4096-integer tiles a unit may span
constexpr u64 kPrepSpins = 1ull << 22;

struct BatchPrepArgs {
    const svb_list *lists;
    const PlanHeader *plan;
    const uint8_t *in;
    WsHeader *hdr;
};

__global__ void __launch_bounds__(kThreads) batch_prep_kernel(BatchPrepArgs a)
{
    __shared__ uint32_t s_off[kMaxSegTiles * kBSubs + 1];
    __shared__ uint32_t s_gap[kMaxSegTiles * kBSubs];
    __shared__ __align__(16) uint8_t s_slot[kWarps][2][kBPrepCtrl + kBPrepData];
    __shared__ __align__(16) uint16_t s_pos[kWarps][kSubQuads];
    __shared__ u64 s_unit, s_d0;
    __shared__ uint32_t s_bad, s_last;

    const uint32_t nsplit = plan_nsplit(a.plan);
    if (nsplit == 0)
        return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u64 etag = epoch_tag(a.hdr);
    PlanUnit *units = plan_units(a.plan);
    TileStatus *recs = plan_recs(a.plan);
    const uint32_t tq = a.plan->tile_quads;   // the plan's tile: units count these
    const bool tq_ok = tq == (uint32_t)kBQuads || tq == 2u * kBQuads;
    if (!tq_ok && tid == 0)
        raise_error(a.hdr, kErrInvalid);
    const uint64_t keep = l2_policy_evict_last();
    while (tq_ok) {
        __syncthreads();
        if (tid == 0)
            s_unit = atomicAdd(&a.hdr->a_counter, 1ull);
        __syncthreads();
        const u64 u = s_unit;
        if (u >= nsplit)
            break;
        const PlanUnit U = units[u];
        const svb_list L = a.lists[U.list];
        const uint32_t nql = (L.n + 3) / 4;
        const uint32_t last_nints = L.n - 4 * (nql - 1);
        const uint8_t *lo = a.in + L.in_off;
        const uint8_t *hi = lo + L.in_len;
        const uint8_t *data = lo + nql;
        const uint32_t qb0 = U.t0 * tq;
        const uint32_t qe = min((U.t0 + U.nt) * tq, nql);
        const uint32_t ns = (qe - qb0 + kSubQuads - 1) / kSubQuads;
        const bool ctrl_ok = (u64)nql <= L.in_len;
        // The list's last unit: no later unit reads its totals, so only its
        // data offset and carry-in (the two look-backs) are found; a stream
        // cut short inside it is reported by the decode.
        const bool last = U.t0 + U.nt >= (nql + tq - 1) / tq;
        // A: data bytes of each sub-tile (byte loads, coalesced across the warp).
        for (uint32_t j = warp; !last && j < ns; j += kWarps) {
            const uint32_t qb = qb0 + j * kSubQuads;
            uint32_t t = 0;
            if (ctrl_ok) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t q = qb + 32 * k + lane;
                    if (q < qe && q < qb + kSubQuads) {
                        uint32_t c = __ldg(lo + q);
                        const uint32_t nints = q == nql - 1 ? last_nints : 4u;
                        if (nints < 4)
                            c &= (1u << (2 * nints)) - 1u;
                        t += quad_count(c, nints);
                    }
                }
            }
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1)
                t += __shfl_xor_sync(0xffffffffu, t, d);
            if (lane == 0)
                s_off[j] = t;
        }
        __syncthreads();
        // B: offsets within the unit (warp 0 scans), then the unit's data offset.
        if (warp == 0) {
            const uint32_t per = last ? 0u : (ns + 31) / 32;
            const uint32_t b = min(lane * per, ns), e = min(b + per, ns);
            uint32_t tot = 0;
            for (uint32_t i = b; i < e; i++)
                tot += s_off[i];
            const uint32_t inc = warp_incl_scan(tot);
            uint32_t c = inc - tot;
            for (uint32_t i = b; i < e; i++) {
                const uint32_t v = s_off[i];
                s_off[i] = c;
                c += v;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);   // 0 for the last unit
            if (lane == 0)
                s_off[ns] = total;
            TileStatus *me = &recs[U.first + U.seg];
            u64 d0 = 0;
            bool ok = true;
            if (U.seg == 0) {
                if (lane == 0 && !last)
                    publish(&me->off_tag, &me->off_pre, total, kFlagPrefix, etag);
            } else {
                if (lane == 0 && !last)
                    publish(&me->off_tag, &me->off_agg, total, kFlagAgg, etag);
                d0 = lookback<false>(recs + U.first, U.seg, etag, kPrepSpins, a.hdr, ok);
                if (lane == 0 && !last)
                    publish(&me->off_tag, &me->off_pre, d0 + total, kFlagPrefix, etag);
            }
            if (lane == 0) {
                if (!ok)
                    raise_error(a.hdr, kErrTimeout);
                s_d0 = d0;
                s_bad = (!ok || !ctrl_ok || (u64)nql + d0 + total > L.in_len) ? 1u : 0u;
            }
        }
        __syncthreads();
        const u64 d0 = s_d0;
        const bool bad = s_bad != 0;
        // C: each sub-tile's gap sum; a warp stages its next sub-tile while it
        // sums the current one.
        uint16_t *pos = s_pos[warp];
        const uintptr_t blo = (uintptr_t)lo, bhi = (uintptr_t)hi;
        auto geom = [&](uint32_t j, uint32_t &qb, uint32_t &nq, u64 &start, uint32_t &len) {
            qb = qb0 + j * kSubQuads;
            nq = min((uint32_t)kSubQuads, qe - qb);
            start = d0 + s_off[j];
            len = s_off[j + 1] - s_off[j];
            const bool full = nq == (uint32_t)kSubQuads && !(qb + nq == nql && last_nints < 4);
            return full && len == 4u * kSubQuads;   // every code zero: a byte sum
        };
        auto stage = [&](uint32_t j, uint8_t *slot) {
            if (bad || last || j >= ns)
                return;
            uint32_t qb, nq, len;
            u64 start;
            if (geom(j, qb, nq, start, len))
                return;
            warp_stage(lo + qb, nq, slot, blo, bhi, keep);
            warp_stage(data + start, len, slot + kBPrepCtrl, blo, bhi, keep);
        };
        stage(warp, s_slot[warp][0]);
        cp_async_commit();
        uint32_t k = 0;
        for (uint32_t j = warp; !last && j < ns; j += kWarps, k++) {
            stage(j + kWarps, s_slot[warp][(k + 1) & 1]);
            cp_async_commit();
            cp_async_wait<1>();   // sub-tile j's copies have landed
            __syncwarp();
            uint32_t sum = 0;
            if (!bad) {
                uint32_t qb, nq, len;
                u64 start;
                if (geom(j, qb, nq, start, len)) {
#pragma unroll
                    for (int i = 0; i < 16; i++)
                        sum += __ldg(data + start + lane + 32 * i);
                } else {
                    const uint8_t *slot = s_slot[warp][k & 1];
                    SubTile t;
                    t.C = slot + ((uintptr_t)(lo + qb) & 15u);
                    t.D = slot + kBPrepCtrl;
                    t.base = (uint32_t)((uintptr_t)(data + start) & 15u);
                    t.nq = nq;
                    t.tail = qb + nq == nql ? last_nints : 4u;
                    const uint32_t w = subtile_ctrl_word(t);
                    subtile_positions(t, w, pos);
                    __syncwarp();
                    uint32_t v[kSubRounds][4];
                    subtile_gather(t, pos, v);
#pragma unroll
                    for (int r = 0; r < kSubRounds; r++)
                        sum += v[r][0] + v[r][1] + v[r][2] + v[r][3];
                }
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1)
                    sum += __shfl_xor_sync(0xffffffffu, sum, d);
            }
            __syncwarp();  // the slot and pos are read before they are refilled
            if (lane == 0)
                s_gap[j] = sum;
        }
        cp_async_wait<0>();
        __syncthreads();
        // D: the unit's carry-in.
        if (warp == 0) {
            uint32_t g = 0;
            for (uint32_t i = lane; !last && i < ns; i += 32)
                g += s_gap[i];
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1)
                g += __shfl_xor_sync(0xffffffffu, g, d);
            TileStatus *me = &recs[U.first + U.seg];
            u64 c0 = L.prev;
            bool ok = true;
            if (U.seg == 0) {
                if (lane == 0 && !last)
                    publish(&me->val_tag, &me->val_pre, (uint32_t)(L.prev + g), kFlagPrefix, etag);
            } else {
                if (lane == 0 && !last)
                    publish(&me->val_tag, &me->val_agg, g, kFlagAgg, etag);
                c0 = lookback<true>(recs + U.first, U.seg, etag, kPrepSpins, a.hdr, ok);
                if (lane == 0 && !last)
                    publish(&me->val_tag, &me->val_pre, (uint32_t)(c0 + g), kFlagPrefix, etag);
            }
            if (lane == 0) {
                if (!ok)
                    raise_error(a.hdr, kErrTimeout);
                units[u].d0 = d0;
                units[u].c0 = (uint32_t)c0;
            }
        }
    }
    // The last CTA readies the claim counters for the decode launch.
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&a.hdr->a_done, 1ull) == (u64)gridDim.x - 1 ? 1u : 0u;
        if (s_last) {
            st_relaxed(&a.hdr->a_counter, 0);
            st_relaxed(&a.hdr->a_done, 0);
        }
    }
}

template <int S, int K, int kMinCtas>
__global__ void __launch_bounds__(kBBlock, kMinCtas) batch_decode_kernel(BatchDecArgs a)
{
    constexpr int kCRing = BPipe<S, K>::kCRing;
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    BPipe<S, K> &P = *reinterpret_cast<BPipe<S, K> *>(dyn_smem);
    __shared__ __align__(16) uint16_t s_pos[kBQuads];   // each warp's quad positions
    __shared__ uint32_t s_sum[2][kWarps];                // sub-tile gap sums, per tile parity

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // A plan made for another tile size: its units do not match this
    // kernel's tiles, so nothing is decoded (every CTA sees the same).
    if (a.plan->tile_quads != (uint32_t)BPipe<S, K>::kTQ) {
        if (tid == 0)
            raise_error(a.hdr, kErrInvalid);
        finish_launch(a.hdr, a.result);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&P.full[s], 32);
            mbar_init(&P.empty[s], kWarps);
        }
        for (int r = 0; r < kCRing; r++)
            mbar_init(&P.cfull[r], 32);
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == kWarps)
        bdec_produce<S, K>(a, P, lane);
    else
        bdec_consume<S, K>(a, P, s_pos, s_sum);

    // Small lists: every warp takes them one by one, staging their pieces in
    // a slot of its own carved from the data stages, which the big-list
    // phase no longer uses once every warp is past it.
    static_assert((kBBlock / 32) * kSmallSlot <= (int)sizeof(P.data), "small-list slots fit");
    __syncthreads();
    uint8_t *slot = &P.data[0][0] + warp * kSmallSlot;
    const uint32_t *small = plan_small(a.plan);
    const uint32_t nsmall = a.plan->nsmall;
    for (;;) {
        uint32_t j = 0;
        if (lane == 0)
            j = (uint32_t)atomicAdd(&a.hdr->a_counter, 1ull);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= nsmall)
            break;
        bdec_small(a, small[j], lane, slot);
    }
    finish_launch(a.hdr, a.result);
}

// ---------------------------------------------------------------------------
// Encode

struct BatchEncArgs {
    const svb_list *lists;
    const PlanHeader *plan;
    const uint32_t *in;
    uint8_t *out;
    u64 *sizes;
    WsHeader *hdr;
    DeviceResult *result;
    uint32_t delta;
};

constexpr int kEStageBytes = 16 * kBQuads + 16;  // 4096 values + 16-byte phase

// Staging depth S of the encode kernel, a compile-time parameter like the
// decode kernel's.
template <int S>
struct EPipe {
    uint8_t vals[S][kEStageBytes];
    uint32_t slice[kWarps][kEncSliceWords];   // each warp's data bytes, phased like the output
    uint64_t full[S];
    uint64_t empty[S];
    uint32_t list[S];
    uint32_t tile[S];
    uint32_t hv[S];  // phase (mod 16) of the staged values
    u64 out_off[S];  // the tile's list: where its stream goes,
    uint32_t n[S], prev[S];   // its integers and start value
};

template <int S>
__device__ void benc_produce(const BatchEncArgs &a, EPipe<S> &P, int lane)
{
    const PlanHeader *plan = a.plan;
    const uint32_t *big = plan_big(plan);
    uint32_t issued = 0, li = kNoList, k = 0, ntl = 0;
    svb_list L = {};
    auto claim = [&]() -> bool {
        uint32_t j = 0;
        if (lane == 0)
            j = (uint32_t)atomicAdd(&a.hdr->tile_counter, 1ull);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= plan->nbig)
            return false;
        li = big[j];
        L = a.lists[li];
        ntl = (L.n + 4 * kBQuads - 1) / (4 * kBQuads);
        k = 0;
        return true;
    };
    bool have = claim();
    for (uint32_t g = 0;; g++) {
        const int s = g % S;
        if (g >= (uint32_t)S) {
            bool ok = mbar_wait_bounded(&P.empty[s], ((g / S) - 1) & 1u, kBPolls);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0)
                    raise_error(a.hdr, kErrTimeout);
                issued = g;
                break;
            }
        }
        if (!have) {
            if (lane == 0) {
                P.list[s] = kNoList;
                mbar_arrive_expect_tx(&P.full[s], 0);
            } else {
                mbar_arrive(&P.full[s]);
            }
            issued = g + 1;
            break;
        }
        const u64 i0 = (u64)k * 4 * kBQuads;
        const uint32_t cnt = (uint32_t)min((u64)4 * kBQuads, (u64)L.n - i0);
        const uint8_t *lo = reinterpret_cast<const uint8_t *>(a.in + L.in_off);
        const uint8_t *gv = lo + 4 * i0;
        const StagePlan pv = stage_plan(gv, 4 * cnt, lo, lo + 4 * (u64)L.n);
        if (pv.edges)
            range_edges(gv, 4 * cnt, P.vals[s], lane);
        if (lane == 0) {
            P.list[s] = li;
            P.tile[s] = k;
            P.hv[s] = (uint32_t)((uintptr_t)gv & 15u);
            P.out_off[s] = L.out_off;
            P.n[s] = L.n;
            P.prev[s] = L.prev;
            mbar_arrive_expect_tx(&P.full[s], pv.bytes);
            if (pv.bytes)
                bulk_g2s(P.vals[s] + pv.dst_off, pv.src, pv.bytes, &P.full[s]);
        } else {
            mbar_arrive(&P.full[s]);
        }
        if (++k == ntl)
            have = claim();
        issued = g + 1;
    }
    if (lane == 0) {
        for (int s = 0; s < S; s++)
            if (issued > (uint32_t)s) {
                uint32_t fills = (issued - 1 - s) / S + 1;
                mbar_wait_bounded(&P.full[s], (fills - 1) & 1u, kBPolls);
            }
    }
    __syncwarp();
}

// Consumer warps of the big-list phase: warp w encodes sub-tile w of every
// tile with the same per-warp code as the single-stream encoder.  A list's
// tiles come in order to one CTA, so its data offset is a running sum: the
// eight warps trade their sub-tile sizes once per tile (one barrier) and each
// keeps the running offset and the list's last integer itself.
template <int S>
__device__ void benc_consume(const BatchEncArgs &a, EPipe<S> &P, uint32_t (*s_size)[kWarps])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t sq0 = warp * kSubQuads;
    u64 run = 0;          // data bytes of the current list written so far
    uint32_t before = 0;  // the list's integer before the current tile (differential)
    for (uint32_t g = 0;; g++) {
        const int s = g % S;
        if (!mbar_wait_bounded(&P.full[s], (g / S) & 1u, kBPolls)) {
            raise_error(a.hdr, kErrTimeout);
            break;
        }
        const uint32_t li = P.list[s];
        if (li == kNoList)
            break;
        const uint32_t n = P.n[s], k = P.tile[s];
        const u64 out_off = P.out_off[s];
        const uint32_t nql = (n + 3) / 4;
        const uint32_t last_nints = n - 4 * (nql - 1);
        const uint32_t q0 = k * kBQuads;
        const uint32_t nq = min((uint32_t)kBQuads, nql - q0);
        const uint32_t cnt = min((uint32_t)(4 * kBQuads), n - 4 * q0);   // values in the tile
        if (k == 0) {
            run = 0;
            before = P.prev[s];
        }
        const uint32_t *V = reinterpret_cast<const uint32_t *>(P.vals[s] + P.hv[s]);
        const uint32_t nvq = nq > sq0 ? min(nq - sq0, (uint32_t)kSubQuads) : 0u;
        const uint32_t tail = q0 + nq == nql ? last_nints : 4u;
        const bool fast = 4 * (sq0 + kSubQuads) <= cnt;   // a whole sub-tile
        uint32_t nints[kEncRounds], d[kEncRounds][4], ctrl[kEncRounds], cb[kEncRounds];
        auto prior = [&]() { return before; };
        if (fast && P.hv[s] == 0)
            subenc_load<true>(V, sq0, nq, tail, a.delta != 0, prior, nints, d, ctrl, cb);
        else if (fast)   // the list's values start 4, 8 or 12 bytes past a 16-byte boundary
            subenc_load<true, decltype(prior), false, false>(V, sq0, nq, tail, a.delta != 0, prior,
                                                            nints, d, ctrl, cb);
        else
            subenc_load<false>(V, sq0, nq, tail, a.delta != 0, prior, nints, d, ctrl, cb);
        const uint32_t tile_last = V[cnt - 1];
        // The control bytes use every staged value this warp loaded.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.empty[s]);

        const uint32_t mine = subenc_bytes(cb);
        uint32_t *sizes = s_size[g & 1];   // double-buffered: the next tile's barrier
        if (lane == 0)                     // orders these reads before the reuse
            sizes[warp] = mine;
        named_sync(1, kThreads);
        uint32_t pre = 0, all = 0;
#pragma unroll
        for (int j = 0; j < kWarps; j++) {
            const uint32_t x = sizes[j];
            pre += j < warp ? x : 0u;
            all += x;
        }
        uint8_t *stream = a.out + out_off;
        if (nvq) {
            uint8_t *cdst = stream + q0 + sq0, *ddst = stream + nql + run + pre;
            if (fast)
                subenc_write<true>(P.slice[warp], cdst, ddst, nvq, nints, ctrl, cb, d);
            else
                subenc_write<false>(P.slice[warp], cdst, ddst, nvq, nints, ctrl, cb, d);
        }
        run += all;
        before = tile_last;
        if (q0 + nq == nql && warp == 0 && lane == 0) {
            a.sizes[li] = nql + run;
            atomicAdd(&a.hdr->total, (u64)nql + run);
        }
    }
}

// One small list, encoded by one warp straight from global memory.
__device__ void benc_small(const BatchEncArgs &a, uint32_t li, int lane)
{
    const svb_list L = a.lists[li];
    const uint32_t n = L.n, nq = (n + 3) / 4;
    const uint32_t *src = a.in + L.in_off;
    uint8_t *ctrl = a.out + L.out_off;
    uint8_t *data = ctrl + nq;
    u64 running = 0;
    uint32_t before = L.prev;
    for (uint32_t q0 = 0; q0 < nq; q0 += 32) {
        const uint32_t q = q0 + lane;
        const uint32_t nints = q >= nq ? 0u : (q == nq - 1 ? n - 4 * q : 4u);
        uint32_t x[4] = {0, 0, 0, 0}, d[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            if ((uint32_t)j < nints)
                x[j] = __ldg(src + 4 * q + j);
        if (a.delta) {
            uint32_t pv = __shfl_up_sync(0xffffffffu, x[3], 1);
            if (lane == 0)
                pv = before;
            d[0] = x[0] - pv;
            d[1] = x[1] - x[0];
            d[2] = x[2] - x[1];
            d[3] = x[3] - x[2];
            before = __shfl_sync(0xffffffffu, x[3], 31);
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                d[j] = x[j];
        }
        uint32_t c = 0, C = 0;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if ((uint32_t)j < nints) {
                const uint32_t Lb = byte_len(d[j]);
                c |= (Lb - 1) << (2 * j);
                C += Lb;
            }
        if (nints)
            ctrl[q] = (uint8_t)c;
        const uint32_t incl = warp_incl_scan(C);
        uint8_t *p = data + running + (incl - C);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if ((uint32_t)j < nints) {
                const uint32_t code = (c >> (2 * j)) & 3u;
#pragma unroll
                for (uint32_t b = 0; b < 4; b++)
                    if (b <= code)
                        p[b] = (uint8_t)(d[j] >> (8 * b));
                p += code + 1;
            }
        }
        running += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        a.sizes[li] = nq + running;
        atomicAdd(&a.hdr->total, (u64)nq + running);
    }
}

template <int S, int kMinCtas>
__global__ void __launch_bounds__(kBBlock, kMinCtas) batch_encode_kernel(BatchEncArgs a)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    EPipe<S> &P = *reinterpret_cast<EPipe<S> *>(dyn_smem);
    __shared__ uint32_t s_size[2][kWarps];   // sub-tile data bytes, per tile parity

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&P.full[s], 32);
            mbar_init(&P.empty[s], kWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == kWarps)
        benc_produce<S>(a, P, lane);
    else
        benc_consume<S>(a, P, s_size);

    const uint32_t *small = plan_small(a.plan);
    const uint32_t nsmall = a.plan->nsmall;
    for (;;) {
        uint32_t j = 0;
        if (lane == 0)
            j = (uint32_t)atomicAdd(&a.hdr->a_counter, 1ull);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= nsmall)
            break;
        benc_small(a, small[j], lane);
    }
    finish_launch(a.hdr, a.result);
}

// ---------------------------------------------------------------------------

template <class K>
static int persistent_grid(K kernel, size_t smem)
{
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kBBlock, smem);
    return (sms > 0 ? sms : 148) * (occ > 0 ? occ : 1);
}

// Staging depths and decode tile sizes the batched kernels are built with,
// and the ones in use (0: the default; set by svb_batch_set_stages and
// svb_batch_set_tile).  Decoding is built for tiles of 4096 integers at
// depths 2, 3 and 4, and for tiles of 8192 at depths 1 and 2.
static std::atomic<int> g_dec_stages{0}, g_enc_stages{0}, g_dec_tile{0};
constexpr int kDecStagesDefault = 2, kEncStagesDefault = 3;
constexpr int kTileIntsDefault = 4 * kBQuads;

int batch_set_stages(int decode_stages, int encode_stages)
{
    const bool dec_ok = decode_stages == 0 || (decode_stages >= 1 && decode_stages <= 4);
    const bool enc_ok = encode_stages == 0 || encode_stages == 2 || encode_stages == 3;
    if (!dec_ok || !enc_ok)
        return 1;
    g_dec_stages.store(decode_stages, std::memory_order_relaxed);
    g_enc_stages.store(encode_stages, std::memory_order_relaxed);
    return 0;
}

int batch_stages(int encode)
{
    const int v = (encode ? g_enc_stages : g_dec_stages).load(std::memory_order_relaxed);
    return v ? v : (encode ? kEncStagesDefault : kDecStagesDefault);
}

int batch_set_tile(int tile_ints)
{
    if (tile_ints != 0 && tile_ints != 4 * kBQuads && tile_ints != 8 * kBQuads)
        return 1;
    g_dec_tile.store(tile_ints, std::memory_order_relaxed);
    return 0;
}

int batch_tile(void)
{
    const int v = g_dec_tile.load(std::memory_order_relaxed);
    return v ? v : kTileIntsDefault;
}

// One instantiation of the decode kernel: S stages, at least kMinCtas CTAs
// per SM (the register cap that lets that many fit).
template <int S, int K, int kMinCtas>
static void launch_bdec(const BatchDecArgs &a, int grid, cudaStream_t stream)
{
    static int g = 0;
    if (!g)
        g = persistent_grid(batch_decode_kernel<S, K, kMinCtas>, sizeof(BPipe<S, K>));
    prof_begin("batch_decode_kernel", stream);
    batch_decode_kernel<S, K, kMinCtas>
        <<<grid > 0 ? grid : g, kBBlock, sizeof(BPipe<S, K>), stream>>>(a);
    prof_end(stream);
}

template <int S, int kMinCtas>
static void launch_benc(const BatchEncArgs &a, int grid, cudaStream_t stream)
{
    static int g = 0;
    if (!g)
        g = persistent_grid(batch_encode_kernel<S, kMinCtas>, sizeof(EPipe<S>));
    prof_begin("batch_encode_kernel", stream);
    batch_encode_kernel<S, kMinCtas>
        <<<grid > 0 ? grid : g, kBBlock, sizeof(EPipe<S>), stream>>>(a);
    prof_end(stream);
}

int launch_batch_decode(const void *d_plan, const svb_list *d_lists, const uint8_t *in,
                        uint32_t *out, bool delta, void *ws, DeviceResult *result,
                        cudaStream_t stream, int grid)
{
    // The instantiation for the tile and depth in use; a pair that is not
    // built is refused before anything is enqueued.
    const int tile = batch_tile(), stages = batch_stages(0);
    const bool built = tile == 4 * kBQuads ? stages >= 2 && stages <= 4 : stages <= 2;
    if (!built)
        return 1;
    BatchDecArgs a;
    a.lists = d_lists;
    a.plan = static_cast<const PlanHeader *>(d_plan);
    a.in = in;
    a.out = out;
    a.hdr = static_cast<WsHeader *>(ws);
    a.result = result;
    a.delta = delta ? 1u : 0u;
    // Units of split lists first: their data offsets and carry-ins (a
    // launch that returns at once when the plan has none).
    static int pg = 0;
    if (!pg) {
        int occ = 0, sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_prep_kernel, kThreads, 0);
        pg = (sms > 0 ? sms : 148) * (occ > 0 ? occ : 1);
    }
    BatchPrepArgs pa;
    pa.lists = d_lists;
    pa.plan = a.plan;
    pa.in = in;
    pa.hdr = a.hdr;
    prof_begin("batch_prep_kernel", stream);
    batch_prep_kernel<<<pg, kThreads, 0, stream>>>(pa);
    prof_end(stream);
    if (tile == 8 * kBQuads) {
        if (stages == 1)
            launch_bdec<1, 2, 4>(a, grid, stream);
        else
            launch_bdec<2, 2, 2>(a, grid, stream);
    } else if (stages == 4) {
        launch_bdec<4, 1, 3>(a, grid, stream);
    } else if (stages == 3) {
        launch_bdec<3, 1, 4>(a, grid, stream);
    } else {
        launch_bdec<2, 1, 4>(a, grid, stream);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_batch_encode(const void *d_plan, const svb_list *d_lists, const uint32_t *in,
                        uint8_t *out, u64 *sizes, bool delta, void *ws, DeviceResult *result,
                        cudaStream_t stream, int grid)
{
    BatchEncArgs a;
    a.lists = d_lists;
    a.plan = static_cast<const PlanHeader *>(d_plan);
    a.in = in;
    a.out = out;
    a.sizes = sizes;
    a.hdr = static_cast<WsHeader *>(ws);
    a.result = result;
    a.delta = delta ? 1u : 0u;
    if (batch_stages(1) == 2)
        launch_benc<2, 4>(a, grid, stream);
    else
        launch_benc<3, 3>(a, grid, stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

uint32_t batch_default_seg_tiles()
{
    return kSegTiles;
}

size_t batch_plan_bytes(size_t num_lists)
{
    const size_t units = num_lists + kExtraUnits;
    return plan_recs_off(num_lists, units) + sizeof(TileStatus) * units;
}

int build_batch_plan(const svb_list *h_lists, size_t num_lists, uint32_t threshold,
                     uint32_t seg_tiles, void *d_plan, cudaStream_t stream)
{
    if (threshold == 0)
        threshold = kDefaultBigThreshold;
    // The plan is made for the decode tile in use: tq quads, units of
    // seg_tiles such tiles (at most kMaxSegTiles tiles of 4096 integers).
    const uint32_t tq = (uint32_t)batch_tile() / 4;
    if ((u64)seg_tiles * tq > (u64)kMaxSegTiles * kBQuads)
        return 1;
    std::vector<uint32_t> big, small;
    for (size_t j = 0; j < num_lists; j++) {
        if (h_lists[j].n == 0)
            continue;
        (h_lists[j].n >= threshold ? big : small).push_back((uint32_t)j);
    }
    // Longest first, so that the last lists handed out are the shortest.
    auto longer = [&](uint32_t x, uint32_t y) {
        return h_lists[x].n != h_lists[y].n ? h_lists[x].n > h_lists[y].n : x < y;
    };
    std::sort(big.begin(), big.end(), longer);
    std::sort(small.begin(), small.end(), longer);
    // Units: a big list longer than a quarter of a CTA's fair share of the
    // big lists' tiles (and than 2 * seg_tiles tiles) is cut into units of seg_tiles
    // tiles, while the plan's unit budget lasts: splitting costs a pass over
    // the list's stream, which pays only when one CTA would otherwise be left
    // decoding it alone at the end.  The split lists' units come first, then
    // one unit per other big list.
    u64 big_tiles = 0;
    for (uint32_t li : big)
        big_tiles += (((u64)h_lists[li].n + 3) / 4 + tq - 1) / tq;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const u64 ctas = 3 * (u64)(sms > 0 ? sms : 148);
    const u64 fair = (big_tiles + ctas - 1) / ctas;
    std::vector<PlanUnit> split, whole;
    const size_t budget = num_lists + kExtraUnits;
    for (uint32_t li : big) {
        const uint32_t nql = (uint32_t)(((u64)h_lists[li].n + 3) / 4);
        const uint32_t ntl = (nql + tq - 1) / tq;
        const uint32_t nseg = seg_tiles ? (ntl + seg_tiles - 1) / seg_tiles : 1u;
        if (seg_tiles && ntl > 2 * seg_tiles && 4 * (u64)ntl > fair &&
            split.size() + nseg + (big.size() - 1) <= budget) {
            const uint32_t first = (uint32_t)split.size();
            for (uint32_t k = 0; k < nseg; k++)
                split.push_back(PlanUnit{li, k * seg_tiles, std::min(seg_tiles, ntl - k * seg_tiles),
                                         k, 0, 0, first});
        } else {
            whole.push_back(PlanUnit{li, 0, ntl, 0, 0, 0, 0});
        }
    }
    const size_t ids = big.size() + small.size();
    const size_t nunits = split.empty() ? 0 : split.size() + whole.size();
    const size_t bytes = nunits ? plan_recs_off(ids, nunits) + sizeof(TileStatus) * nunits
                                : sizeof(PlanHeader) + 4 * ids;
    std::vector<uint8_t> buf(bytes, 0);
    PlanHeader h = {};
    h.nbig = (uint32_t)big.size();
    h.nsmall = (uint32_t)small.size();
    h.threshold = threshold;
    h.nunits = (uint32_t)nunits;
    h.tile_quads = tq;
    std::copy_n(reinterpret_cast<const uint8_t *>(&h), sizeof(h), buf.data());
    uint32_t *w = reinterpret_cast<uint32_t *>(buf.data() + sizeof(PlanHeader));
    std::copy(big.begin(), big.end(), w);
    std::copy(small.begin(), small.end(), w + big.size());
    if (nunits) {
        // Units header (nsplit), the units, then zeroed records: a zero tag
        // never matches a launch's tag.
        *reinterpret_cast<uint32_t *>(buf.data() + plan_units_off(ids)) = (uint32_t)split.size();
        PlanUnit *u = reinterpret_cast<PlanUnit *>(buf.data() + plan_units_off(ids) + 16);
        std::copy(split.begin(), split.end(), u);
        std::copy(whole.begin(), whole.end(), u + split.size());
    }
    // Pageable source: the copy is staged before this call returns.
    return cudaMemcpyAsync(d_plan, buf.data(), buf.size(), cudaMemcpyHostToDevice, stream) ==
                   cudaSuccess
               ? 0
               : 3;
}

}  // namespace svb
