// Stream VByte decoding of one array, reduce-then-decode form.
//
// The decoder's only serial dependency is where each quad's data bytes start:
// the data pointer advances by C in [4,16] per control byte (Sec. 4, Fig. 4),
// the same chain that in varint-GB also hides the next control byte (Sec. 4).
// With the control stream apart, those positions depend on the control bytes
// alone, so:
//   offsets_kernel   reads only the control stream (2 bits per integer) and
//                    writes the data-stream offset of every sub-tile of
//                    kSubQuads quads (512 integers).  Persistent CTAs each sum
//                    a contiguous range, claimed in order, publish the range
//                    total and find their base as the sum of all earlier
//                    ranges' totals, then add it.  It also writes the
//                    stream's size and checks it against in_len.
//   decode_tiled     persistent CTAs with one producer warp and eight
//                    consumer warps.  The producer takes tiles of eight
//                    sub-tiles round-robin, reads their offsets and has the TMA
//                    engine copy each tile's control and data bytes into one of
//                    kStages shared-memory stages (cp.async.bulk completing on
//                    the stage's "full" mbarrier).  Each consumer warp decodes
//                    one sub-tile on its own - warp scans only, no barrier with
//                    the other warps - and releases it on the stage's "empty"
//                    mbarrier.  Nothing waits on another CTA.
// Differential streams need each sub-tile's carry-in: prev plus the sum of all
// earlier gaps (Sec. 2's prefix sum continued across sub-tiles).  By default
// delta_prep_kernel takes the offsets pass's place and also sums each
// sub-tile's gaps into carry-ins (see its own comment); the decode pass then
// adds a known carry.  The earlier form, kept as a decoder variant, runs a
// sums pass after offsets_kernel: the decode pipeline without stores over
// contiguous tile ranges, each warp summing its sub-tile's gaps and one
// look-back per CTA chaining the range totals into per-sub-tile carries.
//
// Bytes outside the stream are never read: each tile's range is copied as its
// 16-byte-aligned interior by the bulk engine plus a ragged head and tail of
// at most 15 bytes each by plain loads.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"
#include "svb_subtile.cuh"

namespace svb {

constexpr int kTileQuads = 1024;                      // quads per tile (4096 integers)
constexpr int kSubs = kTileQuads / kSubQuads;         // sub-tiles per tile = consumer warps
constexpr int kTileData = 16 * kTileQuads;            // data bytes per tile, at most
constexpr int kStageData = kTileData + 64;            // + 16-byte phase + 2-word read slack
constexpr int kStageCtrl = kTileQuads + 32;
constexpr int kStages = 4;
constexpr int kDecBlock = kThreads + 32;              // 8 consumer warps + 1 producer warp
constexpr u64 kBarrierPolls = 1ull << 24;             // bound on one mbarrier wait
constexpr u64 kNoTile = ~0ull;

static_assert(kSubs == kWarps, "one consumer warp per sub-tile");

// ---------------------------------------------------------------------------
// Pass 1: sub-tile offsets from the control stream.

constexpr int kOffGroupQuads = 64 * kThreads;         // quads per CTA iteration (64 per thread)
constexpr int kOffGroupSubs = kOffGroupQuads / kSubQuads;

struct OffsetsArgs {
    const uint8_t *in;
    u64 in_len;
    u64 n, nquads, nsubs;
    u64 groups;      // ceil(nquads / kOffGroupQuads)
    u64 per_cta;     // groups per CTA
    u64 *offs;       // nsubs + 1 entries
    WsHeader *hdr;
    TileStatus *st;
    u64 spin_limit;
    uint32_t in_aligned;
    uint32_t prev;       // delta_prep_kernel: the value before the first integer
    u64 *carries;        // delta_prep_kernel: per sub-tile carry-in (zero-extended)
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

// Sum of the data bytes of 64 quads starting at q (one thread's share); a
// has in, nquads and in_aligned.
template <class Args>
__device__ __forceinline__ uint32_t sum64(const Args &a, u64 q, uint32_t last_nints)
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

// 16 control bytes (quads q .. q + 15) as one chunk, zero past nquads.
template <class Args>
__device__ __forceinline__ uint4 ctrl_chunk(const Args &a, u64 q)
{
    if (q >= a.nquads)
        return make_uint4(0u, 0u, 0u, 0u);
    if (a.in_aligned && q + 16 <= a.nquads)
        return __ldg(reinterpret_cast<const uint4 *>(a.in + q));
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int b = 0; b < 16; b++)
        if (q + b < a.nquads)
            w[b >> 2] |= (uint32_t)__ldg(a.in + q + b) << (8 * (b & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// This CTA's range of groups [g0, g1): the offsets of its sub-tiles relative
// to the range go to offs, the CTA sums the published totals of the ranges
// before (its base), then the base is added.  The CTA holding the last
// group also writes the stream size and the truncation verdict.  Ends with a
// block barrier (the range's offsets are then visible to the whole CTA).
struct RangeBytes {
    u64 base;   // data offset where the range starts
    u64 bytes;  // data bytes of the range
};

__device__ RangeBytes range_offsets(const OffsetsArgs &a, u64 cta, u64 etag, u64 g0, u64 g1,
                                    uint32_t (*s_w)[kWarps], u64 *s_base, u64 *s_part)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));

    // Each iteration: 64 quads per thread, two threads per sub-tile.  On an
    // aligned stream the next group's four 16-byte loads are issued before
    // this group is summed, so each group costs a scan and a barrier, not a
    // round trip to memory as well.
    u64 running = 0;  // this CTA's data bytes so far (every thread)
    int buf = 0;
    auto whole = [&](u64 q) { return a.in_aligned && q + 64 <= a.nquads; };
    uint4 nxt[4] = {};
    if (g0 < g1 && whole(g0 * (u64)kOffGroupQuads + 64u * tid)) {
        const uint4 *p = reinterpret_cast<const uint4 *>(a.in + g0 * (u64)kOffGroupQuads + 64u * tid);
#pragma unroll
        for (int i = 0; i < 4; i++)
            nxt[i] = __ldg(p + i);
    }
    for (u64 g = g0; g < g1; g++, buf ^= 1) {
        const u64 q = g * (u64)kOffGroupQuads + 64u * tid;
        uint4 cur[4];
#pragma unroll
        for (int i = 0; i < 4; i++)
            cur[i] = nxt[i];
        const u64 qn = q + (u64)kOffGroupQuads;
        if (g + 1 < g1 && whole(qn)) {
            const uint4 *p = reinterpret_cast<const uint4 *>(a.in + qn);
#pragma unroll
            for (int i = 0; i < 4; i++)
                nxt[i] = __ldg(p + i);
        }
        uint32_t sum = 0;
        if (whole(q)) {
#pragma unroll
            for (int i = 0; i < 4; i++)
                sum += chunk_bytes(cur[i], q + 16 * i, a.nquads, last_nints);
        } else {
            sum = sum64(a, q, last_nints);
        }
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);   // the sub-tile's bytes
        const uint32_t v = (lane & 1) ? 0u : sum;
        const uint32_t inc = warp_incl_scan(v);
        if (lane == 31)
            s_w[buf][warp] = inc;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
#pragma unroll
        for (int j = 0; j < kWarps; j++) {
            const uint32_t t = s_w[buf][j];
            wpre += j < warp ? t : 0u;
            tot += t;
        }
        const u64 sub = g * kOffGroupSubs + (tid >> 1);
        if (!(lane & 1) && sub < a.nsubs)
            a.offs[sub] = running + wpre + inc - v;
        running += tot;
        // s_w is double-buffered: the next iteration writes the other half,
        // and the barrier of that iteration orders this read before reuse.
    }

    // The range's base: publish this range's total, then the whole CTA sums
    // the totals of every range before it.  Ranges are claimed in order, so
    // each earlier range belongs to a CTA that has started, and a CTA
    // publishes its total without waiting on anyone: no chain of prefixes is
    // needed.  Each thread inspects kBasePer records per pass, their tag
    // loads in flight together; a release store of a tag, a relaxed load that
    // sees it and an acquire fence order the total's load after it.  Every
    // wait is bounded: after spin_limit polling rounds, or once another CTA
    // has raised an error, the thread records a timeout and stops waiting.
    constexpr int kBasePer = 4;
    if (tid == 0)
        publish(&a.st[cta].off_tag, &a.st[cta].off_agg, running, kFlagAgg, etag);
    u64 part = 0;
    for (u64 p0 = 0; p0 < cta; p0 += (u64)kThreads * kBasePer) {
        u64 tags[kBasePer];
        auto rec = [&](int i) { return p0 + (u64)tid + (u64)i * kThreads; };
        auto ready = [&](u64 t) { return (t & ~3ull) == etag && (t & 3ull) != kFlagNone; };
#pragma unroll
        for (int i = 0; i < kBasePer; i++)
            tags[i] = rec(i) < cta ? ld_relaxed(&a.st[rec(i)].off_tag) : (etag | kFlagAgg);
        for (u64 spins = 0;;) {
            bool all = true;
#pragma unroll
            for (int i = 0; i < kBasePer; i++)
                all = all && ready(tags[i]);
            if (all)
                break;
            if (++spins > a.spin_limit || ((spins & 31) == 0 && error_raised(a.hdr))) {
                raise_error(a.hdr, kErrTimeout);
                break;
            }
            if (spins > 4)
                __nanosleep(spins < 64 ? 32 : 256);
#pragma unroll
            for (int i = 0; i < kBasePer; i++)
                if (!ready(tags[i]))
                    tags[i] = ld_relaxed(&a.st[rec(i)].off_tag);
        }
        fence_acq_rel_gpu();
#pragma unroll
        for (int i = 0; i < kBasePer; i++)
            if (rec(i) < cta && ready(tags[i]))
                part += ld_relaxed(&a.st[rec(i)].off_agg);
    }
    part = warp_sum64(part);
    if (lane == 0)
        s_part[warp] = part;
    __syncthreads();
    if (tid == 0) {
        u64 base = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++)
            base += s_part[w];
        if (g1 == a.groups && g0 < g1) {  // the CTA holding the last sub-tile
            const u64 stream = a.nquads + base + running;
            a.offs[a.nsubs] = base + running;
            st_relaxed(&a.hdr->total, stream);
            if (stream > a.in_len)
                raise_error(a.hdr, kErrTruncated);
        }
        *s_base = base;
    }
    __syncthreads();
    const u64 base = *s_base;
    if (base) {
        // Eight loads in flight per thread, then the eight stores.
        const u64 s0 = g0 * kOffGroupSubs, s1 = min(g1 * kOffGroupSubs, a.nsubs);
        for (u64 s = s0 + tid; s < s1; s += 8u * kThreads) {
            u64 v[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const u64 si = s + (u64)i * kThreads;
                v[i] = si < s1 ? a.offs[si] : 0ull;
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const u64 si = s + (u64)i * kThreads;
                if (si < s1)
                    a.offs[si] = v[i] + base;
            }
        }
    }
    __syncthreads();
    return RangeBytes{base, running};
}

// The last CTA of an offsets launch resets its claim and done counters.
__device__ __forceinline__ void offsets_done(const OffsetsArgs &a)
{
    if (threadIdx.x == 0) {
        __threadfence();
        u64 done = atomicAdd(&a.hdr->a_done, 1ull);
        if (done == (u64)gridDim.x - 1) {
            st_relaxed(&a.hdr->a_counter, 0);
            st_relaxed(&a.hdr->a_done, 0);
        }
    }
}

__global__ void __launch_bounds__(kThreads) offsets_kernel(OffsetsArgs a)
{
    __shared__ uint32_t s_w[2][kWarps];
    __shared__ u64 s_cta, s_etag, s_base, s_part[kWarps];

    if (threadIdx.x == 0) {
        s_cta = atomicAdd(&a.hdr->a_counter, 1ull);
        s_etag = epoch_tag(a.hdr);
    }
    __syncthreads();
    const u64 cta = s_cta;
    const u64 g0 = cta * a.per_cta;
    const u64 g1 = min(g0 + a.per_cta, a.groups);
    range_offsets(a, cta, s_etag, g0, g1, s_w, &s_base, s_part);
    offsets_done(a);
}

// Turns the gap sums carries[s0 .. s1) of the sub-tiles of range `cta` into
// carry-ins, computed by one whole warp: each lane takes a contiguous run of
// the sums (its loads all in flight at once), the lane totals are scanned,
// the range total is chained with the ranges before by one look-back (prev
// starts the first range), and each lane writes its run's carries.
__device__ void range_carries(u64 *carries, u64 s0, u64 s1, u64 cta, uint32_t prev,
                              TileStatus *st, u64 etag, u64 spin_limit, WsHeader *hdr)
{
    const int lane = threadIdx.x & 31;
    const u64 per = (s1 - s0 + 31) / 32;
    const u64 b = min(s0 + lane * per, s1), e = min(b + per, s1);
    uint32_t tot = 0;
#pragma unroll 4
    for (u64 i = b; i < e; i++)
        tot += (uint32_t)carries[i];
    const uint32_t inc = warp_incl_scan(tot);
    const uint32_t run = __shfl_sync(0xffffffffu, inc, 31);
    TileStatus *me = &st[cta];
    u64 base = prev;
    bool ok = true;
    if (cta == 0) {
        if (lane == 0)
            publish(&me->val_tag, &me->val_pre, (uint32_t)(prev + run), kFlagPrefix, etag);
    } else {
        if (lane == 0)
            publish(&me->val_tag, &me->val_agg, run, kFlagAgg, etag);
        base = lookback<true>(st, cta, etag, spin_limit, hdr, ok);
        if (ok && lane == 0)
            publish(&me->val_tag, &me->val_pre, (uint32_t)(base + run), kFlagPrefix, etag);
    }
    if (!ok && lane == 0)
        raise_error(hdr, kErrTimeout);
    uint32_t c = (uint32_t)base + inc - tot;
    for (u64 i = b; i < e; i++) {
        const uint32_t v = (uint32_t)carries[i];
        carries[i] = c;
        c += v;
    }
}

// ---------------------------------------------------------------------------
// Pass 1 for differential streams: sub-tile offsets and carry-ins in one
// launch.  Each CTA takes a contiguous range of groups in claim order, finds
// its sub-tiles' data offsets as offsets_kernel does, then sums each
// sub-tile's gaps and turns the sums into carry-ins within the range; the
// last CTA to finish scans the range totals (prev first) into each range's
// carry-in, which the decode pass adds (Sec. 2's prefix sum continued across
// sub-tiles and ranges).
//
// Gap sums: warp w takes 32 consecutive sub-tiles of the range at a time, one
// per lane.  A full sub-tile whose data is 512 bytes has only zero control
// bytes (Sec. 4: a control byte covers 4 + the sum of its codes bytes), so
// it holds 512 one-byte gaps, the common case of sorted lists with small
// gaps.  For each such sub-tile the warp loads the 16-byte-aligned run that
// holds its bytes, one chunk per lane, coalesced, and each lane byte-sums its
// chunk with dp4a; in batches of 8 runs, a reduce-scatter and a butterfly
// over the warp (10 shuffles per batch) leave sub-tile l's run total in lane
// l, and lane l corrects it for the run's ragged ends.  The kernel runs 4
// CTAs per SM: its waits are chains of dependent loads and barriers, so more
// resident warps pay more than deeper per-warp batches.  Every other
// sub-tile is taken by the whole warp: staged into one of the warp's two
// shared slots with cp.async (the next one's copies in flight) and decoded
// with the decode pass's sub-tile code.  The loads keep the stream in L2 (evict-last) for the decode pass,
// which reads it again.  Reads stay inside the stream as far as the CTA's
// own data ends and inside [in, in + in_len): on a stream cut short the sums
// are meaningless, the truncation verdict is set and the decode pass does
// nothing.

constexpr int kPrepCtrl = 144;                        // 15-byte phase + 128 control bytes
constexpr int kPrepData = 16 * kSubQuads + 48;        // phase + 2048 + round-up + read slack
constexpr int kPrepSlot = kPrepCtrl + kPrepData;      // one staged sub-tile
constexpr int kPrepUnroll = 8;                        // sub-tile runs a warp loads together

static_assert(kPrepUnroll == 8, "the reduce-scatter spans lane bits 4, 3, 2");

static_assert(kPrepCtrl % 16 == 0 && kPrepSlot % 16 == 0, "cp.async needs 16-byte slots");

// 16-byte read-only load whose line L2 keeps with the given policy.
__device__ __forceinline__ uint4 ld_keep128(const void *p, uint64_t policy)
{
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(policy));
    return v;
}

// Mask of the low `kept` bytes of a word (kept clamped to [0, 4]).
__device__ __forceinline__ uint32_t low_bytes_mask(int kept)
{
    return kept <= 0 ? 0u : (kept >= 4 ? ~0u : ~0u >> (8 * (4 - kept)));
}

// Sum of the bytes of x that the byte mask m keeps, added to acc.
__device__ __forceinline__ uint32_t bytesum4(uint4 x, uint4 m, uint32_t acc)
{
    acc = __dp4a(x.x & m.x, 0x01010101u, acc);
    acc = __dp4a(x.y & m.y, 0x01010101u, acc);
    acc = __dp4a(x.z & m.z, 0x01010101u, acc);
    return __dp4a(x.w & m.w, 0x01010101u, acc);
}

__device__ __forceinline__ uint32_t bytesum4(uint4 x, uint32_t acc)
{
    acc = __dp4a(x.x, 0x01010101u, acc);
    acc = __dp4a(x.y, 0x01010101u, acc);
    acc = __dp4a(x.z, 0x01010101u, acc);
    return __dp4a(x.w, 0x01010101u, acc);
}

// Gap sums carries[s0 .. s1) of one range into carry-ins relative to the
// range (exclusive prefix); returns the range total.  One whole warp: each
// lane takes a contiguous run of the sums, the lane totals are scanned.
__device__ uint32_t range_local_carries(u64 *carries, u64 s0, u64 s1)
{
    const int lane = threadIdx.x & 31;
    const u64 per = (s1 - s0 + 31) / 32;
    const u64 b = min(s0 + lane * per, s1), e = min(b + per, s1);
    uint32_t tot = 0;
#pragma unroll 4
    for (u64 i = b; i < e; i++)
        tot += (uint32_t)carries[i];
    const uint32_t inc = warp_incl_scan(tot);
    uint32_t c = inc - tot;
    for (u64 i = b; i < e; i++) {
        const uint32_t v = (uint32_t)carries[i];
        carries[i] = c;
        c += v;
    }
    return __shfl_sync(0xffffffffu, inc, 31);
}

__global__ void __launch_bounds__(kThreads, 4) delta_prep_kernel(OffsetsArgs a)
{
    __shared__ uint32_t s_w[2][kWarps];
    __shared__ u64 s_cta, s_etag, s_base, s_part[kWarps];
    __shared__ uint32_t s_last;
    __shared__ uint4 s_lowm[16];  // s_lowm[p] keeps the bytes below p of a 16-byte chunk
    __shared__ __align__(16) uint8_t s_slot[kWarps][2][kPrepSlot];
    __shared__ __align__(16) uint16_t s_pos[kWarps][kSubQuads];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_cta = atomicAdd(&a.hdr->a_counter, 1ull);
        s_etag = epoch_tag(a.hdr);
    }
    if (tid < 16)
        s_lowm[tid] = make_uint4(low_bytes_mask(tid), low_bytes_mask(tid - 4),
                                 low_bytes_mask(tid - 8), low_bytes_mask(tid - 12));
    __syncthreads();
    const u64 cta = s_cta, etag = s_etag;
    const u64 g0 = cta * a.per_cta;
    const u64 g1 = min(g0 + a.per_cta, a.groups);
    const RangeBytes r = range_offsets(a, cta, etag, g0, g1, s_w, &s_base, s_part);

    const u64 s0 = g0 * kOffGroupSubs, s1 = min(g1 * kOffGroupSubs, a.nsubs);
    const u64 range_end = r.base + r.bytes;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    const uint8_t *data = a.in + a.nquads;
    const uint8_t *rdata = data + r.base;  // the range's first data byte
    // Bytes this CTA may read: its control and data bytes lie below the end
    // of its data, and nothing at or past in + in_len is read (in_len may
    // be the "unbounded" ~0 of the unchecked calls: saturate).
    const uintptr_t lo = (uintptr_t)a.in;
    const uintptr_t in_end = a.in_len > ~(uintptr_t)0 - lo ? ~(uintptr_t)0 : lo + a.in_len;
    const uintptr_t hi = min(in_end, (uintptr_t)(data + range_end));
    const uint64_t policy = l2_policy_evict_last();
    uint16_t *pos = s_pos[warp];

    // Warp-wide: stage sub-tile j (data bytes [d0, d1)) into slot b.
    auto stage = [&](u64 j, u64 d0, u64 d1, uint8_t *b) {
        const u64 q0 = j * kSubQuads;
        const uint32_t nq = (uint32_t)min((u64)kSubQuads, a.nquads - q0);
        warp_stage(a.in + q0, nq, b, lo, hi, policy);
        warp_stage(data + d0, (uint32_t)(d1 - d0), b + kPrepCtrl, lo, hi, policy);
    };
    // Warp-wide: the decoded gaps of staged sub-tile j summed (every lane).
    auto staged_sum = [&](u64 j, u64 d0, const uint8_t *b) -> uint32_t {
        const u64 q0 = j * kSubQuads;
        SubTile t;
        t.C = b + ((uintptr_t)(a.in + q0) & 15u);
        t.D = b + kPrepCtrl;
        t.base = (uint32_t)((uintptr_t)(data + d0) & 15u);
        t.nq = (uint32_t)min((u64)kSubQuads, a.nquads - q0);
        t.tail = q0 + t.nq == a.nquads ? last_nints : 4u;
        const uint32_t w = subtile_ctrl_word(t);
        subtile_positions(t, w, pos);
        __syncwarp();
        uint32_t v[kSubRounds][4];
        subtile_gather(t, pos, v);
        uint32_t sum = 0;
#pragma unroll
        for (int rr = 0; rr < kSubRounds; rr++)
            sum += v[rr][0] + v[rr][1] + v[rr][2] + v[rr][3];
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1)
            sum += __shfl_xor_sync(0xffffffffu, sum, d);
        __syncwarp();  // the slot and pos are read before they are refilled
        return sum;
    };

    for (u64 rb = s0 + (u64)warp * 32; rb < s1; rb += (u64)kWarps * 32) {
        const u64 j = rb + lane;
        const bool valid = j < s1;
        uint32_t e0 = 0, e1 = 0;  // the sub-tile's data bytes, from the range's first
        if (valid) {
            e0 = (uint32_t)(a.offs[j] - r.base);
            e1 = (uint32_t)((j + 1 < s1 ? a.offs[j + 1] : range_end) - r.base);
        }
        const u64 q0 = j * kSubQuads;
        const bool full = valid && (q0 + kSubQuads < a.nquads ||
                                    (q0 + kSubQuads == a.nquads && last_nints == 4));
        const uintptr_t g = (uintptr_t)(rdata + e0);
        const uintptr_t a0 = g & ~(uintptr_t)15;
        // The run's chunk 32 (its first g mod 16 bytes end the sub-tile's
        // 512) must lie inside the readable bytes too.
        const bool fast = full && e1 - e0 == 4u * kSubQuads && a0 >= lo && a0 + 16 * 33 <= hi;
        const unsigned F = __ballot_sync(0xffffffffu, fast);
        // Batches of 8 runs: each lane byte-sums its chunk of each run, a
        // reduce-scatter over lane bits 4, 3, 2 and a butterfly over bits
        // 1, 0 leave run u0 + k's total in lanes 4k .. 4k + 3, and lane
        // u0 + k takes it from lane 4k.  Each batch's loads are issued as
        // soon as the batch before has been byte-summed.
        uint32_t sum = 0;  // chunks 0..31 of this lane's run
        uint4 v[kPrepUnroll];
        auto load_batch = [&](int u0) {
#pragma unroll
            for (int i = 0; i < kPrepUnroll; i++) {
                const int u = u0 + i;
                const uint32_t eu = __shfl_sync(0xffffffffu, e0, u);
                v[i] = make_uint4(0u, 0u, 0u, 0u);
                if ((F >> u) & 1u) {
                    const uint4 *run = reinterpret_cast<const uint4 *>(
                        (uintptr_t)(rdata + eu) & ~(uintptr_t)15);
                    v[i] = ld_keep128(run + lane, policy);
                }
            }
        };
        load_batch(0);
#pragma unroll
        for (int u0 = 0; u0 < 32; u0 += kPrepUnroll) {
            uint32_t q[kPrepUnroll];
#pragma unroll
            for (int i = 0; i < kPrepUnroll; i++)
                q[i] = bytesum4(v[i], 0u);
            if (u0 + kPrepUnroll < 32)   // the next batch's loads fly during the shuffles
                load_batch(u0 + kPrepUnroll);
#pragma unroll
            for (int h = kPrepUnroll / 2, bit = 16; h >= 1; h >>= 1, bit >>= 1) {
                const bool upper = (lane & bit) != 0;
#pragma unroll
                for (int i = 0; i < h; i++) {
                    const uint32_t send = upper ? q[i] : q[i + h];
                    const uint32_t keep = upper ? q[i + h] : q[i];
                    q[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
                }
            }
            q[0] += __shfl_xor_sync(0xffffffffu, q[0], 2);
            q[0] += __shfl_xor_sync(0xffffffffu, q[0], 1);
            const uint32_t t = __shfl_sync(0xffffffffu, q[0], ((lane - u0) & 7) << 2);
            if ((lane & ~7) == u0)
                sum = t;
        }
        if (fast) {
            // Bytes [g, g + 512): less the first ph bytes of chunk 0, plus
            // the first ph bytes of chunk 32.
            const uint32_t ph = (uint32_t)(g & 15u);
            if (ph) {
                const uint4 m = s_lowm[ph];
                const uint4 *run = reinterpret_cast<const uint4 *>(a0);
                const uint4 c0 = ld_keep128(run, policy), c32 = ld_keep128(run + 32, policy);
                sum += bytesum4(c32, m, 0u) - bytesum4(c0, m, 0u);
            }
        }
        // The rest, a whole warp per sub-tile, the next one's copies in
        // flight while the current one is summed.
        unsigned slow = __ballot_sync(0xffffffffu, valid && !fast);
        if (slow) {
            const u64 d0 = r.base + e0, d1 = r.base + e1;
            int l = __ffs(slow) - 1;
            uint32_t k = 0;
            stage(__shfl_sync(0xffffffffu, j, l), __shfl_sync(0xffffffffu, d0, l),
                  __shfl_sync(0xffffffffu, d1, l), s_slot[warp][0]);
            cp_async_commit();
            while (slow) {
                slow &= slow - 1;
                const int nl = slow ? __ffs(slow) - 1 : -1;
                if (nl >= 0)
                    stage(__shfl_sync(0xffffffffu, j, nl), __shfl_sync(0xffffffffu, d0, nl),
                          __shfl_sync(0xffffffffu, d1, nl), s_slot[warp][(k + 1) & 1]);
                cp_async_commit();
                cp_async_wait<1>();
                __syncwarp();
                const uint32_t t = staged_sum(__shfl_sync(0xffffffffu, j, l),
                                              __shfl_sync(0xffffffffu, d0, l),
                                              s_slot[warp][k & 1]);
                if (lane == l)
                    sum = t;
                l = nl;
                k++;
            }
            cp_async_wait<0>();
        }
        if (valid)
            a.carries[j] = sum;
    }
    __syncthreads();  // every gap sum of the range is written
    if (warp == 0 && s0 < s1) {
        const uint32_t total = range_local_carries(a.carries, s0, s1);
        if (lane == 0)
            a.st[cta].val_agg = total;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&a.hdr->a_done, 1ull) == (u64)gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last)
        return;
    // The last CTA: carry-in of every range = prev + the totals before it.
    // Thread t scans a contiguous run of the ranges.
    __threadfence();
    const u64 nr = gridDim.x;
    const u64 per = (nr + kThreads - 1) / kThreads;
    const u64 b = min((u64)tid * per, nr), e = min(b + per, nr);
    uint32_t tot = 0;
    for (u64 i = b; i < e; i++)
        tot += (uint32_t)ld_relaxed(&a.st[i].val_agg);
    const uint32_t inc = warp_incl_scan(tot);
    if (lane == 31)
        s_w[0][warp] = inc;
    __syncthreads();
    uint32_t c = a.prev + inc - tot;
    for (int w = 0; w < warp; w++)
        c += s_w[0][w];
    for (u64 i = b; i < e; i++) {
        const uint32_t v = (uint32_t)ld_relaxed(&a.st[i].val_agg);
        a.st[i].val_pre = c;
        c += v;
    }
    if (tid == 0) {
        st_relaxed(&a.hdr->a_counter, 0);
        st_relaxed(&a.hdr->a_done, 0);
    }
}

// ---------------------------------------------------------------------------
// Pass 2: persistent decode, producer warp + consumer warps.

enum TiledMode : int {
    kPlain = 0,  // decode and store
    kDelta = 1,  // decode, running sums plus each sub-tile's carry-in, store
    kSums = 2,   // decode, sum each sub-tile's gaps; write per-sub-tile carries
};

struct TiledArgs {
    const uint8_t *in;
    u64 n, nquads, ntiles, nsubs;
    uint32_t *out;
    const u64 *offs;
    u64 *carries;       // per sub-tile: written by kSums, read by kDelta (zero-extended)
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    u64 per_cta;        // kSums: tiles per CTA (contiguous ranges)
    u64 range_subs;     // kDelta: carries are relative to ranges of this many
                        // sub-tiles, whose carry-ins are st[range].val_pre
                        // (0: the carries are absolute)
    u64 range_magic;    // ceil(2^64 / (range_subs / kSubs)): a tile's range is
                        // the high word of tile * range_magic
    u64 tile0, tile1;   // decoding: the tiles [tile0, tile1) to decode
    u64 in_len;         // decode_chunked_kernel: stream bytes that may be read
    uint32_t prev;
    uint32_t out_aligned;
};

struct Pipe {
    uint8_t data[kStages][kStageData];
    uint8_t ctrl[kStages][kStageCtrl];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    u64 tile[kStages];
    uint32_t hd[kStages], hc[kStages];   // address phase (mod 16) of the data / control range
    uint32_t soff[kStages][kSubs];       // each sub-tile's data offset inside the tile
    uint32_t carry[kStages][kSubs];      // kDelta: each sub-tile's carry-in
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
    const u64 t = a.tile0 + first + (u64)k * gridDim.x;
    return t < a.tile1 ? t : a.ntiles;
}

// Producer warp: fill stages with tiles until none is left, then post one
// stage marked kNoTile.  Lane j < 9 carries the offset of sub-tile j of the
// next tile (the ninth is where the tile ends); lane j < 8 its carry.
template <int kMode>
__device__ void produce(const TiledArgs &a, Pipe &P, u64 first, int lane)
{
    uint32_t issued = 0;  // stage fills posted (iteration k fills stage k % kStages)
    auto fetch = [&](u64 t, u64 &off, uint32_t &car) {
        if (t < a.ntiles && lane <= kSubs) {
            const u64 sb = min(t * kSubs + lane, a.nsubs);
            off = a.offs[sb];
            if (kMode == kDelta && lane < kSubs && sb < a.nsubs) {
                car = (uint32_t)a.carries[sb];
                // A range is a whole number of tiles; t / (tiles per range)
                // by one multiply (exact for t < 2^32: the rounding error
                // of the reciprocal stays below 1 / divisor).
                if (a.range_subs)
                    car += (uint32_t)a.st[__umul64hi(t, a.range_magic)].val_pre;
            }
        }
    };
    const uint8_t *stream_end = a.in + a.nquads + a.offs[a.nsubs];
    // Offsets (and carries) of the next kAhead tiles are in flight at once,
    // so a tile's metadata has kAhead stage fills to arrive in: one round
    // trip per tile would bound a CTA whose tiles decode faster than that.
    constexpr int kAhead = 4;
    u64 qt[kAhead], qoff[kAhead];
    uint32_t qcar[kAhead];
#pragma unroll
    for (int i = 0; i < kAhead; i++) {
        qt[i] = tile_of<kMode>(a, first, i);
        qoff[i] = 0;
        qcar[i] = 0;
        fetch(qt[i], qoff[i], qcar[i]);
    }
    bool done = false;
    for (uint32_t k0 = 0; !done; k0 += kAhead) {
#pragma unroll
    for (int i = 0; i < kAhead; i++) {
        const uint32_t k = k0 + i;
        const int s = k % kStages;
        if (k >= (uint32_t)kStages) {
            bool ok = mbar_wait_bounded(&P.empty[s], ((k / kStages) - 1) & 1u, kBarrierPolls);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0)
                    raise_error(a.hdr, kErrTimeout);
                done = true;
                break;
            }
        }
        const u64 t = qt[i];
        const u64 off = qoff[i];
        const uint32_t car = qcar[i];
        if (t >= a.ntiles) {
            if (lane == 0) {
                P.tile[s] = kNoTile;
                mbar_arrive_expect_tx(&P.full[s], 0);
            } else {
                mbar_arrive(&P.full[s]);
            }
            issued = k + 1;
            done = true;
            break;
        }
        qt[i] = tile_of<kMode>(a, first, k + kAhead);
        fetch(qt[i], qoff[i], qcar[i]);
        const u64 d0 = __shfl_sync(0xffffffffu, off, 0);
        const u64 d1 = __shfl_sync(0xffffffffu, off, kSubs);
        if (lane < kSubs) {
            P.soff[s][lane] = (uint32_t)(off - d0);
            if (kMode == kDelta)
                P.carry[s][lane] = car;
        }
        const u64 q0 = t * kTileQuads;
        const uint32_t clen = (uint32_t)min((u64)kTileQuads, a.nquads - q0);
        const uint8_t *gc = a.in + q0;
        const uint8_t *gd = a.in + a.nquads + d0;
        const uint32_t dlen = (uint32_t)(d1 - d0);
        // Everything in [in, stream end) may be read: a tile's aligned ends
        // are bytes of its neighbours, so almost every tile is one bulk copy
        // per stream and the producer never waits on a load of its own.
        const StagePlan pc = stage_plan(gc, clen, a.in, stream_end);
        const StagePlan pd = stage_plan(gd, dlen, a.in, stream_end);
        if (pc.edges)
            range_edges(gc, clen, P.ctrl[s], lane);
        if (pd.edges)
            range_edges(gd, dlen, P.data[s], lane);
        if (lane == 0) {
            P.tile[s] = t;
            P.hc[s] = (uint32_t)((uintptr_t)gc & 15u);
            P.hd[s] = (uint32_t)((uintptr_t)gd & 15u);
            mbar_arrive_expect_tx(&P.full[s], pc.bytes + pd.bytes);
            if (pc.bytes)
                bulk_g2s(P.ctrl[s] + pc.dst_off, pc.src, pc.bytes, &P.full[s]);
            if (pd.bytes)
                bulk_g2s(P.data[s] + pd.dst_off, pd.src, pd.bytes, &P.full[s]);
        } else {
            mbar_arrive(&P.full[s]);
        }
        issued = k + 1;
    }
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

// A full sub-tile of 512 one-byte gaps at staged position b, decoded into
// running sums from carry_in: lane l holds quad 32r + l in v[r] (the layout
// the stores take).  The in-quad sums of the four rounds are packed into
// 16-bit fields of one 64-bit word (each at most 4 * 255, a warp's total at
// most 32 * 1020 < 2^16), so one warp scan serves all four rounds.
__device__ __forceinline__ void zero_ctrl_delta(const uint8_t *D, uint32_t b, uint32_t carry_in,
                                                uint32_t (&v)[kSubRounds][4])
{
    const int lane = threadIdx.x & 31;
    const uint32_t *W = reinterpret_cast<const uint32_t *>(D);
#pragma unroll
    for (int r = 0; r < kSubRounds; r++) {
        const uint32_t p = b + 128u * r + 4u * lane;
        const uint32_t x = __funnelshift_r(W[p >> 2], W[(p >> 2) + 1], p << 3);
        v[r][0] = __byte_perm(x, 0, 0x4440);
        v[r][1] = v[r][0] + __byte_perm(x, 0, 0x4441);
        v[r][2] = v[r][1] + __byte_perm(x, 0, 0x4442);
        v[r][3] = v[r][2] + __byte_perm(x, 0, 0x4443);
    }
    const u64 pk = (u64)(v[0][3] | (v[1][3] << 16)) | ((u64)(v[2][3] | (v[3][3] << 16)) << 32);
    u64 inc = pk;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const u64 t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d)
            inc += t;
    }
    const u64 ex = inc - pk;
    const u64 tot = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t t0 = (uint32_t)tot & 0xffffu, t1 = (uint32_t)(tot >> 16) & 0xffffu,
                   t2 = (uint32_t)(tot >> 32) & 0xffffu;
    uint32_t add[kSubRounds];
    add[0] = carry_in + ((uint32_t)ex & 0xffffu);
    add[1] = carry_in + t0 + ((uint32_t)(ex >> 16) & 0xffffu);
    add[2] = carry_in + t0 + t1 + ((uint32_t)(ex >> 32) & 0xffffu);
    add[3] = carry_in + t0 + t1 + t2 + (uint32_t)(ex >> 48);
#pragma unroll
    for (int r = 0; r < kSubRounds; r++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            v[r][j] += add[r];
}

// Stores a sub-tile's integers (lane l: quad 32r + l in v[r]).
__device__ __forceinline__ void store_subtile(uint32_t *out, u64 q0, uint32_t nq, bool full,
                                              bool aligned, u64 nquads, uint32_t last_nints,
                                              const uint32_t (&v)[kSubRounds][4])
{
    const int lane = threadIdx.x & 31;
    uint32_t *op = out + 4 * (q0 + lane);
#pragma unroll
    for (int r = 0; r < kSubRounds; r++) {
        const uint32_t lq = r * 32 + lane;
        uint32_t *dst = op + 128 * r;
        if (full && aligned) {
            stg_stream128(dst, make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]));
        } else if (lq < nq) {
            const uint32_t nints = q0 + lq == nquads - 1 ? last_nints : 4u;
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

// Consumer warp `warp`: decodes sub-tile `warp` of every tile, alone.
template <int kMode>
__device__ void consume(const TiledArgs &a, Pipe &P, uint16_t *s_pos)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    uint16_t *pos = s_pos + warp * kSubQuads;   // this warp's staged positions
    for (uint32_t k = 0;; k++) {
        const int s = k % kStages;
        if (!mbar_wait_bounded(&P.full[s], (k / kStages) & 1u, kBarrierPolls)) {
            raise_error(a.hdr, kErrTimeout);  // cannot happen unless a copy is lost
            break;
        }
        const u64 tile = P.tile[s];
        if (tile == kNoTile)
            break;
        const u64 q0 = tile * kTileQuads + (u64)warp * kSubQuads;  // first quad of the sub-tile
        const u64 sb = tile * kSubs + warp;
        if (q0 >= a.nquads) {  // the last tile may have fewer sub-tiles
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&P.empty[s]);
            continue;
        }
        SubTile t;
        t.C = P.ctrl[s] + P.hc[s] + warp * kSubQuads;
        t.D = P.data[s];
        t.base = P.hd[s] + P.soff[s][warp];
        t.nq = (uint32_t)min((u64)kSubQuads, a.nquads - q0);
        t.tail = q0 + t.nq == a.nquads ? last_nints : 4u;
        const bool full = t.full();
        const uint8_t *D = t.D;
        const uint32_t base = t.base;
        const uint32_t carry_in = kMode == kDelta ? P.carry[s][warp] : 0u;
        const uint32_t w = subtile_ctrl_word(t);
        if (kMode == kSums && full && __all_sync(0xffffffffu, w == 0)) {
            // All 512 integers take one byte: the gaps are the data bytes
            // [base, base + 512).
            const uint32_t t = zero_ctrl_sum(D, base);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&P.empty[s]);
            if (lane == 0)
                a.carries[sb] = t;
            continue;
        }
        uint32_t v[kSubRounds][4];
        if (kMode == kDelta && full && __all_sync(0xffffffffu, w == 0)) {
            // Every integer one byte (Sec. 4): no positions to find, one
            // packed scan for the running sums.
            zero_ctrl_delta(D, base, carry_in, v);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&P.empty[s]);
            store_subtile(a.out, q0, t.nq, full, a.out_aligned != 0, a.nquads, last_nints, v);
            continue;
        }
        subtile_positions(t, w, pos);
        __syncwarp();
        uint32_t *op = a.out + 4 * (q0 + lane);
        const uint32_t nq = t.nq;
        subtile_gather(t, pos, v);
        // This warp no longer reads stage s.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&P.empty[s]);

        if (kMode == kSums) {
            uint32_t t = 0;
#pragma unroll
            for (int r = 0; r < kSubRounds; r++)
                t += v[r][0] + v[r][1] + v[r][2] + v[r][3];
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1)
                t += __shfl_xor_sync(0xffffffffu, t, d);
            if (lane == 0)
                a.carries[sb] = t;  // the sub-tile's gap sum; made a carry later
            continue;
        }
        if (kMode == kDelta) {
            // Running sums: within the quad, across the warp's rounds, carry-in.
            uint32_t run = carry_in;
#pragma unroll
            for (int r = 0; r < kSubRounds; r++) {
                v[r][1] += v[r][0];
                v[r][2] += v[r][1];
                v[r][3] += v[r][2];
                const uint32_t qs = v[r][3];
                const uint32_t inc = warp_incl_scan(qs);
                const uint32_t add = run + inc - qs;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    v[r][j] += add;
                run += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
#pragma unroll
        for (int r = 0; r < kSubRounds; r++) {
            const uint32_t lq = r * 32 + lane;
            uint32_t *dst = op + 128 * r;
            if (full && a.out_aligned) {
                stg_stream128(dst, make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]));
            } else if (lq < nq) {
                const uint32_t nints = q0 + lq == a.nquads - 1 ? last_nints : 4u;
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

// kSums epilogue, warp 0: turn this CTA's sub-tile gap sums into carries.
__device__ void sums_to_carries(const TiledArgs &a, u64 first, u64 etag)
{
    const u64 s0 = first * kSubs;
    const u64 s1 = min(min(first + a.per_cta, a.ntiles) * kSubs, a.nsubs);
    const u64 cta = first / (a.per_cta ? a.per_cta : 1);
    range_carries(a.carries, s0, s1, cta, a.prev, a.st, etag, a.spin_limit, a.hdr);
}

// ---------------------------------------------------------------------------
// Single pass for plain streams, by chunks: decode_chunked_kernel.
//
// Persistent CTAs take chunks of kDcTiles tiles in claim order.  A chunk
// warp, one chunk ahead of the decode, reads the chunk's control bytes,
// turns them into each sub-tile's data offset within the chunk (Sec. 4: a
// control byte covers 4 + the sum of its codes bytes), publishes the chunk's
// total and finds the chunk's data offset by decoupled look-back over the
// chunks before it.  The producer warp then stages the chunk's tiles with
// bulk copies and the consumer warps decode them exactly as in the two-pass
// decoder, so no separate offsets pass runs.  A chunk's look-back has the
// decode of the previous chunk to complete in: chunks are claimed about as
// fast as CTAs finish them, so the predecessors it waits on are a window of
// recent claims whose totals were published as soon as their control bytes
// were summed.  The control reads ask L2 to keep the bytes for the
// producer, which stages them again one chunk later; at full size most have
// been evicted by then, so the control stream is read twice.

constexpr int kDcTiles = 16;                   // tiles per chunk (65536 integers)
constexpr int kDcSubs = kDcTiles * kSubs;      // sub-tiles per chunk
constexpr int kDcBlock = kDecBlock + 32;       // consumers, producer, chunk warp
constexpr int kDcVecs = kDcTiles * kTileQuads / 16;   // 16-byte control vectors per chunk
constexpr int kDcLaneSubs = kDcSubs / 32;              // sub-tiles each lane scans
static_assert(kDcSubs % 32 == 0 && kDcVecs % (8 * 32) == 0, "whole batches of vectors");

struct DcChunks {
    u64 chunk[2];                     // chunk index, or kNoTile once none is left
    u64 base[2];                      // the chunk's first data byte (from the data start)
    uint32_t soff[2][kDcSubs + 1];    // sub-tile data offsets in the chunk; [kDcSubs]: its total
    uint32_t bad[2];                  // cut short or failed: decode nothing
    uint64_t ready[2];                // chunk warp -> producer
    uint64_t freed[2];                // producer -> chunk warp
};

// The chunk warp: sums, look-back and hand-over of one chunk after another,
// double-buffered; buffer b is claimed again only once the producer freed it.
__device__ void dc_chunks(const TiledArgs &a, DcChunks &C, uint32_t *s_cnt, u64 etag, int lane)
{
    const u64 nchunks = (a.ntiles + kDcTiles - 1) / kDcTiles;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    const bool aligned = ((uintptr_t)a.in & 15u) == 0;
    const uint64_t keep = l2_policy_evict_last();
    for (uint32_t j = 0;; j++) {
        const int b = j & 1;
        if (j >= 2 && !__all_sync(0xffffffffu, mbar_wait_bounded(&C.freed[b], ((j >> 1) - 1) & 1u,
                                                                  kBarrierPolls))) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            return;   // the producer's own wait for this buffer runs out too
        }
        u64 c = 0;
        if (lane == 0)
            c = atomicAdd(&a.hdr->tile_counter, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= nchunks) {
            if (lane == 0) {
                C.chunk[b] = kNoTile;
                mbar_arrive(&C.ready[b]);
            }
            return;
        }
        // Data bytes of each sub-tile: vector 32i + lane holds quads
        // 16 (32i + lane) .. of the chunk, which lie in sub-tile 4i + lane / 8;
        // the 8 lanes of a sub-tile add up their counts.
        const u64 q0 = c * (u64)kDcTiles * kTileQuads;
#pragma unroll
        for (int h = 0; h < kDcVecs / (8 * 32); h++) {
            uint4 v[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const u64 q = q0 + 16 * (u64)((8 * h + i) * 32 + lane);
                if (q >= a.nquads) {
                    v[i] = make_uint4(0u, 0u, 0u, 0u);
                } else if (aligned && q + 16 <= a.nquads) {
                    v[i] = ld_keep128(a.in + q, keep);
                } else {
                    uint32_t w[4] = {0, 0, 0, 0};
                    for (int k = 0; k < 16; k++)
                        if (q + k < a.nquads)
                            w[k >> 2] |= (uint32_t)__ldg(a.in + q + k) << (8 * (k & 3));
                    v[i] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const u64 q = q0 + 16 * (u64)((8 * h + i) * 32 + lane);
                uint32_t cnt = q < a.nquads ? chunk_bytes(v[i], q, a.nquads, last_nints) : 0u;
                cnt += __shfl_xor_sync(0xffffffffu, cnt, 1);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, 2);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, 4);
                if ((lane & 7) == 0)
                    s_cnt[4 * (8 * h + i) + (lane >> 3)] = cnt;
            }
        }
        __syncwarp();
        uint32_t cs[kDcLaneSubs], lt = 0;
#pragma unroll
        for (int i = 0; i < kDcLaneSubs; i++) {
            cs[i] = s_cnt[kDcLaneSubs * lane + i];
            lt += cs[i];
        }
        const uint32_t inc = warp_incl_scan(lt);
        uint32_t ex = inc - lt;
#pragma unroll
        for (int i = 0; i < kDcLaneSubs; i++) {
            C.soff[b][kDcLaneSubs * lane + i] = ex;
            ex += cs[i];
        }
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        // The chunk's data offset: publish its total, then look back.
        u64 excl = 0;
        bool ok = true;
        if (c == 0) {
            if (lane == 0)
                publish(&a.st[0].off_tag, &a.st[0].off_pre, total, kFlagPrefix, etag);
        } else {
            if (lane == 0)
                publish(&a.st[c].off_tag, &a.st[c].off_agg, total, kFlagAgg, etag);
            excl = lookback<false>(a.st, c, etag, a.spin_limit, a.hdr, ok);
            if (lane == 0 && ok)
                publish(&a.st[c].off_tag, &a.st[c].off_pre, excl + total, kFlagPrefix, etag);
        }
        const u64 end = a.nquads + excl + total;   // stream bytes up to the chunk's end
        if (lane == 0) {
            if (!ok)
                raise_error(a.hdr, kErrTimeout);
            else if (end > a.in_len)
                raise_error(a.hdr, kErrTruncated);
            if (c == nchunks - 1)
                st_relaxed(&a.hdr->total, end);
            C.soff[b][kDcSubs] = total;
            C.base[b] = excl;
            C.chunk[b] = c;
            C.bad[b] = (!ok || end > a.in_len) ? 1u : 0u;
        }
        __syncwarp();   // s_cnt and the buffer are written before the hand-over
        if (lane == 0)
            mbar_arrive(&C.ready[b]);
    }
}

// The producer: each chunk's tiles into the stage ring, with the offsets the
// chunk warp found.  Reads stay inside the stream: below the chunk's own data
// end plus the bytes the integers after it must have (the aligned copy of a
// tile that would pass that bound falls back to its interior plus plain
// loads of the ragged ends).
__device__ void dc_produce(const TiledArgs &a, Pipe &P, DcChunks &C, int lane)
{
    uint32_t k = 0, issued = 0;   // stage fills
    const uint8_t *data = a.in + a.nquads;
    auto wait_empty = [&]() -> bool {
        if (k < (uint32_t)kStages)
            return true;
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&P.empty[k % kStages],
                                                                  ((k / kStages) - 1) & 1u,
                                                                  kBarrierPolls));
        if (!ok && lane == 0)
            raise_error(a.hdr, kErrTimeout);
        return ok;
    };
    for (uint32_t j = 0;; j++) {
        const int b = j & 1;
        if (!__all_sync(0xffffffffu,
                        mbar_wait_bounded(&C.ready[b], (j >> 1) & 1u, kBarrierPolls))) {
            if (lane == 0)
                raise_error(a.hdr, kErrTimeout);
            break;
        }
        const u64 c = C.chunk[b];
        if (c == kNoTile)
            break;
        const u64 t0 = c * kDcTiles, t1 = min(t0 + kDcTiles, a.ntiles);
        const u64 base = C.base[b];
        // Readable up to the chunk's data end plus as many bytes as the
        // integers after the chunk surely have (one each), at most 16.
        const u64 after = a.n - min(a.n, (t1 * kTileQuads) * 4);
        const uint8_t *hi = data + base + C.soff[b][kDcSubs] + min(after, (u64)16);
        if (a.in_len != ~0ull && hi > a.in + a.in_len)
            hi = a.in + a.in_len;
        bool failed = false;
        for (u64 t = C.bad[b] ? t1 : t0; t < t1; t++) {
            if (!wait_empty()) {
                failed = true;
                break;
            }
            const int s = k % kStages;
            const uint32_t i = (uint32_t)(t - t0);
            const uint32_t so = lane <= kSubs ? C.soff[b][i * kSubs + lane] : 0u;
            const uint32_t s0 = __shfl_sync(0xffffffffu, so, 0);
            const uint32_t s1 = __shfl_sync(0xffffffffu, so, kSubs);
            if (lane < kSubs)
                P.soff[s][lane] = so - s0;
            const u64 q0 = t * kTileQuads;
            const uint32_t clen = (uint32_t)min((u64)kTileQuads, a.nquads - q0);
            const uint8_t *gc = a.in + q0;
            const uint8_t *gd = data + base + s0;
            const uint32_t dlen = s1 - s0;
            const StagePlan pc = stage_plan(gc, clen, a.in, hi);
            const StagePlan pd = stage_plan(gd, dlen, a.in, hi);
            if (pc.edges)
                range_edges(gc, clen, P.ctrl[s], lane);
            if (pd.edges)
                range_edges(gd, dlen, P.data[s], lane);
            if (lane == 0) {
                P.tile[s] = t;
                P.hc[s] = (uint32_t)((uintptr_t)gc & 15u);
                P.hd[s] = (uint32_t)((uintptr_t)gd & 15u);
                mbar_arrive_expect_tx(&P.full[s], pc.bytes + pd.bytes);
                if (pc.bytes)
                    bulk_g2s(P.ctrl[s] + pc.dst_off, pc.src, pc.bytes, &P.full[s]);
                if (pd.bytes)
                    bulk_g2s(P.data[s] + pd.dst_off, pd.src, pd.bytes, &P.full[s]);
            } else {
                mbar_arrive(&P.full[s]);
            }
            issued = ++k;
        }
        __syncwarp();   // buffer b is no longer read
        if (lane == 0)
            mbar_arrive(&C.freed[b]);
        if (failed)
            break;
    }
    // No tile left: one stage marked kNoTile ends the consumers' loop.
    if (wait_empty()) {
        const int s = k % kStages;
        if (lane == 0) {
            P.tile[s] = kNoTile;
            mbar_arrive_expect_tx(&P.full[s], 0);
        } else {
            mbar_arrive(&P.full[s]);
        }
        issued = ++k;
    }
    // Let every copy this warp started land before the CTA can exit.
    if (lane == 0) {
        for (int s = 0; s < kStages; s++)
            if (issued > (uint32_t)s) {
                const uint32_t fills = (issued - 1 - s) / kStages + 1;
                mbar_wait_bounded(&P.full[s], (fills - 1) & 1u, kBarrierPolls);
            }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kDcBlock, 3) decode_chunked_kernel(TiledArgs a)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    Pipe &P = *reinterpret_cast<Pipe *>(dyn_smem);
    __shared__ __align__(16) uint16_t s_pos[kWarps * kSubQuads];
    __shared__ DcChunks C;
    __shared__ uint32_t s_cnt[kDcSubs];
    __shared__ u64 s_etag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&P.full[s], 32);        // the 32 producer lanes arrive
            mbar_init(&P.empty[s], kWarps);   // one arrival per consumer warp
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&C.ready[b], 1);
            mbar_init(&C.freed[b], 1);
        }
        fence_mbar_init();
        s_etag = epoch_tag(a.hdr);
    }
    __syncthreads();
    if (warp == kWarps)
        dc_produce(a, P, C, lane);
    else if (warp == kWarps + 1)
        dc_chunks(a, C, s_cnt, s_etag, lane);
    else
        consume<kPlain>(a, P, s_pos);
    finish_launch(a.hdr, a.result);
}

template <int kMode>
__global__ void __launch_bounds__(kDecBlock, 3) decode_tiled_kernel(TiledArgs a)
{
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    Pipe &P = *reinterpret_cast<Pipe *>(dyn_smem);
    __shared__ __align__(16) uint16_t s_pos[kTileQuads];
    __shared__ u64 s_etag, s_first;
    __shared__ uint32_t s_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&P.full[s], 32);        // the 32 producer lanes arrive
            mbar_init(&P.empty[s], kWarps);   // one arrival per consumer warp
        }
        fence_mbar_init();
        s_etag = epoch_tag(a.hdr);
        s_flag = error_raised(a.hdr) ? 1u : 0u;
        // The sums pass takes ranges in claim order, so every range before
        // this one belongs to a CTA that is running or done.
        s_first = kMode == kSums ? atomicAdd(&a.hdr->tile_counter, 1ull) * a.per_cta
                                 : (u64)blockIdx.x;
    }
    __syncthreads();
    if (!s_flag) {  // else the offsets pass failed (truncated stream)
        if (warp == kWarps) {
            produce<kMode>(a, P, s_first, lane);
        } else {
            consume<kMode>(a, P, s_pos);
            if (kMode == kSums) {
                named_sync(1, kThreads);  // every sub-tile sum of the range is written
                if (warp == 0)
                    sums_to_carries(a, s_first, s_etag);
            }
        }
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

static int prep_grid()
{
    static int g = 0;
    if (!g) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, delta_prep_kernel, kThreads, 0);
        g = sm_count() * (occ > 0 ? occ : 1);
    }
    return g;
}

// Arguments of a range-per-CTA pass over the control stream with at most
// max_grid CTAs; *grid receives the launch's CTA count (each has groups).
static OffsetsArgs offsets_args(const uint8_t *in, u64 in_len, u64 n, void *ws, u64 spin_limit,
                                u64 max_grid, u64 *grid)
{
    const WsLayout L = ws_layout(n);
    const u64 nquads = (n + 3) / 4;
    OffsetsArgs o;
    o.in = in;
    o.in_len = in_len;
    o.n = n;
    o.nquads = nquads;
    o.nsubs = (nquads + kSubQuads - 1) / kSubQuads;
    o.groups = (nquads + kOffGroupQuads - 1) / kOffGroupQuads;
    u64 ogrid = min(max_grid, o.groups);
    o.per_cta = (o.groups + ogrid - 1) / ogrid;
    *grid = (o.groups + o.per_cta - 1) / o.per_cta;  // no CTA without groups
    o.offs = reinterpret_cast<u64 *>(static_cast<char *>(ws) + L.offs);
    o.hdr = reinterpret_cast<WsHeader *>(ws);
    o.st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + L.status);
    o.spin_limit = spin_limit;
    o.in_aligned = (((uintptr_t)in) & 15u) == 0;
    o.prev = 0;
    o.carries = reinterpret_cast<u64 *>(static_cast<char *>(ws) + L.carries);
    return o;
}

// Offsets pass alone: sub-tile offsets, stream size and the truncation
// verdict into the workspace (the first half of launch_decode_tiled).
int launch_offsets(const uint8_t *in, u64 in_len, u64 n, void *ws, cudaStream_t stream,
                   u64 spin_limit)
{
    u64 grid = 0;
    const OffsetsArgs o = offsets_args(in, in_len, n, ws, spin_limit, offsets_grid(), &grid);
    prof_begin("offsets_kernel", stream);
    offsets_kernel<<<(unsigned)grid, kThreads, 0, stream>>>(o);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// Offsets and carry-ins of a differential stream in one launch; returns the
// sub-tiles per range (the carries are relative to ranges), 0 on failure.
static u64 launch_delta_prep(const uint8_t *in, u64 in_len, u64 n, uint32_t prev, void *ws,
                             cudaStream_t stream, u64 spin_limit)
{
    u64 grid = 0;
    OffsetsArgs o = offsets_args(in, in_len, n, ws, spin_limit, prep_grid(), &grid);
    o.prev = prev;
    prof_begin("delta_prep_kernel", stream);
    delta_prep_kernel<<<(unsigned)grid, kThreads, 0, stream>>>(o);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? o.per_cta * kOffGroupSubs : 0;
}

// After delta_prep_kernel run from 0: the stream's sum of coded values
// (mod 2^32) is the sum of its ranges' gap totals.  One warp writes out[0] =
// that sum, out[1] = the status, out[2] = the stream's bytes, and readies the
// workspace for the next launch as finish_launch does.
__global__ void gap_total_kernel(WsHeader *hdr, const TileStatus *st, u64 nranges,
                                 unsigned long long *out)
{
    uint32_t sum = 0;
    for (u64 i = threadIdx.x; i < nranges; i += 32)
        sum += (uint32_t)ld_relaxed(&st[i].val_agg);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (threadIdx.x == 0) {
        const u64 err = ld_relaxed(&hdr->error), total = ld_relaxed(&hdr->total);
        out[0] = err ? 0ull : sum;
        out[1] = err;
        out[2] = err ? ~0ull : total;
        st_relaxed(&hdr->error, 0);
        st_relaxed(&hdr->total, 0);
        st_relaxed(&hdr->tile_counter, 0);
        st_relaxed(&hdr->done_counter, 0);
        st_relaxed(&hdr->a_counter, 0);
        st_relaxed(&hdr->a_done, 0);
        st_relaxed(&hdr->epoch, ld_relaxed(&hdr->epoch) + 1);
    }
}

int launch_gap_sum(const uint8_t *in, u64 in_len, u64 n, void *ws, u64 *d_out,
                   cudaStream_t stream, u64 spin_limit)
{
    u64 grid = 0;
    OffsetsArgs o = offsets_args(in, in_len, n, ws, spin_limit, prep_grid(), &grid);
    o.prev = 0;
    prof_begin("delta_prep_kernel", stream);
    delta_prep_kernel<<<(unsigned)grid, kThreads, 0, stream>>>(o);
    prof_end(stream);
    gap_total_kernel<<<1, 32, 0, stream>>>(o.hdr, o.st, grid,
                                           reinterpret_cast<unsigned long long *>(d_out));
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

static TiledArgs tiled_args(const uint8_t *in, u64 n, uint32_t *out, uint32_t prev, void *ws,
                            DeviceResult *result, u64 spin_limit)
{
    const WsLayout L = ws_layout(n);
    const u64 nquads = (n + 3) / 4;
    TiledArgs t;
    t.in = in;
    t.n = n;
    t.nquads = nquads;
    t.ntiles = (nquads + kTileQuads - 1) / kTileQuads;
    t.nsubs = (nquads + kSubQuads - 1) / kSubQuads;
    t.out = out;
    t.offs = reinterpret_cast<u64 *>(static_cast<char *>(ws) + L.offs);
    t.carries = reinterpret_cast<u64 *>(static_cast<char *>(ws) + L.carries);
    t.hdr = reinterpret_cast<WsHeader *>(ws);
    t.st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + L.status);
    t.result = result;
    t.spin_limit = spin_limit;
    t.per_cta = 0;
    t.range_subs = 0;
    t.range_magic = 0;
    t.tile0 = 0;
    t.tile1 = t.ntiles;
    t.prev = prev;
    t.out_aligned = (((uintptr_t)out) & 15u) == 0;
    t.in_len = ~0ull;
    return t;
}

__global__ void set_claim_counter_kernel(WsHeader *hdr, u64 v)
{
    hdr->a_counter = v;
}

// Failure-detection check of the offsets pass's wait for earlier ranges'
// totals: the claim counter starts at 1, so the one CTA launched takes range
// 1 and waits for range 0's total, which no CTA publishes; the wait runs out
// after spin_limit polls and records SVB_ETIMEOUT.  A decode over all tiles
// follows: it sees the error, decodes nothing and readies the workspace
// (counters reset, epoch advanced) for the next call.
int launch_offsets_timeout_check(const uint8_t *in, u64 n, uint32_t *out, void *ws,
                                 DeviceResult *result, cudaStream_t stream, u64 spin_limit)
{
    u64 grid = 0;
    OffsetsArgs o = offsets_args(in, ~0ull, n, ws, spin_limit, 1, &grid);
    set_claim_counter_kernel<<<1, 1, 0, stream>>>(o.hdr, 1);
    offsets_kernel<<<1, kThreads, 0, stream>>>(o);
    TiledArgs t = tiled_args(in, n, out, 0, ws, result, spin_limit);
    const u64 g = max((u64)1, min((u64)tiled_grid<kPlain>(), t.ntiles));
    decode_tiled_kernel<kPlain><<<(unsigned)g, kDecBlock, sizeof(Pipe), stream>>>(t);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

u64 decode_tile_ints()
{
    return 4 * (u64)kTileQuads;
}

// Plain decode of the tiles [tile0, tile1) after launch_offsets; out is the
// whole array's output.  Each launch finishes the workspace's launch record,
// so give each its own result.
int launch_decode_range(const uint8_t *in, u64 n, uint32_t *out, void *ws, DeviceResult *result,
                        cudaStream_t stream, u64 tile0, u64 tile1)
{
    TiledArgs t = tiled_args(in, n, out, 0, ws, result, 0);
    t.tile0 = tile0;
    t.tile1 = min(tile1, t.ntiles);
    const u64 grid = max((u64)1, min((u64)tiled_grid<kPlain>(), t.tile1 - min(tile0, t.tile1)));
    prof_begin("decode_tiled_kernel<plain>", stream);
    decode_tiled_kernel<kPlain><<<(unsigned)grid, kDecBlock, sizeof(Pipe), stream>>>(t);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// The chunked single pass over a plain stream (the caller checked that
// in_len covers the control bytes).
int launch_decode_chunked(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, void *ws,
                          DeviceResult *result, cudaStream_t stream, u64 spin_limit)
{
    static int g = 0;
    if (!g) {
        cudaFuncSetAttribute(decode_chunked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Pipe));
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_chunked_kernel, kDcBlock,
                                                      sizeof(Pipe));
        g = sm_count() * (occ > 0 ? occ : 1);
    }
    TiledArgs t = tiled_args(in, n, out, 0, ws, result, spin_limit);
    t.in_len = in_len;
    const u64 nchunks = (t.ntiles + kDcTiles - 1) / kDcTiles;
    const u64 grid = max((u64)1, min((u64)g, nchunks));
    prof_begin("decode_chunked_kernel", stream);
    decode_chunked_kernel<<<(unsigned)grid, kDcBlock, sizeof(Pipe), stream>>>(t);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_decode_tiled(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                        bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                        u64 spin_limit, bool sums_pass)
{
    TiledArgs t = tiled_args(in, n, out, prev, ws, result, spin_limit);
    const u64 ntiles = t.ntiles;
    if (delta && !sums_pass) {
        // Offsets and carries in one pass, then the decode with carries.
        t.range_subs = launch_delta_prep(in, in_len, n, prev, ws, stream, spin_limit);
        if (!t.range_subs)
            return 3;
        const u64 range_tiles = t.range_subs / kSubs;  // >= 16: ranges are whole groups
        t.range_magic = ~0ull / range_tiles + 1;
        u64 grid = min((u64)tiled_grid<kDelta>(), ntiles);
        prof_begin("decode_tiled_kernel<delta>", stream);
        decode_tiled_kernel<kDelta><<<(unsigned)grid, kDecBlock, sizeof(Pipe), stream>>>(t);
        prof_end(stream);
        return cudaGetLastError() == cudaSuccess ? 0 : 3;
    }
    if (launch_offsets(in, in_len, n, ws, stream, spin_limit) != 0)
        return 3;
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
