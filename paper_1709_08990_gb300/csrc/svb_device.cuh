// Device-side building blocks shared by the Stream VByte kernels:
// the workspace layout, tile-status records, ordered loads and stores, warp
// and block scans, and the bounded decoupled look-back that turns per-tile
// aggregates into exclusive prefixes in one pass.
//
// The paper's decoder walks the stream serially: each control byte tells how
// far the data pointer moves (Sec. 4, Fig. 4), the dependency that Sec. 4
// names as the reason varint-GB resists vectorisation.  On the
// GPU that chain becomes a prefix sum of the per-quad byte counts over the
// whole stream; tiles compute their own sums from their control bytes and
// chain them with a decoupled look-back (a single-pass scan: each tile
// publishes its aggregate early and sums its predecessors' published values).
#pragma once

#include <cstddef>
#include <cstdint>

namespace svb {

typedef unsigned long long u64;

constexpr int kThreads = 256;                      // threads per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kMinQuadsPerTile = 256;              // workspace sizing unit (tile records)
constexpr int kSubQuads = 128;                     // sub-tile: the quads one warp decodes

// Status word low bits: what the tile has published.
constexpr u64 kFlagNone = 0, kFlagAgg = 1, kFlagPrefix = 2;
// Set in every tag, never in any other word the kernels store in a workspace.
constexpr u64 kTagMark = 1ull << 63;

// Error codes written to the workspace (same values as svb_status).
constexpr u64 kErrTruncated = 2, kErrTimeout = 4;

// One tile's published values.  Each scan has a tag word and two slots; a
// reader that has seen a tag reads a slot that is written once per launch
// and before the tag, so it never sees a half-updated record.  The tag is
// kTagMark | ((epoch + 1) << 2) | flag: records left by earlier launches on
// the same workspace never match, so the array is zeroed only once.  Where
// the records lie depends on n (ws_layout), so a call may find in a record's
// place the words an earlier call of another size or kind left there:
// sub-tile offsets and byte totals (below 2^48), carries and gap sums
// (stored zero-extended, below 2^32) or older tags.  None of those has bit
// 63 set together with this launch's epoch, so none reads as ready.
struct __align__(64) TileStatus {
    u64 off_tag, off_agg, off_pre;   // data-stream byte offsets
    u64 val_tag, val_agg, val_pre;   // running sum of deltas (mod 2^32)
    u64 pad0, pad1;
};

// Workspace layout (see ws_layout): [header 128 B][result 16 B, padded to
// 128 B][tile offsets: u64 x (tiles + 1)][TileStatus x tiles]
struct __align__(128) WsHeader {
    u64 tile_counter;   // next dynamic tile id (the decode or encode kernel)
    u64 done_counter;   // CTAs that have finished this launch
    u64 epoch;          // launches finished on this workspace
    u64 error;          // first error of this launch, 0 if none
    u64 total;          // stream size, written by the last tile
    u64 a_counter;      // dynamic CTA id of the offsets pass
    u64 a_done;         // CTAs of the offsets pass that have finished
    u64 pad[9];
};

constexpr size_t kResultOffset = 128;
constexpr size_t kOffsetsOffset = 256;

struct WsLayout {
    size_t offs;     // byte offset of the tile-offset array (u64 x tiles + 1)
    size_t carries;  // byte offset of the per-sub-tile carry array (u64 x subs, zero-extended)
    size_t status;   // byte offset of the TileStatus array
    size_t total;    // workspace bytes
};

// Layout for up to `subs` sub-tiles (offsets and carries, one per kSubQuads
// quads) and `tiles` tile records (one per kMinQuadsPerTile quads or more).
constexpr WsLayout ws_layout_for(u64 subs, u64 tiles)
{
    WsLayout l{};
    l.offs = kOffsetsOffset;
    l.carries = (l.offs + 8 * (subs + 1) + 63) & ~(size_t)63;
    l.status = (l.carries + 8 * (subs ? subs : 1) + 63) & ~(size_t)63;
    l.total = l.status + sizeof(TileStatus) * (tiles ? tiles : 1);
    return l;
}

constexpr WsLayout ws_layout(u64 n)
{
    const u64 nq = (n + 3) / 4;
    return ws_layout_for((nq + kSubQuads - 1) / kSubQuads,
                         (nq + kMinQuadsPerTile - 1) / kMinQuadsPerTile);
}

struct DeviceResult {
    u64 bytes;
    u64 status;
};

// ---- ordered global accesses (GPU scope) ---------------------------------

__device__ __forceinline__ u64 ld_acquire(const u64 *p)
{
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u64 ld_relaxed(const u64 *p)
{
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(u64 *p, u64 v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(u64 *p, u64 v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tag base of the running launch (see TileStatus): or a flag into it.
__device__ __forceinline__ u64 epoch_tag(const WsHeader *h)
{
    return kTagMark | ((ld_relaxed(&h->epoch) + 1) << 2);
}

// Read-only, not-allocating-in-L1 loads of the compressed input.
__device__ __forceinline__ uint4 ldg_stream128(const void *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Output stores that should not linger in L2 (evict-first).
__device__ __forceinline__ void stg_stream128(void *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// One round of a warp's decoded quads (lane l: the four integers of quad l,
// bound for dst + 4l) stored with 16-byte writes although dst is only 4-byte
// aligned: m = (dst / 4) mod 4 in {1, 2, 3}.  The aligned chunk that ends
// with lane l's first 4 - m integers takes its first m from lane l - 1 (one
// shuffle per integer); lane 0 writes its first 4 - m integers and lane 31
// its last m one by one, which the neighbouring rounds' chunks leave out.
// Every lane of the warp must call it, with the same dst and m.
__device__ __forceinline__ void stg_round_realigned(uint32_t *dst, uint4 v, uint32_t m)
{
    const int lane = threadIdx.x & 31;
    const uint32_t p1 = __shfl_up_sync(0xffffffffu, v.y, 1);
    const uint32_t p2 = __shfl_up_sync(0xffffffffu, v.z, 1);
    const uint32_t p3 = __shfl_up_sync(0xffffffffu, v.w, 1);
    uint32_t *own = dst + 4 * lane;
    uint4 c;
    if (m == 1)
        c = make_uint4(p3, v.x, v.y, v.z);
    else if (m == 2)
        c = make_uint4(p2, p3, v.x, v.y);
    else
        c = make_uint4(p1, p2, p3, v.x);
    if (lane > 0)
        stg_stream128(own - m, c);
    if (lane == 0) {
        own[0] = v.x;
        if (m < 3)
            own[1] = v.y;
        if (m < 2)
            own[2] = v.z;
    }
    if (lane == 31) {
        own[3] = v.w;
        if (m > 1)
            own[2] = v.z;
        if (m > 2)
            own[1] = v.y;
    }
}

__device__ __forceinline__ void raise_error(WsHeader *h, u64 code)
{
    atomicCAS(&h->error, 0ull, code);
}

__device__ __forceinline__ bool error_raised(const WsHeader *h)
{
    return ld_relaxed(&h->error) != 0;
}

// ---- scans ---------------------------------------------------------------

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d)
            v += t;
    }
    return v;
}

__device__ __forceinline__ u64 warp_sum64(u64 v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// ---- decoupled look-back ---------------------------------------------------

// Publish one value of a scan: slot first, then the tag with release order.
__device__ __forceinline__ void publish(u64 *tag, u64 *slot, u64 value, u64 flag, u64 etag)
{
    st_relaxed(slot, value);
    st_release(tag, etag | flag);
}

constexpr int kLookbackPerLane = 8;  // predecessors each lane inspects per round trip

__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Exclusive prefix of tile `tile` (> 0) for one scan (kVal: the delta running
// sum, else the byte offsets), computed by one whole warp.  One round trip
// inspects a window of 32 * kLookbackPerLane predecessors (lane l owns the
// run of kLookbackPerLane tiles starting l * kLookbackPerLane tiles back,
// nearest first).  Only the tiles nearer than the window's nearest published
// inclusive prefix matter: while one of them has published nothing yet, those
// (and only those) are polled again; then the window is summed up to that
// prefix, or wholly when it holds none, and the next window is taken.  The
// tag loads are relaxed and independent, so they are in flight together; one
// acquire fence after the tags that matter are valid orders the value loads
// after them (a release store of the tag, a relaxed load that sees it and an
// acquire fence synchronise).  Every wait is bounded: after spin_limit polling
// rounds (backing off to ~0.25 us each), or as soon as another tile has raised
// an error, it returns with ok = false and the caller records the failure.
template <bool kVal>
__device__ u64 lookback(TileStatus *st, u64 tile, u64 etag, u64 spin_limit, WsHeader *hdr,
                        bool &ok)
{
    constexpr int K = kLookbackPerLane;
    constexpr int kWindow = 32 * K;
    const int lane = threadIdx.x & 31;
    u64 excl = 0;
    long long base = (long long)tile - 1;
    u64 spins = 0;
    ok = true;
    auto tag_of = [&](long long p) -> const u64 * {
        return kVal ? &st[p].val_tag : &st[p].off_tag;
    };
    for (;;) {
        u64 tags[K];
#pragma unroll
        for (int j = 0; j < K; j++) {
            const long long p = base - (lane * K + j);
            tags[j] = p >= 0 ? ld_relaxed(tag_of(p)) : (etag | kFlagPrefix);
        }
        int ppos, npos;  // window positions of the nearest prefix / not-ready tile
        for (;;) {
            int pk = K, nk = K;
#pragma unroll
            for (int j = K - 1; j >= 0; j--) {
                const bool ready = (tags[j] & ~3ull) == etag && (tags[j] & 3ull) != kFlagNone;
                if (!ready)
                    nk = j;
                if (ready && (tags[j] & 3ull) == kFlagPrefix)
                    pk = j;
            }
            const unsigned pm = __ballot_sync(0xffffffffu, pk < K);
            const unsigned nm = __ballot_sync(0xffffffffu, nk < K);
            const int pl = pm ? __ffs(pm) - 1 : 0, nl = nm ? __ffs(nm) - 1 : 0;
            const int pk_l = __shfl_sync(0xffffffffu, pk, pl);
            const int nk_l = __shfl_sync(0xffffffffu, nk, nl);
            ppos = pm ? pl * K + pk_l : kWindow;
            npos = nm ? nl * K + nk_l : kWindow;
            if (npos > ppos || npos == kWindow)
                break;  // every tile nearer than the prefix (or in the window) is ready
            if (++spins > spin_limit || ((spins & 31) == 0 && error_raised(hdr))) {
                ok = false;
                return 0;
            }
            if (spins > 4)
                __nanosleep(spins < 64 ? 32 : 256);
#pragma unroll
            for (int j = 0; j < K; j++) {
                const long long p = base - (lane * K + j);
                const bool ready = (tags[j] & ~3ull) == etag && (tags[j] & 3ull) != kFlagNone;
                if (p >= 0 && !ready && lane * K + j < ppos)
                    tags[j] = ld_relaxed(tag_of(p));
            }
        }
        fence_acq_rel_gpu();
        u64 sum = 0;
#pragma unroll
        for (int j = 0; j < K; j++) {
            const long long p = base - (lane * K + j);
            if (p >= 0 && lane * K + j <= ppos) {
                const bool pre = (tags[j] & 3ull) == kFlagPrefix;
                sum += ld_relaxed(kVal ? (pre ? &st[p].val_pre : &st[p].val_agg)
                                       : (pre ? &st[p].off_pre : &st[p].off_agg));
            }
        }
        excl += warp_sum64(sum);
        if (ppos < kWindow)
            break;
        base -= kWindow;
    }
    return kVal ? (excl & 0xffffffffull) : excl;
}

// The last CTA to finish writes the launch's result and readies the
// workspace for the next launch (counters to zero, epoch + 1).
__device__ __forceinline__ void finish_launch(WsHeader *hdr, DeviceResult *result)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        u64 done = atomicAdd(&hdr->done_counter, 1ull);
        if (done == (u64)gridDim.x - 1) {
            __threadfence();
            u64 err = ld_relaxed(&hdr->error);
            u64 total = ld_relaxed(&hdr->total);
            result->bytes = err ? ~0ull : total;
            result->status = err;
            st_relaxed(&hdr->error, 0);
            st_relaxed(&hdr->total, 0);
            st_relaxed(&hdr->tile_counter, 0);
            st_relaxed(&hdr->done_counter, 0);
            st_relaxed(&hdr->a_counter, 0);
            st_relaxed(&hdr->a_done, 0);
            st_relaxed(&hdr->epoch, ld_relaxed(&hdr->epoch) + 1);
        }
    }
}

// ---- bulk asynchronous copies (TMA engine) and mbarriers -----------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk-copy accesses (async proxy) that are ordered after it through an
// mbarrier: a stage's readers issue it before they release the stage, so the
// copy that refills the stage cannot overtake their loads.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, u64 limit)
{
    for (u64 i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (i > 64)
            __nanosleep(64);
    }
    return false;
}

// As mbar_wait_bounded, but each poll may suspend the thread for up to
// `hint_ns` (it resumes as soon as the phase completes), so a long wait costs
// few instructions.  At most limit * hint_ns in all.
__device__ __forceinline__ bool mbar_wait_suspend(uint64_t *bar, uint32_t parity, u64 limit,
                                                  uint32_t hint_ns)
{
    for (u64 i = 0; i < limit; i++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok)
            return true;
    }
    return false;
}

// Barrier among the first `count` threads of the CTA (named barrier `id`).
__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Global -> shared bulk copy completing on an mbarrier.  dst and src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// L2 eviction priority for a bulk copy's source lines.
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bulk_g2s with an L2 cache policy for the source.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// ---- per-thread asynchronous copies (cp.async) ----------------------------

// 16 bytes global -> shared, both 16-byte aligned, the source lines kept in
// L2 with the given eviction policy; completes with cp_async_wait.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint64_t policy)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                 "l"(src), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait until at most `kPending` of this thread's committed groups are in flight.
template <int kPending>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

}  // namespace svb
