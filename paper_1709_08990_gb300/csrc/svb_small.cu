// Stream VByte coding of small arrays (a few hundred tiles) in one launch.
//
// A small array is launch- and latency-bound: the tiled decoder's offsets
// pass and decode pass are two launches of a few microseconds of work each,
// and the single-pass decoder's tiles wait on a chain of look-backs.  Here
// one CTA takes one tile of 4096 integers (eight warps, one 512-integer
// sub-tile each) and the grid, launched cooperatively so that every CTA is
// resident, meets once at a barrier:
//   1. each warp sums its sub-tile's data bytes from the control bytes
//      (Sec. 4: a control byte covers 4 + the sum of its codes bytes), or,
//      encoding, sizes its coded values (Sec. 3: L(v) from the highest set
//      bit) and keeps them in registers; the CTA writes its tile's total;
//   2. grid barrier (one counter, every wait bounded);
//   3. each CTA sums the totals of the tiles before it, which gives its data
//      offset, then decodes its sub-tiles from shared memory (staged by
//      cp.async) or writes its encoded bytes.
// Nothing waits on a chain: the barrier is the only cross-CTA wait, and the
// values an encoder sizes are the values it writes (one read of the input).
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"
#include "svb_quad.cuh"
#include "svb_subenc.cuh"
#include "svb_subtile.cuh"

namespace svb {

constexpr int kSmTileQuads = kWarps * kSubQuads;    // 1024 quads: one sub-tile per warp
constexpr int kSmSlot = 16 * kSubQuads + 48;        // phase + 2048 data bytes + slack
constexpr u64 kSmPolls = 1ull << 22;                // bound on the grid barrier's wait

struct SmallArgs {
    const uint8_t *in;      // decode: the stream
    u64 in_len;
    const uint32_t *vals;   // encode: the integers
    uint8_t *enc_out;       // encode: the stream
    uint32_t *dec_out;      // decode: the integers
    u64 n, nquads;
    u64 *totals;            // one data-byte total per tile (workspace)
    WsHeader *hdr;
    DeviceResult *result;
    u64 spin_limit;
    uint32_t prev;
    uint32_t delta;
    uint32_t out_aligned;
};

// Data bytes of a sub-tile from its control word w (every lane): four quads
// per lane; the pad fields of the stream's last quad cover none.
__device__ __forceinline__ uint32_t small_subtile_bytes(const SubTile &t, uint32_t w)
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

// Steps 1-3's shared part: tile total `mine` published, the grid barrier,
// then the sum of the earlier tiles' totals (the tile's data offset, every
// thread).  The last tile writes the stream size and, decoding, the
// truncation verdict.  Ends with a CTA barrier.
__device__ u64 small_base(const SmallArgs &a, uint32_t mine, u64 *s_part, u64 *s_base)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u64 t = blockIdx.x;
    if (tid == 0) {
        st_relaxed(&a.totals[t], mine);
        __threadfence();
        atomicAdd(&a.hdr->a_counter, 1ull);
        bool ok = false;
        for (u64 i = 0; i < kSmPolls; i++) {
            if (ld_acquire(&a.hdr->a_counter) >= (u64)gridDim.x) {
                ok = true;
                break;
            }
            if ((i & 255) == 255 && error_raised(a.hdr))
                break;
            if (i > 8)
                __nanosleep(64);
        }
        if (!ok)
            raise_error(a.hdr, kErrTimeout);
    }
    __syncthreads();
    u64 part = 0;
    for (u64 i = tid; i < t; i += kThreads)
        part += ld_relaxed(&a.totals[i]);
    part = warp_sum64(part);
    if (lane == 0)
        s_part[warp] = part;
    __syncthreads();
    if (tid == 0) {
        u64 base = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++)
            base += s_part[w];
        *s_base = base;
        if (t + 1 == gridDim.x) {
            const u64 stream = a.nquads + base + mine;
            st_relaxed(&a.hdr->total, stream);
            if (a.in && stream > a.in_len)
                raise_error(a.hdr, kErrTruncated);
        }
    }
    __syncthreads();
    return *s_base;
}

__global__ void __launch_bounds__(kThreads) decode_small_kernel(SmallArgs a)
{
    __shared__ __align__(16) uint8_t s_slot[kWarps][kSmSlot];
    __shared__ __align__(16) uint16_t s_pos[kWarps][kSubQuads];
    __shared__ uint32_t s_sub[kWarps];
    __shared__ u64 s_part[kWarps], s_base;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u64 q0 = (u64)blockIdx.x * kSmTileQuads + (u64)warp * kSubQuads;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    SubTile t;
    t.C = a.in + q0;
    t.nq = q0 < a.nquads ? (uint32_t)min((u64)kSubQuads, a.nquads - q0) : 0u;
    t.tail = t.nq && q0 + t.nq == a.nquads ? last_nints : 4u;
    uint32_t w = 0, bytes = 0;
    if (t.nq) {
        w = subtile_ctrl_word(t);
        bytes = small_subtile_bytes(t, w);
    }
    if (lane == 0)
        s_sub[warp] = bytes;
    __syncthreads();
    uint32_t mine = 0, before = 0;
#pragma unroll
    for (int i = 0; i < kWarps; i++) {
        mine += s_sub[i];
        before += i < warp ? s_sub[i] : 0u;
    }
    const u64 base = small_base(a, mine, s_part, &s_base);
    if (t.nq) {  // (on a stream cut short the reads stop at in_len; the status says so)
        const uint8_t *g = a.in + a.nquads + base + before;
        const uintptr_t lo = (uintptr_t)a.in;
        const uintptr_t hi = a.in_len > ~(uintptr_t)0 - lo ? ~(uintptr_t)0 : lo + a.in_len;
        warp_stage(g, bytes, s_slot[warp], lo, hi, l2_policy_evict_first());
        cp_async_commit();
        t.D = s_slot[warp];
        t.base = (uint32_t)((uintptr_t)g & 15u);
        subtile_positions(t, w, s_pos[warp]);
        cp_async_wait<0>();
        __syncwarp();
        uint32_t v[kSubRounds][4];
        subtile_gather(t, s_pos[warp], v);
        uint32_t *op = a.dec_out + 4 * q0;
        const uint32_t m = (uint32_t)((uintptr_t)a.dec_out >> 2) & 3u;
#pragma unroll
        for (int r = 0; r < kSubRounds; r++) {
            const bool whole = subtile_nints(t, 32u * r + 31u) == 4u;
            const uint4 x = make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]);
            if (whole && a.out_aligned) {
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
    }
    finish_launch(a.hdr, a.result);
}

// Encoding: each warp loads and sizes its sub-tile's coded values (the gaps
// to the previous integer for differential coding, the first from prev or
// the integer before the tile), keeps them in registers across the barrier,
// then writes its control bytes and lays its data bytes end to end from the
// tile's data offset (the chunked encoder's per-warp sub-tile code).
__global__ void __launch_bounds__(kThreads) encode_small_kernel(SmallArgs a)
{
    __shared__ __align__(16) uint32_t s_slice[kWarps][kEncSliceWords];
    __shared__ uint32_t s_sub[kWarps];
    __shared__ u64 s_part[kWarps], s_base;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u64 q0 = (u64)blockIdx.x * kSmTileQuads;   // the tile's first quad
    const uint32_t sq0 = (uint32_t)warp * kSubQuads;
    const uint32_t nq = (uint32_t)min((u64)kSmTileQuads, a.nquads - q0);
    const uint32_t nvq = nq > sq0 ? min(nq - sq0, (uint32_t)kSubQuads) : 0u;
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));
    const uint32_t tail = q0 + nq == a.nquads ? last_nints : 4u;
    const uint32_t *V = a.vals + 4 * q0;
    const bool fast = 4 * (q0 + sq0 + kSubQuads) <= a.n;   // a whole sub-tile
    const bool aligned = ((uintptr_t)V & 15u) == 0;
    auto before = [&]() { return q0 == 0 ? a.prev : __ldg(a.vals + 4 * q0 - 1); };
    uint32_t nints[kEncRounds], d[kEncRounds][4], ctrl[kEncRounds], cb[kEncRounds];
    bool small = false;
    uint32_t bytes = 0;
    if (nvq) {
        if (fast && aligned) {
            subenc_values<true>(V, sq0, nq, tail, a.delta != 0, before, nints, d);
        } else if (fast) {
            subenc_values<true, decltype(before), false>(V, sq0, nq, tail, a.delta != 0, before,
                                                         nints, d);
        } else {
            subenc_values<false>(V, sq0, nq, tail, a.delta != 0, before, nints, d);
        }
        small = fast && subenc_all_small(d);
        if (!small)
            subenc_lengths<false>(nints, d, ctrl, cb);
        bytes = small ? 4u * kSubQuads : subenc_bytes(cb);
    }
    if (lane == 0)
        s_sub[warp] = bytes;
    __syncthreads();
    uint32_t mine = 0, prior = 0;
#pragma unroll
    for (int i = 0; i < kWarps; i++) {
        mine += s_sub[i];
        prior += i < warp ? s_sub[i] : 0u;
    }
    const u64 base = small_base(a, mine, s_part, &s_base);
    if (nvq) {
        uint8_t *dst = a.enc_out + a.nquads + base + prior;
        uint8_t *cdst = a.enc_out + q0 + sq0;
        if (small)
            subenc_write_small(s_slice[warp], cdst, dst, d);
        else if (fast)
            subenc_write<true>(s_slice[warp], cdst, dst, nvq, nints, ctrl, cb, d);
        else
            subenc_write<false>(s_slice[warp], cdst, dst, nvq, nints, ctrl, cb, d);
    }
    finish_launch(a.hdr, a.result);
}

// Cooperative launch of one of the kernels over `tiles` CTAs; 0, or 3 when
// the launch failed or cannot be made here (the grid would not be resident,
// or the stream is being captured), so that the caller takes another path.
template <class K>
static int launch_small(K kernel, const SmallArgs &a, u64 tiles, cudaStream_t stream,
                        const char *name)
{
    static int resident[2] = {0, 0};
    const int which = kernel == decode_small_kernel ? 0 : 1;
    if (!resident[which]) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, 0);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        resident[which] = (occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return 3;
    if (tiles == 0 || tiles > (u64)resident[which])
        return 3;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3((unsigned)tiles);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(name, stream);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, a);
    prof_end(stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 3;
    }
    return 0;
}

static SmallArgs small_args(u64 n, void *ws, DeviceResult *result, u64 spin_limit)
{
    SmallArgs a = {};
    a.n = n;
    a.nquads = (n + 3) / 4;
    a.totals = reinterpret_cast<u64 *>(static_cast<char *>(ws) + ws_layout(n).offs);
    a.hdr = reinterpret_cast<WsHeader *>(ws);
    a.result = result;
    a.spin_limit = spin_limit;
    return a;
}

u64 small_tiles(u64 n)
{
    return ((n + 3) / 4 + kSmTileQuads - 1) / kSmTileQuads;
}

int launch_decode_small(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, void *ws,
                        DeviceResult *result, cudaStream_t stream, u64 spin_limit)
{
    SmallArgs a = small_args(n, ws, result, spin_limit);
    a.in = in;
    a.in_len = in_len;
    a.dec_out = out;
    a.out_aligned = (((uintptr_t)out) & 15u) == 0;
    return launch_small(decode_small_kernel, a, small_tiles(n), stream, "decode_small_kernel");
}

int launch_encode_small(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta,
                        void *ws, DeviceResult *result, cudaStream_t stream, u64 spin_limit)
{
    SmallArgs a = small_args(n, ws, result, spin_limit);
    a.vals = in;
    a.enc_out = out;
    a.prev = prev;
    a.delta = delta ? 1u : 0u;
    return launch_small(encode_small_kernel, a, small_tiles(n), stream, "encode_small_kernel");
}

}  // namespace svb
