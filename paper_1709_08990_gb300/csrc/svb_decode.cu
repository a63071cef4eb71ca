// Stream VByte decoding on sm_103a, plain and differential, in one pass.
//
// What is computed (arXiv 1709.08990, Sec. 4 and Fig. 4): integer i has the
// 2-bit code c_i in control byte i/4 (bits 2(i mod 4)..), takes c_i + 1 data
// bytes, and its value is those bytes read least significant first (the
// shuffle of Sec. 2 zero-fills the high bytes).  Differential streams hold
// gaps; x_i = prev + sum of the first i gaps mod 2^32 (Sec. 2, Sec. 5).
//
// How (one CTA per tile of kQuadsPerTile control bytes = 4 * kQuadsPerTile
// integers; tiles taken in order from an atomic counter so that every tile's
// predecessors are already running):
//   1. load the tile's control bytes and sum the byte counts they imply
//      (per quad C = 4 + sum of codes, C in [4,16], Sec. 4), block scan
//      -> each quad's offset inside the tile and the tile's byte total;
//   2. decoupled look-back over the tiles' byte totals -> the tile's offset
//      in the data stream (the GPU form of the paper's pointer chain);
//   3. stage the tile's data bytes in shared memory with 16-byte loads;
//   4. each lane decodes one quad per round (lanes take consecutive quads, so
//      each warp store writes 512 contiguous bytes); an all-zero control byte
//      in every lane of a warp takes a byte-widening fast path (Sec. 4: the
//      paper special-cases zero control bytes);
//   5. differential: quad, warp and block prefix sums plus a second look-back
//      over the tiles' gap sums give each value its running sum.
// Nothing outside the stream is read: partial 16-byte chunks at the ends of a
// tile's data range are read byte by byte.  Pad fields of an incomplete last
// control byte are masked to zero and contribute no bytes.
#include <cuda_runtime.h>

#include "svb_device.cuh"
#include "svb_internal.h"

namespace svb {

constexpr int kDecQuads = 1024;                     // quads per tile (4096 ints)
constexpr int kDecRounds = kDecQuads / kThreads;    // quads per lane
constexpr int kDecDataMax = 16 * kDecQuads;         // bytes of data per tile, at most
constexpr int kDecStage = kDecDataMax + 64;         // 16-byte head skew + slack for 2-word reads
constexpr int kDecChunks = (kDecDataMax + 16 + 15) / 16;
constexpr int kDecChunkIters = (kDecChunks + kThreads - 1) / kThreads;

struct DecodeArgs {
    const uint8_t *in;
    u64 in_len;      // readable bytes of in
    u64 n;           // integers
    uint32_t *out;
    u64 nquads;      // ceil(n / 4) = control bytes
    u64 ntiles;
    WsHeader *hdr;
    TileStatus *st;
    DeviceResult *result;
    u64 spin_limit;
    u64 tile_base;   // 0 except in the look-back timeout check
    uint32_t prev;
    uint32_t out_aligned;  // out is 16-byte aligned
};

__device__ __forceinline__ uint32_t quad_bytes(uint32_t c, uint32_t nints)
{
    // Sec. 4: C = number of integers + sum of their codes.
    return nints + __popc(c & 0x55u) + 2u * __popc(c & 0xAAu);
}

// Value of the integer at byte p of the staged tile, taking code + 1 bytes.
__device__ __forceinline__ uint32_t extract(const uint32_t *s32, uint32_t p, uint32_t code)
{
    uint32_t w0 = s32[p >> 2], w1 = s32[(p >> 2) + 1];
    uint32_t v = __funnelshift_r(w0, w1, (p & 3u) * 8u);
    return v & (0xffffffffu >> (24u - 8u * code));
}

template <bool kDelta>
__global__ void __launch_bounds__(kThreads, 4) decode_kernel(DecodeArgs a)
{
    __shared__ __align__(16) uint8_t s_data[kDecStage];
    __shared__ __align__(16) uint32_t s_ctrl[kDecQuads / 4];
    __shared__ __align__(16) uint16_t s_qoff[kDecQuads];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ u64 s_tile, s_etag, s_base;
    __shared__ uint32_t s_skip, s_carry;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        s_tile = atomicAdd(&a.hdr->tile_counter, 1ull) + a.tile_base;
        s_etag = epoch_tag(a.hdr);
        s_skip = (s_tile >= a.ntiles || error_raised(a.hdr)) ? 1u : 0u;
    }
    __syncthreads();
    const u64 tile = s_tile, etag = s_etag;
    if (s_skip) {
        finish_launch(a.hdr, a.result);
        return;
    }

    // ---- 1. control bytes -> per-quad byte counts and offsets ------------
    const u64 q0 = tile * kDecQuads;
    const uint32_t nq = (uint32_t)min((u64)kDecQuads, a.nquads - q0);
    const uint32_t last_nints = (uint32_t)(a.n - 4 * (a.nquads - 1));  // 1..4
    const uint8_t *cp = a.in + q0;
    uint32_t w = 0;
    if (4u * tid + 4u <= nq && (((uintptr_t)cp) & 3u) == 0) {
        w = __ldg(reinterpret_cast<const uint32_t *>(cp) + tid);
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (4u * tid + j < nq)
                w |= (uint32_t)__ldg(cp + 4 * tid + j) << (8 * j);
    }
    uint32_t cnt[4], S = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        uint32_t lq = 4u * tid + j;
        uint32_t c = (w >> (8 * j)) & 0xffu;
        uint32_t nints = 4;
        if (q0 + lq == a.nquads - 1 && last_nints < 4) {
            nints = last_nints;
            c &= (1u << (2 * nints)) - 1u;  // pad fields carry no bytes
            w = (w & ~(0xffu << (8 * j))) | (c << (8 * j));
        }
        cnt[j] = lq < nq ? quad_bytes(c, nints) : 0u;
        S += cnt[j];
    }
    s_ctrl[tid] = w;
    uint32_t incl = warp_incl_scan(S);
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0, agg = 0;
#pragma unroll
    for (int k = 0; k < kWarps; k++) {
        uint32_t t = s_warp[k];
        wpre += k < warp ? t : 0u;
        agg += t;
    }
    {
        uint32_t e = wpre + incl - S;
        uint32_t o0 = e, o1 = o0 + cnt[0], o2 = o1 + cnt[1], o3 = o2 + cnt[2];
        uint2 packed = make_uint2(o0 | (o1 << 16), o2 | (o3 << 16));
        reinterpret_cast<uint2 *>(s_qoff)[tid] = packed;
    }

    // ---- 2. tile offset in the data stream (look-back) -------------------
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
            uint32_t skip = 0;
            if (!ok) {
                raise_error(a.hdr, kErrTimeout);
                skip = 1;
            } else if (a.nquads + base + agg > a.in_len) {
                raise_error(a.hdr, kErrTruncated);
                skip = 1;
            } else if (tile == a.ntiles - 1) {
                st_relaxed(&a.hdr->total, a.nquads + base + agg);
            }
            s_base = base;
            s_skip = skip;
        }
    }
    __syncthreads();
    if (s_skip) {
        finish_launch(a.hdr, a.result);
        return;
    }

    // ---- 3. stage the tile's data bytes ----------------------------------
    const uint8_t *src = a.in + a.nquads + s_base;
    const uint32_t h = (uint32_t)((uintptr_t)src & 15u);
    const uint8_t *asrc = src - h;
    const uint32_t nchunks = (h + agg + 15u) >> 4;
    {
        uint4 r[kDecChunkIters];
#pragma unroll
        for (int i = 0; i < kDecChunkIters; i++) {
            uint32_t k = tid + i * kThreads;
            if (k < nchunks && 16u * k >= h && 16u * k + 16u <= h + agg)
                r[i] = ldg_stream128(asrc + 16u * k);
        }
#pragma unroll
        for (int i = 0; i < kDecChunkIters; i++) {
            uint32_t k = tid + i * kThreads;
            if (k < nchunks) {
                if (16u * k >= h && 16u * k + 16u <= h + agg) {
                    *reinterpret_cast<uint4 *>(s_data + 16u * k) = r[i];
                } else {
                    for (uint32_t b = 0; b < 16; b++) {
                        uint32_t idx = 16u * k + b;
                        if (idx >= h && idx < h + agg)
                            s_data[idx] = __ldg(asrc + idx);
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---- 4. decode: one quad per lane per round --------------------------
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(s_data);
    const uint8_t *sctrl = reinterpret_cast<const uint8_t *>(s_ctrl);
    uint32_t v[kDecRounds][4];
#pragma unroll
    for (int r = 0; r < kDecRounds; r++) {
        const uint32_t lq = warp * (32 * kDecRounds) + r * 32 + lane;
        const bool valid = lq < nq;
        const uint32_t c = valid ? sctrl[lq] : 0u;
        const uint32_t p = h + (valid ? s_qoff[lq] : 0u);
        if (__all_sync(0xffffffffu, c == 0)) {
            // Four one-byte integers: widen the four bytes at p.
            uint32_t d = __funnelshift_r(s32[p >> 2], s32[(p >> 2) + 1], (p & 3u) * 8u);
            v[r][0] = __byte_perm(d, 0, 0x4440);
            v[r][1] = __byte_perm(d, 0, 0x4441);
            v[r][2] = __byte_perm(d, 0, 0x4442);
            v[r][3] = __byte_perm(d, 0, 0x4443);
        } else {
            uint32_t q = p;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uint32_t code = (c >> (2 * k)) & 3u;
                v[r][k] = extract(s32, q, code);
                q += code + 1;
            }
        }
        const uint32_t nints = !valid ? 0u : (q0 + lq == a.nquads - 1 ? last_nints : 4u);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if ((uint32_t)k >= nints)
                v[r][k] = 0;
        if (!kDelta && valid) {
            uint32_t *dst = a.out + 4 * (q0 + lq);
            if (nints == 4 && a.out_aligned)
                stg_stream128(dst, make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]));
            else
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if ((uint32_t)k < nints)
                        dst[k] = v[r][k];
        }
    }

    if (kDelta) {
        // ---- 5. running sums: quad, round (warp), block, tiles -----------
        uint32_t qexcl[kDecRounds], wrun = 0;
#pragma unroll
        for (int r = 0; r < kDecRounds; r++) {
            v[r][1] += v[r][0];
            v[r][2] += v[r][1];
            v[r][3] += v[r][2];
            uint32_t qs = v[r][3];
            uint32_t inc = warp_incl_scan(qs);
            qexcl[r] = wrun + inc - qs;
            wrun += __shfl_sync(0xffffffffu, inc, 31);
        }
        __syncthreads();  // s_warp reuse
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
            bool ok = true;
            if (tile == 0) {
                if (lane == 0)
                    publish(&me->val_tag, &me->val_pre, (uint32_t)(a.prev + vagg), kFlagPrefix,
                            etag);
            } else {
                if (lane == 0)
                    publish(&me->val_tag, &me->val_agg, vagg, kFlagAgg, etag);
                carry = lookback<true>(a.st, tile, etag, a.spin_limit, a.hdr, ok);
                if (ok && lane == 0)
                    publish(&me->val_tag, &me->val_pre, (uint32_t)(carry + vagg), kFlagPrefix,
                            etag);
            }
            if (lane == 0) {
                if (!ok)
                    raise_error(a.hdr, kErrTimeout);
                s_carry = (uint32_t)carry;
                s_skip = ok ? 0u : 1u;
            }
        }
        __syncthreads();
        if (!s_skip) {
            const uint32_t base = s_carry + bpre;
#pragma unroll
            for (int r = 0; r < kDecRounds; r++) {
                const uint32_t lq = warp * (32 * kDecRounds) + r * 32 + lane;
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
    }
    finish_launch(a.hdr, a.result);
}

int launch_decode(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                  bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                  u64 spin_limit, u64 tile_base, u64 grid_override)
{
    DecodeArgs a;
    a.in = in;
    a.in_len = in_len;
    a.n = n;
    a.out = out;
    a.nquads = (n + 3) / 4;
    a.ntiles = (a.nquads + kDecQuads - 1) / kDecQuads;
    a.hdr = reinterpret_cast<WsHeader *>(ws);
    a.st = reinterpret_cast<TileStatus *>(static_cast<char *>(ws) + ws_layout(n).status);
    a.result = result;
    a.spin_limit = spin_limit;
    a.tile_base = tile_base;
    a.prev = prev;
    a.out_aligned = (((uintptr_t)out) & 15u) == 0;
    dim3 grid((unsigned)(grid_override ? grid_override : a.ntiles));
    prof_begin(delta ? "decode_kernel<delta>" : "decode_kernel<plain>", stream);
    if (delta)
        decode_kernel<true><<<grid, kThreads, 0, stream>>>(a);
    else
        decode_kernel<false><<<grid, kThreads, 0, stream>>>(a);
    prof_end(stream);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

u64 decode_tiles(u64 n)
{
    u64 nq = (n + 3) / 4;
    return (nq + kDecQuads - 1) / kDecQuads;
}

}  // namespace svb
