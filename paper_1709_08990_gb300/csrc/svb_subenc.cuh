// Encoding one warp's sub-tile (kSubQuads = 128 quads, 512 values) of a
// staged tile, shared by the single-stream and the batched encoders.
//
// subenc_load: each lane takes one quad per round (quad 32r + lane of the
// sub-tile): its integers, their coded values (the gaps to the previous
// integer for differential coding, Sec. 1 and Sec. 5), each value's length
// L(v) - 1 from the index of its highest set bit (Sec. 3), the control byte
// (first integer in the low bits, Fig. 3) and the quad's data bytes.
//
// subenc_write: control bytes go straight to global memory; the data bytes
// are laid end to end (Sec. 4) in the warp's shared slice at the phase of
// their destination - each lane shifts its quad's 4..16 bytes to their byte
// position with funnel shifts, writes the words it completes and passes its
// partial last word to the next lane - and the slice goes out with 16-byte
// streaming stores (ragged ends byte by byte).
#pragma once

#include <cstdint>

#include "svb_device.cuh"

namespace svb {

constexpr int kEncRounds = kSubQuads / 32;                  // quads per lane per sub-tile
// One warp's data bytes (at most 16 per quad) at a phase of up to 15 bytes,
// rounded to 16-byte chunks, plus a spare word no data byte reaches.
constexpr int kEncSliceWords = (16 * kSubQuads + 32) / 4;

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

// The sub-tile starting at tile-local quad sq0 of a staged tile of nq quads
// whose values are V (V[4q + j] = integer j of quad q); tail = integers in
// quad nq - 1 (4 unless it ends the stream).  For differential coding,
// before() gives the integer preceding the tile (called by lane 0 only, when
// sq0 == 0; otherwise the preceding integer is V[4 * sq0 - 1]).  kFast: all
// 128 quads hold 4 integers.  kAligned: V is 16-byte aligned (a quad is one
// 16-byte load; else four 4-byte loads).  Out: per round the
// integers of the lane's quad (0 past the end), the coded values (0 past the
// end), the control byte (left 0 with kSizeOnly, when only sizes are
// needed) and the quad's data bytes.
template <bool kFast, class Before, bool kAligned = true>
__device__ __forceinline__ void subenc_values(const uint32_t *V, uint32_t sq0, uint32_t nq,
                                              uint32_t tail, bool delta, Before before,
                                              uint32_t (&nints)[kEncRounds],
                                              uint32_t (&d)[kEncRounds][4])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < kEncRounds; r++) {
        const uint32_t lq = sq0 + 32 * r + lane;
        nints[r] = kFast ? 4u : (lq >= nq ? 0u : (lq == nq - 1 ? tail : 4u));
        if (kFast) {
            const uint4 v = kAligned
                ? *reinterpret_cast<const uint4 *>(V + 4 * lq)
                : make_uint4(V[4 * lq], V[4 * lq + 1], V[4 * lq + 2], V[4 * lq + 3]);
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
    if (delta) {
        uint32_t carry = 0;  // integer before the lane's first one, in lane 0
        if (lane == 0 && nints[0])
            carry = sq0 ? V[4 * sq0 - 1] : before();
#pragma unroll
        for (int r = 0; r < kEncRounds; r++) {
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

// Control bytes and byte counts of the coded values d (see subenc_load).
template <bool kSizeOnly = false>
__device__ __forceinline__ void subenc_lengths(const uint32_t (&nints)[kEncRounds],
                                               const uint32_t (&d)[kEncRounds][4],
                                               uint32_t (&ctrl)[kEncRounds],
                                               uint32_t (&cb)[kEncRounds])
{
    // Fields past the end are 0 and add nothing.
#pragma unroll
    for (int r = 0; r < kEncRounds; r++) {
        uint32_t c = 0, C = nints[r];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t e = extra_bytes(d[r][j]);
            if (!kSizeOnly)
                c |= e << (2 * j);
            C += e;
        }
        ctrl[r] = c;   // kSizeOnly: 0, only the byte counts are needed
        cb[r] = C;
    }
}

template <bool kFast, class Before, bool kSizeOnly = false, bool kAligned = true>
__device__ __forceinline__ void subenc_load(const uint32_t *V, uint32_t sq0, uint32_t nq,
                                            uint32_t tail, bool delta, Before before,
                                            uint32_t (&nints)[kEncRounds],
                                            uint32_t (&d)[kEncRounds][4],
                                            uint32_t (&ctrl)[kEncRounds],
                                            uint32_t (&cb)[kEncRounds])
{
    subenc_values<kFast, Before, kAligned>(V, sq0, nq, tail, delta, before, nints, d);
    subenc_lengths<kSizeOnly>(nints, d, ctrl, cb);
}

// Whether every coded value of the warp's sub-tile takes one byte (Sec. 3:
// below 2^8); fields past the end are 0.
__device__ __forceinline__ bool subenc_all_small(const uint32_t (&d)[kEncRounds][4])
{
    uint32_t o = 0;
#pragma unroll
    for (int r = 0; r < kEncRounds; r++)
        o |= d[r][0] | d[r][1] | d[r][2] | d[r][3];
    return __all_sync(0xffffffffu, o < 256u);
}

// Data bytes of the sub-tile (all lanes), from subenc_load's byte counts.
__device__ __forceinline__ uint32_t subenc_bytes(const uint32_t (&cb)[kEncRounds])
{
    uint32_t t = 0;
#pragma unroll
    for (int r = 0; r < kEncRounds; r++)
        t += cb[r];
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1)
        t += __shfl_xor_sync(0xffffffffu, t, k);
    return t;
}

// Stores the warp's data bytes [h, h + run) of slice (phased like dst) to
// dst: 16-byte streaming stores, ragged ends byte by byte.
__device__ __forceinline__ void subenc_flush(uint32_t *slice, uint8_t *dst, uint32_t h, uint32_t run)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const uint8_t *sb = reinterpret_cast<const uint8_t *>(slice);
    uint8_t *adst = dst - h;
    const uint32_t end = h + run;
    const uint32_t c0 = (h + 15) >> 4, c1 = end >> 4;   // whole 16-byte chunks [c0, c1)
#pragma unroll
    for (int k = 0; k < (kEncSliceWords * 4 / 16 + 31) / 32; k++) {
        const uint32_t c = c0 + lane + 32 * k;
        if (c < c1)
            stg_stream128(adst + 16 * c, *reinterpret_cast<const uint4 *>(sb + 16 * c));
    }
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

// Writes the sub-tile's nvq quads: control byte of quad i to ctrl_dst[i],
// data bytes to dst onward; slice is the warp's shared scratch
// (kEncSliceWords words, 16-byte aligned).
template <bool kFast>
__device__ __forceinline__ void subenc_write(uint32_t *slice, uint8_t *ctrl_dst, uint8_t *dst,
                                             uint32_t nvq_any,
                                             const uint32_t (&nints)[kEncRounds],
                                             const uint32_t (&ctrl)[kEncRounds],
                                             const uint32_t (&cb)[kEncRounds],
                                             const uint32_t (&d)[kEncRounds][4])
{
    constexpr uint32_t kNone = 0xffffffffu;
    constexpr uint32_t kSpare = kEncSliceWords - 1;   // never holds data bytes
    const int lane = threadIdx.x & 31;
    const uint32_t h = (uint32_t)((uintptr_t)dst & 15u);
    const uint32_t nvq = kFast ? (uint32_t)kSubQuads : nvq_any;
    uint32_t run = 0, carry = 0, fidx = kNone, fword = 0;
#pragma unroll
    for (int r = 0; r < kEncRounds; r++) {
        if (32u * r >= nvq)
            break;
        const uint32_t lq = 32 * r + lane;
        const uint32_t C = cb[r];
        const uint32_t nint = kFast ? 4u : nints[r];
        uint32_t L[4];
#pragma unroll
        for (int j = 0; j < 4; j++)
            L[j] = (uint32_t)j < nint ? ((ctrl[r] >> (2 * j)) & 3u) + 1 : 0u;
        if (nint)
            ctrl_dst[lq] = (uint8_t)ctrl[r];
        const uint32_t inc = warp_incl_scan(C);
        const uint32_t pos = h + run + inc - C;
        run += __shfl_sync(0xffffffffu, inc, 31);
        // The quad's bytes end to end, then moved to their phase in a word.
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
        const uint32_t last = nfull == 0 ? t0 : nfull == 1 ? t1 : nfull == 2 ? t2
                                                : nfull == 3 ? t3 : t4;
        uint32_t pt = __shfl_up_sync(0xffffffffu, last, 1);
        if (lane == 0)
            pt = carry;
        carry = __shfl_sync(0xffffffffu, last, 31);
        const uint32_t w0 = t0 | pt;
        // The words this lane completes; stores it need not make go to the
        // slice's spare last word instead, so there is no branch.
        const uint32_t wi = pos >> 2;
        slice[nfull > 0 ? wi : kSpare] = w0;
        slice[nfull > 1 ? wi + 1 : kSpare] = t1;
        slice[nfull > 2 ? wi + 2 : kSpare] = t2;
        slice[nfull > 3 ? wi + 3 : kSpare] = t3;
        const bool fin = lq + 1 == nvq && ((pos + C) & 3u);   // the sub-tile's last, partial word
        fidx = fin ? (pos + C) >> 2 : fidx;
        fword = fin ? (nfull ? last : w0) : fword;
    }
    slice[fidx != kNone ? fidx : kSpare] = fword;
    subenc_flush(slice, dst, h, run);
}

// A full sub-tile (128 quads) whose 512 coded values all take one byte:
// every control byte is 0 and the data bytes are the values' low bytes in
// order (Sec. 4), so no lengths, scan or shifts per value are needed.  Each
// lane packs its quad's four bytes into a word, shifted to the destination's
// phase with the previous quad's word.
__device__ __forceinline__ void subenc_write_small(uint32_t *slice, uint8_t *ctrl_dst, uint8_t *dst,
                                                   const uint32_t (&d)[kEncRounds][4])
{
    const int lane = threadIdx.x & 31;
    const uint32_t h = (uint32_t)((uintptr_t)dst & 15u);
    const uint32_t hw = h >> 2, sh = 8 * (h & 3);
    if (((uintptr_t)ctrl_dst & 3u) == 0) {
        reinterpret_cast<uint32_t *>(ctrl_dst)[lane] = 0u;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            ctrl_dst[4 * lane + j] = 0;
    }
    uint32_t carry = 0;  // the word of the quad before this round's first
#pragma unroll
    for (int r = 0; r < kEncRounds; r++) {
        const uint32_t w = __byte_perm(__byte_perm(d[r][0], d[r][1], 0x0040),
                                       __byte_perm(d[r][2], d[r][3], 0x0040), 0x5410);
        uint32_t pw = __shfl_up_sync(0xffffffffu, w, 1);
        if (lane == 0)
            pw = carry;
        carry = __shfl_sync(0xffffffffu, w, 31);
        slice[hw + 32 * r + lane] = sh ? __funnelshift_l(pw, w, sh) : w;
    }
    if (lane == 31 && sh)
        slice[hw + kSubQuads] = carry >> (32 - sh);
    subenc_flush(slice, dst, h, 4u * kSubQuads);
}

}  // namespace svb
