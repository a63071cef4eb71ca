// Decoding one warp's sub-tile (up to kSubQuads = 128 quads) from shared
// memory, shared by the single-stream and the batched decoders.
//
// The sub-tile's control bytes C and its data bytes (from D + base on) are
// staged.  Each lane takes four consecutive control bytes, turns their codes
// into the four quads' byte counts (Sec. 4: a control byte covers 4 + the sum
// of its codes bytes) and a warp scan into every quad's data position, kept
// in the warp's `pos` scratch.  Then, in rounds of 32 quads, each lane decodes
// one quad: per integer a funnel shift of two shared words and a mask
// (decode_quad), or, when the whole round's control bytes are zero (every
// integer one byte, Sec. 4), a byte widening (widen_quad).
#pragma once

#include <cstdint>

#include "svb_device.cuh"
#include "svb_quad.cuh"

namespace svb {

constexpr int kSubRounds = kSubQuads / 32;   // quads per lane per sub-tile

struct SubTile {
    const uint8_t *C;   // the sub-tile's control bytes
    const uint8_t *D;   // the stage's data bytes
    uint32_t base;      // the sub-tile's first data byte in D
    uint32_t nq;        // quads in the sub-tile, 1..kSubQuads
    uint32_t tail;      // integers in quad nq - 1: 4 unless it is the stream's last quad
    __device__ bool full() const { return nq == (uint32_t)kSubQuads && tail == 4; }
};

// Control bytes 4l .. 4l + 3 of the sub-tile in lane l (0 past nq).
__device__ __forceinline__ uint32_t subtile_ctrl_word(const SubTile &t)
{
    const int lane = threadIdx.x & 31;
    uint32_t w = 0;
    if (((uintptr_t)t.C & 3u) == 0 && 4u * lane + 4u <= t.nq) {
        w = reinterpret_cast<const uint32_t *>(t.C)[lane];
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (4u * lane + j < t.nq)
                w |= (uint32_t)t.C[4 * lane + j] << (8 * j);
    }
    return w;
}

// Integers in quad lq of the sub-tile (0 past the end).
__device__ __forceinline__ uint32_t subtile_nints(const SubTile &t, uint32_t lq)
{
    return lq >= t.nq ? 0u : (lq == t.nq - 1 ? t.tail : 4u);
}

// Staged data position of each quad of the sub-tile into pos[0 .. nq) (16-bit
// entries, four per lane); w from subtile_ctrl_word.
__device__ __forceinline__ void subtile_positions(const SubTile &t, uint32_t w, uint16_t *pos)
{
    const int lane = threadIdx.x & 31;
    uint32_t o1, o2, o3, tsum;
    if (t.full()) {
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
            const uint32_t nints = subtile_nints(t, 4u * lane + j);
            uint32_t c = (w >> (8 * j)) & 0xffu;
            if (nints < 4)
                c &= (1u << (2 * nints)) - 1u;
            cnt[j] = nints ? quad_count(c, nints) : 0u;
        }
        o1 = cnt[0];
        o2 = o1 + cnt[1];
        o3 = o2 + cnt[2];
        tsum = o3 + cnt[3];
    }
    const uint32_t incl = warp_incl_scan(tsum);
    const uint32_t o0 = t.base + incl - tsum;
    reinterpret_cast<uint2 *>(pos)[lane] =
        make_uint2(o0 | ((o0 + o1) << 16), (o0 + o2) | ((o0 + o3) << 16));
}

// The sub-tile's integers (the coded values: gaps for differential streams):
// lane l holds quad 32r + l in v[r]; fields past the end are 0.  Call after
// subtile_positions and a __syncwarp.
__device__ __forceinline__ void subtile_gather(const SubTile &t, const uint16_t *pos,
                                               uint32_t (&v)[kSubRounds][4])
{
    const int lane = threadIdx.x & 31;
    const bool full = t.full();
#pragma unroll
    for (int r = 0; r < kSubRounds; r++) {
        const uint32_t lq = r * 32 + lane;
        uint4 x;
        if (full) {
            const uint32_t c = t.C[lq];
            const uint32_t p = pos[lq];
            if (__all_sync(0xffffffffu, c == 0))
                x = widen_quad(t.D, p);
            else
                x = decode_quad(t.D, p, c);
        } else {
            const uint32_t nints = subtile_nints(t, lq);
            uint32_t c = nints ? t.C[lq] : 0u;
            if (nints < 4)
                c &= (1u << (2 * nints)) - 1u;
            x = decode_quad(t.D, nints ? pos[lq] : t.base, c);
            x.x = nints > 0 ? x.x : 0u;
            x.y = nints > 1 ? x.y : 0u;
            x.z = nints > 2 ? x.z : 0u;
            x.w = nints > 3 ? x.w : 0u;
        }
        v[r][0] = x.x;
        v[r][1] = x.y;
        v[r][2] = x.z;
        v[r][3] = x.w;
    }
}

// Sum of the 512 one-byte integers at staged positions [base, base + 512) of
// D (a sub-tile whose control bytes are all zero: Sec. 4, an all-zero control
// byte covers 4 bytes), a word at a time with the bytes outside masked; the
// warp's total in every lane.
__device__ __forceinline__ uint32_t zero_ctrl_sum(const uint8_t *D, uint32_t base)
{
    const int lane = threadIdx.x & 31;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(D);
    const uint32_t b0 = base >> 2, b1 = (base + 4 * kSubQuads + 3) >> 2;
    const uint32_t head = base & 3u, tail = (base + 4 * kSubQuads) & 3u;
    uint32_t t = 0;
    for (uint32_t i = b0 + lane; i < b1; i += 32) {
        uint32_t x = Wd[i];
        if (i == b0)
            x &= 0xffffffffu << (8 * head);
        if (i == b1 - 1 && tail)
            x &= 0xffffffffu >> (8 * (4 - tail));
        const uint32_t y = (x & 0x00ff00ffu) + ((x >> 8) & 0x00ff00ffu);
        t += (y & 0xffffu) + (y >> 16);
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        t += __shfl_xor_sync(0xffffffffu, t, d);
    return t;
}

// Copies the bytes of global [g, g + len) that lie inside [lo, hi) so that
// byte g + i lands at dst + (g mod 16) + i (dst 16-byte aligned): whole
// 16-byte chunks by cp.async, a chunk that straddles lo or hi byte by byte
// (none of its bytes outside [lo, hi) is read).  One whole warp; the caller
// commits and waits.
__device__ __forceinline__ void warp_stage(const uint8_t *g, uint32_t len, uint8_t *dst,
                                           uintptr_t lo, uintptr_t hi, uint64_t policy)
{
    const int lane = threadIdx.x & 31;
    const uintptr_t a0 = (uintptr_t)g & ~(uintptr_t)15;
    const uint32_t nch = (uint32_t)((((uintptr_t)g + len + 15) & ~(uintptr_t)15) - a0) >> 4;
    for (uint32_t c = lane; c < nch; c += 32) {
        const uintptr_t src = a0 + 16 * (uintptr_t)c;
        if (src >= lo && src + 16 <= hi) {
            cp_async16(dst + 16 * c, reinterpret_cast<const void *>(src), policy);
        } else {
            for (int i = 0; i < 16; i++)
                if (src + i >= lo && src + i < hi)
                    dst[16 * c + i] = __ldg(reinterpret_cast<const uint8_t *>(src + i));
        }
    }
}

}  // namespace svb
