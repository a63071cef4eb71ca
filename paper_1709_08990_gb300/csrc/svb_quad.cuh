// Device helpers shared by the tiled and batched kernels: staging a byte
// range into shared memory (bulk-copy interior + ragged edges) and decoding
// or encoding one quad of four integers.
#pragma once

#include <cstdint>

#include "svb_device.cuh"

namespace svb {

// Interior of global [g, g + len): the 16-byte-aligned part, copied by the
// bulk engine to smem base + off0 (base + (g mod 16) holds byte g).
__device__ __forceinline__ uint32_t range_interior(const uint8_t *g, uint32_t len,
                                                   const uint8_t *&a0, uint32_t &off0)
{
    uintptr_t s = (uintptr_t)g, e = s + len;
    uintptr_t c0 = (s + 15) & ~(uintptr_t)15, c1 = e & ~(uintptr_t)15;
    a0 = reinterpret_cast<const uint8_t *>(c0);
    off0 = (uint32_t)(c0 - (s & ~(uintptr_t)15));
    return c1 > c0 ? (uint32_t)(c1 - c0) : 0u;
}

// The ragged head and tail of [g, g + len) (< 16 bytes each), by plain loads.
__device__ __forceinline__ void range_edges(const uint8_t *g, uint32_t len, uint8_t *base,
                                            int lane)
{
    uintptr_t s = (uintptr_t)g, e = s + len;
    uintptr_t c0 = (s + 15) & ~(uintptr_t)15, c1 = e & ~(uintptr_t)15;
    uint32_t h = (uint32_t)(s & 15u);
    uint32_t head = (uint32_t)((c0 < e ? c0 : e) - s);                    // bytes [0, head)
    uint32_t tail0 = (uint32_t)((c1 > c0 ? c1 : (c0 < e ? c0 : e)) - s);  // bytes [tail0, len)
    for (uint32_t i = lane; i < head; i += 32)
        base[h + i] = __ldg(g + i);
    for (uint32_t i = tail0 + lane; i < len; i += 32)
        base[h + i] = __ldg(g + i);
}

// How to stage global [g, g + len) so that byte g lands at smem base +
// (g mod 16).  When the 16-byte-aligned range around it lies inside [lo, hi)
// (the bytes the caller may read), one bulk copy of that whole range does it;
// otherwise the aligned interior goes by bulk copy and the ragged ends (under
// 16 bytes each) by plain loads (range_edges).
struct StagePlan {
    const uint8_t *src;
    uint32_t dst_off;
    uint32_t bytes;
    bool edges;
};

__device__ __forceinline__ StagePlan stage_plan(const uint8_t *g, uint32_t len, const uint8_t *lo,
                                                const uint8_t *hi)
{
    StagePlan p;
    const uintptr_t s = (uintptr_t)g, e = s + len;
    const uintptr_t o0 = s & ~(uintptr_t)15, o1 = (e + 15) & ~(uintptr_t)15;
    if (len && o0 >= (uintptr_t)lo && o1 <= (uintptr_t)hi) {
        p.src = reinterpret_cast<const uint8_t *>(o0);
        p.dst_off = 0;
        p.bytes = (uint32_t)(o1 - o0);
        p.edges = false;
    } else {
        p.bytes = range_interior(g, len, p.src, p.dst_off);
        p.edges = len != 0;
    }
    return p;
}

__device__ __forceinline__ uint32_t quad_count(uint32_t c, uint32_t nints)
{
    return nints + __popc(c & 0x55u) + 2u * __popc(c & 0xAAu);
}

// The code + 1 bytes at staged position p, least significant first.  The
// funnel shift uses only the low five bits of its count, so p << 3 selects
// the byte within the first word.
__device__ __forceinline__ uint32_t take(const uint8_t *d, uint32_t p, uint32_t code)
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(d + (p & ~3u));
    return __funnelshift_r(w[0], w[1], p << 3) & (0xffffffffu >> (24u - 8u * code));
}

// One quad: its four integers start at staged position p, lengths from the
// codes of control byte c (Sec. 4: integer j takes code_j + 1 bytes).
__device__ __forceinline__ uint4 decode_quad(const uint8_t *d, uint32_t p, uint32_t c)
{
    const uint32_t c0 = c & 3u, c1 = (c >> 2) & 3u, c2 = (c >> 4) & 3u, c3 = c >> 6;
    const uint32_t p1 = p + c0 + 1, p2 = p1 + c1 + 1, p3 = p2 + c2 + 1;
    return make_uint4(take(d, p, c0), take(d, p1, c1), take(d, p2, c2), take(d, p3, c3));
}

// A quad with control byte 0: four one-byte integers (the zero-control fast
// path the paper also takes, Sec. 4).
__device__ __forceinline__ uint4 widen_quad(const uint8_t *d, uint32_t p)
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(d + (p & ~3u));
    const uint32_t x = __funnelshift_r(w[0], w[1], p << 3);
    return make_uint4(__byte_perm(x, 0, 0x4440), __byte_perm(x, 0, 0x4441),
                      __byte_perm(x, 0, 0x4442), __byte_perm(x, 0, 0x4443));
}

// Sec. 3: bytes needed by v, 1..4 (zero takes one byte).
__device__ __forceinline__ uint32_t byte_len(uint32_t v)
{
    return max(1u, (39u - (uint32_t)__clz(v)) >> 3);
}

}  // namespace svb
