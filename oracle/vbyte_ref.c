/*
 * VByte oracle: a plain, slow, scalar C statement of the VByte format that
 * Stream VByte is compared against (Lemire, Kurz, Rupp, arXiv 1709.08990,
 * Sec. 2 and Sec. 3), used for the compressed-size comparison of Sec. 5
 * (Fig. 5b: extra bits per integer of Stream VByte over VByte).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite and the bench's CPU legs do.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * The format, step by step as the paper states it:
 *   1. differential coding as for Stream VByte: delta_1 = x_1 - prev,
 *      delta_i = x_i - x_{i-1}, modulo 2^32 (Sec. 1, Sec. 5);
 *   2. each coded value is cut into 7-bit groups, least significant group
 *      first (Sec. 2); every byte holds one group in its low seven bits;
 *   3. the most significant bit of a byte is 1 when the next byte continues
 *      the same integer and 0 in the integer's last byte (Sec. 2, Sec. 3:
 *      b_0 .. b_{L-1} in [2^7, 2^8), the last byte in [0, 2^7));
 *   4. so an integer in [2^(7(L-1)), 2^(7L)) takes L bytes, and zero one byte
 *      (Sec. 3); a 32-bit integer takes at most five;
 *   5. decoding sums (b_i mod 2^7) * 2^(7i) over the integer's bytes (Sec. 3)
 *      and, for differential coding, restores x_i = x_{i-1} + delta_i.
 * The decoder reads nothing past in_len and rejects an integer spread over
 * more than five bytes (it cannot be a 32-bit value).
 */
#include <stddef.h>
#include <stdint.h>

#define VBYTE_REF_ERROR ((size_t)-1)

/* Step 4: bytes of one coded value. */
unsigned vbyte_ref_length(uint32_t v)
{
    unsigned bytes = 1;
    while (v >= 128u) {
        v >>= 7;
        bytes++;
    }
    return bytes;
}

/* Step 1: the value coded for position i. */
static uint32_t coded_value(const uint32_t *x, size_t i, int delta, uint32_t prev)
{
    if (!delta)
        return x[i];
    uint32_t before = i ? x[i - 1] : prev;
    return x[i] - before;
}

/* Bytes of the whole VByte stream of n integers. */
size_t vbyte_ref_size(const uint32_t *x, size_t n, int delta, uint32_t prev)
{
    size_t total = 0;
    for (size_t i = 0; i < n; i++)
        total += vbyte_ref_length(coded_value(x, i, delta, prev));
    return total;
}

/* Steps 1-3: writes the stream to out (room for 5n bytes), returns its size. */
size_t vbyte_ref_encode(const uint32_t *x, size_t n, uint8_t *out, int delta, uint32_t prev)
{
    size_t p = 0;
    for (size_t i = 0; i < n; i++) {
        uint32_t v = coded_value(x, i, delta, prev);
        for (;;) {
            uint8_t group = (uint8_t)(v & 127u);
            v >>= 7;
            if (v == 0) {
                out[p++] = group;          /* last byte: high bit 0 */
                break;
            }
            out[p++] = (uint8_t)(group | 128u);   /* another byte follows */
        }
    }
    return p;
}

/* Step 5: decodes n integers, returns the bytes consumed or VBYTE_REF_ERROR
 * if the stream ends early or an integer runs past five bytes. */
size_t vbyte_ref_decode(const uint8_t *in, size_t in_len, size_t n, uint32_t *out, int delta,
                        uint32_t prev)
{
    size_t p = 0;
    uint32_t run = prev;
    for (size_t i = 0; i < n; i++) {
        uint64_t value = 0;
        unsigned k = 0;
        for (;;) {
            if (p >= in_len || k == 5)
                return VBYTE_REF_ERROR;
            uint8_t b = in[p++];
            value += (uint64_t)(b % 128u) << (7 * k);
            k++;
            if (b < 128u)
                break;
        }
        uint32_t v = (uint32_t)value;
        if (delta) {
            run += v;
            out[i] = run;
        } else {
            out[i] = v;
        }
    }
    return p;
}
