/*
 * Stream VByte oracle: a plain, slow, scalar C statement of what the codec
 * computes (Lemire, Kurz, Rupp, "Stream VByte: Faster Byte-Oriented Integer
 * Compression", arXiv 1709.08990).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Every function below follows the paper's definition step by step, in the
 * paper's order, with no blocking, fusion or reordering:
 *   1. differential coding: delta_1 = x_1 - prev, delta_i = x_i - x_{i-1}
 *      (Sec. 1; Sec. 5 on posting lists; all arithmetic mod 2^32);
 *   2. byte length of each coded value, ceil(log_256(v + 1)) in {1,2,3,4}
 *      (Sec. 3, the varint-GB length rule), with v = 0 taking one byte
 *      because code 00 means one byte (Sec. 4: an all-zero control byte
 *      covers four data bytes);
 *   3. control stream: one byte per four integers, two bits per integer,
 *      holding length - 1 (Sec. 3; Fig. 1; Fig. 3).  Integer j of a block of
 *      four sits in bits 2j..2j+1 (first integer in the low bits); pad fields
 *      of an incomplete last block are zero;
 *   4. data stream: right after the ceil(2N/8) control bytes (Sec. 4), each
 *      coded value's length-many low-order bytes, least significant first
 *      (Sec. 2: pshufb zero-fills the high bytes of each 32-bit lane);
 *   5. the compressed size is ceil(N/4) + sum of lengths (Sec. 4; Sec. 5
 *      reports the same storage as varint-GB, whose blocks have this size).
 * Decoding reverses these steps (Sec. 4, Fig. 4): the code of each integer
 * gives its byte count C, the low C bytes are read little-endian, and for
 * differential coding a prefix sum restores x_i = x_{i-1} + delta_i
 * (Sec. 2, differential coding).  The decoder accepts any code, including
 * non-minimal ones, ignores the pad fields of an incomplete last control
 * byte, and never reads past in_len.
 *
 * The N/A cases of the paper (N = 0) return 0 and touch nothing.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SVB_REF_ERROR ((size_t)-1)

/* Sec. 3: an integer x is stored in ceil(log_256(x + 1)) bytes, one of
 * {1,2,3,4}.  x = 0 gives log_256(1) = 0, but the smallest length is one
 * byte (code 00), so zero takes one byte. */
unsigned svb_ref_byte_length(uint32_t x)
{
    if (x < (1u << 8))
        return 1;
    if (x < (1u << 16))
        return 2;
    if (x < (1u << 24))
        return 3;
    return 4;
}

/* Sec. 4: ceil(2N/8) control bytes. */
size_t svb_ref_control_bytes(size_t n)
{
    return (2 * n + 7) / 8;
}

/* Largest possible compressed size: every integer four bytes long. */
size_t svb_ref_max_compressed_size(size_t n)
{
    return svb_ref_control_bytes(n) + 4 * n;
}

/* Encode n integers into out; returns the number of bytes written. */
static size_t encode_stream(const uint32_t *x, size_t n, uint8_t *out,
                            uint32_t prev, int delta)
{
    if (n == 0)
        return 0;

    /* Step 1: the coded values (gaps for differential coding). */
    uint32_t *v = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!v)
        return SVB_REF_ERROR;
    for (size_t i = 0; i < n; i++) {
        if (delta)
            v[i] = x[i] - (i == 0 ? prev : x[i - 1]);
        else
            v[i] = x[i];
    }

    /* Steps 2 and 3: the control stream, first integer in the low bits. */
    size_t nctrl = svb_ref_control_bytes(n);
    memset(out, 0, nctrl);
    for (size_t i = 0; i < n; i++) {
        unsigned len = svb_ref_byte_length(v[i]);
        out[i / 4] |= (uint8_t)((len - 1) << (2 * (i % 4)));
    }

    /* Step 4: the data stream, low-order bytes first. */
    size_t pos = nctrl;
    for (size_t i = 0; i < n; i++) {
        unsigned len = svb_ref_byte_length(v[i]);
        for (unsigned b = 0; b < len; b++)
            out[pos++] = (uint8_t)(v[i] >> (8 * b));
    }

    free(v);
    /* Step 5: ceil(N/4) + sum of lengths. */
    return pos;
}

/* Decode n integers from in[0, in_len); returns the bytes consumed, or
 * SVB_REF_ERROR when the stream is shorter than its control bytes say. */
static size_t decode_stream(const uint8_t *in, size_t in_len, size_t n,
                            uint32_t *x, uint32_t prev, int delta)
{
    if (n == 0)
        return 0;
    size_t nctrl = svb_ref_control_bytes(n);
    if (in_len < nctrl)
        return SVB_REF_ERROR;

    /* Control byte -> byte count -> little-endian value (Sec. 4, Fig. 4). */
    size_t pos = nctrl;
    for (size_t i = 0; i < n; i++) {
        unsigned code = (in[i / 4] >> (2 * (i % 4))) & 3u;
        unsigned len = code + 1;
        if (len > in_len - pos)
            return SVB_REF_ERROR;
        uint32_t v = 0;
        for (unsigned b = 0; b < len; b++)
            v |= (uint32_t)in[pos + b] << (8 * b);
        pos += len;
        x[i] = v;
    }

    /* Differential coding: prefix sum x_i = x_{i-1} + delta_i (Sec. 2). */
    if (delta) {
        uint32_t run = prev;
        for (size_t i = 0; i < n; i++) {
            run += x[i];
            x[i] = run;
        }
    }
    return pos;
}

/* The four entry points of the codec, on host memory. */
size_t svb_ref_encode(const uint32_t *in, size_t n, uint8_t *out)
{
    return encode_stream(in, n, out, 0, 0);
}

size_t svb_ref_delta_encode(const uint32_t *in, size_t n, uint8_t *out,
                            uint32_t prev)
{
    return encode_stream(in, n, out, prev, 1);
}

size_t svb_ref_decode(const uint8_t *in, size_t in_len, size_t n,
                      uint32_t *out)
{
    return decode_stream(in, in_len, n, out, 0, 0);
}

size_t svb_ref_delta_decode(const uint8_t *in, size_t in_len, size_t n,
                            uint32_t *out, uint32_t prev)
{
    return decode_stream(in, in_len, n, out, prev, 1);
}

/* Bytes of data stream that n integers with the given control bytes take
 * (Sec. 4: each control byte covers C in [4,16] bytes; an incomplete last
 * control byte covers only its used fields). */
size_t svb_ref_data_bytes(const uint8_t *ctrl, size_t n)
{
    size_t total = 0;
    for (size_t i = 0; i < n; i++)
        total += ((ctrl[i / 4] >> (2 * (i % 4))) & 3u) + 1;
    return total;
}

/* Seek and select on a compressed array (the operations benchmarked at the
 * end of Sec. 5, Fig. 6): both read the integers in order exactly as
 * decode_stream does - code, then length-many little-endian bytes, then the
 * running sum for differential coding - and stop at the answer.
 *
 *   seek(target)  the index of the first integer >= target, with that
 *                 integer in *value; n (and *value = 0) when there is none;
 *   select(i)     the integer at index i (i < n) in *value, returning 0.
 *
 * All ceil(n/4) control bytes must be present.  Either returns SVB_REF_ERROR
 * when the data stream ends before the integer that decides the answer
 * (for seek without a match, before the last integer), and select does so
 * for i >= n. */
size_t svb_ref_seek(const uint8_t *in, size_t in_len, size_t n, uint32_t prev,
                    int delta, uint32_t target, uint32_t *value)
{
    *value = 0;
    size_t nctrl = svb_ref_control_bytes(n);
    if (in_len < nctrl)
        return SVB_REF_ERROR;
    size_t pos = nctrl;
    uint32_t run = prev;
    for (size_t i = 0; i < n; i++) {
        unsigned len = ((in[i / 4] >> (2 * (i % 4))) & 3u) + 1;
        if (len > in_len - pos)
            return SVB_REF_ERROR;
        uint32_t v = 0;
        for (unsigned b = 0; b < len; b++)
            v |= (uint32_t)in[pos + b] << (8 * b);
        pos += len;
        if (delta) {
            run += v;
            v = run;
        }
        if (v >= target) {
            *value = v;
            return i;
        }
    }
    return n;
}

size_t svb_ref_select(const uint8_t *in, size_t in_len, size_t n, uint32_t prev,
                      int delta, size_t index, uint32_t *value)
{
    *value = 0;
    size_t nctrl = svb_ref_control_bytes(n);
    if (index >= n || in_len < nctrl)
        return SVB_REF_ERROR;
    size_t pos = nctrl;
    uint32_t run = prev;
    for (size_t i = 0; i <= index; i++) {
        unsigned len = ((in[i / 4] >> (2 * (i % 4))) & 3u) + 1;
        if (len > in_len - pos)
            return SVB_REF_ERROR;
        uint32_t v = 0;
        for (unsigned b = 0; b < len; b++)
            v |= (uint32_t)in[pos + b] << (8 * b);
        pos += len;
        run = delta ? run + v : v;
    }
    *value = run;
    return 0;
}
