/*
 * Exhaustive check of the Stream VByte oracle over every byte-length pattern
 * of n <= NMAX integers (4^n patterns for each n, tails n mod 4 != 0
 * included).  Compiled together with one build of the oracle source and run
 * by the test suite.
 *
 * For each pattern the values are chosen with exactly the pattern's lengths
 * (smallest, largest or a hashed value of that length, cycling by position),
 * and the harness checks, from the pattern alone and not from the oracle's
 * own length function:
 *   - the compressed size is ceil(n/4) + sum of lengths (Sec. 4);
 *   - control field i holds length_i - 1, first integer in the low bits,
 *     pad fields zero (Sec. 3, Fig. 3);
 *   - the data bytes are each value's low-order bytes, least significant
 *     first, back to back after the control bytes (Sec. 2, Sec. 4);
 *   - decoding restores the values and consumes exactly the stream;
 *   - differential coding of the running sums (start `prev`) produces the
 *     very same stream, and decodes back to the running sums (Sec. 2).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

size_t svb_ref_encode(const uint32_t *in, size_t n, uint8_t *out);
size_t svb_ref_decode(const uint8_t *in, size_t in_len, size_t n, uint32_t *out);
size_t svb_ref_delta_encode(const uint32_t *in, size_t n, uint8_t *out, uint32_t prev);
size_t svb_ref_delta_decode(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                            uint32_t prev);

static uint32_t hash32(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (uint32_t)(z ^ (z >> 31));
}

static uint32_t value_with_length(unsigned len, unsigned kind, uint64_t salt)
{
    uint64_t lo = len == 1 ? 0 : 1ull << (8 * (len - 1));
    uint64_t hi = (1ull << (8 * len)) - 1;
    if (kind == 0)
        return (uint32_t)lo;
    if (kind == 1)
        return (uint32_t)hi;
    return (uint32_t)(lo + hash32(salt) % (hi - lo + 1));
}

static int fail(const char *what, unsigned n, uint64_t pat)
{
    fprintf(stderr, "FAIL %s n=%u pattern=%llu\n", what, n, (unsigned long long)pat);
    return 1;
}

int main(int argc, char **argv)
{
    unsigned nmax = argc > 1 ? (unsigned)atoi(argv[1]) : 12;
    unsigned delta_every = argc > 2 ? (unsigned)atoi(argv[2]) : 1;
    uint32_t v[16], x[16], back[16];
    uint8_t s[80], s2[80];
    unsigned len[16];
    uint64_t checked = 0;

    for (unsigned n = 0; n <= nmax; n++) {
        uint64_t npat = 1ull << (2 * n);
        for (uint64_t pat = 0; pat < npat; pat++) {
            size_t expect = (n + 3) / 4;
            for (unsigned i = 0; i < n; i++) {
                len[i] = 1 + (unsigned)((pat >> (2 * i)) & 3);
                v[i] = value_with_length(len[i], (unsigned)((pat + i + n) % 3),
                                         (pat << 4) ^ (i * 131u + n));
                expect += len[i];
            }
            size_t got = svb_ref_encode(v, n, s);
            if (got != expect)
                return fail("size", n, pat);
            size_t nctrl = (n + 3) / 4;
            for (unsigned q = 0; q < nctrl; q++) {
                unsigned want = 0;
                for (unsigned j = 0; j < 4 && 4 * q + j < n; j++)
                    want |= (len[4 * q + j] - 1) << (2 * j);
                if (s[q] != want)
                    return fail("control byte", n, pat);
            }
            size_t pos = nctrl;
            for (unsigned i = 0; i < n; i++)
                for (unsigned b = 0; b < len[i]; b++, pos++)
                    if (s[pos] != (uint8_t)(v[i] >> (8 * b)))
                        return fail("data byte", n, pat);
            memset(back, 0xAB, sizeof back);
            if (svb_ref_decode(s, got, n, back) != got)
                return fail("decode size", n, pat);
            if (memcmp(back, v, n * sizeof(uint32_t)) != 0)
                return fail("decode values", n, pat);
            if (got > 0 && svb_ref_decode(s, got - 1, n, back) != (size_t)-1)
                return fail("truncation not detected", n, pat);

            if (pat % delta_every == 0) {
                uint32_t prev = hash32(pat * 7 + n);
                uint32_t run = prev;
                for (unsigned i = 0; i < n; i++) {
                    run += v[i];
                    x[i] = run;
                }
                if (svb_ref_delta_encode(x, n, s2, prev) != got || memcmp(s, s2, got) != 0)
                    return fail("delta encode", n, pat);
                memset(back, 0xCD, sizeof back);
                if (svb_ref_delta_decode(s2, got, n, back, prev) != got)
                    return fail("delta decode size", n, pat);
                if (memcmp(back, x, n * sizeof(uint32_t)) != 0)
                    return fail("delta decode values", n, pat);
            }
            checked++;
        }
    }
    printf("OK %llu patterns\n", (unsigned long long)checked);
    return 0;
}
