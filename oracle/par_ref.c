/*
 * Multi-threaded harness around the Stream VByte oracle, for timing the
 * oracle on all of a host's cores.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite and the bench's CPU-baseline and
 * reference legs do.  It computes nothing of the method itself: every byte
 * count and every decoded integer comes from the oracle's own functions in
 * svb_ref.c, which this file links with and does not change.  Its result is
 * checked against the oracle's single-threaded decode, bit for bit.
 *
 * The single stream is cut into chunks of whole control bytes (Sec. 4: a
 * control byte and its 4 + sum-of-codes data bytes describe four integers
 * on their own), one chunk per thread:
 *   pass 1  each thread counts the data bytes its chunk's control bytes cover
 *           (svb_ref_data_bytes); a prefix over the chunks, in order, gives
 *           each chunk's data offset;
 *   pass 2  each thread copies its chunk's control bytes and data bytes into
 *           one buffer (the oracle's decoder takes a stream laid out as
 *           control bytes then data) and decodes it with the oracle, from 0
 *           for differential streams;
 *   pass 3  (differential streams) each chunk's integers are shifted by prev
 *           plus the sum of all earlier chunks' gaps (Sec. 2: the prefix sum
 *           carried across chunks), taken from the last integer of each
 *           earlier chunk's own decode.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PAR_REF_ERROR ((size_t)-1)

size_t svb_ref_control_bytes(size_t n);
size_t svb_ref_data_bytes(const uint8_t *ctrl, size_t n);
size_t svb_ref_decode(const uint8_t *in, size_t in_len, size_t n, uint32_t *out);
size_t svb_ref_delta_decode(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                            uint32_t prev);

struct chunk {
    const uint8_t *in;  /* the whole stream */
    size_t nctrl;       /* control bytes of the whole stream */
    size_t q0, q1;      /* the chunk's control bytes [q0, q1) */
    size_t i0, i1;      /* its integers [i0, i1) */
    size_t d0, dlen;    /* its data bytes [d0, d0 + dlen) after the control bytes */
    uint32_t *out;
    uint32_t add;       /* pass 3: added to every integer */
    int delta;
    int ok;
};

static void *pass1(void *p)
{
    struct chunk *c = (struct chunk *)p;
    c->dlen = svb_ref_data_bytes(c->in + c->q0, c->i1 - c->i0);
    return NULL;
}

static void *pass2(void *p)
{
    struct chunk *c = (struct chunk *)p;
    size_t m = c->i1 - c->i0, nc = c->q1 - c->q0;
    uint8_t *buf = (uint8_t *)malloc(nc + c->dlen + 1);
    if (!buf) {
        c->ok = 0;
        return NULL;
    }
    memcpy(buf, c->in + c->q0, nc);
    memcpy(buf + nc, c->in + c->nctrl + c->d0, c->dlen);
    const size_t k = c->delta ? svb_ref_delta_decode(buf, nc + c->dlen, m, c->out + c->i0, 0)
                              : svb_ref_decode(buf, nc + c->dlen, m, c->out + c->i0);
    c->ok = k == nc + c->dlen;
    free(buf);
    return NULL;
}

static void *pass3(void *p)
{
    struct chunk *c = (struct chunk *)p;
    for (size_t i = c->i0; i < c->i1; i++)
        c->out[i] += c->add;
    return NULL;
}

static int run_all(struct chunk *cs, int k, void *(*fn)(void *))
{
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)k);
    if (!th)
        return 0;
    int started = 0;
    for (int t = 0; t < k; t++) {
        if (pthread_create(&th[t], NULL, fn, &cs[t]) != 0)
            break;
        started++;
    }
    for (int t = 0; t < started; t++)
        pthread_join(th[t], NULL);
    free(th);
    return started == k;
}

/* Decode n integers from in[0, in_len) into out with `threads` threads;
 * returns the bytes consumed, or PAR_REF_ERROR when the stream is shorter
 * than its control bytes say (or a thread could not be started). */
size_t svb_par_decode(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                      uint32_t prev, int delta, int threads)
{
    if (n == 0)
        return 0;
    size_t nctrl = svb_ref_control_bytes(n);
    if (in_len < nctrl)
        return PAR_REF_ERROR;
    if (threads < 1)
        threads = 1;
    if ((size_t)threads > nctrl)
        threads = (int)nctrl;
    struct chunk *cs = (struct chunk *)calloc((size_t)threads, sizeof(struct chunk));
    if (!cs)
        return PAR_REF_ERROR;
    size_t per = (nctrl + (size_t)threads - 1) / (size_t)threads;
    for (int t = 0; t < threads; t++) {
        struct chunk *c = &cs[t];
        c->in = in;
        c->nctrl = nctrl;
        c->q0 = (size_t)t * per < nctrl ? (size_t)t * per : nctrl;
        c->q1 = c->q0 + per < nctrl ? c->q0 + per : nctrl;
        c->i0 = 4 * c->q0 < n ? 4 * c->q0 : n;
        c->i1 = 4 * c->q1 < n ? 4 * c->q1 : n;
        c->out = out;
        c->delta = delta;
        c->ok = 1;
    }
    size_t res = PAR_REF_ERROR;
    if (!run_all(cs, threads, pass1))
        goto done;
    size_t off = 0;
    for (int t = 0; t < threads; t++) {
        cs[t].d0 = off;
        off += cs[t].dlen;
    }
    if (nctrl + off > in_len)
        goto done;
    if (!run_all(cs, threads, pass2))
        goto done;
    for (int t = 0; t < threads; t++)
        if (!cs[t].ok)
            goto done;
    if (delta) {
        uint32_t run = prev;
        for (int t = 0; t < threads; t++) {
            cs[t].add = run;
            if (cs[t].i1 > cs[t].i0)
                run += out[cs[t].i1 - 1];
        }
        if (!run_all(cs, threads, pass3))
            goto done;
    }
    res = nctrl + off;
done:
    free(cs);
    return res;
}
