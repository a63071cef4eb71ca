/*
 * svb.h - Stream VByte codec on the GPU (sm_103a), C ABI.
 *
 * Format (Lemire, Kurz, Rupp, arXiv 1709.08990, Sec. 4 and Fig. 3): n
 * unsigned 32-bit integers become ceil(n/4) control bytes followed by a data
 * stream.  Integer i has a 2-bit code, length - 1, in control byte i/4 at
 * bits 2(i mod 4)..2(i mod 4)+1 (first integer in the low bits); its value
 * takes `length` bytes of the data stream, least significant byte first.
 * The length of v is ceil(log_256(v + 1)) bytes, one byte for v = 0
 * (Sec. 3).  Pad fields of an incomplete last control byte are written as 0
 * and ignored when decoding.  n is not stored in the stream (Sec. 4 keeps
 * the count outside it); every call takes it.
 *
 * Differential coding (Sec. 1, Sec. 2, Sec. 5): the
 * stream holds delta_1 = x_1 - prev, delta_i = x_i - x_{i-1}, modulo 2^32;
 * decoding computes x_i = prev + delta_1 + ... + delta_i modulo 2^32.  The
 * paper starts from prev = 0; here the caller chooses prev.
 *
 * Memory.  Every data pointer is a DEVICE pointer unless its name starts
 * with h_.  The caller allocates and owns every buffer.  No entry point
 * retains a pointer after it returns (async forms: after the stream reaches
 * the launched work).  Buffers need no particular alignment; 16-byte aligned
 * buffers take the fastest path.
 *
 * Streams.  svb_stream_t is cudaStream_t.  The synchronous forms run on the
 * calling thread's stream set by svb_set_stream (default: the legacy default
 * stream 0) and wait for it.  The async forms enqueue work on the stream they
 * are given and return at once.
 *
 * Errors.  Size-returning calls return SVB_ERROR ((size_t)-1) on failure and
 * set the calling thread's svb_last_error(); int-returning calls return the
 * status code itself.  n = 0 returns 0 and touches nothing.
 */
#ifndef SVB_H
#define SVB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *svb_stream_t; /* == cudaStream_t */

#define SVB_ERROR ((size_t)-1)

enum svb_status {
    SVB_OK = 0,
    SVB_EINVAL = 1,     /* null pointer with n > 0, workspace too small, bad argument */
    SVB_ETRUNCATED = 2, /* the compressed input is shorter than its control bytes require */
    SVB_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    SVB_ETIMEOUT = 4,   /* a cross-tile wait ran past its spin limit; outputs are undefined */
    SVB_ENOMEM = 5      /* the library could not allocate its per-device workspace */
};

/* Written by the device at the end of an async call.  bytes: bytes written
 * (encode) or consumed (decode), or SVB_ERROR; status: an svb_status. */
typedef struct svb_result {
    uint64_t bytes;
    uint64_t status;
} svb_result;

/* ---- sizes -------------------------------------------------------------- */

/* Largest compressed size of n integers: ceil(n/4) + 4n (Sec. 4: control
 * bytes plus at most four data bytes per integer). */
size_t svb_max_compressed_size(size_t n);

/* Compressed size of n integers whose control bytes are ctrl (a HOST copy of
 * the first ceil(n/4) bytes of a stream): ceil(n/4) + sum of the lengths the
 * codes give, pad fields not counted. */
size_t svb_compressed_size_from_control(const uint8_t *h_ctrl, size_t n);

/* ---- the four codec calls (Sec. 4; synchronous) ------------------------ */

/* Encode in[0..n) into out (capacity >= svb_max_compressed_size(n)).
 * Returns the bytes written, ceil(n/4) + sum of lengths. */
size_t svb_encode(const uint32_t *in, size_t n, uint8_t *out);

/* Decode n integers from the stream at in into out[0..n).  The caller
 * guarantees that in holds the whole stream (its length follows from the
 * control bytes; use svb_decode_checked when it is not known).  Returns the
 * bytes consumed.  Reads no byte outside the stream. */
size_t svb_decode(const uint8_t *in, size_t n, uint32_t *out);

/* Differential forms: the stream codes in[0] - prev, then in[i] - in[i-1]
 * for i >= 1, modulo 2^32; decoding restores out[i] = prev + the sum of the
 * first i + 1 coded values, modulo 2^32 (Sec. 2, Sec. 5). */
size_t svb_delta_encode(const uint32_t *in, size_t n, uint8_t *out, uint32_t prev);
size_t svb_delta_decode(const uint8_t *in, size_t n, uint32_t *out, uint32_t prev);

/* Decode with the input length known: in[0..in_len) is all that may be
 * read.  A stream shorter than its control bytes require returns SVB_ERROR
 * with SVB_ETRUNCATED and leaves out partly written.  delta selects
 * differential decoding from prev. */
size_t svb_decode_checked(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                          uint32_t prev, int delta);

/* ---- host-buffer forms (copies inside the call) ------------------------ */

/* Decode a stream held in HOST memory h_in[0..in_len) into HOST memory
 * h_out[0..n).  d_in (>= in_len bytes) and d_out (>= 4n bytes) are caller-
 * owned device staging buffers.  Copies in, decodes and copies out on the
 * calling thread's stream; pinned host memory gives full link speed. */
size_t svb_decode_host(const uint8_t *h_in, size_t in_len, size_t n, uint32_t *h_out,
                       uint32_t prev, int delta, uint8_t *d_in, uint32_t *d_out);

/* Encode HOST h_in[0..n) into HOST h_out (capacity >=
 * svb_max_compressed_size(n)) through device staging buffers d_in (>= 4n
 * bytes) and d_out (>= svb_max_compressed_size(n) bytes). */
size_t svb_encode_host(const uint32_t *h_in, size_t n, uint8_t *h_out, uint32_t prev,
                       int delta, uint32_t *d_in, uint8_t *d_out);

/* ---- streams and errors ------------------------------------------------ */

/* Stream used by the synchronous forms in the calling thread. */
int svb_set_stream(svb_stream_t stream);
svb_stream_t svb_get_stream(void);

/* Status of the calling thread's last failed (or successful) call. */
int svb_last_error(void);
const char *svb_error_string(int status);

/* Spin limit of the cross-tile waits (iterations of a bounded, backing-off
 * poll, about a microsecond each at most).  0 restores the default, which is
 * also overridable with the environment variable SVB_LOOKBACK_SPIN_LIMIT. */
void svb_set_spin_limit(uint64_t iterations);

/* Decoder variant used by every decode call of this process:
 *   SVB_DECODE_AUTO (0)        the default: SVB_DECODE_SMALL for plain
 *                              streams of at most 2^22 integers whose tiles
 *                              can all be resident (launch-bound sizes),
 *                              else SVB_DECODE_SINGLE_PASS up to 2^20
 *                              integers and SVB_DECODE_TWO_PASS above;
 *   SVB_DECODE_SINGLE_PASS (1) one kernel: each tile sums its control bytes,
 *                              finds its data offset by a decoupled look-back
 *                              over its predecessors, then decodes;
 *   SVB_DECODE_TWO_PASS (2)    an offsets pass over the control stream, then
 *                              a persistent decode with bulk-copy staging;
 *                              for differential streams the offsets pass
 *                              also sums each 512-integer sub-tile's gaps
 *                              into its carry-in;
 *   SVB_DECODE_SUMS_PASS (3)   as SVB_DECODE_TWO_PASS, but differential
 *                              streams learn their carry-ins from a separate
 *                              pass over the staged tiles (three launches);
 *   SVB_DECODE_SMALL (4)       plain streams: one cooperative launch, one CTA
 *                              per 4096-integer tile, a grid barrier between
 *                              the tiles' byte totals and the decode; where
 *                              the tiles cannot all be resident at once, or
 *                              the stream is being captured into a graph,
 *                              the decode runs as SVB_DECODE_AUTO would run
 *                              it (single pass up to 2^20 integers, else two
 *                              pass).  Differential streams as
 *                              SVB_DECODE_TWO_PASS;
 *   SVB_DECODE_CHUNKED (5)     plain streams: one persistent launch over
 *                              chunks of 65536 integers; a chunk's data
 *                              offset comes from a decoupled look-back over
 *                              the chunks before it, found one chunk ahead of
 *                              the decode (Sec. 4's offsets without a
 *                              separate pass).  Differential streams, and
 *                              streams whose in_len does not cover their
 *                              control bytes, as SVB_DECODE_TWO_PASS.
 * All give identical results.  Returns SVB_EINVAL for an unknown variant. */
enum svb_decode_variant {
    SVB_DECODE_AUTO = 0,
    SVB_DECODE_SINGLE_PASS = 1,
    SVB_DECODE_TWO_PASS = 2,
    SVB_DECODE_SUMS_PASS = 3,
    SVB_DECODE_SMALL = 4,
    SVB_DECODE_CHUNKED = 5
};
int svb_set_decode_variant(int variant);

/* Encoder variant used by every encode call of this process:
 *   SVB_ENCODE_AUTO (0)           the default: SVB_ENCODE_SMALL for arrays
 *                                 of at most 2^22 integers whose tiles can
 *                                 all be resident, else SVB_ENCODE_CHUNKED;
 *   SVB_ENCODE_TILE_LOOKBACK (1)  one CTA per tile of 4096 integers, which
 *                                 finds its data offset by a look-back over
 *                                 its predecessors' byte totals;
 *   SVB_ENCODE_CHUNKED (2)        persistent CTAs over chunks of 32768
 *                                 integers: a sizing pass, one look-back per
 *                                 chunk, then a writing pass whose second
 *                                 read of the values is served by L2.
 *   SVB_ENCODE_SMALL (3)          one cooperative launch, one CTA per
 *                                 4096-integer tile: each sizes its values,
 *                                 a grid barrier, then each writes them at
 *                                 the offset the earlier tiles' totals give
 *                                 (the values read once); where the tiles
 *                                 cannot all be resident, or the stream is
 *                                 being captured, SVB_ENCODE_CHUNKED runs.
 * All give identical streams.  Returns SVB_EINVAL for an unknown variant. */
enum svb_encode_variant {
    SVB_ENCODE_AUTO = 0,
    SVB_ENCODE_TILE_LOOKBACK = 1,
    SVB_ENCODE_CHUNKED = 2,
    SVB_ENCODE_SMALL = 3
};
int svb_set_encode_variant(int variant);

/* ---- per-kernel timing --------------------------------------------------- */

/* Start recording a CUDA event pair around every kernel the library launches
 * (on the kernel's own stream).  Do not profile while capturing a CUDA graph. */
int svb_profile_begin(void);

/* Stop recording, wait for the recorded events and write one line per kernel,
 * "name launches total_ms", longest total first, into buf (NUL-terminated,
 * truncated to len).  Returns the bytes the full report needs. */
size_t svb_profile_end(char *buf, size_t len);

/* ---- async forms with a caller-owned workspace ------------------------- */

/* Bytes of workspace one async call over n integers needs. */
size_t svb_workspace_size(size_t n);

/* Zero a workspace once before its first use (enqueued on stream).  A
 * workspace serves one call at a time: calls that share one must be ordered
 * on one stream. */
int svb_workspace_init(void *ws, size_t ws_bytes, svb_stream_t stream);

/* Enqueue an encode / decode on stream.  d_result (device memory) receives
 * the byte count and status when the work completes.  in_len bounds the
 * decoder's reads (pass SIZE_MAX when the stream is known to be complete). */
int svb_encode_async(const uint32_t *in, size_t n, uint8_t *out, uint32_t prev, int delta,
                     svb_result *d_result, void *ws, size_t ws_bytes, svb_stream_t stream);
int svb_decode_async(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                     uint32_t prev, int delta, svb_result *d_result, void *ws,
                     size_t ws_bytes, svb_stream_t stream);

/* ---- batched codec: many independent lists in one launch --------------- */

/* One list of a batch.  Decode: in_off / in_len locate the list's stream in
 * the batch's input bytes (in_len = bytes available, at least the stream's
 * size), out_off is the index of its first integer in the output.  Encode:
 * in_off is the index of its first integer in the input, out_off the byte
 * offset of its stream in the output, which must have room for
 * svb_max_compressed_size(n) bytes; in_len is ignored.  prev is the list's
 * start value for differential coding (Sec. 5 starts every list from 0). */
typedef struct svb_list {
    uint64_t in_off;
    uint64_t in_len;
    uint64_t out_off;
    uint32_t n;
    uint32_t prev;
} svb_list;

/* Device bytes of the plan of a batch of num_lists lists. */
size_t svb_batch_plan_bytes(size_t num_lists);

/* Build a batch's work plan on the host from the list lengths in h_lists
 * (HOST memory) and copy it to d_plan (DEVICE, 16-byte aligned,
 * svb_batch_plan_bytes bytes) on stream.  Lists with n >= big_threshold (0:
 * the default, 8192) are decoded by CTAs tile by tile, longest first;
 * shorter ones by one warp each.  A big list of more than 2 * segment_tiles
 * decode tiles (4096 integers unless svb_batch_set_tile chose 8192), and
 * more than a quarter of a CTA's fair share of all big lists' tiles (a GPU's
 * resident decode CTAs sharing them evenly), is cut into units of
 * segment_tiles tiles decoded by several CTAs at once: each batched decode
 * first finds every such unit's data offset and carry-in within its list
 * (one pass over the split lists' streams with a look-back over each list's
 * units), then decodes.  segment_tiles: 0 never splits; at most 32 (16 with
 * tiles of 8192), else SVB_EINVAL.  svb_batch_plan uses the default of 16.
 * A plan stays valid for any batch with the same list
 * lengths; a plan with split lists holds the state of the call using it, so
 * use it in one call at a time, always with the same workspace.  The batched
 * encoder codes every big list whole, whatever the plan. */
int svb_batch_plan(const svb_list *h_lists, size_t num_lists, uint32_t big_threshold,
                   void *d_plan, size_t plan_bytes, svb_stream_t stream);
int svb_batch_plan_segments(const svb_list *h_lists, size_t num_lists, uint32_t big_threshold,
                            uint32_t segment_tiles, void *d_plan, size_t plan_bytes,
                            svb_stream_t stream);

/* Workspace bytes of a batched call (its counters; zero it once with
 * svb_workspace_init, like the single-stream workspace). */
size_t svb_batch_workspace_size(void);

/* Staging depth of the batched kernels, for every later svb_batch_decode /
 * svb_batch_encode of this process: the tiles of compressed bytes (decode)
 * or values (encode) each CTA keeps in flight in shared memory.  Fewer
 * stages take less shared memory, so more CTAs fit on an SM.  Encoding is
 * built at depths 2 and 3; decoding at 2, 3 and 4 for tiles of 4096
 * integers and at 1 and 2 for tiles of 8192 (0 restores the defaults: 2 and
 * 3).  The tuner (autotune.py) picks them per GPU and workload.  No paper
 * counterpart: a launch parameter.  Returns SVB_EINVAL for a depth outside
 * 1..4 (decode) or 2..3 (encode), leaving both settings as they were.
 * svb_batch_get_stages gives the depth in use (encode != 0: the encoder's). */
int svb_batch_set_stages(int decode_stages, int encode_stages);
int svb_batch_get_stages(int encode);

/* Decode tile of the batched decoder, in integers, for every later
 * svb_batch_plan / svb_batch_plan_segments / svb_batch_decode of this
 * process: 4096 (the default; 0 restores it) or 8192.  A CTA's consumer
 * warps decode a tile's sub-tiles of 512 integers, one each (4096) or two
 * each (8192, 32 integers per lane per tile), so larger tiles spread each
 * tile's fixed costs (a stage hand-off, the control-byte scan, one barrier
 * per 4096 integers of differential lists) over more integers.  A plan
 * records the tile it was built for, and its segment_tiles count tiles of
 * that size (segment_tiles * tile at most 32 * 4096 integers):
 * svb_batch_decode with a plan built for another tile decodes nothing and
 * reports SVB_EINVAL in d_result, and svb_batch_decode returns SVB_EINVAL
 * when the depth in use is not built for the tile in use.  The batched
 * encoder keeps tiles of 4096.  No paper counterpart: a launch parameter.
 * Returns SVB_EINVAL for any other size, leaving the setting as it was;
 * svb_batch_get_tile gives the tile in use. */
int svb_batch_set_tile(int tile_ints);
int svb_batch_get_tile(void);

/* Decode / encode every list of the plan in one persistent launch enqueued on
 * stream.  d_lists is the DEVICE copy of the list table.  d_result receives
 * the total bytes consumed / written and the status (SVB_ETRUNCATED when
 * some list's stream is longer than its in_len).  Encode also writes each
 * list's stream size to d_sizes[list] (DEVICE, one uint64_t per list).
 * grid: 0 for one CTA per resident slot, else the number of CTAs. */
int svb_batch_decode(const void *d_plan, const svb_list *d_lists, const uint8_t *in_base,
                     uint32_t *out_base, int delta, svb_result *d_result, void *ws,
                     size_t ws_bytes, int grid, svb_stream_t stream);
int svb_batch_encode(const void *d_plan, const svb_list *d_lists, const uint32_t *in_base,
                     uint8_t *out_base, int delta, uint64_t *d_sizes, svb_result *d_result,
                     void *ws, size_t ws_bytes, int grid, svb_stream_t stream);

/* The same lists coded one list at a time: each list gets its own
 * single-stream call (svb_decode_async / svb_encode_async, the kernels and
 * launches a caller of those gets), all issued from one host loop on
 * `stream`, in table order, sharing one workspace sized for the longest list
 * (svb_workspace_size of it, zeroed once).  h_lists is the HOST copy of the
 * list table, laid out as for svb_batch_decode / svb_batch_encode; the
 * result of list j goes to d_results[j] (DEVICE, num_lists entries).  This
 * is the baseline the batched launch is measured against (Sec. 5 decodes
 * posting lists one at a time).  Returns SVB_OK, or the status of the first
 * call that could not be enqueued (the lists after it are not coded). */
int svb_decode_each(const svb_list *h_lists, size_t num_lists, const uint8_t *in_base,
                    uint32_t *out_base, int delta, svb_result *d_results, void *ws,
                    size_t ws_bytes, svb_stream_t stream);
int svb_encode_each(const svb_list *h_lists, size_t num_lists, const uint32_t *in_base,
                    uint8_t *out_base, int delta, svb_result *d_results, void *ws,
                    size_t ws_bytes, svb_stream_t stream);

/* ---- one array split across several parties ---------------------------- */

/* The per-shard steps of coding one array whose integers are split across P
 * parties (GPUs, or shards on one GPU) at control-byte boundaries: shard p
 * holds integers [4 q_p, min(4 q_{p+1}, n)), i.e. control bytes [q_p,
 * q_{p+1}).  Because the control bytes are kept apart from the data (Sec. 4),
 * one exchange of P byte totals places every shard's data:
 *   decode  (1) svb_control_range_bytes gives the data bytes each shard's
 *           control bytes cover; (2) their exclusive prefix, exchanged, is
 *           each shard's data offset; the shard's control bytes followed by
 *           its data bytes are a stream of its own integers; (3) for
 *           differential streams, svb_gap_sum of each shard's stream, and
 *           prev plus the exclusive prefix of those sums, exchanged, is each
 *           shard's start value (Sec. 2's prefix sum across shards); (4) each
 *           shard decodes its stream (svb_decode_async) from that start.
 *   encode  (1) svb_size_report_async of each shard's integers (for
 *           differential coding from the integer before the shard) less its
 *           control bytes; (2) the exclusive prefix of those, exchanged; (3)
 *           each shard encodes its integers (svb_encode_async); the shards'
 *           control bytes in order, then their data bytes in order, are the
 *           array's stream.
 *
 * svb_control_range_bytes: data bytes that control bytes [q0, q1) of a
 * stream of n integers cover (4 + the sum of codes each; the pad fields of
 * the stream's last control byte count nothing), into *d_bytes (DEVICE) on
 * stream.  Reads in[q0 .. q1) only.  SVB_EINVAL when q0 > q1 or q1 >
 * ceil(n/4).
 *
 * svb_gap_sum: sum mod 2^32 of the n coded values of the stream in[0..in_len)
 * (for a differential stream, the sum of its gaps) into d_out[0], the status
 * into d_out[1] and the stream's bytes into d_out[2] (DEVICE, three
 * uint64_t), on stream, with a caller workspace as for svb_decode_async.
 * Returns SVB_ETRUNCATED at once when in_len < ceil(n/4); a stream cut short
 * inside its data is reported in d_out[1]. */
int svb_control_range_bytes(const uint8_t *in, size_t n, size_t q0, size_t q1,
                            uint64_t *d_bytes, svb_stream_t stream);
int svb_gap_sum(const uint8_t *in, size_t in_len, size_t n, uint64_t *d_out, void *ws,
                size_t ws_bytes, svb_stream_t stream);

/* ---- decoding without allocation --------------------------------------- */

/* Largest n that svb_decode_noalloc accepts. */
#define SVB_NOALLOC_MAX_N ((size_t)1 << 24)

/* Decode like svb_decode_checked, but without allocating anything: no
 * cudaMalloc, cudaFree, pinned host buffer or allocating library call.  The
 * paper has no counterpart; this is for callers that cannot allocate device
 * memory while they decode, such as a custom allocator or memory pool that
 * decodes from inside its own bookkeeping (a nested cudaMalloc would re-enter
 * it), a process whose HBM is already reserved by a framework's caching
 * allocator, or a latency-bound path that cannot afford cudaMalloc/cudaFree,
 * which may synchronize the device.
 *
 * Scratch: a fixed device array of about 1.5 MB inside the library, enough
 * for n <= SVB_NOALLOC_MAX_N; every GPU that loads the library holds it until
 * the process exits.  n > SVB_NOALLOC_MAX_N returns SVB_ERROR with
 * SVB_EINVAL.  The first call on a device looks up the array's device
 * address.  All calls share the array: calls that overlap on the GPU race,
 * so order them on one stream or serialize them on the host.
 *
 * in[0..in_len) is the stream, out[0..n) receives the integers, delta and prev
 * as in svb_decode_checked.  Runs on `stream` and synchronizes it (the byte
 * count comes back through a host copy), so it cannot be called while
 * `stream` is being captured into a CUDA graph.  Returns the bytes consumed,
 * or SVB_ERROR with svb_last_error() set; n = 0 returns 0 with SVB_OK. */
size_t svb_decode_noalloc(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                          uint32_t prev, int delta, svb_stream_t stream);

/* ---- appending ------------------------------------------------------------ */

/* Append k integers to a compressed array without recompressing it (Sec. 4's
 * closing remark: the new data follow the existing data and the control
 * stream grows).  The array is kept as two device buffers that can grow:
 *   ctrl[0 .. ceil(n/4))  its control bytes; room for ceil((n + k)/4);
 *   data[0 .. data_len)   its data bytes; room for data_len + 4k + 3 (n mod 4).
 * Joined, ctrl and data are the usual stream [ctrl][data].  in[0..k) are the
 * new integers (device).  With delta != 0 the array is differentially coded
 * and `last` is its last integer (the start value prev when n = 0); otherwise
 * `last` is unused.  Afterwards the array holds n + k integers, exactly as if
 * all of them had been encoded at once; only the last control byte and the
 * data of its integers are rewritten, so the cost is O(k).  Runs on the
 * current stream and waits for it.  Returns the new data length, or
 * SVB_ERROR with svb_last_error() = SVB_EINVAL (null pointer, too little
 * room, data_len too short for the integers of the last control byte),
 * SVB_ENOMEM, SVB_ECUDA or SVB_ETIMEOUT.  k = 0 returns data_len. */
size_t svb_append(uint8_t *ctrl, size_t ctrl_cap, uint8_t *data, size_t data_cap,
                  size_t data_len, size_t n, const uint32_t *in, size_t k, uint32_t last,
                  int delta);

/* ---- seek and select on compressed lists --------------------------------- */

/* The two operations benchmarked at the end of Sec. 5 (Fig. 6), answered on
 * the compressed bytes of lists held in one pool (a table of svb_list as for
 * the batched codec; out_off is not used), many queries per launch:
 *   SVB_SEEK    arg = target (< 2^32): index of the first integer >= target
 *               and that integer; n and 0 when there is none;
 *   SVB_SELECT  arg = index i < n: the integer at i (index = i).
 * delta != 0 reads every list as differentially coded from its prev (the
 * paper's setting: sorted lists, Sec. 5).  Each answer's status is SVB_OK,
 * SVB_EINVAL (list id >= num_lists, unknown op, select index >= n) or
 * SVB_ETRUNCATED (the list's in_len holds fewer than its ceil(n/4) control
 * bytes, or not the data bytes of the integer that decides the answer).  No
 * byte outside a list's [in_off, in_off + in_len) is read.
 * All pointers are device pointers; answers[k] answers queries[k].  Runs on
 * `stream` and returns at once: SVB_OK, SVB_EINVAL (null pointer with
 * num_queries > 0) or SVB_ECUDA. */
#define SVB_SEEK 0
#define SVB_SELECT 1

typedef struct svb_query {
    uint32_t list;   /* index into the list table */
    uint32_t op;     /* SVB_SEEK or SVB_SELECT */
    uint64_t arg;    /* seek: target; select: index */
} svb_query;

typedef struct svb_answer {
    uint64_t index;  /* seek: position found (n if none); select: the index */
    uint32_t value;  /* the integer there (0 if none or on error) */
    uint32_t status; /* svb_status */
} svb_answer;

int svb_query_batch(const svb_list *d_lists, size_t num_lists, const uint8_t *in_base, int delta,
                    const svb_query *d_queries, size_t num_queries, svb_answer *d_answers,
                    svb_stream_t stream);

/* ---- compressed-size report: Stream VByte against VByte ------------------ */

/* Sizes of n integers coded two ways, without writing either stream (Sec. 5,
 * Fig. 5b: the extra bits per integer of Stream VByte over VByte):
 *   sizes[0]  Stream VByte bytes: ceil(n/4) control bytes plus L(v) =
 *             max(1, ceil(bits(v)/8)) data bytes per coded value (Sec. 3-4);
 *   sizes[1]  VByte bytes: max(1, ceil(bits(v)/7)) per coded value, seven
 *             data bits and one continuation bit per byte (Sec. 2-3).
 * The coded values are the integers, or with delta != 0 their differences
 * x_i - x_{i-1} mod 2^32 with x_{-1} = prev (Sec. 1, Sec. 5).
 * in: device array of n uint32 (any alignment; 16-byte aligned is faster).
 * svb_size_report writes the two sizes to the host array `sizes`, running on
 * the current stream and waiting for it; svb_size_report_async writes them to
 * the device array d_sizes (two uint64) on `stream` and returns at once.
 * Both return SVB_OK, SVB_EINVAL (null sizes, or null in with n > 0) or
 * SVB_ECUDA / SVB_ENOMEM, also left in svb_last_error().  n = 0 gives 0, 0. */
int svb_size_report(const uint32_t *in, size_t n, uint32_t prev, int delta, uint64_t *sizes);
int svb_size_report_async(const uint32_t *in, size_t n, uint32_t prev, int delta,
                          uint64_t *d_sizes, svb_stream_t stream);

/* ---- test hook ---------------------------------------------------------- */

/* Failure-detection check: launches one decode tile whose predecessor is
 * never published, so its cross-tile wait runs out after spin_limit polls.
 * The call must report SVB_ETIMEOUT in d_result and leave the context
 * usable.  stream_in holds a stream of n >= 2 * 4096 integers. */
int svb_testhook_lookback_timeout(const uint8_t *stream_in, size_t n, uint32_t *out,
                                  uint64_t spin_limit, svb_result *d_result, void *ws,
                                  size_t ws_bytes, svb_stream_t stream);

/* Failure-detection check of the offsets pass (the reduce-then-decode
 * decoder's first kernel): its one CTA takes the second range of control
 * bytes and waits for the first range's byte total, which nothing publishes,
 * so the wait runs out after spin_limit polls.  A decode of all tiles
 * follows, which decodes nothing.  d_result must then hold SVB_ETIMEOUT, and
 * the workspace and context stay usable.  stream_in holds a stream of
 * n > 65,536 integers (at least two ranges of 16,384 control bytes);
 * ws is an initialised workspace of svb_workspace_size(n) bytes.  Returns
 * SVB_OK, SVB_EINVAL or SVB_ECUDA. */
int svb_testhook_offsets_timeout(const uint8_t *stream_in, size_t n, uint32_t *out,
                                 uint64_t spin_limit, svb_result *d_result, void *ws,
                                 size_t ws_bytes, svb_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SVB_H */
