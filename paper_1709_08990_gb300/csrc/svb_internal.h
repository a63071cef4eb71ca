// Launchers behind the C ABI (host side of the kernels).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "svb.h"

namespace svb {

typedef unsigned long long u64;
struct DeviceResult;

// Decode n integers; returns an svb_status (0 or SVB_ECUDA for a launch error).
int launch_decode(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                  bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                  u64 spin_limit, u64 tile_base = 0, u64 grid_override = 0);
u64 decode_tiles(u64 n);

// Reduce-then-decode: control-stream offsets pass, then a persistent decode
// with bulk-copy staging.  Differential streams get their carry-ins in the
// offsets pass, or, with sums_pass, from a separate pass over staged tiles.
int launch_decode_chunked(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, void *ws,
                          DeviceResult *result, cudaStream_t stream, u64 spin_limit);
int launch_decode_tiled(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                        bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                        u64 spin_limit, bool sums_pass = false);

// Sum of a stream's n coded values (mod 2^32) into d_out[0], its status into
// d_out[1] and its bytes into d_out[2] (the differential offsets pass run from
// 0, then one warp totals the ranges).
int launch_gap_sum(const uint8_t *in, u64 in_len, u64 n, void *ws, u64 *d_out,
                   cudaStream_t stream, u64 spin_limit);

// Its two halves, for decoding in pieces: the offsets pass (sub-tile offsets,
// stream size and truncation verdict into the workspace), then plain decodes
// of tile ranges [tile0, tile1) of decode_tile_ints() integers each tile.
int launch_offsets(const uint8_t *in, u64 in_len, u64 n, void *ws, cudaStream_t stream,
                   u64 spin_limit);
int launch_decode_range(const uint8_t *in, u64 n, uint32_t *out, void *ws, DeviceResult *result,
                        cudaStream_t stream, u64 tile0, u64 tile1);
// Failure-detection check of the offsets pass's bounded wait (see
// svb_testhook_offsets_timeout).
int launch_offsets_timeout_check(const uint8_t *in, u64 n, uint32_t *out, void *ws,
                                 DeviceResult *result, cudaStream_t stream, u64 spin_limit);
u64 decode_tile_ints();

int launch_encode(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta, void *ws,
                  DeviceResult *result, cudaStream_t stream, u64 spin_limit);
u64 encode_tiles(u64 n);

// Small arrays in one cooperative launch (svb_small.cu): one CTA per tile
// of 4096 integers, a grid barrier between sizing and coding.  Return 0, or
// 3 when the grid cannot be made resident or the stream is being captured
// (the caller then takes another path; nothing was enqueued).
int launch_decode_small(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, void *ws,
                        DeviceResult *result, cudaStream_t stream, u64 spin_limit);
int launch_encode_small(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta,
                        void *ws, DeviceResult *result, cudaStream_t stream, u64 spin_limit);
u64 small_tiles(u64 n);

// Chunked single-pass encoder (svb_encode_tiled.cu).  Control bytes go to
// out; data bytes to out + ceil(n/4), or, when data is given, to
// data - *data_back (data_back a device pointer, or null for 0).
int launch_encode_tiled(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta,
                        void *ws, DeviceResult *result, cudaStream_t stream, u64 spin_limit,
                        uint8_t *data = nullptr, const u64 *data_back = nullptr);

// Append k integers to a stream kept as separate control and data buffers
// (svb_append.cu); scratch holds the re-coded tail and the new values
// (append_scratch_bytes(k)), ws/result are an encoder workspace.  result->bytes
// becomes the new data length.
size_t append_scratch_bytes(u64 k);
int launch_append(uint8_t *ctrl, uint8_t *data, u64 data_len, u64 n, const uint32_t *in, u64 k,
                  uint32_t last, bool delta, void *scratch, void *ws, DeviceResult *result,
                  cudaStream_t stream, u64 spin_limit);

// Batched codec (svb_batch.cu).
// Staging depth of the batched decode (2..4) and encode (2, 3) kernels; 0
// for the default.  Returns 0, or 1 for a depth that is not built.
int batch_set_stages(int decode_stages, int encode_stages);
int batch_stages(int encode);
int batch_set_tile(int tile_ints);
int batch_tile(void);
int launch_batch_decode(const void *d_plan, const svb_list *d_lists, const uint8_t *in,
                        uint32_t *out, bool delta, void *ws, DeviceResult *result,
                        cudaStream_t stream, int grid);
int launch_batch_encode(const void *d_plan, const svb_list *d_lists, const uint32_t *in,
                        uint8_t *out, u64 *sizes, bool delta, void *ws, DeviceResult *result,
                        cudaStream_t stream, int grid);
size_t batch_plan_bytes(size_t num_lists);
int build_batch_plan(const svb_list *h_lists, size_t num_lists, uint32_t threshold,
                     uint32_t seg_tiles, void *d_plan, cudaStream_t stream);
uint32_t batch_default_seg_tiles();

// Seek / select queries on a pool of lists (svb_query.cu).
int launch_query(const svb_list *lists, u64 num_lists, const uint8_t *in, bool delta,
                 const svb_query *queries, u64 num_queries, svb_answer *answers,
                 cudaStream_t stream);

// Stream VByte and VByte sizes of n values into d_sizes[0..2) (svb_size.cu).
int launch_size_report(const uint32_t *in, u64 n, uint32_t prev, bool delta, u64 *d_sizes,
                       cudaStream_t stream);

// Per-kernel CUDA-event timing (svb_profile.cu); no-ops unless profiling is on.
void prof_begin(const char *name, cudaStream_t s);
void prof_end(cudaStream_t s);

// Record the calling thread's status for svb_last_error().
void set_last_error(int code);

}  // namespace svb
