// Launchers behind the C ABI (host side of the kernels).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace svb {

typedef unsigned long long u64;
struct DeviceResult;

// Decode n integers; returns an svb_status (0 or SVB_ECUDA for a launch error).
int launch_decode(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                  bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                  u64 spin_limit, u64 tile_base = 0, u64 grid_override = 0);
u64 decode_tiles(u64 n);

// Reduce-then-decode: control-stream offsets pass, then a persistent decode
// with bulk-copy staging.
int launch_decode_tiled(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                        bool delta, void *ws, DeviceResult *result, cudaStream_t stream,
                        u64 spin_limit);

int launch_encode(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta, void *ws,
                  DeviceResult *result, cudaStream_t stream, u64 spin_limit);
u64 encode_tiles(u64 n);

// Record the calling thread's status for svb_last_error().
void set_last_error(int code);

}  // namespace svb
