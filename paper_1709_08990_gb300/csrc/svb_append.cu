// Appending integers to a compressed array without recompressing it (the
// format section's closing remark, Sec. 4: the new integers' data go after the
// existing data and the control stream occasionally grows).
//
// The stream is kept as two buffers that can grow: control bytes and data
// bytes (joined, they are the usual [ctrl][data] stream).  Appending k
// integers to n:
//   * the r = n mod 4 integers of the incomplete last control byte share
//     their control byte with the first new ones, so they are taken back:
//     their coded values are read from the last bytes of the data stream
//     (their lengths from the control byte, Sec. 4);
//   * those r values, then the k new coded values (gaps, the first from the
//     last existing integer, for differential coding), are encoded by the
//     chunked encoder straight into place: control bytes from index
//     floor(n/4), data bytes from the start of the r values' data.
// Nothing before the last control byte or before those r values' data is
// read or written, so an append costs O(k), not O(n).  The result equals
// encoding all n + k integers at once.
#include <cuda_runtime.h>

#include <algorithm>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"

namespace svb {

// Scratch layout: [u64 tail, u64 bad][uint32 values x (k + 3)].
constexpr size_t kAppendHead = 16;

size_t append_scratch_bytes(u64 k)
{
    return kAppendHead + 4 * (k + 3);
}

struct AppendArgs {
    const uint8_t *ctrl;
    const uint8_t *data;
    u64 data_len, n, k;
    const uint32_t *in;
    uint32_t last;
    uint32_t delta;
    u64 *head;         // [0] tail: data bytes of the r taken-back values; [1] nonzero if
                       // data_len cannot hold them
    uint32_t *vals;    // r + k values to encode
};

__global__ void append_prep_kernel(AppendArgs a)
{
    const uint32_t r = (uint32_t)(a.n % 4);
    const u64 total = r + a.k;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        if (i < r) {
            // Field i of the incomplete last control byte and its bytes.
            const uint32_t c = a.ctrl[a.n / 4];
            uint32_t tail = 0, off = 0;
            for (uint32_t j = 0; j < r; j++) {
                const uint32_t len = ((c >> (2 * j)) & 3u) + 1;
                off += j < i ? len : 0u;
                tail += len;
            }
            const uint32_t len = ((c >> (2 * i)) & 3u) + 1;
            uint32_t v = 0;
            if (tail <= a.data_len) {
                const uint8_t *p = a.data + a.data_len - tail + off;
                for (uint32_t b = 0; b < len; b++)
                    v |= (uint32_t)p[b] << (8 * b);
            }
            a.vals[i] = v;
            if (i == 0) {
                a.head[0] = tail <= a.data_len ? tail : 0;
                a.head[1] = tail <= a.data_len ? 0 : 1;
            }
        } else {
            const u64 j = i - r;
            const uint32_t x = a.in[j];
            a.vals[i] = a.delta ? x - (j ? a.in[j - 1] : a.last) : x;
        }
    }
    if (r == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        a.head[0] = 0;
        a.head[1] = 0;
    }
}

// The encoder reported ceil((r+k)/4) + data bytes of the r + k values; the
// stream's data now ends at data_len - tail + those data bytes.
__global__ void append_finish_kernel(DeviceResult *result, const u64 *head, u64 data_len,
                                     u64 ctrl_bytes)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    if (head[1]) {
        result->bytes = ~0ull;
        result->status = SVB_EINVAL;
        return;
    }
    if (result->status == 0)
        result->bytes = data_len - head[0] + (result->bytes - ctrl_bytes);
}

int launch_append(uint8_t *ctrl, uint8_t *data, u64 data_len, u64 n, const uint32_t *in, u64 k,
                  uint32_t last, bool delta, void *scratch, void *ws, DeviceResult *result,
                  cudaStream_t stream, u64 spin_limit)
{
    const uint32_t r = (uint32_t)(n % 4);
    AppendArgs a;
    a.ctrl = ctrl;
    a.data = data;
    a.data_len = data_len;
    a.n = n;
    a.k = k;
    a.in = in;
    a.last = last;
    a.delta = delta ? 1u : 0u;
    a.head = static_cast<u64 *>(scratch);
    a.vals = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + kAppendHead);
    const u64 total = r + k;
    const unsigned blocks = (unsigned)std::min<u64>((total + 255) / 256, 4096);
    prof_begin("append_prep_kernel", stream);
    append_prep_kernel<<<blocks ? blocks : 1, 256, 0, stream>>>(a);
    prof_end(stream);
    if (cudaGetLastError() != cudaSuccess)
        return SVB_ECUDA;
    // Encode the r + k values into place: control bytes from floor(n/4), data
    // from data + data_len - tail (tail read on the device).
    int st = launch_encode_tiled(a.vals, total, ctrl + n / 4, 0, false, ws, result, stream,
                                 spin_limit, data + data_len, a.head);
    if (st != 0)
        return SVB_ECUDA;
    append_finish_kernel<<<1, 32, 0, stream>>>(result, a.head, data_len, (total + 3) / 4);
    return cudaGetLastError() == cudaSuccess ? SVB_OK : SVB_ECUDA;
}

}  // namespace svb
