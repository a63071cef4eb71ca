// The C ABI of include/svb.h: argument checks, the per-device workspace used
// by the synchronous calls, stream and error bookkeeping.  All computation
// happens in the kernels; nothing here decodes or encodes on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "svb.h"
#include "svb_device.cuh"
#include "svb_internal.h"

using svb::u64;

namespace {

thread_local int t_last_error = SVB_OK;
thread_local cudaStream_t t_stream = nullptr;
std::atomic<u64> g_spin_limit{0};
std::atomic<int> g_decode_variant{SVB_DECODE_AUTO};
std::atomic<int> g_encode_variant{SVB_ENCODE_AUTO};

constexpr u64 kDefaultSpinLimit = 1ull << 21;  // ~2 s of polling at most
constexpr u64 kSmallPlain = 1ull << 20;         // plain streams decoded in one launch
constexpr u64 kSmallArray = 1ull << 22;         // arrays tried with the one-launch kernels

u64 spin_limit()
{
    u64 v = g_spin_limit.load(std::memory_order_relaxed);
    if (v)
        return v;
    static const u64 env = [] {
        const char *s = std::getenv("SVB_LOOKBACK_SPIN_LIMIT");
        if (s && *s) {
            unsigned long long x = std::strtoull(s, nullptr, 10);
            if (x > 0)
                return (u64)x;
        }
        return kDefaultSpinLimit;
    }();
    return env;
}

int decode_dispatch(const uint8_t *in, u64 in_len, u64 n, uint32_t *out, uint32_t prev,
                    bool delta, void *ws, svb::DeviceResult *r, cudaStream_t s)
{
    const int v = g_decode_variant.load(std::memory_order_relaxed);
    // Small plain streams are launch-bound: one launch beats the offsets pass
    // plus the tiled decode there.  The one-launch small-array decoder comes
    // first; where it cannot run (too many tiles to be resident at once, or
    // a stream being captured), the single pass does.
    if (!delta && n && (v == SVB_DECODE_SMALL || (v == SVB_DECODE_AUTO && n <= kSmallArray)) &&
        svb::launch_decode_small(in, in_len, n, out, ws, r, s, spin_limit()) == 0)
        return 0;
    if (v == SVB_DECODE_CHUNKED && !delta && in_len >= (n + 3) / 4)
        return svb::launch_decode_chunked(in, in_len, n, out, ws, r, s, spin_limit());
    if (v == SVB_DECODE_SINGLE_PASS ||
        ((v == SVB_DECODE_AUTO || v == SVB_DECODE_SMALL) && !delta && n <= kSmallPlain))
        return svb::launch_decode(in, in_len, n, out, prev, delta, ws, r, s, spin_limit());
    return svb::launch_decode_tiled(in, in_len, n, out, prev, delta, ws, r, s, spin_limit(),
                                    v == SVB_DECODE_SUMS_PASS);
}

int encode_dispatch(const uint32_t *in, u64 n, uint8_t *out, uint32_t prev, bool delta,
                    void *ws, svb::DeviceResult *r, cudaStream_t s)
{
    const int v = g_encode_variant.load(std::memory_order_relaxed);
    if (v == SVB_ENCODE_TILE_LOOKBACK)
        return svb::launch_encode(in, n, out, prev, delta, ws, r, s, spin_limit());
    if (n && (v == SVB_ENCODE_SMALL || (v == SVB_ENCODE_AUTO && n <= kSmallArray)) &&
        svb::launch_encode_small(in, n, out, prev, delta, ws, r, s, spin_limit()) == 0)
        return 0;
    return svb::launch_encode_tiled(in, n, out, prev, delta, ws, r, s, spin_limit());
}

size_t set_error(int code)
{
    t_last_error = code;
    return code == SVB_OK ? 0 : SVB_ERROR;
}

// Workspace kept per device for the synchronous calls.  The calls on one
// device serialise on its mutex: they share the workspace and wait anyway.
struct DeviceCache {
    std::mutex mu;
    void *ws = nullptr;
    size_t bytes = 0;
    svb_result *h_res = nullptr;  // pinned
};

constexpr int kMaxDevices = 64;
DeviceCache g_cache[kMaxDevices];

// Grows c's workspace to hold a launch over n integers (zeroed when grown);
// call with c.mu held.
int ensure_workspace(DeviceCache &c, size_t n, cudaStream_t s)
{
    size_t need = svb_workspace_size(n);
    if (c.bytes < need) {
        size_t grow = std::max(need, 2 * c.bytes);
        if (c.ws) {
            cudaDeviceSynchronize();
            cudaFree(c.ws);
            c.ws = nullptr;
            c.bytes = 0;
        }
        if (cudaMalloc(&c.ws, grow) != cudaSuccess) {
            cudaGetLastError();
            c.ws = nullptr;
            return SVB_ENOMEM;
        }
        if (cudaMemsetAsync(c.ws, 0, grow, s) != cudaSuccess)
            return SVB_ECUDA;
        c.bytes = grow;
    }
    if (!c.h_res && cudaMallocHost(&c.h_res, sizeof(svb_result)) != cudaSuccess) {
        c.h_res = nullptr;
        return SVB_ENOMEM;
    }
    return SVB_OK;
}

template <class F>
size_t run_sync(size_t n, F &&launch)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(SVB_ECUDA);
    DeviceCache &c = g_cache[dev];
    std::lock_guard<std::mutex> lock(c.mu);
    cudaStream_t s = t_stream;
    if (int st = ensure_workspace(c, n, s))
        return set_error(st);
    auto *d_res = reinterpret_cast<svb::DeviceResult *>(static_cast<char *>(c.ws) +
                                                         svb::kResultOffset);
    int st = launch(c.ws, d_res, s);
    if (st != SVB_OK)
        return set_error(st);
    if (cudaMemcpyAsync(c.h_res, d_res, sizeof(svb_result), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_error(SVB_ECUDA);
    if (c.h_res->status != SVB_OK)
        return set_error((int)c.h_res->status);
    t_last_error = SVB_OK;
    return (size_t)c.h_res->bytes;
}

size_t encode_sync(const uint32_t *in, size_t n, uint8_t *out, uint32_t prev, bool delta)
{
    if (n == 0)
        return set_error(SVB_OK);
    if (!in || !out)
        return set_error(SVB_EINVAL);
    return run_sync(n, [&](void *ws, svb::DeviceResult *r, cudaStream_t s) {
        return encode_dispatch(in, n, out, prev, delta, ws, r, s);
    });
}

size_t decode_sync(const uint8_t *in, u64 in_len, size_t n, uint32_t *out, uint32_t prev,
                   bool delta)
{
    if (n == 0)
        return set_error(SVB_OK);
    if (!in || !out)
        return set_error(SVB_EINVAL);
    if (in_len < ((u64)n + 3) / 4)
        return set_error(SVB_ETRUNCATED);
    return run_sync(n, [&](void *ws, svb::DeviceResult *r, cudaStream_t s) {
        return decode_dispatch(in, in_len, n, out, prev, delta, ws, r, s);
    });
}

// Scratch for appends (the re-coded tail and the new values), per device;
// kept apart from the encoder workspace so its bytes never pass for records.
struct ScratchCache {
    std::mutex mu;
    void *p = nullptr;
    size_t bytes = 0;
};
ScratchCache g_append_scratch[kMaxDevices];

// ---- host-buffer decode in pieces ------------------------------------------
//
// For a plain stream of many tiles the copy in, the decode and the copy out
// overlap: the control bytes go first and the data bytes follow in chunks on
// a second stream; once the offsets pass has placed every tile, each group of
// tiles is decoded as soon as the chunk holding its last data byte has
// landed, and its integers go back to the host on a third stream while the
// next group decodes.  The two copy directions run at the same time.

constexpr u64 kPieceTiles = 4096;          // tiles per decode launch (16 M integers)
constexpr size_t kCopyChunk = 64u << 20;   // bytes per host-to-device copy
constexpr int kMaxPieces = 256;
constexpr int kMaxCopies = 256;

struct HostPipe {
    bool ready = false;
    cudaStream_t s_cmp = nullptr, s_in = nullptr, s_out = nullptr;
    cudaEvent_t start = nullptr, in_done = nullptr, cmp_done = nullptr;
    cudaEvent_t in_ev[kMaxCopies] = {}, dec_ev[kMaxPieces] = {};
    u64 *h_meta = nullptr;                  // pinned: error, total, piece offsets
    svb::DeviceResult *d_res = nullptr;     // one result per piece
    svb_result *h_res = nullptr;            // pinned copy of those
};
HostPipe g_pipe[kMaxDevices];

int pipe_init(HostPipe &p)
{
    if (p.ready)
        return SVB_OK;
    const unsigned ef = cudaEventDisableTiming;
    bool ok = cudaStreamCreateWithFlags(&p.s_cmp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.s_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.start, ef) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.in_done, ef) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.cmp_done, ef) == cudaSuccess;
    for (int i = 0; ok && i < kMaxCopies; i++)
        ok = cudaEventCreateWithFlags(&p.in_ev[i], ef) == cudaSuccess;
    for (int i = 0; ok && i < kMaxPieces; i++)
        ok = cudaEventCreateWithFlags(&p.dec_ev[i], ef) == cudaSuccess;
    ok = ok && cudaMallocHost(&p.h_meta, (2 + kMaxPieces) * sizeof(u64)) == cudaSuccess &&
         cudaMalloc(&p.d_res, kMaxPieces * sizeof(svb::DeviceResult)) == cudaSuccess &&
         cudaMallocHost(&p.h_res, kMaxPieces * sizeof(svb_result)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return SVB_ENOMEM;
    }
    p.ready = true;
    return SVB_OK;
}

size_t decode_host_pieces(const uint8_t *h_in, u64 in_len, u64 n, uint32_t *h_out, uint8_t *d_in,
                          uint32_t *d_out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(SVB_ECUDA);
    DeviceCache &c = g_cache[dev];
    std::lock_guard<std::mutex> lock(c.mu);
    HostPipe &p = g_pipe[dev];
    cudaStream_t caller = t_stream;
    if (int st = pipe_init(p))
        return set_error(st);
    if (int st = ensure_workspace(c, n, caller))
        return set_error(st);
    const u64 nquads = (n + 3) / 4;
    const u64 tile_ints = svb::decode_tile_ints();
    const u64 ntiles = (n + tile_ints - 1) / tile_ints;
    const u64 piece = std::max<u64>(kPieceTiles, (ntiles + kMaxPieces - 1) / kMaxPieces);
    const u64 npieces = (ntiles + piece - 1) / piece;
    const u64 dbytes = in_len - nquads;
    const size_t chunk = std::max<size_t>(kCopyChunk, (dbytes + kMaxCopies - 1) / kMaxCopies);
    const u64 ncopies = (dbytes + chunk - 1) / chunk;
    const svb::WsLayout L = svb::ws_layout(n);
    const u64 *offs = reinterpret_cast<const u64 *>(static_cast<char *>(c.ws) + L.offs);

    // After the caller's earlier work (and the workspace's zeroing).
    if (cudaEventRecord(p.start, caller) != cudaSuccess ||
        cudaStreamWaitEvent(p.s_cmp, p.start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(p.s_in, p.start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(p.s_out, p.start, 0) != cudaSuccess)
        return set_error(SVB_ECUDA);
    bool ok = cudaMemcpyAsync(d_in, h_in, nquads, cudaMemcpyHostToDevice, p.s_cmp) == cudaSuccess;
    for (u64 j = 0; ok && j < ncopies; j++) {
        const u64 o = nquads + j * chunk, len = std::min<u64>(chunk, in_len - o);
        ok = cudaMemcpyAsync(d_in + o, h_in + o, len, cudaMemcpyHostToDevice, p.s_in) ==
                 cudaSuccess &&
             cudaEventRecord(p.in_ev[j], p.s_in) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(p.in_done, p.s_in) == cudaSuccess;
    // Offsets, then the error word, the stream size and each piece's data offset.
    ok = ok && svb::launch_offsets(d_in, in_len, n, c.ws, p.s_cmp, spin_limit()) == 0 &&
         cudaMemcpyAsync(p.h_meta, static_cast<char *>(c.ws) + offsetof(svb::WsHeader, error),
                         2 * sizeof(u64), cudaMemcpyDeviceToHost, p.s_cmp) == cudaSuccess &&
         cudaMemcpy2DAsync(p.h_meta + 2, sizeof(u64), offs, piece * (tile_ints / 512) * sizeof(u64),
                           sizeof(u64), npieces, cudaMemcpyDeviceToHost, p.s_cmp) == cudaSuccess &&
         cudaStreamSynchronize(p.s_cmp) == cudaSuccess;
    if (!ok)
        return set_error(SVB_ECUDA);
    const u64 err = p.h_meta[0], total = p.h_meta[1];
    u64 pieces_run = 0;
    if (err) {
        // One decode over everything: it sees the error, skips the work and
        // readies the workspace for the next call.
        ok = cudaStreamWaitEvent(p.s_cmp, p.in_done, 0) == cudaSuccess &&
             svb::launch_decode_range(d_in, n, d_out, c.ws, p.d_res, p.s_cmp, 0, ntiles) == 0;
        pieces_run = 1;
    } else {
        for (u64 k = 0; ok && k < npieces; k++) {
            const u64 t0 = k * piece, t1 = std::min(t0 + piece, ntiles);
            // Data bytes this piece may read: its own, plus up to 15 of the
            // next piece's (tiles are copied as 16-byte-aligned ranges).
            const u64 dend = k + 1 < npieces ? p.h_meta[2 + k + 1] : total - nquads;
            const u64 need = std::min<u64>(dend + 16, dbytes);
            if (need)
                ok = cudaStreamWaitEvent(p.s_cmp, p.in_ev[std::min<u64>((need - 1) / chunk,
                                                                        ncopies - 1)],
                                         0) == cudaSuccess;
            ok = ok &&
                 svb::launch_decode_range(d_in, n, d_out, c.ws, p.d_res + k, p.s_cmp, t0, t1) ==
                     0 &&
                 cudaEventRecord(p.dec_ev[k], p.s_cmp) == cudaSuccess &&
                 cudaStreamWaitEvent(p.s_out, p.dec_ev[k], 0) == cudaSuccess;
            const u64 i0 = t0 * tile_ints, i1 = std::min(t1 * tile_ints, n);
            ok = ok && cudaMemcpyAsync(h_out + i0, d_out + i0, 4 * (i1 - i0),
                                       cudaMemcpyDeviceToHost, p.s_out) == cudaSuccess;
        }
        pieces_run = npieces;
    }
    ok = ok && cudaEventRecord(p.cmp_done, p.s_cmp) == cudaSuccess &&
         cudaStreamWaitEvent(p.s_out, p.cmp_done, 0) == cudaSuccess &&
         cudaStreamWaitEvent(p.s_out, p.in_done, 0) == cudaSuccess &&
         cudaMemcpyAsync(p.h_res, p.d_res, pieces_run * sizeof(svb_result),
                         cudaMemcpyDeviceToHost, p.s_out) == cudaSuccess &&
         cudaStreamSynchronize(p.s_out) == cudaSuccess;
    if (!ok)
        return set_error(SVB_ECUDA);
    if (err)
        return set_error((int)err);
    for (u64 k = 0; k < pieces_run; k++)
        if (p.h_res[k].status != SVB_OK)
            return set_error((int)p.h_res[k].status);
    t_last_error = SVB_OK;
    return (size_t)total;
}

}  // namespace

void svb::set_last_error(int code)
{
    t_last_error = code;
}

extern "C" {

size_t svb_max_compressed_size(size_t n)
{
    return (n + 3) / 4 + 4 * n;
}

size_t svb_compressed_size_from_control(const uint8_t *h_ctrl, size_t n)
{
    if (n == 0)
        return 0;
    if (!h_ctrl)
        return set_error(SVB_EINVAL);
    size_t nq = (n + 3) / 4, total = nq;
    for (size_t q = 0; q < nq; q++) {
        unsigned c = h_ctrl[q];
        unsigned k = (q == nq - 1) ? (unsigned)(n - 4 * q) : 4u;
        if (k < 4)
            c &= (1u << (2 * k)) - 1u;
        total += k + (unsigned)__builtin_popcount(c & 0x55u) +
                 2u * (unsigned)__builtin_popcount(c & 0xAAu);
    }
    t_last_error = SVB_OK;
    return total;
}

size_t svb_encode(const uint32_t *in, size_t n, uint8_t *out)
{
    return encode_sync(in, n, out, 0, false);
}

size_t svb_decode(const uint8_t *in, size_t n, uint32_t *out)
{
    return decode_sync(in, ~0ull, n, out, 0, false);
}

size_t svb_delta_encode(const uint32_t *in, size_t n, uint8_t *out, uint32_t prev)
{
    return encode_sync(in, n, out, prev, true);
}

size_t svb_delta_decode(const uint8_t *in, size_t n, uint32_t *out, uint32_t prev)
{
    return decode_sync(in, ~0ull, n, out, prev, true);
}

size_t svb_decode_checked(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                          uint32_t prev, int delta)
{
    return decode_sync(in, in_len, n, out, prev, delta != 0);
}

size_t svb_decode_host(const uint8_t *h_in, size_t in_len, size_t n, uint32_t *h_out,
                       uint32_t prev, int delta, uint8_t *d_in, uint32_t *d_out)
{
    if (n == 0)
        return set_error(SVB_OK);
    if (!h_in || !h_out || !d_in || !d_out)
        return set_error(SVB_EINVAL);
    // Large plain streams: copies and decode overlap, piece by piece.
    if (!delta && n >= 2 * kPieceTiles * svb::decode_tile_ints() &&
        in_len >= ((u64)n + 3) / 4 &&
        g_decode_variant.load(std::memory_order_relaxed) != SVB_DECODE_SINGLE_PASS)
        return decode_host_pieces(h_in, in_len, n, h_out, d_in, d_out);
    cudaStream_t s = t_stream;
    if (cudaMemcpyAsync(d_in, h_in, in_len, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return set_error(SVB_ECUDA);
    size_t k = decode_sync(d_in, in_len, n, d_out, prev, delta != 0);
    if (k == SVB_ERROR)
        return k;
    if (cudaMemcpyAsync(h_out, d_out, 4 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_error(SVB_ECUDA);
    t_last_error = SVB_OK;
    return k;
}

size_t svb_encode_host(const uint32_t *h_in, size_t n, uint8_t *h_out, uint32_t prev,
                       int delta, uint32_t *d_in, uint8_t *d_out)
{
    if (n == 0)
        return set_error(SVB_OK);
    if (!h_in || !h_out || !d_in || !d_out)
        return set_error(SVB_EINVAL);
    cudaStream_t s = t_stream;
    if (cudaMemcpyAsync(d_in, h_in, 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return set_error(SVB_ECUDA);
    size_t k = encode_sync(d_in, n, d_out, prev, delta != 0);
    if (k == SVB_ERROR)
        return k;
    if (cudaMemcpyAsync(h_out, d_out, k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_error(SVB_ECUDA);
    t_last_error = SVB_OK;
    return k;
}

size_t svb_append(uint8_t *ctrl, size_t ctrl_cap, uint8_t *data, size_t data_cap,
                  size_t data_len, size_t n, const uint32_t *in, size_t k, uint32_t last,
                  int delta)
{
    if (!ctrl || !data || (k && !in))
        return set_error(SVB_EINVAL);
    if (k == 0) {
        t_last_error = SVB_OK;
        return data_len;
    }
    const size_t r = n % 4;
    if (ctrl_cap < (n + k + 3) / 4 || data_cap < data_len + 4 * k + 3 * r)
        return set_error(SVB_EINVAL);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(SVB_ECUDA);
    ScratchCache &sc = g_append_scratch[dev];
    std::lock_guard<std::mutex> lock(sc.mu);
    const size_t need = svb::append_scratch_bytes(k);
    if (sc.bytes < need) {
        if (sc.p) {
            cudaDeviceSynchronize();
            cudaFree(sc.p);
            sc.p = nullptr;
            sc.bytes = 0;
        }
        const size_t grow = std::max(need, 2 * sc.bytes);
        if (cudaMalloc(&sc.p, grow) != cudaSuccess) {
            cudaGetLastError();
            sc.p = nullptr;
            return set_error(SVB_ENOMEM);
        }
        sc.bytes = grow;
    }
    return run_sync(k + 3, [&](void *ws, svb::DeviceResult *res, cudaStream_t s) {
        return svb::launch_append(ctrl, data, data_len, n, in, k, last, delta != 0, sc.p, ws, res,
                                  s, spin_limit());
    });
}

int svb_set_stream(svb_stream_t stream)
{
    t_stream = reinterpret_cast<cudaStream_t>(stream);
    return SVB_OK;
}

svb_stream_t svb_get_stream(void)
{
    return reinterpret_cast<svb_stream_t>(t_stream);
}

int svb_last_error(void)
{
    return t_last_error;
}

const char *svb_error_string(int status)
{
    switch (status) {
    case SVB_OK: return "ok";
    case SVB_EINVAL: return "invalid argument";
    case SVB_ETRUNCATED: return "compressed input shorter than its control bytes require";
    case SVB_ECUDA: return "CUDA error";
    case SVB_ETIMEOUT: return "cross-tile wait exceeded its spin limit";
    case SVB_ENOMEM: return "out of device memory";
    default: return "unknown status";
    }
}

int svb_set_decode_variant(int variant)
{
    if (variant < SVB_DECODE_AUTO || variant > SVB_DECODE_CHUNKED)
        return SVB_EINVAL;
    g_decode_variant.store(variant, std::memory_order_relaxed);
    return SVB_OK;
}

int svb_set_encode_variant(int variant)
{
    if (variant < SVB_ENCODE_AUTO || variant > SVB_ENCODE_SMALL)
        return SVB_EINVAL;
    g_encode_variant.store(variant, std::memory_order_relaxed);
    return SVB_OK;
}

void svb_set_spin_limit(uint64_t iterations)
{
    g_spin_limit.store(iterations, std::memory_order_relaxed);
}

size_t svb_workspace_size(size_t n)
{
    return svb::ws_layout(n).total;
}

int svb_workspace_init(void *ws, size_t ws_bytes, svb_stream_t stream)
{
    if (!ws || ws_bytes < svb::kOffsetsOffset)
        return SVB_EINVAL;
    return cudaMemsetAsync(ws, 0, ws_bytes, reinterpret_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? SVB_OK
               : SVB_ECUDA;
}

int svb_encode_async(const uint32_t *in, size_t n, uint8_t *out, uint32_t prev, int delta,
                     svb_result *d_result, void *ws, size_t ws_bytes, svb_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!d_result)
        return SVB_EINVAL;
    if (n == 0)
        return cudaMemsetAsync(d_result, 0, sizeof(svb_result), s) == cudaSuccess ? SVB_OK
                                                                                 : SVB_ECUDA;
    if (!in || !out || !ws || ws_bytes < svb_workspace_size(n))
        return SVB_EINVAL;
    return encode_dispatch(in, n, out, prev, delta != 0, ws,
                           reinterpret_cast<svb::DeviceResult *>(d_result), s);
}

int svb_decode_async(const uint8_t *in, size_t in_len, size_t n, uint32_t *out,
                     uint32_t prev, int delta, svb_result *d_result, void *ws,
                     size_t ws_bytes, svb_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!d_result)
        return SVB_EINVAL;
    if (n == 0)
        return cudaMemsetAsync(d_result, 0, sizeof(svb_result), s) == cudaSuccess ? SVB_OK
                                                                                 : SVB_ECUDA;
    if (!in || !out || !ws || ws_bytes < svb_workspace_size(n))
        return SVB_EINVAL;
    if (in_len < ((u64)n + 3) / 4)
        return SVB_ETRUNCATED;
    return decode_dispatch(in, in_len, n, out, prev, delta != 0, ws,
                           reinterpret_cast<svb::DeviceResult *>(d_result), s);
}

int svb_gap_sum(const uint8_t *in, size_t in_len, size_t n, uint64_t *d_out, void *ws,
                size_t ws_bytes, svb_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!d_out)
        return SVB_EINVAL;
    if (n == 0)
        return cudaMemsetAsync(d_out, 0, 3 * sizeof(uint64_t), s) == cudaSuccess ? SVB_OK
                                                                               : SVB_ECUDA;
    if (!in || !ws || ws_bytes < svb_workspace_size(n))
        return SVB_EINVAL;
    if (in_len < ((u64)n + 3) / 4)
        return SVB_ETRUNCATED;
    return svb::launch_gap_sum(in, in_len, n, ws, reinterpret_cast<u64 *>(d_out), s,
                               spin_limit()) == 0
               ? SVB_OK
               : SVB_ECUDA;
}

int svb_decode_each(const svb_list *h_lists, size_t num_lists, const uint8_t *in_base,
                    uint32_t *out_base, int delta, svb_result *d_results, void *ws,
                    size_t ws_bytes, svb_stream_t stream)
{
    if (num_lists == 0)
        return SVB_OK;
    if (!h_lists || !in_base || !out_base || !d_results)
        return SVB_EINVAL;
    for (size_t j = 0; j < num_lists; j++) {
        const svb_list &l = h_lists[j];
        const int st = svb_decode_async(in_base + l.in_off, (size_t)l.in_len, l.n,
                                        out_base + l.out_off, l.prev, delta, d_results + j, ws,
                                        ws_bytes, stream);
        if (st != SVB_OK)
            return st;
    }
    return SVB_OK;
}

int svb_encode_each(const svb_list *h_lists, size_t num_lists, const uint32_t *in_base,
                    uint8_t *out_base, int delta, svb_result *d_results, void *ws,
                    size_t ws_bytes, svb_stream_t stream)
{
    if (num_lists == 0)
        return SVB_OK;
    if (!h_lists || !in_base || !out_base || !d_results)
        return SVB_EINVAL;
    for (size_t j = 0; j < num_lists; j++) {
        const svb_list &l = h_lists[j];
        const int st = svb_encode_async(in_base + l.in_off, l.n, out_base + l.out_off, l.prev,
                                        delta, d_results + j, ws, ws_bytes, stream);
        if (st != SVB_OK)
            return st;
    }
    return SVB_OK;
}

size_t svb_batch_plan_bytes(size_t num_lists)
{
    return svb::batch_plan_bytes(num_lists);
}

int svb_batch_plan_segments(const svb_list *h_lists, size_t num_lists, uint32_t big_threshold,
                            uint32_t segment_tiles, void *d_plan, size_t plan_bytes,
                            svb_stream_t stream)
{
    if ((!h_lists && num_lists) || !d_plan || plan_bytes < svb::batch_plan_bytes(num_lists) ||
        num_lists > 0xffffffffull || segment_tiles > 32 || ((uintptr_t)d_plan & 15u))
        return SVB_EINVAL;
    const int st = svb::build_batch_plan(h_lists, num_lists, big_threshold, segment_tiles, d_plan,
                                         reinterpret_cast<cudaStream_t>(stream));
    return st == 1 ? SVB_EINVAL : st;
}

int svb_batch_plan(const svb_list *h_lists, size_t num_lists, uint32_t big_threshold,
                   void *d_plan, size_t plan_bytes, svb_stream_t stream)
{
    return svb_batch_plan_segments(h_lists, num_lists, big_threshold,
                                   svb::batch_default_seg_tiles(), d_plan, plan_bytes, stream);
}

size_t svb_batch_workspace_size(void)
{
    return svb::kOffsetsOffset;
}

int svb_batch_set_stages(int decode_stages, int encode_stages)
{
    return svb::batch_set_stages(decode_stages, encode_stages) == 0 ? SVB_OK : SVB_EINVAL;
}

int svb_batch_get_stages(int encode)
{
    return svb::batch_stages(encode != 0);
}

int svb_batch_set_tile(int tile_ints)
{
    return svb::batch_set_tile(tile_ints) == 0 ? SVB_OK : SVB_EINVAL;
}

int svb_batch_get_tile(void)
{
    return svb::batch_tile();
}

int svb_batch_decode(const void *d_plan, const svb_list *d_lists, const uint8_t *in_base,
                     uint32_t *out_base, int delta, svb_result *d_result, void *ws,
                     size_t ws_bytes, int grid, svb_stream_t stream)
{
    if (!d_plan || !d_lists || !in_base || !out_base || !d_result || !ws ||
        ws_bytes < svb::kOffsetsOffset || grid < 0)
        return SVB_EINVAL;
    return svb::launch_batch_decode(d_plan, d_lists, in_base, out_base, delta != 0, ws,
                                    reinterpret_cast<svb::DeviceResult *>(d_result),
                                    reinterpret_cast<cudaStream_t>(stream), grid);
}

int svb_batch_encode(const void *d_plan, const svb_list *d_lists, const uint32_t *in_base,
                     uint8_t *out_base, int delta, uint64_t *d_sizes, svb_result *d_result,
                     void *ws, size_t ws_bytes, int grid, svb_stream_t stream)
{
    if (!d_plan || !d_lists || !in_base || !out_base || !d_sizes || !d_result || !ws ||
        ws_bytes < svb::kOffsetsOffset || grid < 0)
        return SVB_EINVAL;
    return svb::launch_batch_encode(d_plan, d_lists, in_base, out_base,
                                    reinterpret_cast<u64 *>(d_sizes), delta != 0, ws,
                                    reinterpret_cast<svb::DeviceResult *>(d_result),
                                    reinterpret_cast<cudaStream_t>(stream), grid);
}

int svb_testhook_lookback_timeout(const uint8_t *stream_in, size_t n, uint32_t *out,
                                  uint64_t spin_limit_, svb_result *d_result, void *ws,
                                  size_t ws_bytes, svb_stream_t stream)
{
    if (!stream_in || !out || !d_result || !ws || ws_bytes < svb_workspace_size(n))
        return SVB_EINVAL;
    if (svb::decode_tiles(n) < 2)
        return SVB_EINVAL;
    // One CTA that takes tile 1; tile 0 is never launched, so its status is
    // never published in this launch and the wait must run out.
    return svb::launch_decode(stream_in, ~0ull, n, out, 0, false, ws,
                              reinterpret_cast<svb::DeviceResult *>(d_result),
                              reinterpret_cast<cudaStream_t>(stream), spin_limit_, 1, 1);
}

int svb_testhook_offsets_timeout(const uint8_t *stream_in, size_t n, uint32_t *out,
                                 uint64_t spin_limit_, svb_result *d_result, void *ws,
                                 size_t ws_bytes, svb_stream_t stream)
{
    if (!stream_in || !out || !d_result || !ws || ws_bytes < svb_workspace_size(n))
        return SVB_EINVAL;
    if (n <= 64 * (u64)svb::kThreads * 4)  // at least two ranges of the offsets pass
        return SVB_EINVAL;
    return svb::launch_offsets_timeout_check(stream_in, n, out, ws,
                                             reinterpret_cast<svb::DeviceResult *>(d_result),
                                             reinterpret_cast<cudaStream_t>(stream),
                                             spin_limit_);
}

}  // extern "C"
