// noalloc.cu -- dqj_render_noalloc: the plain render (march + bisection passes)
// with its scratch in a fixed, file-scope device array instead of memory the
// library allocates.  For callers that must not allocate device memory: a host
// application that reserves all device memory for its own pool before loading
// this library, or a frame loop that must not block on the allocator.
//
// The array is DQJ_NOALLOC_MAX_PIXELS hit-list entries (16 B each) plus a
// 256-byte counter block, about 4 MiB.  Its device address is looked up once
// per device with cudaGetSymbolAddress, on the first call made while that
// device is current.  Under lazy module loading (the CUDA default) that first
// call is also when the array is placed on the device, so make it before the
// caller reserves the device's memory for its own pool and before any stream
// capture; from then on the device holds the array until the process exits.
// The address is kept for the life of the process: a cudaDeviceReset after the
// first call is not supported.  All calls share the array: the counter block
// is cleared at the start of every call, and calls that overlap on the GPU
// (other streams or threads) race on it.  The march kernel and tile shape are
// dqj_render's defaults (default_tile_shape, DQJ_MARCH_VARIANT included).
#include <mutex>

#include "runtime.h"

namespace {

constexpr size_t kCounterBytes = 256;
constexpr size_t kHitBytes = (size_t)DQJ_NOALLOC_MAX_PIXELS * sizeof(int4);
static_assert(sizeof(dqj::Counters) <= kCounterBytes, "counter block");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterBytes + kHitBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_num_sms[kMaxDevices];

dqj_status check_planes(const dqj_params &p, const dqj_outputs *out)
{
    if (!out) return dqj::fail(DQJ_ERR_INVALID, "outputs is NULL");
    if (out->pitch_px < p.width) return dqj::fail(DQJ_ERR_INVALID, "pitch_px must be >= width");
    const void *planes[4] = {out->iter, out->depth, out->normal, out->rgba};
    for (const void *q : planes)
        if (q && (reinterpret_cast<uintptr_t>(q) & 3u))
            return dqj::fail(DQJ_ERR_INVALID, "output planes must be 4-byte aligned");
    return DQJ_OK;
}

}  // namespace

extern "C" dqj_status dqj_render_noalloc(const dqj_params *p, const dqj_outputs *out, void *cuda_stream)
{
    return dqj::guarded([&]() -> dqj_status {
        dqj_status s = dqj::validate(p);
        if (s != DQJ_OK) return s;
        const uint64_t pixels = (uint64_t)p->width * (uint64_t)p->height;
        if (pixels > DQJ_NOALLOC_MAX_PIXELS)
            return dqj::fail(DQJ_ERR_INVALID, "dqj_render_noalloc: width * height exceeds DQJ_NOALLOC_MAX_PIXELS (" +
                                                  std::to_string(DQJ_NOALLOC_MAX_PIXELS) + ")");
        if (p->precision == DQJ_FP32_RECHECK)
            return dqj::fail(DQJ_ERR_INVALID, "dqj_render_noalloc supports DQJ_FP32 and DQJ_FP64 only");
        s = check_planes(*p, out);
        if (s != DQJ_OK) return s;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return dqj::cuda_fail(e, "render_noalloc: cudaGetDevice");
        if (dev < 0 || dev >= kMaxDevices) return dqj::fail(DQJ_ERR_INVALID, "render_noalloc: device ordinal too large");
        void *base = nullptr;
        int sms = 0;
        {
            std::lock_guard<std::mutex> lk(g_setup_mu);
            if (!g_scratch_addr[dev]) {
                void *addr = nullptr;
                e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
                if (e != cudaSuccess) return dqj::cuda_fail(e, "render_noalloc: cudaGetSymbolAddress");
                int n = 0;
                e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
                if (e != cudaSuccess) return dqj::cuda_fail(e, "render_noalloc: cudaDeviceGetAttribute");
                g_num_sms[dev] = n;
                g_scratch_addr[dev] = addr;
            }
            base = g_scratch_addr[dev];
            sms = g_num_sms[dev];
        }
        dqj::Scratch sc{};
        sc.ctr = static_cast<dqj::Counters *>(base);
        sc.hits = reinterpret_cast<int4 *>(static_cast<unsigned char *>(base) + kCounterBytes);
        sc.hit_cap = DQJ_NOALLOC_MAX_PIXELS;

        int variant, tw, th;
        dqj::default_tile_shape(*p, variant, tw, th);
        dqj::FrameDesc fd;
        dqj::derive_frame(*p, fd, tw, th);
        fd.march_variant = variant;
        fd.pitch = out->pitch_px;
        fd.iter = out->iter;
        fd.depth = out->depth;
        fd.normal = out->normal;
        fd.rgba = out->rgba;
        fd.epoch = 1;

        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        // launch errors are read back with cudaGetLastError: start from a clean
        // slate, so an earlier failed call of the caller's is not taken for ours
        (void)cudaGetLastError();
        e = cudaMemsetAsync(sc.ctr, 0, kCounterBytes, st);
        if (e != cudaSuccess) return dqj::cuda_fail(e, "render_noalloc: clear counters");
        e = dqj::launch_frame(fd, sc, st, sms);
        if (e != cudaSuccess) return dqj::cuda_fail(e, "render_noalloc: kernel launch");
        if (out->stats) {
            e = cudaMemcpyAsync(out->stats, sc.ctr->stats, DQJ_NSTATS * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return dqj::cuda_fail(e, "render_noalloc: stats copy");
        }
        return DQJ_OK;
    });
}
