// autotune.cpp -- tile-shape autotuner and its cache.
//
// The march kernels give each warp a screen tile of 32 rays (one per lane) or
// 64 rays (two per lane).  The tile's shape trades how alike neighbouring rays'
// escape counts are (lockstep waste) against tail effects, and the best shape
// depends on the frame size and iteration limit.  dqj_autotune renders a probe
// frame for every (frame-size class, iteration bucket) with every candidate
// shape, keeps the fastest (CUDA-event time, best of three), stores the choice in
// the context and writes it to the cache file.  dqj_create reads the cache when
// it matches the device (name and SM count).
//
// Cache format (JSON): {"device": "<name>", "sms": <n>, "entries":
// [[variant, size_class, iter_bucket, tile_w, tile_h], ...]}
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <vector>

#include "runtime.h"

namespace dqj {

dqj_status render_on_stream(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, cudaStream_t st);

int tile_key(int variant, int size_class, int bucket) { return (variant * 4 + size_class) * 4 + bucket; }

static std::string device_name(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    return prop.name;
}

std::string cache_path_of(const dqj_ctx *ctx)
{
    if (!ctx->cache_path.empty()) return ctx->cache_path;
    if (const char *e = std::getenv("DQJ_AUTOTUNE_CACHE")) return e;
    return "";
}

void load_tile_cache(dqj_ctx *ctx)
{
    const std::string path = cache_path_of(ctx);
    if (path.empty()) return;
    std::ifstream f(path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string text = ss.str();
    const size_t dp = text.find("\"device\"");
    const size_t sp = text.find("\"sms\"");
    const size_t ep = text.find("\"entries\"");
    if (dp == std::string::npos || sp == std::string::npos || ep == std::string::npos) return;
    const size_t q1 = text.find('"', text.find(':', dp) + 1), q2 = text.find('"', q1 + 1);
    if (q1 == std::string::npos || q2 == std::string::npos) return;
    if (text.substr(q1 + 1, q2 - q1 - 1) != device_name(ctx->device)) return;
    if (std::atoi(text.c_str() + text.find(':', sp) + 1) != ctx->num_sms) return;
    const char *c = text.c_str() + text.find('[', ep) + 1;
    int v, sc, b, tw, th, n = 0;
    while ((c = std::strchr(c, '[')) != nullptr) {
        if (std::sscanf(c, "[%d,%d,%d,%d,%d]", &v, &sc, &b, &tw, &th) == 5 ||
            std::sscanf(c, "[%d, %d, %d, %d, %d]", &v, &sc, &b, &tw, &th) == 5) {
            if (v >= 0 && v <= 1 && sc >= 0 && sc < 4 && b >= 0 && b < 4 && tw >= 1 && th >= 1 &&
                tw * th == (v == 1 ? 64 : 32))
                ctx->tiles[tile_key(v, sc, b)] = {tw, th};
            ++n;
        }
        ++c;
    }
}

static dqj_status write_tile_cache(dqj_ctx *ctx)
{
    const std::string path = cache_path_of(ctx);
    if (path.empty()) return DQJ_OK;
    std::ofstream f(path);
    if (!f) return fail(DQJ_ERR_INVALID, "autotune: cannot write cache file " + path);
    f << "{\"device\": \"" << device_name(ctx->device) << "\", \"sms\": " << ctx->num_sms << ", \"entries\": [";
    bool first = true;
    std::lock_guard<std::mutex> lk(ctx->tiles_mu);
    for (const auto &kv : ctx->tiles) {
        const int key = kv.first;
        const int b = key % 4, sc = (key / 4) % 4, v = key / 16;
        f << (first ? "" : ", ") << "[" << v << ", " << sc << ", " << b << ", " << kv.second.first << ", "
          << kv.second.second << "]";
        first = false;
    }
    f << "]}\n";
    return f ? DQJ_OK : fail(DQJ_ERR_INVALID, "autotune: write failed");
}

}  // namespace dqj

using namespace dqj;

extern "C" {

dqj_status dqj_autotune(dqj_ctx *ctx, int32_t max_classes)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        if (ctx->device == DQJ_DEVICE_MOCK) return fail(DQJ_ERR_INVALID, "a mock context cannot autotune");
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(e, "autotune: cudaSetDevice");
        static const int sizes[4][2] = {{256, 256}, {512, 512}, {1024, 1024}, {1920, 1080}};
        static const int iters[4] = {10, 16, 24, 32};
        static const int shapes1[][2] = {{8, 8}, {16, 4}, {4, 16}, {32, 2}, {64, 1}};
        const int nclass = max_classes > 0 && max_classes < 4 ? max_classes : 4;
        void *planes = nullptr;
        const size_t px_max = (size_t)sizes[nclass - 1][0] * sizes[nclass - 1][1];
        e = cudaMalloc(&planes, px_max * 24);
        if (e != cudaSuccess) return cuda_fail(e, "autotune: planes");
        cudaStream_t st = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        dqj_status result = e == cudaSuccess ? DQJ_OK : cuda_fail(e, "autotune: stream/events");
        for (int sc = 0; sc < nclass && result == DQJ_OK; ++sc) {
            for (int bk = 0; bk < 4 && result == DQJ_OK; ++bk) {
                dqj_params p;
                dqj_default_params(&p);
                p.width = sizes[sc][0];
                p.height = sizes[sc][1];
                p.max_iter = iters[bk];
                p.march_steps = 512;
                p.bisect_steps = 10;
                dqj_outputs out{};
                char *pb = static_cast<char *>(planes);
                const size_t px = (size_t)p.width * p.height;
                out.pitch_px = p.width;
                out.iter = reinterpret_cast<int32_t *>(pb);
                out.depth = reinterpret_cast<float *>(pb + px * 4);
                out.normal = reinterpret_cast<float *>(pb + px * 8);
                out.rgba = reinterpret_cast<uint8_t *>(pb + px * 20);
                float best = 1e30f;
                std::pair<int, int> best_shape{8, 8};
                for (const auto &sh : shapes1) {
                    {
                        std::lock_guard<std::mutex> lk(ctx->tiles_mu);
                        ctx->tiles[tile_key(1, sc, bk)] = {sh[0], sh[1]};
                    }
                    float t = 1e30f;
                    for (int rep = 0; rep < 3 && result == DQJ_OK; ++rep) {
                        cudaEventRecord(a, st);
                        result = render_on_stream(ctx, &p, &out, st);
                        cudaEventRecord(b, st);
                        e = cudaEventSynchronize(b);
                        float ms = 0.f;
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                        if (e != cudaSuccess && result == DQJ_OK) result = cuda_fail(e, "autotune: timing");
                        if (rep > 0 && ms < t) t = ms;  // first repetition warms up
                    }
                    if (t < best) {
                        best = t;
                        best_shape = {sh[0], sh[1]};
                    }
                }
                std::lock_guard<std::mutex> lk(ctx->tiles_mu);
                ctx->tiles[tile_key(1, sc, bk)] = best_shape;
            }
        }
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (st) cudaStreamDestroy(st);
        cudaFree(planes);
        if (result != DQJ_OK) return result;
        return write_tile_cache(ctx);
    });
}

dqj_status dqj_tile_shape(dqj_ctx *ctx, const dqj_params *p, int32_t *variant, int32_t *tile_w, int32_t *tile_h)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx || !p || !variant || !tile_w || !tile_h) return fail(DQJ_ERR_INVALID, "NULL argument");
        dqj_status s = validate(p);
        if (s != DQJ_OK) return s;
        int v, tw, th;
        pick_tile_shape(ctx, *p, v, tw, th);
        *variant = v;
        *tile_w = tw;
        *tile_h = th;
        return DQJ_OK;
    });
}

}  // extern "C"
