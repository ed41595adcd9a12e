// runtime.h -- host-side context of libdqj (internal).
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dqj.h"
#include "dqj_internal.h"

namespace dqj {

// Thread-local error message behind dqj_last_error().
dqj_status fail(dqj_status st, const std::string &msg);
dqj_status cuda_fail(cudaError_t e, const char *what);
// Status for the exception in flight (call only inside a catch block): a host
// allocation failure or a thread that could not start gives DQJ_ERR_NOMEM,
// anything else DQJ_ERR_INVALID, each with its message.
dqj_status exception_status() noexcept;
// Runs an entry point's body so that no C++ exception crosses the C ABI.
template <typename F>
dqj_status guarded(F &&body) noexcept
{
    try {
        return body();
    } catch (...) {
        return exception_status();
    }
}

// Validation and derivation of the per-frame constants (host, double).
dqj_status validate(const dqj_params *p);
// Output planes: pitch >= width, every non-NULL plane 4-byte aligned.
dqj_status check_outputs(const dqj_params &p, const dqj_outputs *out);
void derive_frame(const dqj_params &p, FrameDesc &fd, int tile_w, int tile_h);
// Exact thresholds of the axis-slice first step's tests (see PairConsts).
void axis_first_thresholds(const FrameT<float> &F, int modulus_mode, PairConsts &P);

// Scratch block sized for a pixel count; grow-only.
struct ScratchBuf {
    void *base = nullptr;
    size_t bytes = 0;
    uint32_t pixels = 0;
    bool with_queue = false;
    uint64_t part_entries = 0;  // split-march partial results
    Scratch view{};
    uint32_t epoch = 0;
};
dqj_status scratch_ensure(ScratchBuf &s, uint64_t pixels, bool need_queue, uint64_t part_entries = 0);
void scratch_free(ScratchBuf &s);

struct ServeState;  // serving loop, serve.cpp

dqj_status serve_start(dqj_ctx *ctx);

}  // namespace dqj

struct dqj_ctx {
    int device = 0;
    int num_sms = 0;
    dqj_config cfg{};
    std::string cache_path;
    std::mutex mu;                   // orders renders on this context
    dqj::ScratchBuf scratch;
    cudaEvent_t done_ev = nullptr;   // last render's completion on its stream
    unsigned long long done_capture = 0;  // stream-capture id done_ev was last recorded under (0: none)
    // dqj_render_host planes
    // dqj_render_host / dqj_render_host_batch: two device plane sets, so that
    // one frame's copy back overlaps the next frame's render
    cudaStream_t host_stream = nullptr;       // renders
    cudaStream_t host_copy_stream = nullptr;  // device -> host copies
    void *host_planes[2] = {nullptr, nullptr};
    size_t host_planes_bytes[2] = {0, 0};
    cudaEvent_t host_rendered[2] = {nullptr, nullptr}, host_copied[2] = {nullptr, nullptr};
    // tile shapes chosen by the autotuner, keyed by (pixel-count class, iter bucket)
    std::map<int, std::pair<int, int>> tiles;
    std::mutex tiles_mu;             // guards tiles (read by the serving thread too)
    dqj::ServeState *serve = nullptr;
    std::atomic<int> serve_policy{DQJ_SERVE_FIFO};  // order of packed requests in the persistent launch
    // frame pipelines (dqj_render_batch, dqj_render_host_batch): a second
    // scratch set and two lane streams, so that a frame's bisection and FP64
    // passes run beside the next frame's march
    dqj::ScratchBuf scratch2;
    cudaStream_t lane_stream[2] = {nullptr, nullptr};
    cudaEvent_t lane_ev[2][5] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[2] = {nullptr, nullptr};
    // dqj_voxelize scratch: counter block + FP64 recheck queue; grow-only
    void *vox_scratch = nullptr;
    size_t vox_bytes = 0;
    // profiling ring: ring_frames x 5 events, next slot, renders recorded
    std::vector<cudaEvent_t> ev;
    int ring_frames = 0;
    uint64_t ring_next = 0;
};

namespace dqj {
// March kernel variant and tile shape for a frame (autotuned choice or default).
void pick_tile_shape(dqj_ctx *ctx, const dqj_params &p, int &variant, int &tw, int &th);
// The default choice without a context: the paired kernel on 8 x 8 tiles (FP32)
// or one ray per lane on 8 x 4 (FP64), DQJ_MARCH_VARIANT (0 or 1) overriding
// the FP32 kernel.
void default_tile_shape(const dqj_params &p, int &variant, int &tw, int &th);
// Autotuner cache (autotune.cpp): key of a (variant, size class, iteration bucket)
// and loading of the cache file named by the context or DQJ_AUTOTUNE_CACHE.
int tile_key(int variant, int size_class, int bucket);
void load_tile_cache(dqj_ctx *ctx);
}  // namespace dqj
