// serve.cpp -- serving entry points of libdqj: dqj_submit / dqj_poll /
// dqj_destroy and the scheduler thread behind them (continuous batching).
//
// A request is queued on the host at dqj_submit.  The scheduler thread admits
// queued requests in the order of the serving policy (arrival, or earliest
// estimated finish) while the sum of the admitted requests' footprints (output
// planes + scratch + slot) fits the context's memory budget and a device slot
// is free.  dqj_poll reads ticket states under a lock of their own, never the
// scheduler's.  Admitted FP32 / algebraic / EUCLID8 requests are
// written into device slots and run together in one persistent launch
// (serve.cu); requests arriving while it runs join it.  FP32 + FP64 recheck
// requests run in it too, with their recheck and re-render phases.  Other
// precisions and modes run as ordinary stream-ordered frames on the serving
// stream.  Completed
// requests release their budget, and dqj_poll hands back their status once.
//
// The scheduler talks to the device through a small backend interface.  The
// GPU backend is the real one; contexts created with device = DQJ_DEVICE_MOCK
// use a CPU-only mock whose completion delay, allocation failure or
// never-completing behaviour is set from the environment, so the admission,
// budget, BUSY, TIMEOUT and CANCELLED paths are testable without a GPU.
#include <algorithm>
#include <chrono>
#include <deque>
#include <unordered_map>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "runtime.h"
#include "serve_internal.h"

namespace dqj {

dqj_status render_on_stream(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, cudaStream_t st);

namespace {

using clk = std::chrono::steady_clock;

int64_t env_int(const char *name, int64_t dflt)
{
    const char *e = std::getenv(name);
    return e ? std::strtoll(e, nullptr, 10) : dflt;
}

struct Request {
    dqj_ticket ticket = 0;
    dqj_params p{};
    dqj_outputs out{};
    uint64_t footprint = 0;
    bool packed = false;     // runs in the persistent launch
    int slot = -1;
    unsigned block = ~0u;    // control block of a packed request
    uint64_t seq = 0;
    uint64_t prio = 0;       // the persistent launch serves the smallest key first
    clk::time_point submitted{};
    // device resources
    void *scratch = nullptr;
    cudaEvent_t done_ev = nullptr;
    clk::time_point admitted{};
};

bool packable(const dqj_params &p)
{
    return (p.precision == DQJ_FP32 || p.precision == DQJ_FP32_RECHECK) && p.square_mode == DQJ_SQUARE_ALGEBRAIC &&
           p.modulus_mode == DQJ_MODULUS_EUCLID8 && p.traversal == DQJ_TRAVERSAL_MARCH;
}

// Recheck scratch per pixel: queue (4 entries), per-pixel tag, re-render list.
constexpr uint64_t kRecheckBytesPerPixel = 4 * sizeof(int4) + 8;

uint64_t scratch_bytes(const dqj_params &p, bool packed)
{
    const uint64_t px = (uint64_t)p.width * (uint64_t)p.height;
    uint64_t b = 256 + px * sizeof(int4);                                  // counters + hit list
    if (p.precision == DQJ_FP32_RECHECK) b += px * kRecheckBytesPerPixel;   // queue, tags, list
    (void)packed;
    return b;
}

// Per-request bookkeeping counted against the budget (control block and slot).
constexpr uint64_t kRequestOverhead = 2048;
static_assert(sizeof(ReqBlock) + sizeof(ServeSlot) <= kRequestOverhead, "request overhead");

uint64_t footprint(const dqj_params &p, bool packed)
{
    const uint64_t px = (uint64_t)p.width * (uint64_t)p.height;
    return px * 24 + scratch_bytes(p, packed) + kRequestOverhead;
}

// -------------------------------------------------------------------------
// backends
// -------------------------------------------------------------------------
struct Backend {
    virtual ~Backend() = default;
    // Start running a batch of requests (slots already chosen for packed ones);
    // writes each request's status into st[i].
    virtual void admit(Request *const *rs, int n, dqj_status *st) = 0;
    virtual int poll(Request &r) = 0;             // 1 done, 0 running, -1 failed (message set)
    virtual dqj_status kick(bool packed_active) = 0;
    virtual void hold(bool on) = 0;               // the host has queued or running work
    virtual void release(Request &r) = 0;
    virtual dqj_status shutdown(int64_t timeout_ms) = 0;
    virtual void launch_counts(int64_t &launches, int64_t &restarts) const
    {
        launches = 0;
        restarts = 0;
    }
    // Requests in the persistent launch whose device execution (first item
    // claimed to completion) overlapped another request's.
    virtual int64_t overlapped() const { return 0; }
};

class GpuBackend : public Backend {
  public:
    explicit GpuBackend(dqj_ctx *ctx) : ctx_(ctx) {}
    ~GpuBackend() override { free_all(); }

    dqj_status init()
    {
        cudaError_t e = cudaSetDevice(ctx_->device);
        if (e == cudaSuccess) e = cudaMalloc(&d_slots_, sizeof(ServeSlot) * kMaxSlots);
        if (e == cudaSuccess) e = cudaMalloc(&d_blocks_, sizeof(ReqBlock) * kReqBlocks);
        if (e == cudaSuccess) e = cudaMalloc(&d_exit_, 256);
        if (e == cudaSuccess) e = cudaMemset(d_blocks_, 0, sizeof(ReqBlock) * kReqBlocks);
        if (e == cudaSuccess) e = cudaHostAlloc(&h_flags_, sizeof(unsigned) * (kMaxSlots + 2), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(h_flags_, 0, sizeof(unsigned) * (kMaxSlots + 2));
            h_flags_[kMaxSlots] = 1;  // source of the host's exit request
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_flags_), h_flags_, 0);
        }
        if (e == cudaSuccess) e = cudaHostAlloc(&h_times_, sizeof(unsigned long long) * 2 * kMaxSlots, cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(h_times_, 0, sizeof(unsigned long long) * 2 * kMaxSlots);
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_times_), h_times_, 0);
        }
        if (e == cudaSuccess) e = cudaHostAlloc(&h_slots_, sizeof(ServeSlot) * kMaxSlots, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&h_blocks_, sizeof(ReqBlock) * kReqBlocks, cudaHostAllocDefault);
        if (e == cudaSuccess) {
            std::memset(h_slots_, 0, sizeof(ServeSlot) * kMaxSlots);
            for (int s = 0; s < kMaxSlots; ++s) h_slots_[s].block = ~0u;  // no block
            e = cudaMemcpy(d_slots_, h_slots_, sizeof(ServeSlot) * kMaxSlots, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&kstream_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cstream_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pstream_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&kevent_, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "serve: init");
        for (unsigned b = 0; b < (unsigned)kReqBlocks; ++b) free_blocks_.push_back({b, 0});
        for (int s = 0; s < kMaxSlots; ++s) slot_block_[s] = ~0u;
        idle_ns_ = (unsigned long long)env_int("DQJ_SERVE_IDLE_US", 2000) * 1000ull;
        return DQJ_OK;
    }

    // Packed requests: write their control blocks, wait for the copies, then
    // publish the slots.  Plain requests: enqueue an ordinary frame.
    void admit(Request *const *rs, int n, dqj_status *status) override
    {
        cudaError_t e = cudaSetDevice(ctx_->device);
        for (int i = 0; i < n; ++i) status[i] = e == cudaSuccess ? DQJ_OK : cuda_fail(e, "serve: cudaSetDevice");
        if (e != cudaSuccess) return;
        std::vector<unsigned> staged;  // blocks whose bodies were staged, in request order
        bool packed_any = false;
        for (int i = 0; i < n; ++i) {
            Request &r = *rs[i];
            status[i] = r.packed ? stage_packed(r) : launch_plain(r);
            if (r.packed && status[i] == DQJ_OK) {
                staged.push_back(r.block);
                packed_any = true;
            }
        }
        if (!packed_any) return;
        // bodies: one copy per run of consecutive block indices
        std::sort(staged.begin(), staged.end());
        for (size_t i = 0; i < staged.size() && e == cudaSuccess;) {
            size_t j = i + 1;
            while (j < staged.size() && staged[j] == staged[j - 1] + 1) ++j;
            e = cudaMemcpyAsync(d_blocks_ + staged[i], h_blocks_ + staged[i], sizeof(ReqBlock) * (j - i),
                                cudaMemcpyHostToDevice, cstream_);
            i = j;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(cstream_);  // bodies visible before any slot names them
        if (e == cudaSuccess) {
            for (int i = 0; i < n; ++i) {
                Request &r = *rs[i];
                if (!r.packed || status[i] != DQJ_OK) continue;
                retire_block(slot_block_[r.slot]);  // the slot's previous request's block
                slot_block_[r.slot] = r.block;
                h_slots_[r.slot].block = r.block;
                h_slots_[r.slot].prio = r.prio;
                h_slots_[r.slot].seq = r.seq;
            }
            // the host holds the only copy that changes: rewrite the whole table
            e = cudaMemcpyAsync(d_slots_, h_slots_, sizeof(ServeSlot) * kMaxSlots, cudaMemcpyHostToDevice, cstream_);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(cstream_);
        if (e != cudaSuccess) {
            const dqj_status f = cuda_fail(e, "serve: publish requests");
            for (int i = 0; i < n; ++i) {
                Request &r = *rs[i];
                if (!r.packed) continue;
                if (status[i] == DQJ_OK && slot_block_[r.slot] != r.block) retire_block(r.block);  // never published
                status[i] = f;
            }
        }
    }

    void hold(bool on) override
    {
        if (h_flags_) *reinterpret_cast<volatile unsigned *>(&h_flags_[kMaxSlots + 1]) = on ? 1u : 0u;
    }

  private:
    FrameDesc frame_of(Request &r)
    {
        int variant, tw, th;
        pick_tile_shape(ctx_, r.p, variant, tw, th);
        FrameDesc fd;
        derive_frame(r.p, fd, tw, th);
        fd.march_variant = variant;
        fd.pitch = r.out.pitch_px;
        fd.iter = r.out.iter;
        fd.depth = r.out.depth;
        fd.normal = r.out.normal;
        fd.rgba = r.out.rgba;
        fd.stats = r.out.stats;
        fd.epoch = 1;
        return fd;
    }

    // Launch ids: a block retired while launch L (the last one started) may run
    // is reusable once launch L has exited.
    void update_completed()
    {
        if (launched_ && completed_ < launches_ && cudaEventQuery(kevent_) == cudaSuccess) completed_ = launches_;
    }

    void retire_block(unsigned b)
    {
        if (b < (unsigned)kReqBlocks) free_blocks_.push_back({b, launches_});
    }

    // A control block that no launch can still be reading.  When every free block
    // may still be seen by the running launch, stop it (claimed items finish; the
    // next launch continues from the claim counters) and wait for it to exit.
    dqj_status take_block(unsigned &b)
    {
        update_completed();
        if (free_blocks_.empty()) return fail(DQJ_ERR_NOMEM, "serve: control-block pool exhausted");
        if (free_blocks_.front().second > completed_) {
            const dqj_status s = stop_launch(10000);
            if (s != DQJ_OK) return s;
            ++restarts_;
        }
        b = free_blocks_.front().first;
        free_blocks_.pop_front();
        return DQJ_OK;
    }

    // Raise the launch's exit flag with a copy-engine write (no SM needed while
    // the persistent grid occupies them) and wait, bounded, for the launch to end.
    dqj_status stop_launch(int64_t timeout_ms)
    {
        if (!launched_ || completed_ == launches_) return DQJ_OK;
        cudaError_t e = cudaMemcpyAsync(d_exit_, &h_flags_[kMaxSlots], sizeof(unsigned), cudaMemcpyHostToDevice,
                                        cstream_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cstream_);
        if (e != cudaSuccess) return cuda_fail(e, "serve: exit request");
        const auto t0 = clk::now();
        for (;;) {
            const cudaError_t q = cudaEventQuery(kevent_);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return cuda_fail(q, "serve: persistent kernel");
            if (clk::now() - t0 > std::chrono::milliseconds(timeout_ms))
                return fail(DQJ_ERR_TIMEOUT, "serve: persistent kernel did not stop in time");
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        completed_ = launches_;
        return DQJ_OK;
    }

    // Stage a packed request's control block in host memory.  Each slot owns a
    // grow-only scratch buffer laid out by its pixel capacity: the hit list,
    // then (recheck mode) the recheck queue, the per-pixel tags and the
    // re-render list.  The tags of a new buffer start at zero and those of
    // later requests in the slot are told apart by their generation (the
    // frame's epoch).  The zeros come by a copy-engine copy from page-locked
    // host memory: a memset may run as a kernel, which could not start while
    // the persistent grid holds every SM.
    dqj_status stage_packed(Request &r)
    {
        const uint64_t px = (uint64_t)r.p.width * (uint64_t)r.p.height;
        const bool rq = r.p.precision == DQJ_FP32_RECHECK;
        cudaError_t e = cudaSuccess;
        if (slot_px_[r.slot] < px || (rq && !slot_rq_[r.slot])) {
            const uint64_t cap = std::max<uint64_t>(px, slot_px_[r.slot]);
            const bool with_rq = rq || slot_rq_[r.slot];
            if (slot_scratch_[r.slot]) e = cudaFreeAsync(slot_scratch_[r.slot], cstream_);
            slot_scratch_[r.slot] = nullptr;
            slot_px_[r.slot] = 0;
            slot_rq_[r.slot] = false;
            const size_t bytes = cap * (sizeof(int4) + (with_rq ? kRecheckBytesPerPixel : 0));
            if (e == cudaSuccess) e = cudaMallocAsync(&slot_scratch_[r.slot], bytes, cstream_);
            if (e == cudaSuccess && with_rq) {
                const size_t tag_bytes = cap * sizeof(uint32_t);
                if (zeros_bytes_ < tag_bytes) {  // grow-only zero source; the stream is idle here
                    e = cudaStreamSynchronize(cstream_);
                    if (e == cudaSuccess && zeros_) e = cudaFreeHost(zeros_);
                    zeros_ = nullptr;
                    zeros_bytes_ = 0;
                    if (e == cudaSuccess) e = cudaHostAlloc(&zeros_, tag_bytes, cudaHostAllocDefault);
                    if (e == cudaSuccess) {
                        std::memset(zeros_, 0, tag_bytes);
                        zeros_bytes_ = tag_bytes;
                    }
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(static_cast<char *>(slot_scratch_[r.slot]) + cap * 5 * sizeof(int4), zeros_,
                                        tag_bytes, cudaMemcpyHostToDevice, cstream_);
            }
            if (e != cudaSuccess) return cuda_fail(e, "serve: slot scratch");
            slot_px_[r.slot] = cap;
            slot_rq_[r.slot] = with_rq;
        }
        unsigned bi = 0;
        dqj_status s = take_block(bi);
        if (s != DQJ_OK) return s;
        r.block = bi;
        ReqBlock &h = h_blocks_[bi];
        std::memset(&h, 0, sizeof h);
        h.phase = kPhaseMarch;
        h.fd = frame_of(r);
        h.fd.epoch = (uint32_t)r.seq;  // non-zero, unique per admission
        h.ntiles = (unsigned)h.fd.tiles_x * (unsigned)h.fd.tiles_y;
        h.slot = (unsigned)r.slot;
        h.gen = (unsigned)r.seq;
        h.recheck = rq ? 1u : 0u;
        char *base = static_cast<char *>(slot_scratch_[r.slot]);
        const uint64_t cap = slot_px_[r.slot];
        h.sc.ctr = &d_blocks_[bi].ctr;
        h.sc.hits = reinterpret_cast<int4 *>(base);
        h.sc.hit_cap = (uint32_t)px;
        if (rq) {
            h.sc.queue = reinterpret_cast<int4 *>(base + cap * sizeof(int4));
            h.sc.queue_cap = (uint32_t)(4 * cap);
            h.sc.dirty_flag = reinterpret_cast<uint32_t *>(base + cap * 5 * sizeof(int4));
            h.sc.dirty_list = reinterpret_cast<int32_t *>(base + cap * (5 * sizeof(int4) + 4));
            h.sc.dirty_cap = (uint32_t)px;
        }
        return DQJ_OK;
    }

    // Other precisions and modes: an ordinary frame on the serving stream.
    dqj_status launch_plain(Request &r)
    {
        const uint64_t px = (uint64_t)r.p.width * (uint64_t)r.p.height;
        cudaError_t e = cudaMallocAsync(&r.scratch, scratch_bytes(r.p, false), pstream_);
        if (e == cudaSuccess) e = cudaMemsetAsync(r.scratch, 0, 256, pstream_);
        if (e != cudaSuccess) return cuda_fail(e, "serve: scratch");
        char *b = static_cast<char *>(r.scratch);
        Scratch sc{};
        sc.ctr = reinterpret_cast<Counters *>(b);
        sc.hits = reinterpret_cast<int4 *>(b + 256);
        sc.hit_cap = (uint32_t)px;
        if (r.p.precision == DQJ_FP32_RECHECK) {
            char *q = b + 256 + px * sizeof(int4);
            sc.queue = reinterpret_cast<int4 *>(q);
            sc.queue_cap = (uint32_t)(3 * px);
            sc.dirty_flag = reinterpret_cast<uint32_t *>(q + 3 * px * sizeof(int4));
            sc.dirty_list = reinterpret_cast<int32_t *>(q + 3 * px * sizeof(int4) + px * 4);
            sc.dirty_cap = (uint32_t)px;
            e = cudaMemsetAsync(sc.dirty_flag, 0, px * 4, pstream_);
            if (e != cudaSuccess) return cuda_fail(e, "serve: clear flags");
        }
        const FrameDesc fd = frame_of(r);
        e = launch_frame(fd, sc, pstream_, ctx_->num_sms);
        if (e == cudaSuccess && r.out.stats)
            e = cudaMemcpyAsync(r.out.stats, sc.ctr->stats, DQJ_NSTATS * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                pstream_);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r.done_ev, pstream_);
        if (e != cudaSuccess) return cuda_fail(e, "serve: frame launch");
        return DQJ_OK;
    }

  public:
    int poll(Request &r) override
    {
        if (r.packed) {
            const unsigned v = *reinterpret_cast<volatile unsigned *>(&h_flags_[r.slot]);
            if (v == (unsigned)r.seq) {
                record_interval(r.slot);
                return 1;
            }
            if (launched_) {
                const cudaError_t e = cudaEventQuery(kevent_);
                if (e != cudaSuccess && e != cudaErrorNotReady) {
                    cuda_fail(e, "serve: persistent kernel");
                    return -1;
                }
            }
            return 0;
        }
        const cudaError_t e = cudaEventQuery(r.done_ev);
        if (e == cudaSuccess) return 1;
        if (e == cudaErrorNotReady) return 0;
        cuda_fail(e, "serve: frame");
        return -1;
    }

    dqj_status kick(bool packed_active) override
    {
        if (!packed_active) return DQJ_OK;
        if (launched_) {
            const cudaError_t q = cudaEventQuery(kevent_);
            if (q == cudaErrorNotReady) return DQJ_OK;  // still running: it picks up new slots
            if (q != cudaSuccess) return cuda_fail(q, "serve: persistent kernel");
            completed_ = launches_;
        }
        cudaError_t e = cudaSetDevice(ctx_->device);
        ServeCtl ctl{d_slots_, d_blocks_, d_flags_, d_exit_, d_flags_ + kMaxSlots + 1, d_times_, idle_ns_, 1000000000ull};
        if (e == cudaSuccess) e = cudaMemsetAsync(d_exit_, 0, sizeof(unsigned), kstream_);  // ordered before the launch
        if (e == cudaSuccess) e = serve_launch(ctl, ctx_->num_sms, kstream_);
        if (e == cudaSuccess) e = cudaEventRecord(kevent_, kstream_);
        if (e != cudaSuccess) return cuda_fail(e, "serve: launch");
        launched_ = true;
        ++launches_;
        return DQJ_OK;
    }

    void release(Request &r) override
    {
        cudaSetDevice(ctx_->device);
        if (r.done_ev) {
            cudaEventDestroy(r.done_ev);
            r.done_ev = nullptr;
        }
        if (r.scratch) {  // plain-path scratch; packed requests use their slot's hit list
            cudaFreeAsync(r.scratch, pstream_);
            r.scratch = nullptr;
        }
        // a packed request's control block stays named by its slot until the
        // slot is republished (admit retires it then)
    }

    dqj_status shutdown(int64_t timeout_ms) override
    {
        cudaSetDevice(ctx_->device);
        const dqj_status st = stop_launch(timeout_ms);
        if (st == DQJ_OK) {
            cudaStreamSynchronize(pstream_);
            cudaStreamSynchronize(cstream_);
        }
        return st;
    }

    void launch_counts(int64_t &launches, int64_t &restarts) const override
    {
        launches = (int64_t)launches_;
        restarts = (int64_t)restarts_;
    }

    int64_t overlapped() const override { return overlapped_; }

  private:
    // The device interval of a finished request (written by the kernel to
    // mapped memory before the completion flag), checked against the last
    // kIntervals finished requests: an overlap means both ran on the device at
    // the same time.
    static constexpr int kIntervals = 256;
    void record_interval(int slot)
    {
        volatile unsigned long long *t = h_times_ + 2 * slot;
        const unsigned long long a = t[0], b = t[1];
        bool over = false;
        for (int i = 0; i < n_iv_; ++i) over = over || (a < iv_[i][1] && iv_[i][0] < b);
        if (over) ++overlapped_;
        iv_[iv_next_][0] = a;
        iv_[iv_next_][1] = b;
        iv_next_ = (iv_next_ + 1) % kIntervals;
        n_iv_ = std::min(n_iv_ + 1, kIntervals);
    }

    void free_all()
    {
        cudaSetDevice(ctx_->device);
        for (auto &p : slot_scratch_)
            if (p) cudaFree(p);
        if (d_slots_) cudaFree(d_slots_);
        if (d_blocks_) cudaFree(d_blocks_);
        if (d_exit_) cudaFree(d_exit_);
        if (h_flags_) cudaFreeHost(h_flags_);
        if (h_times_) cudaFreeHost(h_times_);
        if (zeros_) cudaFreeHost(zeros_);
        if (h_slots_) cudaFreeHost(h_slots_);
        if (h_blocks_) cudaFreeHost(h_blocks_);
        if (kevent_) cudaEventDestroy(kevent_);
        if (kstream_) cudaStreamDestroy(kstream_);
        if (cstream_) cudaStreamDestroy(cstream_);
        if (pstream_) cudaStreamDestroy(pstream_);
    }

    dqj_ctx *ctx_;
    ServeSlot *d_slots_ = nullptr, *h_slots_ = nullptr;  // h_slots_: the authoritative copy
    ReqBlock *d_blocks_ = nullptr, *h_blocks_ = nullptr;
    std::deque<std::pair<unsigned, uint64_t>> free_blocks_;  // (block, launch id when retired), oldest first
    unsigned slot_block_[kMaxSlots] = {};
    void *slot_scratch_[kMaxSlots] = {};
    uint64_t slot_px_[kMaxSlots] = {};  // pixel capacity of the slot's scratch
    bool slot_rq_[kMaxSlots] = {};      // ... and whether it holds the recheck regions
    unsigned long long *h_times_ = nullptr, *d_times_ = nullptr;  // per slot {first item, finished}
    void *zeros_ = nullptr;  // page-locked zeros for new tag regions
    size_t zeros_bytes_ = 0;
    unsigned long long iv_[kIntervals][2] = {};
    int n_iv_ = 0, iv_next_ = 0;
    int64_t overlapped_ = 0;
    unsigned *h_flags_ = nullptr, *d_flags_ = nullptr;  // [0, kMaxSlots) done flags, [kMaxSlots] = 1, then hold
    unsigned *d_exit_ = nullptr;
    cudaStream_t kstream_ = nullptr, cstream_ = nullptr, pstream_ = nullptr;
    cudaEvent_t kevent_ = nullptr;
    bool launched_ = false;
    uint64_t launches_ = 0, completed_ = 0, restarts_ = 0;
    unsigned long long idle_ns_ = 0;
};

// CPU-only stand-in for the device: a request "runs" for DQJ_MOCK_DELAY_US
// microseconds after admission.  DQJ_MOCK_FAIL=nomem fails every admission with
// DQJ_ERR_NOMEM; DQJ_MOCK_FAIL=hang never completes any request.
class MockBackend : public Backend {
  public:
    MockBackend()
    {
        delay_us_ = env_int("DQJ_MOCK_DELAY_US", 1000);
        const char *f = std::getenv("DQJ_MOCK_FAIL");
        nomem_ = f && std::strcmp(f, "nomem") == 0;
        hang_ = f && std::strcmp(f, "hang") == 0;
        throw_admit_ = f && std::strcmp(f, "throw_admit") == 0;
        if (f && std::strcmp(f, "throw_start") == 0) throw std::bad_alloc();  // a host allocation that fails
    }
    void admit(Request *const *rs, int n, dqj_status *st) override
    {
        if (throw_admit_) throw std::bad_alloc();
        for (int i = 0; i < n; ++i) {
            if (nomem_) {
                st[i] = fail(DQJ_ERR_NOMEM, "serve (mock): injected allocation failure");
                continue;
            }
            rs[i]->admitted = clk::now();
            ++running_;
            st[i] = DQJ_OK;
        }
    }
    void hold(bool) override {}
    int poll(Request &r) override
    {
        if (hang_) return 0;
        if (clk::now() - r.admitted >= std::chrono::microseconds(delay_us_)) {
            --running_;
            return 1;
        }
        return 0;
    }
    dqj_status kick(bool) override { return DQJ_OK; }
    void release(Request &) override {}
    dqj_status shutdown(int64_t) override
    {
        return running_ > 0 ? fail(DQJ_ERR_TIMEOUT, "serve (mock): requests never completed") : DQJ_OK;
    }

  private:
    int64_t delay_us_;
    bool nomem_ = false, hang_ = false, throw_admit_ = false;
    int running_ = 0;
};

}  // namespace

// -------------------------------------------------------------------------
// scheduler
// -------------------------------------------------------------------------
// DQJ_SERVE_SHORTEST key: the request's arrival (ns since the scheduler
// started) plus an estimate of its own march time, pixels x (march_steps + 1)
// samples at 2^-9 ns each (a 1920x1080 frame of 513 samples: 2.1 ms, close to
// its measured 1.8-2.0 ms).  A request is overtaken only by requests whose
// estimated finish comes first, and by none that arrive after its own
// estimated finish, so none waits without bound.
uint64_t shortest_key(const Request &r, clk::time_point t0)
{
    const int64_t arrival = std::chrono::duration_cast<std::chrono::nanoseconds>(r.submitted - t0).count();
    const double cost = (double)r.p.width * (double)r.p.height * (double)(r.p.march_steps + 1) / 512.0;
    return (uint64_t)(arrival > 0 ? arrival : 0) + (uint64_t)cost;
}

struct ServeState {
    dqj_ctx *ctx = nullptr;
    std::unique_ptr<Backend> backend;
    std::mutex mu;
    std::condition_variable cv;
    // Queued requests in admission order: by (key, ticket), the key being the
    // ticket under DQJ_SERVE_FIFO and the estimated finish (shortest_key) under
    // DQJ_SERVE_SHORTEST, as set at dqj_submit.
    std::map<std::pair<uint64_t, dqj_ticket>, std::unique_ptr<Request>> pending;
    std::map<dqj_ticket, std::unique_ptr<Request>> active;  // admitted, not finished
    // Ticket states for dqj_poll, under their own lock (tmu): a client polling
    // in a tight loop never contends for the scheduler's lock (mu), whose
    // unfair hand-over could otherwise starve the scheduler thread.  Lock
    // order: mu before tmu.
    struct TicketState {
        bool done = false;
        dqj_status status = DQJ_OK;
    };
    std::mutex tmu;
    std::unordered_map<dqj_ticket, TicketState> tickets;
    Request *slot_req[kMaxSlots] = {};
    uint64_t used = 0;
    dqj_ticket next_ticket = 1;
    uint64_t next_seq = 1;
    bool draining = false, stop = false;
    std::atomic<bool> failed{false};  // the scheduler thread stopped on a host exception
    const clk::time_point t0 = clk::now();
    std::thread thr;
    int64_t n_packed = 0, n_plain = 0, n_batches = 0, admit_ns = 0, n_completed = 0, n_loops = 0, max_active = 0;

    void set_done(dqj_ticket t, dqj_status st)
    {
        std::lock_guard<std::mutex> lk(tmu);
        TicketState &ts = tickets[t];
        ts.done = true;
        ts.status = st;
    }

    void complete(Request *r, dqj_status st)
    {
        backend->release(*r);
        if (r->slot >= 0) slot_req[r->slot] = nullptr;
        used -= r->footprint;
        set_done(r->ticket, st);
        ++n_completed;
    }

    // The scheduler thread threw (a host allocation inside it failed): queued
    // requests end with DQJ_ERR_NOMEM and later submits are refused.  Admitted
    // requests stay unfinished, since their device work may still be running,
    // so dqj_destroy waits for them and reports DQJ_ERR_TIMEOUT.
    void on_failure() noexcept
    {
        failed = true;
        try {
            std::lock_guard<std::mutex> lk(mu);
            for (auto &kv : pending) set_done(kv.first.second, DQJ_ERR_NOMEM);
            pending.clear();
            cv.notify_all();
        } catch (...) {
        }
    }

    void loop()
    {
        std::unique_lock<std::mutex> lk(mu);
        std::vector<Request *> batch;
        std::vector<dqj_status> st;
        while (!stop) {
            ++n_loops;
            // completions
            for (auto it = active.begin(); it != active.end();) {
                Request *r = it->second.get();
                const int s = r->seq ? backend->poll(*r) : 0;
                if (s != 0) {
                    complete(r, s > 0 ? DQJ_OK : DQJ_ERR_CUDA);
                    it = active.erase(it);
                } else {
                    ++it;
                }
            }
            // choose admissions in queue order while the budget and a slot allow;
            // they count as active (dqj_poll sees them) while being written
            batch.clear();
            while (!draining && !pending.empty()) {
                Request *r = pending.begin()->second.get();
                if (used + r->footprint > ctx->cfg.mem_budget_bytes) break;
                int slot = -1;
                if (r->packed) {
                    for (int s = 0; s < kMaxSlots && slot < 0; ++s)
                        if (!slot_req[s]) slot = s;
                    if (slot < 0) break;
                    slot_req[slot] = r;
                }
                r->slot = slot;
                used += r->footprint;
                active.emplace(r->ticket, std::move(pending.begin()->second));
                pending.erase(pending.begin());
                batch.push_back(r);
            }
            max_active = std::max<int64_t>(max_active, (int64_t)active.size());
            backend->hold(!pending.empty() || !active.empty());
            if (!batch.empty()) {
                const int policy = ctx->serve_policy.load(std::memory_order_relaxed);
                for (Request *r : batch) {
                    r->seq = next_seq++;
                    if ((unsigned)r->seq == 0) r->seq = next_seq++;  // generation 0 means "empty"
                    r->prio = policy == DQJ_SERVE_SHORTEST ? shortest_key(*r, t0) : r->seq;
                }
                // write the slots / launch the frames without holding the lock
                st.assign(batch.size(), DQJ_OK);
                lk.unlock();
                const auto ta = clk::now();
                backend->admit(batch.data(), (int)batch.size(), st.data());
                const int64_t dt = std::chrono::duration_cast<std::chrono::nanoseconds>(clk::now() - ta).count();
                lk.lock();
                admit_ns += dt;
                ++n_batches;
                for (Request *r : batch) ++(r->packed ? n_packed : n_plain);
                for (size_t i = 0; i < batch.size(); ++i) {
                    if (st[i] == DQJ_OK) continue;
                    complete(batch[i], st[i]);
                    active.erase(batch[i]->ticket);
                }
            }
            bool packed_active = false;
            for (auto &kv : active) packed_active = packed_active || kv.second->packed;
            if (backend->kick(packed_active) != DQJ_OK) {
                for (auto &kv : active) complete(kv.second.get(), DQJ_ERR_CUDA);
                active.clear();
            }
            cv.notify_all();
            if (!active.empty())
                cv.wait_for(lk, std::chrono::microseconds(20));
            else
                cv.wait(lk, [&] { return stop || (!pending.empty() && !draining); });
        }
        backend->hold(false);
    }
};

dqj_status serve_start(dqj_ctx *ctx)
{
    if (ctx->serve) return DQJ_OK;
    auto st = std::make_unique<ServeState>();
    st->ctx = ctx;
    if (ctx->device == DQJ_DEVICE_MOCK) {
        st->backend = std::make_unique<MockBackend>();
    } else {
        auto g = std::make_unique<GpuBackend>(ctx);
        dqj_status s = g->init();
        if (s != DQJ_OK) return s;
        st->backend = std::move(g);
    }
    ServeState *raw = st.release();
    raw->thr = std::thread([raw] {
        try {
            raw->loop();
        } catch (...) {
            raw->on_failure();
        }
    });
    ctx->serve = raw;
    return DQJ_OK;
}

}  // namespace dqj

using namespace dqj;

extern "C" {

dqj_status dqj_submit(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, dqj_ticket *ticket)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx || !ticket) return fail(DQJ_ERR_INVALID, "ctx or ticket is NULL");
        dqj_status s = validate(p);
        if (s != DQJ_OK) return s;
        if (!out) return fail(DQJ_ERR_INVALID, "outputs is NULL");
        if (out->pitch_px < p->width) return fail(DQJ_ERR_INVALID, "pitch_px must be >= width");
        const void *planes[4] = {out->iter, out->depth, out->normal, out->rgba};
        for (const void *q : planes)
            if (q && (reinterpret_cast<uintptr_t>(q) & 3u)) return fail(DQJ_ERR_INVALID, "planes must be 4-byte aligned");
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            s = serve_start(ctx);
            if (s != DQJ_OK) return s;
        }
        ServeState &S = *ctx->serve;
        auto r = std::make_unique<Request>();
        r->p = *p;
        r->out = *out;
        r->packed = ctx->device != DQJ_DEVICE_MOCK && packable(*p);
        r->footprint = footprint(*p, r->packed);
        if (r->footprint > ctx->cfg.mem_budget_bytes)
            return fail(DQJ_ERR_NOMEM, "request footprint exceeds the context's memory budget");
        std::lock_guard<std::mutex> lk(S.mu);
        if (S.draining) return fail(DQJ_ERR_CANCELLED, "context is being destroyed");
        if (S.failed) return fail(DQJ_ERR_NOMEM, "serving stopped after a host allocation failure");
        if ((int64_t)S.pending.size() >= ctx->cfg.max_pending) return fail(DQJ_ERR_BUSY, "serving queue is full");
        r->ticket = S.next_ticket++;
        r->submitted = clk::now();
        const uint64_t key = ctx->serve_policy.load(std::memory_order_relaxed) == DQJ_SERVE_SHORTEST
                                 ? shortest_key(*r, S.t0)
                                 : r->ticket;
        {
            std::lock_guard<std::mutex> tl(S.tmu);
            S.tickets.emplace(r->ticket, ServeState::TicketState{});
        }
        *ticket = r->ticket;
        S.pending.emplace(std::make_pair(key, r->ticket), std::move(r));
        S.cv.notify_all();
        return DQJ_OK;
    });
}

dqj_status dqj_serve_policy(dqj_ctx *ctx, int32_t policy)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        if (policy != DQJ_SERVE_FIFO && policy != DQJ_SERVE_SHORTEST)
            return fail(DQJ_ERR_INVALID, "policy must be DQJ_SERVE_FIFO or DQJ_SERVE_SHORTEST");
        ctx->serve_policy.store(policy, std::memory_order_relaxed);
        return DQJ_OK;
    });
}

dqj_status dqj_serve_stats(dqj_ctx *ctx, int64_t *out)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx || !out) return fail(DQJ_ERR_INVALID, "ctx or out is NULL");
        for (int i = 0; i < DQJ_NSERVE_STATS; ++i) out[i] = 0;
        if (!ctx->serve) return DQJ_OK;
        ServeState &S = *ctx->serve;
        std::lock_guard<std::mutex> lk(S.mu);
        S.backend->launch_counts(out[0], out[1]);
        out[2] = S.n_packed;
        out[3] = S.n_plain;
        out[4] = S.n_batches;
        out[5] = S.admit_ns;
        out[6] = S.n_completed;
        out[7] = S.n_loops;
        out[8] = S.max_active;
        out[9] = S.backend->overlapped();
        return DQJ_OK;
    });
}

dqj_status dqj_poll(dqj_ctx *ctx, dqj_ticket ticket, int *done, dqj_status *result)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx || !done || !result) return fail(DQJ_ERR_INVALID, "ctx, done or result is NULL");
        if (!ctx->serve) return fail(DQJ_ERR_NOT_FOUND, "unknown ticket");
        ServeState &S = *ctx->serve;
        std::lock_guard<std::mutex> lk(S.tmu);
        auto f = S.tickets.find(ticket);
        if (f == S.tickets.end()) return fail(DQJ_ERR_NOT_FOUND, "unknown or already consumed ticket");
        *done = f->second.done ? 1 : 0;
        if (f->second.done) {
            *result = f->second.status;
            S.tickets.erase(f);
        }
        return DQJ_OK;
    });
}

dqj_status dqj_destroy(dqj_ctx *ctx)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        const bool device_ctx = ctx->device != DQJ_DEVICE_MOCK;
        dqj_status result = DQJ_OK;
        if (ctx->serve) {
            ServeState &S = *ctx->serve;
            const int64_t timeout_ms = env_int("DQJ_DESTROY_TIMEOUT_MS", 10000);
            {
                std::unique_lock<std::mutex> lk(S.mu);
                S.draining = true;
                for (auto &kv : S.pending) S.set_done(kv.first.second, DQJ_ERR_CANCELLED);
                S.pending.clear();
                S.cv.notify_all();
                S.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return S.active.empty(); });
                S.stop = true;
                S.cv.notify_all();
            }
            S.thr.join();
            result = S.backend->shutdown(S.active.empty() ? timeout_ms : 0);
            if (!S.active.empty() && result == DQJ_OK)
                result = fail(DQJ_ERR_TIMEOUT, "requests still running when the context was destroyed");
            if (result == DQJ_OK || ctx->device == DQJ_DEVICE_MOCK) {
                for (auto &kv : S.active) S.backend->release(*kv.second);
                delete ctx->serve;
                ctx->serve = nullptr;
            } else {
                // the device may still be using the requests' memory: leak it rather than free it under the kernel
                ctx->serve = nullptr;
            }
        }
        if (ctx->device != DQJ_DEVICE_MOCK) {
            cudaSetDevice(ctx->device);
            if (ctx->done_capture)  // the last render was captured in a graph: its event is a graph node
                cudaDeviceSynchronize();
            else if (ctx->done_ev)
                cudaEventSynchronize(ctx->done_ev);
            if (ctx->host_stream) cudaStreamSynchronize(ctx->host_stream);
            if (ctx->host_copy_stream) cudaStreamSynchronize(ctx->host_copy_stream);
            for (int l = 0; l < 2; ++l)
                if (ctx->lane_stream[l]) cudaStreamSynchronize(ctx->lane_stream[l]);
            scratch_free(ctx->scratch);
            scratch_free(ctx->scratch2);
            for (int l = 0; l < 2; ++l) {
                if (ctx->lane_stream[l]) cudaStreamDestroy(ctx->lane_stream[l]);
                for (cudaEvent_t &v : ctx->lane_ev[l])
                    if (v) cudaEventDestroy(v);
                if (ctx->join_ev[l]) cudaEventDestroy(ctx->join_ev[l]);
            }
            if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
            for (int b = 0; b < 2; ++b) {
                if (ctx->host_planes[b]) cudaFree(ctx->host_planes[b]);
                if (ctx->host_rendered[b]) cudaEventDestroy(ctx->host_rendered[b]);
                if (ctx->host_copied[b]) cudaEventDestroy(ctx->host_copied[b]);
            }
            if (ctx->vox_scratch) cudaFree(ctx->vox_scratch);
            if (ctx->host_stream) cudaStreamDestroy(ctx->host_stream);
            if (ctx->host_copy_stream) cudaStreamDestroy(ctx->host_copy_stream);
            if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
            for (auto &v : ctx->ev)
                if (v) cudaEventDestroy(v);
            ctx->ev.clear();
        }
        delete ctx;
        if (device_ctx) (void)cudaGetLastError();  // teardown leaves no error behind for the caller
        return result;
    });
}

}  // extern "C"
