// serve.cpp -- serving entry points of libdqj: dqj_submit / dqj_poll /
// dqj_destroy and the scheduler thread behind them (continuous batching).
//
// A request is queued on the host at dqj_submit.  The scheduler thread admits
// queued requests in arrival order while the sum of the admitted requests'
// footprints (output planes + scratch + slot) fits the context's memory budget
// and a device slot is free.  Admitted FP32 / algebraic / EUCLID8 requests are
// written into device slots and run together in one persistent launch
// (serve.cu); requests arriving while it runs join it.  Other precisions and
// modes run as ordinary stream-ordered frames on the serving stream.  Completed
// requests release their budget, and dqj_poll hands back their status once.
//
// The scheduler talks to the device through a small backend interface.  The
// GPU backend is the real one; contexts created with device = DQJ_DEVICE_MOCK
// use a CPU-only mock whose completion delay, allocation failure or
// never-completing behaviour is set from the environment, so the admission,
// budget, BUSY, TIMEOUT and CANCELLED paths are testable without a GPU.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <memory>

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
    uint64_t seq = 0;
    // device resources
    void *scratch = nullptr;
    cudaEvent_t done_ev = nullptr;
    clk::time_point admitted{};
};

bool packable(const dqj_params &p)
{
    return p.precision == DQJ_FP32 && p.square_mode == DQJ_SQUARE_ALGEBRAIC && p.modulus_mode == DQJ_MODULUS_EUCLID8;
}

uint64_t scratch_bytes(const dqj_params &p, bool packed)
{
    const uint64_t px = (uint64_t)p.width * (uint64_t)p.height;
    uint64_t b = 256 + px * sizeof(int4);                                  // counters + hit list
    if (!packed && p.precision == DQJ_FP32_RECHECK) b += px * (4 * sizeof(int4) + 8);  // queue, tags, list
    return b;
}

uint64_t footprint(const dqj_params &p, bool packed)
{
    const uint64_t px = (uint64_t)p.width * (uint64_t)p.height;
    return px * 24 + scratch_bytes(p, packed) + sizeof(ServeSlot);
}

// -------------------------------------------------------------------------
// backends
// -------------------------------------------------------------------------
struct Backend {
    virtual ~Backend() = default;
    virtual dqj_status admit(Request &r) = 0;     // start running r (slot already chosen when packed)
    virtual int poll(Request &r) = 0;             // 1 done, 0 running, -1 failed (message set)
    virtual dqj_status kick(bool packed_active) = 0;
    virtual void release(Request &r) = 0;
    virtual dqj_status shutdown(int64_t timeout_ms) = 0;
};

class GpuBackend : public Backend {
  public:
    explicit GpuBackend(dqj_ctx *ctx) : ctx_(ctx) {}
    ~GpuBackend() override { free_all(); }

    dqj_status init()
    {
        cudaError_t e = cudaSetDevice(ctx_->device);
        if (e == cudaSuccess) e = cudaMalloc(&d_slots_, sizeof(ServeSlot) * kMaxSlots);
        if (e == cudaSuccess) e = cudaMemset(d_slots_, 0, sizeof(ServeSlot) * kMaxSlots);
        if (e == cudaSuccess) e = cudaHostAlloc(&h_flags_, sizeof(unsigned) * (kMaxSlots + 1), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(h_flags_, 0, sizeof(unsigned) * (kMaxSlots + 1));
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&d_flags_), h_flags_, 0);
        }
        if (e == cudaSuccess) e = cudaHostAlloc(&h_stage_, sizeof(ServeSlot) * kMaxSlots, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&kstream_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cstream_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pstream_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&kevent_, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "serve: init");
        idle_ns_ = (unsigned long long)env_int("DQJ_SERVE_IDLE_US", 2000) * 1000ull;
        return DQJ_OK;
    }

    dqj_status admit(Request &r) override
    {
        cudaError_t e = cudaSetDevice(ctx_->device);
        if (e != cudaSuccess) return cuda_fail(e, "serve: cudaSetDevice");
        const uint64_t px = (uint64_t)r.p.width * (uint64_t)r.p.height;
        const uint64_t sb = scratch_bytes(r.p, r.packed);
        cudaStream_t st = r.packed ? cstream_ : pstream_;
        e = cudaMallocAsync(&r.scratch, sb, st);
        if (e != cudaSuccess) return cuda_fail(e, "serve: scratch");
        e = cudaMemsetAsync(r.scratch, 0, 256, st);
        if (e != cudaSuccess) return cuda_fail(e, "serve: clear counters");
        char *b = static_cast<char *>(r.scratch);
        Scratch sc{};
        sc.ctr = reinterpret_cast<Counters *>(b);
        sc.hits = reinterpret_cast<int4 *>(b + 256);
        sc.hit_cap = (uint32_t)px;
        if (!r.packed && r.p.precision == DQJ_FP32_RECHECK) {
            char *q = b + 256 + px * sizeof(int4);
            sc.queue = reinterpret_cast<int4 *>(q);
            sc.queue_cap = (uint32_t)(3 * px);
            sc.dirty_flag = reinterpret_cast<uint32_t *>(q + 3 * px * sizeof(int4));
            sc.dirty_list = reinterpret_cast<int32_t *>(q + 3 * px * sizeof(int4) + px * 4);
            sc.dirty_cap = (uint32_t)px;
            e = cudaMemsetAsync(sc.dirty_flag, 0, px * 4, st);
            if (e != cudaSuccess) return cuda_fail(e, "serve: clear flags");
        }
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
        if (!r.packed) {
            e = launch_frame(fd, sc, st, ctx_->num_sms);
            if (e == cudaSuccess && r.out.stats)
                e = cudaMemcpyAsync(r.out.stats, sc.ctr->stats, DQJ_NSTATS * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                    st);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(r.done_ev, st);
            if (e != cudaSuccess) return cuda_fail(e, "serve: frame launch");
            return DQJ_OK;
        }
        // packed: write the slot (seq = 0, body, then seq) -- see serve.cu
        const unsigned gen = (unsigned)r.seq;
        const unsigned long long tag = (unsigned long long)gen << 32;
        ServeSlot &h = h_stage_[r.slot];
        std::memset(&h, 0, sizeof h);
        h.seq = 0;
        h.phase = tag | kPhaseMarch;
        h.tile_claim = h.tile_done = h.hit_claim = h.hit_done = tag;
        h.ntiles = (unsigned)fd.tiles_x * (unsigned)fd.tiles_y;
        h.hit_total = 0;
        h.sc = sc;
        h.fd = fd;
        ServeSlot *d = d_slots_ + r.slot;
        e = cudaMemsetAsync(&d->seq, 0, sizeof(unsigned long long), cstream_);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(reinterpret_cast<char *>(d) + sizeof(unsigned long long),
                                reinterpret_cast<char *>(&h) + sizeof(unsigned long long),
                                sizeof(ServeSlot) - sizeof(unsigned long long), cudaMemcpyHostToDevice, cstream_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cstream_);
        if (e == cudaSuccess) {
            seq_stage_[r.slot] = r.seq;
            e = cudaMemcpyAsync(&d->seq, &seq_stage_[r.slot], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                cstream_);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(cstream_);
        if (e != cudaSuccess) return cuda_fail(e, "serve: publish slot");
        return DQJ_OK;
    }

    int poll(Request &r) override
    {
        if (r.packed) {
            const unsigned v = *reinterpret_cast<volatile unsigned *>(&h_flags_[r.slot]);
            if (v == (unsigned)r.seq) return 1;
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
        }
        cudaError_t e = cudaSetDevice(ctx_->device);
        ServeCtl ctl{d_slots_, d_flags_, d_flags_ + kMaxSlots, idle_ns_};
        h_flags_[kMaxSlots] = 0;
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
        if (r.scratch) {
            cudaFreeAsync(r.scratch, r.packed ? cstream_ : pstream_);
            r.scratch = nullptr;
        }
    }

    dqj_status shutdown(int64_t timeout_ms) override
    {
        cudaSetDevice(ctx_->device);
        if (h_flags_) *reinterpret_cast<volatile unsigned *>(&h_flags_[kMaxSlots]) = 1;  // stop
        dqj_status st = DQJ_OK;
        if (launched_) {
            const auto t0 = clk::now();
            for (;;) {
                const cudaError_t q = cudaEventQuery(kevent_);
                if (q == cudaSuccess) break;
                if (q != cudaErrorNotReady) {
                    st = cuda_fail(q, "serve: persistent kernel");
                    break;
                }
                if (clk::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
                    st = fail(DQJ_ERR_TIMEOUT, "serve: persistent kernel did not stop in time");
                    break;
                }
                std::this_thread::sleep_for(std::chrono::microseconds(100));
            }
        }
        if (st == DQJ_OK) {
            cudaStreamSynchronize(pstream_);
            cudaStreamSynchronize(cstream_);
        }
        return st;
    }

    uint64_t launches() const { return launches_; }

  private:
    void free_all()
    {
        cudaSetDevice(ctx_->device);
        if (d_slots_) cudaFree(d_slots_);
        if (h_flags_) cudaFreeHost(h_flags_);
        if (h_stage_) cudaFreeHost(h_stage_);
        if (kevent_) cudaEventDestroy(kevent_);
        if (kstream_) cudaStreamDestroy(kstream_);
        if (cstream_) cudaStreamDestroy(cstream_);
        if (pstream_) cudaStreamDestroy(pstream_);
    }

    dqj_ctx *ctx_;
    ServeSlot *d_slots_ = nullptr;
    ServeSlot *h_stage_ = nullptr;
    unsigned long long seq_stage_[kMaxSlots] = {};
    unsigned *h_flags_ = nullptr, *d_flags_ = nullptr;
    cudaStream_t kstream_ = nullptr, cstream_ = nullptr, pstream_ = nullptr;
    cudaEvent_t kevent_ = nullptr;
    bool launched_ = false;
    uint64_t launches_ = 0;
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
    }
    dqj_status admit(Request &r) override
    {
        if (nomem_) return fail(DQJ_ERR_NOMEM, "serve (mock): injected allocation failure");
        r.admitted = clk::now();
        ++running_;
        return DQJ_OK;
    }
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
    bool nomem_ = false, hang_ = false;
    int running_ = 0;
};

}  // namespace

// -------------------------------------------------------------------------
// scheduler
// -------------------------------------------------------------------------
struct ServeState {
    dqj_ctx *ctx = nullptr;
    std::unique_ptr<Backend> backend;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Request>> pending;
    std::map<dqj_ticket, std::unique_ptr<Request>> active;  // admitted, not finished
    std::map<dqj_ticket, dqj_status> finished;              // awaiting dqj_poll
    Request *slot_req[kMaxSlots] = {};
    uint64_t used = 0;
    dqj_ticket next_ticket = 1;
    uint64_t next_seq = 1;
    bool draining = false, stop = false;
    std::thread thr;

    void complete(Request *r, dqj_status st)
    {
        backend->release(*r);
        if (r->slot >= 0) slot_req[r->slot] = nullptr;
        used -= r->footprint;
        finished[r->ticket] = st;
    }

    void loop()
    {
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            // completions
            for (auto it = active.begin(); it != active.end();) {
                const int s = backend->poll(*it->second);
                if (s != 0) {
                    complete(it->second.get(), s > 0 ? DQJ_OK : DQJ_ERR_CUDA);
                    it = active.erase(it);
                } else {
                    ++it;
                }
            }
            // admissions, in arrival order, while the budget and a slot allow
            while (!draining && !pending.empty()) {
                Request *r = pending.front().get();
                if (used + r->footprint > ctx->cfg.mem_budget_bytes) break;
                int slot = -1;
                if (r->packed) {
                    for (int s = 0; s < kMaxSlots && slot < 0; ++s)
                        if (!slot_req[s]) slot = s;
                    if (slot < 0) break;
                }
                std::unique_ptr<Request> own = std::move(pending.front());
                pending.pop_front();
                r->slot = slot;
                r->seq = next_seq++;
                if ((unsigned)r->seq == 0) r->seq = next_seq++;  // generation 0 means "empty"
                const dqj_status st = backend->admit(*r);
                if (st != DQJ_OK) {
                    backend->release(*r);
                    finished[r->ticket] = st;
                    continue;
                }
                if (slot >= 0) slot_req[slot] = r;
                used += r->footprint;
                active.emplace(r->ticket, std::move(own));
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
    raw->thr = std::thread([raw] { raw->loop(); });
    ctx->serve = raw;
    return DQJ_OK;
}

}  // namespace dqj

using namespace dqj;

extern "C" {

dqj_status dqj_submit(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, dqj_ticket *ticket)
{
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
    if ((int64_t)S.pending.size() >= ctx->cfg.max_pending) return fail(DQJ_ERR_BUSY, "serving queue is full");
    r->ticket = S.next_ticket++;
    *ticket = r->ticket;
    S.pending.push_back(std::move(r));
    S.cv.notify_all();
    return DQJ_OK;
}

dqj_status dqj_poll(dqj_ctx *ctx, dqj_ticket ticket, int *done, dqj_status *result)
{
    if (!ctx || !done || !result) return fail(DQJ_ERR_INVALID, "ctx, done or result is NULL");
    if (!ctx->serve) return fail(DQJ_ERR_NOT_FOUND, "unknown ticket");
    ServeState &S = *ctx->serve;
    std::lock_guard<std::mutex> lk(S.mu);
    auto f = S.finished.find(ticket);
    if (f != S.finished.end()) {
        *done = 1;
        *result = f->second;
        S.finished.erase(f);
        return DQJ_OK;
    }
    if (S.active.count(ticket)) {
        *done = 0;
        return DQJ_OK;
    }
    for (auto &r : S.pending)
        if (r->ticket == ticket) {
            *done = 0;
            return DQJ_OK;
        }
    return fail(DQJ_ERR_NOT_FOUND, "unknown or already consumed ticket");
}

dqj_status dqj_destroy(dqj_ctx *ctx)
{
    if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
    dqj_status result = DQJ_OK;
    if (ctx->serve) {
        ServeState &S = *ctx->serve;
        const int64_t timeout_ms = env_int("DQJ_DESTROY_TIMEOUT_MS", 10000);
        {
            std::unique_lock<std::mutex> lk(S.mu);
            S.draining = true;
            for (auto &r : S.pending) S.finished[r->ticket] = DQJ_ERR_CANCELLED;
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
        if (ctx->done_ev) cudaEventSynchronize(ctx->done_ev);
        if (ctx->host_stream) cudaStreamSynchronize(ctx->host_stream);
        scratch_free(ctx->scratch);
        if (ctx->host_planes) cudaFree(ctx->host_planes);
        if (ctx->host_stream) cudaStreamDestroy(ctx->host_stream);
        if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
        for (auto &v : ctx->ev)
            if (v) cudaEventDestroy(v);
        ctx->ev.clear();
    }
    delete ctx;
    return result;
}

}  // extern "C"
