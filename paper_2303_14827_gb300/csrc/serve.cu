// serve.cu -- persistent serving kernel: render requests of different sizes run
// together in one launch.
//
// The host admits a request by writing a control block (ReqBlock: frame
// constants, counters, claim counters) and then publishing its index in a slot
// (ServeSlot).  Each warp of the persistent grid repeatedly picks the published
// request with the smallest priority key that still has unclaimed work (the
// host sets the key: admission order, or arrival time plus the request's
// estimated cost), claims one work item from it with an atomic add and runs it:
//   MARCH phase : one 64-ray tile of the paired march (march2_tile);
//   BISECT phase: 32 hit-list entries (bisect_chunk).
// The warp that completes a request's last march tile switches it to the
// bisection phase (or finishes it when it has no hits).  The warp that completes
// its last bisection chunk copies the request's counters to the caller's stats
// array and writes the request's generation to the slot's completion flag in
// mapped host memory.  A request's results are those of dqj_render: every
// pixel's arithmetic is independent of which warp, tile order or neighbouring
// requests ran it.
//
// Apart from its counters a control block is immutable while published, and the
// host reuses one only after every warp of any launch that could have seen it
// has exited.  A warp acting on a stale view of a slot therefore meets only the
// exhausted claim counters of a finished request.  A launch that the host stops
// leaves no claimed item unfinished, so the next launch carries on from the
// claim counters.
//
// Every wait is bounded: an idle warp rescans for at most `idle_ns` of
// %globaltimer time and then ends the launch (the host relaunches when new work
// arrives).  While the host has queued or running requests it raises a hold
// flag, and idle warps then keep rescanning for up to `hold_ns`.  A launch ends
// as a whole: the warp that gives up raises the exit flag in device memory and
// every other warp leaves after its current item, so the host never mistakes a
// few remaining warps for a running launch.  The host raises the same flag (by a
// copy-engine write) to stop the launch.
#include "render_common.cuh"
#include "serve_internal.h"

namespace dqj {

namespace {

__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ unsigned ld_vol32(const unsigned *p) { return *reinterpret_cast<const volatile unsigned *>(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void finish_request(ReqBlock *b, const ServeCtl &ctl, int64_t *stats)
{
    if (stats) {
        for (int i = 0; i < DQJ_NSTATS_DEV; ++i) stats[i] = (int64_t)ld_vol64(&b->ctr.stats[i]);
    }
    __threadfence_system();
    st_release(&b->phase, kPhaseDone);
    *reinterpret_cast<volatile unsigned *>(&ctl.done_flags[__ldcg(&b->slot)]) = __ldcg(&b->gen);
    __threadfence_system();
}

// Has the request in block b unclaimed work?  (A hint: the claim re-checks.)
__device__ __forceinline__ bool has_work(const ReqBlock *b)
{
    const unsigned ph = ld_vol32(&b->phase);
    if (ph == kPhaseMarch) return ld_vol64(&b->tile_claim) < (unsigned long long)__ldcg(&b->ntiles);
    if (ph == kPhaseBisect) return ld_vol64(&b->hit_claim) < (unsigned long long)ld_vol32(&b->hit_total);
    return false;
}

__device__ __forceinline__ Scratch load_scratch(const Scratch *src)
{
    static_assert(sizeof(Scratch) % sizeof(uint4) == 0, "Scratch is copied as uint4");
    uint4 tmp[sizeof(Scratch) / sizeof(uint4)];
#pragma unroll
    for (int i = 0; i < (int)(sizeof(Scratch) / sizeof(uint4)); ++i)
        tmp[i] = __ldcg(reinterpret_cast<const uint4 *>(src) + i);
    Scratch sc;
    memcpy(&sc, tmp, sizeof(Scratch));
    return sc;
}

}  // namespace

__global__ void __launch_bounds__(kBlock, 4) serve_kernel(ServeCtl ctl)
{
    __shared__ FrameDesc s_fd[kBlock / 32];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    FrameDesc &fd = s_fd[wib];
    int cached = -1;  // block whose FrameDesc is in s_fd
    unsigned long long idle_since = 0;
    for (;;) {
        if (__shfl_sync(kFull, lane == 0 ? ld_vol32(ctl.exit_flag) : 0u, 0)) break;
        // ---- the published request with the smallest key and unclaimed work (two slots per lane)
        unsigned long long best = ~0ull;
        int best_block = -1;
#pragma unroll
        for (int h = 0; h < kMaxSlots / 32; ++h) {
            const ServeSlot *sl = &ctl.slots[lane + 32 * h];
            if (ld_vol64(&sl->seq) == 0) continue;
            const unsigned long long key = ld_vol64(&sl->prio);
            if (key >= best) continue;
            const unsigned bi = ld_vol32(&sl->block);
            if (bi < (unsigned)kReqBlocks && has_work(&ctl.blocks[bi])) {
                best = key;
                best_block = (int)bi;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(kFull, best, o);
            const int obk = __shfl_xor_sync(kFull, best_block, o);
            if (ob < best) {
                best = ob;
                best_block = obk;
            }
        }
        // ---- claim one work item (lane 0)
        ReqBlock *b = best_block >= 0 ? &ctl.blocks[best_block] : nullptr;
        unsigned item = 0;
        int kind = 0;  // 1 march tile, 2 bisection chunk
        if (b && lane == 0) {
            const unsigned ph = ld_acquire(&b->phase);
            if (ph == kPhaseMarch) {
                const unsigned long long c = atomicAdd(&b->tile_claim, 1ull);
                if (c < (unsigned long long)__ldcg(&b->ntiles)) {
                    item = (unsigned)c;
                    kind = 1;
                }
            } else if (ph == kPhaseBisect) {
                // hit_total was written before the phase was released
                const unsigned nh = ld_vol32(&b->hit_total);
                if (ld_vol64(&b->hit_claim) < nh) {
                    const unsigned long long c = atomicAdd(&b->hit_claim, 32ull);
                    if (c < nh) {
                        item = (unsigned)c;
                        kind = 2;
                    }
                }
            }
        }
        kind = __shfl_sync(kFull, kind, 0);
        item = __shfl_sync(kFull, item, 0);
        if (kind == 0) {
            int quit = 0;
            if (lane == 0) {  // one clock reading per warp keeps the decision uniform
                const unsigned long long now = globaltimer_ns();
                if (idle_since == 0) idle_since = now;
                const unsigned long long idle = now - idle_since;
                // the hold flag lives in host memory: read it only once idle_ns has passed
                quit = idle > ctl.idle_ns && (idle > ctl.hold_ns || !ld_vol32(ctl.hold));
                if (quit) atomicExch(ctl.exit_flag, 1u);
            }
            if (__shfl_sync(kFull, quit, 0)) break;
            if (best_block < 0) __nanosleep(1000);
            continue;
        }
        idle_since = 0;
        if (cached != best_block) {  // immutable while published: copy once per launch
            const uint4 *src = reinterpret_cast<const uint4 *>(&b->fd);
            uint4 *dst = reinterpret_cast<uint4 *>(&fd);
            for (int i = lane; i < (int)(sizeof(FrameDesc) / sizeof(uint4)); i += 32) dst[i] = __ldcg(src + i);
            __syncwarp();
            cached = best_block;
        }
        const Scratch sc = load_scratch(&b->sc);
        LaneStats st;
        if (kind == 1) {
            PairConsts P = fd.p2;
            if (fd.axis_slice)
                march2_tile<0, 0, false, true>(fd, P, sc, item, st);
            else
                march2_tile<0, 0, false, false>(fd, P, sc, item, st);
            flush_lane_stats<false>(sc, st, true);
            __threadfence();
            unsigned long long done = 0;
            if (lane == 0) done = atomicAdd(&b->tile_done, 1ull) + 1ull;
            done = __shfl_sync(kFull, done, 0);
            if (lane == 0 && done == (unsigned long long)__ldcg(&b->ntiles)) {
                const unsigned nh = min(ld_vol32(&b->ctr.hit_count), sc.hit_cap);
                *reinterpret_cast<volatile unsigned *>(&b->hit_total) = nh;
                __threadfence();
                if (nh == 0)
                    finish_request(b, ctl, fd.stats);
                else
                    st_release(&b->phase, kPhaseBisect);
            }
        } else {
            const unsigned nh = ld_vol32(&b->hit_total);
            bisect_chunk<float, 0, 0, false>(fd, sc, item, nh, st);
            flush_lane_stats<false>(sc, st, false);
            __threadfence();
            const unsigned n = min(32u, nh - item);
            unsigned long long done = 0;
            if (lane == 0) done = atomicAdd(&b->hit_done, (unsigned long long)n) + n;
            done = __shfl_sync(kFull, done, 0);
            if (lane == 0 && done == (unsigned long long)nh) finish_request(b, ctl, fd.stats);
        }
    }
}

cudaError_t serve_launch(const ServeCtl &ctl, int num_sms, cudaStream_t st)
{
    static std::atomic<int> per_sm{0};
    serve_kernel<<<num_sms * resident_per_sm(per_sm, serve_kernel), kBlock, 0, st>>>(ctl);
    return cudaGetLastError();
}

}  // namespace dqj
