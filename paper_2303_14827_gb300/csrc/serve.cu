// serve.cu -- persistent serving kernel: render requests of different sizes run
// together in one launch.
//
// The host admits a request by writing a control block (ReqBlock: frame
// constants, counters, claim counters) and then publishing its index in a slot
// (ServeSlot).  Each warp of the persistent grid repeatedly picks the published
// request with the smallest priority key that still has unclaimed work (the
// host sets the key: admission order, or arrival time plus the request's
// estimated cost), claims one work item from it with an atomic add and runs it:
//   MARCH phase  : one 64-ray tile of the paired march (march4_tile, or
//                  march2_tile with DQJ_MARCH_SAMPLES=1; in the recheck mode
//                  with the FP64 recheck of its staged samples);
//   BISECT phase : 32 hit-list entries (bisect_chunk);
//   RECHECK phase: 32 recheck-queue entries (recheck_entry), recheck mode only;
//   FIXUP phase  : one pixel to re-render in FP64 (fixup_pixel), recheck mode.
// The warp that completes a phase's last item moves the request to the next
// phase that has work.  The warp that completes its last item copies the
// request's counters to the caller's stats array and writes the request's
// generation to the slot's completion flag in mapped host memory (the time of
// its first claimed item and of its completion beside it).  A request's
// results are those of dqj_render: every pixel's arithmetic is independent of
// which warp, tile order or neighbouring requests ran it, and the passes run
// in the same order.
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
#include "../../include/dqj.h"

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

__device__ __forceinline__ void finish_request(ReqBlock *b, const ServeCtl &ctl, int64_t *stats)
{
    if (stats) {
        for (int i = 0; i < DQJ_NSTATS_DEV; ++i) stats[i] = (int64_t)ld_vol64(&b->ctr.stats[i]);
    }
    const unsigned slot = __ldcg(&b->slot);
    *reinterpret_cast<volatile unsigned long long *>(&ctl.times[2 * slot + 1]) = globaltimer_ns();
    __threadfence_system();
    st_release(&b->phase, kPhaseDone);
    *reinterpret_cast<volatile unsigned *>(&ctl.done_flags[slot]) = __ldcg(&b->gen);
    __threadfence_system();
}

// Move a request whose phase `from` has completed to the next phase with work,
// or finish it (one lane).  The counts of the next phases are final here: every
// warp that added to them did so before it counted its item as done.
__device__ __forceinline__ void next_phase(ReqBlock *b, const ServeCtl &ctl, const FrameDesc &fd, unsigned from)
{
    if (from == kPhaseMarch) {
        const unsigned nh = min(ld_vol32(&b->ctr.hit_count), __ldcg(&b->sc.hit_cap));
        *reinterpret_cast<volatile unsigned *>(&b->hit_total) = nh;
        if (nh > 0) {
            __threadfence();
            st_release(&b->phase, kPhaseBisect);
            return;
        }
        from = kPhaseBisect;
    }
    if (from == kPhaseBisect) {
        if (!__ldcg(&b->recheck)) {
            finish_request(b, ctl, fd.stats);
            return;
        }
        const unsigned nq = min(ld_vol32(&b->ctr.queue_count), __ldcg(&b->sc.queue_cap));
        *reinterpret_cast<volatile unsigned *>(&b->q_total) = nq;
        if (nq > 0) {
            __threadfence();
            st_release(&b->phase, kPhaseRecheck);
            return;
        }
        from = kPhaseRecheck;
    }
    if (from == kPhaseRecheck) {
        const unsigned nd = min(ld_vol32(&b->ctr.dirty_count), __ldcg(&b->sc.dirty_cap));
        *reinterpret_cast<volatile unsigned *>(&b->f_total) = nd;
        if (nd > 0) {
            __threadfence();
            st_release(&b->phase, kPhaseFixup);
            return;
        }
    }
    finish_request(b, ctl, fd.stats);
}

// Has the request in block b unclaimed work?  (A hint: the claim re-checks.)
__device__ __forceinline__ bool has_work(const ReqBlock *b)
{
    const unsigned ph = ld_vol32(&b->phase);
    if (ph == kPhaseMarch) return ld_vol64(&b->tile_claim) < (unsigned long long)__ldcg(&b->ntiles);
    if (ph == kPhaseBisect) return ld_vol64(&b->hit_claim) < (unsigned long long)ld_vol32(&b->hit_total);
    if (ph == kPhaseRecheck) return ld_vol64(&b->q_claim) < (unsigned long long)ld_vol32(&b->q_total);
    if (ph == kPhaseFixup) return ld_vol64(&b->f_claim) < (unsigned long long)ld_vol32(&b->f_total);
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

// The work items run behind calls of their own: the march with two samples
// per round takes 121-158 registers, and inlined into one loop with the
// scheduler it spilled registers in the hot loop.  The march takes the form
// dqj_render takes (fd.march_samples), so a served request's counters equal
// those of the alone render.
template <bool RECHECK, bool AXIS>
__device__ __noinline__ void march_item4(const FrameDesc &fd, const Scratch &sc, unsigned tile, int4 *stage)
{
    LaneStats st;
    march4_tile<0, 0, RECHECK, AXIS>(fd, fd.p2, sc, tile, st, stage);
    flush_lane_stats<false>(sc, st, true);
}

template <bool RECHECK, bool AXIS>
__device__ __noinline__ void march_item2(const FrameDesc &fd, const Scratch &sc, unsigned tile, int4 *stage)
{
    LaneStats st;
    march2_tile<0, 0, RECHECK, AXIS>(fd, fd.p2, sc, tile, st, stage);
    flush_lane_stats<false>(sc, st, true);
}

template <bool RECHECK, bool AXIS>
__device__ __forceinline__ void march_item(const FrameDesc &fd, const Scratch &sc, unsigned tile, int4 *stage)
{
    if (fd.march_samples == 2)
        march_item4<RECHECK, AXIS>(fd, sc, tile, stage);
    else
        march_item2<RECHECK, AXIS>(fd, sc, tile, stage);
}

template <bool RECHECK>
__device__ __noinline__ void bisect_item(const FrameDesc &fd, const Scratch &sc, unsigned base, unsigned nh)
{
    LaneStats st;
    bisect_chunk<float, 0, 0, RECHECK>(fd, sc, base, nh, st);
    flush_lane_stats<RECHECK>(sc, st, false);
}

__device__ __noinline__ void recheck_item(const FrameDesc &fd, const Scratch &sc, unsigned base, unsigned nq)
{
    const int lane = threadIdx.x & 31;
    if (base + lane < nq) recheck_entry<0, 0>(fd, sc, __ldcg(sc.queue + base + lane));
}

__device__ __noinline__ void fixup_item(const FrameDesc &fd, const Scratch &sc, unsigned i)
{
    unsigned long long its = 0, npx = 0;
    fixup_pixel<0, 0>(fd, __ldcg(sc.dirty_list + i), its, npx);
    flush_stat(&sc.ctr->stats[6], its);
    flush_stat(&sc.ctr->stats[5], npx);
}

// Claim up to `step` items of a phase (lane 0): the first claimed index, or
// ~0u when the phase has none left.
__device__ __forceinline__ unsigned claim(unsigned long long *ctr, unsigned total, unsigned step)
{
    if (ld_vol64(ctr) >= total) return ~0u;
    const unsigned long long c = atomicAdd(ctr, (unsigned long long)step);
    return c < total ? (unsigned)c : ~0u;
}

__global__ void __launch_bounds__(kBlock, 3) serve_kernel(ServeCtl ctl)
{
    __shared__ FrameDesc s_fd[kBlock / 32];
    __shared__ int4 s_stage[kBlock / 32][kQStage];  // recheck entries of a march tile, per warp
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
        unsigned item = ~0u, ph = kPhaseDone;
        if (b && lane == 0) {
            ph = ld_acquire(&b->phase);  // a phase's total was written before the phase was released
            if (ph == kPhaseMarch) {
                item = claim(&b->tile_claim, __ldcg(&b->ntiles), 1);
                if (item == 0) {  // the request's first item: its start on the device
                    *reinterpret_cast<volatile unsigned long long *>(&ctl.times[2 * __ldcg(&b->slot)]) =
                        globaltimer_ns();
                    __threadfence_system();  // visible to the host before the request's completion
                }
            } else if (ph == kPhaseBisect) {
                item = claim(&b->hit_claim, ld_vol32(&b->hit_total), 32);
            } else if (ph == kPhaseRecheck) {
                item = claim(&b->q_claim, ld_vol32(&b->q_total), 32);
            } else if (ph == kPhaseFixup) {
                item = claim(&b->f_claim, ld_vol32(&b->f_total), 1);
            }
        }
        item = __shfl_sync(kFull, item, 0);
        ph = __shfl_sync(kFull, ph, 0);
        if (item == ~0u) {
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
        const bool recheck = fd.precision == DQJ_FP32_RECHECK;
        unsigned long long *done_ctr;
        unsigned n_items, total;
        if (ph == kPhaseMarch) {
            if (recheck) {
                if (fd.axis_slice)
                    march_item<true, true>(fd, sc, item, s_stage[wib]);
                else
                    march_item<true, false>(fd, sc, item, s_stage[wib]);
            } else {
                if (fd.axis_slice)
                    march_item<false, true>(fd, sc, item, nullptr);
                else
                    march_item<false, false>(fd, sc, item, nullptr);
            }
            done_ctr = &b->tile_done;
            n_items = 1;
            total = __ldcg(&b->ntiles);
        } else if (ph == kPhaseBisect) {
            const unsigned nh = ld_vol32(&b->hit_total);
            if (recheck)
                bisect_item<true>(fd, sc, item, nh);
            else
                bisect_item<false>(fd, sc, item, nh);
            done_ctr = &b->hit_done;
            n_items = min(32u, nh - item);
            total = nh;
        } else if (ph == kPhaseRecheck) {
            const unsigned nq = ld_vol32(&b->q_total);
            recheck_item(fd, sc, item, nq);
            done_ctr = &b->q_done;
            n_items = min(32u, nq - item);
            total = nq;
        } else {
            fixup_item(fd, sc, item);
            done_ctr = &b->f_done;
            n_items = 1;
            total = ld_vol32(&b->f_total);
        }
        __threadfence();
        unsigned long long done = 0;
        if (lane == 0) done = atomicAdd(done_ctr, (unsigned long long)n_items) + n_items;
        done = __shfl_sync(kFull, done, 0);
        if (lane == 0 && done == (unsigned long long)total) next_phase(b, ctl, fd, ph);
    }
}

cudaError_t serve_launch(const ServeCtl &ctl, int num_sms, cudaStream_t st)
{
    static std::atomic<int> per_sm{0};
    serve_kernel<<<num_sms * resident_per_sm(per_sm, serve_kernel), kBlock, 0, st>>>(ctl);
    return cudaGetLastError();
}

}  // namespace dqj
