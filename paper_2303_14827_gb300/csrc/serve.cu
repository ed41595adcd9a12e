// serve.cu -- persistent serving kernel: render requests of different sizes run
// together in one launch.
//
// The host admits requests into device-resident slots (ServeSlot).  Each warp of
// the persistent grid repeatedly picks the oldest slot that still has work,
// claims one work item from it and runs it:
//   MARCH phase : one 64-ray tile of the paired march (march2_tile);
//   BISECT phase: 32 hit-list entries (bisect_chunk);
// The warp that completes a request's last march tile switches it to the
// bisection phase (or finishes it when it has no hits).  The warp that completes
// its last bisection chunk copies the request's counters to the caller's stats
// array and writes the request's generation to a completion flag in mapped host
// memory.  A request's results are those of dqj_render: every pixel's arithmetic
// is independent of which warp, tile order or neighbouring requests ran it.
//
// Slots are rewritten by the host while the kernel runs, so slot reads follow a
// sequence lock: a slot is empty while its seq is 0, the host writes the body and
// then the new seq, and a warp accepts a body only if seq reads the same before
// and after copying it.  Work claims are compare-and-swap on 64-bit words tagged
// with the request's generation (the low 32 bits of seq), so a warp holding a
// stale view of a reused slot can neither claim nor corrupt the new request.
// Every wait is bounded: an idle warp rescans for at most `idle_ns` of
// %globaltimer time and then exits (the host relaunches when new work arrives),
// and a warp also exits when the host raises the stop flag.
#include "render_common.cuh"
#include "serve_internal.h"

namespace dqj {

namespace {

__device__ __forceinline__ unsigned long long ld_vol64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ unsigned ld_vol32(const unsigned *p) { return *reinterpret_cast<const volatile unsigned *>(p); }

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Claim `inc` items from a generation-tagged counter word if its generation is
// gen and its count is below limit.  Bounded number of attempts.
__device__ __forceinline__ bool claim(unsigned long long *w, unsigned gen, unsigned limit, unsigned inc,
                                      unsigned &got)
{
    unsigned long long old = ld_vol64(w);
    for (int tries = 0; tries < 256; ++tries) {
        if ((unsigned)(old >> 32) != gen) return false;
        const unsigned cnt = (unsigned)old;
        if (cnt >= limit) return false;
        const unsigned long long prev = atomicCAS(w, old, old + inc);
        if (prev == old) {
            got = cnt;
            return true;
        }
        old = prev;
    }
    return false;
}

__device__ __forceinline__ void finish_request(ServeSlot *slot, const ServeCtl &ctl, const Scratch &sc,
                                               int64_t *stats, unsigned gen, int slot_index)
{
    if (stats) {
        for (int i = 0; i < DQJ_NSTATS_DEV; ++i)
            stats[i] = (int64_t)*(volatile unsigned long long *)&sc.ctr->stats[i];
    }
    __threadfence_system();
    atomicExch(&slot->phase, ((unsigned long long)gen << 32) | kPhaseDone);
    *(volatile unsigned *)&ctl.done_flags[slot_index] = gen;
    __threadfence_system();
}

}  // namespace

__global__ void __launch_bounds__(kBlock, 4) serve_kernel(ServeCtl ctl)
{
    __shared__ FrameDesc s_fd[kBlock / 32];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    FrameDesc &fd = s_fd[wib];
    unsigned long long cached_seq = 0;
    int cached_slot = -1;
    Scratch sc{};
    unsigned long long idle_since = 0;
    for (;;) {
        if (*(volatile unsigned *)ctl.stop) break;
        // ---- pick the oldest slot with claimable work (two slots per lane)
        unsigned long long best = ~0ull;
        int best_slot = -1;
#pragma unroll
        for (int h = 0; h < kMaxSlots / 32; ++h) {
            const int s = lane + 32 * h;
            ServeSlot *sl = &ctl.slots[s];
            const unsigned long long seq = ld_vol64(&sl->seq);
            if (seq == 0) continue;
            const unsigned gen = (unsigned)seq;
            const unsigned long long ph = ld_vol64(&sl->phase);
            if ((unsigned)(ph >> 32) != gen) continue;
            bool work = false;
            if ((ph & 3u) == kPhaseMarch) {
                const unsigned long long c = ld_vol64(&sl->tile_claim);
                work = (unsigned)(c >> 32) == gen && (unsigned)c < ld_vol32(&sl->ntiles);
            } else if ((ph & 3u) == kPhaseBisect) {
                const unsigned long long c = ld_vol64(&sl->hit_claim);
                work = (unsigned)(c >> 32) == gen && (unsigned)c < ld_vol32(&sl->hit_total);
            }
            if (work && seq < best) {
                best = seq;
                best_slot = s;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(kFull, best, o);
            const int os = __shfl_xor_sync(kFull, best_slot, o);
            if (ob < best) {
                best = ob;
                best_slot = os;
            }
        }
        if (best_slot < 0) {
            const unsigned long long now = globaltimer_ns();
            if (idle_since == 0) idle_since = now;
            if (now - idle_since > ctl.idle_ns) break;
            __nanosleep(2000);
            continue;
        }
        ServeSlot *sl = &ctl.slots[best_slot];
        const unsigned gen = (unsigned)best;
        // ---- take a consistent copy of the slot body (sequence lock)
        if (cached_slot != best_slot || cached_seq != best) {
            const uint4 *src = reinterpret_cast<const uint4 *>(&sl->fd);
            uint4 *dst = reinterpret_cast<uint4 *>(&fd);
            for (int i = lane; i < (int)(sizeof(FrameDesc) / sizeof(uint4)); i += 32) dst[i] = __ldcg(src + i);
            const uint4 *ssrc = reinterpret_cast<const uint4 *>(&sl->sc);
            uint4 tmp[sizeof(Scratch) / sizeof(uint4)];
#pragma unroll
            for (int i = 0; i < (int)(sizeof(Scratch) / sizeof(uint4)); ++i) tmp[i] = __ldcg(ssrc + i);
            memcpy(&sc, tmp, sizeof(Scratch));
            __threadfence();
            __syncwarp();
            cached_slot = best_slot;
            cached_seq = best;
        }
        unsigned item = 0;
        int kind = 0;  // 1 march tile, 2 bisection chunk
        if (lane == 0) {
            if (ld_vol64(&sl->seq) == best) {
                const unsigned long long ph = ld_vol64(&sl->phase);
                if ((unsigned)(ph >> 32) == gen) {
                    if ((ph & 3u) == kPhaseMarch && claim(&sl->tile_claim, gen, ld_vol32(&sl->ntiles), 1u, item))
                        kind = 1;
                    else if ((ph & 3u) == kPhaseBisect &&
                             claim(&sl->hit_claim, gen, ld_vol32(&sl->hit_total), 32u, item))
                        kind = 2;
                }
            }
        }
        kind = __shfl_sync(kFull, kind, 0);
        item = __shfl_sync(kFull, item, 0);
        if (kind == 0) {
            cached_slot = -1;  // re-validate next time
            const unsigned long long now = globaltimer_ns();
            if (idle_since == 0) idle_since = now;
            if (now - idle_since > ctl.idle_ns) break;
            continue;
        }
        idle_since = 0;
        LaneStats st;
        if (kind == 1) {
            PairConsts P = fd.p2;
            march2_tile<0, 0, false>(fd, P, sc, item, st);
            flush_lane_stats<false>(sc, st, true);
            __threadfence();
            unsigned long long done = 0;
            if (lane == 0) done = atomicAdd(&sl->tile_done, 1ull) + 1ull;
            done = __shfl_sync(kFull, done, 0);
            if (lane == 0 && (unsigned)done == ld_vol32(&sl->ntiles)) {
                const unsigned nh = min(*(volatile unsigned *)&sc.ctr->hit_count, sc.hit_cap);
                *reinterpret_cast<volatile unsigned *>(&sl->hit_total) = nh;
                __threadfence();
                if (nh == 0)
                    finish_request(sl, ctl, sc, fd.stats, gen, best_slot);
                else
                    atomicExch(&sl->phase, ((unsigned long long)gen << 32) | kPhaseBisect);
            }
        } else {
            const unsigned nh = ld_vol32(&sl->hit_total);
            bisect_chunk<float, 0, 0, false>(fd, sc, item, nh, st);
            flush_lane_stats<false>(sc, st, false);
            __threadfence();
            const unsigned n = min(32u, nh - item);
            unsigned long long done = 0;
            if (lane == 0) done = atomicAdd(&sl->hit_done, (unsigned long long)n) + n;
            done = __shfl_sync(kFull, done, 0);
            if (lane == 0 && (unsigned)done == nh) finish_request(sl, ctl, sc, fd.stats, gen, best_slot);
        }
    }
}

cudaError_t serve_launch(const ServeCtl &ctl, int num_sms, cudaStream_t st)
{
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kBlock, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    serve_kernel<<<per_sm * num_sms, kBlock, 0, st>>>(ctl);
    return cudaGetLastError();
}

}  // namespace dqj
