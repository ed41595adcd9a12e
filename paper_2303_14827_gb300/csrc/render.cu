// render.cu -- sm_103a kernels of the dual-quaternion Julia isosurface renderer.
//
// One frame runs as up to four stream-ordered passes:
//   march   : one ray per lane, 32 rays of a screen tile per warp.  The lanes
//             march in step: every trip of the warp classifies sample k of each
//             lane's ray (Method, "Ray-Marching": fixed steps over the box), so
//             neighbouring rays - which see almost the same escape counts - share
//             trips and no lane diverges.  Misses write their final outputs;
//             hits are appended to a compacted hit list.
//   bisect  : one hit per lane: B bisection steps of the first outside->inside
//             bracket, then the six central-difference evaluations of the normal
//             field (Method, "Lighting/Illumination") and Eq. phong shading
//             (ambient + diffuse).  Splitting hits from the march keeps the long
//             near-surface classifications together instead of stalling warps
//             that are still marching.
//   recheck : (FP32_RECHECK) samples whose modulus came within the margin of R^2
//             are re-evaluated in FP64 from FP64 ray parameters, one per thread;
//             a pixel whose FP64 escape count differs is queued for
//   fixup   : a complete FP64 re-render of that pixel, one per thread.
// Iteration counts are the algorithmic ones (escape count, or max_iter for an
// inside sample), accumulated per lane and added once per warp.
#include <cstdio>
#include <cstdlib>

#include "render_common.cuh"
#include "../../include/dqj.h"

namespace dqj {

namespace {

// ---------------------------------------------------------------------------
// march
// ---------------------------------------------------------------------------
template <typename T, int SQ, int MOD, bool RECHECK>
__global__ void __launch_bounds__(kBlock) march_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<T> &F = frame<T>(fd);
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    unsigned long long s_iters = 0, s_samples = 0, s_hits = 0, s_rechecks = 0;
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(&sc.ctr->tile_next, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        tile = subset_tile(fd, tile);
        const int tx = (int)(tile % (unsigned)fd.tiles_x), ty = (int)(tile / (unsigned)fd.tiles_x);
        const int x = tx * fd.tile_w + lane % fd.tile_w;
        const int y = ty * fd.tile_h + lane / fd.tile_w;
        const bool valid = x < fd.W && y < fd.H;
        T d[3] = {T(0), T(0), T(1)};
        T t_in = T(0), t_out = T(0);
        bool active = valid && camera_clip<T>(F, fd.W, fd.H, x, y, d, t_in, t_out);
        if (!active) t_in = t_out = T(0);
        T D[8];
        slice_dir<T>(F, d, D);
        const T delta = (t_out - t_in) / T(fd.N);
        // FP32 general slice: the first-iterate form of the paired kernel, same
        // operations per ray
        const bool it1 = sizeof(T) == 4 && !fd.axis_slice;
        T Q0[8], Q1[8], Q2[8], dot = T(0);
        if constexpr (sizeof(T) == 4)
            if (it1) first_iterate_coeffs<float, SQ>(F.A, D, F.c, dot, Q0, Q1, Q2);
        const T s_in = it1 ? (T)vadd((float)t_in, (float)dot) : t_in;
        int esc_max = 0, k_first = -1;
        unsigned iters = 0, samples = 0;
        for (int k = 0; k <= fd.N; ++k) {
            if (!__any_sync(kFull, active)) break;
            T z[8];
            bool mg;
            int n;
            if (it1) {
                if constexpr (sizeof(T) == 4) first_iterate<float, 8>(vfma((float)k, delta, s_in), Q0, Q1, Q2, z);
                n = classify_lockstep_it1<T, SQ, MOD, RECHECK>(z, F, fd.max_iter, active, mg);
            } else {
                const T t = dfma(T(k), delta, t_in);
#pragma unroll
                for (int i = 0; i < 8; ++i) z[i] = dfma(t, D[i], F.A[i]);
                n = classify_lockstep<T, SQ, MOD, RECHECK>(z, F, fd.max_iter, active, mg);
            }
            if (RECHECK) {
                const bool push = active && mg;
                if (warp_push(push, make_int4(y * fd.W + x, k | (kMarchSample << 16), 0, n), sc.queue,
                              sc.queue_cap, &sc.ctr->queue_count)) {
                    atomicAdd(&sc.ctr->stats[7], 1ull);
                    mark_dirty(fd, sc, y * fd.W + x);
                }
                s_rechecks += push ? 1 : 0;
            }
            if (active) {
                iters += n ? (unsigned)n : (unsigned)fd.max_iter;
                samples += 1;
                if (n == 0) {
                    k_first = k;
                    active = false;
                } else {
                    esc_max = n > esc_max ? n : esc_max;
                }
            }
        }
        s_iters += iters;
        s_samples += samples;
        const bool hit = valid && k_first >= 0;
        if (valid && !hit) write_miss<T>(fd, x, y, esc_max);
        s_hits += hit ? 1 : 0;
        warp_push(hit, make_int4(y * fd.W + x, k_first, 0, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
    }
    flush_stat(&sc.ctr->stats[0], s_iters);
    flush_stat(&sc.ctr->stats[8], s_iters);
    flush_stat(&sc.ctr->stats[2], s_samples);
    flush_stat(&sc.ctr->stats[3], s_hits);
    if (RECHECK) flush_stat(&sc.ctr->stats[4], s_rechecks);
}

// ---------------------------------------------------------------------------
// march, paired: two rays per lane, tile slots `lane` and `lane + 32` of a
// 64-ray tile, advanced together in the two halves of float2 registers by the
// paired FP32 instructions.  Same per-ray arithmetic as march_kernel<float>.
// Per ray it keeps only running sums: sum_* (steps stayed bounded, summed over
// samples), max_* (largest escape count - 1) and the first inside sample kf_*;
// the iteration and sample counts follow from them once the ray is done.  The
// escape count of the sample before a hit is classified again by the
// bisection pass, which needs it only for hits.
// ---------------------------------------------------------------------------
template <int SQ, int MOD, bool RECHECK, bool AXIS>
__global__ void __launch_bounds__(kBlock, AXIS ? 5 : 4)  // the general form keeps 24 coefficients per ray pair
    march2_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    __shared__ int4 stage[RECHECK ? kBlock / 32 : 1][RECHECK ? kQStage : 1];  // recheck entries, per warp
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(&sc.ctr->tile_next, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        tile = subset_tile(fd, tile);
        // counters are added per tile, so none stays live across the march loop
        LaneStats st;
        march2_tile<SQ, MOD, RECHECK, AXIS>(fd, fd.p2, sc, tile, st, stage[RECHECK ? threadIdx.x >> 5 : 0]);
        flush_lane_stats<false>(sc, st, true);
    }
}

// march2_kernel with two samples of each ray per round (march4_tile).  Its
// four sets of iterates take more registers: four CTAs per SM on an axis
// slice, three with the general form's first-iterate coefficients.
template <int SQ, int MOD, bool RECHECK, bool AXIS>
__global__ void __launch_bounds__(kBlock, AXIS ? 4 : 3) march4_kernel(const __grid_constant__ FrameDesc fd,
                                                                      const Scratch sc)
{
    __shared__ int4 stage[RECHECK ? kBlock / 32 : 1][RECHECK ? kQStage : 1];  // recheck entries, per warp
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(&sc.ctr->tile_next, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        tile = subset_tile(fd, tile);
        LaneStats st;
        march4_tile<SQ, MOD, RECHECK, AXIS>(fd, fd.p2, sc, tile, st, stage[RECHECK ? threadIdx.x >> 5 : 0]);
        flush_lane_stats<false>(sc, st, true);
    }
}

// ---------------------------------------------------------------------------
// split march, for frames with fewer tiles than the GPU has resident warps: a
// work item is one 64-ray tile and one of fd.k_split contiguous ranges of the
// samples, so that more warps share a small frame.  Ranges past a ray's first
// inside sample do work the march would not do (less when an earlier range
// has already recorded its hit: the ray is skipped); march_merge_kernel keeps
// only the ranges up to the first inside sample, so outputs and iteration
// counts are the march's.
// ---------------------------------------------------------------------------
template <int SQ, int MOD, bool AXIS>
__global__ void __launch_bounds__(kBlock, AXIS ? 5 : 4) march2_split_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    const unsigned items = ntiles * (unsigned)fd.k_split;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&sc.ctr->tile_next, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= items) break;
        // lower ranges first, so that later ones find the rays they can skip
        const unsigned r = item / ntiles, tile = subset_tile(fd, item % ntiles);
        const int kb = (int)r * fd.k_chunk, ke = min(kb + fd.k_chunk, fd.N + 1);
        LaneStats st;
        march2_tile<SQ, MOD, false, AXIS, true>(fd, fd.p2, sc, tile, st, nullptr, kb, ke);
    }
}

// march2_split_kernel with two samples of each ray per round (march4_tile).
template <int SQ, int MOD, bool AXIS>
__global__ void __launch_bounds__(kBlock, AXIS ? 4 : 3) march4_split_kernel(const __grid_constant__ FrameDesc fd,
                                                                            const Scratch sc)
{
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    const unsigned items = ntiles * (unsigned)fd.k_split;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&sc.ctr->tile_next, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= items) break;
        const unsigned r = item / ntiles, tile = subset_tile(fd, item % ntiles);
        const int kb = (int)r * fd.k_chunk, ke = min(kb + fd.k_chunk, fd.N + 1);
        LaneStats st;
        march4_tile<SQ, MOD, false, AXIS, true>(fd, fd.p2, sc, tile, st, nullptr, kb, ke);
    }
}

// Per pixel: the ranges of the split march in sample order up to the first
// with an inside sample give the pixel's result (a miss's largest escape count,
// or the hit's first inside sample for the bisection pass) and its iterations
// and samples.
__global__ void __launch_bounds__(kBlock) march_merge_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const int64_t npx = (int64_t)fd.W * fd.H;
    LaneStats st;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < npx; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pixel = base + threadIdx.x;
        const int x = (int)(pixel % fd.W), y = (int)(pixel / fd.W);
        // only the pixels of the frame's tile subset (dqj_render_tiles)
        const unsigned tile = (unsigned)(y / fd.tile_h) * (unsigned)fd.tiles_x + (unsigned)(x / fd.tile_w);
        const bool part = pixel < npx && tile % (unsigned)fd.tile_parts == (unsigned)fd.tile_part;
        int kf = -1, m = 0;
        unsigned iters = 0, samples = 0;
        // the first range with an inside sample is part_hit (the smallest range
        // that recorded one), so the ranges to read are known up front and
        // their loads need not wait on one another
        const unsigned rh = part ? __ldcg(sc.part_hit + pixel) : 0u;
        const int nr = part ? (rh < (unsigned)fd.k_split ? (int)rh + 1 : fd.k_split) : 0;
#pragma unroll 4
        for (int r = 0; r < nr; ++r) {
            const int4 e = __ldcg(sc.part + (int64_t)r * npx + pixel);
            iters += (unsigned)e.y;
            samples += (unsigned)e.w;
            if (r == (int)rh) kf = e.x;
            else m = max(m, e.z);
        }
        const bool hit = kf >= 0;
        st.iters += iters;
        st.samples += samples;
        st.hits += hit ? 1 : 0;
        if (part && !hit) write_miss<float>(fd, x, y, m);
        warp_push(hit, make_int4((int)pixel, kf, 0, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
    }
    flush_lane_stats<false>(sc, st, true);
}

// ---------------------------------------------------------------------------
// bisect + normal + shade over the hit list
// ---------------------------------------------------------------------------
// Hit lists shorter than group_below take group_lanes (4) lanes per hit
// (bisect_group): one lane per hit would give the launch's warps too few hits
// to hide the bisection's dependent chain.  Longer lists take one lane per hit
// (the least work per hit).  Both forms give the same results.
template <typename T, int SQ, int MOD, bool RECHECK>
__global__ void __launch_bounds__(kBlock) bisect_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc,
                                                        unsigned group_below, int group_lanes)
{
    const int lane = threadIdx.x & 31;
    const unsigned nhits = min(*(volatile unsigned *)&sc.ctr->hit_count, sc.hit_cap);
    const int lanes = nhits < group_below ? group_lanes : 1;
    const unsigned per = 32u / (unsigned)lanes;
    LaneStats st;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&sc.ctr->hit_next, per);
        base = __shfl_sync(kFull, base, 0);
        if (base >= nhits) break;
        if (lanes == 4)
            bisect_group<T, SQ, MOD, RECHECK, 4>(fd, sc, base, nhits, st);
        else
            bisect_chunk<T, SQ, MOD, RECHECK>(fd, sc, base, nhits, st);
    }
    flush_lane_stats<RECHECK>(sc, st, false);
}

// ---------------------------------------------------------------------------
// FP64 recheck of queued samples and FP64 re-render of disagreeing pixels
// ---------------------------------------------------------------------------
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) recheck_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const unsigned total = *(volatile unsigned *)&sc.ctr->queue_count;
    const unsigned nq = min(total, sc.queue_cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x)
        recheck_entry<SQ, MOD>(fd, sc, sc.queue[i]);
    // a full queue: pixels whose samples did not fit were flagged by the pushers
}

// FP64 re-render of the pixels queued by the recheck, one pixel per warp
// (fixup_pixel).  Pixels go to warps of different blocks first, so a short
// list spreads over the SMs.
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) fixup_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const int lane = threadIdx.x & 31;
    const unsigned nd = min(*(volatile unsigned *)&sc.ctr->dirty_count, sc.dirty_cap);
    const unsigned warp = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = gridDim.x * (blockDim.x >> 5);
    unsigned long long its = 0, npx = 0;
    for (unsigned i = warp; i < nd; i += nwarps) fixup_pixel<SQ, MOD>(fd, sc.dirty_list[i], its, npx);
    const unsigned long long v = warp_sum(its), p = warp_sum(npx);
    if (lane == 0) {
        if (v) atomicAdd(&sc.ctr->stats[6], v);
        if (p) atomicAdd(&sc.ctr->stats[5], p);
    }
}

// Lanes per hit of a short hit list, and the hit-list length below which a
// list counts as short: fewer hits than 32 per resident warp of the bisection
// launch (capb CTAs of four warps).  DQJ_BISECT_GROUP = 1 or 4 forces that
// many lanes per hit for every list.  (Eight lanes per hit, three tree levels
// per round, measured slower than four at every list length.)
int bisect_forced_lanes()
{
    static const int forced = [] {
        const char *e = std::getenv("DQJ_BISECT_GROUP");
        const long v = e ? std::strtol(e, nullptr, 10) : 0L;
        return v == 1 || v == 4 ? (int)v : 0;
    }();
    return forced;
}
int bisect_group_lanes() { return 4; }
unsigned bisect_group_below(int capb)
{
    if (bisect_forced_lanes() == 1) return 0u;
    if (bisect_forced_lanes() > 1) return 0xffffffffu;
    return (unsigned)capb * 4u * 32u;
}

template <typename T, int SQ, int MOD, bool RECHECK>
cudaError_t launch_passes(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    static std::atomic<int> g_march{0}, g_march2a{0}, g_march2g{0}, g_bisect{0};
    const unsigned ntiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    if (ev) cudaEventRecord(ev[0], st);
    if constexpr (sizeof(T) == 4 && !RECHECK) {
        if (fd.march_variant == 1 && fd.k_split > 1) {
            static std::atomic<int> g_sa{0}, g_sg{0}, g_mg{0};
            const unsigned items = ntiles * (unsigned)fd.k_split;
            if (fd.march_samples == 2) {
                static std::atomic<int> g_s4a{0}, g_s4g{0};
                if (fd.axis_slice) {
                    const int cap = num_sms * resident_per_sm(g_s4a, march4_split_kernel<SQ, MOD, true>);
                    march4_split_kernel<SQ, MOD, true>
                        <<<(int)min((unsigned)cap, (items + 3u) / 4u), kBlock, 0, st>>>(fd, sc);
                } else {
                    const int cap = num_sms * resident_per_sm(g_s4g, march4_split_kernel<SQ, MOD, false>);
                    march4_split_kernel<SQ, MOD, false>
                        <<<(int)min((unsigned)cap, (items + 3u) / 4u), kBlock, 0, st>>>(fd, sc);
                }
            } else if (fd.axis_slice) {
                const int cap = num_sms * resident_per_sm(g_sa, march2_split_kernel<SQ, MOD, true>);
                march2_split_kernel<SQ, MOD, true><<<(int)min((unsigned)cap, (items + 3u) / 4u), kBlock, 0, st>>>(fd, sc);
            } else {
                const int cap = num_sms * resident_per_sm(g_sg, march2_split_kernel<SQ, MOD, false>);
                march2_split_kernel<SQ, MOD, false><<<(int)min((unsigned)cap, (items + 3u) / 4u), kBlock, 0, st>>>(fd, sc);
            }
            const unsigned npx = (unsigned)fd.W * (unsigned)fd.H;
            const int capm = num_sms * resident_per_sm(g_mg, march_merge_kernel);
            march_merge_kernel<<<(int)min((unsigned)capm, (npx + kBlock - 1) / kBlock), kBlock, 0, st>>>(fd, sc);
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (fd.march_variant == 1 && !(fd.k_split > 1 && !RECHECK)) {
            // a persistent grid per instantiation: the axis and general forms
            // have different register counts and resident CTAs per SM
            if (fd.axis_slice && fd.march_samples == 2) {
                static std::atomic<int> g_march4a{0};
                const int cap = num_sms * resident_per_sm(g_march4a, march4_kernel<SQ, MOD, RECHECK, true>);
                const int gm = (int)min((unsigned)cap, (ntiles + 3u) / 4u);
                march4_kernel<SQ, MOD, RECHECK, true><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
            } else if (!fd.axis_slice && fd.march_samples == 2) {
                static std::atomic<int> g_march4g{0};
                const int cap = num_sms * resident_per_sm(g_march4g, march4_kernel<SQ, MOD, RECHECK, false>);
                const int gm = (int)min((unsigned)cap, (ntiles + 3u) / 4u);
                march4_kernel<SQ, MOD, RECHECK, false><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
            } else if (fd.axis_slice) {
                const int cap = num_sms * resident_per_sm(g_march2a, march2_kernel<SQ, MOD, RECHECK, true>);
                const int gm = (int)min((unsigned)cap, (ntiles + 3u) / 4u);
                march2_kernel<SQ, MOD, RECHECK, true><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
            } else {
                const int cap = num_sms * resident_per_sm(g_march2g, march2_kernel<SQ, MOD, RECHECK, false>);
                const int gm = (int)min((unsigned)cap, (ntiles + 3u) / 4u);
                march2_kernel<SQ, MOD, RECHECK, false><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
            }
        }
    }
    if (sizeof(T) != 4 || fd.march_variant != 1) {
        const int cap = num_sms * resident_per_sm(g_march, march_kernel<T, SQ, MOD, RECHECK>);
        const int gm = (int)min((unsigned)cap, (ntiles + 3u) / 4u);
        march_kernel<T, SQ, MOD, RECHECK><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
    }
    if (ev) cudaEventRecord(ev[1], st);
    const int capb = num_sms * resident_per_sm(g_bisect, bisect_kernel<T, SQ, MOD, RECHECK>);
    const unsigned maxw = ((unsigned)fd.W * (unsigned)fd.H + 31u) / 32u;
    const int gb = (int)min((unsigned)capb, (maxw + 3u) / 4u);
    bisect_kernel<T, SQ, MOD, RECHECK><<<gb > 0 ? gb : 1, kBlock, 0, st>>>(fd, sc, bisect_group_below(capb),
                                                                          bisect_group_lanes());
    if (ev) cudaEventRecord(ev[2], st);
    if (RECHECK) {
        static std::atomic<int> g_re{0}, g_fx{0};
        recheck_kernel<SQ, MOD><<<num_sms * resident_per_sm(g_re, recheck_kernel<SQ, MOD>), kBlock, 0, st>>>(fd, sc);
        if (ev) cudaEventRecord(ev[3], st);
        fixup_kernel<SQ, MOD><<<num_sms * resident_per_sm(g_fx, fixup_kernel<SQ, MOD>), kBlock, 0, st>>>(fd, sc);
        if (ev) cudaEventRecord(ev[4], st);
    } else if (ev) {
        cudaEventRecord(ev[3], st);
        cudaEventRecord(ev[4], st);
    }
    return cudaGetLastError();
}

template <int SQ, int MOD>
cudaError_t launch_mode(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    switch (fd.precision) {
    case 0: return launch_passes<float, SQ, MOD, false>(fd, sc, st, num_sms, ev);
    case 1: return launch_passes<float, SQ, MOD, true>(fd, sc, st, num_sms, ev);
    default: return launch_passes<double, SQ, MOD, false>(fd, sc, st, num_sms, ev);
    }
}

}  // namespace

int march_samples_per_round()
{
    static const int n = [] {
        const char *e = std::getenv("DQJ_MARCH_SAMPLES");
        return e && std::strtol(e, nullptr, 10) == 1 ? 1 : 2;
    }();
    return n;
}

int march_split(const FrameDesc &fd, int num_sms)
{
    static std::atomic<int> g_occ{0};
    if (fd.precision != DQJ_FP32 || fd.march_variant != 1 || fd.traversal != DQJ_TRAVERSAL_MARCH) return 1;
    if (const char *e = std::getenv("DQJ_MARCH_SPLIT")) {  // 0: never split; n > 1: n ranges
        const long n = std::strtol(e, nullptr, 10);
        if (n <= 1) return 1;
        return (int)std::min<long>(std::min<long>(n, 64), (long)fd.N + 1);
    }
    static std::atomic<int> g_occ4{0};
    const int per_sm = fd.march_samples == 2 ? resident_per_sm(g_occ4, march4_split_kernel<0, 0, true>)
                                             : resident_per_sm(g_occ, march2_split_kernel<0, 0, true>);
    const long long warps = (long long)num_sms * per_sm * (kBlock / 32);
    const long long tiles = subset_tiles(fd, (unsigned)fd.tiles_x * (unsigned)fd.tiles_y);
    if (tiles >= warps || tiles == 0) return 1;
    // about four waves of items: later waves skip the rays earlier ranges hit
    const long long p = (4 * warps + tiles - 1) / tiles;
    return (int)std::min<long long>(std::min<long long>(p, 16), (long long)fd.N + 1);
}

cudaError_t launch_frame(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    if (fd.traversal == DQJ_TRAVERSAL_DE) return launch_de(fd, sc, st, num_sms, ev);
    const int m = fd.square_mode * 2 + fd.modulus_mode;
    switch (m) {
    case 0: return launch_mode<0, 0>(fd, sc, st, num_sms, ev);
    case 1: return launch_mode<0, 1>(fd, sc, st, num_sms, ev);
    case 2: return launch_mode<1, 0>(fd, sc, st, num_sms, ev);
    default: return launch_mode<1, 1>(fd, sc, st, num_sms, ev);
    }
}

}  // namespace dqj
