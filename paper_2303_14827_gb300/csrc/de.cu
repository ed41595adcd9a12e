// de.cu -- the paper's own traversal: sphere tracing by the distance estimate
// (Method, "Ray-Marching", Eq. distfract2 with the derivative recurrence of
// Eq. distfract), and the normal + shading pass over its hits.
//
// One ray per lane over 8x4 screen tiles claimed by warps of a persistent grid.
// Every lane advances its own ray (its own t); a round samples every active
// ray once, iterating in lockstep until no lane still has a bounded sample,
// and ends when no lane is active.  The derivative is carried squared,
// |zeta'_{n+1}|^2 = 4 |zeta_n|^2 |zeta'_n|^2, so a step needs no square root;
// the estimate 0.5 |zeta| / |zeta'| ln |zeta| = 0.25 sqrt(m / dr2) ln m is
// formed once per sample from the modulus m and dr2 at the escape step, in
// FP32 with the fast reciprocal square root and logarithm.  (In FP32 dr2
// overflows only past ~21 steps, where the estimate is ~1e-15: an overflow
// gives 0, which is below any epsilon, the same decision.)
// Hits go to the hit list as (pixel, depth bits, n*); misses write their
// planes directly.
#include "render_common.cuh"
#include "runtime.h"
#include "../../include/dqj.h"

namespace dqj {

namespace {

constexpr int kDeTileW = 8, kDeTileH = 4;

// Lockstep classification with the squared derivative: returns the escape
// count (0 = inside) and, for an escaped sample, the distance estimate.  AXIS:
// only z[0..2] are set (the rest are zero) and the first step takes the axis
// form (same results).
// dm returns the smallest |modulus - R^2| of the steps tested up to and
// including the escaping one (the recheck's margin distance).
template <typename T, int SQ, int MOD, bool AXIS>
__device__ __forceinline__ int classify_de(T (&z)[8], const FrameT<T> &F, int max_iter, bool part, T &dist, T &dm)
{
    bool alive = part;
    int cnt = 0;
    dm = tinf<T>();
    T sp, m;
    if (AXIS) {
        sp = dfma(z[2], z[2], z[1] * z[1]);
        m = dfma(z[2], z[2], dfma(z[1], z[1], z[0] * z[0]));
    } else {
        sp = dq_sp<T>(z);
        m = modulus<T, MOD>(z);
    }
    T dr2 = T(4) * m, m_esc = T(0), dr2_esc = T(1);
    // the first step, peeled so that it can take the axis form
    m = AXIS ? dq_iter_axis_first<T, MOD>(z, z, sp, F.c) : dq_iter<T, SQ, MOD>(z, z, sp, F.c);
    if (alive) dm = fmin(dm, fabs(m - F.R2));
    if (alive && !(m <= F.R2)) {
        m_esc = m;
        dr2_esc = dr2;
    }
    alive = alive && (m <= F.R2);
    cnt += alive ? 1 : 0;
    if (__any_sync(kFull, alive)) {
        for (int n = 1; n < max_iter; ++n) {
            dr2 = T(4) * m * dr2;
            m = dq_iter<T, SQ, MOD>(z, z, sp, F.c);
            if (alive) dm = fmin(dm, fabs(m - F.R2));
            if (alive && !(m <= F.R2)) {
                m_esc = m;
                dr2_esc = dr2;
            }
            alive = alive && (m <= F.R2);
            cnt += alive ? 1 : 0;
            if (!__any_sync(kFull, alive)) break;
        }
    }
    // a long orbit counts as marginal (see late_step): its FP32 count may move
    // with the sample's position
    if (part && max_iter > late_step<MOD>() && cnt >= late_step<MOD>()) dm = T(0);
    if (!part || alive) {
        dist = T(0);
        return 0;
    }
    // 0.5 |zeta| / |zeta'| ln |zeta| = 0.25 sqrt(m / dr2) ln m = 0.25 m / sqrt(m dr2) ln m
    if constexpr (sizeof(T) == 4)
        dist = 0.25f * m_esc * rsqrtf(m_esc * dr2_esc) * __logf(m_esc);  // fast forms in FP32
    else
        dist = T(0.25) * sqrt(m_esc / dr2_esc) * log(m_esc);
    return cnt + 1;
}

// Sphere tracing of one ray per lane (all 32 lanes call; `valid` = the lane
// has a pixel): from the entry into the box (and the bounding sphere), sample,
// stop at an inside sample or one whose estimate is below epsilon (a hit at
// that sample), else advance by the step scale times the estimate; leaving the
// volume or running out of steps is a miss.  Returns whether the ray hit, with
// its depth, n*, the largest escape count over its samples, and its direction.
// RECHECK (FP32): the FP32 trace's ray parameter accumulates the rounding of
// every estimate, so its hit depth can differ from the FP64 trace's by more
// than the depth tolerance: every hit pixel is queued for the FP64 re-trace.
// For the others, samples whose escape test came within the margin of R^2 or
// whose estimate lies within kDeEpsBand * epsilon of epsilon are queued for the
// FP64 recheck, and a step that lands within kDeExitBand of the exit queues
// the pixel for the FP64 re-trace directly.
constexpr float kDeEpsBand = 0.02f;   // relative to epsilon
constexpr float kDeExitBand = 1e-5f;  // scene units (relative above 1)

template <typename T, int SQ, int MOD, bool AXIS, bool RECHECK>
__device__ __forceinline__ bool de_trace_lane(const FrameDesc &fd, const Scratch &sc, int x, int y, bool valid,
                                              LaneStats &st, T (&d)[3], T (&D)[8], T &depth, int &n_star,
                                              int &esc_max)
{
    const FrameT<T> &F = frame<T>(fd);
    d[0] = d[1] = T(0);
    d[2] = T(1);
    T t0 = T(0), t1 = T(0);
    bool act = valid && camera_clip<T>(F, fd.W, fd.H, x, y, d, t0, t1);
    if (act && F.de_rb > T(0)) {  // bounding sphere about the origin
        const T b = F.eye[0] * d[0] + F.eye[1] * d[1] + F.eye[2] * d[2];
        const T c = F.eye[0] * F.eye[0] + F.eye[1] * F.eye[1] + F.eye[2] * F.eye[2] - F.de_rb * F.de_rb;
        const T disc = b * b - c;
        if (disc > T(0)) {
            const T q = sqrt(disc);
            t0 = max(t0, -b - q);
            t1 = min(t1, -b + q);
            act = t0 < t1;
        } else {
            act = false;
        }
    }
    slice_dir<T>(F, d, D);
    T t = t0;
    depth = T(0);
    int steps = 0;
    esc_max = 0;
    n_star = 0;
    bool hit = false;
    const int pixel = y * fd.W + x;
    while (__any_sync(kFull, act)) {
        T z[8];
#pragma unroll
        for (int i = 0; i < (AXIS ? 3 : 8); ++i) z[i] = dfma(t, D[i], F.A[i]);  // AXIS: the rest are 0
        T dist, dm;
        const int n = classify_de<T, SQ, MOD, AXIS>(z, F, fd.max_iter, act, dist, dm);
        const bool stop = n == 0 || dist < F.de_eps;
        if (RECHECK) {
            const bool push = act && (dm <= F.margin || (n != 0 && fabs(dist - F.de_eps) <= T(kDeEpsBand) * F.de_eps));
            // {pixel, step, t bits, FP32 escape count | FP32 stop decision << 16}
            if (warp_push(push, make_int4(pixel, steps, __float_as_int((float)t), n | (stop ? 1 << 16 : 0)), sc.queue,
                          sc.queue_cap, &sc.ctr->queue_count)) {
                atomicAdd(&sc.ctr->stats[7], 1ull);
                mark_dirty(fd, sc, pixel);
            }
            st.rechecks += push ? 1 : 0;
        }
        if (act) {
            ++steps;
            st.iters += n ? (unsigned)n : (unsigned)fd.max_iter;
            if (n > esc_max) esc_max = n;
            if (stop) {
                hit = true;
                depth = t;
                n_star = n ? n : fd.max_iter;
                act = false;
            } else {
                t = t + F.de_scale * dist;
                act = steps < fd.de_max_steps && t <= t1;
                if (RECHECK && fabs(t - t1) <= T(kDeExitBand) * max(T(1), fabs(t1))) mark_dirty(fd, sc, pixel);
            }
        }
    }
    st.samples += (unsigned)steps;
    st.hits += hit ? 1 : 0;
    if (RECHECK && hit) mark_dirty(fd, sc, pixel);
    return hit;
}

template <typename T, int SQ, int MOD, bool AXIS, bool RECHECK>
__global__ void __launch_bounds__(kBlock) de_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const int lane = threadIdx.x & 31;
    const int tiles_x = (fd.W + kDeTileW - 1) / kDeTileW;
    const unsigned ntiles = subset_tiles(fd, (unsigned)tiles_x * (unsigned)((fd.H + kDeTileH - 1) / kDeTileH));
    LaneStats st;
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(&sc.ctr->tile_next, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        tile = subset_tile(fd, tile);
        const int x = (int)(tile % (unsigned)tiles_x) * kDeTileW + lane % kDeTileW;
        const int y = (int)(tile / (unsigned)tiles_x) * kDeTileH + lane / kDeTileW;
        const bool valid = x < fd.W && y < fd.H;
        T d[3], D[8], depth;
        int n_star, esc_max;
        const bool hit = de_trace_lane<T, SQ, MOD, AXIS, RECHECK>(fd, sc, x, y, valid, st, d, D, depth, n_star,
                                                                  esc_max);
        if (valid && !hit) write_miss<T>(fd, x, y, esc_max);
        int4 e = make_int4(y * fd.W + x, 0, 0, n_star);
        if constexpr (sizeof(T) == 8) {
            const long long b = __double_as_longlong((double)depth);
            e.y = (int)(unsigned)(b & 0xffffffffll);
            e.z = (int)(b >> 32);
        } else {
            e.y = __float_as_int((float)depth);
        }
        // RECHECK: hits are re-traced and shaded by de_fixup_kernel
        warp_push(hit && !RECHECK, e, sc.hits, sc.hit_cap, &sc.ctr->hit_count);
    }
    flush_lane_stats<RECHECK>(sc, st, true);
}

// FP64 recheck of the queued samples of the FP32 trace: each is classified in
// FP64 at the FP32 trace's own position (its t, exact in double) on the FP64
// ray.  The pixel is re-traced in FP64 when the escape count or the stop
// decision differs, or when the FP64 values lie close enough to a threshold
// (modulus within a tenth of the margin, estimate within half the band) that
// the FP32 trace's rounding of its positions could move the FP64 trace's
// decision.
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) de_recheck_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<double> &F = fd.d;
    const unsigned nq = min(*(volatile unsigned *)&sc.ctr->queue_count, sc.queue_cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        const int4 e = sc.queue[i];
        const int pixel = e.x;
        const int x = pixel % fd.W, y = pixel / fd.W;
        double d[3], t_in, t_out, D[8];
        camera_clip<double>(F, fd.W, fd.H, x, y, d, t_in, t_out);
        slice_dir<double>(F, d, D);
        const double t = (double)__int_as_float(e.z);
        double z[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) z[j] = fma(t, D[j], F.A[j]);
        double dist, dm;
        const int n = classify_de<double, SQ, MOD, false>(z, F, fd.max_iter, true, dist, dm);
        const bool stop = n == 0 || dist < F.de_eps;
        const bool differs = n != (e.w & 0xffff) || stop != ((e.w >> 16) != 0);
        const bool close = dm <= 0.1 * F.margin || (n != 0 && fabs(dist - F.de_eps) <= 0.5 * kDeEpsBand * F.de_eps);
        if (differs || close) mark_dirty(fd, sc, pixel);
    }
}

// FP64 re-trace of the pixels queued by the recheck, 32 per warp (one per
// lane, in lockstep like de_kernel), shaded in place.  AXIS: an axis-aligned
// slice, whose samples take the axis form of the first step (same results).
template <int SQ, int MOD, bool AXIS>
__global__ void __launch_bounds__(kBlock) de_fixup_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<double> &F = fd.d;
    const int lane = threadIdx.x & 31;
    const unsigned nd = min(*(volatile unsigned *)&sc.ctr->dirty_count, sc.dirty_cap);
    const unsigned warp = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = gridDim.x * (blockDim.x >> 5);
    LaneStats st, st_fix;
    for (unsigned base = warp * 32; base < nd; base += nwarps * 32) {
        const bool valid = base + lane < nd;
        const int pixel = valid ? sc.dirty_list[base + lane] : 0;
        const int x = pixel % fd.W, y = pixel / fd.W;
        double d[3], D[8], depth;
        int n_star, esc_max;
        const bool hit =
            de_trace_lane<double, SQ, MOD, AXIS, false>(fd, sc, x, y, valid, st_fix, d, D, depth, n_star, esc_max);
        if (valid && !hit) write_miss<double>(fd, x, y, esc_max);
        normal_shade<double, SQ, MOD>(fd, F, x, y, d, D, depth, n_star, hit, st_fix);
        st.hits += valid ? 1 : 0;
    }
    flush_stat(&sc.ctr->stats[5], st.hits);
    flush_stat(&sc.ctr->stats[6], st_fix.iters + st_fix.niters);
}

template <typename T, int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) de_shade_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<T> &F = frame<T>(fd);
    const int lane = threadIdx.x & 31;
    const unsigned nhits = min(*(volatile unsigned *)&sc.ctr->hit_count, sc.hit_cap);
    LaneStats st;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&sc.ctr->hit_next, 32u);
        base = __shfl_sync(kFull, base, 0);
        if (base >= nhits) break;
        const unsigned idx = base + lane;
        const bool part = idx < nhits;
        int4 e = make_int4(0, 0, 0, 0);
        if (part) e = __ldcg(sc.hits + idx);
        const int x = e.x % fd.W, y = e.x / fd.W;
        T depth;
        if constexpr (sizeof(T) == 8)
            depth = __longlong_as_double(((long long)e.z << 32) | (long long)(unsigned)e.y);
        else
            depth = __int_as_float(e.y);
        T d[3] = {T(0), T(0), T(1)};
        T t_in, t_out;
        if (part) camera_clip<T>(F, fd.W, fd.H, x, y, d, t_in, t_out);
        T D[8];
        slice_dir<T>(F, d, D);
        normal_shade<T, SQ, MOD>(fd, F, x, y, d, D, part ? depth : T(0), e.w, part, st);
    }
    flush_stat(&sc.ctr->stats[1], st.niters);
}

template <typename T, int SQ, int MOD, bool RECHECK>
cudaError_t launch_de_t(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    static std::atomic<int> g_de{0}, g_sh{0};
    const int cap_de = num_sms * resident_per_sm(g_de, de_kernel<T, SQ, MOD, false, RECHECK>);
    const int cap_sh = num_sms * resident_per_sm(g_sh, de_shade_kernel<T, SQ, MOD>);
    const unsigned ntiles =
        subset_tiles(fd, (unsigned)((fd.W + kDeTileW - 1) / kDeTileW) * (unsigned)((fd.H + kDeTileH - 1) / kDeTileH));
    const int gd = (int)min((unsigned)cap_de, (ntiles + 3u) / 4u);
    const unsigned maxw = ((unsigned)fd.W * (unsigned)fd.H + 31u) / 32u;
    const int gs = (int)min((unsigned)cap_sh, (maxw + 3u) / 4u);
    if (ev) cudaEventRecord(ev[0], st);
    if (fd.axis_slice)
        de_kernel<T, SQ, MOD, true, RECHECK><<<gd > 0 ? gd : 1, kBlock, 0, st>>>(fd, sc);
    else
        de_kernel<T, SQ, MOD, false, RECHECK><<<gd > 0 ? gd : 1, kBlock, 0, st>>>(fd, sc);
    if (ev) cudaEventRecord(ev[1], st);
    de_shade_kernel<T, SQ, MOD><<<gs > 0 ? gs : 1, kBlock, 0, st>>>(fd, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if constexpr (RECHECK) {
        static std::atomic<int> g_re{0}, g_fx{0}, g_fxg{0};
        de_recheck_kernel<SQ, MOD><<<num_sms * resident_per_sm(g_re, de_recheck_kernel<SQ, MOD>), kBlock, 0, st>>>(
            fd, sc);
        if (ev) cudaEventRecord(ev[3], st);
        if (fd.axis_slice)
            de_fixup_kernel<SQ, MOD, true>
                <<<num_sms * resident_per_sm(g_fx, de_fixup_kernel<SQ, MOD, true>), kBlock, 0, st>>>(fd, sc);
        else
            de_fixup_kernel<SQ, MOD, false>
                <<<num_sms * resident_per_sm(g_fxg, de_fixup_kernel<SQ, MOD, false>), kBlock, 0, st>>>(fd, sc);
        if (ev) cudaEventRecord(ev[4], st);
    } else if (ev) {
        cudaEventRecord(ev[3], st);
        cudaEventRecord(ev[4], st);
    }
    return cudaGetLastError();
}

template <int SQ, int MOD>
cudaError_t launch_de_m(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    switch (fd.precision) {
    case DQJ_FP64: return launch_de_t<double, SQ, MOD, false>(fd, sc, st, num_sms, ev);
    case DQJ_FP32_RECHECK: return launch_de_t<float, SQ, MOD, true>(fd, sc, st, num_sms, ev);
    default: return launch_de_t<float, SQ, MOD, false>(fd, sc, st, num_sms, ev);
    }
}

}  // namespace

cudaError_t launch_de(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    switch (fd.square_mode * 2 + fd.modulus_mode) {
    case 0: return launch_de_m<0, 0>(fd, sc, st, num_sms, ev);
    case 1: return launch_de_m<0, 1>(fd, sc, st, num_sms, ev);
    case 2: return launch_de_m<1, 0>(fd, sc, st, num_sms, ev);
    default: return launch_de_m<1, 1>(fd, sc, st, num_sms, ev);
    }
}

}  // namespace dqj
