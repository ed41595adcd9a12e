// render_common.cuh -- device helpers shared by the render kernels and the
// persistent serving kernel: camera ray and box clip, slice map, warp-aggregated
// queue pushes, output writes and shading, and the per-tile bodies of the march
// and bisection passes.
#pragma once

#include <atomic>

#include "dq_math.cuh"

namespace dqj {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 128;  // 4 warps per CTA

// Resident CTAs of `kernel` per SM at `block` threads, cached in `slot` (one slot
// per kernel instantiation).  The count depends on the kernel's registers and
// shared memory only, so it holds for every device of this single-architecture
// build; callers multiply it by the launching device's SM count.  Threads that
// race on an empty slot compute and store the same value.
template <typename K>
inline int resident_per_sm(std::atomic<int> &slot, K kernel, int block = kBlock)
{
    int v = slot.load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, block, 0) != cudaSuccess || v < 1) {
        cudaGetLastError();
        return 1;
    }
    slot.store(v, std::memory_order_relaxed);
    return v;
}

// The frame's tile subset (dqj_render_tiles): the number of its tiles out of
// ntiles, and the tile index of the subset's i-th tile.
__host__ __device__ __forceinline__ unsigned subset_tiles(const FrameDesc &fd, unsigned ntiles)
{
    const unsigned part = (unsigned)fd.tile_part, parts = (unsigned)fd.tile_parts;
    return part < ntiles ? (ntiles - part + parts - 1) / parts : 0u;
}
__device__ __forceinline__ unsigned subset_tile(const FrameDesc &fd, unsigned i)
{
    return i * (unsigned)fd.tile_parts + (unsigned)fd.tile_part;
}

// Per-lane counters, added to the frame's stats once per warp (DQJ_STAT_*).
struct LaneStats {
    unsigned long long iters = 0, samples = 0, hits = 0, rechecks = 0, niters = 0;
};


template <typename T>
__device__ __forceinline__ const FrameT<T> &frame(const FrameDesc &fd);
template <>
__device__ __forceinline__ const FrameT<float> &frame<float>(const FrameDesc &fd) { return fd.f; }
template <>
__device__ __forceinline__ const FrameT<double> &frame<double>(const FrameDesc &fd) { return fd.d; }

template <typename T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ float tinf<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double tinf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

// Pinhole camera ray through pixel centre (x + 0.5, y + 0.5), row 0 at the top,
// and its slab clip against the box, t >= 0.  Returns false when the ray misses
// the box (t_in >= t_out).  The FP64 form follows the reference formula term by
// term; the FP32 form folds the pixel-to-screen map into one FMA per axis.
template <typename T>
__device__ __forceinline__ bool camera_clip(const FrameT<T> &F, int W, int H, int x, int y, T (&d)[3], T &t_in,
                                            T &t_out)
{
    T sx, sy;
    if constexpr (sizeof(T) == 4) {
        sx = dfma(T(x) + T(0.5), F.sxa, F.sxb);
        sy = dfma(T(y) + T(0.5), F.sya, F.syb);
    } else {
        sx = (T(2) * (T(x) + T(0.5)) / T(W) - T(1)) * F.th * F.aspect;
        sy = (T(1) - T(2) * (T(y) + T(0.5)) / T(H)) * F.th;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = F.fwd[a] + sx * F.right[a] + sy * F.upv[a];
    const T len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = d[a] / len;
    T t0 = -tinf<T>(), t1 = tinf<T>();
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == T(0)) {
            if (F.eye[a] < F.bmin[a] || F.eye[a] > F.bmax[a]) ok = false;
        } else {
            T ta = (F.bmin[a] - F.eye[a]) / d[a];
            T tb = (F.bmax[a] - F.eye[a]) / d[a];
            if (ta > tb) {
                const T tmp = ta;
                ta = tb;
                tb = tmp;
            }
            t0 = ta > t0 ? ta : t0;
            t1 = tb < t1 ? tb : t1;
        }
    }
    if (t0 < T(0)) t0 = T(0);
    t_in = t0;
    t_out = t1;
    return ok && (t0 < t1);
}

// FP64 camera ray and box clip for the recheck of a queued sample: the
// quantities of camera_clip<double> with the pixel-to-screen map folded into one
// FMA per axis and reciprocals in place of divisions (far fewer FP64
// instructions; FP64 runs at 1/64 of the FP32 rate).  Each value may differ from the reference formula's in the
// last place, as the FP64 iteration's contracted FMAs already do: far below
// what moves a recheck decision, which is taken against a margin of 1e-3
// relative.
__device__ __forceinline__ bool camera_clip_rcp(const FrameT<double> &F, int x, int y, double (&d)[3],
                                                double &t_in, double &t_out)
{
    const double sx = fma(double(x) + 0.5, F.sxa, F.sxb);
    const double sy = fma(double(y) + 0.5, F.sya, F.syb);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = F.fwd[a] + sx * F.right[a] + sy * F.upv[a];
    const double il = rsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = d[a] * il;
    double t0 = -tinf<double>(), t1 = tinf<double>();
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (F.eye[a] < F.bmin[a] || F.eye[a] > F.bmax[a]) ok = false;
        } else {
            const double inv = __drcp_rn(d[a]);
            double ta = (F.bmin[a] - F.eye[a]) * inv;
            double tb = (F.bmax[a] - F.eye[a]) * inv;
            if (ta > tb) {
                const double tmp = ta;
                ta = tb;
                tb = tmp;
            }
            t0 = ta > t0 ? ta : t0;
            t1 = tb < t1 ? tb : t1;
        }
    }
    if (t0 < 0.0) t0 = 0.0;
    t_in = t0;
    t_out = t1;
    return ok && (t0 < t1);
}

// D = E d: direction of the ray in the 8-D slice.
template <typename T>
__device__ __forceinline__ void slice_dir(const FrameT<T> &F, const T (&d)[3], T (&D)[8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) D[i] = dfma(d[0], F.E[0][i], dfma(d[1], F.E[1][i], d[2] * F.E[2][i]));
}

// Warp-aggregated append of one int4 per flagged lane.  All lanes must call.
// Returns true on the lanes whose entry did not fit (the caller falls back).
__device__ __forceinline__ bool warp_push(bool flag, int4 v, int4 *buf, unsigned cap, unsigned *count)
{
    const unsigned m = __ballot_sync(kFull, flag);
    if (m == 0) return false;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!flag) return false;
    const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
    if (slot < cap) {
        buf[slot] = v;
        return false;
    }
    return true;
}

// Queue a pixel for an FP64 re-render once per frame.
__device__ __forceinline__ void mark_dirty(const FrameDesc &fd, const Scratch &sc, int pixel)
{
    const uint32_t old = atomicExch(&sc.dirty_flag[pixel], fd.epoch);
    if (old != fd.epoch) {
        const unsigned slot = atomicAdd(&sc.ctr->dirty_count, 1u);
        if (slot < sc.dirty_cap) sc.dirty_list[slot] = pixel;
    }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void flush_stat(unsigned long long *dst, unsigned long long v)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

template <typename T>
__device__ __forceinline__ void write_miss(const FrameDesc &fd, int x, int y, int iter)
{
    const int64_t o = (int64_t)y * fd.pitch + x;
    if (fd.iter) fd.iter[o] = iter;
    if (fd.depth) fd.depth[o] = tinf<float>();
    if (fd.normal) {
        fd.normal[3 * o + 0] = 0.f;
        fd.normal[3 * o + 1] = 0.f;
        fd.normal[3 * o + 2] = 0.f;
    }
    if (fd.rgba) *reinterpret_cast<uchar4 *>(fd.rgba + 4 * o) = make_uchar4(0, 0, 0, 0);
}

__device__ __forceinline__ unsigned char to_u8(double v)
{
    double x = floor(255.0 * v + 0.5);
    x = x < 0.0 ? 0.0 : (x > 255.0 ? 255.0 : x);
    return (unsigned char)x;
}
__device__ __forceinline__ unsigned char to_u8(float v)
{
    float x = floorf(255.f * v + 0.5f);
    x = x < 0.f ? 0.f : (x > 255.f ? 255.f : x);
    return (unsigned char)x;
}

// Largest normal-field value used for a gradient, 2^100 (exact in float and
// double): larger or non-finite field values select the fallback normal -d.
__device__ __forceinline__ float normal_fmax(float) { return 1.2676506002282294e30f; }
__device__ __forceinline__ double normal_fmax(double) { return 1.2676506002282294e30; }

// Normalise the central-difference gradient (fallback -d when guard is set or
// the gradient vanishes), shade with the ambient and diffuse terms of Eq. phong
// and write a hit pixel.  The gradient is scaled by its largest component first
// so that its squared length cannot overflow.
template <typename T>
__device__ __forceinline__ void shade_write(const FrameDesc &fd, const FrameT<T> &F, int x, int y, int iter,
                                            T depth, const T (&g)[3], bool guard, const T (&d)[3])
{
    T n[3];
    const T s = fmax(fabs(g[0]), fmax(fabs(g[1]), fabs(g[2])));
    if (guard || !(s > T(0))) {
        n[0] = -d[0];
        n[1] = -d[1];
        n[2] = -d[2];
    } else {
        const T g0 = g[0] / s, g1 = g[1] / s, g2 = g[2] / s;
        const T gl = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
        n[0] = g0 / gl;
        n[1] = g1 / gl;
        n[2] = g2 / gl;
    }
    T ndl = n[0] * F.light[0] + n[1] * F.light[1] + n[2] * F.light[2];
    T spec = T(0);
    if (F.ks > T(0) && ndl > T(0)) {  // reflected light r = 2n(n.l) - l against v = -d
        const T rv = -((T(2) * ndl * n[0] - F.light[0]) * d[0] + (T(2) * ndl * n[1] - F.light[1]) * d[1] +
                       (T(2) * ndl * n[2] - F.light[2]) * d[2]);
        if (rv > T(0)) spec = F.ks * pow(rv, F.shin);
    }
    ndl = ndl > T(0) ? ndl : T(0);
    T v = F.ka + F.kd * ndl + spec;
    v = v < T(0) ? T(0) : (v > T(1) ? T(1) : v);
    const int64_t o = (int64_t)y * fd.pitch + x;
    if (fd.iter) fd.iter[o] = iter;
    if (fd.depth) fd.depth[o] = (float)depth;
    if (fd.normal) {
        fd.normal[3 * o + 0] = (float)n[0];
        fd.normal[3 * o + 1] = (float)n[1];
        fd.normal[3 * o + 2] = (float)n[2];
    }
    if (fd.rgba)
        *reinterpret_cast<uchar4 *>(fd.rgba + 4 * o) =
            make_uchar4(to_u8(v * F.albedo[0]), to_u8(v * F.albedo[1]), to_u8(v * F.albedo[2]), 255);
}

// FP64 recheck of one queued sample {pixel, k | b << 16, path, n32}: the sample
// is recomputed from the FP64 camera ray with the oracle's formulas (a march
// sample t_in + k delta, or bisection level b of the bracket (k - 1, k) replayed
// from the path bits), classified in FP64, and the pixel is queued for an FP64
// re-render when its FP64 escape count differs from the FP32 one.
template <int SQ, int MOD>
__device__ __forceinline__ void recheck_entry(const FrameDesc &fd, const Scratch &sc, int4 e)
{
    const FrameT<double> &F = fd.d;
    const int pixel = e.x, k = e.y & 0xffff, b = e.y >> 16;
    const int x = pixel % fd.W, y = pixel / fd.W;
    double d[3], t_in, t_out;
    camera_clip_rcp(F, x, y, d, t_in, t_out);
    const double delta = (t_out - t_in) / (double)fd.N;
    double t;
    if (b == kMarchSample) {
        t = t_in + (double)k * delta;
    } else {
        double lo = t_in + (double)(k - 1) * delta, hi = t_in + (double)k * delta;
        for (int l = 0; l < b; ++l) {
            const double mid = lo + 0.5 * (hi - lo);
            if ((unsigned)e.z >> l & 1u)
                lo = mid;
            else
                hi = mid;
        }
        t = lo + 0.5 * (hi - lo);
    }
    double z[8];
    int n64;
    if (fd.axis_slice) {
        // components 3..7 of the slice point are zero (the general sum below
        // gives +-0 there), so the first step takes the axis form, whose
        // operations are those of dq_iter on those zeros: the same iterate
#pragma unroll
        for (int j = 0; j < 3; ++j)
            z[j] = F.O[j] + (F.eye[0] + t * d[0]) * F.E[0][j] + (F.eye[1] + t * d[1]) * F.E[1][j] +
                   (F.eye[2] + t * d[2]) * F.E[2][j];
#pragma unroll
        for (int j = 3; j < 8; ++j) z[j] = 0.0;
        n64 = classify_scalar_axis<double, SQ, MOD>(z, F, fd.max_iter);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            z[j] = F.O[j] + (F.eye[0] + t * d[0]) * F.E[0][j] + (F.eye[1] + t * d[1]) * F.E[1][j] +
                   (F.eye[2] + t * d[2]) * F.E[2][j];
        n64 = classify_scalar<double, SQ, MOD>(z, F, fd.max_iter);
    }
    if (n64 != e.w) mark_dirty(fd, sc, pixel);
}

// Re-render of one pixel by one warp (all 32 lanes call), with the oracle's
// formulas for the sample positions (the reference sequence of steps) in FP64;
// a march or bisection sample is classified in FP32 and again in FP64 only
// when it is marginal (the premise of the recheck mode); the bisection runs
// five levels per round across the lanes; the normal is FP64.  The lanes classify 32 consecutive march samples at a time; a ballot
// finds the first inside one and warp reductions give the largest escape count
// before it, so the result and the iteration count are those of the
// sample-by-sample loop.  Bisection runs on every lane alike; the six normal
// evaluations run on lanes 0..5.  Adds the iterations to its (per lane) and the
// pixel to npx (lane 0).
template <int SQ, int MOD>
__device__ __forceinline__ void fixup_pixel(const FrameDesc &fd, int pixel, unsigned long long &its,
                                            unsigned long long &npx)
{
    const FrameT<double> &F = fd.d;
    const int lane = threadIdx.x & 31;
    do {
        const int x = pixel % fd.W, y = pixel / fd.W;
        npx += lane == 0 ? 1 : 0;
        double d[3], t_in, t_out;
        if (!camera_clip<double>(F, fd.W, fd.H, x, y, d, t_in, t_out)) {
            if (lane == 0) write_miss<double>(fd, x, y, 0);
            break;
        }
        const double delta = (t_out - t_in) / (double)fd.N;
        auto slice = [&](double t, double (&z)[8]) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                z[j] = F.O[j] + (F.eye[0] + t * d[0]) * F.E[0][j] + (F.eye[1] + t * d[1]) * F.E[1][j] +
                       (F.eye[2] + t * d[2]) * F.E[2][j];
        };
        // FP64 classification; an axis-aligned slice takes the axis form of the
        // first step (the same iterate, see classify_scalar_axis)
        auto cls64 = [&](double (&z)[8]) {
            return fd.axis_slice ? classify_scalar_axis<double, SQ, MOD>(z, F, fd.max_iter)
                                 : classify_scalar<double, SQ, MOD>(z, F, fd.max_iter);
        };
        // a march sample: FP32 first, FP64 only when some FP32 modulus came within
        // the recheck margin of R^2 (the premise of the recheck mode: outside the
        // margin FP32 decides as FP64 does)
        auto cls_march = [&](double t) {
            double z[8];
            slice(t, z);
            float zf[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) zf[j] = (float)z[j];
            bool marginal;
            const int n32 = classify_scalar_margin<float, SQ, MOD>(zf, fd.f, fd.max_iter, marginal);
            return marginal ? cls64(z) : n32;
        };
        int esc_max = 0, n_prev = 0, k_first = -1;
        for (int k0 = 0; k0 <= fd.N; k0 += 32) {
            const int k = k0 + lane;
            const bool part = k <= fd.N;
            const int n = part ? cls_march(t_in + (double)k * delta) : 1;
            const unsigned inside = __ballot_sync(kFull, part && n == 0);
            const int first = inside ? __ffs(inside) - 1 : 32;  // samples before it escaped
            if (part && lane <= first) its += n ? (unsigned)n : (unsigned)fd.max_iter;
            int m = part && lane < first ? n : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
            esc_max = max(esc_max, m);
            if (inside) {
                if (first > 0) n_prev = __shfl_sync(kFull, n, first - 1);  // else: last of the previous chunk
                k_first = k0 + first;
                break;
            }
            n_prev = __shfl_sync(kFull, n, 31);
        }
        if (k_first < 0) {
            if (lane == 0) write_miss<double>(fd, x, y, esc_max);
            break;
        }
        double depth = t_in;
        int n_star = fd.max_iter;
        if (k_first > 0) {
            double lo = t_in + (double)(k_first - 1) * delta, hi = t_in + (double)k_first * delta;
            n_star = n_prev;
            // Bisection, up to five levels per round: lane j - 1 holds node j of the
            // level tree (node 1 the next midpoint, children 2j: inside -> [lo, mid],
            // 2j + 1: outside -> [mid, hi]), derives its interval with the same
            // operations as the sequential halvings and classifies its midpoint
            // (FP32 first, FP64 when marginal, as the march samples); the path is
            // then replayed, so the bracket is the sequential one.
            for (int b0 = 0; b0 < fd.B; b0 += 5) {
                const int levels = min(5, fd.B - b0);
                const int node = lane + 1;
                const int depth_j = 31 - __clz(node);  // level of the node
                int n = 1;
                if (depth_j < levels) {
                    double l = lo, h = hi;
                    for (int q = depth_j - 1; q >= 0; --q) {  // path bits below the leading one
                        const double mid = l + 0.5 * (h - l);
                        if ((node >> q) & 1)
                            l = mid;
                        else
                            h = mid;
                    }
                    n = cls_march(l + 0.5 * (h - l));
                }
                int cur = 1;
                for (int q = 0; q < levels; ++q) {
                    const int nq = __shfl_sync(kFull, n, cur - 1);
                    const double mid = lo + 0.5 * (hi - lo);
                    if (lane == 0) its += nq ? (unsigned)nq : (unsigned)fd.max_iter;
                    if (nq == 0) {
                        hi = mid;
                        cur = 2 * cur;
                    } else {
                        lo = mid;
                        n_star = nq;
                        cur = 2 * cur + 1;
                    }
                }
            }
            depth = lo + 0.5 * (hi - lo);
        }
        // normal: lane 2a + s evaluates F at p +- h e_a
        double fv = 0.0;
        if (lane < 6) {
            const int a = lane >> 1;
            double p[3] = {F.eye[0] + depth * d[0], F.eye[1] + depth * d[1], F.eye[2] + depth * d[2]};
            p[a] += (lane & 1) == 0 ? F.h : -F.h;
            double z[8];
            for (int j = 0; j < 8; ++j) z[j] = F.O[j] + p[0] * F.E[0][j] + p[1] * F.E[1][j] + p[2] * F.E[2][j];
            double sp = dq_sp<double>(z);
            for (int n = 0; n < n_star; ++n) dq_iter<double, SQ, MOD>(z, z, sp, F.c);
            its += (unsigned)n_star;
            fv = modulus<double, MOD>(z);
        }
        const bool bad = lane < 6 && !(fv <= normal_fmax(0.0));
        const bool guard = __any_sync(kFull, bad);
        double g[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) g[a] = __shfl_sync(kFull, fv, 2 * a) - __shfl_sync(kFull, fv, 2 * a + 1);
        if (lane == 0) shade_write<double>(fd, F, x, y, n_star, depth, g, guard, d);
    } while (false);
}

// Device clock in nanoseconds, for the time limits of bounded waits.
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Recheck entries of one warp are staged in shared memory.  At the end of its
// tile the warp rechecks them itself in FP64 (recheck_staged): that FP64 work
// overlaps with the FP32 march of the other warps on the SM instead of running
// as a pass of its own after the march.  A tile that fills the stage
// (kQStage entries per warp; a round adds at most 64) appends the staged
// entries to the frame's queue instead, in one block (one atomic), for the
// recheck pass.
constexpr int kQStage = 256;
// Ray parameter of a half without a sample in the recheck march: its first
// iterate overflows (modulus +inf) and the later ones are infinite or NaN, so
// its distance from R^2 never falls within a recheck band.
constexpr float kFarT = 1e18f;

// Append a warp's staged entries qs[0, qn) to the recheck queue (qn warp-uniform)
// and count them as rechecks; entries beyond the queue's capacity re-render
// their pixel in FP64.
__device__ __forceinline__ void flush_staged(const FrameDesc &fd, const Scratch &sc, const int4 *qs, int qn)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    unsigned base = 0;
    if (lane == 0) {
        base = atomicAdd(&sc.ctr->queue_count, (unsigned)qn);
        atomicAdd(&sc.ctr->stats[4], (unsigned long long)qn);
    }
    base = __shfl_sync(kFull, base, 0);
    for (int i = lane; i < qn; i += 32) {
        const int4 e = qs[i];
        if (base + (unsigned)i < sc.queue_cap) {
            sc.queue[base + i] = e;
        } else {
            atomicAdd(&sc.ctr->stats[7], 1ull);
            mark_dirty(fd, sc, e.x);
        }
    }
    __syncwarp();
}

// FP64 recheck of a warp's staged entries qs[0, qn) (qn warp-uniform), one per
// lane, counted as rechecks.
template <int SQ, int MOD>
__device__ __forceinline__ void recheck_staged(const FrameDesc &fd, const Scratch &sc, const int4 *qs, int qn)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane == 0) atomicAdd(&sc.ctr->stats[4], (unsigned long long)qn);
    for (int i = lane; i < qn; i += 32) recheck_entry<SQ, MOD>(fd, sc, qs[i]);
    __syncwarp();
}

// One 64-ray tile of the paired march (see march2_kernel); all 32 lanes call.
// A lane holds tile slots `lane` and `lane + 32`.  RECHECK: qs is the warp's
// staging buffer of kQStage entries in shared memory, rechecked at the end of
// the tile.  SPLIT: only samples
// [kb, ke) of each ray, with the range's partial result written to sc.part
// (range r = kb / fd.k_chunk) for march_merge_kernel instead of the outputs;
// a ray for which a lower range has already found an inside sample is
// skipped (the merge stops at that range), and a range that finds one records
// itself in sc.part_hit.
template <int SQ, int MOD, bool RECHECK, bool AXIS = false, bool SPLIT = false>
__device__ __forceinline__ void march2_tile(const FrameDesc &fd, const PairConsts &P, const Scratch &sc, unsigned tile,
                                            LaneStats &st, int4 *qs = nullptr, int kb = 0, int ke = 0)
{
    const FrameT<float> &F = fd.f;
    const int lane = threadIdx.x & 31;
    const int N = fd.N, max_iter = fd.max_iter;
    const int tx = (int)(tile % (unsigned)fd.tiles_x), ty = (int)(tile / (unsigned)fd.tiles_x);
    // pixel of tile slot s; formed again at the end of the tile rather than kept
    // live across the march loop (the recheck mode keeps the linear indices)
    auto px = [&](int slot) { return tx * fd.tile_w + slot % fd.tile_w; };
    auto py = [&](int slot) { return ty * fd.tile_h + slot / fd.tile_w; };
    int pixa = 0, pixb = 0;
    bool acta, actb, skipa = false, skipb = false;
    // Axis-aligned slice: zeta_0 = A + t D (components 0..2).  Otherwise the
    // first-iterate form (first_iterate_coeffs): zeta_1 = Q0 + s (Q1 + s Q2),
    // s = t + dot, with Q0 kept in D and t + dot in tin.
    float2 D[8], tin, dl;
    float2 Q1[AXIS ? 1 : 8], Q2[AXIS ? 1 : 8];
    {
        const int xa = px(lane), ya = py(lane), xb = px(lane + 32), yb = py(lane + 32);
        if (RECHECK) {
            pixa = ya * fd.W + xa;
            pixb = yb * fd.W + xb;
        }
        const bool va = xa < fd.W && ya < fd.H, vb = xb < fd.W && yb < fd.H;
        float da[3] = {0.f, 0.f, 1.f}, db[3] = {0.f, 0.f, 1.f};
        float tia = 0.f, toa = 0.f, tib = 0.f, tob = 0.f;
        acta = va && camera_clip<float>(F, fd.W, fd.H, xa, ya, da, tia, toa);
        actb = vb && camera_clip<float>(F, fd.W, fd.H, xb, yb, db, tib, tob);
        if constexpr (SPLIT) {
            const unsigned r = (unsigned)(kb / fd.k_chunk);
            skipa = va && __ldcg(sc.part_hit + ya * fd.W + xa) < r;
            skipb = vb && __ldcg(sc.part_hit + yb * fd.W + xb) < r;
            acta = acta && !skipa;
            actb = actb && !skipb;
        }
        if (!acta) tia = toa = 0.f;
        if (!actb) tib = tob = 0.f;
        dl = make_float2((toa - tia) / (float)N, (tob - tib) / (float)N);
        if (RECHECK) {  // a half without a ray samples far away: never within the recheck band
            if (!acta) tia = kFarT;
            if (!actb) tib = kFarT;
        }
        float Da[8], Db[8];
        slice_dir<float>(F, da, Da);
        slice_dir<float>(F, db, Db);
#pragma unroll
        for (int i = 0; i < 8; ++i) D[i] = make_float2(Da[i], Db[i]);
        tin = make_float2(tia, tib);
        if constexpr (!AXIS) {
            // each ray's coefficients by the scalar code of march_kernel and
            // bisect_chunk (same operations, so the same values), then paired
            float Qa[3][8], Qb[3][8], dota, dotb;
            first_iterate_coeffs<float, SQ>(F.A, Da, F.c, dota, Qa[0], Qa[1], Qa[2]);
            first_iterate_coeffs<float, SQ>(F.A, Db, F.c, dotb, Qb[0], Qb[1], Qb[2]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                D[i] = make_float2(Qa[0][i], Qb[0][i]);
                Q1[i] = make_float2(Qa[1][i], Qb[1][i]);
                Q2[i] = make_float2(Qa[2][i], Qb[2][i]);
            }
            tin = make_float2(vadd(tia, dota), vadd(tib, dotb));
        }
    }
    const bool boxa = acta, boxb = actb;
    int suma = 0, sumb = 0, maxa = 0, maxb = 0, kfa = -1, kfb = -1;
    int qn = 0;  // staged recheck entries (warp-uniform)
    const int k0 = SPLIT ? kb : 0, k1 = SPLIT ? ke : N + 1;
    float2 kf = make_float2((float)k0, (float)k0);
    // `more`: some ray of the warp still marches.  It changes only in a round
    // that found a ray inside, so it is voted on only then.
    bool more = __any_sync(kFull, acta || actb);
    for (int k = k0; k < k1 && more; ++k) {
        const float2 t = f2fma(kf, dl, tin);
        kf = f2add(kf, make_float2(1.f, 1.f));
        float2 z[8];
        bool ina = acta, inb = actb, live;
        int ca, cb;
        float2 dm;
        if constexpr (AXIS) {
#pragma unroll
            for (int i = 0; i < 3; ++i) z[i] = f2fma(t, D[i], P.A[i]);  // the rest are 0
            classify_lockstep2<SQ, MOD, RECHECK, true>(z, P, F.R2, max_iter, ina, inb, ca, cb, dm, live);
        } else {
            first_iterate<float2, 8>(t, D, Q1, Q2, z);
            classify_lockstep2_it1<SQ, MOD, RECHECK>(z, P, F.R2, max_iter, ina, inb, ca, cb, dm, live);
        }
        if (RECHECK && __any_sync(kFull, fminf(dm.x, dm.y) <= P.margin_t)) {
            // a marginal sample in this round (rare): stage it
            const bool pa = acta && dm.x <= P.margin_t, pb = actb && dm.y <= P.margin_t;
            const unsigned ba = __ballot_sync(kFull, pa), bb = __ballot_sync(kFull, pb);
            const unsigned below = (1u << lane) - 1u;
            const int nqa = __popc(ba), nq = nqa + __popc(bb);
            if (pa) qs[qn + __popc(ba & below)] = make_int4(pixa, k | (kMarchSample << 16), 0, ina ? 0 : ca + 1);
            if (pb) qs[qn + nqa + __popc(bb & below)] = make_int4(pixb, k | (kMarchSample << 16), 0, inb ? 0 : cb + 1);
            qn += nq;
            if (qn > kQStage - 64) {
                flush_staged(fd, sc, qs, qn);
                qn = 0;
            }
        }
        // ina / inb imply acta / actb (they start equal and only clear)
        suma += ca;
        sumb += cb;
        maxa = max(maxa, ca);
        maxb = max(maxb, cb);
        if (live) {  // some half stayed bounded: those rays are inside at sample k
            if (ina) kfa = k;
            if (inb) kfb = k;
            if (RECHECK) {  // a finished ray samples far away from now on (see above)
                if (ina) tin.x = kFarT;
                if (inb) tin.y = kFarT;
            }
            acta = acta && !ina;
            actb = actb && !inb;
            more = __any_sync(kFull, acta || actb);
        }
    }
    if (RECHECK && qn > 0) recheck_staged<SQ, MOD>(fd, sc, qs, qn);
    const bool hita = kfa >= 0, hitb = kfb >= 0;
    // iterations = sum of (escape count) over escaped samples + max_iter per inside sample
    //            = sum of bounded steps + number of escaped samples
    const int nesca = (hita ? kfa : k1) - k0, nescb = (hitb ? kfb : k1) - k0;
    if constexpr (SPLIT) {  // this range's partial result per ray (see march_merge_kernel)
        const int xa = px(lane), ya = py(lane), xb = px(lane + 32), yb = py(lane + 32);
        const unsigned r = (unsigned)(kb / fd.k_chunk);
        const int64_t npx = (int64_t)fd.W * fd.H, base = (int64_t)r * npx;
        if (xa < fd.W && ya < fd.H && !skipa) {
            const int pa = ya * fd.W + xa;
            sc.part[base + pa] = boxa ? make_int4(kfa, suma + nesca, maxa + 1, nesca + (hita ? 1 : 0))
                                      : make_int4(-1, 0, 0, 0);
            if (hita) atomicMin(sc.part_hit + pa, r);
        }
        if (xb < fd.W && yb < fd.H && !skipb) {
            const int pb = yb * fd.W + xb;
            sc.part[base + pb] = boxb ? make_int4(kfb, sumb + nescb, maxb + 1, nescb + (hitb ? 1 : 0))
                                      : make_int4(-1, 0, 0, 0);
            if (hitb) atomicMin(sc.part_hit + pb, r);
        }
        return;
    }
    st.iters += (boxa ? suma + nesca : 0) + (boxb ? sumb + nescb : 0);
    st.samples += (boxa ? nesca + (hita ? 1 : 0) : 0) + (boxb ? nescb + (hitb ? 1 : 0) : 0);
    st.hits += (hita ? 1 : 0) + (hitb ? 1 : 0);
    const int xa = px(lane), ya = py(lane), xb = px(lane + 32), yb = py(lane + 32);
    const bool va = xa < fd.W && ya < fd.H, vb = xb < fd.W && yb < fd.H;
    if (va && !hita) write_miss<float>(fd, xa, ya, boxa ? maxa + 1 : 0);
    if (vb && !hitb) write_miss<float>(fd, xb, yb, boxb ? maxb + 1 : 0);
    warp_push(hita, make_int4(ya * fd.W + xa, kfa, 0, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
    warp_push(hitb, make_int4(yb * fd.W + xb, kfb, 0, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
}

// march2_tile with two samples of each ray per round (samples k and k + 1,
// classify_lockstep4_axis / classify_lockstep4_it1): the same per-sample
// arithmetic, so the same results, iteration counts and recheck entries.  A
// sample k + 1 after an inside sample k is classified but not counted or
// staged, as the one-sample march never reaches it.  SPLIT: samples [kb, ke)
// of each ray with the range's partial result, as in march2_tile.
template <int SQ, int MOD, bool RECHECK, bool AXIS = true, bool SPLIT = false>
__device__ __forceinline__ void march4_tile(const FrameDesc &fd, const PairConsts &P, const Scratch &sc, unsigned tile,
                                            LaneStats &st, int4 *qs = nullptr, int kb = 0, int ke = 0)
{
    const FrameT<float> &F = fd.f;
    const int lane = threadIdx.x & 31;
    const int N = fd.N, max_iter = fd.max_iter;
    const int tx = (int)(tile % (unsigned)fd.tiles_x), ty = (int)(tile / (unsigned)fd.tiles_x);
    auto px = [&](int slot) { return tx * fd.tile_w + slot % fd.tile_w; };
    auto py = [&](int slot) { return ty * fd.tile_h + slot / fd.tile_w; };
    int pixa = 0, pixb = 0;
    bool acta, actb, skipa = false, skipb = false;
    // as in march2_tile: zeta_0 = A + t D on an axis slice, else the first
    // iterate Q0 + s (Q1 + s Q2) with Q0 in D and s = t + dot
    float2 D[AXIS ? 3 : 8], tin, dl;
    float2 Q1[AXIS ? 1 : 8], Q2[AXIS ? 1 : 8];
    {
        const int xa = px(lane), ya = py(lane), xb = px(lane + 32), yb = py(lane + 32);
        if (RECHECK) {
            pixa = ya * fd.W + xa;
            pixb = yb * fd.W + xb;
        }
        const bool va = xa < fd.W && ya < fd.H, vb = xb < fd.W && yb < fd.H;
        float da[3] = {0.f, 0.f, 1.f}, db[3] = {0.f, 0.f, 1.f};
        float tia = 0.f, toa = 0.f, tib = 0.f, tob = 0.f;
        acta = va && camera_clip<float>(F, fd.W, fd.H, xa, ya, da, tia, toa);
        actb = vb && camera_clip<float>(F, fd.W, fd.H, xb, yb, db, tib, tob);
        if constexpr (SPLIT) {
            const unsigned r = (unsigned)(kb / fd.k_chunk);
            skipa = va && __ldcg(sc.part_hit + ya * fd.W + xa) < r;
            skipb = vb && __ldcg(sc.part_hit + yb * fd.W + xb) < r;
            acta = acta && !skipa;
            actb = actb && !skipb;
        }
        if (!acta) tia = toa = 0.f;
        if (!actb) tib = tob = 0.f;
        dl = make_float2((toa - tia) / (float)N, (tob - tib) / (float)N);
        if (RECHECK) {  // a half without a ray samples far away: never within the recheck band
            if (!acta) tia = kFarT;
            if (!actb) tib = kFarT;
        }
        float Da[8], Db[8];
        slice_dir<float>(F, da, Da);
        slice_dir<float>(F, db, Db);
        if constexpr (AXIS) {
#pragma unroll
            for (int i = 0; i < 3; ++i) D[i] = make_float2(Da[i], Db[i]);
            tin = make_float2(tia, tib);
        } else {
            float Qa[3][8], Qb[3][8], dota, dotb;
            first_iterate_coeffs<float, SQ>(F.A, Da, F.c, dota, Qa[0], Qa[1], Qa[2]);
            first_iterate_coeffs<float, SQ>(F.A, Db, F.c, dotb, Qb[0], Qb[1], Qb[2]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                D[i] = make_float2(Qa[0][i], Qb[0][i]);
                Q1[i] = make_float2(Qa[1][i], Qb[1][i]);
                Q2[i] = make_float2(Qa[2][i], Qb[2][i]);
            }
            tin = make_float2(vadd(tia, dota), vadd(tib, dotb));
        }
    }
    const bool boxa = acta, boxb = actb;
    int suma = 0, sumb = 0, maxa = 0, maxb = 0, kfa = -1, kfb = -1;
    int qn = 0;  // staged recheck entries (warp-uniform)
    const int k0 = SPLIT ? kb : 0, k1 = SPLIT ? ke : N + 1;
    float2 kf = make_float2((float)k0, (float)k0);
    const float2 one = make_float2(1.f, 1.f), two = make_float2(2.f, 2.f), far = make_float2(kFarT, kFarT);
    bool more = __any_sync(kFull, acta || actb);
    for (int k = k0; k < k1 && more; k += 2) {
        const bool has2 = k + 1 < k1;  // warp-uniform: an odd number of samples ends in a round of one
        const float2 t = f2fma(kf, dl, tin);
        const float2 t2 = has2 ? f2fma(f2add(kf, one), dl, tin) : far;
        kf = f2add(kf, two);
        float2 z[8], y[8];
        bool ina = acta, inb = actb, ina2 = acta && has2, inb2 = actb && has2, live;
        int ca, cb, ca2, cb2;
        float2 dm, dm2;
        if constexpr (AXIS) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                z[i] = f2fma(t, D[i], P.A[i]);
                y[i] = f2fma(t2, D[i], P.A[i]);
            }
            classify_lockstep4_axis<SQ, MOD, RECHECK>(z, y, P, F.R2, max_iter, ina, inb, ina2, inb2, ca, cb, ca2,
                                                      cb2, dm, dm2, live);
        } else {
            first_iterate<float2, 8>(t, D, Q1, Q2, z);
            first_iterate<float2, 8>(t2, D, Q1, Q2, y);
            classify_lockstep4_it1<SQ, MOD, RECHECK>(z, y, P, F.R2, max_iter, ina, inb, ina2, inb2, ca, cb, ca2,
                                                     cb2, dm, dm2, live);
        }
        if (RECHECK && __any_sync(kFull, fminf(fminf(dm.x, dm.y), fminf(dm2.x, dm2.y)) <= P.margin_t)) {
            // marginal samples in this round (rare): stage sample k's, then sample k + 1's
            const unsigned below = (1u << lane) - 1u;
            {
                const bool pa = acta && dm.x <= P.margin_t, pb = actb && dm.y <= P.margin_t;
                const unsigned ba = __ballot_sync(kFull, pa), bb = __ballot_sync(kFull, pb);
                const int nqa = __popc(ba);
                if (pa) qs[qn + __popc(ba & below)] = make_int4(pixa, k | (kMarchSample << 16), 0, ina ? 0 : ca + 1);
                if (pb) qs[qn + nqa + __popc(bb & below)] = make_int4(pixb, k | (kMarchSample << 16), 0, inb ? 0 : cb + 1);
                qn += nqa + __popc(bb);
                if (qn > kQStage - 64) {
                    flush_staged(fd, sc, qs, qn);
                    qn = 0;
                }
            }
            {
                const bool pa = acta && has2 && !ina && dm2.x <= P.margin_t;
                const bool pb = actb && has2 && !inb && dm2.y <= P.margin_t;
                const unsigned ba = __ballot_sync(kFull, pa), bb = __ballot_sync(kFull, pb);
                const int nqa = __popc(ba);
                const int k2 = k + 1;
                if (pa) qs[qn + __popc(ba & below)] = make_int4(pixa, k2 | (kMarchSample << 16), 0, ina2 ? 0 : ca2 + 1);
                if (pb) qs[qn + nqa + __popc(bb & below)] = make_int4(pixb, k2 | (kMarchSample << 16), 0, inb2 ? 0 : cb2 + 1);
                qn += nqa + __popc(bb);
                if (qn > kQStage - 64) {
                    flush_staged(fd, sc, qs, qn);
                    qn = 0;
                }
            }
        }
        // sample k + 1 counts only after an outside sample k (ca2 = 0 without a sample)
        suma += ca + (ina ? 0 : ca2);
        sumb += cb + (inb ? 0 : cb2);
        maxa = max(maxa, max(ca, ina ? 0 : ca2));
        maxb = max(maxb, max(cb, inb ? 0 : cb2));
        if (live) {  // some half stayed bounded: those rays are inside at sample k or k + 1
            const bool da = ina || ina2, db = inb || inb2;
            if (da) kfa = ina ? k : k + 1;
            if (db) kfb = inb ? k : k + 1;
            if (RECHECK) {  // a finished ray samples far away from now on (see above)
                if (da) tin.x = kFarT;
                if (db) tin.y = kFarT;
            }
            acta = acta && !da;
            actb = actb && !db;
            more = __any_sync(kFull, acta || actb);
        }
    }
    if (RECHECK && qn > 0) recheck_staged<SQ, MOD>(fd, sc, qs, qn);
    const bool hita = kfa >= 0, hitb = kfb >= 0;
    const int nesca = (hita ? kfa : k1) - k0, nescb = (hitb ? kfb : k1) - k0;
    if constexpr (SPLIT) {  // this range's partial result per ray (see march_merge_kernel)
        const int xa = px(lane), ya = py(lane), xb = px(lane + 32), yb = py(lane + 32);
        const unsigned r = (unsigned)(kb / fd.k_chunk);
        const int64_t npx = (int64_t)fd.W * fd.H, base = (int64_t)r * npx;
        if (xa < fd.W && ya < fd.H && !skipa) {
            const int pa = ya * fd.W + xa;
            sc.part[base + pa] = boxa ? make_int4(kfa, suma + nesca, maxa + 1, nesca + (hita ? 1 : 0))
                                      : make_int4(-1, 0, 0, 0);
            if (hita) atomicMin(sc.part_hit + pa, r);
        }
        if (xb < fd.W && yb < fd.H && !skipb) {
            const int pb = yb * fd.W + xb;
            sc.part[base + pb] = boxb ? make_int4(kfb, sumb + nescb, maxb + 1, nescb + (hitb ? 1 : 0))
                                      : make_int4(-1, 0, 0, 0);
            if (hitb) atomicMin(sc.part_hit + pb, r);
        }
        return;
    }
    st.iters += (boxa ? suma + nesca : 0) + (boxb ? sumb + nescb : 0);
    st.samples += (boxa ? nesca + (hita ? 1 : 0) : 0) + (boxb ? nescb + (hitb ? 1 : 0) : 0);
    st.hits += (hita ? 1 : 0) + (hitb ? 1 : 0);
    const int xa = px(lane), ya = py(lane), xb = px(lane + 32), yb = py(lane + 32);
    const bool va = xa < fd.W && ya < fd.H, vb = xb < fd.W && yb < fd.H;
    if (va && !hita) write_miss<float>(fd, xa, ya, boxa ? maxa + 1 : 0);
    if (vb && !hitb) write_miss<float>(fd, xb, yb, boxb ? maxb + 1 : 0);
    warp_push(hita, make_int4(ya * fd.W + xa, kfa, 0, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
    warp_push(hitb, make_int4(yb * fd.W + xb, kfb, 0, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
}

// Normal (central differences of F(p) = modulus(zeta_{n*}(p)) at p +- h e_a,
// iterated n* times from zeta0 = A + depth D +- h E_a, the slice image of
// eye + depth d +- h e_a), shading and the pixel's outputs for a hit at depth;
// lanes with part == false only join the warp-wide loop bound.
template <typename T, int SQ, int MOD>
__device__ __forceinline__ void normal_shade(const FrameDesc &fd, const FrameT<T> &F, int x, int y, const T (&d)[3],
                                             const T (&D)[8], T depth, int n_star, bool part, LaneStats &st)
{
    int nmax = part ? n_star : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(kFull, nmax, o));
    T g[3];
    bool guard = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T fv[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T hs = s == 0 ? F.h : -F.h;
            T z[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) z[i] = dfma(hs, F.E[a][i], dfma(depth, D[i], F.A[i]));
            T sp = dq_sp<T>(z);
            for (int n = 0; n < nmax; ++n)
                if (n < n_star) dq_iter<T, SQ, MOD>(z, z, sp, F.c);
            fv[s] = modulus<T, MOD>(z);
            guard = guard || !(fv[s] <= normal_fmax(T(0)));
        }
        g[a] = fv[0] - fv[1];
    }
    if (part) {
        st.niters += 6ull * (unsigned)n_star;
        shade_write<T>(fd, F, x, y, n_star, depth, g, guard, d);
    }
}

// Bisection, normal and shading of hit-list entries [base, base + 32) clipped to
// nhits, one per lane (see bisect_kernel); all 32 lanes call.
template <typename T, int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ void bisect_chunk(const FrameDesc &fd, const Scratch &sc, unsigned base, unsigned nhits,
                                             LaneStats &st)
{
    const FrameT<T> &F = frame<T>(fd);
    const int lane = threadIdx.x & 31;
    const unsigned idx = base + lane;
    const bool part = idx < nhits;
    int4 e = make_int4(0, 0, 0, 0);
    if (part) e = __ldcg(sc.hits + idx);  // L2: the list may be rewritten within one serving launch
    const int pixel = e.x, k_first = e.y;
    const int x = pixel % fd.W, y = pixel / fd.W;
    T d[3] = {T(0), T(0), T(1)};
    T t_in = T(0), t_out = T(0);
    if (part) camera_clip<T>(F, fd.W, fd.H, x, y, d, t_in, t_out);
    T D[8];
    slice_dir<T>(F, d, D);
    const T delta = (t_out - t_in) / T(fd.N);
    bool bis = part && k_first > 0;
    T lo = bis ? dfma(T(k_first - 1), delta, t_in) : t_in;
    T hi = bis ? dfma(T(k_first), delta, t_in) : t_in;
    // n* starts as the escape count of the last outside march sample, k_first - 1:
    // the march keeps no per-sample counts, so it is classified again here, with
    // the march's own position and arithmetic (not counted as new iterations)
    int n_lo = fd.max_iter;
    {
        T z[8];
        bool mg;
        int n;
        bool it1 = false;
        if constexpr (sizeof(T) == 4) {
            if (!fd.axis_slice) {  // the FP32 march's first-iterate form and sample position
                it1 = true;
                float Q0[8], Q1[8], Q2[8], dot;
                first_iterate_coeffs<float, SQ>(F.A, D, F.c, dot, Q0, Q1, Q2);
                first_iterate<float, 8>(vfma((float)(k_first - 1), delta, vadd(t_in, dot)), Q0, Q1, Q2, z);
            }
        }
        if (it1) {
            n = classify_lockstep_it1<T, SQ, MOD, false>(z, F, fd.max_iter, bis, mg);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) z[i] = dfma(lo, D[i], F.A[i]);
            n = classify_lockstep<T, SQ, MOD, false>(z, F, fd.max_iter, bis, mg);
        }
        if (bis) n_lo = n;
    }
    unsigned path = 0;
    unsigned iters = 0, samples = 0;
    for (int b = 0; b < fd.B; ++b) {
        const T mid = lo + T(0.5) * (hi - lo);
        T z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = dfma(mid, D[i], F.A[i]);
        bool mg;
        const int n = classify_lockstep<T, SQ, MOD, RECHECK>(z, F, fd.max_iter, bis, mg);
        if (RECHECK) {
            const bool push = bis && mg;
            if (warp_push(push, make_int4(pixel, k_first | (b << 16), (int)path, n), sc.queue, sc.queue_cap,
                          &sc.ctr->queue_count)) {
                atomicAdd(&sc.ctr->stats[7], 1ull);
                mark_dirty(fd, sc, pixel);
            }
            st.rechecks += push ? 1 : 0;
        }
        if (bis) {
            iters += n ? (unsigned)n : (unsigned)fd.max_iter;
            samples += 1;
            if (n == 0) {
                hi = mid;
            } else {
                lo = mid;
                n_lo = n;
                path |= 1u << b;
            }
        }
    }
    const T depth = bis ? lo + T(0.5) * (hi - lo) : t_in;
    // RECHECK: the FP32 field of a normal of more than late_step steps carries
    // its rounding amplified along the orbit, so those normals are evaluated in
    // FP64 (on the FP64 ray, at the bisection's depth); the others in FP32
    const bool n64 = RECHECK && sizeof(T) == 4 && part && n_lo > late_step<MOD>();
    normal_shade<T, SQ, MOD>(fd, F, x, y, d, D, depth, n_lo, part && !n64, st);
    if (RECHECK && sizeof(T) == 4 && __any_sync(kFull, n64)) {
        const FrameT<double> &Fd = fd.d;
        double dd[3] = {0.0, 0.0, 1.0}, ti = 0.0, to = 0.0, Dd[8];
        if (n64) camera_clip<double>(Fd, fd.W, fd.H, x, y, dd, ti, to);
        slice_dir<double>(Fd, dd, Dd);
        normal_shade<double, SQ, MOD>(fd, Fd, x, y, dd, Dd, (double)depth, n_lo, n64, st);
    }
    st.iters += iters;
    st.samples += samples;
}

// Normal and shading of the hits of an L-lane group (see bisect_group):
// evaluation q = 2a + s (F at depth -+ h e_a, s = 0: +h) runs on lane q mod L of
// the group, in round q / L; `part` is uniform within a group.  All 32 lanes
// call.  Same values as normal_shade<U>.
template <typename U, int SQ, int MOD, int L>
__device__ __forceinline__ void group_normal(const FrameDesc &fd, const FrameT<U> &F, int x, int y, const U (&d)[3],
                                             const U (&D)[8], U depth, int n_lo, bool part, LaneStats &st)
{
    const int lane = threadIdx.x & 31;
    const int j = lane & (L - 1), gb = lane & ~(L - 1);
    int nmax = part ? n_lo : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(kFull, nmax, o));
    U fvq[6];
    bool guard = false;
#pragma unroll
    for (int q0 = 0; q0 < 6; q0 += L) {
        const int q = q0 + j;
        const int a = q < 6 ? q >> 1 : 0;
        const U hs = (q & 1) == 0 ? F.h : -F.h;
        U z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = dfma(hs, F.E[a][i], dfma(depth, D[i], F.A[i]));
        U sp = dq_sp<U>(z);
        const int ns = part && q < 6 ? n_lo : 0;
        for (int n = 0; n < nmax; ++n)
            if (n < ns) dq_iter<U, SQ, MOD>(z, z, sp, F.c);
        const U fv = modulus<U, MOD>(z);
        const unsigned bad = __ballot_sync(kFull, q < 6 && !(fv <= normal_fmax(U(0))));
        guard = guard || ((bad >> gb) & ((1u << L) - 1u)) != 0;
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (q0 + i < 6) fvq[q0 + i] = __shfl_sync(kFull, fv, gb + i);
    }
    if (part && j == 0) {
        U g[3] = {fvq[0] - fvq[1], fvq[2] - fvq[3], fvq[4] - fvq[5]};
        st.niters += 6ull * (unsigned)n_lo;
        shade_write<U>(fd, F, x, y, n_lo, depth, g, guard, d);
    }
}

// The same bisection, normal and shading for hit-list entries [base, base +
// 32 / L) clipped to nhits, L lanes per hit (L = 4 or 8; lane group g = lane / L
// takes entry base + g; all 32 lanes call).  For frames with few hits per SM,
// where one lane per hit leaves the bisection's dependent chain of B + 7
// classifications exposed: here the lanes of a group classify the midpoints of
// log2(L) levels of the bisection tree at once (lane j < L - 1 holds node j + 1:
// node 1 the next midpoint, children 2i inside -> [lo, mid] and 2i + 1 outside
// -> [mid, hi]), each deriving its interval with the sequential halvings' own
// operations, and the group replays the path; the six normal evaluations are
// spread over the group's lanes.  Brackets, n*, depths, normals, queued
// rechecks and the counted iterations (only the nodes on the path count) are
// those of bisect_chunk.
template <typename T, int SQ, int MOD, bool RECHECK, int L>
__device__ __forceinline__ void bisect_group(const FrameDesc &fd, const Scratch &sc, unsigned base, unsigned nhits,
                                             LaneStats &st)
{
    static_assert(L == 4 || L == 8, "four or eight lanes per hit");
    constexpr int kLevels = L == 8 ? 3 : 2;  // tree levels per round
    const FrameT<T> &F = frame<T>(fd);
    const int lane = threadIdx.x & 31;
    const int j = lane & (L - 1), gb = lane & ~(L - 1);  // lane in the group, the group's first lane
    const unsigned idx = base + (unsigned)(lane / L);
    const bool part = idx < nhits;
    int4 e = make_int4(0, 0, 0, 0);
    if (part) e = __ldcg(sc.hits + idx);  // L2: the list may be rewritten within one serving launch
    const int pixel = e.x, k_first = e.y;
    const int x = pixel % fd.W, y = pixel / fd.W;
    T d[3] = {T(0), T(0), T(1)};
    T t_in = T(0), t_out = T(0);
    if (part) camera_clip<T>(F, fd.W, fd.H, x, y, d, t_in, t_out);
    T D[8];
    slice_dir<T>(F, d, D);
    const T delta = (t_out - t_in) / T(fd.N);
    const bool bis = part && k_first > 0;
    T lo = bis ? dfma(T(k_first - 1), delta, t_in) : t_in;
    T hi = bis ? dfma(T(k_first), delta, t_in) : t_in;
    // n* starts as the escape count of march sample k_first - 1, classified
    // again with the march's position and arithmetic (not counted): on the
    // group's last lane, in the first round where that form is the midpoints'
    // form, else (the FP32 march's first-iterate form of a general slice) before
    int n_lo = fd.max_iter;
    bool lo_in_round0 = true;
    if constexpr (sizeof(T) == 4) {
        if (!fd.axis_slice) {
            lo_in_round0 = false;
            T z[8];
            float Q0[8], Q1[8], Q2[8], dot;
            first_iterate_coeffs<float, SQ>(F.A, D, F.c, dot, Q0, Q1, Q2);
            first_iterate<float, 8>(vfma((float)(k_first - 1), delta, vadd(t_in, dot)), Q0, Q1, Q2, z);
            bool mg;
            const int n = classify_lockstep_it1<T, SQ, MOD, false>(z, F, fd.max_iter, bis && j == L - 1, mg);
            const int nl = __shfl_sync(kFull, n, gb + L - 1);
            if (bis) n_lo = nl;
        }
    }
    unsigned path = 0;
    unsigned iters = 0, samples = 0, rechecks = 0;
    const int node = j + 1, level = 31 - __clz(node);  // last lane: node L, level kLevels (no node)
    for (int b0 = 0; b0 < fd.B || (b0 == 0 && lo_in_round0); b0 += kLevels) {
        const int levels = min(kLevels, fd.B - b0);
        const bool lo_lane = b0 == 0 && lo_in_round0 && j == L - 1;
        T l = lo, h = hi;
        for (int q = level - 1; q >= 0; --q) {  // path bits below the node's leading one
            const T mid = l + T(0.5) * (h - l);
            if ((node >> q) & 1)
                l = mid;
            else
                h = mid;
        }
        const T pos = lo_lane ? lo : l + T(0.5) * (h - l);
        const bool act = bis && (lo_lane || level < levels);
        T z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = dfma(pos, D[i], F.A[i]);
        bool mg;
        const int n = classify_lockstep<T, SQ, MOD, RECHECK>(z, F, fd.max_iter, act, mg);
        if (b0 == 0 && lo_in_round0) {
            const int nl = __shfl_sync(kFull, n, gb + L - 1);
            if (bis) n_lo = nl;
        }
        // replay the path through the levels of this round
        int cur = 1;
        for (int lv = 0; lv < kLevels; ++lv) {
            const int nc = __shfl_sync(kFull, n, gb + cur - 1);
            const bool mc = RECHECK ? __shfl_sync(kFull, mg, gb + cur - 1) : false;
            if (lv >= levels) break;  // warp-uniform
            const int b = b0 + lv;
            if (RECHECK) {
                const bool push = bis && mc && j == 0;
                if (warp_push(push, make_int4(pixel, k_first | (b << 16), (int)path, nc), sc.queue, sc.queue_cap,
                              &sc.ctr->queue_count)) {
                    atomicAdd(&sc.ctr->stats[7], 1ull);
                    mark_dirty(fd, sc, pixel);
                }
                rechecks += push ? 1 : 0;
            }
            const T mid = lo + T(0.5) * (hi - lo);
            if (bis) {
                iters += nc ? (unsigned)nc : (unsigned)fd.max_iter;
                samples += 1;
                if (nc == 0) {
                    hi = mid;
                } else {
                    lo = mid;
                    n_lo = nc;
                    path |= 1u << b;
                }
            }
            cur = 2 * cur + (nc != 0 ? 1 : 0);
        }
    }
    const T depth = bis ? lo + T(0.5) * (hi - lo) : t_in;
    // RECHECK: a normal of more than late_step steps is evaluated in FP64 (see
    // bisect_chunk), the others in T
    const bool n64 = RECHECK && sizeof(T) == 4 && part && n_lo > late_step<MOD>();
    group_normal<T, SQ, MOD, L>(fd, F, x, y, d, D, depth, n_lo, part && !n64, st);
    if (RECHECK && sizeof(T) == 4 && __any_sync(kFull, n64)) {
        const FrameT<double> &Fd = fd.d;
        double dd[3] = {0.0, 0.0, 1.0}, ti = 0.0, to = 0.0, Dd[8];
        if (n64) camera_clip<double>(Fd, fd.W, fd.H, x, y, dd, ti, to);
        slice_dir<double>(Fd, dd, Dd);
        group_normal<double, SQ, MOD, L>(fd, Fd, x, y, dd, Dd, (double)depth, n_lo, n64, st);
    }
    if (part && j == 0) {
        st.iters += iters;
        st.samples += samples;
        if (RECHECK) st.rechecks += rechecks;
    }
}

// Add a warp's lane counters to the frame's stats.
template <bool RECHECK>
__device__ __forceinline__ void flush_lane_stats(const Scratch &sc, const LaneStats &st, bool march)
{
    flush_stat(&sc.ctr->stats[0], st.iters);
    if (march) flush_stat(&sc.ctr->stats[8], st.iters);
    flush_stat(&sc.ctr->stats[1], st.niters);
    flush_stat(&sc.ctr->stats[2], st.samples);
    flush_stat(&sc.ctr->stats[3], st.hits);
    if (RECHECK) flush_stat(&sc.ctr->stats[4], st.rechecks);
}

}  // namespace dqj
