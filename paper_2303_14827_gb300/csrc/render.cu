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

#include "dq_math.cuh"

namespace dqj {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 128;  // 4 warps per CTA

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
    ndl = ndl > T(0) ? ndl : T(0);
    T v = F.ka + F.kd * ndl;
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

// ---------------------------------------------------------------------------
// march
// ---------------------------------------------------------------------------
template <typename T, int SQ, int MOD, bool RECHECK>
__global__ void __launch_bounds__(kBlock) march_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<T> &F = frame<T>(fd);
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = (unsigned)fd.tiles_x * (unsigned)fd.tiles_y;
    unsigned long long s_iters = 0, s_samples = 0, s_hits = 0, s_rechecks = 0;
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(&sc.ctr->tile_next, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
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
        int esc_max = 0, n_prev = 0, k_first = -1;
        unsigned iters = 0, samples = 0;
        for (int k = 0; k <= fd.N; ++k) {
            if (!__any_sync(kFull, active)) break;
            const T t = dfma(T(k), delta, t_in);
            T z[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) z[i] = dfma(t, D[i], F.A[i]);
            bool mg;
            const int n = classify_lockstep<T, SQ, MOD, RECHECK>(z, F, fd.max_iter, active, mg);
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
                    n_prev = n;
                }
            }
        }
        s_iters += iters;
        s_samples += samples;
        const bool hit = valid && k_first >= 0;
        if (valid && !hit) write_miss<T>(fd, x, y, esc_max);
        s_hits += hit ? 1 : 0;
        warp_push(hit, make_int4(y * fd.W + x, k_first, n_prev, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
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
// samples), max_* (largest escape count - 1), prev_* (escape count - 1 of the
// latest outside sample) and the first inside sample kf_*; the iteration and
// sample counts follow from them once the ray is done.
// ---------------------------------------------------------------------------
template <int SQ, int MOD, bool RECHECK>
__global__ void __launch_bounds__(kBlock, 5) march2_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<float> &F = fd.f;
    const PairConsts &P = fd.p2;
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = (unsigned)fd.tiles_x * (unsigned)fd.tiles_y;
    const int N = fd.N, max_iter = fd.max_iter;
    unsigned long long s_iters = 0, s_samples = 0, s_hits = 0, s_rechecks = 0;
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(&sc.ctr->tile_next, 1u);
        tile = __shfl_sync(kFull, tile, 0);
        if (tile >= ntiles) break;
        const int tx = (int)(tile % (unsigned)fd.tiles_x), ty = (int)(tile / (unsigned)fd.tiles_x);
        const int sb = lane + 32;
        const int xa = tx * fd.tile_w + lane % fd.tile_w, ya = ty * fd.tile_h + lane / fd.tile_w;
        const int xb = tx * fd.tile_w + sb % fd.tile_w, yb = ty * fd.tile_h + sb / fd.tile_w;
        const bool va = xa < fd.W && ya < fd.H, vb = xb < fd.W && yb < fd.H;
        float da[3] = {0.f, 0.f, 1.f}, db[3] = {0.f, 0.f, 1.f};
        float tia = 0.f, toa = 0.f, tib = 0.f, tob = 0.f;
        const bool boxa = va && camera_clip<float>(F, fd.W, fd.H, xa, ya, da, tia, toa);
        const bool boxb = vb && camera_clip<float>(F, fd.W, fd.H, xb, yb, db, tib, tob);
        if (!boxa) tia = toa = 0.f;
        if (!boxb) tib = tob = 0.f;
        float2 D[8];
        {
            float Da[8], Db[8];
            slice_dir<float>(F, da, Da);
            slice_dir<float>(F, db, Db);
#pragma unroll
            for (int i = 0; i < 8; ++i) D[i] = make_float2(Da[i], Db[i]);
        }
        const float2 tin = make_float2(tia, tib);
        const float2 dl = make_float2((toa - tia) / (float)N, (tob - tib) / (float)N);
        bool acta = boxa, actb = boxb;
        int suma = 0, sumb = 0, maxa = 0, maxb = 0, preva = 0, prevb = 0, kfa = -1, kfb = -1;
        float2 kf = make_float2(0.f, 0.f);
        for (int k = 0; k <= N; ++k) {
            if (!__any_sync(kFull, acta || actb)) break;
            const float2 t = f2fma(kf, dl, tin);
            kf = f2add(kf, make_float2(1.f, 1.f));
            float2 z[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) z[i] = f2fma(t, D[i], P.A[i]);
            bool ina = acta, inb = actb, mga, mgb;
            int ca, cb;
            classify_lockstep2<SQ, MOD, RECHECK>(z, P, F.R2, F.margin, max_iter, ina, inb, ca, cb, mga, mgb);
            if (RECHECK) {
                const bool pa = acta && mga, pb = actb && mgb;
                if (warp_push(pa, make_int4(ya * fd.W + xa, k | (kMarchSample << 16), 0, ina ? 0 : ca + 1), sc.queue,
                              sc.queue_cap, &sc.ctr->queue_count)) {
                    atomicAdd(&sc.ctr->stats[7], 1ull);
                    mark_dirty(fd, sc, ya * fd.W + xa);
                }
                if (warp_push(pb, make_int4(yb * fd.W + xb, k | (kMarchSample << 16), 0, inb ? 0 : cb + 1), sc.queue,
                              sc.queue_cap, &sc.ctr->queue_count)) {
                    atomicAdd(&sc.ctr->stats[7], 1ull);
                    mark_dirty(fd, sc, yb * fd.W + xb);
                }
                s_rechecks += (pa ? 1 : 0) + (pb ? 1 : 0);
            }
            // ina / inb imply acta / actb (they start equal and only clear)
            suma += ca;
            sumb += cb;
            maxa = max(maxa, ca);
            maxb = max(maxb, cb);
            if (acta && !ina) preva = ca;
            if (actb && !inb) prevb = cb;
            if (ina) kfa = k;
            if (inb) kfb = k;
            acta = acta && !ina;
            actb = actb && !inb;
        }
        const bool hita = kfa >= 0, hitb = kfb >= 0;
        // iterations = sum of (escape count) over escaped samples + max_iter per inside sample
        //            = sum of bounded steps + number of escaped samples
        const int nesca = hita ? kfa : N + 1, nescb = hitb ? kfb : N + 1;
        s_iters += (boxa ? suma + nesca : 0) + (boxb ? sumb + nescb : 0);
        s_samples += (boxa ? nesca + (hita ? 1 : 0) : 0) + (boxb ? nescb + (hitb ? 1 : 0) : 0);
        s_hits += (hita ? 1 : 0) + (hitb ? 1 : 0);
        if (va && !hita) write_miss<float>(fd, xa, ya, boxa ? maxa + 1 : 0);
        if (vb && !hitb) write_miss<float>(fd, xb, yb, boxb ? maxb + 1 : 0);
        warp_push(hita, make_int4(ya * fd.W + xa, kfa, preva + 1, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
        warp_push(hitb, make_int4(yb * fd.W + xb, kfb, prevb + 1, 0), sc.hits, sc.hit_cap, &sc.ctr->hit_count);
    }
    flush_stat(&sc.ctr->stats[0], s_iters);
    flush_stat(&sc.ctr->stats[8], s_iters);
    flush_stat(&sc.ctr->stats[2], s_samples);
    flush_stat(&sc.ctr->stats[3], s_hits);
    if (RECHECK) flush_stat(&sc.ctr->stats[4], s_rechecks);
}

// ---------------------------------------------------------------------------
// bisect + normal + shade over the hit list
// ---------------------------------------------------------------------------
template <typename T, int SQ, int MOD, bool RECHECK>
__global__ void __launch_bounds__(kBlock) bisect_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<T> &F = frame<T>(fd);
    const int lane = threadIdx.x & 31;
    const unsigned nhits = min(*(volatile unsigned *)&sc.ctr->hit_count, sc.hit_cap);
    unsigned long long s_iters = 0, s_samples = 0, s_niters = 0, s_rechecks = 0;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&sc.ctr->hit_next, 32u);
        base = __shfl_sync(kFull, base, 0);
        if (base >= nhits) break;
        const unsigned idx = base + lane;
        const bool part = idx < nhits;
        int4 e = make_int4(0, 0, 0, 0);
        if (part) e = sc.hits[idx];
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
        int n_lo = bis ? e.z : fd.max_iter;
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
                s_rechecks += push ? 1 : 0;
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
        const int n_star = n_lo;
        // Normal: F(p) = modulus(zeta_{n*}(p)) at p +- h e_a, iterated n* times.
        // zeta0 = A + depth D +- h E_a (the slice image of eye + depth d +- h e_a).
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
            s_niters += 6ull * (unsigned)n_star;
            shade_write<T>(fd, F, x, y, n_star, depth, g, guard, d);
        }
        s_iters += iters;
        s_samples += samples;
    }
    flush_stat(&sc.ctr->stats[0], s_iters);
    flush_stat(&sc.ctr->stats[1], s_niters);
    flush_stat(&sc.ctr->stats[2], s_samples);
    if (RECHECK) flush_stat(&sc.ctr->stats[4], s_rechecks);
}

// ---------------------------------------------------------------------------
// FP64 recheck of queued samples and FP64 re-render of disagreeing pixels
// ---------------------------------------------------------------------------
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) recheck_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<double> &F = fd.d;
    const unsigned total = *(volatile unsigned *)&sc.ctr->queue_count;
    const unsigned nq = min(total, sc.queue_cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        const int4 e = sc.queue[i];
        const int pixel = e.x, k = e.y & 0xffff, b = e.y >> 16;
        const int x = pixel % fd.W, y = pixel / fd.W;
        double d[3], t_in, t_out;
        camera_clip<double>(F, fd.W, fd.H, x, y, d, t_in, t_out);
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
#pragma unroll
        for (int j = 0; j < 8; ++j)
            z[j] = F.O[j] + (F.eye[0] + t * d[0]) * F.E[0][j] + (F.eye[1] + t * d[1]) * F.E[1][j] +
                   (F.eye[2] + t * d[2]) * F.E[2][j];
        const int n64 = classify_scalar<double, SQ, MOD>(z, F, fd.max_iter);
        if (n64 != e.w) mark_dirty(fd, sc, pixel);
    }
    // a full queue: pixels whose samples did not fit were flagged by the pushers
}

// Full FP64 render of one pixel per thread (the reference sequence of steps).
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) fixup_kernel(const __grid_constant__ FrameDesc fd, const Scratch sc)
{
    const FrameT<double> &F = fd.d;
    const unsigned nd = min(*(volatile unsigned *)&sc.ctr->dirty_count, sc.dirty_cap);
    unsigned long long its = 0, npx = 0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) {
        const int pixel = sc.dirty_list[i];
        const int x = pixel % fd.W, y = pixel / fd.W;
        npx += 1;
        double d[3], t_in, t_out;
        if (!camera_clip<double>(F, fd.W, fd.H, x, y, d, t_in, t_out)) {
            write_miss<double>(fd, x, y, 0);
            continue;
        }
        const double delta = (t_out - t_in) / (double)fd.N;
        auto cls = [&](double t) {
            double z[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                z[j] = F.O[j] + (F.eye[0] + t * d[0]) * F.E[0][j] + (F.eye[1] + t * d[1]) * F.E[1][j] +
                       (F.eye[2] + t * d[2]) * F.E[2][j];
            const int n = classify_scalar<double, SQ, MOD>(z, F, fd.max_iter);
            its += n ? n : fd.max_iter;
            return n;
        };
        int esc_max = 0, n_prev = 0, k_first = -1;
        for (int k = 0; k <= fd.N; ++k) {
            const int n = cls(t_in + (double)k * delta);
            if (n == 0) {
                k_first = k;
                break;
            }
            esc_max = n > esc_max ? n : esc_max;
            n_prev = n;
        }
        if (k_first < 0) {
            write_miss<double>(fd, x, y, esc_max);
            continue;
        }
        double depth = t_in;
        int n_star = fd.max_iter;
        if (k_first > 0) {
            double lo = t_in + (double)(k_first - 1) * delta, hi = t_in + (double)k_first * delta;
            n_star = n_prev;
            for (int b = 0; b < fd.B; ++b) {
                const double mid = lo + 0.5 * (hi - lo);
                const int n = cls(mid);
                if (n == 0) {
                    hi = mid;
                } else {
                    lo = mid;
                    n_star = n;
                }
            }
            depth = lo + 0.5 * (hi - lo);
        }
        double g[3];
        bool guard = false;
        for (int a = 0; a < 3; ++a) {
            double fv[2];
            for (int s = 0; s < 2; ++s) {
                double p[3] = {F.eye[0] + depth * d[0], F.eye[1] + depth * d[1], F.eye[2] + depth * d[2]};
                p[a] += s == 0 ? F.h : -F.h;
                double z[8];
                for (int j = 0; j < 8; ++j) z[j] = F.O[j] + p[0] * F.E[0][j] + p[1] * F.E[1][j] + p[2] * F.E[2][j];
                double sp = dq_sp<double>(z);
                for (int n = 0; n < n_star; ++n) dq_iter<double, SQ, MOD>(z, z, sp, F.c);
                its += n_star;
                fv[s] = modulus<double, MOD>(z);
                guard = guard || !(fv[s] <= normal_fmax(0.0));
            }
            g[a] = fv[0] - fv[1];
        }
        shade_write<double>(fd, F, x, y, n_star, depth, g, guard, d);
    }
    unsigned long long v = warp_sum(its), p = warp_sum(npx);
    if ((threadIdx.x & 31) == 0) {
        if (v) atomicAdd(&sc.ctr->stats[6], v);
        if (p) atomicAdd(&sc.ctr->stats[5], p);
    }
}

template <typename K>
int persistent_grid(K kernel, int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms;
}

template <typename T, int SQ, int MOD, bool RECHECK>
cudaError_t launch_passes(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    static int g_march = 0, g_march2 = 0, g_bisect = 0;
    const unsigned ntiles = (unsigned)fd.tiles_x * (unsigned)fd.tiles_y;
    if (ev) cudaEventRecord(ev[0], st);
    if constexpr (sizeof(T) == 4) {
        if (fd.march_variant == 1) {
            if (!g_march2) g_march2 = persistent_grid(march2_kernel<SQ, MOD, RECHECK>, num_sms);
            const int gm = (int)min((unsigned)g_march2, (ntiles + 3u) / 4u);
            march2_kernel<SQ, MOD, RECHECK><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
        }
    }
    if (sizeof(T) != 4 || fd.march_variant != 1) {
        if (!g_march) g_march = persistent_grid(march_kernel<T, SQ, MOD, RECHECK>, num_sms);
        const int gm = (int)min((unsigned)g_march, (ntiles + 3u) / 4u);
        march_kernel<T, SQ, MOD, RECHECK><<<gm > 0 ? gm : 1, kBlock, 0, st>>>(fd, sc);
    }
    if (ev) cudaEventRecord(ev[1], st);
    if (!g_bisect) g_bisect = persistent_grid(bisect_kernel<T, SQ, MOD, RECHECK>, num_sms);
    const unsigned maxw = ((unsigned)fd.W * (unsigned)fd.H + 31u) / 32u;
    const int gb = (int)min((unsigned)g_bisect, (maxw + 3u) / 4u);
    bisect_kernel<T, SQ, MOD, RECHECK><<<gb > 0 ? gb : 1, kBlock, 0, st>>>(fd, sc);
    if (ev) cudaEventRecord(ev[2], st);
    if (RECHECK) {
        static int g_re = 0, g_fx = 0;
        if (!g_re) g_re = persistent_grid(recheck_kernel<SQ, MOD>, num_sms);
        if (!g_fx) g_fx = persistent_grid(fixup_kernel<SQ, MOD>, num_sms);
        recheck_kernel<SQ, MOD><<<g_re, kBlock, 0, st>>>(fd, sc);
        if (ev) cudaEventRecord(ev[3], st);
        fixup_kernel<SQ, MOD><<<g_fx, kBlock, 0, st>>>(fd, sc);
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

cudaError_t launch_frame(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev)
{
    const int m = fd.square_mode * 2 + fd.modulus_mode;
    switch (m) {
    case 0: return launch_mode<0, 0>(fd, sc, st, num_sms, ev);
    case 1: return launch_mode<0, 1>(fd, sc, st, num_sms, ev);
    case 2: return launch_mode<1, 0>(fd, sc, st, num_sms, ev);
    default: return launch_mode<1, 1>(fd, sc, st, num_sms, ev);
    }
}

}  // namespace dqj
