// dq_math.cuh -- dual-quaternion Julia step with its escape test, templated on
// float / double, plus a paired FP32 form that advances two samples per thread.
//
// A dual quaternion zeta = q_r + q_d eps is kept in 8 registers (q_r | q_d),
// scalar first in each half (appendix, quaternion and dual-quaternion
// definitions).  The square is expanded in closed form instead of the general
// product:
//   ALGEBRAIC (eps^2 = 0, appendix product):
//     q_r^2             = (r0^2 - r1^2 - r2^2 - r3^2, 2 r0 r1, 2 r0 r2, 2 r0 r3)
//                         (Eq. quatsq)
//     q_r q_d + q_d q_r = 2 (r0 d0 - v_r . v_d, r0 v_d + d0 v_r)
//                         (the cross products cancel)
//   PAPER_COMPONENTWISE (the equation printed beside Eq. dqjulia2):
//     q_r^2 + q_d^2 eps, each half by Eq. quatsq.
// The escape test compares the modulus with R^2 (Method, "Practical
// Considerations"); EUCLID8 takes |q_r|^2 + |q_d|^2, DUALNUM |q_r|^2.
//
// One step computes zeta_{n+1} = zeta_n^2 + c and m = modulus(zeta_{n+1}).  The
// partial sum sp = r1^2 + r2^2 + r3^2 of the escape test of step n is carried
// into step n+1, whose real scalar r0^2 - r1^2 - r2^2 - r3^2 + c0 is
// r0^2 + (c0 - sp): the three squares are formed once, not twice.  (Offsetting
// sp by -R^2 would save nothing and cost accuracy: c0 - R^2 and sp - R^2 are
// both near -R^2, and their difference loses bits when the iterate is small.)
#pragma once

#include "dqj_internal.h"

namespace dqj {

// FP32 recheck mode: a sample whose orbit runs past late_step<MOD>() steps is
// always rechecked in FP64, whatever its distance from R^2, and a hit whose
// normal field takes more steps than that is re-rendered in FP64.  An FP32
// sample position is rounded (about 6e-8 relative) and each step multiplies a
// position difference by 2 |zeta_n|; on a long enough orbit the amplified
// difference exceeds the recheck margin (1e-3 relative) and moves an escape
// decision that no tested modulus came close to, and it moves the normal
// field's central differences.  With the dual-number modulus, whose escape
// test ignores the dual half, orbits near the real half's own Julia set run
// long: decisions moved at steps 14-24 on 11 of 42 random frames with max_iter
// 16-24, hence 12.  With the 8-component modulus the dual half grows with the
// orbit's sensitivity and ends such orbits early: no decision moved in 180
// random frames with max_iter 12-32, but normals drifted on one frame with
// max_iter 32, hence 20.  The march kernels apply the rule for the
// dual-number modulus only (no cost per round otherwise); the bisection, the
// re-render and sphere tracing apply it for both.
template <int MOD>
__host__ __device__ constexpr int late_step() { return MOD == 1 ? 12 : 20; }

__device__ __forceinline__ float dfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return fma(a, b, c); }

// sp of zeta: r1^2 + r2^2 + r3^2
template <typename T>
__device__ __forceinline__ T dq_sp(const T (&z)[8])
{
    return dfma(z[3], z[3], dfma(z[2], z[2], z[1] * z[1]));
}

// zo = zi^2 + c; returns modulus(zo) and updates sp.  zo and zi may be the
// same array; loops that alternate two arrays avoid copying the state back.
template <typename T, int SQ, int MOD>
__device__ __forceinline__ T dq_iter(const T (&zi)[8], T (&z)[8], T &sp, const T (&c)[8])
{
    const T r0 = zi[0], r1 = zi[1], r2 = zi[2], r3 = zi[3];
    const T d0 = zi[4], d1 = zi[5], d2 = zi[6], d3 = zi[7];
    const T tr0 = r0 + r0;
    z[0] = dfma(r0, r0, dfma(sp, T(-1), c[0]));
    z[1] = dfma(tr0, r1, c[1]);
    z[2] = dfma(tr0, r2, c[2]);
    z[3] = dfma(tr0, r3, c[3]);
    const T td0 = d0 + d0;
    if (SQ == 0) {
        T q = r1 * d1;
        q = dfma(r2, d2, q);
        q = dfma(r3, d3, q);
        z[4] = dfma(q, T(-2), dfma(tr0, d0, c[4]));
        z[5] = dfma(tr0, d1, dfma(td0, r1, c[5]));
        z[6] = dfma(tr0, d2, dfma(td0, r2, c[6]));
        z[7] = dfma(tr0, d3, dfma(td0, r3, c[7]));
    } else {
        T q = d1 * d1;
        q = dfma(d2, d2, q);
        q = dfma(d3, d3, q);
        z[4] = dfma(q, T(-1), dfma(d0, d0, c[4]));
        z[5] = dfma(td0, d1, c[5]);
        z[6] = dfma(td0, d2, c[6]);
        z[7] = dfma(td0, d3, c[7]);
    }
    sp = dq_sp<T>(z);
    T x = dfma(z[0], z[0], sp);
    if (MOD == 0) {
        x = dfma(z[4], z[4], x);
        x = dfma(z[5], z[5], x);
        x = dfma(z[6], z[6], x);
        x = dfma(z[7], z[7], x);
    }
    return x;
}

// modulus(zeta), the scalar field of the normal estimate
template <typename T, int MOD>
__device__ __forceinline__ T modulus(const T (&z)[8])
{
    T x = z[0] * z[0];
    x = dfma(z[1], z[1], x);
    x = dfma(z[2], z[2], x);
    x = dfma(z[3], z[3], x);
    if (MOD == 0) {
        x = dfma(z[4], z[4], x);
        x = dfma(z[5], z[5], x);
        x = dfma(z[6], z[6], x);
        x = dfma(z[7], z[7], x);
    }
    return x;
}

// Escape-time classification of one sample per lane, all 32 lanes in step.
// Every lane runs the same straight-line iteration each trip; a lane that has
// escaped keeps iterating (its result is no longer used) so that no lane ever
// diverges.  The trip loop ends when no lane in the warp is still bounded, or at
// max_iter.  `part` = the lane has a sample.  Returns the escape count in
// 1..max_iter, or 0 when the sample stayed bounded for max_iter steps.  With
// RECHECK, `marginal` reports whether any tested modulus lay within F.margin of
// R^2 (up to and including the escaping step).
template <typename T, int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ int classify_lockstep(T (&z)[8], const FrameT<T> &F, int max_iter, bool part,
                                                 bool &marginal)
{
    bool alive = part;
    bool mg = false;
    int cnt = 0;
    T sp = dq_sp<T>(z);
    T w[8];
    // two steps per trip, z -> w -> z, with the escape test after each
    for (int n = 0; n < max_iter; n += 2) {
        T m = dq_iter<T, SQ, MOD>(z, w, sp, F.c);
        if (RECHECK) mg = mg || (alive && fabs(m - F.R2) <= F.margin);
        alive = alive && (m <= F.R2);
        cnt += alive ? 1 : 0;
        if (!__any_sync(0xffffffffu, alive) || n + 1 >= max_iter) break;
        m = dq_iter<T, SQ, MOD>(w, z, sp, F.c);
        if (RECHECK) mg = mg || (alive && fabs(m - F.R2) <= F.margin);
        alive = alive && (m <= F.R2);
        cnt += alive ? 1 : 0;
        if (!__any_sync(0xffffffffu, alive)) break;
    }
    if (RECHECK && part && max_iter > late_step<MOD>() && cnt >= late_step<MOD>()) mg = true;  // a long orbit
    marginal = mg;
    return cnt >= max_iter ? 0 : cnt + 1;
}

// The modulus of zeta given its sp = r1^2 + r2^2 + r3^2: the tail of dq_iter.
template <typename T, int MOD>
__device__ __forceinline__ T modulus_sp(const T (&z)[8], T sp)
{
    T x = dfma(z[0], z[0], sp);
    if (MOD == 0) {
        x = dfma(z[4], z[4], x);
        x = dfma(z[5], z[5], x);
        x = dfma(z[6], z[6], x);
        x = dfma(z[7], z[7], x);
    }
    return x;
}

// classify_lockstep for a sample given by its first iterate zeta_1 (the FP32
// march forms zeta_1 directly, see first_iterate_coeffs): step 1 tests
// modulus(zeta_1), the remaining max_iter - 1 steps iterate from zeta_1.
template <typename T, int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ int classify_lockstep_it1(T (&z)[8], const FrameT<T> &F, int max_iter, bool part,
                                                     bool &marginal)
{
    bool alive = part;
    T sp = dq_sp<T>(z);
    T m = modulus_sp<T, MOD>(z, sp);
    bool mg = RECHECK && alive && fabs(m - F.R2) <= F.margin;
    alive = alive && (m <= F.R2);
    int cnt = alive ? 1 : 0;
    T w[8];
    if (__any_sync(0xffffffffu, alive)) {
        for (int n = 1; n < max_iter; n += 2) {
            m = dq_iter<T, SQ, MOD>(z, w, sp, F.c);
            if (RECHECK) mg = mg || (alive && fabs(m - F.R2) <= F.margin);
            alive = alive && (m <= F.R2);
            cnt += alive ? 1 : 0;
            if (!__any_sync(0xffffffffu, alive) || n + 1 >= max_iter) break;
            m = dq_iter<T, SQ, MOD>(w, z, sp, F.c);
            if (RECHECK) mg = mg || (alive && fabs(m - F.R2) <= F.margin);
            alive = alive && (m <= F.R2);
            cnt += alive ? 1 : 0;
            if (!__any_sync(0xffffffffu, alive)) break;
        }
    }
    if (RECHECK && part && max_iter > late_step<MOD>() && cnt >= late_step<MOD>()) mg = true;  // a long orbit
    marginal = mg;
    return cnt >= max_iter ? 0 : cnt + 1;
}

// Scalar (per-thread) classification with early exit, for FP64 rechecks and
// re-renders.  Same return convention.
// Scalar form of dq_iter2_axis_first: the first step of a sample whose
// components 3..7 are zero; same operations and order as dq_iter, so the same
// result.  zi and z may be the same array.
template <typename T, int MOD>
__device__ __forceinline__ T dq_iter_axis_first(const T (&zi)[8], T (&z)[8], T &sp, const T (&c)[8])
{
    const T r0 = zi[0], r1 = zi[1], r2 = zi[2];
    const T tr0 = r0 + r0;
    z[0] = dfma(r0, r0, dfma(sp, T(-1), c[0]));
    z[1] = dfma(tr0, r1, c[1]);
    z[2] = dfma(tr0, r2, c[2]);
#pragma unroll
    for (int i = 3; i < 8; ++i) z[i] = c[i];
    sp = dq_sp<T>(z);
    T x = dfma(z[0], z[0], sp);
    if (MOD == 0) {
        x = dfma(z[4], z[4], x);
        x = dfma(z[5], z[5], x);
        x = dfma(z[6], z[6], x);
        x = dfma(z[7], z[7], x);
    }
    return x;
}

// classify_scalar for a sample of an axis-aligned slice (components 3..7 of z
// zero): the first step takes dq_iter_axis_first, the same iterate as dq_iter
// there.  Same return convention.
template <typename T, int SQ, int MOD>
__device__ __forceinline__ int classify_scalar_axis(T (&z)[8], const FrameT<T> &F, int max_iter)
{
    T sp = dfma(z[2], z[2], z[1] * z[1]);
    if (max_iter < 1) return 0;
    if (dq_iter_axis_first<T, MOD>(z, z, sp, F.c) > F.R2) return 1;
    for (int n = 2; n <= max_iter; ++n)
        if (dq_iter<T, SQ, MOD>(z, z, sp, F.c) > F.R2) return n;
    return 0;
}

// classify_scalar that also reports whether any tested modulus, up to and
// including the escaping one, lay within F.margin of R^2.
template <typename T, int SQ, int MOD>
__device__ __forceinline__ int classify_scalar_margin(T (&z)[8], const FrameT<T> &F, int max_iter, bool &marginal)
{
    T sp = dq_sp<T>(z);
    marginal = false;
    const bool long_orbits = max_iter > late_step<MOD>();  // steps past late_step count as marginal
    for (int n = 1; n <= max_iter; ++n) {
        const T m = dq_iter<T, SQ, MOD>(z, z, sp, F.c);
        marginal = marginal || fabs(m - F.R2) <= F.margin || (long_orbits && n > late_step<MOD>());
        if (m > F.R2) return n;
    }
    return 0;
}

template <typename T, int SQ, int MOD>
__device__ __forceinline__ int classify_scalar(T (&z)[8], const FrameT<T> &F, int max_iter)
{
    T sp = dq_sp<T>(z);
    for (int n = 1; n <= max_iter; ++n)
        if (dq_iter<T, SQ, MOD>(z, z, sp, F.c) > F.R2) return n;
    return 0;
}

// ---------------------------------------------------------------------------
// Paired form: two independent samples per thread, one in each half of a
// float2, advanced together by the sm_100+ paired FP32 instructions
// (fma.rn.f32x2, add.rn.f32x2, mul.rn.f32x2).  Per half the arithmetic is
// exactly dq_iter<float>, so both forms round identically.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float2 dq_sp2(const float2 (&z)[8])
{
    return f2fma(z[3], z[3], f2fma(z[2], z[2], f2mul(z[1], z[1])));
}

// ---------------------------------------------------------------------------
// First-iterate form of a march sample.  Along a ray the slice point is
// zeta_0(t) = A + t D (A the slice image of the eye, D = E d), so its first
// iterate zeta_1(t) = zeta_0(t)^2 + c is a quadratic in t.  With t* = -(A . D)
// (the parameter where the slice line passes closest to the slice origin;
// |D| = 1) and A' = A + t* D:
//     zeta_1 = Q0 + s (Q1 + s Q2),   s = t - t*,
//     Q0 = A'^2 + c,   Q1 = A' D + D A',   Q2 = D^2
// (products in the frame's square mode).  Shifting the origin to A' keeps the
// three terms of the size of zeta_1 near the set instead of |A|^2, so the form
// rounds like the direct square.  The coefficients are formed once per ray;
// each sample then costs two FMAs per component instead of forming zeta_0 and
// squaring it.  Written once over the lane type V (float, or float2 for two
// rays per lane) so that the scalar and paired kernels round identically.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return f2fma(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return f2mul(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return f2add(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

// o = a^2 (Eq. quatsq) for quaternions a[0..3], scalar first
template <typename V>
__device__ __forceinline__ void quat_sq_v(const V *a, V *o)
{
    const V ta0 = vadd(a[0], a[0]);
    V q = vmul(a[1], a[1]);
    q = vfma(a[2], a[2], q);
    q = vfma(a[3], a[3], q);
    o[0] = vfma(a[0], a[0], vneg(q));
    o[1] = vmul(ta0, a[1]);
    o[2] = vmul(ta0, a[2]);
    o[3] = vmul(ta0, a[3]);
}

// o = a b + b a = 2 (a0 b0 - av . bv, a0 bv + b0 av) (the cross products cancel)
template <typename V>
__device__ __forceinline__ void quat_sym_v(const V *a, const V *b, V *o)
{
    V q = vmul(a[1], b[1]);
    q = vfma(a[2], b[2], q);
    q = vfma(a[3], b[3], q);
    const V r = vfma(a[0], b[0], vneg(q));
    o[0] = vadd(r, r);
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        const V t = vfma(a[0], b[i], vmul(b[0], a[i]));
        o[i] = vadd(t, t);
    }
}

// o = a^2 in square mode SQ (0 algebraic: (a_r^2, a_r a_d + a_d a_r);
// 1 component-wise: (a_r^2, a_d^2))
template <typename V, int SQ>
__device__ __forceinline__ void dq_sq_v(const V (&a)[8], V (&o)[8])
{
    quat_sq_v(a, o);
    if (SQ == 0)
        quat_sym_v(a, a + 4, o + 4);
    else
        quat_sq_v(a + 4, o + 4);
}

// o = a b + b a in square mode SQ (the cross term of (a + s b)^2)
template <typename V, int SQ>
__device__ __forceinline__ void dq_sym_v(const V (&a)[8], const V (&b)[8], V (&o)[8])
{
    quat_sym_v(a, b, o);
    if (SQ == 0) {
        V u[4], w[4];
        quat_sym_v(a, b + 4, u);
        quat_sym_v(a + 4, b, w);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[4 + i] = vadd(u[i], w[i]);
    } else {
        quat_sym_v(a + 4, b + 4, o + 4);
    }
}

// Coefficients of the first-iterate form of one ray (see above); dot = A . D,
// so s = t + dot.
template <typename V, int SQ>
__device__ __forceinline__ void first_iterate_coeffs(const V (&A)[8], const V (&D)[8], const V (&c)[8], V &dot,
                                                     V (&Q0)[8], V (&Q1)[8], V (&Q2)[8])
{
    V d = vmul(A[0], D[0]);
#pragma unroll
    for (int i = 1; i < 8; ++i) d = vfma(A[i], D[i], d);
    dot = d;
    const V ts = vneg(d);
    V Ap[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) Ap[i] = vfma(ts, D[i], A[i]);
    dq_sq_v<V, SQ>(Ap, Q0);
#pragma unroll
    for (int i = 0; i < 8; ++i) Q0[i] = vadd(Q0[i], c[i]);
    dq_sym_v<V, SQ>(Ap, D, Q1);
    dq_sq_v<V, SQ>(D, Q2);
}

// zeta_1 at s: Q0 + s (Q1 + s Q2), components [0, n)
template <typename V, int n>
__device__ __forceinline__ void first_iterate(V s, const V (&Q0)[8], const V (&Q1)[8], const V (&Q2)[8], V (&z)[8])
{
#pragma unroll
    for (int i = 0; i < n; ++i) z[i] = vfma(s, vfma(s, Q2[i], Q1[i]), Q0[i]);
}

template <int SQ, int MOD>
__device__ __forceinline__ float2 dq_iter2(const float2 (&zi)[8], float2 (&z)[8], float2 &sp, const PairConsts &P)
{
    const float2 r0 = zi[0], r1 = zi[1], r2 = zi[2], r3 = zi[3];
    const float2 d0 = zi[4], d1 = zi[5], d2 = zi[6], d3 = zi[7];
    const float2 tr0 = f2add(r0, r0);
    z[0] = f2fma(r0, r0, f2fma(sp, P.neg1, P.c[0]));
    z[1] = f2fma(tr0, r1, P.c[1]);
    z[2] = f2fma(tr0, r2, P.c[2]);
    z[3] = f2fma(tr0, r3, P.c[3]);
    const float2 td0 = f2add(d0, d0);
    if (SQ == 0) {
        float2 q = f2mul(r1, d1);
        q = f2fma(r2, d2, q);
        q = f2fma(r3, d3, q);
        z[4] = f2fma(q, P.neg2, f2fma(tr0, d0, P.c[4]));
        z[5] = f2fma(tr0, d1, f2fma(td0, r1, P.c[5]));
        z[6] = f2fma(tr0, d2, f2fma(td0, r2, P.c[6]));
        z[7] = f2fma(tr0, d3, f2fma(td0, r3, P.c[7]));
    } else {
        float2 q = f2mul(d1, d1);
        q = f2fma(d2, d2, q);
        q = f2fma(d3, d3, q);
        z[4] = f2fma(q, P.neg1, f2fma(d0, d0, P.c[4]));
        z[5] = f2fma(td0, d1, P.c[5]);
        z[6] = f2fma(td0, d2, P.c[6]);
        z[7] = f2fma(td0, d3, P.c[7]);
    }
    sp = dq_sp2(z);
    float2 x = f2fma(z[0], z[0], sp);
    if (MOD == 0) {
        x = f2fma(z[4], z[4], x);
        x = f2fma(z[5], z[5], x);
        x = f2fma(z[6], z[6], x);
        x = f2fma(z[7], z[7], x);
    }
    return x;
}

// First step of the paired iteration for a sample of an axis-aligned slice:
// components 3..7 of the input are zero (the slice origin and basis vanish
// there), so every product with them is zero and the step reduces to the terms
// below.  The operations kept are those of dq_iter2 in the same order, so the
// iterate is the same (up to the sign of zero components, which no later
// modulus or comparison sees).  Both squaring modes give the same step here.
// Returns a = z0^2 + sp only: the rest of the modulus adds the fixed c4..c7
// terms, and the step's tests use the thresholds on a in P (t_esc, t_mlo,
// t_mhi), which decide exactly as the full modulus would.
__device__ __forceinline__ float2 dq_iter2_axis_first(const float2 (&zi)[8], float2 (&z)[8], float2 &sp,
                                                      const PairConsts &P)
{
    const float2 r0 = zi[0], r1 = zi[1], r2 = zi[2];
    const float2 tr0 = f2add(r0, r0);
    z[0] = f2fma(r0, r0, f2fma(sp, P.neg1, P.c[0]));
    z[1] = f2fma(tr0, r1, P.c[1]);
    z[2] = f2fma(tr0, r2, P.c[2]);
#pragma unroll
    for (int i = 3; i < 8; ++i) z[i] = P.c[i];
    sp = f2fma(z[3], z[3], f2fma(z[2], z[2], f2mul(z[1], z[1])));
    return f2fma(z[0], z[0], sp);
}

// Lockstep classification of two samples per lane (halves .x and .y), same
// conventions as classify_lockstep.  On entry aa / ab say whether each half has
// a sample; on return they say whether it stayed bounded (inside), and ca / cb
// hold the number of steps it stayed bounded (escape count - 1, or max_iter).
// AXIS: the samples lie in an axis-aligned slice, only z[0..2] are set on entry
// (components 3..7 are zero) and the first step takes dq_iter2_axis_first.
// `live` (warp-uniform) is false when the warp's last vote saw no bounded half:
// then no half is inside.
// RECHECK: dm returns, per half with a sample, the smallest distance from R^2
// of its tested moduli, up to and including the escaping one, and of the
// moduli of the steps the half takes after escaping while other halves of the
// warp are still bounded: the sample is marginal when dm <= P.margin_t.  Each
// later step costs one paired subtraction and a minimum per half; taking the
// minimum only while the half is bounded cost 4 % of the march.  A modulus
// after the escape that comes within the band (about 2e-4 of the flagged
// samples) only adds a recheck, which confirms the FP32 count, so the flagged
// set, but not the result, depends on how many samples share the warp's
// steps.  The axis-form first step
// measures |a - a_c| instead (see PairConsts), for every half alike, so a half
// without a sample must carry a z whose first step is far outside the band
// (march2_tile gives it a ray parameter of 1e18: a = +inf).  Without AXIS such
// a half keeps dm = +inf.
template <int SQ, int MOD, bool RECHECK, bool AXIS = false>
__device__ __forceinline__ void classify_lockstep2(float2 (&z)[8], const PairConsts &P, float R2, int max_iter,
                                                   bool &aa, bool &ab, int &ca, int &cb, float2 &dm, bool &live)
{
    const float inf = __int_as_float(0x7f800000);
    dm = make_float2(inf, inf);
    bool v = true;
    int na = 0, nb = 0;
    float2 sp = AXIS ? f2fma(z[2], z[2], f2mul(z[1], z[1])) : dq_sp2(z);
    float2 w[8];
    // one tested step: escape test, count, and the margin distance while bounded
    auto test = [&](float2 x) {
        if (RECHECK) {
            const float2 u = f2add(x, P.negR2);
            dm.x = fminf(dm.x, fabsf(u.x));
            dm.y = fminf(dm.y, fabsf(u.y));
        }
        aa = aa && (x.x <= R2);
        ab = ab && (x.y <= R2);
        na += aa ? 1 : 0;
        nb += ab ? 1 : 0;
    };
    int n0 = 0;
    if constexpr (AXIS) {  // the first trip, peeled so that its first step takes the axis form
        n0 = max_iter;
        const float2 a = dq_iter2_axis_first(z, w, sp, P);  // tests on a (see PairConsts)
        if (RECHECK) {  // a half without a sample must come with a far-away z (see march2_tile)
            const float2 u = f2add(a, P.neg_ac);
            dm.x = fabsf(u.x);
            dm.y = fabsf(u.y);
        }
        aa = aa && (a.x < P.t_esc);
        ab = ab && (a.y < P.t_esc);
        na += aa ? 1 : 0;
        nb += ab ? 1 : 0;
        v = __any_sync(0xffffffffu, aa || ab);
        if (v && max_iter > 1) {
            test(dq_iter2<SQ, MOD>(w, z, sp, P));
            v = __any_sync(0xffffffffu, aa || ab);
            if (v) n0 = 2;
        }
    }
    // two steps per trip, z -> w -> z, with the escape test after each
    for (int n = n0; n < max_iter; n += 2) {
        test(dq_iter2<SQ, MOD>(z, w, sp, P));
        v = __any_sync(0xffffffffu, aa || ab);
        if (!v || n + 1 >= max_iter) break;
        test(dq_iter2<SQ, MOD>(w, z, sp, P));
        v = __any_sync(0xffffffffu, aa || ab);
        if (!v) break;
    }
    if (RECHECK && MOD == 1 && max_iter > late_step<MOD>()) {  // a long orbit is always rechecked
        if (na >= late_step<MOD>()) dm.x = 0.f;
        if (nb >= late_step<MOD>()) dm.y = 0.f;
    }
    live = v;
    ca = na;
    cb = nb;
}

// classify_lockstep2 for samples given by their first iterate zeta_1 (the
// first-iterate form of a general slice, see first_iterate_coeffs): step 1 is
// the escape test of zeta_1, the remaining max_iter - 1 steps iterate from it.
// Same outputs and recheck distance as classify_lockstep2.
template <int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ void classify_lockstep2_it1(float2 (&z)[8], const PairConsts &P, float R2, int max_iter,
                                                       bool &aa, bool &ab, int &ca, int &cb, float2 &dm, bool &live)
{
    const float inf = __int_as_float(0x7f800000);
    dm = make_float2(inf, inf);
    int na = 0, nb = 0;
    float2 sp = dq_sp2(z);
    float2 w[8];
    auto test = [&](float2 x) {
        if (RECHECK) {
            const float2 u = f2add(x, P.negR2);
            dm.x = fminf(dm.x, fabsf(u.x));
            dm.y = fminf(dm.y, fabsf(u.y));
        }
        aa = aa && (x.x <= R2);
        ab = ab && (x.y <= R2);
        na += aa ? 1 : 0;
        nb += ab ? 1 : 0;
    };
    {
        float2 x = f2fma(z[0], z[0], sp);
        if (MOD == 0) {
            x = f2fma(z[4], z[4], x);
            x = f2fma(z[5], z[5], x);
            x = f2fma(z[6], z[6], x);
            x = f2fma(z[7], z[7], x);
        }
        test(x);
    }
    bool v = __any_sync(0xffffffffu, aa || ab);
    if (v) {
        // two steps per trip, z -> w -> z, with the escape test after each
        for (int n = 1; n < max_iter; n += 2) {
            test(dq_iter2<SQ, MOD>(z, w, sp, P));
            v = __any_sync(0xffffffffu, aa || ab);
            if (!v || n + 1 >= max_iter) break;
            test(dq_iter2<SQ, MOD>(w, z, sp, P));
            v = __any_sync(0xffffffffu, aa || ab);
            if (!v) break;
        }
    }
    if (RECHECK && MOD == 1 && max_iter > late_step<MOD>()) {  // a long orbit is always rechecked
        if (na >= late_step<MOD>()) dm.x = 0.f;
        if (nb >= late_step<MOD>()) dm.y = 0.f;
    }
    live = v;
    ca = na;
    cb = nb;
}

// classify_lockstep2 (AXIS form) for two samples of each of a lane's two rays
// at once: set 0 (z; halves a, b) and set 1 (y; halves a2, b2).  The sets
// advance in the same steps with one vote per step over all four halves, so
// per sample the vote, the loop and the round's bookkeeping cost half as
// much, and the two sets' independent chains hide each other's latency.  Each
// half's outputs are those classify_lockstep2 gives it alone (the same
// operations on its own values; a half only stops counting earlier or later).
template <int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ void classify_lockstep4_axis(float2 (&z)[8], float2 (&y)[8], const PairConsts &P, float R2,
                                                        int max_iter, bool &aa, bool &ab, bool &aa2, bool &ab2,
                                                        int &ca, int &cb, int &ca2, int &cb2, float2 &dm,
                                                        float2 &dm2, bool &live)
{
    bool v = true;
    int na = 0, nb = 0, na2 = 0, nb2 = 0;
    float2 sp = f2fma(z[2], z[2], f2mul(z[1], z[1]));
    float2 sq = f2fma(y[2], y[2], f2mul(y[1], y[1]));
    float2 w[8], u[8];
    auto test = [&](float2 x, float2 x2) {
        if (RECHECK) {  // as in classify_lockstep2: every step, no predicate
            const float2 e = f2add(x, P.negR2), e2 = f2add(x2, P.negR2);
            dm.x = fminf(dm.x, fabsf(e.x));
            dm.y = fminf(dm.y, fabsf(e.y));
            dm2.x = fminf(dm2.x, fabsf(e2.x));
            dm2.y = fminf(dm2.y, fabsf(e2.y));
        }
        aa = aa && (x.x <= R2);
        ab = ab && (x.y <= R2);
        aa2 = aa2 && (x2.x <= R2);
        ab2 = ab2 && (x2.y <= R2);
        na += aa ? 1 : 0;
        nb += ab ? 1 : 0;
        na2 += aa2 ? 1 : 0;
        nb2 += ab2 ? 1 : 0;
    };
    int n0 = max_iter;
    {
        const float2 a = dq_iter2_axis_first(z, w, sp, P);
        const float2 a2 = dq_iter2_axis_first(y, u, sq, P);
        if (RECHECK) {  // halves without a sample come with a far-away z (see march2_tile)
            const float2 e = f2add(a, P.neg_ac), e2 = f2add(a2, P.neg_ac);
            dm = make_float2(fabsf(e.x), fabsf(e.y));
            dm2 = make_float2(fabsf(e2.x), fabsf(e2.y));
        }
        aa = aa && (a.x < P.t_esc);
        ab = ab && (a.y < P.t_esc);
        aa2 = aa2 && (a2.x < P.t_esc);
        ab2 = ab2 && (a2.y < P.t_esc);
        na += aa ? 1 : 0;
        nb += ab ? 1 : 0;
        na2 += aa2 ? 1 : 0;
        nb2 += ab2 ? 1 : 0;
        v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
        if (v && max_iter > 1) {
            test(dq_iter2<SQ, MOD>(w, z, sp, P), dq_iter2<SQ, MOD>(u, y, sq, P));
            v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
            if (v) n0 = 2;
        }
    }
    for (int n = n0; n < max_iter; n += 2) {
        test(dq_iter2<SQ, MOD>(z, w, sp, P), dq_iter2<SQ, MOD>(y, u, sq, P));
        v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
        if (!v || n + 1 >= max_iter) break;
        test(dq_iter2<SQ, MOD>(w, z, sp, P), dq_iter2<SQ, MOD>(u, y, sq, P));
        v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
        if (!v) break;
    }
    if (RECHECK && MOD == 1 && max_iter > late_step<MOD>()) {  // a long orbit is always rechecked
        if (na >= late_step<MOD>()) dm.x = 0.f;
        if (nb >= late_step<MOD>()) dm.y = 0.f;
        if (na2 >= late_step<MOD>()) dm2.x = 0.f;
        if (nb2 >= late_step<MOD>()) dm2.y = 0.f;
    }
    live = v;
    ca = na;
    cb = nb;
    ca2 = na2;
    cb2 = nb2;
}

// classify_lockstep2_it1 for two samples of each of a lane's two rays at once
// (see classify_lockstep4_axis): z and y hold the first iterates of samples
// k and k + 1.  Same outputs per half as classify_lockstep2_it1.
template <int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ void classify_lockstep4_it1(float2 (&z)[8], float2 (&y)[8], const PairConsts &P, float R2,
                                                       int max_iter, bool &aa, bool &ab, bool &aa2, bool &ab2,
                                                       int &ca, int &cb, int &ca2, int &cb2, float2 &dm,
                                                       float2 &dm2, bool &live)
{
    const float inf = __int_as_float(0x7f800000);
    dm = dm2 = make_float2(inf, inf);
    int na = 0, nb = 0, na2 = 0, nb2 = 0;
    float2 sp = dq_sp2(z), sq = dq_sp2(y);
    float2 w[8], u[8];
    auto test = [&](float2 x, float2 x2) {
        if (RECHECK) {  // as in classify_lockstep2: every step, no predicate
            const float2 e = f2add(x, P.negR2), e2 = f2add(x2, P.negR2);
            dm.x = fminf(dm.x, fabsf(e.x));
            dm.y = fminf(dm.y, fabsf(e.y));
            dm2.x = fminf(dm2.x, fabsf(e2.x));
            dm2.y = fminf(dm2.y, fabsf(e2.y));
        }
        aa = aa && (x.x <= R2);
        ab = ab && (x.y <= R2);
        aa2 = aa2 && (x2.x <= R2);
        ab2 = ab2 && (x2.y <= R2);
        na += aa ? 1 : 0;
        nb += ab ? 1 : 0;
        na2 += aa2 ? 1 : 0;
        nb2 += ab2 ? 1 : 0;
    };
    {
        float2 x = f2fma(z[0], z[0], sp), x2 = f2fma(y[0], y[0], sq);
        if (MOD == 0) {
#pragma unroll
            for (int i = 4; i < 8; ++i) {
                x = f2fma(z[i], z[i], x);
                x2 = f2fma(y[i], y[i], x2);
            }
        }
        test(x, x2);
    }
    bool v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
    if (v) {
        for (int n = 1; n < max_iter; n += 2) {
            test(dq_iter2<SQ, MOD>(z, w, sp, P), dq_iter2<SQ, MOD>(y, u, sq, P));
            v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
            if (!v || n + 1 >= max_iter) break;
            test(dq_iter2<SQ, MOD>(w, z, sp, P), dq_iter2<SQ, MOD>(u, y, sq, P));
            v = __any_sync(0xffffffffu, aa || ab || aa2 || ab2);
            if (!v) break;
        }
    }
    if (RECHECK && MOD == 1 && max_iter > late_step<MOD>()) {  // a long orbit is always rechecked
        if (na >= late_step<MOD>()) dm.x = 0.f;
        if (nb >= late_step<MOD>()) dm.y = 0.f;
        if (na2 >= late_step<MOD>()) dm2.x = 0.f;
        if (nb2 >= late_step<MOD>()) dm2.y = 0.f;
    }
    live = v;
    ca = na;
    cb = nb;
    ca2 = na2;
    cb2 = nb2;
}

}  // namespace dqj
