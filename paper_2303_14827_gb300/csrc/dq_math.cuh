// dq_math.cuh -- dual-quaternion Julia step, escape modulus and lockstep
// classification on the device, templated on float / double.
//
// A dual quaternion zeta = q_r + q_d eps is kept in 8 registers (q_r | q_d),
// scalar first in each half (appendix, quaternion and dual-quaternion
// definitions).  The square is expanded in closed form instead of the general
// product:
//   ALGEBRAIC (eps^2 = 0, appendix product):
//     q_r^2           = (r0^2 - r1^2 - r2^2 - r3^2, 2 r0 r1, 2 r0 r2, 2 r0 r3)
//                       (Eq. quatsq)
//     q_r q_d + q_d q_r = 2 (r0 d0 - v_r . v_d, r0 v_d + d0 v_r)
//                       (the cross products cancel)
//   PAPER_COMPONENTWISE (the equation printed beside Eq. dqjulia2):
//     q_r^2 + q_d^2 eps, each half by Eq. quatsq.
// The escape test compares the modulus with R^2 (Method, "Practical
// Considerations"); EUCLID8 takes |q_r|^2 + |q_d|^2, DUALNUM |q_r|^2.
#pragma once

#include "dqj_internal.h"

namespace dqj {

__device__ __forceinline__ float dfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return fma(a, b, c); }

// zeta <- zeta^2 + c
template <typename T, int SQ>
__device__ __forceinline__ void dq_step(T (&z)[8], const T (&c)[8])
{
    const T r0 = z[0], r1 = z[1], r2 = z[2], r3 = z[3];
    const T d0 = z[4], d1 = z[5], d2 = z[6], d3 = z[7];
    const T tr0 = r0 + r0;
    T nr0 = dfma(r0, r0, c[0]);
    nr0 = dfma(-r1, r1, nr0);
    nr0 = dfma(-r2, r2, nr0);
    nr0 = dfma(-r3, r3, nr0);
    z[0] = nr0;
    z[1] = dfma(tr0, r1, c[1]);
    z[2] = dfma(tr0, r2, c[2]);
    z[3] = dfma(tr0, r3, c[3]);
    if (SQ == 0) {
        const T td0 = d0 + d0;
        T p = r0 * d0;
        p = dfma(-r1, d1, p);
        p = dfma(-r2, d2, p);
        p = dfma(-r3, d3, p);
        z[4] = dfma(T(2), p, c[4]);
        z[5] = dfma(tr0, d1, dfma(td0, r1, c[5]));
        z[6] = dfma(tr0, d2, dfma(td0, r2, c[6]));
        z[7] = dfma(tr0, d3, dfma(td0, r3, c[7]));
    } else {
        const T td0 = d0 + d0;
        T nd0 = dfma(d0, d0, c[4]);
        nd0 = dfma(-d1, d1, nd0);
        nd0 = dfma(-d2, d2, nd0);
        nd0 = dfma(-d3, d3, nd0);
        z[4] = nd0;
        z[5] = dfma(td0, d1, c[5]);
        z[6] = dfma(td0, d2, c[6]);
        z[7] = dfma(td0, d3, c[7]);
    }
}

// modulus(zeta) - R^2, with R^2 folded into the first term
template <typename T, int MOD>
__device__ __forceinline__ T modulus_minus(const T (&z)[8], T R2)
{
    T x = dfma(z[0], z[0], -R2);
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

template <typename T, int MOD>
__device__ __forceinline__ T modulus(const T (&z)[8])
{
    return modulus_minus<T, MOD>(z, T(0));
}

// Escape-time classification of one sample per lane, all 32 lanes in step.
// Every lane runs the same straight-line iteration each trip; a lane that has
// escaped keeps iterating (its result is no longer used) so that no lane ever
// diverges.  The trip loop ends when no lane in the warp is still bounded, or at
// max_iter.  `part` = the lane has a sample.  Returns the escape count in
// 1..max_iter, or 0 when the sample stayed bounded for max_iter steps.  With
// RECHECK, *marginal reports whether any tested modulus lay within F.margin of
// R^2 (up to and including the escaping step).
template <typename T, int SQ, int MOD, bool RECHECK>
__device__ __forceinline__ int classify_lockstep(T (&z)[8], const FrameT<T> &F, int max_iter, bool part,
                                                 bool &marginal)
{
    bool alive = part;
    bool mg = false;
    int cnt = 0;
    for (int n = 0; n < max_iter; ++n) {
        dq_step<T, SQ>(z, F.c);
        const T x = modulus_minus<T, MOD>(z, F.R2);
        if (RECHECK) mg = mg || (alive && fabs(x) <= F.margin);
        alive = alive && (x <= T(0));
        cnt += alive ? 1 : 0;
        if (!__any_sync(0xffffffffu, alive)) break;
    }
    marginal = mg;
    return cnt >= max_iter ? 0 : cnt + 1;
}

// Scalar (per-thread) classification with early exit, for FP64 rechecks and
// re-renders.  Same return convention.
template <typename T, int SQ, int MOD>
__device__ __forceinline__ int classify_scalar(T (&z)[8], const FrameT<T> &F, int max_iter)
{
    for (int n = 1; n <= max_iter; ++n) {
        dq_step<T, SQ>(z, F.c);
        if (modulus_minus<T, MOD>(z, F.R2) > T(0)) return n;
    }
    return 0;
}

}  // namespace dqj
