/*
 * dqj_oracle.c -- plain, slow, FP64 CPU oracle for the dual-quaternion Julia
 * isosurface renderer (Kenwright, "Dual-Quaternion Julia Fractals").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is compared
 * against.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with the
 * CUDA path, and the CUDA path never calls it.
 *
 * Everything is IEEE double, built with -O2 -ffp-contract=off (no fused
 * multiply-add, no fast-math), so every formula below is evaluated exactly in the
 * order written.  Quaternion and dual-quaternion products are the GENERAL
 * products of the paper's appendix; the iteration squares a dual quaternion by
 * multiplying it with itself (no specialised square), so that a reader can check
 * each step against the paper by eye.
 *
 * Conventions (readings of places where the paper is silent or garbled):
 *  - A quaternion is stored scalar first, [s, v] = (q0, q1, q2, q3) (appendix,
 *    quaternion definition; Eq. quatsq also puts the real component first).
 *  - A dual quaternion zeta = q_r + q_d eps is stored as 8 doubles (q_r | q_d)
 *    (appendix, dual-quaternion definition).
 *  - Squaring (Method, "Dual-Quaternion Julia Sets"): square mode 0 (ALGEBRAIC)
 *    is zeta*zeta with the appendix product, i.e. q_r^2 + (q_r q_d + q_d q_r) eps,
 *    which respects eps^2 = 0 (Introduction, dual numbers).  Square mode 1
 *    (PAPER_COMPONENTWISE) squares each quaternion on its own, q_r^2 + q_d^2 eps,
 *    as the equation beside Eq. dqjulia2 is written.
 *  - Modulus used by the escape test: modulus mode 0 (EUCLID8) is
 *    |q_r|^2 + |q_d|^2, the appendix quaternion magnitude applied to both halves;
 *    mode 1 (DUALNUM) is |q_r|^2, the modulus of a dual number (Introduction:
 *    ||a + b eps|| = |a|) applied to zeta zeta* (appendix magnitude).
 *  - Escape (Method, Julia sets and "Practical Considerations"): after each
 *    update n = 1..max_iter the sample escapes at the first n with
 *    modulus > R^2 (strict).  No escape by max_iter means "inside".
 *  - Slice (Method, "Dimension Reduction"): a 3-D scene point p maps to
 *    zeta0 = origin + p_x E0 + p_y E1 + p_z E2, with E an orthonormal 3-frame in
 *    R^8.  The default frame is the first three unit vectors.
 *  - Ray marching (Method, "Ray-Marching"): fixed-step march over the ray's
 *    intersection with an axis-aligned box, N+1 samples t_k = t_in + k*Delta,
 *    Delta = (t_out - t_in)/N; the first inside sample ends the march, then B
 *    bisection steps refine the crossing.
 *  - Normal (Method, "Lighting/Illumination"): central differences of the scalar
 *    field F(p) = modulus(zeta_{n*}(p)) along the scene axes, n* the escape count
 *    of the final outside bisection end, iterated exactly n* times.  When any of
 *    the six values exceeds 2^100 or is not finite (a neighbour that escaped
 *    long before n*), or the gradient is zero, the normal is -d.
 *  - Shading (Eq. phong): ambient plus diffuse terms only.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------- */
/* Scene description, owned by the oracle (the CUDA path has its own).        */
/* ------------------------------------------------------------------------- */
typedef struct {
    double c[8];
    double slice_origin[8];
    double slice_basis[3][8];
    double eye[3], target[3], up[3];
    double fov_y_deg;
    int32_t width, height, max_iter;
    double escape_radius;
    int32_t march_steps, bisect_steps;
    double normal_h;
    double box_min[3], box_max[3];
    double light_dir[3];
    double k_ambient, k_diffuse;
    double albedo[3];
    int32_t square_mode;  /* 0 ALGEBRAIC, 1 PAPER_COMPONENTWISE */
    int32_t modulus_mode; /* 0 EUCLID8, 1 DUALNUM */
    double k_specular;    /* Eq. phong k_s (0: no specular term) */
    double shininess;     /* Eq. phong exponent s */
    int32_t traversal;    /* 0 fixed-step march + bisection, 1 distance-estimate sphere tracing */
    int32_t de_max_steps; /* DE: step limit per ray */
    double de_epsilon;    /* DE: a sample whose estimate is below this is a hit */
    double de_step_scale; /* DE: step = scale * estimate */
    double de_bound_radius; /* DE: bounding sphere about the origin (0: box only) */
} or_scene;

/* Per-pixel trace, for tests that check the march and bisection logic. */
typedef struct {
    int32_t box_hit;      /* ray meets the box with t_in < t_out               */
    int32_t hit;          /* some march sample is inside                        */
    int32_t k_first;      /* index of the first inside march sample, or -1      */
    int32_t n_star;       /* escape count used for the normal field            */
    int32_t esc_max;      /* max escape count over the (outside) march samples  */
    int32_t pad;
    double t_in, t_out, delta;
    double lo, hi, depth;
    double o[3], d[3];
    int64_t class_iters;  /* DQ iterations with escape test (march + bisection) */
    int64_t normal_iters; /* DQ iterations of the six normal evaluations        */
    int32_t de_steps;     /* DE: samples taken                                  */
    int32_t pad2;
} or_trace;

/* ------------------------------------------------------------------------- */
/* Quaternion operations (appendix, "Quaternion Operations").                 */
/* ------------------------------------------------------------------------- */

/* q1 q2 = [s1 s2 - v1.v2, s1 v2 + s2 v1 + v1 x v2]  (appendix, multiplication) */
void or_quat_mul(const double *a, const double *b, double *out)
{
    double s1 = a[0], s2 = b[0];
    const double *v1 = a + 1, *v2 = b + 1;
    double dot = v1[0] * v2[0] + v1[1] * v2[1] + v1[2] * v2[2];
    double cx = v1[1] * v2[2] - v1[2] * v2[1];
    double cy = v1[2] * v2[0] - v1[0] * v2[2];
    double cz = v1[0] * v2[1] - v1[1] * v2[0];
    double r[4];
    r[0] = s1 * s2 - dot;
    r[1] = s1 * v2[0] + s2 * v1[0] + cx;
    r[2] = s1 * v2[1] + s2 * v1[1] + cy;
    r[3] = s1 * v2[2] + s2 * v1[2] + cz;
    memcpy(out, r, sizeof r);
}

/* q1 + q2 = [s1 + s2, v1 + v2]  (appendix, addition) */
static void quat_add(const double *a, const double *b, double *out)
{
    for (int i = 0; i < 4; ++i) out[i] = a[i] + b[i];
}

/* q* = [s, -v]  (appendix, conjugate) */
static void quat_conj(const double *a, double *out)
{
    out[0] = a[0];
    out[1] = -a[1];
    out[2] = -a[2];
    out[3] = -a[3];
}

/* ||q||^2 = s^2 + |v|^2  (appendix, magnitude, squared) */
static double quat_norm2(const double *a)
{
    return a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
}

/* q1 . q2  (appendix, dot product) */
double or_quat_dot(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

/* ------------------------------------------------------------------------- */
/* Dual-quaternion operations (appendix, "Dual-Quaternion Operations"), with  */
/* the two typos of that list read as follows: the real part of a sum is      */
/* q_r1 + q_r2, and the real part of a product is q_r1 q_r2.                  */
/* ------------------------------------------------------------------------- */

/* zeta1 + zeta2 = (q_r1 + q_r2) + (q_d1 + q_d2) eps */
void or_dq_add(const double *a, const double *b, double *out)
{
    quat_add(a, b, out);
    quat_add(a + 4, b + 4, out + 4);
}

/* zeta1 zeta2 = q_r1 q_r2 + (q_r1 q_d2 + q_d1 q_r2) eps */
void or_dq_mul(const double *a, const double *b, double *out)
{
    double rr[4], rd[4], dr[4], r[8];
    or_quat_mul(a, b, rr);
    or_quat_mul(a, b + 4, rd);
    or_quat_mul(a + 4, b, dr);
    memcpy(r, rr, sizeof rr);
    quat_add(rd, dr, r + 4);
    memcpy(out, r, sizeof r);
}

/* zeta* = q_r* + q_d* eps */
void or_dq_conj(const double *a, double *out)
{
    double r[8];
    quat_conj(a, r);
    quat_conj(a + 4, r + 4);
    memcpy(out, r, sizeof r);
}

/* ||zeta|| = zeta zeta*  (appendix, magnitude): returned as a dual quaternion. */
void or_dq_magnitude(const double *a, double *out)
{
    double cj[8];
    or_dq_conj(a, cj);
    or_dq_mul(a, cj, out);
}

/* zeta^2 for the two readings of the Method section (see file header). */
void or_dq_square(const double *z, int square_mode, double *out)
{
    if (square_mode == 1) {
        double r[8];
        or_quat_mul(z, z, r);
        or_quat_mul(z + 4, z + 4, r + 4);
        memcpy(out, r, sizeof r);
    } else {
        or_dq_mul(z, z, out);
    }
}

/* Escape-test modulus for the two readings (see file header). */
double or_modulus(const double *z, int modulus_mode)
{
    if (modulus_mode == 1) return quat_norm2(z);
    return quat_norm2(z) + quat_norm2(z + 4);
}

/* n plain steps of Eq. dqjulia2, zeta <- zeta^2 + c, with no escape test. */
void or_dq_julia(const double *z0, const double *c, int n, int square_mode, double *out)
{
    double z[8], sq[8];
    memcpy(z, z0, sizeof z);
    for (int i = 0; i < n; ++i) {
        or_dq_square(z, square_mode, sq);
        or_dq_add(sq, c, z);
    }
    memcpy(out, z, sizeof z);
}

/* n plain steps of the quaternion Julia map, Eq. dqjulia, q <- q^2 + c. */
void or_quat_julia(const double *q0, const double *c, int n, double *out)
{
    double q[4], sq[4];
    memcpy(q, q0, sizeof q);
    for (int i = 0; i < n; ++i) {
        or_quat_mul(q, q, sq);
        quat_add(sq, c, q);
    }
    memcpy(out, q, sizeof q);
}

/*
 * Escape-time classification of one sample (Method, Eq. dqjulia2 and
 * "Practical Considerations").  Returns the escape count n in 1..max_iter, or 0
 * when the sample has not escaped after max_iter steps (inside).  *m_last gets
 * the modulus after the last step taken; *iters the number of steps taken.
 */
int or_classify(const double *z0, const double *c, int max_iter, double escape_radius,
                int square_mode, int modulus_mode, double *m_last, int64_t *iters)
{
    double z[8], sq[8];
    double r2 = escape_radius * escape_radius;
    double m = or_modulus(z0, modulus_mode);
    memcpy(z, z0, sizeof z);
    for (int n = 1; n <= max_iter; ++n) {
        or_dq_square(z, square_mode, sq);
        or_dq_add(sq, c, z);
        m = or_modulus(z, modulus_mode);
        if (m > r2) {
            if (m_last) *m_last = m;
            if (iters) *iters += n;
            return n;
        }
    }
    if (m_last) *m_last = m;
    if (iters) *iters += max_iter;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Scene geometry.                                                            */
/* ------------------------------------------------------------------------- */

static void v3_sub(const double *a, const double *b, double *o)
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}

static double v3_dot(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void v3_cross(const double *a, const double *b, double *o)
{
    double r[3];
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
    memcpy(o, r, sizeof r);
}

static void v3_normalize(double *a)
{
    double len = sqrt(v3_dot(a, a));
    a[0] /= len;
    a[1] /= len;
    a[2] /= len;
}

/*
 * Pinhole camera.  The paper only names the view vector of Eq. phong; this is
 * the reading used: forward f = normalize(target - eye), right =
 * normalize(f x up), true up = right x f; vertical field of view fov_y, aspect
 * width/height; the ray passes through the pixel centre (i + 0.5, j + 0.5), row 0
 * at the top, column 0 at the left.  Returns 0.
 */
int or_camera_ray(const or_scene *s, int i, int j, double *o, double *d)
{
    double f[3], r[3], u[3];
    v3_sub(s->target, s->eye, f);
    v3_normalize(f);
    v3_cross(f, s->up, r);
    v3_normalize(r);
    v3_cross(r, f, u);
    double th = tan(0.5 * s->fov_y_deg * (M_PI / 180.0));
    double aspect = (double)s->width / (double)s->height;
    double sx = (2.0 * ((double)i + 0.5) / (double)s->width - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * ((double)j + 0.5) / (double)s->height) * th;
    for (int a = 0; a < 3; ++a) d[a] = f[a] + sx * r[a] + sy * u[a];
    v3_normalize(d);
    o[0] = s->eye[0];
    o[1] = s->eye[1];
    o[2] = s->eye[2];
    return 0;
}

/*
 * Slab clip of the ray o + t d against [box_min, box_max], t >= 0.  Returns 1 and
 * the interval when t_in < t_out, else 0.  An axis with d = 0 constrains nothing
 * when the origin lies within that slab, and misses otherwise.
 */
int or_box_clip(const or_scene *s, const double *o, const double *d, double *t_in, double *t_out)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < s->box_min[a] || o[a] > s->box_max[a]) return 0;
            continue;
        }
        double ta = (s->box_min[a] - o[a]) / d[a];
        double tb = (s->box_max[a] - o[a]) / d[a];
        if (ta > tb) {
            double tmp = ta;
            ta = tb;
            tb = tmp;
        }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t0 < 0.0) t0 = 0.0;
    *t_in = t0;
    *t_out = t1;
    return t0 < t1;
}

/* Dimension reduction by a 3-D slice (Method, "Dimension Reduction"). */
void or_slice_point(const or_scene *s, const double *p, double *z0)
{
    for (int i = 0; i < 8; ++i)
        z0[i] = s->slice_origin[i] + p[0] * s->slice_basis[0][i] + p[1] * s->slice_basis[1][i] +
                p[2] * s->slice_basis[2][i];
}

static int classify_point(const or_scene *s, const double *p, int64_t *iters)
{
    double z0[8];
    or_slice_point(s, p, z0);
    return or_classify(z0, s->c, s->max_iter, s->escape_radius, s->square_mode, s->modulus_mode,
                       NULL, iters);
}

static void ray_point(const double *o, const double *d, double t, double *p)
{
    p[0] = o[0] + t * d[0];
    p[1] = o[1] + t * d[1];
    p[2] = o[2] + t * d[2];
}

/* Scalar field of the normal estimate: modulus of zeta_{n} at p, n plain steps. */
static double normal_field(const or_scene *s, const double *p, int n, int64_t *iters)
{
    double z0[8], zn[8];
    or_slice_point(s, p, z0);
    or_dq_julia(z0, s->c, n, s->square_mode, zn);
    *iters += n;
    return or_modulus(zn, s->modulus_mode);
}

/* Largest normal-field value used for a gradient: 2^100 (exact in float and
 * double).  Larger or non-finite values select the fallback normal -d. */
#define NORMAL_FMAX 1267650600228229401496703205376.0

/* ------------------------------------------------------------------------- */
/* One pixel: camera ray, box clip, march, bisection, normal, shading.        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t iter;
    double depth;
    double normal[3];
    uint8_t rgba[4];
} pixel_out;

static uint8_t to_u8(double v)
{
    double x = floor(255.0 * v + 0.5);
    if (x < 0.0) x = 0.0;
    if (x > 255.0) x = 255.0;
    return (uint8_t)x;
}

/*
 * Distance estimate at a scene point p (Method, "Ray-Marching", Eq. distfract2,
 * with the derivative recurrence of Eq. distfract read as
 * |zeta'_{n+1}| = 2 |zeta_n| |zeta'_n|, |zeta'_0| = 1).  Iterates from the slice
 * image of p until the modulus exceeds R^2 at step n, and returns n with
 * *dist = 0.5 |zeta_n| / |zeta'_n| ln |zeta_n|, |zeta| = sqrt(modulus).  Returns 0
 * (inside, *dist = 0) when no escape happens within max_iter steps.
 */
int or_de_distance(const or_scene *s, const double *p, double *dist, int64_t *iters)
{
    double z[8], sq[8];
    double r2 = s->escape_radius * s->escape_radius;
    double dr = 1.0;
    or_slice_point(s, p, z);
    for (int n = 1; n <= s->max_iter; ++n) {
        dr = 2.0 * sqrt(or_modulus(z, s->modulus_mode)) * dr;
        or_dq_square(z, s->square_mode, sq);
        or_dq_add(sq, s->c, z);
        double m = or_modulus(z, s->modulus_mode);
        if (m > r2) {
            double a = sqrt(m);
            if (iters) *iters += n;
            *dist = 0.5 * a / dr * log(a);
            return n;
        }
    }
    if (iters) *iters += s->max_iter;
    *dist = 0.0;
    return 0;
}

/* Sphere tracing along the ray (Method, "Ray-Marching"): from the entry into
 * the box (and the bounding sphere, when its radius is positive), sample,
 * stop at an inside sample or one whose estimate is below de_epsilon (a hit
 * at that sample), else advance by de_step_scale times the estimate; a ray
 * that leaves the volume or runs out of steps misses.  Sets t->hit, t->depth,
 * t->n_star (escape count at the hit sample, max_iter when inside) and
 * t->esc_max (the largest escape count over the samples). */
static void de_trace(const or_scene *s, or_trace *t)
{
    double t0 = t->t_in, t1 = t->t_out;
    if (s->de_bound_radius > 0.0) {
        double b = v3_dot(t->o, t->d);
        double c = v3_dot(t->o, t->o) - s->de_bound_radius * s->de_bound_radius;
        double disc = b * b - c;
        if (!(disc > 0.0)) return;
        double q = sqrt(disc);
        if (-b - q > t0) t0 = -b - q;
        if (-b + q < t1) t1 = -b + q;
        if (!(t0 < t1)) return;
    }
    double tt = t0, p[3], dist;
    for (int step = 0; step < s->de_max_steps && tt <= t1; ++step) {
        ray_point(t->o, t->d, tt, p);
        int n = or_de_distance(s, p, &dist, &t->class_iters);
        t->de_steps += 1;
        if (n == 0 || dist < s->de_epsilon) {
            t->hit = 1;
            t->depth = tt;
            t->n_star = n == 0 ? s->max_iter : n;
            if (n != 0 && n > t->esc_max) t->esc_max = n;
            return;
        }
        if (n > t->esc_max) t->esc_max = n;
        tt += s->de_step_scale * dist;
    }
}

static void render_pixel(const or_scene *s, int i, int j, pixel_out *po, or_trace *tr)
{
    or_trace t;
    memset(&t, 0, sizeof t);
    t.k_first = -1;
    or_camera_ray(s, i, j, t.o, t.d);

    po->iter = 0;
    po->depth = INFINITY;
    po->normal[0] = po->normal[1] = po->normal[2] = 0.0;
    po->rgba[0] = po->rgba[1] = po->rgba[2] = po->rgba[3] = 0;

    t.box_hit = or_box_clip(s, t.o, t.d, &t.t_in, &t.t_out);
    if (!t.box_hit) {
        if (tr) *tr = t;
        return;
    }

    int n_star;
    if (s->traversal == 1) {
        de_trace(s, &t);
        if (!t.hit) {
            po->iter = t.esc_max;
            if (tr) *tr = t;
            return;
        }
        n_star = t.n_star;
        goto shade;
    }

    /* March: N+1 samples in order, stop at the first inside one. */
    int n_steps = s->march_steps;
    t.delta = (t.t_out - t.t_in) / (double)n_steps;
    int esc_max = 0, n_prev = 0;
    double p[3];
    for (int k = 0; k <= n_steps; ++k) {
        double tk = t.t_in + (double)k * t.delta;
        ray_point(t.o, t.d, tk, p);
        int n = classify_point(s, p, &t.class_iters);
        if (n == 0) {
            t.k_first = k;
            break;
        }
        if (n > esc_max) esc_max = n;
        n_prev = n;
    }
    t.esc_max = esc_max;

    if (t.k_first < 0) {
        po->iter = esc_max;
        if (tr) *tr = t;
        return;
    }
    t.hit = 1;

    /* Bisection of the first outside -> inside bracket. */
    if (t.k_first == 0) {
        t.lo = t.hi = t.depth = t.t_in;
        n_star = s->max_iter;
    } else {
        double lo = t.t_in + (double)(t.k_first - 1) * t.delta;
        double hi = t.t_in + (double)t.k_first * t.delta;
        int n_lo = n_prev;
        for (int b = 0; b < s->bisect_steps; ++b) {
            double mid = lo + 0.5 * (hi - lo);
            ray_point(t.o, t.d, mid, p);
            int n = classify_point(s, p, &t.class_iters);
            if (n == 0) {
                hi = mid;
            } else {
                lo = mid;
                n_lo = n;
            }
        }
        t.lo = lo;
        t.hi = hi;
        t.depth = lo + 0.5 * (hi - lo);
        n_star = n_lo;
    }
    t.n_star = n_star;
shade:
    po->iter = n_star;
    po->depth = t.depth;

    /* Normal: central differences of F along the scene axes.  Overflow guard
     * (the paper gives none): when any of the six field values exceeds
     * NORMAL_FMAX = 2^100 or is not finite, the normal is -d. */
    double ph[3], g[3];
    int guard = 0;
    ray_point(t.o, t.d, t.depth, ph);
    for (int a = 0; a < 3; ++a) {
        double pp[3] = {ph[0], ph[1], ph[2]};
        double pm[3] = {ph[0], ph[1], ph[2]};
        pp[a] += s->normal_h;
        pm[a] -= s->normal_h;
        double fp = normal_field(s, pp, n_star, &t.normal_iters);
        double fm = normal_field(s, pm, n_star, &t.normal_iters);
        if (!(fp <= NORMAL_FMAX) || !(fm <= NORMAL_FMAX)) guard = 1;
        g[a] = fp - fm;
    }
    double gl = sqrt(v3_dot(g, g));
    if (guard || !(gl > 0.0)) {
        po->normal[0] = -t.d[0];
        po->normal[1] = -t.d[1];
        po->normal[2] = -t.d[2];
    } else {
        po->normal[0] = g[0] / gl;
        po->normal[1] = g[1] / gl;
        po->normal[2] = g[2] / gl;
    }

    /* Shading, Eq. phong: ambient, diffuse and (when k_s > 0) specular terms
     * with unit light intensities.  The specular term uses the reflected light
     * r = 2 n (n.l) - l and the unit vector to the eye v = -d, and counts only
     * when the light is in front (n.l > 0) and r.v > 0. */
    double l[3] = {s->light_dir[0], s->light_dir[1], s->light_dir[2]};
    v3_normalize(l);
    double ndl = v3_dot(po->normal, l);
    double spec = 0.0;
    if (s->k_specular > 0.0 && ndl > 0.0) {
        double r[3], rv = 0.0;
        for (int a = 0; a < 3; ++a) r[a] = 2.0 * ndl * po->normal[a] - l[a];
        for (int a = 0; a < 3; ++a) rv -= r[a] * t.d[a];
        if (rv > 0.0) spec = s->k_specular * pow(rv, s->shininess);
    }
    if (ndl < 0.0) ndl = 0.0;
    double v = s->k_ambient + s->k_diffuse * ndl + spec;
    if (v < 0.0) v = 0.0;
    if (v > 1.0) v = 1.0;
    po->rgba[0] = to_u8(v * s->albedo[0]);
    po->rgba[1] = to_u8(v * s->albedo[1]);
    po->rgba[2] = to_u8(v * s->albedo[2]);
    po->rgba[3] = 255;
    if (tr) *tr = t;
}

/* Trace of one pixel, for tests. */
void or_trace_pixel(const or_scene *s, int i, int j, or_trace *tr)
{
    pixel_out po;
    render_pixel(s, i, j, &po, tr);
}

/* ------------------------------------------------------------------------- */
/* Whole images and pixel lists on a pool of threads.                          */
/* ------------------------------------------------------------------------- */
typedef struct {
    const or_scene *s;
    const int64_t *pix; /* NULL: all pixels, row-major */
    int64_t npix;
    int32_t *iter;
    double *depth, *normal;
    uint8_t *rgba;
    int64_t *pix_iters; /* optional per-output class iterations */
    atomic_llong next;
    atomic_llong class_iters, normal_iters;
} job;

enum { CHUNK = 64 };

static void *worker(void *arg)
{
    job *jb = (job *)arg;
    int64_t ci = 0, ni = 0;
    for (;;) {
        int64_t start = atomic_fetch_add(&jb->next, CHUNK);
        if (start >= jb->npix) break;
        int64_t end = start + CHUNK < jb->npix ? start + CHUNK : jb->npix;
        for (int64_t q = start; q < end; ++q) {
            int64_t lin = jb->pix ? jb->pix[q] : q;
            int i = (int)(lin % jb->s->width), j = (int)(lin / jb->s->width);
            pixel_out po;
            or_trace tr;
            render_pixel(jb->s, i, j, &po, &tr);
            ci += tr.class_iters;
            ni += tr.normal_iters;
            if (jb->iter) jb->iter[q] = po.iter;
            if (jb->depth) jb->depth[q] = po.depth;
            if (jb->normal) memcpy(jb->normal + 3 * q, po.normal, sizeof po.normal);
            if (jb->rgba) memcpy(jb->rgba + 4 * q, po.rgba, sizeof po.rgba);
            if (jb->pix_iters) jb->pix_iters[q] = tr.class_iters;
        }
    }
    atomic_fetch_add(&jb->class_iters, ci);
    atomic_fetch_add(&jb->normal_iters, ni);
    return NULL;
}

/* Number of worker threads a call with nthreads <= 0 uses. */
int or_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static int run_job(job *jb, int nthreads)
{
    if (nthreads <= 0) nthreads = or_default_threads();
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[started], NULL, worker, jb) != 0) break;
        ++started;
    }
    worker(jb);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return started + 1;
}

/*
 * Render pixels.  pix == NULL renders the whole width x height image in
 * row-major order (npix ignored); otherwise output q belongs to linear pixel
 * index pix[q] = row * width + col.  Output arrays may be NULL.  normal is 3
 * doubles per output, rgba 4 bytes.  Returns the number of threads used;
 * *class_iters / *normal_iters get the DQ iteration totals.
 */
int or_render(const or_scene *s, const int64_t *pix, int64_t npix, int nthreads, int32_t *iter,
              double *depth, double *normal, uint8_t *rgba, int64_t *pix_iters,
              int64_t *class_iters, int64_t *normal_iters)
{
    job jb;
    memset(&jb, 0, sizeof jb);
    jb.s = s;
    jb.pix = pix;
    jb.npix = pix ? npix : (int64_t)s->width * (int64_t)s->height;
    jb.iter = iter;
    jb.depth = depth;
    jb.normal = normal;
    jb.rgba = rgba;
    jb.pix_iters = pix_iters;
    atomic_init(&jb.next, 0);
    atomic_init(&jb.class_iters, 0);
    atomic_init(&jb.normal_iters, 0);
    int used = run_job(&jb, nthreads);
    if (class_iters) *class_iters = atomic_load(&jb.class_iters);
    if (normal_iters) *normal_iters = atomic_load(&jb.normal_iters);
    return used;
}

/* ------------------------------------------------------------------------- */
/* Voxel occupancy grid (Fig. voxels: the paper's voxel prototype).           */
/* The grid has G cells per axis over the march box; cell (i, j, k) is        */
/* classified at its centre p_a = box_min_a + (idx_a + 1/2) (box_max_a -      */
/* box_min_a) / G, mapped into the slice like a ray sample.  Linear index     */
/* (k G + j) G + i, x fastest.  occupancy 1 = inside (no escape by max_iter), */
/* count = escape count (0 inside), as or_classify.                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    const or_scene *s;
    int32_t g;
    const int64_t *idx;
    int64_t n;
    uint8_t *occ;
    int32_t *count;
    atomic_llong next;
    atomic_llong iters;
} vox_job;

void or_voxel_center(const or_scene *s, int32_t g, int64_t lin, double *p)
{
    int64_t i = lin % g, j = (lin / g) % g, k = lin / ((int64_t)g * g);
    int64_t ix[3] = {i, j, k};
    for (int a = 0; a < 3; ++a)
        p[a] = s->box_min[a] + ((double)ix[a] + 0.5) * (s->box_max[a] - s->box_min[a]) / (double)g;
}

static void *vox_worker(void *arg)
{
    vox_job *jb = (vox_job *)arg;
    int64_t it = 0;
    for (;;) {
        int64_t start = atomic_fetch_add(&jb->next, CHUNK);
        if (start >= jb->n) break;
        int64_t end = start + CHUNK < jb->n ? start + CHUNK : jb->n;
        for (int64_t q = start; q < end; ++q) {
            double p[3];
            or_voxel_center(jb->s, jb->g, jb->idx ? jb->idx[q] : q, p);
            int n = classify_point(jb->s, p, &it);
            if (jb->occ) jb->occ[q] = n == 0 ? 1 : 0;
            if (jb->count) jb->count[q] = n;
        }
    }
    atomic_fetch_add(&jb->iters, it);
    return NULL;
}

/*
 * Classify voxel cells.  idx == NULL classifies the whole g^3 grid (n ignored);
 * otherwise output q belongs to linear cell index idx[q].  Returns the number of
 * threads used; *iters gets the DQ iteration total.
 */
int or_voxelize(const or_scene *s, int32_t g, const int64_t *idx, int64_t n, int nthreads, uint8_t *occ,
                int32_t *count, int64_t *iters)
{
    vox_job jb;
    memset(&jb, 0, sizeof jb);
    jb.s = s;
    jb.g = g;
    jb.idx = idx;
    jb.n = idx ? n : (int64_t)g * g * g;
    jb.occ = occ;
    jb.count = count;
    atomic_init(&jb.next, 0);
    atomic_init(&jb.iters, 0);
    if (nthreads <= 0) nthreads = or_default_threads();
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[started], NULL, vox_worker, &jb) != 0) break;
        ++started;
    }
    vox_worker(&jb);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    if (iters) *iters = atomic_load(&jb.iters);
    return started + 1;
}

/* ------------------------------------------------------------------------- */
/* Image of a voxel grid from the scene camera (Fig. voxels compares the     */
/* ray-traced image with renders of 50^3 and 100^3 grids).  Reading: a grid   */
/* is drawn as the union of its occupied cells, each the closed cube          */
/* [box_min + idx s, box_min + (idx + 1) s] per axis, s = (box_max -          */
/* box_min) / G; a pixel shows the first such cube its camera ray crosses.    */
/*   depth  = the ray parameter where the ray enters that cube (t_in of the   */
/*            box when the first cell crossed is occupied); +inf on a miss;   */
/*   normal = outward unit normal of the entered face, -sign(d_a) e_a, a the  */
/*            axis of that face (-d when the eye is inside the hit cube);     */
/*   iter   = cells crossed up to and including the hit cube (all cells       */
/*            crossed inside the box on a miss, 0 when the ray misses the     */
/*            box);                                                           */
/*   rgba   = Eq. phong with that normal, as for the ray-traced image.        */
/* Two forms: the cell-by-cell walk along the ray (Amanatides and Woo's grid  */
/* traversal, 1987) and, for tiny grids, the plain definition: the smallest   */
/* entry parameter over all occupied cubes the ray crosses with positive      */
/* length.                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t iter;
    int32_t axis;   /* axis of the entered face, -1 when the eye is inside the hit cube, -2 on a miss */
    double depth;
    double gap;     /* smallest margin of a floating-point decision of the walk (scene units) */
} vox_hit;

static void vox_shade(const or_scene *s, const double *d, int axis, double *normal, uint8_t *rgba)
{
    if (axis < 0) {
        normal[0] = -d[0];
        normal[1] = -d[1];
        normal[2] = -d[2];
    } else {
        normal[0] = normal[1] = normal[2] = 0.0;
        normal[axis] = d[axis] > 0.0 ? -1.0 : 1.0;
    }
    double l[3] = {s->light_dir[0], s->light_dir[1], s->light_dir[2]};
    v3_normalize(l);
    double ndl = v3_dot(normal, l);
    double spec = 0.0;
    if (s->k_specular > 0.0 && ndl > 0.0) {
        double r[3], rv = 0.0;
        for (int a = 0; a < 3; ++a) r[a] = 2.0 * ndl * normal[a] - l[a];
        for (int a = 0; a < 3; ++a) rv -= r[a] * d[a];
        if (rv > 0.0) spec = s->k_specular * pow(rv, s->shininess);
    }
    if (ndl < 0.0) ndl = 0.0;
    double v = s->k_ambient + s->k_diffuse * ndl + spec;
    if (v < 0.0) v = 0.0;
    if (v > 1.0) v = 1.0;
    rgba[0] = to_u8(v * s->albedo[0]);
    rgba[1] = to_u8(v * s->albedo[1]);
    rgba[2] = to_u8(v * s->albedo[2]);
    rgba[3] = 255;
}

/* Axis whose slab the ray enters last at the box entry (the face it comes in
 * through); -1 when t_in was clipped to 0 (eye inside the box). */
static int box_entry_axis(const or_scene *s, const double *o, const double *d)
{
    double best = -INFINITY;
    int axis = -1;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        double ta = (s->box_min[a] - o[a]) / d[a];
        double tb = (s->box_max[a] - o[a]) / d[a];
        double te = ta < tb ? ta : tb;
        if (te > best) {
            best = te;
            axis = a;
        }
    }
    return best < 0.0 ? -1 : axis;
}

/* The walk: start in the cell that holds the box entry point, then step to the
 * neighbour across whichever cell face the ray reaches first. */
static vox_hit voxel_walk(const or_scene *s, int32_t g, const uint8_t *occ, const double *o, const double *d)
{
    vox_hit h = {0, -2, INFINITY, INFINITY};
    double t_in, t_out;
    if (!or_box_clip(s, o, d, &t_in, &t_out)) return h;
    double size[3], p[3];
    int64_t idx[3], stp[3];
    double tmax[3], tdel[3];
    int entry = box_entry_axis(s, o, d);
    ray_point(o, d, t_in, p);
    for (int a = 0; a < 3; ++a) {
        size[a] = (s->box_max[a] - s->box_min[a]) / (double)g;
        double u = (p[a] - s->box_min[a]) / size[a];
        double f = floor(u);
        if (a != entry) {
            /* margin of the cell choice: distance of the entry point to the
             * nearest cell plane of this axis */
            double m = fabs(u - floor(u + 0.5)) * size[a];
            if (m < h.gap) h.gap = m;
        }
        if (f < 0.0) f = 0.0;
        if (f > (double)(g - 1)) f = (double)(g - 1);
        idx[a] = (int64_t)f;
        if (d[a] > 0.0) {
            stp[a] = 1;
            tmax[a] = (s->box_min[a] + (double)(idx[a] + 1) * size[a] - o[a]) / d[a];
            tdel[a] = size[a] / d[a];
        } else if (d[a] < 0.0) {
            stp[a] = -1;
            tmax[a] = (s->box_min[a] + (double)idx[a] * size[a] - o[a]) / d[a];
            tdel[a] = -size[a] / d[a];
        } else {
            stp[a] = 0;
            tmax[a] = INFINITY;
            tdel[a] = INFINITY;
        }
    }
    int axis = entry;
    double t = t_in;
    for (int64_t n = 1;; ++n) {
        if (occ[(idx[2] * g + idx[1]) * g + idx[0]]) {
            h.iter = (int32_t)n;
            h.axis = axis;
            h.depth = t;
            return h;
        }
        /* next face: the smallest tmax, ties to the lower axis */
        int a = 0;
        for (int b = 1; b < 3; ++b)
            if (tmax[b] < tmax[a]) a = b;
        for (int b = 0; b < 3; ++b)
            if (b != a && tmax[b] - tmax[a] < h.gap) h.gap = tmax[b] - tmax[a];
        idx[a] += stp[a];
        if (idx[a] < 0 || idx[a] >= g) {
            h.iter = (int32_t)n;
            return h;
        }
        t = tmax[a];
        tmax[a] += tdel[a];
        axis = a;
    }
}

/* The plain definition, by brute force over every occupied cube (tiny grids). */
static vox_hit voxel_brute(const or_scene *s, int32_t g, const uint8_t *occ, const double *o, const double *d)
{
    vox_hit h = {0, -2, INFINITY, INFINITY};
    double t_in, t_out;
    if (!or_box_clip(s, o, d, &t_in, &t_out)) return h;
    double size[3];
    for (int a = 0; a < 3; ++a) size[a] = (s->box_max[a] - s->box_min[a]) / (double)g;
    int32_t crossed_before = 0;
    for (int64_t lin = 0; lin < (int64_t)g * g * g; ++lin) {
        int64_t ix[3] = {lin % g, (lin / g) % g, lin / ((int64_t)g * g)};
        double t0 = t_in, t1 = t_out;
        int ax = -1;
        for (int a = 0; a < 3; ++a) {
            double lo = s->box_min[a] + (double)ix[a] * size[a];
            double hi = s->box_min[a] + (double)(ix[a] + 1) * size[a];
            if (d[a] == 0.0) {
                if (o[a] < lo || o[a] > hi) t1 = -INFINITY;
                continue;
            }
            double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
            if (ta > tb) {
                double tmp = ta;
                ta = tb;
                tb = tmp;
            }
            if (ta > t0) {
                t0 = ta;
                ax = a;
            }
            if (tb < t1) t1 = tb;
        }
        if (!(t0 < t1) || !occ[lin]) continue;
        if (t0 < h.depth) {
            h.depth = t0;
            h.axis = ax;
        }
    }
    if (h.axis == -1 && t_in > 0.0) h.axis = box_entry_axis(s, o, d);
    /* cells crossed up to the hit: those whose entry lies before the hit's */
    for (int64_t lin = 0; lin < (int64_t)g * g * g; ++lin) {
        int64_t ix[3] = {lin % g, (lin / g) % g, lin / ((int64_t)g * g)};
        double t0 = t_in, t1 = t_out;
        for (int a = 0; a < 3; ++a) {
            double lo = s->box_min[a] + (double)ix[a] * size[a];
            double hi = s->box_min[a] + (double)(ix[a] + 1) * size[a];
            if (d[a] == 0.0) {
                if (o[a] < lo || o[a] > hi) t1 = -INFINITY;
                continue;
            }
            double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
            if (ta > tb) {
                double tmp = ta;
                ta = tb;
                tb = tmp;
            }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        }
        if (t0 < t1 && t0 <= h.depth) ++crossed_before;
    }
    h.iter = crossed_before;
    return h;
}

typedef struct {
    const or_scene *s;
    int32_t g;
    const uint8_t *occ;
    int brute;
    const int64_t *pix;
    int64_t npix;
    int32_t *iter;
    double *depth, *normal, *gap;
    uint8_t *rgba;
    atomic_llong next;
} vrender_job;

static void *vrender_worker(void *arg)
{
    vrender_job *jb = (vrender_job *)arg;
    for (;;) {
        int64_t start = atomic_fetch_add(&jb->next, CHUNK);
        if (start >= jb->npix) break;
        int64_t end = start + CHUNK < jb->npix ? start + CHUNK : jb->npix;
        for (int64_t q = start; q < end; ++q) {
            int64_t lin = jb->pix ? jb->pix[q] : q;
            int i = (int)(lin % jb->s->width), j = (int)(lin / jb->s->width);
            double o[3], d[3], n[3] = {0.0, 0.0, 0.0};
            uint8_t c[4] = {0, 0, 0, 0};
            or_camera_ray(jb->s, i, j, o, d);
            vox_hit h = jb->brute ? voxel_brute(jb->s, jb->g, jb->occ, o, d)
                                  : voxel_walk(jb->s, jb->g, jb->occ, o, d);
            if (h.axis != -2) vox_shade(jb->s, d, h.axis, n, c);
            if (jb->iter) jb->iter[q] = h.iter;
            if (jb->depth) jb->depth[q] = h.depth;
            if (jb->normal) memcpy(jb->normal + 3 * q, n, sizeof n);
            if (jb->rgba) memcpy(jb->rgba + 4 * q, c, sizeof c);
            if (jb->gap) jb->gap[q] = h.gap;
        }
    }
    return NULL;
}

/*
 * Image of the g^3 occupancy grid occ (linear index (k g + j) g + i) from the
 * scene camera, by the walk (brute = 0) or by the plain definition (brute = 1,
 * tiny grids only).  pix / npix / outputs as or_render; gap (optional) gets, per
 * output, the smallest margin of a floating-point decision the walk took (the
 * cell of the entry point and each choice of the next face), in scene units.
 * Returns the number of threads used.
 */
int or_voxel_render(const or_scene *s, int32_t g, const uint8_t *occ, int brute, const int64_t *pix, int64_t npix,
                    int nthreads, int32_t *iter, double *depth, double *normal, uint8_t *rgba, double *gap)
{
    vrender_job jb;
    memset(&jb, 0, sizeof jb);
    jb.s = s;
    jb.g = g;
    jb.occ = occ;
    jb.brute = brute;
    jb.pix = pix;
    jb.npix = pix ? npix : (int64_t)s->width * (int64_t)s->height;
    jb.iter = iter;
    jb.depth = depth;
    jb.normal = normal;
    jb.rgba = rgba;
    jb.gap = gap;
    atomic_init(&jb.next, 0);
    if (nthreads <= 0) nthreads = or_default_threads();
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[started], NULL, vrender_worker, &jb) != 0) break;
        ++started;
    }
    vrender_worker(&jb);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return started + 1;
}
