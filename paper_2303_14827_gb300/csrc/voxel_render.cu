// voxel_render.cu -- image of a voxel occupancy grid from the scene camera
// (Fig. voxels: the paper sets its ray-traced image beside renders of 50^3 and
// 100^3 voxel grids).  The grid is drawn as the union of its occupied cells,
// each a closed axis-aligned cube of the march box; a pixel shows the first cube
// its camera ray crosses, found by walking the ray cell by cell (Amanatides and
// Woo's grid traversal, 1987): start in the cell of the box entry point, then
// step to the neighbour across whichever cell face the ray reaches first.
//
// One pixel per thread, 16 x 8 pixel tiles per CTA, so a warp's rays walk
// neighbouring cells and share the occupancy bytes through L1/L2.  The camera
// ray, the start cell and the hit depth are FP64; the per-step choice of the
// next face compares FP32 face distances against a rigorous error bound and
// falls back to FP64 within it, so every choice is the one an FP64 walk makes
// except where two faces lie within FP64 rounding of each other (FP64 runs at
// 1/64 of the FP32 rate on this part).  A ray crosses at most 3 g - 2 cells.
#include "render_common.cuh"
#include "runtime.h"

namespace dqj {

namespace {

constexpr int kVrTileW = 16, kVrTileH = 8;
static_assert(kVrTileW * kVrTileH == kBlock, "one pixel per thread");

// Grid-uniform FP64 constants, computed once on the host.
struct GridGeom {
    double size[3];      // cell edge per axis, (box_max - box_min) / g
    double inv_size[3];  // g / (box_max - box_min)
    double lo_e[3];      // box_min - eye
    double hi_e[3];      // box_max - eye
    double sxa, sxb;     // screen x = (x + 0.5) sxa + sxb  (pinhole camera)
    double sya, syb;     // screen y = (y + 0.5) sya + syb
};

// Hit pixel: the entered face's outward normal (-d when the eye is inside the
// hit cube) and the ambient, diffuse and specular terms of Eq. phong, shaded in
// FP32 (the FP32 frame constants; the normal is exact and the depth FP64).
__device__ __forceinline__ void write_face_hit(const FrameDesc &fd, int x, int y, int iter, double depth, int axis,
                                               const double (&d)[3])
{
    const FrameT<float> &F = fd.f;
    float n[3], df[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        df[b] = (float)d[b];
        n[b] = axis < 0 ? -df[b] : (axis == b ? (d[b] > 0.0 ? -1.f : 1.f) : 0.f);
    }
    float ndl = n[0] * F.light[0] + n[1] * F.light[1] + n[2] * F.light[2];
    float spec = 0.f;
    if (F.ks > 0.f && ndl > 0.f) {  // reflected light r = 2n(n.l) - l against v = -d
        const float rv = -((2.f * ndl * n[0] - F.light[0]) * df[0] + (2.f * ndl * n[1] - F.light[1]) * df[1] +
                           (2.f * ndl * n[2] - F.light[2]) * df[2]);
        if (rv > 0.f) spec = F.ks * powf(rv, F.shin);
    }
    ndl = ndl > 0.f ? ndl : 0.f;
    float v = F.ka + F.kd * ndl + spec;
    v = v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
    const int64_t o = (int64_t)y * fd.pitch + x;
    if (fd.iter) fd.iter[o] = iter;
    if (fd.depth) fd.depth[o] = (float)depth;
    if (fd.normal) {
        fd.normal[3 * o + 0] = n[0];
        fd.normal[3 * o + 1] = n[1];
        fd.normal[3 * o + 2] = n[2];
    }
    if (fd.rgba)
        *reinterpret_cast<uchar4 *>(fd.rgba + 4 * o) =
            make_uchar4(to_u8(v * F.albedo[0]), to_u8(v * F.albedo[1]), to_u8(v * F.albedo[2]), 255);
}

__global__ void __launch_bounds__(kBlock) voxel_render_kernel(const __grid_constant__ FrameDesc fd,
                                                              const uint8_t *__restrict__ occ, int g,
                                                              const __grid_constant__ GridGeom geo)
{
    const FrameT<double> &F = fd.d;
    const int x = blockIdx.x * kVrTileW + (int)(threadIdx.x % kVrTileW);
    const int y = blockIdx.y * kVrTileH + (int)(threadIdx.x / kVrTileW);
    if (x >= fd.W || y >= fd.H) return;
    // FP64 camera ray and slab clip (the pinhole formula of the march), with
    // reciprocals instead of divisions: an FP64 division or square root is a
    // sequence of FP64 operations, and FP64 runs at 1/64 of the FP32 rate here,
    // so this per-pixel setup, not the walk, bounds small grids.
    double d[3];
    {
        const double sx = fma((double)x + 0.5, geo.sxa, geo.sxb);
        const double sy = fma((double)y + 0.5, geo.sya, geo.syb);
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = F.fwd[a] + sx * F.right[a] + sy * F.upv[a];
        const double il = rsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] *= il;
    }
    // Per axis: the ray reaches cell plane k (bmin + k size) at
    // t = base + k sd, base = (bmin - eye) / d, sd = size / d.  The box is
    // entered through the face of the axis whose slab is entered last (none
    // when the eye is inside the box and t_in is clipped to 0).
    double b64[3], d64[3], t0 = -tinf<double>(), t1 = tinf<double>();
    int axis = -1;
    bool in_box = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (F.eye[a] < F.bmin[a] || F.eye[a] > F.bmax[a]) in_box = false;
            b64[a] = d64[a] = 0.0;
            continue;
        }
        const double id = __drcp_rn(d[a]);
        const double ta = geo.lo_e[a] * id, tb = geo.hi_e[a] * id;
        b64[a] = ta;
        d64[a] = geo.size[a] * id;
        const double te = ta < tb ? ta : tb, tx = ta < tb ? tb : ta;
        if (te > t0) {
            t0 = te;
            axis = a;
        }
        t1 = tx < t1 ? tx : t1;
    }
    if (t0 < 0.0) {
        t0 = 0.0;
        axis = -1;
    }
    const double t_in = t0;
    if (!in_box || !(t0 < t1)) {
        write_miss<double>(fd, x, y, 0);
        return;
    }
    // The walk compares the FP32 values m = fma(k, sd, base) of the face
    // distances; each lies within E = 2^-21 (g |sd| + |base|) of its FP64
    // value (three roundings of at most 2^-24 relative each, with a factor 2 to
    // spare), so when the two nearest faces differ by more than the sum of the
    // bounds the FP32 order is the FP64 order; otherwise the choice is made in
    // FP64.
    int i0, i1, i2, k0, k1, k2, s0, s1, s2;
    float b32[3], d32[3], m[3];
    float tol = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double p = F.eye[a] + t_in * d[a];
        double c = floor((p - F.bmin[a]) * geo.inv_size[a]);
        c = c < 0.0 ? 0.0 : (c > (double)(g - 1) ? (double)(g - 1) : c);
        const int ia = (int)c;
        const int sa = d[a] > 0.0 ? 1 : (d[a] < 0.0 ? -1 : 0);
        const int ka = ia + (sa > 0 ? 1 : 0);
        b32[a] = (float)b64[a];
        d32[a] = (float)d64[a];
        // an axis whose FP32 face distances overflow (|d| below ~1e-38) crosses
        // no cell plane inside the box, like an axis the ray runs parallel to
        if (sa != 0 && isfinite(d32[a]) && isfinite(b32[a])) {
            m[a] = fmaf((float)ka, d32[a], b32[a]);
            tol += 4.76837158203125e-7f * ((float)g * fabsf(d32[a]) + fabsf(b32[a]));
        } else {
            m[a] = tinf<float>();
        }
        if (a == 0) { i0 = ia; k0 = ka; s0 = sa; }
        if (a == 1) { i1 = ia; k1 = ka; s1 = sa; }
        if (a == 2) { i2 = ia; k2 = ka; s2 = sa; }
    }
    // Each step moves to the neighbour across the nearest face.  The step is
    // written without branches: neighbouring lanes choose different axes, and
    // a three-way branch would run all three paths for the warp.  A cell
    // records how it was entered (code = axis | plane << 2 for a step across
    // cell plane `plane` of `axis`; 3 for the start cell, entered at the box
    // entry through face axis0).  g <= 1024, so cell indices fit in 32 bits.
    // (Measured and not kept: walking a few cells ahead to batch their loads,
    // plane indices carried as floats, and the FP64 choice out of line; each
    // was slower.)
    const int axis0 = axis;
    float m0 = m[0], m1 = m[1], m2 = m[2];
    const uint32_t gu = (uint32_t)g;
    const int32_t st0 = s0, st1 = s1 * g, st2 = s2 * g * g;
    uint32_t lin = ((uint32_t)i2 * gu + (uint32_t)i1) * gu + (uint32_t)i0;
    uint32_t code = 3u;
    int n = 0;  // cells tested
    bool hit = false;
    const int max_cells = 3 * g;  // a ray crosses at most 3 g - 2 cells
    while (n < max_cells) {
        ++n;
        if (__ldg(occ + lin)) {
            hit = true;
            break;
        }
        // the nearest face, ties to the lower axis
        int a = (m0 <= m1 && m0 <= m2) ? 0 : (m1 <= m2 ? 1 : 2);
        const float lo = fminf(m0, fminf(m1, m2));
        const float mid = fmaxf(fminf(m0, m1), fminf(fmaxf(m0, m1), m2));
        if (mid - lo <= tol) {  // too close for FP32: decide in FP64
            const double t0 = m[0] != tinf<float>() ? fma((double)k0, d64[0], b64[0]) : tinf<double>();
            const double t1 = m[1] != tinf<float>() ? fma((double)k1, d64[1], b64[1]) : tinf<double>();
            const double t2 = m[2] != tinf<float>() ? fma((double)k2, d64[2], b64[2]) : tinf<double>();
            a = (t0 <= t1 && t0 <= t2) ? 0 : (t1 <= t2 ? 1 : 2);
        }
        const bool x0 = a == 0, x1 = a == 1, x2 = a == 2;
        i0 += x0 ? s0 : 0;
        i1 += x1 ? s1 : 0;
        i2 += x2 ? s2 : 0;
        const bool out = ((unsigned)i0 >= gu) | ((unsigned)i1 >= gu) | ((unsigned)i2 >= gu);
        const int kc = x0 ? k0 : (x1 ? k1 : k2);
        const int sa = x0 ? s0 : (x1 ? s1 : s2);
        code = (uint32_t)a | ((uint32_t)kc << 2);
        k0 += x0 ? s0 : 0;
        k1 += x1 ? s1 : 0;
        k2 += x2 ? s2 : 0;
        lin += (uint32_t)(x0 ? st0 : (x1 ? st1 : st2));
        const float mk = fmaf((float)(kc + sa), x0 ? d32[0] : (x1 ? d32[1] : d32[2]), x0 ? b32[0] : (x1 ? b32[1] : b32[2]));
        m0 = x0 ? mk : m0;
        m1 = x1 ? mk : m1;
        m2 = x2 ? mk : m2;
        if (out) break;  // the cell just tested was the last inside the grid
    }
    if (!hit) {
        write_miss<double>(fd, x, y, n);
        return;
    }
    const int sa = (int)(code & 3u);
    const double kc = (double)(code >> 2);
    double t = t_in;  // the start cell is entered at the box entry
    if (sa == 0) t = fma(kc, d64[0], b64[0]);
    if (sa == 1) t = fma(kc, d64[1], b64[1]);
    if (sa == 2) t = fma(kc, d64[2], b64[2]);
    write_face_hit(fd, x, y, n, t, sa == 3 ? axis0 : sa, d);
}

}  // namespace

}  // namespace dqj

using namespace dqj;

extern "C" dqj_status dqj_render_voxels(dqj_ctx *ctx, const dqj_params *p, int32_t grid_n, const uint8_t *occupancy,
                                        const dqj_outputs *out, void *cuda_stream)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        dqj_status s = validate(p);
        if (s != DQJ_OK) return s;
        if (grid_n < 1 || grid_n > DQJ_VOXEL_MAX_GRID)
            return fail(DQJ_ERR_INVALID, "grid_n must be in 1.." + std::to_string(DQJ_VOXEL_MAX_GRID));
        if (!occupancy) return fail(DQJ_ERR_INVALID, "occupancy is NULL");
        s = check_outputs(*p, out);
        if (s != DQJ_OK) return s;
        if (ctx->device == DQJ_DEVICE_MOCK) return fail(DQJ_ERR_INVALID, "a mock context cannot render voxels");
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(e, "render_voxels: cudaSetDevice");
        FrameDesc fd;
        derive_frame(*p, fd, 8, 8);
        fd.pitch = out->pitch_px;
        fd.iter = out->iter;
        fd.depth = out->depth;
        fd.normal = out->normal;
        fd.rgba = out->rgba;
        GridGeom geo;
        for (int a = 0; a < 3; ++a) {
            const double ext = p->box_max[a] - p->box_min[a];
            geo.size[a] = ext / (double)grid_n;
            geo.inv_size[a] = (double)grid_n / ext;
            geo.lo_e[a] = p->box_min[a] - p->eye[a];
            geo.hi_e[a] = p->box_max[a] - p->eye[a];
        }
        // the pinhole map of the FP64 camera, 2 (x + 0.5) / W - 1 and
        // 1 - 2 (y + 0.5) / H scaled by tan(fov_y / 2) (and the aspect for x)
        geo.sxa = 2.0 * fd.d.th * fd.d.aspect / (double)p->width;
        geo.sxb = -fd.d.th * fd.d.aspect;
        geo.sya = -2.0 * fd.d.th / (double)p->height;
        geo.syb = fd.d.th;
        const dim3 grid((unsigned)((p->width + kVrTileW - 1) / kVrTileW), (unsigned)((p->height + kVrTileH - 1) / kVrTileH));
        voxel_render_kernel<<<grid, kBlock, 0, static_cast<cudaStream_t>(cuda_stream)>>>(fd, occupancy, grid_n, geo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "render_voxels: launch");
        return DQJ_OK;
    });
}
