// voxel_render.cu -- image of a voxel occupancy grid from the scene camera
// (Fig. voxels: the paper sets its ray-traced image beside renders of 50^3 and
// 100^3 voxel grids).  The grid is drawn as the union of its occupied cells,
// each a closed axis-aligned cube of the march box; a pixel shows the first cube
// its camera ray crosses, found by walking the ray cell by cell (Amanatides and
// Woo's grid traversal, 1987): start in the cell of the box entry point, then
// step to the neighbour across whichever cell face the ray reaches first.
//
// One pixel per thread, 16 x 8 pixel tiles per CTA, so a warp's rays walk
// neighbouring cells and share the occupancy bytes through L1/L2.  The walk runs
// in FP64 (camera ray, face distances and their comparisons), so its choices of
// the next face agree with an FP64 restatement except where two faces lie within
// rounding of each other.  A ray crosses at most 3 g - 2 cells.
#include "render_common.cuh"
#include "runtime.h"

namespace dqj {

namespace {

constexpr int kVrTileW = 16, kVrTileH = 8;
static_assert(kVrTileW * kVrTileH == kBlock, "one pixel per thread");

__global__ void __launch_bounds__(kBlock) voxel_render_kernel(const __grid_constant__ FrameDesc fd,
                                                              const uint8_t *__restrict__ occ, int g)
{
    const FrameT<double> &F = fd.d;
    const int x = blockIdx.x * kVrTileW + (int)(threadIdx.x % kVrTileW);
    const int y = blockIdx.y * kVrTileH + (int)(threadIdx.x / kVrTileW);
    if (x >= fd.W || y >= fd.H) return;
    double d[3], t_in, t_out;
    if (!camera_clip<double>(F, fd.W, fd.H, x, y, d, t_in, t_out)) {
        write_miss<double>(fd, x, y, 0);
        return;
    }
    // Face the ray enters the box through: the axis whose slab it enters last
    // (none when the eye is inside the box and t_in was clipped to 0).
    int axis = -1;
    {
        double best = -tinf<double>();
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] == 0.0) continue;
            const double ta = (F.bmin[a] - F.eye[a]) / d[a], tb = (F.bmax[a] - F.eye[a]) / d[a];
            const double te = ta < tb ? ta : tb;
            if (te > best) {
                best = te;
                axis = a;
            }
        }
        if (best < 0.0) axis = -1;
    }
    int idx[3], stp[3];
    double tmax[3], tdel[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double size = (F.bmax[a] - F.bmin[a]) / (double)g;
        const double p = F.eye[a] + t_in * d[a];
        double f = floor((p - F.bmin[a]) / size);
        f = f < 0.0 ? 0.0 : (f > (double)(g - 1) ? (double)(g - 1) : f);
        idx[a] = (int)f;
        if (d[a] > 0.0) {
            stp[a] = 1;
            tmax[a] = (F.bmin[a] + (double)(idx[a] + 1) * size - F.eye[a]) / d[a];
            tdel[a] = size / d[a];
        } else if (d[a] < 0.0) {
            stp[a] = -1;
            tmax[a] = (F.bmin[a] + (double)idx[a] * size - F.eye[a]) / d[a];
            tdel[a] = -size / d[a];
        } else {
            stp[a] = 0;
            tmax[a] = tinf<double>();
            tdel[a] = tinf<double>();
        }
    }
    // The walk keeps one scalar per axis (no runtime-indexed arrays, which
    // would live in local memory).
    int i0 = idx[0], i1 = idx[1], i2 = idx[2];
    double m0 = tmax[0], m1 = tmax[1], m2 = tmax[2];
    const uint64_t gg = (uint64_t)g;
    double t = t_in;
    const int max_cells = 3 * g;  // each step moves one index one cell towards its exit
    for (int n = 1; n <= max_cells; ++n) {
        const uint64_t lin = ((uint64_t)i2 * gg + (uint64_t)i1) * gg + (uint64_t)i0;
        if (__ldg(occ + lin)) {
            double nv[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) nv[b] = axis == b ? (d[b] > 0.0 ? -1.0 : 1.0) : 0.0;
            shade_write<double>(fd, F, x, y, n, t, nv, axis < 0, d);
            return;
        }
        bool out;
        if (m0 <= m1 && m0 <= m2) {  // the nearest face, ties to the lower axis
            i0 += stp[0];
            out = (unsigned)i0 >= (unsigned)g;
            t = m0;
            m0 += tdel[0];
            axis = 0;
        } else if (m1 <= m2) {
            i1 += stp[1];
            out = (unsigned)i1 >= (unsigned)g;
            t = m1;
            m1 += tdel[1];
            axis = 1;
        } else {
            i2 += stp[2];
            out = (unsigned)i2 >= (unsigned)g;
            t = m2;
            m2 += tdel[2];
            axis = 2;
        }
        if (out) {
            write_miss<double>(fd, x, y, n);
            return;
        }
    }
    write_miss<double>(fd, x, y, max_cells);  // not reached: the walk leaves the grid first
}

}  // namespace

}  // namespace dqj

using namespace dqj;

extern "C" dqj_status dqj_render_voxels(dqj_ctx *ctx, const dqj_params *p, int32_t grid_n, const uint8_t *occupancy,
                                        const dqj_outputs *out, void *cuda_stream)
{
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
    const dim3 grid((unsigned)((p->width + kVrTileW - 1) / kVrTileW), (unsigned)((p->height + kVrTileH - 1) / kVrTileH));
    voxel_render_kernel<<<grid, kBlock, 0, static_cast<cudaStream_t>(cuda_stream)>>>(fd, occupancy, grid_n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "render_voxels: launch");
    return DQJ_OK;
}
