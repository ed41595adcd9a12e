// voxel.cu -- voxel occupancy grid (Fig. voxels, the paper's voxel prototype):
// every cell of a g x g x g grid over the march box is classified at its centre
// like a ray sample (slice map, then the escape-time iteration), giving an
// occupancy byte (1 = no escape by max_iter) and the escape count.
//
// Work unit of the FP32 kernel: a 32 x 2 segment (x = x0 .. x0+31 in rows
// 2 jp and 2 jp + 1 of slice k).  The rows' slice images of (0, y, z) are
// warp-uniform; each lane advances its column's two cells in float2 halves
// with the paired march classification, so a cell costs the same arithmetic
// as a march sample.  Warps claim segments through an atomic counter
// (persistent grid).
// FP64 runs one cell per lane; FP32 + recheck queues cells whose modulus came
// within the margin of R^2 and re-classifies them in FP64 afterwards (a queue
// overflow re-runs the whole grid in FP64).
#include "render_common.cuh"
#include "runtime.h"

namespace dqj {

namespace {

struct VoxelArgs {
    int32_t g;
    uint32_t segs_per_row;
    uint64_t nsegs;
    uint8_t *occ;       // g^3 or NULL
    uint16_t *count;    // g^3 or NULL
    Counters *ctr;      // stats in DQJ_STAT_* order, tile_next = segment claim, queue_count
    uint32_t *queue;    // FP32 + recheck: cells to re-classify in FP64
    uint32_t queue_cap;
};

// Scene-space step of the grid along each axis.
template <typename T>
__device__ __forceinline__ void grid_step(const FrameT<T> &F, int g, T (&step)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) step[a] = (F.bmax[a] - F.bmin[a]) / T(g);
}

// Slice image of the cell centre (x, y, z) = (p0, row's y, row's z): the row
// part O + y E_1 + z E_2 is shared by the whole row.
template <typename T>
__device__ __forceinline__ void row_base(const FrameT<T> &F, const T (&step)[3], int j, int k, T (&base)[8])
{
    const T y = dfma(T(j) + T(0.5), step[1], F.bmin[1]);
    const T z = dfma(T(k) + T(0.5), step[2], F.bmin[2]);
#pragma unroll
    for (int i = 0; i < 8; ++i) base[i] = dfma(z, F.E[2][i], dfma(y, F.E[1][i], F.O[i]));
}

__device__ __forceinline__ void write_cell(const VoxelArgs &va, uint64_t lin, bool inside, int esc)
{
    if (va.occ) va.occ[lin] = inside ? 1 : 0;
    if (va.count) va.count[lin] = (uint16_t)(inside ? 0 : esc);
}

// Re-classify cell lin in FP64 (n = its FP64 escape count) and overwrite it
// where the result differs; returns the change of the inside count.
__device__ __forceinline__ long long fix_cell(const VoxelArgs &va, uint64_t lin, int n, unsigned long long &fixed)
{
    const bool inside = n == 0;
    const bool was = va.occ ? va.occ[lin] != 0 : va.count[lin] == 0;
    const bool changed = was != inside || (va.count && va.count[lin] != (uint16_t)n);
    if (!changed) return 0;
    write_cell(va, lin, inside, n);
    fixed += 1;
    return (inside ? 1 : 0) - (was ? 1 : 0);
}

// Segments are claimed kBatch at a time; inside a batch the row coordinates
// advance incrementally (no division per segment).
constexpr uint32_t kBatch = 16;

// Paired FP32 classification of two cells per lane.  A segment is 32 x 2
// cells: 32 along x in the row pair (2 jp, 2 jp + 1) of one z slice; lane l
// takes column x0 + l of both rows, so its two cells share px and differ only
// in the rows' (warp-uniform) slice bases, and each warp store covers 32
// consecutive cells of a row.  32 x 2 segments keep the warp's cells closer
// together than 64 x 1 rows, so its lockstep rounds wait less for the slowest
// cell (escape counts of the default grid at 1024^3: 0.945 of the steps are
// useful against 0.904).  Cell indices fit in 32 bits (g <= 1024); per-lane
// counts are 32-bit within a batch.
template <int SQ, int MOD, bool RECHECK, bool AXIS>
__global__ void __launch_bounds__(kBlock, 5) voxel2_kernel(const __grid_constant__ FrameDesc fd, const VoxelArgs va)
{
    const FrameT<float> &F = fd.f;
    const int lane = threadIdx.x & 31;
    const int g = va.g;
    const uint32_t gu = (uint32_t)g;
    const uint32_t spr = va.segs_per_row, nsegs = (uint32_t)va.nsegs;
    const uint32_t npairs = (gu + 1u) / 2u;
    const uint32_t max_iter = (uint32_t)fd.max_iter;
    float step[3];
    grid_step<float>(F, g, step);
    unsigned long long iters = 0, inside_n = 0, rechecks = 0, cells = 0;
    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(&va.ctr->tile_next, kBatch);
        first = __shfl_sync(kFull, first, 0);
        if (first >= nsegs) break;
        const uint32_t last = min(first + kBatch, nsegs);
        uint32_t rp = first / spr;
        int x0 = (int)(first - rp * spr) * 32;
        int jp = (int)(rp % npairs), k = (int)(rp / npairs);
        float ba[8], bb[8];  // slice bases of the two rows (row 2 jp + 1 = g of an odd grid is unused)
        row_base<float>(F, step, 2 * jp, k, ba);
        row_base<float>(F, step, 2 * jp + 1, k, bb);
        uint32_t it32 = 0, in32 = 0, cl32 = 0, re32 = 0;
        for (uint32_t seg = first; seg < last; ++seg) {
            const int x = x0 + lane, j0 = 2 * jp;
            const bool two = j0 + 1 < g;
            bool aa = x < g, ab = aa && two;
            const float p = fmaf((float)x + 0.5f, step[0], F.bmin[0]);
            const float2 px = make_float2(p, p);
            float2 z[8];
#pragma unroll
            for (int i = 0; i < (AXIS ? 3 : 8); ++i)  // AXIS: components 3..7 are zero
                z[i] = f2fma(px, make_float2(F.E[0][i], F.E[0][i]), make_float2(ba[i], bb[i]));
            int ca, cb;
            bool live;
            float2 dm;
            const bool va_ = aa, vb_ = ab;
            classify_lockstep2<SQ, MOD, RECHECK, AXIS>(z, fd.p2, F.R2, fd.max_iter, aa, ab, ca, cb, dm, live);
            const bool mga = dm.x <= fd.p2.margin_t, mgb = dm.y <= fd.p2.margin_t;
            const uint32_t la = ((uint32_t)k * gu + (uint32_t)j0) * gu + (uint32_t)x, lb = la + gu;
            if (lane == 0) cl32 += (uint32_t)min(32, g - x0) * (two ? 2u : 1u);
            if (va_) {
                write_cell(va, la, aa, ca + 1);
                it32 += aa ? max_iter : (uint32_t)(ca + 1);
                in32 += aa ? 1u : 0u;
            }
            if (vb_) {
                write_cell(va, lb, ab, cb + 1);
                it32 += ab ? max_iter : (uint32_t)(cb + 1);
                in32 += ab ? 1u : 0u;
            }
            if (RECHECK) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool push = h == 0 ? (va_ && mga) : (vb_ && mgb);
                    const unsigned m = __ballot_sync(kFull, push);
                    if (m == 0) continue;
                    const int leader = __ffs(m) - 1;
                    unsigned b = 0;
                    if (lane == leader) b = atomicAdd(&va.ctr->queue_count, (unsigned)__popc(m));
                    b = __shfl_sync(kFull, b, leader);
                    if (push) {
                        const unsigned slot = b + __popc(m & ((1u << lane) - 1u));
                        if (slot < va.queue_cap)
                            va.queue[slot] = h == 0 ? la : lb;
                        else
                            atomicAdd(&va.ctr->stats[7], 1ull);  // overflow: the FP64 pass re-runs the grid
                        re32 += 1;
                    }
                }
            }
            x0 += 32;  // next segment: same row pair, or the start of the next one
            if (x0 >= g) {
                x0 = 0;
                if (++jp == (int)npairs) {
                    jp = 0;
                    ++k;
                }
                if (seg + 1 < last) {
                    row_base<float>(F, step, 2 * jp, k, ba);
                    row_base<float>(F, step, 2 * jp + 1, k, bb);
                }
            }
        }
        iters += it32;
        inside_n += in32;
        cells += cl32;
        rechecks += re32;
    }
    flush_stat(&va.ctr->stats[0], iters);
    flush_stat(&va.ctr->stats[2], cells);
    flush_stat(&va.ctr->stats[3], inside_n);
    if (RECHECK) flush_stat(&va.ctr->stats[4], rechecks);
}

// FP64 classification, one cell per lane (32-cell row segments).
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) voxel64_kernel(const __grid_constant__ FrameDesc fd, const VoxelArgs va)
{
    const FrameT<double> &F = fd.d;
    const int lane = threadIdx.x & 31;
    const int g = va.g;
    const uint32_t spr = (uint32_t)((g + 31) / 32);
    const uint32_t nsegs = (uint32_t)g * (uint32_t)g * spr;
    double step[3];
    grid_step<double>(F, g, step);
    unsigned long long iters = 0, inside_n = 0, cells = 0;
    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(&va.ctr->tile_next, kBatch);
        first = __shfl_sync(kFull, first, 0);
        if (first >= nsegs) break;
        const uint32_t last = min(first + kBatch, nsegs);
        for (uint32_t seg = first; seg < last; ++seg) {
            const uint32_t row = seg / spr;
            const int x = (int)(seg - row * spr) * 32 + lane;
            const int j = (int)(row % (uint32_t)g), k = (int)(row / (uint32_t)g);
            double base[8], z[8];
            row_base<double>(F, step, j, k, base);
            const double p0 = fma((double)x + 0.5, step[0], F.bmin[0]);
#pragma unroll
            for (int i = 0; i < 8; ++i) z[i] = fma(p0, F.E[0][i], base[i]);
            bool mg;
            const bool part = x < g;
            const int n = classify_lockstep<double, SQ, MOD, false>(z, F, fd.max_iter, part, mg);
            if (part) {
                write_cell(va, (uint64_t)row * (uint64_t)g + x, n == 0, n);
                iters += n ? (unsigned)n : (unsigned)fd.max_iter;
                inside_n += n == 0 ? 1 : 0;
                cells += 1;
            }
        }
    }
    flush_stat(&va.ctr->stats[0], iters);
    flush_stat(&va.ctr->stats[2], cells);
    flush_stat(&va.ctr->stats[3], inside_n);
}

// FP64 re-classification of one cell (recheck and overflow passes).
template <int SQ, int MOD>
__device__ __forceinline__ int cell_fp64(const FrameDesc &fd, int g, uint64_t lin, unsigned long long &it)
{
    const FrameT<double> &F = fd.d;
    double step[3], base[8], z[8];
    grid_step<double>(F, g, step);
    const int x = (int)(lin % (uint64_t)g);
    const uint64_t row = lin / (uint64_t)g;
    row_base<double>(F, step, (int)(row % (uint64_t)g), (int)(row / (uint64_t)g), base);
    const double p0 = fma((double)x + 0.5, step[0], F.bmin[0]);
#pragma unroll
    for (int i = 0; i < 8; ++i) z[i] = fma(p0, F.E[0][i], base[i]);
    const int n = classify_scalar<double, SQ, MOD>(z, F, fd.max_iter);
    it += n ? (unsigned)n : (unsigned)fd.max_iter;
    return n;
}

template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) voxel_recheck_kernel(const __grid_constant__ FrameDesc fd, const VoxelArgs va)
{
    const unsigned nq = min(*(volatile unsigned *)&va.ctr->queue_count, va.queue_cap);
    unsigned long long fixed = 0, it = 0;
    long long delta = 0;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint64_t lin = va.queue[q];
        delta += fix_cell(va, lin, cell_fp64<SQ, MOD>(fd, va.g, lin, it), fixed);
    }
    flush_stat(&va.ctr->stats[5], fixed);
    flush_stat(&va.ctr->stats[6], it);
    flush_stat(&va.ctr->stats[3], (unsigned long long)delta);
}

// After a queue overflow: every cell again in FP64 (and the inside count with it).
template <int SQ, int MOD>
__global__ void __launch_bounds__(kBlock) voxel_overflow_kernel(const __grid_constant__ FrameDesc fd, const VoxelArgs va)
{
    if (*(volatile unsigned long long *)&va.ctr->stats[7] == 0) return;
    const uint64_t n = (uint64_t)va.g * (uint64_t)va.g * (uint64_t)va.g;
    unsigned long long fixed = 0, it = 0;
    long long delta = 0;
    for (uint64_t lin = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < n;
         lin += (uint64_t)gridDim.x * blockDim.x)
        delta += fix_cell(va, lin, cell_fp64<SQ, MOD>(fd, va.g, lin, it), fixed);
    flush_stat(&va.ctr->stats[5], fixed);
    flush_stat(&va.ctr->stats[6], it);
    flush_stat(&va.ctr->stats[3], (unsigned long long)delta);
}

template <int SQ, int MOD>
cudaError_t launch_voxels_t(const FrameDesc &fd, const VoxelArgs &va, cudaStream_t st, int num_sms)
{
    static std::atomic<int> g64{0}, g2{0}, gre{0}, gov{0};
    if (fd.precision == DQJ_FP64) {
        voxel64_kernel<SQ, MOD><<<num_sms * resident_per_sm(g64, voxel64_kernel<SQ, MOD>), kBlock, 0, st>>>(fd, va);
        return cudaGetLastError();
    }
    const bool re = fd.precision == DQJ_FP32_RECHECK;
    const int gm = (int)min((uint64_t)num_sms * resident_per_sm(g2, voxel2_kernel<SQ, MOD, false, false>),
                            (va.nsegs + 4 * kBatch - 1) / (4 * kBatch));
    const int gg = gm > 0 ? gm : 1;
    if (re) {
        if (fd.axis_slice)
            voxel2_kernel<SQ, MOD, true, true><<<gg, kBlock, 0, st>>>(fd, va);
        else
            voxel2_kernel<SQ, MOD, true, false><<<gg, kBlock, 0, st>>>(fd, va);
        voxel_recheck_kernel<SQ, MOD><<<num_sms * resident_per_sm(gre, voxel_recheck_kernel<SQ, MOD>), kBlock, 0, st>>>(fd, va);
        voxel_overflow_kernel<SQ, MOD><<<num_sms * resident_per_sm(gov, voxel_overflow_kernel<SQ, MOD>), kBlock, 0, st>>>(fd, va);
    } else if (fd.axis_slice) {
        voxel2_kernel<SQ, MOD, false, true><<<gg, kBlock, 0, st>>>(fd, va);
    } else {
        voxel2_kernel<SQ, MOD, false, false><<<gg, kBlock, 0, st>>>(fd, va);
    }
    return cudaGetLastError();
}

cudaError_t launch_voxels(const FrameDesc &fd, const VoxelArgs &va, cudaStream_t st, int num_sms)
{
    if (fd.square_mode == 0)
        return fd.modulus_mode == 0 ? launch_voxels_t<0, 0>(fd, va, st, num_sms)
                                    : launch_voxels_t<0, 1>(fd, va, st, num_sms);
    return fd.modulus_mode == 0 ? launch_voxels_t<1, 0>(fd, va, st, num_sms) : launch_voxels_t<1, 1>(fd, va, st, num_sms);
}

}  // namespace

}  // namespace dqj

using namespace dqj;

extern "C" dqj_status dqj_voxelize(dqj_ctx *ctx, const dqj_params *p, int32_t grid_n, uint8_t *occupancy,
                                   uint16_t *counts, int64_t *stats, void *cuda_stream)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        dqj_status s = validate(p);
        if (s != DQJ_OK) return s;
        if (grid_n < 1 || grid_n > DQJ_VOXEL_MAX_GRID)
            return fail(DQJ_ERR_INVALID, "grid_n must be in 1.." + std::to_string(DQJ_VOXEL_MAX_GRID));
        if (counts && (reinterpret_cast<uintptr_t>(counts) & 1u)) return fail(DQJ_ERR_INVALID, "counts must be 2-byte aligned");
        if (stats && (reinterpret_cast<uintptr_t>(stats) & 7u)) return fail(DQJ_ERR_INVALID, "stats must be 8-byte aligned");
        if (!occupancy && !counts) return fail(DQJ_ERR_INVALID, "occupancy and counts are both NULL");
        if (ctx->device == DQJ_DEVICE_MOCK) return fail(DQJ_ERR_INVALID, "a mock context cannot voxelize");
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(e, "voxelize: cudaSetDevice");
        const uint64_t cells = (uint64_t)grid_n * (uint64_t)grid_n * (uint64_t)grid_n;
        const bool re = p->precision == DQJ_FP32_RECHECK;
        const uint64_t qcap = re ? std::min<uint64_t>(cells, 1ull << 24) : 0;
        const size_t need = 256 + qcap * sizeof(uint32_t);
        if (ctx->vox_bytes < need) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "voxelize: synchronize");
            if (ctx->vox_scratch) cudaFree(ctx->vox_scratch);
            ctx->vox_scratch = nullptr;
            ctx->vox_bytes = 0;
            e = cudaMalloc(&ctx->vox_scratch, need);
            if (e != cudaSuccess) return cuda_fail(e, "voxelize: cudaMalloc");
            ctx->vox_bytes = need;
        }
        FrameDesc fd;
        derive_frame(*p, fd, 8, 8);
        VoxelArgs va{};
        va.g = grid_n;
        va.segs_per_row = (uint32_t)((grid_n + 31) / 32);  // 32 x 2 segments of the FP32 kernel
        va.nsegs = (uint64_t)grid_n * (uint64_t)((grid_n + 1) / 2) * va.segs_per_row;
        va.occ = occupancy;
        va.count = counts;
        va.ctr = static_cast<Counters *>(ctx->vox_scratch);
        va.queue = reinterpret_cast<uint32_t *>(static_cast<char *>(ctx->vox_scratch) + 256);
        va.queue_cap = (uint32_t)qcap;
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        e = cudaStreamWaitEvent(st, ctx->done_ev, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(va.ctr, 0, sizeof(Counters), st);
        if (e == cudaSuccess) e = launch_voxels(fd, va, st, ctx->num_sms);
        if (e == cudaSuccess && stats)
            e = cudaMemcpyAsync(stats, va.ctr->stats, DQJ_NSTATS * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->done_ev, st);
        if (e != cudaSuccess) return cuda_fail(e, "voxelize: launch");
        return DQJ_OK;
    });
}
