// fma_peak.cu -- FP32 / FP64 FMA throughput microbenchmark (the roofline
// denominator of the renderer, which is bound by the FP32 FMA pipe).
//
// Each thread runs independent dependency chains x <- x * a + b (a < 1, so the
// values stay normal), enough of them that latency is hidden.  Variants:
//   0  scalar fma.rn.f32, 8 chains
//   1  paired fma.rn.f32x2 (__ffma2_rn), 8 float2 chains
//   2  as 0 plus 2 integer ops per 8 FMAs (does non-FMA work cost FMA slots?)
//   3  as 1 plus 2 integer ops per 8 paired FMAs
//   4  fma.rn.f64, 8 chains
// Only FMAs are counted as flops (2 each).
#include "dqj_internal.h"

namespace dqj {

namespace {

constexpr int kPeakBlock = 256;

template <int V>
__global__ void __launch_bounds__(kPeakBlock) fma_kernel(int iters, float a, float b, float *sink)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (V == 0 || V == 2) {
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = 1.0f + 1e-3f * (float)(tid + i);
        unsigned u = tid, w = tid * 7u;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
                if constexpr (V == 2) {
                    u = u * 1664525u + w;
                    w ^= u >> 7;
                }
            }
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += x[i];
        if (s == -1.0f || (V == 2 && u == 0x12345u && w == 7u)) sink[tid] = s;
    } else if constexpr (V == 1 || V == 3) {
        float2 x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = make_float2(1.0f + 1e-3f * (float)(tid + i), 1.0f - 1e-3f * (float)i);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        unsigned u = tid, w = tid * 7u;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
                if constexpr (V == 3) {
                    u = u * 1664525u + w;
                    w ^= u >> 7;
                }
            }
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
        if (s == -1.0f || (V == 3 && u == 0x12345u && w == 7u)) sink[tid] = s;
    } else {
        double x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = 1.0 + 1e-3 * (double)(tid + i);
        const double ad = a, bd = b;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fma(x[i], ad, bd);
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += x[i];
        if (s == -1.0) sink[tid] = (float)s;
    }
}

template <int V>
cudaError_t run(int num_sms, float *sink, cudaStream_t st, double *flops)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_kernel<V>, kPeakBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = per_sm * num_sms;
    const int iters = V == 4 ? 256 : 8192;
    // FMAs per thread per iteration
    const double fmas_per_iter = (V == 0 || V == 2) ? 32.0 : (V == 1 || V == 3) ? 32.0 : 8.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_kernel<V><<<grid, kPeakBlock, 0, st>>>(iters / 4, 0.999f, 0.001f, sink);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        fma_kernel<V><<<grid, kPeakBlock, 0, st>>>(iters, 0.999f, 0.001f, sink);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    e = cudaGetLastError();
    const double total = (double)grid * kPeakBlock * iters * fmas_per_iter * 2.0;
    *flops = total / (best * 1e-3);
    return e;
}

}  // namespace

cudaError_t fma_peak_launch(int variant, int num_sms, float *sink, cudaStream_t st, double *flops)
{
    switch (variant) {
    case 0: return run<0>(num_sms, sink, st, flops);
    case 1: return run<1>(num_sms, sink, st, flops);
    case 2: return run<2>(num_sms, sink, st, flops);
    case 3: return run<3>(num_sms, sink, st, flops);
    case 4: return run<4>(num_sms, sink, st, flops);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dqj
