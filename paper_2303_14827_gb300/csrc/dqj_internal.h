// dqj_internal.h -- structures shared by the host runtime and the CUDA kernels
// of libdqj.  Not part of the public ABI (include/dqj.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace dqj {

// Per-frame constants derived on the host in double, stored in the precision the
// kernel computes in.  Passed by value as a kernel parameter, so the kernels read
// them straight from the constant bank.
template <typename T>
struct FrameT {
    T c[8];        // Julia constant (q_r | q_d)
    T A[8];        // slice_origin + E * eye: slice image of the camera position
    T O[8];        // slice_origin
    T E[3][8];     // slice frame, scene axis a -> R^8
    T eye[3];
    T fwd[3], right[3], upv[3];
    T th, aspect;  // tan(fov_y / 2), width / height (FP64 camera formula)
    T sxa, sxb;    // FP32 camera: sx = (x + 0.5) * sxa + sxb
    T sya, syb;    //              sy = (y + 0.5) * sya + syb
    T bmin[3], bmax[3];
    T R2;          // escape threshold on the modulus, R^2
    T margin;      // recheck band: |modulus - R^2| <= margin (= recheck_margin * R^2)
    T h;           // normal step
    T light[3];    // unit vector to the light
    T ka, kd, albedo[3];
    T ks, shin;  // Eq. phong specular coefficient and exponent (ks = 0: off)
    T de_eps, de_scale, de_rb;  // distance-estimate traversal: hit threshold, step scale, bounding radius
};

// Encoding of a queued FP64 recheck: which sample of which pixel.
//   b == kMarchSample : march sample t_in + k * delta
//   b <  kMarchSample : bisection sample at level b of bracket (k-1, k);
//                       bit i of path = 1 when level i moved lo up to mid
constexpr int kMarchSample = 31;

// Broadcast pairs (v, v) for the paired FP32 march kernel (see dq_math.cuh).
struct PairConsts {
    float2 c[8];
    float2 A[8];
    float2 neg1, neg2;
    float2 negR2;   // (-R^2, -R^2): modulus - R^2 of both halves in one paired add
    float2 neg_ac;  // (-a_c, -a_c): centre of the first step's recheck band on a (below)
    // Axis-slice first step: its modulus is a = z0^2 + sp followed by the fixed
    // FMAs with c4..c7 (EUCLID8), a monotone function of a, so its tests are
    // thresholds on a, found on the host: escape <=> a >= t_esc (exact); the
    // recheck band |modulus - R^2| <= margin is a in [t_mlo, t_mhi].  The paired
    // kernels test the band as |a - a_c| <= margin_t, and later steps as
    // |modulus - R^2| <= margin_t, where margin_t >= margin is the smallest
    // float for which [a_c - margin_t, a_c + margin_t] contains [t_mlo, t_mhi]:
    // a superset of the exact band by at most a few units in the last place.
    float t_esc, t_mlo, t_mhi, margin_t;
};

struct alignas(16) FrameDesc {
    FrameT<float> f;
    FrameT<double> d;
    PairConsts p2;
    int32_t W, H, max_iter, N, B;
    int32_t square_mode, modulus_mode, precision;
    int32_t march_variant;   // FP32 march: 0 one ray per lane, 1 two rays per lane (paired FP32)
    int32_t tile_w, tile_h, tiles_x, tiles_y;
    int32_t traversal;       // DQJ_TRAVERSAL_MARCH or DQJ_TRAVERSAL_DE
    int32_t de_max_steps;
    int64_t pitch;
    int32_t *iter;
    float *depth;
    float *normal;
    uint8_t *rgba;
    int64_t *stats;   // served requests: caller's DQJ_NSTATS counters (device), or NULL
    uint32_t epoch;   // tag for per-pixel dirty flags, changes every frame
    uint32_t axis_slice;  // 1: slice origin and basis are zero in components 3..7
    int32_t k_split;      // march samples split into this many ranges across warps (1: not split)
    int32_t k_chunk;      // samples per range
    int32_t tile_part;    // the frame's tiles t with t mod tile_parts == tile_part are rendered
    int32_t tile_parts;   // (1: every tile)
    int32_t march_samples;  // paired FP32 march on an axis-aligned slice: samples of each ray per round (1, 2)
};

// Counters at the head of the scratch block; zeroed before every frame.
struct Counters {
    unsigned long long stats[10]; // DQJ_STAT_* order
    unsigned int tile_next;       // next tile to claim in the march
    unsigned int hit_count;       // entries in the hit list
    unsigned int hit_next;        // next hit entry to claim in the bisection pass
    unsigned int queue_count;     // entries pushed to the recheck queue (may exceed cap)
    unsigned int queue_next;
    unsigned int dirty_count;     // pixels to re-render in FP64
    unsigned int dirty_next;
    unsigned int pad[5];
};
static_assert(sizeof(Counters) == 128, "Counters layout");

// Views into one scratch allocation owned by a context.
struct alignas(16) Scratch {
    Counters *ctr;
    int4 *hits;           // march: {pixel, k_first, 0, 0}; sphere tracing: {pixel, depth bits, n*}
    uint32_t hit_cap;
    int4 *queue;          // {pixel, k | b << 16, path, n32}
    uint32_t queue_cap;
    uint32_t *dirty_flag; // per pixel, == epoch when the pixel is queued for re-render
    int32_t *dirty_list;
    uint32_t dirty_cap;
    int4 *part;           // split march: per range and pixel {first inside k or -1, iterations, max escape count, samples}
    uint32_t *part_hit;   // split march: per pixel, the lowest range that found an inside sample (~0u: none yet)
    uint32_t part_cap;    // entries of part
    uint32_t pad_[3];
};

// Host-side launch helpers implemented in render.cu.
// Enqueue the passes of one frame on st.  ev (optional, 5 events) is recorded
// before the march and after the march, bisect, recheck and fixup passes.
cudaError_t launch_frame(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms,
                         cudaEvent_t *ev = nullptr);
// The distance-estimate traversal (de.cu): sphere tracing, then normal and
// shading of its hits; same events (the last three after the shading pass).
cudaError_t launch_de(const FrameDesc &fd, const Scratch &sc, cudaStream_t st, int num_sms, cudaEvent_t *ev);
cudaError_t fma_peak_launch(int variant, int num_sms, float *sink, cudaStream_t st, double *flops);
// Ranges the paired FP32 march of a frame splits its samples into (1: none):
// enough for the frame's tiles to fill the resident warps of num_sms SMs.
int march_split(const FrameDesc &fd, int num_sms);
// Samples of each ray per round of the paired FP32 march on an axis-aligned
// slice: 2 unless DQJ_MARCH_SAMPLES = 1 (read once per process).  Both give
// the same results.
int march_samples_per_round();

}  // namespace dqj
