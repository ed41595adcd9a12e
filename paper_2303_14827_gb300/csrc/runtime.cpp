// runtime.cpp -- C ABI entry points, parameter validation, per-frame constants
// and scratch management of libdqj.
#include "runtime.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <system_error>

namespace dqj {

static thread_local std::string g_err;

// The message is best effort: if the host cannot allocate it, the previous
// one is cleared and the status still returns.
static void set_error(const char *msg) noexcept
{
    try {
        g_err = msg;
    } catch (...) {
        g_err.clear();
    }
}

dqj_status fail(dqj_status st, const std::string &msg)
{
    set_error(msg.c_str());
    return st;
}

dqj_status cuda_fail(cudaError_t e, const char *what)
{
    const dqj_status st = e == cudaErrorMemoryAllocation ? DQJ_ERR_NOMEM : DQJ_ERR_CUDA;
    try {
        g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    } catch (...) {
        set_error(what);
    }
    return st;
}

dqj_status exception_status() noexcept
{
    try {
        throw;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return DQJ_ERR_NOMEM;
    } catch (const std::system_error &e) {  // e.g. a thread could not be started
        set_error(e.what());
        return DQJ_ERR_NOMEM;
    } catch (const std::exception &e) {
        set_error(e.what());
        return DQJ_ERR_INVALID;
    } catch (...) {
        set_error("unknown C++ exception");
        return DQJ_ERR_INVALID;
    }
}

static bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

dqj_status validate(const dqj_params *p)
{
    if (!p) return fail(DQJ_ERR_INVALID, "params is NULL");
    if (p->width < 1 || p->width > 16384) return fail(DQJ_ERR_INVALID, "width must be in 1..16384");
    if (p->height < 1 || p->height > 16384) return fail(DQJ_ERR_INVALID, "height must be in 1..16384");
    if (p->max_iter < 1 || p->max_iter > 1024) return fail(DQJ_ERR_INVALID, "max_iter must be in 1..1024");
    if (!(p->escape_radius > 0.0) || !std::isfinite(p->escape_radius))
        return fail(DQJ_ERR_INVALID, "escape_radius must be finite and > 0");
    if (p->march_steps < 1 || p->march_steps > 65535) return fail(DQJ_ERR_INVALID, "march_steps must be in 1..65535");
    if (p->bisect_steps < 0 || p->bisect_steps > 30) return fail(DQJ_ERR_INVALID, "bisect_steps must be in 0..30");
    if (!(p->fov_y_deg > 0.0 && p->fov_y_deg < 180.0)) return fail(DQJ_ERR_INVALID, "fov_y_deg must be in (0, 180)");
    if (!(p->normal_h > 0.0) || !std::isfinite(p->normal_h))
        return fail(DQJ_ERR_INVALID, "normal_h must be finite and > 0");
    if (p->precision < DQJ_FP32 || p->precision > DQJ_FP64)
        return fail(DQJ_ERR_INVALID, "precision must be DQJ_FP32, DQJ_FP32_RECHECK or DQJ_FP64");
    if (!(p->recheck_margin >= 0.0 && p->recheck_margin <= 0.5))
        return fail(DQJ_ERR_INVALID, "recheck_margin must be in [0, 0.5]");
    if (p->square_mode < 0 || p->square_mode > 1) return fail(DQJ_ERR_INVALID, "square_mode must be 0 or 1");
    if (p->modulus_mode < 0 || p->modulus_mode > 1) return fail(DQJ_ERR_INVALID, "modulus_mode must be 0 or 1");
    if (!finite_all(p->c, 8)) return fail(DQJ_ERR_INVALID, "c must be finite");
    if (!finite_all(p->slice_origin, 8)) return fail(DQJ_ERR_INVALID, "slice_origin must be finite");
    if (!finite_all(&p->slice_basis[0][0], 24)) return fail(DQJ_ERR_INVALID, "slice_basis must be finite");
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double dot = 0.0;
            for (int i = 0; i < 8; ++i) dot += p->slice_basis[a][i] * p->slice_basis[b][i];
            if (std::fabs(dot - (a == b ? 1.0 : 0.0)) > 1e-9)
                return fail(DQJ_ERR_INVALID, "slice_basis rows must be orthonormal (to 1e-9)");
        }
    if (!finite_all(p->eye, 3) || !finite_all(p->target, 3) || !finite_all(p->up, 3))
        return fail(DQJ_ERR_INVALID, "eye, target and up must be finite");
    double f[3] = {p->target[0] - p->eye[0], p->target[1] - p->eye[1], p->target[2] - p->eye[2]};
    const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0)) return fail(DQJ_ERR_INVALID, "eye and target must differ");
    const double cx = f[1] * p->up[2] - f[2] * p->up[1], cy = f[2] * p->up[0] - f[0] * p->up[2],
                 cz = f[0] * p->up[1] - f[1] * p->up[0];
    const double ul = std::sqrt(p->up[0] * p->up[0] + p->up[1] * p->up[1] + p->up[2] * p->up[2]);
    if (!(std::sqrt(cx * cx + cy * cy + cz * cz) > 1e-12 * fl * ul))
        return fail(DQJ_ERR_INVALID, "up must not be parallel to the view direction");
    if (!finite_all(p->box_min, 3) || !finite_all(p->box_max, 3)) return fail(DQJ_ERR_INVALID, "box must be finite");
    for (int a = 0; a < 3; ++a)
        if (!(p->box_min[a] < p->box_max[a])) return fail(DQJ_ERR_INVALID, "box_min must be < box_max");
    if (!finite_all(p->light_dir, 3)) return fail(DQJ_ERR_INVALID, "light_dir must be finite");
    if (!(p->light_dir[0] * p->light_dir[0] + p->light_dir[1] * p->light_dir[1] + p->light_dir[2] * p->light_dir[2] >
          0.0))
        return fail(DQJ_ERR_INVALID, "light_dir must be non-zero");
    if (!std::isfinite(p->k_ambient) || !std::isfinite(p->k_diffuse))
        return fail(DQJ_ERR_INVALID, "k_ambient and k_diffuse must be finite");
    if (!(p->k_specular >= 0.0 && p->k_specular <= 1e6))
        return fail(DQJ_ERR_INVALID, "k_specular must be finite and >= 0");
    if (!(p->shininess >= 0.0 && p->shininess <= 1e4)) return fail(DQJ_ERR_INVALID, "shininess must be in [0, 10000]");
    if (p->traversal != DQJ_TRAVERSAL_MARCH && p->traversal != DQJ_TRAVERSAL_DE)
        return fail(DQJ_ERR_INVALID, "traversal must be DQJ_TRAVERSAL_MARCH or DQJ_TRAVERSAL_DE");
    if (p->traversal == DQJ_TRAVERSAL_DE) {
        if (p->de_max_steps < 1 || p->de_max_steps > 1000000)
            return fail(DQJ_ERR_INVALID, "de_max_steps must be in 1..1000000");
        if (!(p->de_epsilon > 0.0 && p->de_epsilon < 1e30)) return fail(DQJ_ERR_INVALID, "de_epsilon must be > 0");
        if (!(p->de_step_scale > 0.0 && p->de_step_scale <= 1.0))
            return fail(DQJ_ERR_INVALID, "de_step_scale must be in (0, 1]");
        if (!(p->de_bound_radius >= 0.0 && p->de_bound_radius < 1e30))
            return fail(DQJ_ERR_INVALID, "de_bound_radius must be >= 0");
    }
    for (int a = 0; a < 3; ++a)
        if (!(p->albedo[a] >= 0.0 && p->albedo[a] <= 1.0)) return fail(DQJ_ERR_INVALID, "albedo must be in [0, 1]");
    return DQJ_OK;
}

template <typename T>
static void cast_frame(const FrameT<double> &d, FrameT<T> &f)
{
    const double *src = reinterpret_cast<const double *>(&d);
    T *dst = reinterpret_cast<T *>(&f);
    static_assert(sizeof(FrameT<double>) % sizeof(double) == 0, "FrameT is an array of doubles");
    for (size_t i = 0; i < sizeof(FrameT<double>) / sizeof(double); ++i) dst[i] = (T)src[i];
}

// The modulus after the axis-slice first step, as the device forms it from the
// partial sum a = z0^2 + sp: EUCLID8 adds c4^2 .. c7^2 by four rounded FMAs
// (every component 3..7 equals c there), DUALNUM adds nothing.
static float axis_first_modulus(float a, const FrameT<float> &F, int modulus_mode)
{
    if (modulus_mode == 0)
        for (int i = 4; i < 8; ++i) a = std::fmaf(F.c[i], F.c[i], a);
    return a;
}

// Smallest non-negative float (by bit pattern, which orders them) for which a
// monotone false -> true predicate holds; 0x7f800001 when none does.
template <typename Pred>
static uint32_t first_true(Pred pred)
{
    auto as_f = [](uint32_t b) {
        float f;
        std::memcpy(&f, &b, sizeof f);
        return f;
    };
    uint32_t lo = 0, hi = 0x7f800000u;  // +0 .. +inf
    if (!pred(as_f(hi))) return 0x7f800001u;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (pred(as_f(mid)))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Thresholds of the axis-slice first step on a = z0^2 + sp >= 0: every rounded
// FMA is non-decreasing in a, so "modulus > R^2" holds exactly from t_esc up,
// and "|modulus - R^2| <= margin" (the recheck test, in FP32 as the device
// forms it) exactly on [t_mlo, t_mhi] (empty when t_mlo > t_mhi).
void axis_first_thresholds(const FrameT<float> &F, int modulus_mode, PairConsts &P)
{
    auto bits_f = [](uint32_t b) {
        float f;
        std::memcpy(&f, &b, sizeof f);
        return f;
    };
    const float R2 = F.R2, margin = F.margin;
    auto x = [&](float a) { return axis_first_modulus(a, F, modulus_mode); };
    P.t_esc = bits_f(first_true([&](float a) { return x(a) > R2; }));
    const uint32_t lo = first_true([&](float a) { return x(a) - R2 >= -margin; });
    const uint32_t above = first_true([&](float a) { return x(a) - R2 > margin; });
    if (lo > 0x7f800000u || above == 0 || above <= lo) {
        P.t_mlo = INFINITY;
        P.t_mhi = -1.f;
    } else {
        P.t_mlo = bits_f(lo);
        P.t_mhi = bits_f(above - 1);
    }
    // centre a_c and half-width margin_t of the paired kernels' band test (exact
    // in double: every bound below is a float or the difference of two floats)
    double need = margin;
    float ac = INFINITY;  // empty band: |a - inf| is never within margin_t
    if (P.t_mlo <= P.t_mhi) {
        ac = (float)(0.5 * ((double)P.t_mlo + (double)P.t_mhi));
        need = std::max(need, std::max((double)ac - (double)P.t_mlo, (double)P.t_mhi - (double)ac));
    }
    float mt = (float)need;
    if ((double)mt < need) mt = std::nextafter(mt, INFINITY);
    P.neg_ac = make_float2(-ac, -ac);
    P.margin_t = mt;
}

void derive_frame(const dqj_params &p, FrameDesc &fd, int tile_w, int tile_h)
{
    std::memset(&fd, 0, sizeof fd);
    FrameT<double> &F = fd.d;
    for (int i = 0; i < 8; ++i) {
        F.c[i] = p.c[i];
        F.O[i] = p.slice_origin[i];
        for (int a = 0; a < 3; ++a) F.E[a][i] = p.slice_basis[a][i];
        F.A[i] = p.slice_origin[i] + p.eye[0] * p.slice_basis[0][i] + p.eye[1] * p.slice_basis[1][i] +
                 p.eye[2] * p.slice_basis[2][i];
    }
    // a slice through the first three components only: zeta_0 is zero in 3..7
    fd.axis_slice = 1;
    for (int i = 3; i < 8; ++i)
        if (p.slice_origin[i] != 0.0 || p.slice_basis[0][i] != 0.0 || p.slice_basis[1][i] != 0.0 ||
            p.slice_basis[2][i] != 0.0)
            fd.axis_slice = 0;
    double f[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) f[a] = p.target[a] - p.eye[a];
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] /= fl;
    r[0] = f[1] * p.up[2] - f[2] * p.up[1];
    r[1] = f[2] * p.up[0] - f[0] * p.up[2];
    r[2] = f[0] * p.up[1] - f[1] * p.up[0];
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    for (int a = 0; a < 3; ++a) {
        F.eye[a] = p.eye[a];
        F.fwd[a] = f[a];
        F.right[a] = r[a];
        F.upv[a] = u[a];
        F.bmin[a] = p.box_min[a];
        F.bmax[a] = p.box_max[a];
        F.albedo[a] = p.albedo[a];
    }
    F.th = std::tan(0.5 * p.fov_y_deg * (M_PI / 180.0));
    F.aspect = (double)p.width / (double)p.height;
    F.sxa = 2.0 * F.th * F.aspect / (double)p.width;
    F.sxb = -F.th * F.aspect;
    F.sya = -2.0 * F.th / (double)p.height;
    F.syb = F.th;
    F.R2 = p.escape_radius * p.escape_radius;
    F.margin = p.recheck_margin * F.R2;
    F.h = p.normal_h;
    const double ll = std::sqrt(p.light_dir[0] * p.light_dir[0] + p.light_dir[1] * p.light_dir[1] +
                                p.light_dir[2] * p.light_dir[2]);
    for (int a = 0; a < 3; ++a) F.light[a] = p.light_dir[a] / ll;
    F.ka = p.k_ambient;
    F.kd = p.k_diffuse;
    F.ks = p.k_specular;
    F.shin = p.shininess;
    F.de_eps = p.de_epsilon;
    F.de_scale = p.de_step_scale;
    F.de_rb = p.de_bound_radius;
    cast_frame<float>(F, fd.f);
    for (int i = 0; i < 8; ++i) {
        fd.p2.c[i] = make_float2(fd.f.c[i], fd.f.c[i]);
        fd.p2.A[i] = make_float2(fd.f.A[i], fd.f.A[i]);
    }
    fd.p2.neg1 = make_float2(-1.f, -1.f);
    fd.p2.neg2 = make_float2(-2.f, -2.f);
    fd.p2.negR2 = make_float2(-fd.f.R2, -fd.f.R2);
    axis_first_thresholds(fd.f, p.modulus_mode, fd.p2);
    fd.W = p.width;
    fd.H = p.height;
    fd.max_iter = p.max_iter;
    fd.N = p.march_steps;
    fd.B = p.bisect_steps;
    fd.square_mode = p.square_mode;
    fd.modulus_mode = p.modulus_mode;
    fd.precision = p.precision;
    fd.traversal = p.traversal;
    fd.de_max_steps = p.de_max_steps;
    fd.tile_w = tile_w;
    fd.tile_h = tile_h;
    fd.tiles_x = (p.width + tile_w - 1) / tile_w;
    fd.tiles_y = (p.height + tile_h - 1) / tile_h;
    fd.k_split = 1;
    fd.k_chunk = fd.N + 1;
    fd.tile_part = 0;
    fd.tile_parts = 1;
    fd.march_samples = march_samples_per_round();
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void scratch_free(ScratchBuf &s)
{
    if (s.base) cudaFree(s.base);
    s = ScratchBuf{};
}

dqj_status scratch_ensure(ScratchBuf &s, uint64_t pixels, bool need_queue, uint64_t part_entries)
{
    if (s.base && pixels <= s.pixels && (!need_queue || s.with_queue) && part_entries <= s.part_entries)
        return DQJ_OK;
    const uint64_t px = std::max<uint64_t>(pixels, s.pixels);
    const bool wq = need_queue || s.with_queue;
    const uint64_t qcap = wq ? 4 * px : 0;
    const uint64_t pcap = std::max<uint64_t>(part_entries, s.part_entries);
    size_t off = 0;
    const size_t o_ctr = off;
    off = align_up(off + sizeof(Counters), 256);
    const size_t o_hits = off;
    off = align_up(off + px * sizeof(int4), 256);
    const size_t o_queue = off;
    off = align_up(off + qcap * sizeof(int4), 256);
    const size_t o_flag = off;
    off = align_up(off + px * sizeof(uint32_t), 256);
    const size_t o_list = off;
    off = align_up(off + px * sizeof(int32_t), 256);
    const size_t o_part = off;
    off = align_up(off + pcap * sizeof(int4), 256);
    const size_t o_phit = off;
    off = align_up(off + (pcap ? px * sizeof(uint32_t) : 0), 256);
    void *base = nullptr;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "scratch: synchronize");
    if (s.base) cudaFree(s.base);
    s = ScratchBuf{};
    e = cudaMalloc(&base, off);
    if (e != cudaSuccess) return cuda_fail(e, "scratch: cudaMalloc");
    e = cudaMemset(base, 0, off);
    if (e != cudaSuccess) {
        cudaFree(base);
        return cuda_fail(e, "scratch: cudaMemset");
    }
    char *b = static_cast<char *>(base);
    s.base = base;
    s.bytes = off;
    s.pixels = (uint32_t)px;
    s.with_queue = wq;
    s.epoch = 0;
    s.view.ctr = reinterpret_cast<Counters *>(b + o_ctr);
    s.view.hits = reinterpret_cast<int4 *>(b + o_hits);
    s.view.hit_cap = (uint32_t)px;
    s.view.queue = wq ? reinterpret_cast<int4 *>(b + o_queue) : nullptr;
    s.view.queue_cap = (uint32_t)qcap;
    s.view.dirty_flag = reinterpret_cast<uint32_t *>(b + o_flag);
    s.view.dirty_list = reinterpret_cast<int32_t *>(b + o_list);
    s.view.dirty_cap = (uint32_t)px;
    s.part_entries = pcap;
    s.view.part = pcap ? reinterpret_cast<int4 *>(b + o_part) : nullptr;
    s.view.part_hit = pcap ? reinterpret_cast<uint32_t *>(b + o_phit) : nullptr;
    s.view.part_cap = (uint32_t)pcap;
    return DQJ_OK;
}

// March kernel and tile shape of a frame: the autotuned choice for its class,
// else the paired kernel on 8 x 8 tiles (FP32) or one ray per lane on 8 x 4
// (FP64).  The environment variable DQJ_MARCH_VARIANT (0 or 1) overrides the
// FP32 kernel: 0 one ray per lane, 1 two rays per lane.
void default_tile_shape(const dqj_params &p, int &variant, int &tw, int &th)
{
    variant = p.precision == DQJ_FP64 ? 0 : 1;
    if (const char *e = std::getenv("DQJ_MARCH_VARIANT"))
        if (e[0] == '0' || e[0] == '1') variant = p.precision == DQJ_FP64 ? 0 : e[0] - '0';
    tw = 8;
    th = variant >= 1 ? 8 : 4;
}

void pick_tile_shape(dqj_ctx *ctx, const dqj_params &p, int &variant, int &tw, int &th)
{
    default_tile_shape(p, variant, tw, th);
    const int64_t px = (int64_t)p.width * p.height;
    const int cls = px <= 65536 ? 0 : px <= 262144 ? 1 : px <= 1048576 ? 2 : 3;
    const int bucket = p.max_iter <= 12 ? 0 : p.max_iter <= 20 ? 1 : p.max_iter <= 28 ? 2 : 3;
    {
        std::lock_guard<std::mutex> lk(ctx->tiles_mu);
        auto it = ctx->tiles.find(tile_key(variant, cls, bucket));
        if (it != ctx->tiles.end()) {
            tw = it->second.first;
            th = it->second.second;
        }
    }
    // a warp covers 32 rays (one per lane) or 64 (two per lane)
    if (tw < 1 || th < 1 || tw * th != (variant >= 1 ? 64 : 32)) {
        tw = 8;
        th = variant >= 1 ? 8 : 4;
    }
}

// Enqueue the passes of one frame (of its tiles t with t mod parts == part) on
// stream st with scratch set sb; ctx->mu held.  Ordered after the context's
// previous render through ctx->done_ev unless `lane` is given: then the caller
// (a batch) orders the frame, lane holds five events for the passes (used
// unless the profiling ring is on), and *march_done returns the event recorded
// after the frame's march.
static dqj_status enqueue_frame_on(dqj_ctx *ctx, const dqj_params &p, const dqj_outputs &out, cudaStream_t st,
                                   int part, int parts, ScratchBuf &sb, cudaEvent_t *lane,
                                   cudaEvent_t *march_done = nullptr)
{
    int variant, tw, th;
    pick_tile_shape(ctx, p, variant, tw, th);
    FrameDesc fd;
    derive_frame(p, fd, tw, th);
    fd.march_variant = variant;
    fd.tile_part = part;
    fd.tile_parts = parts;
    fd.pitch = out.pitch_px;
    fd.iter = out.iter;
    fd.depth = out.depth;
    fd.normal = out.normal;
    fd.rgba = out.rgba;
    const uint64_t px = (uint64_t)p.width * (uint64_t)p.height;
    // Under stream capture (a CUDA graph) nothing may allocate or synchronize, a
    // wait on an event recorded outside the capture is not allowed, and a
    // replay repeats the frame's constants, so the per-pixel tags of the
    // recheck mode are cleared by the frame itself instead of changing epoch.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    unsigned long long cap_id = 0;
    // launch errors are read back with cudaGetLastError: start from a clean
    // slate, so an earlier failed call of the caller's is not taken for ours
    (void)cudaGetLastError();
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cap, &cap_id);
    if (e != cudaSuccess) return cuda_fail(e, "render: cudaStreamGetCaptureInfo");
    const bool capturing = cap == cudaStreamCaptureStatusActive;
    const bool recheck = p.precision == DQJ_FP32_RECHECK;
    // a frame with fewer tiles than resident warps splits its samples into ranges
    fd.k_split = march_split(fd, ctx->num_sms);
    fd.k_chunk = (fd.N + 1 + fd.k_split - 1) / fd.k_split;
    fd.k_split = (fd.N + 1 + fd.k_chunk - 1) / fd.k_chunk;  // every range holds a sample
    const uint64_t part_entries = fd.k_split > 1 ? (uint64_t)fd.k_split * px : 0;
    if (capturing &&
        !(sb.base && px <= sb.pixels && (!recheck || sb.with_queue) && part_entries <= sb.part_entries))
        return fail(DQJ_ERR_INVALID, "render: under stream capture the context's scratch must already fit the frame "
                                     "(render the largest frame once before capturing)");
    dqj_status s = scratch_ensure(sb, px, recheck, part_entries);
    if (s != DQJ_OK) return s;
    if (capturing) {
        if (recheck) {
            e = cudaMemsetAsync(sb.view.dirty_flag, 0, (size_t)sb.pixels * sizeof(uint32_t), st);
            if (e != cudaSuccess) return cuda_fail(e, "render: clear flags");
        }
        fd.epoch = 1;
    } else {
        if (++sb.epoch == 0) {  // tags wrapped: clear the per-pixel flags
            e = cudaMemsetAsync(sb.view.dirty_flag, 0, (size_t)sb.pixels * sizeof(uint32_t), st);
            if (e != cudaSuccess) return cuda_fail(e, "render: clear flags");
            sb.epoch = 1;
        }
        fd.epoch = sb.epoch;
    }
    // the previous render's event: waited on only when it was recorded in the
    // same capture state (a record inside a graph is ordered by its replays)
    if (!lane && ctx->done_capture == (capturing ? cap_id : 0ull)) {
        e = cudaStreamWaitEvent(st, ctx->done_ev, 0);
        if (e != cudaSuccess) return cuda_fail(e, "render: cudaStreamWaitEvent");
    }
    e = cudaMemsetAsync(sb.view.ctr, 0, sizeof(Counters), st);
    if (e != cudaSuccess) return cuda_fail(e, "render: clear counters");
    if (fd.k_split > 1) {
        e = cudaMemsetAsync(sb.view.part_hit, 0xff, px * sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "render: clear split-march hits");
    }
    cudaEvent_t *ev = lane;
    if (ctx->ring_frames > 0) ev = &ctx->ev[5 * (ctx->ring_next++ % (uint64_t)ctx->ring_frames)];
    e = launch_frame(fd, sb.view, st, ctx->num_sms, ev);
    if (e != cudaSuccess) return cuda_fail(e, "render: kernel launch");
    if (march_done) *march_done = ev ? ev[1] : nullptr;
    if (out.stats) {
        e = cudaMemcpyAsync(out.stats, sb.view.ctr->stats, DQJ_NSTATS * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "render: stats copy");
    }
    if (!lane) {
        e = cudaEventRecord(ctx->done_ev, st);
        if (e != cudaSuccess) return cuda_fail(e, "render: cudaEventRecord");
        ctx->done_capture = capturing ? cap_id : 0;
    }
    return DQJ_OK;
}

static dqj_status enqueue_frame(dqj_ctx *ctx, const dqj_params &p, const dqj_outputs &out, cudaStream_t st,
                                int part = 0, int parts = 1)
{
    return enqueue_frame_on(ctx, p, out, st, part, parts, ctx->scratch, nullptr);
}

// The frames of a batch alternate between the context's two scratch sets and
// two lane streams, and each frame's march waits only for the previous frame's
// march: a frame's bisection, recheck and re-render passes (short, and bound by
// latency) run beside the next frame's march instead of after it, while the
// marches themselves stay one at a time.  ctx->mu held from open to close.
struct FramePipe {
    dqj_ctx *ctx;
    cudaEvent_t prev = nullptr;  // after the previous frame's march
    int next = 0;
    bool used[2] = {false, false};

    // order the batch after the context's previous render and the caller's
    // stream st, and fork the lanes from st
    dqj_status open(cudaStream_t st)
    {
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
            if (!ctx->lane_stream[l]) e = cudaStreamCreateWithFlags(&ctx->lane_stream[l], cudaStreamNonBlocking);
            for (int k = 0; k < 5 && e == cudaSuccess; ++k)
                if (!ctx->lane_ev[l][k]) e = cudaEventCreateWithFlags(&ctx->lane_ev[l][k], cudaEventDisableTiming);
            if (e == cudaSuccess && !ctx->join_ev[l]) e = cudaEventCreateWithFlags(&ctx->join_ev[l], cudaEventDisableTiming);
        }
        if (e == cudaSuccess && !ctx->fork_ev) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
        if (e == cudaSuccess && ctx->done_capture == 0) e = cudaStreamWaitEvent(st, ctx->done_ev, 0);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->fork_ev, st);
        for (int l = 0; l < 2 && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(ctx->lane_stream[l], ctx->fork_ev, 0);
        if (e != cudaSuccess) return cuda_fail(e, "render batch: lane streams");
        return DQJ_OK;
    }

    // enqueue the next frame, after `after` too when given; *lane returns the
    // stream it runs on
    dqj_status frame(const dqj_params &p, const dqj_outputs &out, cudaStream_t *lane = nullptr,
                     cudaEvent_t after = nullptr)
    {
        const int l = next++ & 1;
        cudaStream_t ls = ctx->lane_stream[l];
        cudaError_t e = cudaSuccess;
        if (prev) e = cudaStreamWaitEvent(ls, prev, 0);
        if (e == cudaSuccess && after) e = cudaStreamWaitEvent(ls, after, 0);
        if (e != cudaSuccess) return cuda_fail(e, "render batch: cudaStreamWaitEvent");
        used[l] = true;
        if (lane) *lane = ls;
        return enqueue_frame_on(ctx, p, out, ls, 0, 1, l ? ctx->scratch2 : ctx->scratch, ctx->lane_ev[l], &prev);
    }

    // join the lanes into st and make st the context's last render
    dqj_status close(cudaStream_t st)
    {
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
            if (!used[l]) continue;
            e = cudaEventRecord(ctx->join_ev[l], ctx->lane_stream[l]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[l], 0);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->done_ev, st);
        if (e != cudaSuccess) return cuda_fail(e, "render batch: join");
        ctx->done_capture = 0;
        return DQJ_OK;
    }
};

dqj_status check_outputs(const dqj_params &p, const dqj_outputs *out)
{
    if (!out) return fail(DQJ_ERR_INVALID, "outputs is NULL");
    if (out->pitch_px < p.width) return fail(DQJ_ERR_INVALID, "pitch_px must be >= width");
    if (out->rgba && (reinterpret_cast<uintptr_t>(out->rgba) & 3u))
        return fail(DQJ_ERR_INVALID, "rgba must be 4-byte aligned");
    if (out->iter && (reinterpret_cast<uintptr_t>(out->iter) & 3u))
        return fail(DQJ_ERR_INVALID, "iter must be 4-byte aligned");
    if (out->depth && (reinterpret_cast<uintptr_t>(out->depth) & 3u))
        return fail(DQJ_ERR_INVALID, "depth must be 4-byte aligned");
    if (out->normal && (reinterpret_cast<uintptr_t>(out->normal) & 3u))
        return fail(DQJ_ERR_INVALID, "normal must be 4-byte aligned");
    return DQJ_OK;
}

dqj_status render_on_stream(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, cudaStream_t st, int part,
                            int parts)
{
    dqj_status s = validate(p);
    if (s != DQJ_OK) return s;
    s = check_outputs(*p, out);
    if (s != DQJ_OK) return s;
    if (parts < 1 || parts > 65536 || part < 0 || part >= parts)
        return fail(DQJ_ERR_INVALID, "tile parts must satisfy 0 <= part < parts <= 65536");
    if (ctx->device == DQJ_DEVICE_MOCK) return fail(DQJ_ERR_INVALID, "a mock context cannot render");
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "render: cudaSetDevice");
    return enqueue_frame(ctx, *p, *out, st, part, parts);
}

dqj_status render_on_stream(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, cudaStream_t st)
{
    return render_on_stream(ctx, p, out, st, 0, 1);
}

}  // namespace dqj

using namespace dqj;

extern "C" {

const char *dqj_last_error(void) { return g_err.c_str(); }

dqj_status dqj_default_params(dqj_params *p)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!p) return fail(DQJ_ERR_INVALID, "params is NULL");
        std::memset(p, 0, sizeof *p);
        const double c[8] = {-0.2, 0.6, 0.2, 0.2, 0.1, 0.0, 0.0, 0.05};
        for (int i = 0; i < 8; ++i) p->c[i] = c[i];
        for (int a = 0; a < 3; ++a) p->slice_basis[a][a] = 1.0;
        p->eye[2] = 3.5;
        p->up[1] = 1.0;
        p->fov_y_deg = 45.0;
        p->width = 256;
        p->height = 256;
        p->max_iter = 12;
        p->escape_radius = 4.0;
        p->march_steps = 256;
        p->bisect_steps = 8;
        p->normal_h = 1e-4;
        for (int a = 0; a < 3; ++a) {
            p->box_min[a] = -2.0;
            p->box_max[a] = 2.0;
            p->light_dir[a] = 1.0;
            p->albedo[a] = 1.0;
        }
        p->k_ambient = 0.15;
        p->k_diffuse = 0.85;
        p->precision = DQJ_FP32;
        p->recheck_margin = 1e-3;
        p->square_mode = DQJ_SQUARE_ALGEBRAIC;
        p->modulus_mode = DQJ_MODULUS_EUCLID8;
        p->k_specular = 0.0;
        p->shininess = 32.0;
        p->traversal = DQJ_TRAVERSAL_MARCH;
        p->de_max_steps = 512;
        p->de_epsilon = 1e-3;
        p->de_step_scale = 1.0;
        p->de_bound_radius = 0.0;
        return DQJ_OK;
    });
}

dqj_status dqj_validate_params(const dqj_params *p)
{
    return dqj::guarded([&]() -> dqj_status { return validate(p); });
}

dqj_status dqj_create(const dqj_config *cfg, dqj_ctx **out)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!out) return fail(DQJ_ERR_INVALID, "out is NULL");
        *out = nullptr;
        dqj_config c{};
        if (cfg) c = *cfg;
        if (c.mem_budget_bytes == 0) c.mem_budget_bytes = 16ull << 30;
        if (c.max_pending <= 0) c.max_pending = 4096;
        if (c.device == DQJ_DEVICE_MOCK) {
            dqj_ctx *ctx = new (std::nothrow) dqj_ctx();
            if (!ctx) return fail(DQJ_ERR_NOMEM, "create: out of host memory");
            ctx->device = DQJ_DEVICE_MOCK;
            ctx->cfg = c;
            if (c.autotune_cache) ctx->cache_path = c.autotune_cache;
            ctx->cfg.autotune_cache = nullptr;
            load_tile_cache(ctx);  // a cache written for device "unknown" with 0 SMs applies
            *out = ctx;
            return DQJ_OK;
        }
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess) return cuda_fail(e, "create: cudaGetDeviceCount");
        if (c.device < 0 || c.device >= ndev) return fail(DQJ_ERR_INVALID, "device ordinal out of range");
        e = cudaSetDevice(c.device);
        if (e != cudaSuccess) return cuda_fail(e, "create: cudaSetDevice");
        dqj_ctx *ctx = new (std::nothrow) dqj_ctx();
        if (!ctx) return fail(DQJ_ERR_NOMEM, "create: out of host memory");
        ctx->device = c.device;
        ctx->cfg = c;
        if (c.autotune_cache) ctx->cache_path = c.autotune_cache;
        ctx->cfg.autotune_cache = nullptr;
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, c.device);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->host_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            dqj_status s = cuda_fail(e, "create");
            if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
            delete ctx;
            return s;
        }
        load_tile_cache(ctx);
        *out = ctx;
        return DQJ_OK;
    });
}

dqj_status dqj_render(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, void *cuda_stream)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        return render_on_stream(ctx, p, out, static_cast<cudaStream_t>(cuda_stream));
    });
}

dqj_status dqj_render_tiles(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, void *cuda_stream,
                            int32_t part, int32_t parts)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        return render_on_stream(ctx, p, out, static_cast<cudaStream_t>(cuda_stream), part, parts);
    });
}

dqj_status dqj_render_batch(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, int32_t n, void *cuda_stream)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        if (ctx->device == DQJ_DEVICE_MOCK) return fail(DQJ_ERR_INVALID, "a mock context cannot render");
        if (n < 0 || (n > 0 && (!p || !out))) return fail(DQJ_ERR_INVALID, "bad frame count or NULL arrays");
        for (int32_t i = 0; i < n; ++i) {
            dqj_status s = validate(&p[i]);
            if (s != DQJ_OK) return s;
            s = check_outputs(p[i], &out[i]);
            if (s != DQJ_OK) return s;
        }
        if (n == 0) return DQJ_OK;
        const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(e, "render batch: cudaSetDevice");
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cap);
        if (e != cudaSuccess) return cuda_fail(e, "render batch: cudaStreamIsCapturing");
        if (cap != cudaStreamCaptureStatusNone)
            return fail(DQJ_ERR_INVALID, "render batch: not under stream capture (capture dqj_render calls instead)");
        if (n == 1) return enqueue_frame(ctx, p[0], out[0], st);
        FramePipe pipe{ctx};
        dqj_status s = pipe.open(st);
        for (int32_t i = 0; i < n && s == DQJ_OK; ++i) s = pipe.frame(p[i], out[i]);
        const dqj_status c = pipe.close(st);  // joined even after a failed frame, so st stays ordered
        return s != DQJ_OK ? s : c;
    });
}

dqj_status dqj_render_host_batch(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *host_out, int32_t n)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        if (ctx->device == DQJ_DEVICE_MOCK) return fail(DQJ_ERR_INVALID, "a mock context cannot render");
        if (n < 0 || (n > 0 && (!p || !host_out))) return fail(DQJ_ERR_INVALID, "bad frame count or NULL arrays");
        size_t need = 0;
        for (int32_t i = 0; i < n; ++i) {
            dqj_status s = validate(&p[i]);
            if (s != DQJ_OK) return s;
            s = check_outputs(p[i], &host_out[i]);
            if (s != DQJ_OK) return s;
            const size_t px = (size_t)p[i].width * (size_t)p[i].height;
            need = std::max(need, align_up(px * 24, 256) + DQJ_NSTATS * sizeof(int64_t));
        }
        if (n == 0) return DQJ_OK;
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_fail(e, "render_host: cudaSetDevice");
        if (!ctx->host_copy_stream) e = cudaStreamCreateWithFlags(&ctx->host_copy_stream, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            if (!ctx->host_rendered[b]) e = cudaEventCreateWithFlags(&ctx->host_rendered[b], cudaEventDisableTiming);
            if (e == cudaSuccess && !ctx->host_copied[b])
                e = cudaEventCreateWithFlags(&ctx->host_copied[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "render_host: streams and events");
        const int nbuf = n > 1 ? 2 : 1;
        for (int b = 0; b < nbuf; ++b) {
            if (need <= ctx->host_planes_bytes[b]) continue;
            e = cudaStreamSynchronize(ctx->host_copy_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->host_stream);
            if (e == cudaSuccess && ctx->host_planes[b]) e = cudaFree(ctx->host_planes[b]);
            ctx->host_planes[b] = nullptr;
            ctx->host_planes_bytes[b] = 0;
            if (e == cudaSuccess) e = cudaMalloc(&ctx->host_planes[b], need);
            if (e != cudaSuccess) return cuda_fail(e, "render_host: device planes");
            ctx->host_planes_bytes[b] = need;
        }
        cudaStream_t rs = ctx->host_stream, cs = ctx->host_copy_stream;
        // two or more frames run through the frame pipeline (lane l = i % 2
        // renders into plane set b = i % 2); one frame renders on host_stream
        FramePipe pipe{ctx};
        if (n > 1) {
            const dqj_status s = pipe.open(rs);
            if (s != DQJ_OK) return s;
        }
        for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
            const int b = i % nbuf;
            const dqj_params &pi = p[i];
            const dqj_outputs &ho = host_out[i];
            const size_t px = (size_t)pi.width * (size_t)pi.height;
            char *base = static_cast<char *>(ctx->host_planes[b]);
            dqj_outputs dev{};
            dev.pitch_px = pi.width;
            dev.iter = ho.iter ? reinterpret_cast<int32_t *>(base) : nullptr;
            dev.depth = ho.depth ? reinterpret_cast<float *>(base + px * 4) : nullptr;
            dev.normal = ho.normal ? reinterpret_cast<float *>(base + px * 8) : nullptr;
            dev.rgba = ho.rgba ? reinterpret_cast<uint8_t *>(base + px * 20) : nullptr;
            dev.stats = ho.stats ? reinterpret_cast<int64_t *>(base + align_up(px * 24, 256)) : nullptr;
            // the render into plane set b waits for that set's previous copy back
            cudaStream_t ls = rs;
            dqj_status s = DQJ_OK;
            if (n > 1) {
                s = pipe.frame(pi, dev, &ls, ctx->host_copied[b]);
            } else {
                e = cudaStreamWaitEvent(rs, ctx->host_copied[b], 0);
                if (e != cudaSuccess) break;
                s = enqueue_frame(ctx, pi, dev, rs);
            }
            if (s != DQJ_OK) {
                if (n > 1) pipe.close(rs);
                cudaStreamSynchronize(cs);
                return s;
            }
            e = cudaEventRecord(ctx->host_rendered[b], ls);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ctx->host_rendered[b], 0);
            const size_t w = (size_t)pi.width, hp = (size_t)ho.pitch_px;
            auto copy2d = [&](void *dst, const void *src, size_t elem) {
                return cudaMemcpy2DAsync(dst, hp * elem, src, w * elem, w * elem, (size_t)pi.height,
                                         cudaMemcpyDeviceToHost, cs);
            };
            if (e == cudaSuccess && ho.iter) e = copy2d(ho.iter, dev.iter, 4);
            if (e == cudaSuccess && ho.depth) e = copy2d(ho.depth, dev.depth, 4);
            if (e == cudaSuccess && ho.normal) e = copy2d(ho.normal, dev.normal, 12);
            if (e == cudaSuccess && ho.rgba) e = copy2d(ho.rgba, dev.rgba, 4);
            if (e == cudaSuccess && ho.stats)
                e = cudaMemcpyAsync(ho.stats, dev.stats, DQJ_NSTATS * sizeof(int64_t), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->host_copied[b], cs);
        }
        const dqj_status c = n > 1 ? pipe.close(rs) : DQJ_OK;
        const cudaError_t e2 = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return cuda_fail(e, "render_host: copy back");
        return c;
    });
}

dqj_status dqj_render_host(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *host_out)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!p || !host_out) return fail(DQJ_ERR_INVALID, "params or outputs is NULL");
        return dqj_render_host_batch(ctx, p, host_out, 1);
    });
}

static void free_ring(dqj_ctx *ctx)
{
    for (auto &v : ctx->ev)
        if (v) cudaEventDestroy(v);
    ctx->ev.clear();
    ctx->ring_frames = 0;
    ctx->ring_next = 0;
}

dqj_status dqj_set_profiling(dqj_ctx *ctx, int32_t ring_frames)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
        if (ring_frames < 0 || ring_frames > 4096) return fail(DQJ_ERR_INVALID, "ring_frames must be in 0..4096");
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e == cudaSuccess && ctx->done_ev) e = cudaEventSynchronize(ctx->done_ev);
        if (e != cudaSuccess) return cuda_fail(e, "set_profiling");
        free_ring(ctx);
        if (ring_frames == 0) return DQJ_OK;
        ctx->ev.assign((size_t)ring_frames * 5, nullptr);
        for (auto &v : ctx->ev) {
            e = cudaEventCreate(&v);
            if (e != cudaSuccess) {
                free_ring(ctx);
                return cuda_fail(e, "set_profiling: cudaEventCreate");
            }
        }
        ctx->ring_frames = ring_frames;
        return DQJ_OK;
    });
}

dqj_status dqj_pass_ms(dqj_ctx *ctx, int32_t frames, float *ms)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!ctx || !ms) return fail(DQJ_ERR_INVALID, "ctx or ms is NULL");
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (frames < 1 || frames > ctx->ring_frames) return fail(DQJ_ERR_INVALID, "frames must be in 1..ring_frames");
        if ((uint64_t)frames > ctx->ring_next) return fail(DQJ_ERR_NOT_FOUND, "fewer renders were recorded");
        cudaError_t e = cudaSetDevice(ctx->device);
        for (int f = 0; f < frames && e == cudaSuccess; ++f) {
            const uint64_t idx = ctx->ring_next - (uint64_t)frames + (uint64_t)f;
            cudaEvent_t *ev = &ctx->ev[5 * (idx % (uint64_t)ctx->ring_frames)];
            e = cudaEventSynchronize(ev[4]);
            for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[4 * f + i], ev[i], ev[i + 1]);
        }
        if (e != cudaSuccess) return cuda_fail(e, "pass_ms");
        return DQJ_OK;
    });
}

dqj_status dqj_fma_peak(int32_t device, int32_t variant, int32_t launches, double *flops_per_s)
{
    return dqj::guarded([&]() -> dqj_status {
        if (!flops_per_s) return fail(DQJ_ERR_INVALID, "flops_per_s is NULL");
        if (variant < 0 || variant > 4) return fail(DQJ_ERR_INVALID, "variant must be in 0..4");
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) return cuda_fail(e, "fma_peak: cudaSetDevice");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return cuda_fail(e, "fma_peak: attribute");
        float *sink = nullptr;
        e = cudaMalloc(&sink, (size_t)sms * 2048 * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(e, "fma_peak: cudaMalloc");
        double best = 0.0;
        for (int i = 0; i < (launches > 0 ? launches : 1) && e == cudaSuccess; ++i) {
            double f = 0.0;
            e = fma_peak_launch(variant, sms, sink, nullptr, &f);
            if (f > best) best = f;
        }
        cudaFree(sink);
        if (e != cudaSuccess) return cuda_fail(e, "fma_peak: launch");
        *flops_per_s = best;
        return DQJ_OK;
    });
}

}  // extern "C"
