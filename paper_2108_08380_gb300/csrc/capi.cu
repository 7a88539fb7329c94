// C ABI entry points: context, parameters, validation and dispatch to the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <algorithm>
#include <vector>

#include "bd_internal.h"

namespace bd {

static std::atomic<unsigned long long> g_launches{0};

void note_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

static thread_local TraceScope *t_scope = nullptr;

static void trace_record(TraceScope *sc, cudaStream_t st, const char *label)
{
    bd_ctx *ctx = sc->ctx;
    if (!ctx || !ctx->trace)
        return;
    cudaEvent_t ev = nullptr;
    if (sc->captured) {
        // under capture a plain record only orders nodes: record an external event node
        if (cudaEventCreate(&ev) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        sc->captured->push_back({ev, label});
        if (cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) != cudaSuccess)
            cudaGetLastError();
        return;
    } else {
        if (ctx->trace_next == ctx->trace_pool.size()) {
            if (cudaEventCreate(&ev) != cudaSuccess)
                return;
            ctx->trace_pool.push_back(ev);
        }
        ev = ctx->trace_pool[ctx->trace_next++];
        ctx->marks.push_back({ev, label});
    }
    if (cudaEventRecord(ev, st) != cudaSuccess)
        cudaGetLastError();
}

TraceScope::TraceScope(bd_ctx *c, cudaStream_t st, std::vector<TraceMark> *cap)
    : ctx(c), captured(cap), prev(t_scope)
{
    t_scope = this;
    trace_record(this, st, "begin");
}

TraceScope::~TraceScope() { t_scope = prev; }

void trace_kernel(cudaStream_t st, const char *label)
{
    if (t_scope)
        trace_record(t_scope, st, label);
}

bd_status set_err(bd_ctx *ctx, bd_status s, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

bd_status cuda_err(bd_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess)
        return BD_OK;
    return set_err(ctx, e == cudaErrorMemoryAllocation ? BD_ERR_NOMEM : BD_ERR_CUDA, "%s: %s (%d)",
                   what, cudaGetErrorString(e), (int)e);
}

bd_status ensure_scratch(bd_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_bytes)
        return BD_OK;
    const size_t want = align_up(bytes, (size_t)2 << 20);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "scratch: stream synchronize");
    if (ctx->scratch) {
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) {
        ctx->scratch = nullptr;
        return cuda_err(ctx, e, "scratch: cudaMalloc");
    }
    ctx->scratch_bytes = want;
    return BD_OK;
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode_fn()
{
    static PFN_encodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

bool encode_tmap_2d_bf16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer)
{
    PFN_encodeTiled fn = get_encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_tmap_2d_u8(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                       uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer)
{
    PFN_encodeTiled fn = get_encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess)
            ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

static bool image_ok(int w, int h, int pitch)
{
    if (w < 1 || h < 1 || w > kMaxImageSide || h > kMaxImageSide || pitch < w)
        return false;
    return 255.0 * (double)w * (double)h < 4294967296.0;
}

static long long floor_div(long long a, long long b)
{
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0)))
        --q;
    return q;
}

}  // namespace bd

using namespace bd;

#define BD_GUARD(ctx)                                                        \
    if (!(ctx))                                                              \
        return BD_ERR_INVALID;                                               \
    DeviceGuard _guard((ctx)->device);                                       \
    if (!_guard.ok)                                                          \
        return set_err((ctx), BD_ERR_CUDA, "cannot make device %d current", (ctx)->device)

#define BD_LAUNCH(ctx, expr, what)                                           \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess)                                               \
            return cuda_err((ctx), _e, (what));                              \
    } while (0)

extern "C" {

bd_status bd_create(int device, void *stream, bd_ctx **out)
{
    if (!out)
        return BD_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return BD_ERR_INVALID;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return BD_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3)
        return BD_ERR_UNSUPPORTED;  // built for sm_103a only
    bd_ctx *ctx = new bd_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    ctx->sm_count = prop.multiProcessorCount;
    DeviceGuard g(device);
    if (!g.ok || cudaMalloc(&ctx->status, sizeof(DeviceStatus)) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(DeviceStatus)) != cudaSuccess) {
        if (ctx->status)
            cudaFree(ctx->status);
        delete ctx;
        return BD_ERR_NOMEM;
    }
    *out = ctx;
    return BD_OK;
}

void bd_destroy(bd_ctx *ctx)
{
    if (!ctx)
        return;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        for (cudaEvent_t ev : ctx->trace_pool)
            cudaEventDestroy(ev);
        if (ctx->scratch)
            cudaFree(ctx->scratch);
        if (ctx->arrivals)
            cudaFree(ctx->arrivals);
        if (ctx->status)
            cudaFree(ctx->status);
    }
    delete ctx;
}

bd_status bd_set_stream(bd_ctx *ctx, void *stream)
{
    if (!ctx)
        return BD_ERR_INVALID;
    ctx->stream = (cudaStream_t)stream;
    return BD_OK;
}

const char *bd_last_error(const bd_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t bd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

bd_status bd_trace_enable(bd_ctx *ctx, int on)
{
    if (!ctx)
        return BD_ERR_INVALID;
    ctx->trace = on != 0;
    return BD_OK;
}

bd_status bd_trace_reset(bd_ctx *ctx)
{
    if (!ctx)
        return BD_ERR_INVALID;
    ctx->marks.clear();
    ctx->trace_next = 0;
    return BD_OK;
}

int bd_trace_read(bd_ctx *ctx, int max, float *ms, const char **labels)
{
    if (!ctx || max < 0)
        return -1;
    DeviceGuard g(ctx->device);
    if (ctx->marks.empty())
        return 0;
    if (cudaEventSynchronize(ctx->marks.back().ev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    int n = 0;
    for (size_t i = 1; i < ctx->marks.size() && n < max; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ctx->marks[i - 1].ev, ctx->marks[i].ev) != cudaSuccess) {
            cudaGetLastError();  // leave no pending error behind for the next launch check
            t = -1.f;
        }
        if (ms)
            ms[n] = t;
        if (labels)
            labels[n] = ctx->marks[i].label;
        ++n;
    }
    return n;
}

bd_status bd_sync_status(bd_ctx *ctx, uint32_t *flags)
{
    BD_GUARD(ctx);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_sync_status: synchronize");
    unsigned long long f = 0;
    e = cudaMemcpy(&f, &ctx->status->flags, sizeof(f), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_sync_status: read flags");
    e = cudaMemset(&ctx->status->flags, 0, sizeof(f));
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_sync_status: clear flags");
    if (flags)
        *flags = (uint32_t)f;
    if (f & BD_FLAG_TIMEOUT)
        return set_err(ctx, BD_ERR_TIMEOUT, "a device-side wait timed out");
    if (f)
        return set_err(ctx, BD_ERR_DEVICE_CHECK, "device flags 0x%llx", f);
    return BD_OK;
}

bd_status bd_rescued_count(bd_ctx *ctx, uint64_t *count, int reset)
{
    BD_GUARD(ctx);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_rescued_count: synchronize");
    unsigned long long c = 0;
    e = cudaMemcpy(&c, &ctx->status->rescued, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_rescued_count: read");
    if (count)
        *count = c;
    if (reset) {
        e = cudaMemset(&ctx->status->rescued, 0, sizeof(c));
        if (e != cudaSuccess)
            return cuda_err(ctx, e, "bd_rescued_count: reset");
    }
    return BD_OK;
}

bd_status bd_reserve(bd_ctx *ctx, size_t bytes)
{
    BD_GUARD(ctx);
    return ensure_scratch(ctx, bytes);
}

size_t bd_scratch_bytes_bad(int w, int h)
{
    if (!image_ok(w, h, w))
        return 0;
    return align_up((size_t)(h + 1) * (size_t)(w + 1) * 4, 256) + integral_scratch_bytes(w, h);
}

size_t bd_scratch_bytes_hashsift(int n)
{
    if (n < 0)
        return 0;
    return align_up((size_t)n * kHistDim * 4, 256);
}

size_t bd_scratch_bytes_match(int nq, int nt, int nbits)
{
    // sized for the largest GPU the library supports (the split count grows with the SM count)
    return match_scratch_bytes(nq, nt, nbits, 256);
}

// ---------------------------------------------------------------------------
// BAD parameters
// ---------------------------------------------------------------------------

bd_status bd_bad_params_create(bd_ctx *ctx, int nbits, const uint8_t *centres,
                               const uint8_t *sides, const int32_t *thr_num, int32_t thr_den,
                               int n_angle_bins, const float *level_scales, int n_levels,
                               bd_bad_params **out)
{
    BD_GUARD(ctx);
    if (!out || !centres || !sides || !thr_num || !level_scales)
        return set_err(ctx, BD_ERR_INVALID, "bd_bad_params_create: null pointer");
    *out = nullptr;
    if (nbits != 256 && nbits != 512)
        return set_err(ctx, BD_ERR_INVALID, "nbits must be 256 or 512 (got %d)", nbits);
    if (thr_den <= 0)
        return set_err(ctx, BD_ERR_INVALID, "thr_den must be > 0");
    if (n_angle_bins < 1 || n_angle_bins > kMaxAngleBins)
        return set_err(ctx, BD_ERR_INVALID, "n_angle_bins must be in [1, %d]", kMaxAngleBins);
    if (n_levels < 1 || n_levels > kMaxLevels)
        return set_err(ctx, BD_ERR_INVALID, "n_levels must be in [1, %d]", kMaxLevels);
    for (int l = 0; l < n_levels; ++l) {
        const float s = level_scales[l];
        if (!(s > 0.f) || s > 32.f || (l > 0 && !(s > level_scales[l - 1])))
            return set_err(ctx, BD_ERR_INVALID,
                           "level_scales must be strictly increasing in (0, 32]");
    }
    for (int k = 0; k < nbits; ++k) {
        if (sides[k] < 1 || sides[k] > 64)
            return set_err(ctx, BD_ERR_INVALID, "box side %d of pair %d not in [1, 64]", sides[k], k);
        for (int q = 0; q < 4; ++q)
            if (centres[k * 4 + q] > 31)
                return set_err(ctx, BD_ERR_INVALID, "box centre of pair %d outside 0..31", k);
    }

    bd_bad_params *p = new bd_bad_params();
    p->ctx = ctx;
    p->nbits = nbits;
    p->nbins = n_angle_bins;
    p->nlevels = n_levels;
    p->thr_den = thr_den;
    const double kPi = 3.14159265358979323846;
    p->angle_scale = (float)((double)n_angle_bins / (2.0 * kPi));
    for (int l = 0; l + 1 < n_levels; ++l)
        p->level_mid[l] = (float)sqrt((double)level_scales[l] * (double)level_scales[l + 1]);

    // Rotated, scaled box geometry per (level, angle bin): the patch frame offset
    // d = u - (16,16) maps to round(sigma * R(theta_b) d), R in image coordinates
    // (y down), theta_b = 2 pi b / NB; the side scales to max(1, round(s sigma)).
    const size_t nt = (size_t)n_levels * n_angle_bins * nbits;
    p->h_offsets = new int32_t[nt * 4];
    p->h_sides = new int32_t[(size_t)n_levels * nbits];
    std::vector<short4> corner(nt);
    std::vector<int2> side_thr((size_t)n_levels * nbits);
    for (int l = 0; l < n_levels; ++l) {
        const double sg = (double)level_scales[l];
        for (int k = 0; k < nbits; ++k) {
            long long sp = llround((double)sides[k] * sg);
            if (sp < 1)
                sp = 1;
            p->h_sides[(size_t)l * nbits + k] = (int32_t)sp;
            // den*(sum1 - sum2) <= num*s'^2  <=>  sum1 - sum2 <= floor(num*s'^2 / den)
            long long t = floor_div((long long)thr_num[k] * sp * sp, (long long)thr_den);
            if (t > 2147483647LL)
                t = 2147483647LL;
            if (t < -2147483647LL - 1)
                t = -2147483647LL - 1;
            side_thr[(size_t)l * nbits + k] = make_int2((int)sp, (int)t);
        }
        for (int b = 0; b < n_angle_bins; ++b) {
            const double th = 2.0 * kPi * (double)b / (double)n_angle_bins;
            const double c = cos(th), s = sin(th);
            for (int k = 0; k < nbits; ++k) {
                const size_t e = ((size_t)l * n_angle_bins + b) * nbits + k;
                const int sp = p->h_sides[(size_t)l * nbits + k];
                int o[4];
                for (int j = 0; j < 2; ++j) {
                    const double dx = (double)centres[k * 4 + j * 2 + 0] - 16.0;
                    const double dy = (double)centres[k * 4 + j * 2 + 1] - 16.0;
                    o[j * 2 + 0] = (int)llround(sg * (c * dx - s * dy));
                    o[j * 2 + 1] = (int)llround(sg * (s * dx + c * dy));
                }
                for (int q = 0; q < 4; ++q)
                    p->h_offsets[e * 4 + q] = o[q];
                const int half = sp / 2;
                corner[e] = make_short4((short)(o[0] - half), (short)(o[1] - half),
                                        (short)(o[2] - half), (short)(o[3] - half));
            }
        }
    }
    // The kernels' table: per (level, bin) the 2K boxes (x, y, side, id = 2 k + j),
    // sorted by top-left row, side and column so that a warp's 32 consecutive
    // boxes fall on few image rows.
    std::vector<short4> box(nt * 2);
    for (int l = 0; l < n_levels; ++l)
        for (int b = 0; b < n_angle_bins; ++b) {
            const size_t base = ((size_t)l * n_angle_bins + b) * nbits;
            short4 *dst = box.data() + base * 2;
            for (int k = 0; k < nbits; ++k) {
                const short4 c = corner[base + k];
                const short sp = (short)side_thr[(size_t)l * nbits + k].x;
                dst[2 * k] = make_short4(c.x, c.y, sp, (short)(2 * k));
                dst[2 * k + 1] = make_short4(c.z, c.w, sp, (short)(2 * k + 1));
            }
            std::sort(dst, dst + 2 * nbits, [](const short4 &a, const short4 &c) {
                if (a.y != c.y)
                    return a.y < c.y;
                if (a.z != c.z)
                    return a.z < c.z;
                if (a.x != c.x)
                    return a.x < c.x;
                return a.w < c.w;
            });
        }
    std::vector<int> thr(side_thr.size());
    for (size_t i = 0; i < thr.size(); ++i)
        thr[i] = side_thr[i].y;
    std::vector<short4> pbox(nbits);
    std::vector<int> pside(nbits);
    for (int k = 0; k < nbits; ++k) {
        const int s = sides[k];
        pside[k] = s;
        pbox[k] = make_short4((short)(centres[k * 4 + 0] - s / 2), (short)(centres[k * 4 + 1] - s / 2),
                              (short)(centres[k * 4 + 2] - s / 2), (short)(centres[k * 4 + 3] - s / 2));
    }
    cudaError_t e = cudaMalloc(&p->d_box, box.size() * sizeof(short4));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->d_patch_box, nbits * sizeof(short4));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->d_patch_side, nbits * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_patch_box, pbox.data(), nbits * sizeof(short4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_patch_side, pside.data(), nbits * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&p->d_thr, side_thr.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_box, box.data(), box.size() * sizeof(short4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_thr, thr.data(), thr.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        bd_bad_params_destroy(p);
        return cuda_err(ctx, e, "bd_bad_params_create: upload");
    }
    *out = p;
    return BD_OK;
}

void bd_bad_params_destroy(bd_bad_params *p)
{
    if (!p)
        return;
    {
        DeviceGuard g(p->ctx->device);
        if (p->d_box)
            cudaFree(p->d_box);
        if (p->d_thr)
            cudaFree(p->d_thr);
        if (p->d_patch_box)
            cudaFree(p->d_patch_box);
        if (p->d_patch_side)
            cudaFree(p->d_patch_side);
    }
    delete[] p->h_offsets;
    delete[] p->h_sides;
    delete p;
}

bd_status bd_bad_params_table(const bd_bad_params *p, int32_t *offsets, int32_t *sides_out)
{
    if (!p || !offsets || !sides_out)
        return BD_ERR_INVALID;
    const size_t nt = (size_t)p->nlevels * p->nbins * p->nbits;
    memcpy(offsets, p->h_offsets, nt * 4 * sizeof(int32_t));
    memcpy(sides_out, p->h_sides, (size_t)p->nlevels * p->nbits * sizeof(int32_t));
    return BD_OK;
}

// ---------------------------------------------------------------------------
// HashSIFT parameters
// ---------------------------------------------------------------------------

bd_status bd_hs_params_create(bd_ctx *ctx, int nbits, const float *W, const float *bias,
                              float spacing, int precision, float band, bd_hs_params **out)
{
    BD_GUARD(ctx);
    if (!out || !W || !bias)
        return set_err(ctx, BD_ERR_INVALID, "bd_hs_params_create: null pointer");
    *out = nullptr;
    if (nbits != 256 && nbits != 512)
        return set_err(ctx, BD_ERR_INVALID, "nbits must be 256 or 512 (got %d)", nbits);
    if (!(spacing > 0.f) || spacing > 16.f)
        return set_err(ctx, BD_ERR_INVALID, "spacing must be in (0, 16]");
    if (precision != BD_HS_FP32 && precision != BD_HS_BF16_RESCUE)
        return set_err(ctx, BD_ERR_INVALID, "unknown precision %d", precision);
    if (!isfinite(band))
        return set_err(ctx, BD_ERR_INVALID, "band must be finite");
    const int K = nbits;
    for (size_t i = 0; i < (size_t)128 * K; ++i)
        if (!isfinite(W[i]))
            return set_err(ctx, BD_ERR_INVALID, "W has a non-finite entry");
    for (int k = 0; k < K; ++k)
        if (!isfinite(bias[k]))
            return set_err(ctx, BD_ERR_INVALID, "bias has a non-finite entry");

    bd_hs_params *p = new bd_hs_params();
    p->ctx = ctx;
    p->nbits = K;
    p->precision = precision;
    p->spacing = spacing;
    std::vector<float> Wt((size_t)K * 128), bnd(K);
    std::vector<__nv_bfloat16> Whi((size_t)K * 128), Wlo((size_t)K * 128);
    bool has_lo = false;
    for (int k = 0; k < K; ++k) {
        double nn = 0.0;
        for (int i = 0; i < 128; ++i) {
            const float v = W[(size_t)i * K + k];
            Wt[(size_t)k * 128 + i] = v;
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            Whi[(size_t)k * 128 + i] = hi;
            Wlo[(size_t)k * 128 + i] = lo;
            has_lo = has_lo || __bfloat162float(hi) != v;  // W is exactly BF16 only without this
            nn += (double)v * (double)v;
        }
        // With x = hi + lo + d, |d| <= 2^-16 |x| (two BF16 roundings), the three
        // products hi*hi + lo*hi + hi*lo miss |W||f| by at most 3*2^-16 + O(2^-24);
        // FP32 accumulation of 384 products adds <= 384*2^-24, the FP32 path's own
        // 128-term rounding <= 128*2^-24.  All of it, times ||W_k||_2 ||f||_2
        // (||f|| = 1), stays below 2^-13 ||W_k||_2.
        const double c = ldexp(1.0, -13);
        bnd[k] = band < 0.f ? (float)(c * sqrt(nn)) : band;
    }
    p->w_has_lo = has_lo;
    cudaError_t e = cudaMalloc(&p->d_W, sizeof(float) * 128 * K);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_Wt, sizeof(float) * 128 * K);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_Wt16_hi, sizeof(__nv_bfloat16) * 128 * K);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_Wt16_lo, sizeof(__nv_bfloat16) * 128 * K);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_bias, sizeof(float) * K);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_band, sizeof(float) * K);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_W, W, sizeof(float) * 128 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_Wt, Wt.data(), sizeof(float) * 128 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_Wt16_hi, Whi.data(), sizeof(__nv_bfloat16) * 128 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_Wt16_lo, Wlo.data(), sizeof(__nv_bfloat16) * 128 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_bias, bias, sizeof(float) * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_band, bnd.data(), sizeof(float) * K, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        bd_hs_params_destroy(p);
        return cuda_err(ctx, e, "bd_hs_params_create: upload");
    }
    p->tmap_ok = encode_tmap_2d_bf16(&p->tmap_w_hi, p->d_Wt16_hi, 128, (uint64_t)K, 256, 64, 128) &&
                 encode_tmap_2d_bf16(&p->tmap_w_lo, p->d_Wt16_lo, 128, (uint64_t)K, 256, 64, 128);
    if (precision == BD_HS_BF16_RESCUE && !p->tmap_ok) {
        bd_hs_params_destroy(p);
        return set_err(ctx, BD_ERR_UNSUPPORTED, "cannot encode the TMA descriptor of W");
    }
    e = prepare_hs_proj_tc();
    if (e != cudaSuccess) {
        bd_hs_params_destroy(p);
        return cuda_err(ctx, e, "bd_hs_params_create: projection kernel attribute");
    }
    *out = p;
    return BD_OK;
}

bd_status bd_hs_params_set_variant(bd_hs_params *p, int flags)
{
    if (!p)
        return BD_ERR_INVALID;
    if (flags & ~(BD_HS_VARIANT_TRILINEAR | BD_HS_VARIANT_CLIP | BD_HS_VARIANT_ROOT))
        return set_err(p->ctx, BD_ERR_INVALID, "bd_hs_params_set_variant: unknown flags 0x%x", flags);
    p->variant = flags;
    return BD_OK;
}

void bd_hs_params_destroy(bd_hs_params *p)
{
    if (!p)
        return;
    DeviceGuard g(p->ctx->device);
    if (p->d_W) cudaFree(p->d_W);
    if (p->d_Wt) cudaFree(p->d_Wt);
    if (p->d_Wt16_hi) cudaFree(p->d_Wt16_hi);
    if (p->d_Wt16_lo) cudaFree(p->d_Wt16_lo);
    if (p->d_bias) cudaFree(p->d_bias);
    if (p->d_band) cudaFree(p->d_band);
    delete p;
}

// ---------------------------------------------------------------------------
// work
// ---------------------------------------------------------------------------

bd_status bd_integral(bd_ctx *ctx, const uint8_t *img, int w, int h, int pitch, uint32_t *ii,
                      int ii_stride)
{
    BD_GUARD(ctx);
    if (!img || !ii || !image_ok(w, h, pitch) || ii_stride < w + 1)
        return set_err(ctx, BD_ERR_INVALID, "bd_integral: bad arguments");
    bd_status s = ensure_scratch(ctx, integral_scratch_bytes(w, h));
    if (s != BD_OK)
        return s;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_integral(img, w, h, pitch, ii, ii_stride,
                              integral_scratch_carve(ctx->scratch, w, h), ctx->stream),
              "integral kernels");
    return BD_OK;
}

bd_status bd_bad_describe(bd_ctx *ctx, const bd_bad_params *p, const uint8_t *img, int w, int h,
                          int pitch, const bd_keypoint *kps, int n, uint32_t *out)
{
    BD_GUARD(ctx);
    if (!p || !img || !image_ok(w, h, pitch) || n < 0 || (n > 0 && (!kps || !out)))
        return set_err(ctx, BD_ERR_INVALID, "bd_bad_describe: bad arguments");
    if (n == 0)
        return BD_OK;
    const int stride = w + 1;
    const size_t ii_bytes = align_up((size_t)(h + 1) * stride * 4, 256);
    bd_status s = ensure_scratch(ctx, ii_bytes + integral_scratch_bytes(w, h));
    if (s != BD_OK)
        return s;
    uint32_t *ii = (uint32_t *)ctx->scratch;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_integral(img, w, h, pitch, ii, stride,
                              integral_scratch_carve((char *)ctx->scratch + ii_bytes, w, h),
                              ctx->stream),
              "integral kernels");
    BD_LAUNCH(ctx, launch_bad_gather(p, ii, stride, w, h, kps, n, out, ctx->status, ctx->stream),
              "BAD gather kernel");
    return BD_OK;
}

bd_status bd_hashsift_warp(bd_ctx *ctx, const bd_hs_params *p, const uint8_t *img, int w, int h,
                           int pitch, const bd_keypoint *kps, int n, float *patches)
{
    BD_GUARD(ctx);
    if (!p || !img || !image_ok(w, h, pitch) || n < 0 || (n > 0 && (!kps || !patches)))
        return set_err(ctx, BD_ERR_INVALID, "bd_hashsift_warp: bad arguments");
    if (n == 0)
        return BD_OK;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_hs_warp(p, img, w, h, pitch, kps, n, patches, ctx->status, ctx->stream,
                             ctx->sm_count),
              "patch warp kernel");
    return BD_OK;
}

bd_status bd_hashsift_hist(bd_ctx *ctx, const float *patches, int n, float *hist)
{
    BD_GUARD(ctx);
    if (n < 0 || (n > 0 && (!patches || !hist)))
        return set_err(ctx, BD_ERR_INVALID, "bd_hashsift_hist: bad arguments");
    if (n == 0)
        return BD_OK;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx, launch_hs_hist_patches(patches, n, hist, ctx->stream, ctx->sm_count),
              "histogram kernel");
    return BD_OK;
}

static bd_status project(bd_ctx *ctx, const bd_hs_params *p, const float *hist, int n,
                         uint32_t *out, const bd_keypoint *kps)
{
    if (p->precision == BD_HS_FP32) {
        BD_LAUNCH(ctx, launch_hs_proj_fp32(p, hist, n, out, ctx->stream, kps),
                  "FP32 projection kernel");
        return BD_OK;
    }
    BD_LAUNCH(ctx, launch_hs_proj_tc(p, hist, n, out, ctx->status, ctx->stream, kps),
              "tcgen05 projection kernel");
    return BD_OK;
}

bd_status bd_hashsift_project(bd_ctx *ctx, const bd_hs_params *p, const float *hist, int n,
                              uint32_t *out)
{
    BD_GUARD(ctx);
    if (!p || n < 0 || (n > 0 && (!hist || !out)))
        return set_err(ctx, BD_ERR_INVALID, "bd_hashsift_project: bad arguments");
    if (n == 0)
        return BD_OK;
    if (p->precision == BD_HS_BF16_RESCUE && ((uintptr_t)hist & 15))
        return set_err(ctx, BD_ERR_INVALID, "bd_hashsift_project: hist must be 16-byte aligned");
    TraceScope scope(ctx, ctx->stream);
    return project(ctx, p, hist, n, out, nullptr);
}

bd_status bd_hashsift_describe(bd_ctx *ctx, const bd_hs_params *p, const uint8_t *img, int w,
                               int h, int pitch, const bd_keypoint *kps, int n, uint32_t *out,
                               float *hist_out)
{
    BD_GUARD(ctx);
    if (!p || !img || !image_ok(w, h, pitch) || n < 0 || (n > 0 && (!kps || !out)))
        return set_err(ctx, BD_ERR_INVALID, "bd_hashsift_describe: bad arguments");
    if (hist_out && ((uintptr_t)hist_out & 15))
        return set_err(ctx, BD_ERR_INVALID, "bd_hashsift_describe: hist_out must be 16-byte aligned");
    if (n == 0)
        return BD_OK;
    bd_status s = ensure_scratch(ctx, bd_scratch_bytes_hashsift(n));
    if (s != BD_OK)
        return s;
    float *h32 = hist_out ? hist_out : (float *)ctx->scratch;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_hs_hist_image(p, img, w, h, pitch, kps, n, h32, ctx->status, ctx->stream,
                                   ctx->sm_count),
              "fused warp + histogram kernel");
    return project(ctx, p, h32, n, out, kps);
}

static bd_status ensure_arrivals(bd_ctx *ctx, int qblocks)
{
    if (qblocks <= ctx->arrivals_cap)
        return BD_OK;
    const int cap = qblocks < 4096 ? 4096 : qblocks;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && ctx->arrivals)
        e = cudaFree(ctx->arrivals);
    ctx->arrivals = nullptr;
    ctx->arrivals_cap = 0;
    if (e == cudaSuccess)
        e = cudaMalloc(&ctx->arrivals, sizeof(unsigned int) * cap);
    if (e == cudaSuccess)
        e = cudaMemset(ctx->arrivals, 0, sizeof(unsigned int) * cap);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "arrival counters");
    ctx->arrivals_cap = cap;
    return BD_OK;
}

bd_status bd_match_tc(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits,
                      int ratio_num, int ratio_den, bd_match_result *out)
{
    BD_GUARD(ctx);
    if (((uintptr_t)q & 15) || ((uintptr_t)t & 15) || ((uintptr_t)out & 3))
        return set_err(ctx, BD_ERR_INVALID,
                       "bd_match_tc: descriptor arrays must be 16-byte and out 4-byte aligned");
    if ((nbits != 256 && nbits != 512) || nq < 0 || nt < 0 || nt > (int)kMatchIdxMask ||
        ratio_den <= 0 || ratio_num <= 0 || ratio_num > ratio_den || (nq > 0 && (!q || !out)) ||
        (nt > 0 && !t) || (nq + 127) / 128 > 65535)
        return set_err(ctx, BD_ERR_INVALID, "bd_match_tc: bad arguments");
    if (nq == 0)
        return BD_OK;
    bd_status s = ensure_scratch(ctx, match_tc_scratch_bytes(nq, nt, nbits, ctx->sm_count));
    if (s == BD_OK)
        s = ensure_arrivals(ctx, match_tc_query_blocks(nq));
    if (s != BD_OK)
        return s;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_match_tc(ctx, q, nq, t, nt, nbits, ratio_num, ratio_den, out, ctx->scratch,
                              ctx->stream, ctx->arrivals),
              "tensor-core matching kernels");
    return BD_OK;
}

bd_status bd_match(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits,
                   int ratio_num, int ratio_den, bd_match_result *out)
{
    BD_GUARD(ctx);
    if (((uintptr_t)q & 15) || ((uintptr_t)t & 15) || ((uintptr_t)out & 3))
        return set_err(ctx, BD_ERR_INVALID,
                       "bd_match: descriptor arrays must be 16-byte and out 4-byte aligned");
    if ((nbits != 256 && nbits != 512) || nq < 0 || nt < 0 || nt > (int)kMatchIdxMask ||
        ratio_den <= 0 || ratio_num <= 0 || ratio_num > ratio_den || (nq > 0 && (!q || !out)) ||
        (nt > 0 && !t))
        return set_err(ctx, BD_ERR_INVALID, "bd_match: bad arguments");
    if (nq == 0)
        return BD_OK;
    bd_status s = ensure_scratch(ctx, match_scratch_bytes(nq, nt, nbits, ctx->sm_count));
    if (s != BD_OK)
        return s;
    s = ensure_arrivals(ctx, match_query_blocks(nq));
    if (s != BD_OK)
        return s;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_match(q, nq, t, nt, nbits, ratio_num, ratio_den, out, ctx->scratch,
                           ctx->sm_count, ctx->stream, ctx->arrivals),
              "matching kernel");
    return BD_OK;
}

bd_status bd_match_batch(bd_ctx *ctx, const bd_match_job *jobs, int n_jobs)
{
    BD_GUARD(ctx);
    if (n_jobs < 0 || n_jobs > BD_MATCH_MAX_JOBS || (n_jobs > 0 && !jobs))
        return set_err(ctx, BD_ERR_INVALID, "bd_match_batch: bad job count");
    for (int k = 0; k < n_jobs; ++k) {
        const bd_match_job &a = jobs[k];
        if (((uintptr_t)a.q & 15) || ((uintptr_t)a.t & 15) || ((uintptr_t)a.out & 3) ||
            (a.nbits != 256 && a.nbits != 512) || a.nq < 0 || a.nt < 0 ||
            a.nt > (int)kMatchIdxMask || a.ratio_den <= 0 || a.ratio_num <= 0 ||
            a.ratio_num > a.ratio_den || (a.nq > 0 && (!a.q || !a.out)) || (a.nt > 0 && !a.t))
            return set_err(ctx, BD_ERR_INVALID, "bd_match_batch: job %d has bad arguments", k);
    }
    bd_status s = ensure_scratch(ctx, match_batch_scratch_bytes(jobs, n_jobs, ctx->sm_count));
    if (s == BD_OK)
        s = ensure_arrivals(ctx, match_batch_query_blocks(jobs, n_jobs));
    if (s != BD_OK)
        return s;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_match_batch(jobs, n_jobs, ctx->scratch, ctx->sm_count, ctx->stream,
                                 ctx->arrivals),
              "batched matching kernel");
    return BD_OK;
}

bd_status bd_match_mnn(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                       int nbits, int ratio_num, int ratio_den, int tensor_cores,
                       bd_match_result *out, int32_t *mnn)
{
    BD_GUARD(ctx);
    if (((uintptr_t)q & 15) || ((uintptr_t)t & 15) || ((uintptr_t)out & 3) || ((uintptr_t)mnn & 3))
        return set_err(ctx, BD_ERR_INVALID,
                       "bd_match_mnn: descriptor arrays must be 16-byte, out and mnn 4-byte aligned");
    if ((nbits != 256 && nbits != 512) || nq < 0 || nt < 0 || nt > (int)kMatchIdxMask ||
        nq > (int)kMatchIdxMask || ratio_den <= 0 || ratio_num <= 0 || ratio_num > ratio_den ||
        (nq > 0 && (!q || !out || !mnn)) || (nt > 0 && !t) ||
        (tensor_cores && ((nq + 127) / 128 > 65535 || (nt + 127) / 128 > 65535)))
        return set_err(ctx, BD_ERR_INVALID, "bd_match_mnn: bad arguments");
    if (nq == 0)
        return BD_OK;
    // reverse records first in the scratch area, the matchings' own scratch after them
    const size_t rev_bytes = align_up((size_t)(nt > 0 ? nt : 1) * sizeof(bd_match_result), 256);
    size_t need = tensor_cores ? match_tc_scratch_bytes(nq, nt, nbits, ctx->sm_count)
                               : match_scratch_bytes(nq, nt, nbits, ctx->sm_count);
    int qblocks = tensor_cores ? match_tc_query_blocks(nq) : match_query_blocks(nq);
    if (nt > 0) {
        const size_t rn = tensor_cores ? match_tc_scratch_bytes(nt, nq, nbits, ctx->sm_count)
                                       : match_scratch_bytes(nt, nq, nbits, ctx->sm_count);
        const int rb = tensor_cores ? match_tc_query_blocks(nt) : match_query_blocks(nt);
        need = need > rn ? need : rn;
        qblocks = qblocks > rb ? qblocks : rb;
    }
    bd_status s = ensure_scratch(ctx, rev_bytes + need);
    if (s == BD_OK)
        s = ensure_arrivals(ctx, qblocks);
    if (s != BD_OK)
        return s;
    bd_match_result *rev = (bd_match_result *)ctx->scratch;
    void *work = (char *)ctx->scratch + rev_bytes;
    TraceScope scope(ctx, ctx->stream);
    if (tensor_cores) {
        BD_LAUNCH(ctx,
                  launch_match_tc(ctx, q, nq, t, nt, nbits, ratio_num, ratio_den, out, work,
                                  ctx->stream, ctx->arrivals),
                  "tensor-core matching kernels");
        if (nt > 0)
            BD_LAUNCH(ctx,
                      launch_match_tc(ctx, t, nt, q, nq, nbits, ratio_num, ratio_den, rev, work,
                                      ctx->stream, ctx->arrivals),
                      "tensor-core matching kernels (reverse)");
    } else {
        BD_LAUNCH(ctx,
                  launch_match(q, nq, t, nt, nbits, ratio_num, ratio_den, out, work, ctx->sm_count,
                               ctx->stream, ctx->arrivals),
                  "matching kernel");
        if (nt > 0)
            BD_LAUNCH(ctx,
                      launch_match(t, nt, q, nq, nbits, ratio_num, ratio_den, rev, work,
                                   ctx->sm_count, ctx->stream, ctx->arrivals),
                      "matching kernel (reverse)");
    }
    BD_LAUNCH(ctx, launch_mnn_cross(out, rev, nq, mnn, ctx->stream), "mutual check kernel");
    return BD_OK;
}

bd_status bd_select_feature(bd_ctx *ctx, const uint8_t *patches, int n, const int32_t *sim_ap,
                            const int32_t *sim_an, int tau, const int32_t *centres,
                            const int32_t *sides, int J, int32_t *theta_q, int64_t *loss,
                            int32_t *best)
{
    BD_GUARD(ctx);
    if (n < 1 || n > (1 << 20) || J < 1 || J >= (1 << 20) || !patches || !sim_ap || !sim_an ||
        !centres || !sides || !theta_q || !loss || !best || ((uintptr_t)loss & 7) ||
        ((uintptr_t)sim_ap & 3) || ((uintptr_t)sim_an & 3) || ((uintptr_t)theta_q & 3) ||
        ((uintptr_t)best & 3) || tau < -(1 << 20) || tau > (1 << 20))
        return set_err(ctx, BD_ERR_INVALID, "bd_select_feature: bad arguments");
    int max_side = 1;
    for (int j = 0; j < J; ++j) {
        max_side = sides[j] > max_side ? sides[j] : max_side;
        if (sides[j] < 1 || sides[j] > 32)
            return set_err(ctx, BD_ERR_INVALID, "bd_select_feature: side of candidate %d", j);
        for (int q = 0; q < 4; ++q)
            if (centres[4 * j + q] <= -(1 << 15) || centres[4 * j + q] >= (1 << 15))
                return set_err(ctx, BD_ERR_INVALID, "bd_select_feature: centre of candidate %d", j);
    }
    // scratch: [candidates][state + keys], the keys capped at 1 GiB per pass
    const size_t cand_bytes = align_up((size_t)J * 16, 256) + align_up((size_t)J * 4, 256);
    size_t work = select_scratch_bytes(n, J);
    const size_t cap = ((size_t)1 << 30) + 256;
    if (work > cap)
        work = cap;
    if (work < select_scratch_bytes_pass(n, J, 1))
        work = select_scratch_bytes_pass(n, J, 1);
    bd_status s = ensure_scratch(ctx, cand_bytes + work);
    if (s != BD_OK)
        return s;
    int32_t *d_xy = (int32_t *)ctx->scratch;
    int32_t *d_side = (int32_t *)((char *)ctx->scratch + align_up((size_t)J * 16, 256));
    cudaError_t e = cudaMemcpyAsync(d_xy, centres, (size_t)J * 16, cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_side, sides, (size_t)J * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_select_feature: candidate upload");
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_select_feature(patches, n, sim_ap, sim_an, tau, d_xy, d_side, max_side, J, theta_q, loss,
                                    best, (char *)ctx->scratch + cand_bytes, work, ctx->stream),
              "feature selection kernels");
    return BD_OK;
}

bd_status bd_probe(bd_ctx *ctx, int kind, const uint32_t *table, size_t table_words,
                   size_t window_words, int reps, uint32_t *sink, uint64_t *units)
{
    BD_GUARD(ctx);
    if (!units)
        return set_err(ctx, BD_ERR_INVALID, "bd_probe: null units");
    unsigned long long u = 0;
    bool bad = false;
    TraceScope scope(ctx, ctx->stream);
    BD_LAUNCH(ctx,
              launch_probe(kind, table, table_words, window_words, reps, sink, ctx->sm_count,
                           ctx->stream, &u, &bad),
              "probe kernel");
    if (bad)
        return set_err(ctx, BD_ERR_INVALID, "bd_probe: bad kind, repetitions or gather geometry");
    *units = (uint64_t)u;
    return BD_OK;
}

}  // extern "C"
