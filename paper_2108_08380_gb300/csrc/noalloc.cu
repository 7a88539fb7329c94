// BAD description without any device allocation in the call.
//
// Some callers cannot call cudaMalloc: processes whose device memory is all
// reserved up front by another allocator (a framework's caching pool), so a
// fresh cudaMalloc fails or fragments what the pool holds; real-time loops
// that cannot take the device-wide synchronisation cudaFree implies; and
// plug-ins run inside a host program that forbids allocation once it is up.
// bd_bad_describe_noalloc serves them: the integral image and its tile
// carries live in one file-scope static device array, so the call launches
// the same two integral kernels and the same gather kernel as
// bd_bad_describe without allocating anything.
//
// Host code cannot use the array's name as a device address (it names a host
// stand-in), so the device address is looked up with cudaGetSymbolAddress,
// with the device current, once per device context (keyed by the driver's
// context id, so a context created after cudaDeviceReset gets a fresh lookup
// instead of a stale address), and cached.
#include <mutex>

#include "bd_internal.h"

namespace bd {
namespace {

// The integral image and carries of up to ~2.3 megapixels (1920x1088 fits).
constexpr size_t kStaticScratchBytes = BD_BAD_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_bad_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
    void *addr = nullptr;
    unsigned long long ctx_id = 0;  // driver id of the context the address belongs to
};
Cached g_scratch[kMaxDevices];

typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long *);

void *driver_fn(const char *name)
{
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return p;
}

// Id of the context current on this thread; 0 when there is none or the
// driver cannot say.
unsigned long long current_ctx_id()
{
    static PFN_ctxGetCurrent get_current = (PFN_ctxGetCurrent)driver_fn("cuCtxGetCurrent");
    static PFN_ctxGetId get_id = (PFN_ctxGetId)driver_fn("cuCtxGetId");
    if (!get_current || !get_id)
        return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

bd_status static_scratch(bd_ctx *ctx, int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices)
        return set_err(ctx, BD_ERR_UNSUPPORTED, "device index %d out of range", dev);
    Cached &c = g_scratch[dev];
    const unsigned long long id = current_ctx_id();
    if (!c.addr || id == 0 || id != c.ctx_id) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_bad_static_scratch);
        if (e != cudaSuccess || !ptr)
            return cuda_err(ctx, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                            "bd_bad_describe_noalloc: cudaGetSymbolAddress");
        c.addr = ptr;
        c.ctx_id = current_ctx_id();  // the lookup has made the device's context current
    }
    *out = c.addr;
    return BD_OK;
}

}  // namespace
}  // namespace bd

using namespace bd;

extern "C" bd_status bd_bad_describe_noalloc(const bd_bad_params *p, const uint8_t *img, int w,
                                             int h, int pitch, const bd_keypoint *kps, int n,
                                             uint32_t *out, void *stream)
{
    if (!p)
        return BD_ERR_INVALID;
    bd_ctx *ctx = p->ctx;
    if (!img || w < 1 || h < 1 || w > kMaxImageSide || h > kMaxImageSide || pitch < w || n < 0 ||
        (n > 0 && (!kps || !out)))
        return set_err(ctx, BD_ERR_INVALID, "bd_bad_describe_noalloc: bad arguments");
    const int stride = w + 1;
    const size_t ii_bytes = align_up((size_t)(h + 1) * stride * 4, 256);
    const size_t need = ii_bytes + integral_scratch_bytes(w, h);
    if (need > kStaticScratchBytes)
        return set_err(ctx, BD_ERR_INVALID,
                       "bd_bad_describe_noalloc: a %dx%d image needs %zu bytes of scratch, more "
                       "than the %zu-byte static area; use bd_bad_describe",
                       w, h, need, kStaticScratchBytes);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_bad_describe_noalloc: cudaGetDevice");
    if (dev != ctx->device)
        return set_err(ctx, BD_ERR_INVALID,
                       "bd_bad_describe_noalloc: current device %d is not the parameters' device %d",
                       dev, ctx->device);
    if (n == 0)
        return BD_OK;
    void *scratch = nullptr;
    bd_status s = static_scratch(ctx, dev, &scratch);
    if (s != BD_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *ii = (uint32_t *)scratch;
    e = launch_integral(img, w, h, pitch, ii, stride,
                        integral_scratch_carve((char *)scratch + ii_bytes, w, h), st);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_bad_describe_noalloc: integral kernels");
    e = launch_bad_gather(p, ii, stride, w, h, kps, n, out, nullptr, st);
    if (e != cudaSuccess)
        return cuda_err(ctx, e, "bd_bad_describe_noalloc: gather kernel");
    return BD_OK;
}
