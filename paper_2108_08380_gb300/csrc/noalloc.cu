// BAD description without any device allocation in the call.
//
// Some callers cannot call cudaMalloc: code that enqueues work while a CUDA
// stream capture in global mode is active (cudaMalloc is an error there),
// processes whose device memory is entirely owned by another allocator, and
// real-time loops that cannot take the implicit synchronisation of
// cudaMalloc / cudaFree.  bd_bad_describe_noalloc serves them: the integral
// image and its tile carries live in one file-scope static device array, so
// the call launches the same two integral kernels and the same gather kernel
// as bd_bad_describe without allocating anything.
//
// Host code cannot use the array's name as a device address (it names a host
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "bd_internal.h"

namespace bd {
namespace {

// The integral image and carries of up to ~2.3 megapixels (1920x1088 fits).
constexpr size_t kStaticScratchBytes = BD_BAD_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_bad_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

bd_status static_scratch(bd_ctx *ctx, int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices)
        return set_err(ctx, BD_ERR_UNSUPPORTED, "device index %d out of range", dev);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_bad_static_scratch);
        if (e != cudaSuccess || !ptr)
            return cuda_err(ctx, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                            "bd_bad_describe_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
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
