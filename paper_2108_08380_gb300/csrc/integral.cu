// Integral image of one image: two launches over 32x128 tiles (tile routines
// and the carry scheme are in integral_dev.cuh).
#include "integral_dev.cuh"

namespace bd {
namespace {

__global__ void __launch_bounds__(dev::IITC) ii_stats_kernel(const uint8_t *__restrict__ img, int w,
                                                             int h, int pitch, uint32_t *colsum,
                                                             uint32_t *rowsum, uint32_t *tiletot,
                                                             int ntx)
{
    __shared__ dev::IiStatsSmem S;
    dev::ii_stats_tile(S, img, w, h, pitch, colsum, rowsum, tiletot, ntx, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(dev::IITC) ii_final_kernel(const uint8_t *__restrict__ img, int w,
                                                             int h, int pitch,
                                                             const uint32_t *colsum,
                                                             const uint32_t *rowsum,
                                                             const uint32_t *tiletot, int ntx,
                                                             uint32_t *ii, int stride)
{
    __shared__ dev::IiFinalSmem S;
    dev::ii_final_tile(S, img, w, h, pitch, colsum, rowsum, tiletot, ntx, ii, stride, blockIdx.x,
                       blockIdx.y);
}

}  // namespace

size_t integral_scratch_bytes(int w, int h)
{
    const size_t ntx = (w + dev::IITC - 1) / dev::IITC, nty = (h + dev::IITR - 1) / dev::IITR;
    return align_up(nty * w * 4, 256) + align_up((size_t)h * ntx * 4, 256) +
           align_up(nty * ntx * 4, 256);
}

IntegralScratch integral_scratch_carve(void *base, int w, int h)
{
    const size_t ntx = (w + dev::IITC - 1) / dev::IITC, nty = (h + dev::IITR - 1) / dev::IITR;
    char *p = (char *)base;
    IntegralScratch s;
    s.colsum = (uint32_t *)p;
    p += align_up(nty * w * 4, 256);
    s.rowsum = (uint32_t *)p;
    p += align_up((size_t)h * ntx * 4, 256);
    s.tiletot = (uint32_t *)p;
    return s;
}

cudaError_t launch_integral(const uint8_t *img, int w, int h, int pitch, uint32_t *ii,
                            int ii_stride, const IntegralScratch &s, cudaStream_t st)
{
    const int ntx = (w + dev::IITC - 1) / dev::IITC, nty = (h + dev::IITR - 1) / dev::IITR;
    dim3 grid(ntx, nty);
    ii_stats_kernel<<<grid, dev::IITC, 0, st>>>(img, w, h, pitch, s.colsum, s.rowsum, s.tiletot, ntx);
    trace_kernel(st, "ii_stats");
    ii_final_kernel<<<grid, dev::IITC, 0, st>>>(img, w, h, pitch, s.colsum, s.rowsum, s.tiletot,
                                                ntx, ii, ii_stride);
    trace_kernel(st, "ii_final");
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace bd
