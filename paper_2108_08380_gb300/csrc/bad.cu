// BAD descriptor gather over the keypoints of one image: one warp per
// keypoint (the per-keypoint routine is in bad_dev.cuh).
#include "bad_dev.cuh"

namespace bd {
namespace {

template <int NW>
__global__ void __launch_bounds__(256, 2) bad_gather_kernel(dev::BadTables T,
                                                            const uint32_t *__restrict__ ii,
                                                            int stride, int w, int h,
                                                            const bd_keypoint *__restrict__ kps,
                                                            int n, uint32_t *__restrict__ out,
                                                            DeviceStatus *status)
{
    __shared__ uint32_t sums[8][2 * NW * 32];  // the box sums of each warp's keypoint
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps)
        dev::bad_describe_warp<NW, true>(T, ii, stride, w, h, kps[i], out + (size_t)i * NW, status,
                                         sums[threadIdx.x >> 5]);
}

}  // namespace

cudaError_t launch_bad_gather(const bd_bad_params *p, const uint32_t *ii, int ii_stride, int w,
                              int h, const bd_keypoint *kps, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st)
{
    const int sm_count = p->ctx->sm_count > 0 ? p->ctx->sm_count : 1;
    const dev::BadTables T = dev::bad_tables(p);
    const int warps_per_block = 8;
    int blocks = (n + warps_per_block - 1) / warps_per_block;
    const int cap = sm_count * 16;  // 8 warps per CTA, two CTAs per SM: eight waves
    if (blocks > cap)
        blocks = cap;
    if (p->nbits == 256)
        bad_gather_kernel<8><<<blocks, 256, 0, st>>>(T, ii, ii_stride, w, h, kps, n, out, status);
    else
        bad_gather_kernel<16><<<blocks, 256, 0, st>>>(T, ii, ii_stride, w, h, kps, n, out, status);
    trace_kernel(st, "bad_gather");
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
