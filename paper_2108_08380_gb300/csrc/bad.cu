// BAD descriptor gather (Sec. III-A): one warp per keypoint.  Lane j owns
// bits j, j+32, ...; for each bit it reads the pair's rotated/scaled corner
// offsets from the (level, angle-bin) table, takes the two box sums from the
// integral image (4 lookups each, zero outside the image), applies the exact
// integer stump  sum1 - sum2 <= floor(num * s'^2 / den)  and the warp packs
// 32 stumps per __ballot_sync.
#include "bd_internal.h"

namespace bd {
namespace {

struct LevelMids {
    float v[kMaxLevels];
};

__device__ __forceinline__ uint32_t box_sum(const uint32_t *__restrict__ ii, int stride, int w,
                                            int h, int x0, int y0, int s)
{
    const int xa = min(max(x0, 0), w), xb = min(max(x0 + s, 0), w);
    const int ya = min(max(y0, 0), h), yb = min(max(y0 + s, 0), h);
    const uint32_t *ra = ii + (size_t)ya * stride;
    const uint32_t *rb = ii + (size_t)yb * stride;
    return __ldg(rb + xb) - __ldg(ra + xb) - __ldg(rb + xa) + __ldg(ra + xa);
}

template <int NW>
__global__ void __launch_bounds__(256, 2) bad_gather_kernel(
    const short4 *__restrict__ corner, const int2 *__restrict__ side_thr, int nbins, int nlevels,
    float angle_scale, LevelMids mids, const uint32_t *__restrict__ ii, int stride, int w, int h,
    const bd_keypoint *__restrict__ kps, int n, uint32_t *__restrict__ out, DeviceStatus *status)
{
    constexpr int K = NW * 32;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const bd_keypoint kp = kps[i];
        if (!dev::kp_valid(kp)) {
            if (lane < NW)
                out[(size_t)i * NW + lane] = 0u;
            if (lane == 0)
                dev::raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
            continue;
        }
        const int ix = dev::round_coord(kp.x);
        const int iy = dev::round_coord(kp.y);
        int l = 0;
#pragma unroll
        for (int q = 0; q + 1 < kMaxLevels; ++q)
            l += (q + 1 < nlevels && mids.v[q] < kp.scale) ? 1 : 0;
        int b = (int)floorf(__fadd_rn(__fmul_rn(kp.angle, angle_scale), 0.5f)) % nbins;
        if (b < 0)
            b += nbins;
        const short4 *tab = corner + ((size_t)l * nbins + b) * K;
        const int2 *st = side_thr + (size_t)l * K;
        uint32_t mine = 0;
        // all of a group's table reads first, then all its gathers: the warp keeps
        // 8 * 8 independent loads in flight instead of walking the bits in series
        constexpr int G = NW < 8 ? NW : 8;
#pragma unroll 1
        for (int j0 = 0; j0 < NW; j0 += G) {
            short4 c[G];
            int2 s[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                c[g] = __ldg(tab + (j0 + g) * 32 + lane);
                s[g] = __ldg(st + (j0 + g) * 32 + lane);
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t s1 = box_sum(ii, stride, w, h, ix + c[g].x, iy + c[g].y, s[g].x);
                const uint32_t s2 = box_sum(ii, stride, w, h, ix + c[g].z, iy + c[g].w, s[g].x);
                const bool bit = ((int)s1 - (int)s2) <= s[g].y;
                const uint32_t word = __ballot_sync(0xffffffffu, bit);
                if (lane == j0 + g)
                    mine = word;
            }
        }
        if (lane < NW)
            out[(size_t)i * NW + lane] = mine;
    }
}

}  // namespace

cudaError_t launch_bad_gather(const bd_bad_params *p, const uint32_t *ii, int ii_stride, int w,
                              int h, const bd_keypoint *kps, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st)
{
    LevelMids mids;
    for (int q = 0; q < kMaxLevels; ++q)
        mids.v[q] = p->level_mid[q];
    const int warps_per_block = 8;
    int blocks = (n + warps_per_block - 1) / warps_per_block;
    const int cap = 152 * 16;
    if (blocks > cap)
        blocks = cap;
    if (p->nbits == 256)
        bad_gather_kernel<8><<<blocks, 256, 0, st>>>(p->d_corner, p->d_side_thr, p->nbins,
                                                     p->nlevels, p->angle_scale, mids, ii,
                                                     ii_stride, w, h, kps, n, out, status);
    else
        bad_gather_kernel<16><<<blocks, 256, 0, st>>>(p->d_corner, p->d_side_thr, p->nbins,
                                                      p->nlevels, p->angle_scale, mids, ii,
                                                      ii_stride, w, h, kps, n, out, status);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
