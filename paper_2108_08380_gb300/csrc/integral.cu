// Integral image (summed-area table) of an 8-bit image, Sec. III-A / IV-F:
// box means of BAD come from four lookups in it.
//
// Two launches over 32x128 tiles.  The first reduces every tile to its
// column sums, row sums and total; the second rebuilds each tile's outputs
// from its own pixels plus those small carries:
//   ii[y+1][x+1] = G(tile) + sum_{x' in tile, x' <= x} V(x')        (everything above the band)
//                + sum_{y' in band, y' <= y} (R(y') + rowprefix(y', x))
// with V(x) the column sums of all bands above, R(y) the row sums of all
// tiles to the left and G the total of the tiles above-left.  HBM traffic is
// two reads of the image and one write of the table (6 B per pixel).
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int TR = kIiTileRows;  // 32
constexpr int TC = kIiTileCols;  // 128

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(TC) ii_stats_kernel(const uint8_t *__restrict__ img, int w, int h,
                                                      int pitch, uint32_t *__restrict__ colsum,
                                                      uint32_t *__restrict__ rowsum,
                                                      uint32_t *__restrict__ tiletot, int ntx)
{
    __shared__ uint32_t tile[TR][TC + 1];
    __shared__ uint32_t wsum[TC / 32];
    const int tx = blockIdx.x, ty = blockIdx.y, t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;
    const int x = tx * TC + t, y0 = ty * TR;
    uint32_t cs = 0;
#pragma unroll 8
    for (int r = 0; r < TR; ++r) {
        const int y = y0 + r;
        const uint32_t v = (x < w && y < h) ? (uint32_t)__ldg(img + (size_t)y * pitch + x) : 0u;
        tile[r][t] = v;
        cs += v;
    }
    if (x < w)
        colsum[(size_t)ty * w + x] = cs;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TR / (TC / 32); ++q) {
        const int r = wp * (TR / (TC / 32)) + q;
        uint32_t s = tile[r][lane] + tile[r][lane + 32] + tile[r][lane + 64] + tile[r][lane + 96];
        s = warp_sum(s);
        if (lane == 0 && y0 + r < h)
            rowsum[(size_t)(y0 + r) * ntx + tx] = s;
    }
    cs = warp_sum(cs);
    if (lane == 0)
        wsum[wp] = cs;
    __syncthreads();
    if (t == 0)
        tiletot[(size_t)ty * ntx + tx] = wsum[0] + wsum[1] + wsum[2] + wsum[3];
}

__global__ void __launch_bounds__(TC) ii_final_kernel(const uint8_t *__restrict__ img, int w, int h,
                                                      int pitch,
                                                      const uint32_t *__restrict__ colsum,
                                                      const uint32_t *__restrict__ rowsum,
                                                      const uint32_t *__restrict__ tiletot,
                                                      int ntx, uint32_t *__restrict__ ii,
                                                      int stride)
{
    __shared__ uint32_t rowinc[TR][TC + 1];
    __shared__ uint32_t R[TR];
    __shared__ uint32_t wtot[TC / 32];
    __shared__ uint32_t gpart[TC / 32];
    const int tx = blockIdx.x, ty = blockIdx.y, t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;
    const int x = tx * TC + t, y0 = ty * TR;

    // column sums of all bands above this one
    uint32_t v = 0;
    if (x < w) {
#pragma unroll 8
        for (int a = 0; a < ty; ++a)
            v += __ldg(colsum + (size_t)a * w + x);
    }
    // total of the tiles above-left
    uint32_t g = 0;
    const int nab = ty * tx;
#pragma unroll 4
    for (int i = t; i < nab; i += TC)
        g += __ldg(tiletot + (size_t)(i / tx) * ntx + (i % tx));
    g = warp_sum(g);
    // inclusive scan of v across the tile's columns
    uint32_t vs = warp_incl_scan(v, lane);
    if (lane == 31)
        wtot[wp] = vs;
    if (lane == 0)
        gpart[wp] = g;
    // row sums of the tiles to the left
    if (wp == 0) {
        uint32_t r = 0;
        const int y = y0 + lane;
        if (y < h) {
#pragma unroll 8
            for (int a = 0; a < tx; ++a)
                r += __ldg(rowsum + (size_t)y * ntx + a);
        }
        R[lane] = r;
    }
    __syncthreads();
    for (int q = 0; q < wp; ++q)
        vs += wtot[q];
    uint32_t acc = gpart[0] + gpart[1] + gpart[2] + gpart[3] + vs;

    // per-row inclusive prefix inside the tile, plus the carry from the left
#pragma unroll 2
    for (int q = 0; q < TR / (TC / 32); ++q) {
        const int r = wp * (TR / (TC / 32)) + q;
        const int y = y0 + r;
        const int c0 = tx * TC + lane * 4;
        uint32_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        if (y < h) {
            const uint8_t *row = img + (size_t)y * pitch;
            p0 = c0 + 0 < w ? __ldg(row + c0 + 0) : 0u;
            p1 = c0 + 1 < w ? __ldg(row + c0 + 1) : 0u;
            p2 = c0 + 2 < w ? __ldg(row + c0 + 2) : 0u;
            p3 = c0 + 3 < w ? __ldg(row + c0 + 3) : 0u;
        }
        p1 += p0;
        p2 += p1;
        p3 += p2;
        const uint32_t incl = warp_incl_scan(p3, lane);
        const uint32_t base = incl - p3 + R[r];
        rowinc[r][lane * 4 + 0] = base + p0;
        rowinc[r][lane * 4 + 1] = base + p1;
        rowinc[r][lane * 4 + 2] = base + p2;
        rowinc[r][lane * 4 + 3] = base + p3;
    }
    __syncthreads();
    // running column sums down the band
    for (int r = 0; r < TR; ++r) {
        const int y = y0 + r;
        if (y >= h)
            break;
        acc += rowinc[r][t];
        if (x < w)
            ii[(size_t)(y + 1) * stride + x + 1] = acc;
    }
    // zero first row and first column
    if (ty == 0) {
        if (x < w)
            ii[x + 1] = 0;
        if (tx == 0 && t == 0)
            ii[0] = 0;
    }
    if (tx == 0 && t < TR && y0 + t < h)
        ii[(size_t)(y0 + t + 1) * stride] = 0;
}

}  // namespace

size_t integral_scratch_bytes(int w, int h)
{
    const size_t ntx = (w + TC - 1) / TC, nty = (h + TR - 1) / TR;
    return align_up(nty * w * 4, 256) + align_up((size_t)h * ntx * 4, 256) +
           align_up(nty * ntx * 4, 256);
}

IntegralScratch integral_scratch_carve(void *base, int w, int h)
{
    const size_t ntx = (w + TC - 1) / TC, nty = (h + TR - 1) / TR;
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
    const int ntx = (w + TC - 1) / TC, nty = (h + TR - 1) / TR;
    dim3 grid(ntx, nty);
    ii_stats_kernel<<<grid, TC, 0, st>>>(img, w, h, pitch, s.colsum, s.rowsum, s.tiletot, ntx);
    ii_final_kernel<<<grid, TC, 0, st>>>(img, w, h, pitch, s.colsum, s.rowsum, s.tiletot, ntx, ii,
                                         ii_stride);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace bd
