// Tile routines of the integral image (summed-area table), Sec. III-A / IV-F:
// box means of BAD come from four lookups in it.  Shared by the per-image
// kernels (integral.cu) and the batched persistent kernel (batch.cu).
//
// The image is cut into 32x128 tiles.  Two passes (the per-image kernels):
// pass 1 reduces each tile to its column
// sums, row sums and total.  Pass 2 rebuilds the tile's table entries from its
// own pixels plus those carries:
//   ii[y+1][x+1] = G + sum_{tile columns x' <= x} V(x')
//                + sum_{band rows y' <= y} (R(y') + rowprefix(y', x))
// with V(x) the column sums of all bands above, R(y) the row sums of all
// tiles to the left and G the total of the tiles above-left.  HBM traffic is
// two reads of the image and one write of the table (6 B per pixel).
// Carries are read with ld.global.cg: in the persistent kernel they were
// written by other CTAs of the same launch.
#pragma once

#include "bd_internal.h"

namespace bd {
namespace dev {

constexpr int IITR = kIiTileRows;  // 32
constexpr int IITC = kIiTileCols;  // 128, = threads per CTA

struct IiStatsSmem {
    uint32_t tile[IITR][IITC + 1];
    uint32_t wsum[IITC / 32];
};

struct IiFinalSmem {
    uint32_t rowinc[IITR][IITC + 1];
    uint32_t R[IITR];
    uint32_t wtot[IITC / 32];
    uint32_t gpart[IITC / 32];
};

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1 for tile (tx, ty); called by all 128 threads of the CTA.
__device__ __forceinline__ void ii_stats_tile(IiStatsSmem &S, const uint8_t *__restrict__ img,
                                              int w, int h, int pitch, uint32_t *colsum,
                                              uint32_t *rowsum, uint32_t *tiletot, int ntx, int tx,
                                              int ty)
{
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int x = tx * IITC + t, y0 = ty * IITR;
    // all 32 loads in flight at once: one memory round trip per tile
    uint32_t px[IITR];
#pragma unroll
    for (int r = 0; r < IITR; ++r) {
        const int y = y0 + r;
        px[r] = (x < w && y < h) ? (uint32_t)__ldg(img + (size_t)y * pitch + x) : 0u;
    }
    uint32_t cs = 0;
#pragma unroll
    for (int r = 0; r < IITR; ++r) {
        S.tile[r][t] = px[r];
        cs += px[r];
    }
    if (x < w)
        colsum[(size_t)ty * w + x] = cs;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < IITR / (IITC / 32); ++q) {
        const int r = wp * (IITR / (IITC / 32)) + q;
        uint32_t s = S.tile[r][lane] + S.tile[r][lane + 32] + S.tile[r][lane + 64] + S.tile[r][lane + 96];
        s = warp_sum_u32(s);
        if (lane == 0 && y0 + r < h)
            rowsum[(size_t)(y0 + r) * ntx + tx] = s;
    }
    cs = warp_sum_u32(cs);
    if (lane == 0)
        S.wsum[wp] = cs;
    __syncthreads();
    if (t == 0)
        tiletot[(size_t)ty * ntx + tx] = S.wsum[0] + S.wsum[1] + S.wsum[2] + S.wsum[3];
}

// Pass 2 for tile (tx, ty); called by all 128 threads of the CTA.
__device__ __forceinline__ void ii_final_tile(IiFinalSmem &S, const uint8_t *__restrict__ img,
                                              int w, int h, int pitch, const uint32_t *colsum,
                                              const uint32_t *rowsum, const uint32_t *tiletot,
                                              int ntx, uint32_t *ii, int stride, int tx, int ty)
{
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int x = tx * IITC + t, y0 = ty * IITR;

    constexpr int RPW = IITR / (IITC / 32);  // rows rebuilt per warp (8)
    // this warp's rows first (4 bytes per lane each, one word load when
    // aligned): they do not depend on the carries, so their round trip
    // overlaps the carry reads below
    uint32_t px[RPW];
    {
        const int c0 = tx * IITC + lane * 4;
        const bool words = ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 3) == 0 && c0 + 3 < w;
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int y = y0 + wp * RPW + q;
            uint32_t v = 0u;
            if (y < h) {
                const uint8_t *row = img + (size_t)y * pitch + c0;
                if (words) {
                    v = __ldg(reinterpret_cast<const uint32_t *>(row));
                } else {
                    const uint32_t b0 = c0 + 0 < w ? __ldg(row + 0) : 0u;
                    const uint32_t b1 = c0 + 1 < w ? __ldg(row + 1) : 0u;
                    const uint32_t b2 = c0 + 2 < w ? __ldg(row + 2) : 0u;
                    const uint32_t b3 = c0 + 3 < w ? __ldg(row + 3) : 0u;
                    v = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
                }
            }
            px[q] = v;
        }
    }

    // column sums of all bands above this one
    uint32_t v = 0;
    if (x < w) {
#pragma unroll 16
        for (int a = 0; a < ty; ++a)
            v += __ldcg(colsum + (size_t)a * w + x);
    }
    // total of the tiles above-left
    uint32_t g = 0;
    const int nab = ty * tx;
#pragma unroll 4
    for (int i = t; i < nab; i += IITC)
        g += __ldcg(tiletot + (size_t)(i / tx) * ntx + (i % tx));
    g = warp_sum_u32(g);
    // row sums of the tiles to the left
    uint32_t rl = 0;
    if (wp == 0) {
        const int y = y0 + lane;
        if (y < h) {
#pragma unroll 8
            for (int a = 0; a < tx; ++a)
                rl += __ldcg(rowsum + (size_t)y * ntx + a);
        }
    }
    // inclusive scan of v across the tile's columns
    uint32_t vs = warp_incl_scan_u32(v, lane);
    if (lane == 31)
        S.wtot[wp] = vs;
    if (lane == 0)
        S.gpart[wp] = g;
    if (wp == 0)
        S.R[lane] = rl;
    __syncthreads();
    for (int q = 0; q < wp; ++q)
        vs += S.wtot[q];
    uint32_t acc = S.gpart[0] + S.gpart[1] + S.gpart[2] + S.gpart[3] + vs;

    // per-row inclusive prefix inside the tile, plus the carry from the left
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        const int r = wp * RPW + q;
        const uint32_t p0 = px[q] & 0xFFu;
        const uint32_t p1 = p0 + ((px[q] >> 8) & 0xFFu);
        const uint32_t p2 = p1 + ((px[q] >> 16) & 0xFFu);
        const uint32_t p3 = p2 + (px[q] >> 24);
        const uint32_t incl = warp_incl_scan_u32(p3, lane);
        const uint32_t base = incl - p3 + S.R[r];
        S.rowinc[r][lane * 4 + 0] = base + p0;
        S.rowinc[r][lane * 4 + 1] = base + p1;
        S.rowinc[r][lane * 4 + 2] = base + p2;
        S.rowinc[r][lane * 4 + 3] = base + p3;
    }
    __syncthreads();
    // running column sums down the band
    for (int r = 0; r < IITR; ++r) {
        const int y = y0 + r;
        if (y >= h)
            break;
        acc += S.rowinc[r][t];
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
    if (tx == 0 && t < IITR && y0 + t < h)
        ii[(size_t)(y0 + t + 1) * stride] = 0;
}

// ---------------------------------------------------------------------------
// Single pass (the batched persistent kernel): a tile computes the same
// aggregates as pass 1 from pixels it keeps on chip, publishes them, waits
// only for the tiles it needs (those to its left in its band and every tile
// of the bands above, all earlier in the work queue, which publish before
// they wait), then adds the carries exactly as pass 2 does.  The image is
// read once: 1 B read + 4 B written per pixel, plus the aggregates.

struct IiOneSmem {
    uint32_t rowinc[IITR][IITC + 1];  // in-tile row prefix (no carry from the left)
    uint32_t colpart[IITC / 32][IITC];  // column sums over each warp's 8 rows
    uint32_t rowtot[IITR];
    uint32_t R[IITR];
    uint32_t wtot[IITC / 32];
    uint32_t gpart[IITC / 32];
};

// Local part of tile (tx, ty): loads its pixels, keeps the in-tile row
// prefixes in shared memory and writes its column sums, row sums and total.
// Called by all 128 threads; ends with a barrier.
__device__ __forceinline__ void ii_one_local(IiOneSmem &S, const uint8_t *__restrict__ img, int w,
                                             int h, int pitch, uint32_t *colsum, uint32_t *rowsum,
                                             uint32_t *tiletot, int ntx, int tx, int ty)
{
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int y0 = ty * IITR;
    constexpr int RPW = IITR / (IITC / 32);  // rows per warp (8)
    uint32_t px[RPW];
    {
        const int c0 = tx * IITC + lane * 4;
        const bool words = ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 3) == 0 && c0 + 3 < w;
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int y = y0 + wp * RPW + q;
            uint32_t v = 0u;
            if (y < h) {
                const uint8_t *row = img + (size_t)y * pitch + c0;
                if (words) {
                    v = __ldg(reinterpret_cast<const uint32_t *>(row));
                } else {
                    const uint32_t b0 = c0 + 0 < w ? __ldg(row + 0) : 0u;
                    const uint32_t b1 = c0 + 1 < w ? __ldg(row + 1) : 0u;
                    const uint32_t b2 = c0 + 2 < w ? __ldg(row + 2) : 0u;
                    const uint32_t b3 = c0 + 3 < w ? __ldg(row + 3) : 0u;
                    v = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
                }
            }
            px[q] = v;
        }
    }
    uint32_t cp0 = 0, cp1 = 0, cp2 = 0, cp3 = 0;
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        const int r = wp * RPW + q;
        const uint32_t b0 = px[q] & 0xFFu, b1 = (px[q] >> 8) & 0xFFu;
        const uint32_t b2 = (px[q] >> 16) & 0xFFu, b3 = px[q] >> 24;
        cp0 += b0;
        cp1 += b1;
        cp2 += b2;
        cp3 += b3;
        const uint32_t p1 = b0 + b1, p2 = p1 + b2, p3 = p2 + b3;
        const uint32_t incl = warp_incl_scan_u32(p3, lane);
        const uint32_t base = incl - p3;
        S.rowinc[r][lane * 4 + 0] = base + b0;
        S.rowinc[r][lane * 4 + 1] = base + p1;
        S.rowinc[r][lane * 4 + 2] = base + p2;
        S.rowinc[r][lane * 4 + 3] = base + p3;
        if (lane == 31)
            S.rowtot[r] = incl;
    }
    S.colpart[wp][lane * 4 + 0] = cp0;
    S.colpart[wp][lane * 4 + 1] = cp1;
    S.colpart[wp][lane * 4 + 2] = cp2;
    S.colpart[wp][lane * 4 + 3] = cp3;
    __syncthreads();
    const int x = tx * IITC + t;
    if (x < w)
        colsum[(size_t)ty * w + x] = S.colpart[0][t] + S.colpart[1][t] + S.colpart[2][t] + S.colpart[3][t];
    if (t < IITR && y0 + t < h)
        rowsum[(size_t)(y0 + t) * ntx + tx] = S.rowtot[t];
    if (wp == 0) {
        const uint32_t tot = warp_sum_u32(S.rowtot[lane]);
        if (lane == 0)
            tiletot[(size_t)ty * ntx + tx] = tot;
    }
    __syncthreads();
}

// Carries of tile (tx, ty) from the aggregates of the tiles above and to the
// left (read through L2: other CTAs of the launch wrote them), then the
// table entries of the tile.  Called by all 128 threads after ii_one_local.
__device__ __forceinline__ void ii_one_finish(IiOneSmem &S, int w, int h, const uint32_t *colsum,
                                              const uint32_t *rowsum, const uint32_t *tiletot,
                                              int ntx, uint32_t *ii, int stride, int tx, int ty)
{
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    const int x = tx * IITC + t, y0 = ty * IITR;
    uint32_t v = 0;
    if (x < w) {
#pragma unroll 16
        for (int a = 0; a < ty; ++a)
            v += __ldcg(colsum + (size_t)a * w + x);
    }
    uint32_t g = 0;
    const int nab = ty * tx;
#pragma unroll 4
    for (int i = t; i < nab; i += IITC)
        g += __ldcg(tiletot + (size_t)(i / tx) * ntx + (i % tx));
    g = warp_sum_u32(g);
    uint32_t rl = 0;
    if (wp == 0) {
        const int y = y0 + lane;
        if (y < h) {
#pragma unroll 8
            for (int a = 0; a < tx; ++a)
                rl += __ldcg(rowsum + (size_t)y * ntx + a);
        }
    }
    uint32_t vs = warp_incl_scan_u32(v, lane);
    if (lane == 31)
        S.wtot[wp] = vs;
    if (lane == 0)
        S.gpart[wp] = g;
    if (wp == 0)
        S.R[lane] = rl;
    __syncthreads();
    for (int q = 0; q < wp; ++q)
        vs += S.wtot[q];
    uint32_t acc = S.gpart[0] + S.gpart[1] + S.gpart[2] + S.gpart[3] + vs;
    for (int r = 0; r < IITR; ++r) {
        const int y = y0 + r;
        if (y >= h)
            break;
        acc += S.rowinc[r][t] + S.R[r];
        if (x < w)
            ii[(size_t)(y + 1) * stride + x + 1] = acc;
    }
    if (ty == 0) {
        if (x < w)
            ii[x + 1] = 0;
        if (tx == 0 && t == 0)
            ii[0] = 0;
    }
    if (tx == 0 && t < IITR && y0 + t < h)
        ii[(size_t)(y0 + t + 1) * stride] = 0;
}

}  // namespace dev
}  // namespace bd
