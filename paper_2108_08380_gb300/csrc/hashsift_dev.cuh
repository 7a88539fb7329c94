// HashSIFT per-keypoint routines (Sec. III-B), FP32 on CUDA cores; shared by
// the per-image kernels (hashsift.cu), the batched persistent kernel and the
// training step.
//
//  - the 32x32 patch, sampled bilinearly around the keypoint (Sec. IV-F:
//    HashSIFT describes a normalised 32x32 patch, not an image pyramid);
//  - the SIFT-style histogram: central-difference gradients, 8 orientation
//    bins with linear voting between neighbours, 4x4 cells of 8x8 pixels, a
//    sigma = 16 Gaussian weight about the patch centre, L2 normalisation.
//
// One warp describes one keypoint (hs_hist_warp), in three phases:
//  1. sample the 1024 patch pixels in 4x8 blocks (one block per warp-wide
//     load: a compact block of a rotated patch touches a few image rows,
//     where a 32-pixel patch row can touch one row per pixel) into the
//     warp's patch buffer in shared memory, rows padded to 40 floats so both
//     the block writes and the row reads are conflict-free;
//  2. lane j walks down patch column j with the vertical neighbours in
//     registers and the horizontal ones from the neighbouring lanes, voting
//     into a lane-private histogram of the four cells its column crosses,
//     laid out [cell row][bin][lane] (conflict-free, no atomics);
//  3. each lane sums four of the 128 (cell, bin) entries over the cell's 8
//     columns and the warp normalises them.
// There is no CTA-wide barrier: the warps of a CTA run independent keypoints.
#pragma once

#include "bd_internal.h"

namespace bd {
namespace dev {

constexpr int HS_NT = 128;       // threads per keypoint
constexpr int PS = kPatch;       // 32
constexpr int PSP = kPatch + 1;  // padded smem row
constexpr int NT = HS_NT;

struct Frame {
    int ix, iy;
    float fx, fy, A, B;  // A = scale*spacing*cos(angle), B = scale*spacing*sin(angle)
};

__device__ __forceinline__ Frame make_frame(const bd_keypoint &kp, float spacing)
{
    Frame f;
    f.ix = round_coord(kp.x);
    f.iy = round_coord(kp.y);
    f.fx = kp.x - (float)f.ix;  // exact: both operands are within a factor of 2
    f.fy = kp.y - (float)f.iy;
    float s, c;
    sincosf(kp.angle, &s, &c);
    const float sg = kp.scale * spacing;
    f.A = sg * c;
    f.B = sg * s;
    return f;
}

// Bilinear sample (clamp-to-edge taps) of patch pixel (i, j): the offset from
// the rounded keypoint is kept small so FP32 keeps ~1e-6 px of precision.
__device__ __forceinline__ float sample(const uint8_t *__restrict__ img, int w, int h, int pitch,
                                        const Frame &f, int i, int j)
{
    const float u = (float)j - 15.5f, v = (float)i - 15.5f;
    const float ox = fmaf(f.A, u, fmaf(-f.B, v, f.fx));
    const float oy = fmaf(f.B, u, fmaf(f.A, v, f.fy));
    const float flx = floorf(ox), fly = floorf(oy);
    float ax = ox - flx, ay = oy - fly;
    int x0 = f.ix + (int)flx, y0 = f.iy + (int)fly;
    float i00, i01, i10, i11;
    if (w >= 2 && h >= 2) {
        // Clamp-to-edge without clamping each tap: a sample left of / above the
        // image reads column / row 0 with weight 0 on the next one, a sample at
        // or beyond the last column / row reads it with weight 1.
        if (x0 < 0) {
            x0 = 0;
            ax = 0.0f;
        } else if (x0 > w - 2) {
            x0 = w - 2;
            ax = 1.0f;
        }
        if (y0 < 0) {
            y0 = 0;
            ay = 0.0f;
        } else if (y0 > h - 2) {
            y0 = h - 2;
            ay = 1.0f;
        }
        const uint8_t *p = img + (size_t)y0 * pitch + x0;
        i00 = (float)__ldg(p);
        i01 = (float)__ldg(p + 1);
        i10 = (float)__ldg(p + pitch);
        i11 = (float)__ldg(p + pitch + 1);
    } else {
        const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
        const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
        const uint8_t *ra = img + (size_t)ya * pitch;
        const uint8_t *rb = img + (size_t)yb * pitch;
        i00 = (float)__ldg(ra + xa);
        i01 = (float)__ldg(ra + xb);
        i10 = (float)__ldg(rb + xa);
        i11 = (float)__ldg(rb + xb);
    }
    const float top = fmaf(ax, i01 - i00, i00);
    const float bot = fmaf(ax, i11 - i10, i10);
    return fmaf(ay, bot - top, top);
}

// Orientation bin pair of the gradient (gx, gy) != (0, 0).  The angle
// atan2(gy, gx) wrapped to [0, 2 pi) is q pi/4; the vote goes to bin floor(q)
// with weight 1 - frac(q) and to the next bin with frac(q) = w1.  The
// first-octant angle u = (4/pi) atan(r), r = min/max of |gx|, |gy| in [0, 1],
// comes from an odd degree-15 polynomial r * P(r^2) whose coefficients are a
// least-squares fit of (4/pi) atan(r) on Chebyshev nodes of [0, 1]; its
// largest error on a 2-million-point grid of [0, 1) is 1.0e-7 evaluated in
// double precision and 2.1e-7 evaluated as below in FP32 (a CPU test parses
// the coefficients from this file and checks both bounds).  u is exact at
// r = 0 and set to exactly 1 at r = 1, so exact multiples of 45 degrees fall
// on exact bin edges.  The octant o (0..7) follows from the signs and the
// |gy| > |gx| test: q = o + u in even octants and o + 1 - u in odd ones, so
// the bin is o and w1 is u or 1 - u, with no rounding of q itself.
__device__ __forceinline__ int orient_bin(float gx, float gy, float &w1)
{
    const float ax = fabsf(gx), ay = fabsf(gy);
    const float mn = fminf(ax, ay), mx = fmaxf(ax, ay);
    const float r = __fdividef(mn, mx);
    const float z = r * r;
    float p = -0.005162368528544903f;
    p = fmaf(p, z, 0.027836523950099945f);
    p = fmaf(p, z, -0.07118938118219376f);
    p = fmaf(p, z, 0.12276794016361237f);
    p = fmaf(p, z, -0.17709001898765564f);
    p = fmaf(p, z, 0.2539675235748291f);
    p = fmaf(p, z, -0.4243689775466919f);
    p = fmaf(p, z, 1.2732386589050293f);
    const float u = mn == mx ? 1.0f : p * r;
    // quadrant k = 2 sy + (sx ^ sy) starts at octant 2k; within it the
    // second octant is the one nearer the next axis (sw flipped in odd k)
    const int sx = gx < 0.0f, sy = gy < 0.0f, sw = ay > ax;
    const int t = sx ^ sy;
    const int odd = t ^ sw;
    w1 = odd ? 1.0f - u : u;
    return 4 * sy + 2 * t + odd;
}

// Per-thread constants of the 128-thread histogram layout used by the
// training backward (thread t: cell t/8, pixel row t%8 of it): pixel row i,
// first column j0 and the separable Gaussian weights gi * gj[q] (sigma = 16).
struct HistLane {
    int i, j0;
    float g[8];
};

__device__ __forceinline__ HistLane hist_lane(int t)
{
    HistLane L;
    const int cell = t >> 3;
    L.i = (cell >> 2) * 8 + (t & 7);
    L.j0 = (cell & 3) * 8;
    // separable weight exp(-(di^2 + dj^2) / 512); __expf's relative error
    // (~2^-21) is far below the histogram tolerance
    const float di = (float)L.i - 15.5f;
    const float gi = __expf(-di * di * (1.0f / 512.0f));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float dj = (float)(L.j0 + q) - 15.5f;
        L.g[q] = gi * __expf(-dj * dj * (1.0f / 512.0f));
    }
    return L;
}

// ---------------------------------------------------------------------------
// warp per keypoint

constexpr unsigned kFull = 0xffffffffu;

// Splits x (|x| < 2^21) into x = i + f exactly, with i an integer and f in
// [0, 1]: i = floor(x), or floor(x) - 1 with f = 1 when x is an integer.
// Adding 1.5 * 2^23 rounds to an integer in the mantissa, so this takes FP32
// adds and one integer subtract instead of conversion instructions.  Either
// split gives the same bilinear value and the same orientation votes.
__device__ __forceinline__ int split_floor(float x, float &f)
{
    const float M = 12582912.0f;  // 1.5 * 2^23, bit pattern 0x4B400000
    const float t = __fadd_rn(__fadd_rn(x, -0.5f), M);
    f = __fadd_rn(x, -__fadd_rn(t, -M));
    return __float_as_int(t) - 0x4B400000;
}

// uint8 value as FP32 through the mantissa (exact for b < 2^23).
__device__ __forceinline__ float u8f(uint32_t b)
{
    return __uint_as_float(0x4B000000u | b) - 8388608.0f;
}

// Bilinear sampler of patch column j of a keypoint: pixel (i, j) samples
// (x, y) + scale * spacing * R(angle) (j - 15.5, i - 15.5), clamp to edge.
// The offset from the rounded keypoint is kept small so FP32 keeps ~1e-6 px.
// Interior = true (decided once per keypoint, see col_interior) reads the
// four taps without clamping: the whole footprint lies inside the image.
struct ColFrame {
    const uint8_t *img;
    int w, h, pitch, ix, iy;
    float A, B, cx, cy;
};

__device__ __forceinline__ ColFrame col_frame(const uint8_t *img, int w, int h, int pitch,
                                              const Frame &f, int j = 0)
{
    ColFrame c;
    c.img = img;
    c.w = w;
    c.h = h;
    c.pitch = pitch;
    c.ix = f.ix;
    c.iy = f.iy;
    c.A = f.A;
    c.B = f.B;
    c.cx = f.fx;
    c.cy = f.fy;
    (void)j;
    return c;
}

// True when every tap of the patch is inside the image with a margin:
// |offset| <= 15.5 (|A| + |B|) + 0.5, taps reach one pixel beyond, and
// split_floor may step one more to the left / top.
__device__ __forceinline__ bool col_interior(const Frame &f, int w, int h)
{
    const float reach = 15.5f * (fabsf(f.A) + fabsf(f.B));
    if (!(reach < 1.0e6f) || w < 2 || h < 2)
        return false;
    const int m = (int)reach + 5;
    return f.ix - m >= 0 && f.ix + m < w && f.iy - m >= 0 && f.iy + m < h;
}

template <bool Interior>
struct ColSampler {
    ColFrame c;

    __device__ __forceinline__ float at(int i, int j) const
    {
        const float u = (float)j - 15.5f, v = (float)i - 15.5f;
        float ox = fmaf(c.A, u, fmaf(-c.B, v, c.cx));
        float oy = fmaf(c.B, u, fmaf(c.A, v, c.cy));
        if (!Interior) {  // keep split_floor in range; the taps clamp to the edge anyway
            ox = fminf(fmaxf(ox, -1048576.0f), 1048576.0f);
            oy = fminf(fmaxf(oy, -1048576.0f), 1048576.0f);
        }
        float ax, ay;
        int x0 = split_floor(ox, ax) + c.ix;
        int y0 = split_floor(oy, ay) + c.iy;
        float i00, i01, i10, i11;
        if (Interior) {
            const uint8_t *p = c.img + (size_t)y0 * c.pitch + x0;
            i00 = u8f(__ldg(p));
            i01 = u8f(__ldg(p + 1));
            i10 = u8f(__ldg(p + c.pitch));
            i11 = u8f(__ldg(p + c.pitch + 1));
        } else if (c.w >= 2 && c.h >= 2) {
            // a sample left of / above the image reads column / row 0 with
            // weight 0 on the next one; at or beyond the last column / row it
            // reads that one with weight 1
            if (x0 < 0) {
                x0 = 0;
                ax = 0.0f;
            } else if (x0 > c.w - 2) {
                x0 = c.w - 2;
                ax = 1.0f;
            }
            if (y0 < 0) {
                y0 = 0;
                ay = 0.0f;
            } else if (y0 > c.h - 2) {
                y0 = c.h - 2;
                ay = 1.0f;
            }
            const uint8_t *p = c.img + (size_t)y0 * c.pitch + x0;
            i00 = u8f(__ldg(p));
            i01 = u8f(__ldg(p + 1));
            i10 = u8f(__ldg(p + c.pitch));
            i11 = u8f(__ldg(p + c.pitch + 1));
        } else {
            const int xa = min(max(x0, 0), c.w - 1), xb = min(max(x0 + 1, 0), c.w - 1);
            const int ya = min(max(y0, 0), c.h - 1), yb = min(max(y0 + 1, 0), c.h - 1);
            const uint8_t *ra = c.img + (size_t)ya * c.pitch;
            const uint8_t *rb = c.img + (size_t)yb * c.pitch;
            i00 = u8f(__ldg(ra + xa));
            i01 = u8f(__ldg(ra + xb));
            i10 = u8f(__ldg(rb + xa));
            i11 = u8f(__ldg(rb + xb));
        }
        const float top = fmaf(ax, i01 - i00, i00);
        const float bot = fmaf(ax, i11 - i10, i10);
        return fmaf(ay, bot - top, top);
    }
};

// A patch already in memory ([32][32] FP32, row-major).
struct PatchMem {
    const float *p;
    __device__ __forceinline__ float at(int i, int j) const { return __ldg(p + i * PS + j); }
};

constexpr int kPRow = 40;  // padded patch row: bank (8 i + j) % 32 is distinct per block and per row

struct WarpHist {
    union {
        float P[PS][kPRow];               // patch samples [row][column]
        uint32_t win[PS * kPRow];         // or the keypoint's image footprint (bytes)
    };
    float priv[4][8][32];  // [cell row][bin][lane]
    float wss[4];          // per-warp sums of squares (cooperative mode)
};
constexpr int kWinBytes = PS * kPRow * 4;

// Image footprint of a keypoint staged in shared memory: image rows
// [y0, y0 + nr), bytes [x0, x0 + 4 wpr) of each (x0 word-aligned), row
// stride S bytes with S / 4 odd so that rows fall on different banks.
struct WinGeom {
    int x0, y0, nr, wpr, S;
};

// Footprint of the keypoint's 32x32 samples (every bilinear tap, with the
// split_floor step) when it lies inside the image, fits kWinBytes and the
// image rows are word-aligned; false otherwise (the sampler reads global
// memory then).
__device__ __forceinline__ bool win_geom(const Frame &f, const uint8_t *img, int w, int h,
                                         int pitch, WinGeom &g)
{
    if ((reinterpret_cast<uintptr_t>(img) & 3) || (pitch & 3))
        return false;
    const float reach = 15.5f * (fabsf(f.A) + fabsf(f.B));  // |sample offset| <= reach + 0.5
    if (!(reach < 60.0f))
        return false;
    const int m = (int)reach + 3;  // taps reach one pixel beyond; split_floor may step one back
    const int x0 = (f.ix - m) & ~3, x1 = f.ix + m + 2;
    const int y0 = f.iy - m, y1 = f.iy + m + 2;
    if (f.ix - m < 0 || y0 < 0 || y1 > h)
        return false;
    const int wpr = (x1 - x0 + 3) >> 2;
    if (wpr > 32 || x0 + 4 * wpr > w)
        return false;
    const int S = 4 * (wpr | 1);
    if ((y1 - y0) * S > kWinBytes)
        return false;
    g.x0 = x0;
    g.y0 = y0;
    g.nr = y1 - y0;
    g.wpr = wpr;
    g.S = S;
    return true;
}

// Copies the footprint into the window with word loads, threads t0 .. t0 +
// nthr - 1 of the caller's group (32: one warp; 128: the CTA); rows are
// spread over the group in blocks of the next power of two >= wpr words.
__device__ __forceinline__ void win_stage(uint32_t *win, const WinGeom &g, const uint8_t *img,
                                          int pitch, int tid, int nthr)
{
    const int wp2 = g.wpr <= 8 ? 8 : (g.wpr <= 16 ? 16 : 32);
    const int rpi = nthr / wp2;  // rows per pass
    const int rr = tid / wp2, c = tid % wp2;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(img + (size_t)g.y0 * pitch + g.x0);
    const int pw = pitch >> 2, sw = g.S >> 2;
    if (c < g.wpr)
        for (int r = rr; r < g.nr; r += rpi)
            win[r * sw + c] = __ldg(src + (size_t)r * pw + c);
}

// Bilinear sample (i, j) of the patch from the staged footprint, with the
// same arithmetic as ColSampler (identical values).
__device__ __forceinline__ float win_sample(const uint8_t *win, const WinGeom &g,
                                            const ColFrame &c, int i, int j)
{
    const float u = (float)j - 15.5f, v = (float)i - 15.5f;
    const float ox = fmaf(c.A, u, fmaf(-c.B, v, c.cx));
    const float oy = fmaf(c.B, u, fmaf(c.A, v, c.cy));
    float ax, ay;
    const int x0 = split_floor(ox, ax) + c.ix - g.x0;
    const int y0 = split_floor(oy, ay) + c.iy - g.y0;
    const uint8_t *p = win + y0 * g.S + x0;
    const float i00 = u8f(p[0]), i01 = u8f(p[1]);
    const float i10 = u8f(p[g.S]), i11 = u8f(p[g.S + 1]);
    const float top = fmaf(ax, i01 - i00, i00);
    const float bot = fmaf(ax, i11 - i10, i10);
    return fmaf(ay, bot - top, top);
}

// Gaussian weight exp(-(d^2) / 512) of row / column index i (sigma = 16 about
// 15.5); __expf's relative error (~2^-21) is far below the histogram tolerance.
__device__ __forceinline__ float gauss16(int i)
{
    const float d = (float)i - 15.5f;
    return __expf(-d * d * (1.0f / 512.0f));
}

// Votes of pixel (i, lane) with vertical neighbours up / down and the row's
// value here.  gx, gy are twice the central differences, so the weight is
// halved (exact).  Lanes 0 and 31 get their own value from the shuffles,
// which is the replicated edge.  A zero gradient votes zero (no branch).
__device__ __forceinline__ void vote_px(WarpHist &S, int lane, int i, float up, float here,
                                        float down, float g_half)
{
    const float left = __shfl_up_sync(kFull, here, 1);
    const float right = __shfl_down_sync(kFull, here, 1);
    const float gx = right - left;
    const float gy = down - up;
    const float m2 = gx * gx + gy * gy;
    const float gi = __shfl_sync(kFull, g_half, i);  // lane i holds half its weight
    const bool any = m2 > 0.0f;
    const float m = any ? m2 * rsqrtf(m2) : 0.0f;
    float w1;
    const int b0 = orient_bin(any ? gx : 1.0f, gy, w1);
    const int b1 = (b0 + 1) & 7;
    // (g_i g_j) |grad|: gi and g_half carry a factor 1/2 each, m a factor 2
    const float gm = (2.0f * gi * g_half) * m;
    const float v1 = gm * w1;
    float *col = &S.priv[i >> 3][0][lane];
    col[b0 * 32] += gm - v1;
    col[b1 * 32] += v1;
}

// Zeroes the lane-private histogram (warp mode: all four cell rows).
__device__ __forceinline__ void priv_zero_warp(WarpHist &S, int lane)
{
    float4 *z = reinterpret_cast<float4 *>(&S.priv[0][0][0]);
#pragma unroll
    for (int q = 0; q < 8; ++q)
        z[q * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// SIFT variants after L2 normalisation (flags: HS_CLIP 0.2 clip and
// renormalise, HS_ROOT L1-normalise and take square roots) of a histogram
// spread over the warp, n entries per lane.
template <int N>
__device__ __forceinline__ void variants_warp(float (&h)[N], int flags)
{
    if (flags & BD_HS_VARIANT_CLIP) {
        float ss = 0.0f;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            h[q] = fminf(h[q], 0.2f);
            ss += h[q] * h[q];
        }
        const float nrm = sqrtf(warp_sum_f(ss));
#pragma unroll
        for (int q = 0; q < N; ++q)
            h[q] = nrm > 0.0f ? h[q] / nrm : 0.0f;
    }
    if (flags & BD_HS_VARIANT_ROOT) {
        float l1 = 0.0f;
#pragma unroll
        for (int q = 0; q < N; ++q)
            l1 += h[q];
        l1 = warp_sum_f(l1);
#pragma unroll
        for (int q = 0; q < N; ++q)
            h[q] = l1 > 0.0f ? sqrtf(h[q] / l1) : 0.0f;
    }
}

// Cell sums, L2 norm, variants and output of a warp-mode histogram: lane
// (cell column cj, bin b) owns entries ci*32 + lane, ci = 0..3.
__device__ __forceinline__ void warp_finish(WarpHist &S, int lane, bool valid,
                                            float *__restrict__ hist, size_t k,
                                            float *__restrict__ norm_out, int flags)
{
    const int cj = lane >> 3, b = lane & 7;
    float H[4];
    float ss = 0.0f;
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            s += S.priv[ci][b][cj * 8 + ((q + b) & 7)];
        H[ci] = s;
        ss += s * s;
    }
    const float nrm = sqrtf(warp_sum_f(ss));
    if (norm_out && lane == 0)
        norm_out[k] = valid ? nrm : 0.0f;
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
        H[ci] = (valid && nrm > 0.0f) ? H[ci] / nrm : 0.0f;
    if (flags)
        variants_warp<4>(H, flags);
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
        hist[k * kHistDim + ci * 32 + lane] = H[ci];
    __syncwarp();
}

// Histogram of one keypoint by one warp: rows from `src` (a ColSampler or a
// PatchMem), output like the oracle's [cell][bin] order, L2-normalised,
// with the optional norm.
template <class Src>
__device__ __forceinline__ void hs_hist_warp(WarpHist &S, const Src &src, bool valid, int lane,
                                             float *__restrict__ hist, size_t k,
                                             float *__restrict__ norm_out, int flags)
{
    {
        float4 *z = reinterpret_cast<float4 *>(&S.priv[0][0][0]);
#pragma unroll
        for (int q = 0; q < 8; ++q)
            z[q * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncwarp();
    if (valid) {
        // 1. samples in 4x8 blocks: block bb covers rows 4 (bb / 4) + [0, 4),
        //    columns 8 (bb % 4) + [0, 8); lane -> (lane / 8, lane % 8)
        const int bi = lane >> 3, bj = lane & 7;
#pragma unroll 8
        for (int bb = 0; bb < 32; ++bb) {
            const int i = 4 * (bb >> 2) + bi, j = 8 * (bb & 3) + bj;
            S.P[i][j] = src.at(i, j);
        }
        __syncwarp();
        // 2. votes down this lane's column
        const float g_half = 0.5f * gauss16(lane);
        float up = S.P[0][lane];  // replicated row -1
        float here = up;
#pragma unroll 8
        for (int i = 0; i < PS; ++i) {
            const float down = S.P[i < PS - 1 ? i + 1 : PS - 1][lane];
            vote_px(S, lane, i, up, here, down, g_half);
            up = here;
            here = down;
        }
    }
    __syncwarp();
    warp_finish(S, lane, valid, hist, k, norm_out, flags);
}

// CTA-wide sum of one float per thread (the four warps of a 128-thread CTA).
__device__ __forceinline__ float cta_sum4(WarpHist &S, float v, int lane, int w)
{
    v = warp_sum_f(v);
    __syncthreads();  // earlier readers of wss are done
    if (lane == 0)
        S.wss[w] = v;
    __syncthreads();
    return S.wss[0] + S.wss[1] + S.wss[2] + S.wss[3];
}

// Cell sums of warp w's cell row, L2 norm over the CTA, variants, output.
__device__ __forceinline__ void cta_finish(WarpHist &S, int t, bool valid,
                                           float *__restrict__ hist, size_t k,
                                           float *__restrict__ norm_out, int flags)
{
    const int lane = t & 31, w = t >> 5;
    const int cj = lane >> 3, b = lane & 7;
    float H = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        H += S.priv[w][b][cj * 8 + ((q + b) & 7)];
    const float nrm = sqrtf(cta_sum4(S, H * H, lane, w));
    if (norm_out && t == 0)
        norm_out[k] = valid ? nrm : 0.0f;
    float hv = (valid && nrm > 0.0f) ? H / nrm : 0.0f;
    if (flags & BD_HS_VARIANT_CLIP) {
        hv = fminf(hv, 0.2f);
        const float n2 = sqrtf(cta_sum4(S, hv * hv, lane, w));
        hv = n2 > 0.0f ? hv / n2 : 0.0f;
    }
    if (flags & BD_HS_VARIANT_ROOT) {
        const float l1 = cta_sum4(S, hv, lane, w);
        hv = l1 > 0.0f ? sqrtf(hv / l1) : 0.0f;
    }
    hist[k * kHistDim + w * 32 + lane] = hv;
    __syncthreads();  // S is reused by the next keypoint
}

// The same histogram by the four warps of a 128-thread CTA sharing one
// keypoint (lower latency when keypoints are few): warp w samples and votes
// rows [8w, 8w + 8), i.e. cell row w, and normalises its 32 entries with the
// CTA's sum of squares.  All 128 threads call it; S is the CTA's buffer.
template <class Src>
__device__ __forceinline__ void hs_hist_cta(WarpHist &S, const Src &src, bool valid,
                                            float *__restrict__ hist, size_t k,
                                            float *__restrict__ norm_out, int flags)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    {
        float4 *z = reinterpret_cast<float4 *>(&S.priv[w][0][0]);
        z[lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        z[lane + 32] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (valid) {
        const int bi = lane >> 3, bj = lane & 7;
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // blocks 8w .. 8w + 7: rows 8w .. 8w + 7
            const int bb = 8 * w + q;
            const int i = 4 * (bb >> 2) + bi, j = 8 * (bb & 3) + bj;
            S.P[i][j] = src.at(i, j);
        }
    }
    __syncthreads();
    if (valid) {
        const float g_half = 0.5f * gauss16(lane);
        float up = S.P[w > 0 ? 8 * w - 1 : 0][lane];
        float here = S.P[8 * w][lane];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int i = 8 * w + r;
            const float down = S.P[i < PS - 1 ? i + 1 : PS - 1][lane];
            vote_px(S, lane, i, up, here, down, g_half);
            up = here;
            here = down;
        }
    }
    __syncwarp();
    cta_finish(S, t, valid, hist, k, norm_out, flags);
}

// Warp mode from a staged footprint: the lane samples its column on the fly
// (one sample per pixel, taps from shared memory) while it votes.
__device__ __forceinline__ void hs_hist_warp_win(WarpHist &S, const WinGeom &g, const ColFrame &c,
                                                 const uint8_t *img, int pitch, int lane,
                                                 float *__restrict__ hist, size_t k, int flags)
{
    priv_zero_warp(S, lane);
    win_stage(S.win, g, img, pitch, lane, 32);
    __syncwarp();
    const uint8_t *win = reinterpret_cast<const uint8_t *>(S.win);
    const float g_half = 0.5f * gauss16(lane);
    float here = win_sample(win, g, c, 0, lane);
    float up = here;  // replicated row -1
#pragma unroll 4
    for (int i = 0; i < PS; ++i) {
        const float down = i < PS - 1 ? win_sample(win, g, c, i + 1, lane) : here;
        vote_px(S, lane, i, up, here, down, g_half);
        up = here;
        here = down;
    }
    __syncwarp();
    warp_finish(S, lane, true, hist, k, nullptr, flags);
}

// CTA mode from a staged footprint: the CTA stages it, warp w samples rows
// 8w - 1 .. 8w + 8 on the fly and votes rows [8w, 8w + 8).
__device__ __forceinline__ void hs_hist_cta_win(WarpHist &S, const WinGeom &g, const ColFrame &c,
                                                const uint8_t *img, int pitch,
                                                float *__restrict__ hist, size_t k, int flags)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    {
        float4 *z = reinterpret_cast<float4 *>(&S.priv[w][0][0]);
        z[lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        z[lane + 32] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    win_stage(S.win, g, img, pitch, t, 128);
    __syncthreads();
    const uint8_t *win = reinterpret_cast<const uint8_t *>(S.win);
    const float g_half = 0.5f * gauss16(lane);
    float up = win_sample(win, g, c, w > 0 ? 8 * w - 1 : 0, lane);
    float here = win_sample(win, g, c, 8 * w, lane);
#pragma unroll 4
    for (int r = 0; r < 8; ++r) {
        const int i = 8 * w + r;
        const float down = i < PS - 1 ? win_sample(win, g, c, i + 1, lane) : here;
        vote_px(S, lane, i, up, here, down, g_half);
        up = here;
        here = down;
    }
    __syncwarp();
    cta_finish(S, t, true, hist, k, nullptr, flags);
}

// ---------------------------------------------------------------------------
// trilinear binning (SIFT variant): a vote is shared by the two nearest cell
// rows and columns, cell c centred at pixel 8c + 3.5 with weight 1 - |x - (8c +
// 3.5)| / 8.  Lane j's column always splits between the same two cell columns
// c0 = floor((j - 3.5) / 8) and c0 + 1 (slots 0 and 1), so the lane keeps a
// private [cell row][slot][bin] histogram; the finish sums, for each cell
// column, slot 0 of the lanes with c0 = cj and slot 1 of those with c0 = cj - 1.

struct WarpHistTri {
    float P[PS][kPRow];
    float priv[4][2][8][32];  // [cell row][slot][bin][lane]
};

template <class Src>
__device__ __forceinline__ void hs_hist_warp_tri(WarpHistTri &S, const Src &src, bool valid,
                                                 int lane, float *__restrict__ hist, size_t k,
                                                 int flags)
{
    {
        float4 *z = reinterpret_cast<float4 *>(&S.priv[0][0][0][0]);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            z[q * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncwarp();
    if (valid) {
        const int bi = lane >> 3, bj = lane & 7;
#pragma unroll 8
        for (int bb = 0; bb < 32; ++bb) {
            const int i = 4 * (bb >> 2) + bi, j = 8 * (bb & 3) + bj;
            S.P[i][j] = src.at(i, j);
        }
        __syncwarp();
        // this lane's column weights
        const float xc = ((float)lane - 3.5f) * 0.125f;
        const int c0 = (int)floorf(xc);
        const float wx1 = xc - (float)c0;
        const float wxs[2] = {c0 >= 0 ? 1.0f - wx1 : 0.0f, c0 + 1 <= 3 ? wx1 : 0.0f};
        const float g_half = 0.5f * gauss16(lane);
        float up = S.P[0][lane];
        float here = up;
#pragma unroll 4
        for (int i = 0; i < PS; ++i) {
            const float down = S.P[i < PS - 1 ? i + 1 : PS - 1][lane];
            const float left = __shfl_up_sync(kFull, here, 1);
            const float right = __shfl_down_sync(kFull, here, 1);
            const float gx = right - left;
            const float gy = down - up;
            const float m2 = gx * gx + gy * gy;
            const float gi = __shfl_sync(kFull, g_half, i);
            const bool any = m2 > 0.0f;
            const float m = any ? m2 * rsqrtf(m2) : 0.0f;
            float w1;
            const int b0 = orient_bin(any ? gx : 1.0f, gy, w1);
            const int b1 = (b0 + 1) & 7;
            const float gm = (2.0f * gi * g_half) * m;
            const float yc = ((float)i - 3.5f) * 0.125f;
            const int r0 = (int)floorf(yc);
            const float wy1 = yc - (float)r0;
#pragma unroll
            for (int dr = 0; dr < 2; ++dr) {
                const int ci = r0 + dr;
                if (ci < 0 || ci > 3)
                    continue;
                const float wy = dr ? wy1 : 1.0f - wy1;
#pragma unroll
                for (int sl = 0; sl < 2; ++sl) {
                    const float v = gm * (wy * wxs[sl]);
                    const float v1 = v * w1;
                    float *col = &S.priv[ci][sl][0][lane];
                    col[b0 * 32] += v - v1;
                    col[b1 * 32] += v1;
                }
            }
            up = here;
            here = down;
        }
    }
    __syncwarp();
    // entry (ci, cj, b): slot 0 of lanes [8cj + 4, 8cj + 12), slot 1 of lanes [8cj - 4, 8cj + 4)
    const int cj = lane >> 3, b = lane & 7;
    float H[4];
    float ss = 0.0f;
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int la = 8 * cj + 4 + ((q + b) & 7);
            const int lb = 8 * cj - 4 + ((q + b) & 7);
            if (la < 32)
                s += S.priv[ci][0][b][la];
            if (lb >= 0)
                s += S.priv[ci][1][b][lb];
        }
        H[ci] = s;
        ss += s * s;
    }
    const float nrm = sqrtf(warp_sum_f(ss));
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
        H[ci] = (valid && nrm > 0.0f) ? H[ci] / nrm : 0.0f;
    if (flags & (BD_HS_VARIANT_CLIP | BD_HS_VARIANT_ROOT))
        variants_warp<4>(H, flags);
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
        hist[k * kHistDim + ci * 32 + lane] = H[ci];
    __syncwarp();
}

// Trilinear histogram of keypoint k sampled from the image (warp mode).
__device__ __forceinline__ void hs_hist_image_warp_tri(WarpHistTri &S, const uint8_t *img, int w,
                                                       int h, int pitch, const bd_keypoint &kp,
                                                       float spacing, float *hist, size_t k,
                                                       DeviceStatus *status, int flags)
{
    const int lane = threadIdx.x & 31;
    const bool valid = kp_valid(kp);
    ColSampler<false> edge;
    if (!valid) {
        if (lane == 0)
            raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
        hs_hist_warp_tri(S, edge, false, lane, hist, k, flags);
        return;
    }
    const Frame f = make_frame(kp, spacing);
    if (col_interior(f, w, h)) {
        ColSampler<true> in;
        in.c = col_frame(img, w, h, pitch, f, lane);
        hs_hist_warp_tri(S, in, true, lane, hist, k, flags);
    } else {
        edge.c = col_frame(img, w, h, pitch, f, lane);
        hs_hist_warp_tri(S, edge, true, lane, hist, k, flags);
    }
}

// Histogram of keypoint k of n sampled from the image by the whole CTA.
// UseWin: stage the footprint in shared memory when it fits (the per-image
// kernel; the batched kernel keeps the smaller code without it).
template <bool UseWin>
__device__ __forceinline__ void hs_hist_image_cta(WarpHist &S, const uint8_t *img, int w, int h,
                                                  int pitch, const bd_keypoint &kp, float spacing,
                                                  float *hist, size_t k, DeviceStatus *status,
                                                  int flags)
{
    const bool valid = kp_valid(kp);
    ColSampler<false> edge;
    if (!valid) {
        if (threadIdx.x == 0)
            raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
        hs_hist_cta(S, edge, false, hist, k, nullptr, flags);
        return;
    }
    const Frame f = make_frame(kp, spacing);
    WinGeom g;
    if (UseWin && win_geom(f, img, w, h, pitch, g)) {
        hs_hist_cta_win(S, g, col_frame(img, w, h, pitch, f), img, pitch, hist, k, flags);
    } else if (col_interior(f, w, h)) {
        ColSampler<true> in;
        in.c = col_frame(img, w, h, pitch, f);
        hs_hist_cta(S, in, true, hist, k, nullptr, flags);
    } else {
        edge.c = col_frame(img, w, h, pitch, f);
        hs_hist_cta(S, edge, true, hist, k, nullptr, flags);
    }
}

// Histogram of keypoint k of n sampled from the image; all 32 lanes call it.
template <bool UseWin>
__device__ __forceinline__ void hs_hist_image_warp(WarpHist &S, const uint8_t *img, int w, int h,
                                                   int pitch, const bd_keypoint &kp, float spacing,
                                                   float *hist, size_t k, DeviceStatus *status,
                                                   int flags)
{
    const int lane = threadIdx.x & 31;
    const bool valid = kp_valid(kp);
    ColSampler<false> edge;
    if (!valid) {
        if (lane == 0)
            raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
        hs_hist_warp(S, edge, false, lane, hist, k, nullptr, flags);
        return;
    }
    const Frame f = make_frame(kp, spacing);
    WinGeom g;
    if (UseWin && win_geom(f, img, w, h, pitch, g)) {
        hs_hist_warp_win(S, g, col_frame(img, w, h, pitch, f, lane), img, pitch, lane, hist, k,
                         flags);
    } else if (col_interior(f, w, h)) {
        ColSampler<true> in;
        in.c = col_frame(img, w, h, pitch, f, lane);
        hs_hist_warp(S, in, true, lane, hist, k, nullptr, flags);
    } else {
        edge.c = col_frame(img, w, h, pitch, f, lane);
        hs_hist_warp(S, edge, true, lane, hist, k, nullptr, flags);
    }
}

}  // namespace dev
}  // namespace bd
