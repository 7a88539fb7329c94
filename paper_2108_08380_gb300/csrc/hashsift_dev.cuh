// HashSIFT per-keypoint routines (Sec. III-B), FP32 on CUDA cores; shared by
// the per-image kernels (hashsift.cu) and the batched persistent kernel.
//
//  - the 32x32 patch, sampled bilinearly around the keypoint (Sec. IV-F:
//    HashSIFT describes a normalised 32x32 patch, not an image pyramid);
//  - the SIFT-style histogram: central-difference gradients, 8 orientation
//    bins with linear voting between neighbours, 4x4 cells of 8x8 pixels, a
//    sigma = 16 Gaussian weight about the patch centre, L2 normalisation.
//
// One CTA of 128 threads describes one keypoint.  Thread t owns cell t/8 and
// pixel row t%8 of that cell: its 8 pixels vote into a thread-private 8-bin
// histogram in shared memory laid out [bin][thread] (conflict-free), and
// thread t then sums bin t%8 of cell t/8 over the cell's 8 threads.  No
// atomics are needed.
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

// Orientation of the gradient (gx, gy) in units of pi/4, on [0, 8]: the same
// quantity as atan2(gy, gx) wrapped to [0, 2 pi) times 4/pi.  The first-octant
// angle u = (4/pi) atan(r), r = min/max of |gx|, |gy| in [0, 1], comes from an
// odd polynomial r * P(r^2) fitted here by weighted least squares on [0, 1]
// (max error 5e-8 in exact arithmetic, 2.2e-7 evaluated in FP32); the signs
// and the |gy| > |gx| test place it in its octant.  (gx, gy) != (0, 0).
__device__ __forceinline__ float orientation8(float gx, float gy)
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
    const float u = p * r;
    float q = ay > ax ? 2.0f - u : u;  // first quadrant, [0, 2]
    if (gx < 0.0f)
        q = 4.0f - q;                  // second quadrant (gy >= 0)
    if (gy < 0.0f)
        q = 8.0f - q;                  // third / fourth quadrant
    return q;
}

struct HistSmem {
    float P[PS][PSP];
    float priv[8][NT];
    float wss[NT / 32];
    int valid;
};

// Per-thread constants of the histogram mapping: pixel row i, first column j0
// and the separable Gaussian weights gi * gj[q] (Sec. III-B; sigma = 16).
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

// Votes of this thread's 8 pixels into its private histogram column.
__device__ __forceinline__ void vote(HistSmem &S, const HistLane &L, int t)
{
    const int i = L.i;
    const int iu = max(i - 1, 0), id = min(i + 1, PS - 1);
    float left = S.P[i][max(L.j0 - 1, 0)];
    float mid = S.P[i][L.j0];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = L.j0 + q;
        const float right = S.P[i][min(j + 1, PS - 1)];
        const float gx = 0.5f * (right - left);
        const float gy = 0.5f * (S.P[id][j] - S.P[iu][j]);
        left = mid;
        mid = right;
        const float m2 = gx * gx + gy * gy;
        if (!(m2 > 0.0f))
            continue;  // no gradient, no vote
        const float m = m2 * rsqrtf(m2);
        const float tt = orientation8(gx, gy);  // 8 phi / (2 pi)
        const float fl = floorf(tt);
        const float w1 = tt - fl;
        const int b0 = ((int)fl) & 7;
        const int b1 = (b0 + 1) & 7;
        const float gm = L.g[q] * m;
        const float v1 = gm * w1;
        S.priv[b0][t] += gm - v1;
        S.priv[b1][t] += v1;
    }
}

// Sum of the cell's 8 private columns for bin t%8, L2 norm, output.
__device__ __forceinline__ void hist_finish(HistSmem &S, int t, bool valid, float *__restrict__ hist,
                                       __nv_bfloat16 *__restrict__ hist16, size_t kp, size_t nkp,
                                       float *__restrict__ norm_out = nullptr)
{
    const int cell = t >> 3, b = t & 7;
    float H = 0.0f;
#pragma unroll
    for (int s = 0; s < 8; ++s)
        H += S.priv[b][cell * 8 + ((s + b) & 7)];
    float ss = H * H;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((t & 31) == 0)
        S.wss[t >> 5] = ss;
    __syncthreads();
    const float tot = S.wss[0] + S.wss[1] + S.wss[2] + S.wss[3];
    const float nrm = sqrtf(tot);
    if (norm_out && t == 0)
        norm_out[kp] = valid ? nrm : 0.0f;
    const float h = (valid && nrm > 0.0f) ? H / nrm : 0.0f;
    hist[kp * kHistDim + t] = h;
    if (hist16) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(h);
        hist16[kp * kHistDim + t] = hi;
        hist16[(nkp + kp) * kHistDim + t] = __float2bfloat16_rn(h - __bfloat162float(hi));
    }
}


// Histogram (and BF16 head/tail copies) of keypoint k of n, sampled from the
// image; all 128 threads of the CTA call it with the same keypoint.
__device__ __forceinline__ void hs_hist_one(HistSmem &S, const HistLane &L, const uint8_t *img,
                                            int w, int h, int pitch, const bd_keypoint &kp,
                                            float spacing, float *hist, __nv_bfloat16 *hist16,
                                            size_t k, size_t n, DeviceStatus *status)
{
    const int t = threadIdx.x;
    const bool valid = kp_valid(kp);
    if (valid) {
        const Frame f = make_frame(kp, spacing);
#pragma unroll
        for (int r = 0; r < PS * PS / NT; ++r) {
            const int p = t + r * NT;
            S.P[p >> 5][p & 31] = sample(img, w, h, pitch, f, p >> 5, p & 31);
        }
    } else if (t == 0) {
        raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
    }
#pragma unroll
    for (int b = 0; b < 8; ++b)
        S.priv[b][t] = 0.0f;
    __syncthreads();
    if (valid)
        vote(S, L, t);
    __syncthreads();
    hist_finish(S, t, valid, hist, hist16, k, n);
}

}  // namespace dev
}  // namespace bd
