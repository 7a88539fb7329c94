// BAD descriptor of one keypoint by one warp (Sec. III-A).  Shared by the
// per-image gather kernel (bad.cu) and the batched persistent kernel.
//
// Lane j owns bits j, j+32, ...; for each bit it reads the pair's rotated and
// scaled corner offsets from the (level, angle-bin) table, takes the two box
// sums from the integral image (4 lookups each, zero outside the image),
// applies the exact integer stump  sum1 - sum2 <= floor(num * s'^2 / den)
// and the warp packs 32 stumps per __ballot_sync.
#pragma once

#include "bd_internal.h"

namespace bd {
namespace dev {

struct BadTables {
    const short4 *corner;   // [L][NB][K] top-left corner offsets (x1, y1, x2, y2)
    const int2 *side_thr;   // [L][K] (scaled side, integer threshold)
    int nbins, nlevels;
    float angle_scale;      // float(NB / 2 pi)
    float mids[kMaxLevels]; // float(sqrt(s_l s_{l+1}))
};

// Table reads go through the read-only path; integral reads too unless the
// table was written earlier in the same launch (persistent kernel: ReadOnly = false).
template <bool ReadOnly>
__device__ __forceinline__ uint32_t ld_ii(const uint32_t *p)
{
    if (ReadOnly)
        return __ldg(p);
    return __ldca(p);
}

template <bool ReadOnly>
__device__ __forceinline__ uint32_t box_sum(const uint32_t *ii, int stride, int w, int h, int x0,
                                            int y0, int s)
{
    const int xa = min(max(x0, 0), w), xb = min(max(x0 + s, 0), w);
    const int ya = min(max(y0, 0), h), yb = min(max(y0 + s, 0), h);
    const uint32_t *ra = ii + (size_t)ya * stride;
    const uint32_t *rb = ii + (size_t)yb * stride;
    return ld_ii<ReadOnly>(rb + xb) - ld_ii<ReadOnly>(ra + xb) - ld_ii<ReadOnly>(rb + xa) +
           ld_ii<ReadOnly>(ra + xa);
}

// Quantised pyramid level and angle bin of a (valid) keypoint.
__device__ __forceinline__ void bad_cell(const BadTables &T, const bd_keypoint &kp, int &l, int &b)
{
    l = 0;
#pragma unroll
    for (int q = 0; q + 1 < kMaxLevels; ++q)
        l += (q + 1 < T.nlevels && T.mids[q] < kp.scale) ? 1 : 0;
    b = (int)floorf(__fadd_rn(__fmul_rn(kp.angle, T.angle_scale), 0.5f)) % T.nbins;
    if (b < 0)
        b += T.nbins;
}

// Writes words [word0, word0 + WPW) of the NW words of keypoint kp to
// out[word0 ..]; all 32 lanes of the warp call it.  WPW = NW: the whole
// descriptor by one warp; WPW = NW / 4: the four warps of a CTA share the
// keypoint (its integral-image window is then read by one CTA, not four).
template <int NW, int WPW, bool ReadOnly>
__device__ __forceinline__ void bad_describe_words(const BadTables &T, const uint32_t *ii,
                                                   int stride, int w, int h, const bd_keypoint &kp,
                                                   uint32_t *out, DeviceStatus *status, int word0)
{
    constexpr int K = NW * 32;
    const int lane = threadIdx.x & 31;
    if (!kp_valid(kp)) {
        if (lane < WPW)
            out[word0 + lane] = 0u;
        if (lane == 0)
            raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
        return;
    }
    const int ix = round_coord(kp.x);
    const int iy = round_coord(kp.y);
    int l, b;
    bad_cell(T, kp, l, b);
    const short4 *tab = T.corner + ((size_t)l * T.nbins + b) * K;
    const int2 *st = T.side_thr + (size_t)l * K;
    uint32_t mine = 0;
    // a group's table reads first, then all its gathers: the warp keeps
    // 8 x 8 independent loads in flight instead of walking the bits in series
    constexpr int G = WPW < 8 ? WPW : 8;
#pragma unroll 1
    for (int j0 = word0; j0 < word0 + WPW; j0 += G) {
        short4 c[G];
        int2 s[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            c[g] = __ldg(tab + (j0 + g) * 32 + lane);
            s[g] = __ldg(st + (j0 + g) * 32 + lane);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t s1 = box_sum<ReadOnly>(ii, stride, w, h, ix + c[g].x, iy + c[g].y, s[g].x);
            const uint32_t s2 = box_sum<ReadOnly>(ii, stride, w, h, ix + c[g].z, iy + c[g].w, s[g].x);
            const bool bit = ((int)s1 - (int)s2) <= s[g].y;
            const uint32_t word = __ballot_sync(0xffffffffu, bit);
            if (lane == j0 - word0 + g)
                mine = word;
        }
    }
    if (lane < WPW)
        out[word0 + lane] = mine;
}

// Writes the NW words of keypoint kp to out[0..NW); all 32 lanes call it.
template <int NW, bool ReadOnly>
__device__ __forceinline__ void bad_describe_warp(const BadTables &T, const uint32_t *ii, int stride,
                                                  int w, int h, const bd_keypoint &kp,
                                                  uint32_t *out, DeviceStatus *status)
{
    bad_describe_words<NW, NW, ReadOnly>(T, ii, stride, w, h, kp, out, status, 0);
}

inline BadTables bad_tables(const bd_bad_params *p)
{
    BadTables T;
    T.corner = p->d_corner;
    T.side_thr = p->d_side_thr;
    T.nbins = p->nbins;
    T.nlevels = p->nlevels;
    T.angle_scale = p->angle_scale;
    for (int q = 0; q < kMaxLevels; ++q)
        T.mids[q] = p->level_mid[q];
    return T;
}

}  // namespace dev
}  // namespace bd
