// BAD descriptor of one keypoint (Sec. III-A).  Shared by the per-image
// gather kernel (bad.cu) and the batched persistent kernel.
//
// Each bit compares two equal-sized boxes: h = +1 iff the exact integer stump
// sum1 - sum2 <= floor(num * s'^2 / den) holds, the sums taken from the
// integral image (4 lookups each, zero outside the image) at the box
// positions of the keypoint's (level, angle-bin) table.  The 2K boxes of a
// table are stored sorted by top-left row (then side, then column), so the
// 32 boxes of one warp-wide load sit on a few image rows: about 9 cache
// lines per load on the batched workload's tables instead of 27 when lane j
// takes bit j.  The box sums go to shared memory by box id; then lane j of
// word w forms bit 32 w + j and the warp packs 32 stumps per __ballot_sync.
#pragma once

#include "bd_internal.h"

namespace bd {
namespace dev {

struct BadTables {
    const short4 *box;      // [L][NB][2K] (x, y, side, id = 2 k + j) of box j of pair k,
                            // top-left corner from the keypoint's pixel; sorted per table
    const int *thr;         // [L][K] integer threshold on sum1 - sum2
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

// Barrier of the P warps sharing a keypoint: the warp itself, or named
// barrier `id` (1 or 2, immediates so that the kernel reserves only those)
// over their 32 P threads.
template <int P>
__device__ __forceinline__ void bad_sync(int id)
{
    if (P == 1)
        __syncwarp();
    else if (id == 1)
        asm volatile("bar.sync 1, %0;" ::"n"(32 * P) : "memory");
    else
        asm volatile("bar.sync 2, %0;" ::"n"(32 * P) : "memory");
}

// The NW words of keypoint kp to out[0..NW), by P warps (1, 2 or 4) that all
// call it with the same kp: `part` is this warp's index among them, `sums`
// 2K words of shared memory they share, `bar` their named barrier (P > 1).
// Warp `part` sums box groups [part 2NW/P, (part + 1) 2NW/P) of 32 boxes and
// forms words [part NW/P, (part + 1) NW/P).
template <int NW, int P, bool ReadOnly>
__device__ __forceinline__ void bad_describe_boxes(const BadTables &T, const uint32_t *ii,
                                                   int stride, int w, int h, const bd_keypoint &kp,
                                                   uint32_t *out, DeviceStatus *status,
                                                   uint32_t *sums, int part, int bar)
{
    constexpr int K = NW * 32;
    constexpr int GPW = 2 * NW / P;  // box groups of this warp
    constexpr int WPW = NW / P;      // output words of this warp
    const int lane = threadIdx.x & 31;
    if (!kp_valid(kp)) {  // the same branch in every warp of the group
        if (lane < WPW)
            out[part * WPW + lane] = 0u;
        if (lane == 0)
            raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
        return;
    }
    const int ix = round_coord(kp.x);
    const int iy = round_coord(kp.y);
    int l, b;
    bad_cell(T, kp, l, b);
    const short4 *tab = T.box + ((size_t)l * T.nbins + b) * (2 * K) + (size_t)part * GPW * 32;
    const int *st = T.thr + (size_t)l * K + part * WPW * 32;
    int thr[WPW];
#pragma unroll
    for (int q = 0; q < WPW; ++q)
        thr[q] = __ldg(st + q * 32 + lane);
    // a group's table reads first, then all its gathers: 8 x 4 loads in flight
    constexpr int G = GPW < 8 ? GPW : 8;
#pragma unroll 1
    for (int g0 = 0; g0 < GPW; g0 += G) {
        short4 e[G];
#pragma unroll
        for (int q = 0; q < G; ++q)
            e[q] = __ldg(tab + (g0 + q) * 32 + lane);
#pragma unroll
        for (int q = 0; q < G; ++q)
            sums[e[q].w] = box_sum<ReadOnly>(ii, stride, w, h, ix + e[q].x, iy + e[q].y, e[q].z);
    }
    bad_sync<P>(bar);
    uint32_t mine = 0;
#pragma unroll
    for (int q = 0; q < WPW; ++q) {
        const int k = (part * WPW + q) * 32 + lane;
        const uint2 pr = *reinterpret_cast<const uint2 *>(sums + 2 * k);
        const uint32_t word = __ballot_sync(0xffffffffu, ((int)pr.x - (int)pr.y) <= thr[q]);
        if (lane == q)
            mine = word;
    }
    if (lane < WPW)
        out[part * WPW + lane] = mine;
    bad_sync<P>(bar);  // the sums may be overwritten by the next keypoint
}

// One warp, the whole descriptor; sums: 2K words of the warp's shared memory.
template <int NW, bool ReadOnly>
__device__ __forceinline__ void bad_describe_warp(const BadTables &T, const uint32_t *ii, int stride,
                                                  int w, int h, const bd_keypoint &kp,
                                                  uint32_t *out, DeviceStatus *status,
                                                  uint32_t *sums)
{
    bad_describe_boxes<NW, 1, ReadOnly>(T, ii, stride, w, h, kp, out, status, sums, 0, 0);
}

inline BadTables bad_tables(const bd_bad_params *p)
{
    BadTables T;
    T.box = p->d_box;
    T.thr = p->d_thr;
    T.nbins = p->nbins;
    T.nlevels = p->nlevels;
    T.angle_scale = p->angle_scale;
    for (int q = 0; q < kMaxLevels; ++q)
        T.mids[q] = p->level_mid[q];
    return T;
}

}  // namespace dev
}  // namespace bd
