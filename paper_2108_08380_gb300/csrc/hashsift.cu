// HashSIFT feature extraction (Sec. III-B) on CUDA cores, FP32:
//  - the 32x32 patch, sampled bilinearly around the keypoint (Sec. III-A/IV-F:
//    HashSIFT describes a normalised 32x32 patch, not an image pyramid);
//  - the SIFT-style histogram: central-difference gradients, 8 orientation
//    bins with linear voting between neighbours, 4x4 cells of 8x8 pixels, a
//    sigma = 16 Gaussian weight about the patch centre, L2 normalisation;
//  - the plain FP32 projection D = sgn(W^T f + b) used as the reference GPU
//    path (the tensor-core projection lives in proj_tc.cu).
//
// One CTA of 128 threads describes one keypoint at a time (grid-stride).
// Thread t owns cell t/8 and pixel row t%8 of that cell: its 8 pixels vote
// into a thread-private 8-bin histogram in shared memory laid out [bin][thread]
// (conflict-free), and thread t then sums bin t%8 of cell t/8 over the cell's
// 8 threads.  No atomics are needed.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int NT = 128;          // threads per CTA
constexpr int PS = kPatch;       // 32
constexpr int PSP = kPatch + 1;  // padded smem row

struct Frame {
    int ix, iy;
    float fx, fy, A, B;  // A = scale*spacing*cos(angle), B = scale*spacing*sin(angle)
};

__device__ __forceinline__ Frame make_frame(const bd_keypoint &kp, float spacing)
{
    Frame f;
    f.ix = dev::round_coord(kp.x);
    f.iy = dev::round_coord(kp.y);
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
    const float ax = ox - flx, ay = oy - fly;
    const int x0 = f.ix + (int)flx, y0 = f.iy + (int)fly;
    const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    const uint8_t *ra = img + (size_t)ya * pitch;
    const uint8_t *rb = img + (size_t)yb * pitch;
    const float i00 = (float)__ldg(ra + xa), i01 = (float)__ldg(ra + xb);
    const float i10 = (float)__ldg(rb + xa), i11 = (float)__ldg(rb + xb);
    const float top = fmaf(ax, i01 - i00, i00);
    const float bot = fmaf(ax, i11 - i10, i10);
    return fmaf(ay, bot - top, top);
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
    const float di = (float)L.i - 15.5f;
    const float gi = expf(-di * di * (1.0f / 512.0f));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float dj = (float)(L.j0 + q) - 15.5f;
        L.g[q] = gi * expf(-dj * dj * (1.0f / 512.0f));
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
        const float m = sqrtf(gx * gx + gy * gy);
        float phi = atan2f(gy, gx);
        if (phi < 0.0f)
            phi += 6.28318530717958647692f;
        const float tt = phi * 1.27323954473516268615f;  // 8 / (2 pi)
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
__device__ __forceinline__ void finish(HistSmem &S, int t, bool valid, float *__restrict__ hist,
                                       __nv_bfloat16 *__restrict__ hist16, size_t kp, size_t nkp)
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
    const float h = (valid && nrm > 0.0f) ? H / nrm : 0.0f;
    hist[kp * kHistDim + t] = h;
    if (hist16) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(h);
        hist16[kp * kHistDim + t] = hi;
        hist16[(nkp + kp) * kHistDim + t] = __float2bfloat16_rn(h - __bfloat162float(hi));
    }
}

__global__ void __launch_bounds__(NT) hs_hist_image_kernel(
    const uint8_t *__restrict__ img, int w, int h, int pitch, const bd_keypoint *__restrict__ kps,
    int n, float spacing, float *__restrict__ hist, __nv_bfloat16 *__restrict__ hist16,
    DeviceStatus *status)
{
    __shared__ HistSmem S;
    const int t = threadIdx.x;
    const HistLane L = hist_lane(t);
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const bd_keypoint kp = kps[k];
        const bool valid = dev::kp_valid(kp);
        if (valid) {
            const Frame f = make_frame(kp, spacing);
#pragma unroll
            for (int r = 0; r < PS * PS / NT; ++r) {
                const int p = t + r * NT;
                S.P[p >> 5][p & 31] = sample(img, w, h, pitch, f, p >> 5, p & 31);
            }
        } else if (t == 0) {
            dev::raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b)
            S.priv[b][t] = 0.0f;
        __syncthreads();
        if (valid)
            vote(S, L, t);
        __syncthreads();
        finish(S, t, valid, hist, hist16, (size_t)k, (size_t)n);
    }
}

__global__ void __launch_bounds__(NT) hs_hist_patch_kernel(const float *__restrict__ patches,
                                                           int n, float *__restrict__ hist,
                                                           __nv_bfloat16 *__restrict__ hist16)
{
    __shared__ HistSmem S;
    const int t = threadIdx.x;
    const HistLane L = hist_lane(t);
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const float *src = patches + (size_t)k * PS * PS;
#pragma unroll
        for (int r = 0; r < PS * PS / NT; ++r) {
            const int p = t + r * NT;
            S.P[p >> 5][p & 31] = __ldg(src + p);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b)
            S.priv[b][t] = 0.0f;
        __syncthreads();
        vote(S, L, t);
        __syncthreads();
        finish(S, t, true, hist, hist16, (size_t)k, (size_t)n);
    }
}

__global__ void __launch_bounds__(NT) hs_warp_kernel(const uint8_t *__restrict__ img, int w, int h,
                                                     int pitch,
                                                     const bd_keypoint *__restrict__ kps, int n,
                                                     float spacing, float *__restrict__ patches,
                                                     DeviceStatus *status)
{
    const int t = threadIdx.x;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const bd_keypoint kp = kps[k];
        float *dst = patches + (size_t)k * PS * PS;
        if (!dev::kp_valid(kp)) {
            for (int p = t; p < PS * PS; p += NT)
                dst[p] = 0.0f;
            if (t == 0)
                dev::raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
            continue;
        }
        const Frame f = make_frame(kp, spacing);
#pragma unroll
        for (int r = 0; r < PS * PS / NT; ++r) {
            const int p = t + r * NT;
            dst[p] = sample(img, w, h, pitch, f, p >> 5, p & 31);
        }
    }
}

__global__ void hs_to_bf16_kernel(const float *__restrict__ src, size_t count,
                                  __nv_bfloat16 *__restrict__ dst)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        const float v = src[i];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        dst[i] = hi;
        dst[count + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// ---------------------------------------------------------------------------
// FP32 projection: margins m = W^T f + b accumulated in the order i = 0..127
// (the tensor-core path's FP32 re-check uses the same order, so both paths
// give the same bits), bit = m > 0.  Tile: 64 keypoints x 128 bits per CTA,
// 4 x 8 outputs per thread.
// ---------------------------------------------------------------------------
constexpr int PBM = 64, PBN = 128, PBK = 32;

__global__ void __launch_bounds__(256) hs_proj_fp32_kernel(const float *__restrict__ hist, int n,
                                                           const float *__restrict__ W, int K,
                                                           const float *__restrict__ bias,
                                                           const bd_keypoint *__restrict__ kps,
                                                           uint8_t *__restrict__ out)
{
    __shared__ float Hs[PBK][PBM + 4];
    __shared__ float Ws[PBK][PBN];
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;
    const int m0 = blockIdx.x * PBM, n0 = blockIdx.y * PBN;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = 0.0f;
    for (int k0 = 0; k0 < kHistDim; k0 += PBK) {
        __syncthreads();
        for (int e = t; e < PBM * PBK; e += 256) {
            const int r = e / PBK, c = e % PBK;
            const int row = m0 + r;
            Hs[c][r] = row < n ? __ldg(hist + (size_t)row * kHistDim + k0 + c) : 0.0f;
        }
        for (int e = t; e < PBK * PBN; e += 256) {
            const int r = e / PBN, c = e % PBN;
            Ws[r][c] = __ldg(W + (size_t)(k0 + r) * K + n0 + c);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < PBK; ++kk) {
            float hv[4], wv[8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
                hv[a] = Hs[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 8; ++b)
                wv[b] = Ws[kk][tx * 8 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    acc[a][b] = fmaf(hv[a], wv[b], acc[a][b]);
        }
    }
    float bv[8];
#pragma unroll
    for (int b = 0; b < 8; ++b)
        bv[b] = __ldg(bias + n0 + tx * 8 + b);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int row = m0 + ty * 4 + a;
        if (row >= n)
            continue;
        const bool ok = kps ? dev::kp_valid(kps[row]) : true;
        uint32_t byte = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            byte |= (ok && (acc[a][b] + bv[b]) > 0.0f) ? (1u << b) : 0u;
        out[(size_t)row * (K / 8) + (n0 + tx * 8) / 8] = (uint8_t)byte;
    }
}

int grid_for(int n, int sm_count, int per_sm)
{
    long long g = (long long)sm_count * per_sm;
    return (int)(n < g ? n : g);
}

}  // namespace

cudaError_t launch_hs_warp(const bd_hs_params *p, const uint8_t *img, int w, int h, int pitch,
                           const bd_keypoint *kps, int n, float *patches, DeviceStatus *status,
                           cudaStream_t st, int sm_count)
{
    hs_warp_kernel<<<grid_for(n, sm_count, 16), NT, 0, st>>>(img, w, h, pitch, kps, n, p->spacing,
                                                             patches, status);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hs_hist_patches(const float *patches, int n, float *hist,
                                   __nv_bfloat16 *hist16, cudaStream_t st, int sm_count)
{
    hs_hist_patch_kernel<<<grid_for(n, sm_count, 12), NT, 0, st>>>(patches, n, hist, hist16);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hs_hist_image(const bd_hs_params *p, const uint8_t *img, int w, int h, int pitch,
                                 const bd_keypoint *kps, int n, float *hist,
                                 __nv_bfloat16 *hist16, DeviceStatus *status, cudaStream_t st,
                                 int sm_count)
{
    hs_hist_image_kernel<<<grid_for(n, sm_count, 12), NT, 0, st>>>(img, w, h, pitch, kps, n,
                                                                   p->spacing, hist, hist16,
                                                                   status);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hs_to_bf16(const float *hist, int n, __nv_bfloat16 *hist16, cudaStream_t st)
{
    const size_t cnt = (size_t)n * kHistDim;
    int blocks = (int)((cnt + 255) / 256);
    if (blocks > 4096)
        blocks = 4096;
    hs_to_bf16_kernel<<<blocks, 256, 0, st>>>(hist, cnt, hist16);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hs_proj_fp32(const bd_hs_params *p, const float *hist, int n, uint32_t *out,
                                cudaStream_t st, const bd_keypoint *kps)
{
    dim3 grid((n + PBM - 1) / PBM, p->nbits / PBN);
    hs_proj_fp32_kernel<<<grid, 256, 0, st>>>(hist, n, p->d_W, p->nbits, p->d_bias, kps,
                                              reinterpret_cast<uint8_t *>(out));
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
