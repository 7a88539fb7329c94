// HashSIFT extraction kernels over the keypoints of one image (Sec. III-B):
// patch warp, fused warp + histogram, histogram of given patches (one CTA of
// 128 threads per keypoint, grid-stride; routines in hashsift_dev.cuh), and
// the plain FP32 projection D = sgn(W^T f + b) used as the reference GPU path
// (the tensor-core projection lives in proj_tc.cu).

#include "hashsift_dev.cuh"

namespace bd {
namespace {

using dev::NT;
using dev::PS;

// Coop = false: one warp per keypoint (hs_hist_warp), the CTA's warps take
// independent keypoints; Coop = true: the CTA's four warps share each
// keypoint (hs_hist_cta), for few keypoints.
template <bool Coop>
__global__ void __launch_bounds__(NT) hs_hist_image_kernel(
    const uint8_t *__restrict__ img, int w, int h, int pitch, const bd_keypoint *__restrict__ kps,
    int n, float spacing, float *__restrict__ hist, DeviceStatus *status, int flags)
{
    __shared__ dev::WarpHist S[Coop ? 1 : NT / 32];
    if (Coop) {
        for (int k = blockIdx.x; k < n; k += gridDim.x)
            dev::hs_hist_image_cta<true>(S[0], img, w, h, pitch, kps[k], spacing, hist, (size_t)k,
                                         status, flags);
    } else {
        const int warp = threadIdx.x >> 5;
        for (int k = blockIdx.x * (NT / 32) + warp; k < n; k += gridDim.x * (NT / 32))
            dev::hs_hist_image_warp<true>(S[warp], img, w, h, pitch, kps[k], spacing, hist,
                                          (size_t)k, status, flags);
    }
}

// Trilinear-binned histograms (SIFT variant), one warp per keypoint, two
// warps per CTA (13 KB of shared memory each).
constexpr int NT_TRI = 64;
__global__ void __launch_bounds__(NT_TRI) hs_hist_image_tri_kernel(
    const uint8_t *__restrict__ img, int w, int h, int pitch, const bd_keypoint *__restrict__ kps,
    int n, float spacing, float *__restrict__ hist, DeviceStatus *status, int flags)
{
    __shared__ dev::WarpHistTri S[NT_TRI / 32];
    const int warp = threadIdx.x >> 5;
    for (int k = blockIdx.x * (NT_TRI / 32) + warp; k < n; k += gridDim.x * (NT_TRI / 32))
        dev::hs_hist_image_warp_tri(S[warp], img, w, h, pitch, kps[k], spacing, hist, (size_t)k,
                                    status, flags);
}

__global__ void __launch_bounds__(NT) hs_hist_patch_kernel(const float *__restrict__ patches,
                                                           int n, float *__restrict__ hist,
                                                           float *__restrict__ norm_out)
{
    __shared__ dev::WarpHist S[NT / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = blockIdx.x * (NT / 32) + warp; k < n; k += gridDim.x * (NT / 32)) {
        dev::PatchMem src;
        src.p = patches + (size_t)k * PS * PS;
        dev::hs_hist_warp(S[warp], src, true, lane, hist, (size_t)k, norm_out, 0);
    }
}

// Standalone patch warp (bd_hashsift_warp): the same sampler as the histogram.
__global__ void __launch_bounds__(NT) hs_warp_kernel(const uint8_t *__restrict__ img, int w, int h,
                                                     int pitch,
                                                     const bd_keypoint *__restrict__ kps, int n,
                                                     float spacing, float *__restrict__ patches,
                                                     DeviceStatus *status)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = blockIdx.x * (NT / 32) + warp; k < n; k += gridDim.x * (NT / 32)) {
        const bd_keypoint kp = kps[k];
        float *dst = patches + (size_t)k * PS * PS + lane;
        if (!dev::kp_valid(kp)) {
            for (int i = 0; i < PS; ++i)
                dst[i * PS] = 0.0f;
            if (lane == 0)
                dev::raise_flag(status, BD_FLAG_INVALID_KEYPOINT);
            continue;
        }
        const dev::Frame f = dev::make_frame(kp, spacing);
        if (dev::col_interior(f, w, h)) {
            dev::ColSampler<true> cs;
            cs.c = dev::col_frame(img, w, h, pitch, f, lane);
#pragma unroll 8
            for (int i = 0; i < PS; ++i)
                dst[i * PS] = cs.at(i, lane);
        } else {
            dev::ColSampler<false> cs;
            cs.c = dev::col_frame(img, w, h, pitch, f, lane);
#pragma unroll 8
            for (int i = 0; i < PS; ++i)
                dst[i * PS] = cs.at(i, lane);
        }
    }
}


// ---------------------------------------------------------------------------
// FP32 projection: margins m = W^T f + b, bit = m > 0.  The sum runs in four
// chunks of 32 terms, each a sequential fmaf chain from zero, combined as
// ((c0 + c1) + c2) + c3 before the bias; the tensor-core path's FP32
// re-check evaluates the same expression, so both paths give the same bits.
// Tile: 64 keypoints x 128 bits per CTA, 4 x 8 outputs per thread: rows
// 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3, so
// that a warp's 16-byte shared loads are contiguous; the two threads of a
// byte combine their nibbles by a shuffle.
// ---------------------------------------------------------------------------
constexpr int PBM = 64, PBN = 128, PBK = 32;

__global__ void __launch_bounds__(256) hs_proj_fp32_kernel(const float *__restrict__ hist, int n,
                                                           const float *__restrict__ W, int K,
                                                           const float *__restrict__ bias,
                                                           const bd_keypoint *__restrict__ kps,
                                                           uint8_t *__restrict__ out)
{
    __shared__ __align__(16) float Hs[PBK][PBM + 4];
    __shared__ __align__(16) float Ws[PBK][PBN];
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;
    const int m0 = blockIdx.x * PBM, n0 = blockIdx.y * PBN;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = 0.0f;
    // this thread's share of a 32-deep K chunk (8 histogram and 16 W values),
    // loaded into registers one chunk ahead so that the loads of chunk k + 1
    // are in flight during chunk k's FMAs
    constexpr int HQ = PBM * PBK / 256, WQ = PBK * PBN / 256;
    float hq[HQ], wq[WQ];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < HQ; ++q) {
            const int e = t + 256 * q;
            const int row = m0 + e / PBK;
            hq[q] = row < n ? __ldg(hist + (size_t)row * kHistDim + k0 + e % PBK) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            const int e = t + 256 * q;
            wq[q] = __ldg(W + (size_t)(k0 + e / PBN) * K + n0 + e % PBN);
        }
    };
    load(0);
    for (int k0 = 0; k0 < kHistDim; k0 += PBK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < HQ; ++q) {
            const int e = t + 256 * q;
            Hs[e % PBK][e / PBK] = hq[q];
        }
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            const int e = t + 256 * q;
            Ws[e / PBN][e % PBN] = wq[q];
        }
        __syncthreads();
        if (k0 + PBK < kHistDim)
            load(k0 + PBK);
        float part[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b)
                part[a][b] = 0.0f;
#pragma unroll 8
        for (int kk = 0; kk < PBK; ++kk) {
            const float4 h4 = *reinterpret_cast<const float4 *>(&Hs[kk][ty * 4]);
            const float4 w0 = *reinterpret_cast<const float4 *>(&Ws[kk][tx * 4]);
            const float4 w1 = *reinterpret_cast<const float4 *>(&Ws[kk][64 + tx * 4]);
            const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    part[a][b] = fmaf(hv[a], wv[b], part[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b)
                acc[a][b] = k0 == 0 ? part[a][b] : acc[a][b] + part[a][b];
    }
    float bv[8];
#pragma unroll
    for (int b = 0; b < 8; ++b)
        bv[b] = __ldg(bias + n0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4));
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int row = m0 + ty * 4 + a;
        const bool in = row < n;
        const bool ok = in && (kps ? dev::kp_valid(kps[row]) : true);
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            lo |= (ok && (acc[a][b] + bv[b]) > 0.0f) ? (1u << b) : 0u;
            hi |= (ok && (acc[a][b + 4] + bv[b + 4]) > 0.0f) ? (1u << b) : 0u;
        }
        // even tx: the low nibble of bytes tx / 2 and 8 + tx / 2; odd tx: the high
        const uint32_t lo_p = __shfl_xor_sync(0xffffffffu, lo, 1), hi_p = __shfl_xor_sync(0xffffffffu, hi, 1);
        if (in && !(tx & 1)) {
            uint8_t *o = out + (size_t)row * (K / 8) + n0 / 8;
            o[tx >> 1] = (uint8_t)(lo | (lo_p << 4));
            o[8 + (tx >> 1)] = (uint8_t)(hi | (hi_p << 4));
        }
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
    hs_warp_kernel<<<grid_for((n + 3) / 4, sm_count, 16), NT, 0, st>>>(img, w, h, pitch, kps, n, p->spacing,
                                                             patches, status);
    trace_kernel(st, "hs_warp");
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hs_hist_patches(const float *patches, int n, float *hist, cudaStream_t st,
                                   int sm_count,
                                   float *norm_out)
{
    hs_hist_patch_kernel<<<grid_for((n + 3) / 4, sm_count, 12), NT, 0, st>>>(patches, n, hist,
                                                                   norm_out);
    trace_kernel(st, "hs_hist_patch");
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hs_hist_image(const bd_hs_params *p, const uint8_t *img, int w, int h, int pitch,
                                 const bd_keypoint *kps, int n, float *hist,
                                 DeviceStatus *status, cudaStream_t st,
                                 int sm_count)
{
    const int flags = p->variant;
    // few keypoints: the CTA shares each one (latency); many: one per warp (throughput)
    if (flags & BD_HS_VARIANT_TRILINEAR)
        hs_hist_image_tri_kernel<<<grid_for((n + 1) / 2, sm_count, 16), NT_TRI, 0, st>>>(
            img, w, h, pitch, kps, n, p->spacing, hist, status, flags);
    else if (n <= 2 * 12 * sm_count)
        hs_hist_image_kernel<true><<<grid_for(n, sm_count, 12), NT, 0, st>>>(
            img, w, h, pitch, kps, n, p->spacing, hist, status, flags);
    else
        hs_hist_image_kernel<false><<<grid_for((n + 3) / 4, sm_count, 12), NT, 0, st>>>(
            img, w, h, pitch, kps, n, p->spacing, hist, status, flags);
    trace_kernel(st, "hs_hist_image");
    note_launches(1);
    return cudaGetLastError();
}


cudaError_t launch_hs_proj_fp32(const bd_hs_params *p, const float *hist, int n, uint32_t *out,
                                cudaStream_t st, const bd_keypoint *kps)
{
    dim3 grid((n + PBM - 1) / PBM, p->nbits / PBN);
    hs_proj_fp32_kernel<<<grid, 256, 0, st>>>(hist, n, p->d_W, p->nbits, p->d_bias, kps,
                                              reinterpret_cast<uint8_t *>(out));
    trace_kernel(st, "hs_proj_fp32");
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
