// HashSIFT hash D = sgn(W^T f + b) (Sec. III-B) on the 5th-generation tensor
// cores: the projection is a dense 128-deep contraction, so it runs as
// tcgen05.mma kind::f16 with BF16 operands and an FP32 accumulator in TMEM.
//
// CTA = 128 threads, tile = 128 keypoints x 256 bits.
//  - thread 0 loads the two operand tiles with TMA (128-byte swizzle, two
//    64-wide K chunks each), then issues 8 MMAs of K = 16 and commits them to
//    an mbarrier;
//  - each warp reads its 32 TMEM lanes (= keypoints) back 32 columns at a
//    time, adds the FP32 bias and takes the sign;
//  - every bit whose BF16 margin lies inside the band |m| < band_k is queued
//    and recomputed from the FP32 histogram and FP32 W (same accumulation
//    order as the FP32 projection kernel, so the two paths agree bit for bit
//    whenever the band bounds the BF16 error).
// Waits on mbarriers are bounded; on a timeout the CTA raises
// BD_FLAG_TIMEOUT, waits once more for its MMAs, frees TMEM and returns.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int A_CHUNK = BM * 128;       // bytes of one 64-wide BF16 K chunk of A
constexpr int B_CHUNK = BN * 128;       // ... of B
constexpr int TILE_BYTES = 2 * A_CHUNK + 2 * B_CHUNK;  // 98304
constexpr int SMEM_BYTES = TILE_BYTES + 1024;           // + alignment slack

__global__ void __launch_bounds__(128) hs_proj_tc_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const float *__restrict__ hist32, const float *__restrict__ Wt32,
    const float *__restrict__ bias, const float *__restrict__ band,
    const bd_keypoint *__restrict__ kps, int n, int K, uint32_t *__restrict__ out,
    DeviceStatus *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + 2 * A_CHUNK;
    __shared__ uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int list_n[BN / 32];
    __shared__ float bias_s[BN], band_s[BN];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

    if (t == 0) {
        dev::mbar_init(&bar_tma, 1);
        dev::mbar_init(&bar_mma, 1);
        dev::fence_mbar_init();
        abort_flag = 0;
    }
    if (t < BN / 32)
        list_n[t] = 0;
    for (int c = t; c < BN; c += 128) {
        bias_s[c] = __ldg(bias + n0 + c);
        band_s[c] = __ldg(band + n0 + c);
    }
    if (warp == 0)
        dev::tmem_alloc(&tmem_slot, BN);
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    const uint32_t tmem = tmem_slot;

    bool issued = false;
    if (t == 0) {
        dev::mbar_arrive_expect_tx(&bar_tma, TILE_BYTES);
        dev::tma_load_2d(sA, &tmA, 0, m0, &bar_tma);
        dev::tma_load_2d(sA + A_CHUNK, &tmA, 64, m0, &bar_tma);
        dev::tma_load_2d(sB, &tmB, 0, n0, &bar_tma);
        dev::tma_load_2d(sB + B_CHUNK, &tmB, 64, n0, &bar_tma);
        if (!dev::mbar_wait_bounded(&bar_tma, 0)) {
            abort_flag = 1;
        } else {
            dev::tc_fence_after();
            const uint32_t idesc = dev::umma_idesc_bf16_f32(BM, BN);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int chunk = kk >> 2, sub = kk & 3;
                const uint64_t a = dev::umma_desc_sw128(dev::smem_u32(sA + chunk * A_CHUNK + sub * 32));
                const uint64_t b = dev::umma_desc_sw128(dev::smem_u32(sB + chunk * B_CHUNK + sub * 32));
                dev::umma_bf16(tmem, a, b, idesc, kk > 0 ? 1u : 0u);
            }
            dev::umma_commit(&bar_mma);
            issued = true;
        }
    }
    __syncthreads();
    bool ok = abort_flag == 0;
    if (ok)
        ok = dev::mbar_wait_bounded(&bar_mma, 0);
    ok = __syncthreads_and(ok) != 0;
    dev::tc_fence_after();

    if (ok) {
        // operand tiles are dead now: reuse them for the output tile and the rescue queue
        uint32_t *out_tile = reinterpret_cast<uint32_t *>(sA);             // [128][8]
        uint16_t *queue = reinterpret_cast<uint16_t *>(sA + BM * 8 * 4);   // <= 128*32 entries
        const int row = warp * 32 + lane;
        const int kp = m0 + row;
        const bool valid = kp < n && (kps == nullptr || dev::kp_valid(kps[kp]));
        unsigned long long rescued = 0;
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t r[32];
            dev::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), r);
            uint32_t word = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float m = __uint_as_float(r[j]) + bias_s[c * 32 + j];
                word |= (m > 0.0f) ? (1u << j) : 0u;
                if (valid && fabsf(m) < band_s[c * 32 + j]) {
                    const int q = atomicAdd(&list_n[c], 1);
                    queue[q] = (uint16_t)((row << 5) | j);
                }
            }
            out_tile[row * 8 + c] = valid ? word : 0u;
            __syncthreads();
            const int cnt = list_n[c];
            for (int e = t; e < cnt; e += 128) {
                const int ent = queue[e];
                const int rr = ent >> 5, jj = ent & 31;
                const int col = n0 + c * 32 + jj;
                const float4 *hv = reinterpret_cast<const float4 *>(hist32 + (size_t)(m0 + rr) * kHistDim);
                const float4 *wv = reinterpret_cast<const float4 *>(Wt32 + (size_t)col * kHistDim);
                float acc = 0.0f;
#pragma unroll 8
                for (int i = 0; i < kHistDim / 4; ++i) {
                    const float4 a = __ldg(hv + i), b = __ldg(wv + i);
                    acc = fmaf(a.x, b.x, acc);
                    acc = fmaf(a.y, b.y, acc);
                    acc = fmaf(a.z, b.z, acc);
                    acc = fmaf(a.w, b.w, acc);
                }
                const float m32 = acc + bias_s[c * 32 + jj];
                if (m32 > 0.0f)
                    atomicOr(&out_tile[rr * 8 + c], 1u << jj);
                else
                    atomicAnd(&out_tile[rr * 8 + c], ~(1u << jj));
            }
            rescued += (unsigned long long)cnt;
            __syncthreads();
        }
        if (t == 0 && rescued)
            atomicAdd(&status->rescued, rescued);
        if (kp < n) {
            uint32_t *dst = out + (size_t)kp * (K / 32) + n0 / 32;
#pragma unroll
            for (int c = 0; c < BN / 32; ++c)
                dst[c] = out_tile[row * 8 + c];
        }
    } else if (t == 0) {
        dev::raise_flag(status, BD_FLAG_TIMEOUT);
        if (issued)
            dev::mbar_wait_bounded(&bar_mma, 0);  // let issued MMAs drain before freeing TMEM
    }
    dev::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        dev::tmem_dealloc(tmem, BN);
}

}  // namespace

cudaError_t launch_hs_proj_tc(const bd_hs_params *p, const CUtensorMap &tmap_hist,
                              const float *hist, int n, uint32_t *out, DeviceStatus *status,
                              cudaStream_t st, const bd_keypoint *kps)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(hs_proj_tc_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
        configured = true;
    }
    dim3 grid((n + BM - 1) / BM, p->nbits / BN);
    hs_proj_tc_kernel<<<grid, 128, SMEM_BYTES, st>>>(tmap_hist, p->tmap_w, hist, p->d_Wt,
                                                     p->d_bias, p->d_band, kps, n, p->nbits, out,
                                                     status);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
