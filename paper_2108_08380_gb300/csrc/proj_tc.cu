// HashSIFT hash D = sgn(W^T f + b) (Sec. III-B) on the 5th-generation tensor
// cores: the projection is a dense 128-deep contraction, so it runs as
// tcgen05.mma kind::f16 with BF16 operands and an FP32 accumulator in TMEM.
//
// Precision: f and W are each split into a BF16 head and a BF16 tail
// (x = hi + lo + O(2^-16 |x|)); three MMAs accumulate f_hi W_hi + f_lo W_hi +
// f_hi W_lo in FP32 (the third is skipped when W is exactly BF16).  The
// margin is then within ~8e-5 ||W_k|| of the exact one, so only bits with
// |m| below the band (default 2^-13 ||W_k||_2) are queued and recomputed from
// the FP32 histogram and FP32 W, in the FP32 projection kernel's order: the
// result equals the FP32 path bit for bit.
//
// CTA = 256 threads, tile = 128 keypoints x 128 bits, K = 128 in two 64-wide
// phases through one 64 KB shared-memory stage:
//  - thread 0 loads the phase's four operand tiles with TMA (128-byte
//    swizzle) and issues 4 x (2 or 3) MMAs of K = 16, committed to an mbarrier;
//  - warps w and w+4 read TMEM lane quadrant w%4 (= 32 keypoints), each half
//    of the columns, add the FP32 bias, take the sign and queue band bits;
//  - four threads re-evaluate each queued bit in FP32: thread q sums terms
//    [32q, 32q+32) from zero, and the four partials are combined in the FP32
//    projection kernel's order.
// Waits on mbarriers are bounded; on a timeout the CTA raises
// BD_FLAG_TIMEOUT, waits once more for its MMAs, frees TMEM and returns.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int TILE = BM * 128;             // bytes of one 64-wide BF16 K chunk of a 128-row operand
constexpr int STAGE_BYTES = 4 * TILE;      // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGE_BYTES + 1024;
constexpr int NTH = 256;                   // threads per CTA
static_assert(2048 + 2 * BM * BN <= STAGE_BYTES, "epilogue does not fit the stage");

__global__ void __launch_bounds__(NTH) hs_proj_tc_kernel(
    const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int w_has_lo,
    const float *__restrict__ hist32, const float *__restrict__ Wt32,
    const float *__restrict__ bias, const float *__restrict__ band,
    const bd_keypoint *__restrict__ kps, int n, int K, uint32_t *__restrict__ out,
    DeviceStatus *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sAh = smem, *sAl = smem + TILE, *sBh = smem + 2 * TILE, *sBl = smem + 3 * TILE;
    __shared__ uint64_t bar_tma, bar_mma0, bar_mma1;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int list_n;
    __shared__ float bias_s[BN], band_s[BN];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // the bit tiles of one keypoint tile are neighbours in launch order, so they
    // read the same histogram rows while those are still in L2
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    if (t == 0) {
        dev::mbar_init(&bar_tma, 1);
        dev::mbar_init(&bar_mma0, 1);
        dev::mbar_init(&bar_mma1, 1);
        dev::fence_mbar_init();
        abort_flag = 0;
    }
    if (t == 0)
        list_n = 0;
    if (t < BN) {
        bias_s[t] = __ldg(bias + n0 + t);
        band_s[t] = __ldg(band + n0 + t);
    }
    static_assert(BN <= NTH, "one thread per bias entry");
    // programmatic launch: the prologue above overlaps the previous kernel
    // (which writes the histograms read below)
    dev::griddep_wait();
    dev::griddep_launch_dependents();
    if (warp == 0)
        dev::tmem_alloc(&tmem_slot, BN);
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    const uint32_t tmem = tmem_slot;

    int issued = 0;  // commits issued (thread 0)
    if (t == 0) {
        const uint32_t idesc = dev::umma_idesc_bf16_f32(BM, BN);
        bool ok = true;
        for (int p = 0; p < 2 && ok; ++p) {
            if (p == 1 && !dev::mbar_wait_bounded(&bar_mma0, 0)) {  // stage free again
                ok = false;
                break;
            }
            dev::mbar_arrive_expect_tx(&bar_tma, w_has_lo ? STAGE_BYTES : 3 * TILE);
            dev::tma_load_2d(sAh, &tmAh, 64 * p, m0, &bar_tma);
            dev::tma_load_2d(sAl, &tmAl, 64 * p, m0, &bar_tma);
            dev::tma_load_2d(sBh, &tmBh, 64 * p, n0, &bar_tma);
            if (w_has_lo)
                dev::tma_load_2d(sBl, &tmBl, 64 * p, n0, &bar_tma);
            if (!dev::mbar_wait_bounded(&bar_tma, (uint32_t)p)) {
                ok = false;
                break;
            }
            dev::tc_fence_after();
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint64_t ah = dev::umma_desc_sw128(dev::smem_u32(sAh + s * 32));
                const uint64_t al = dev::umma_desc_sw128(dev::smem_u32(sAl + s * 32));
                const uint64_t bh = dev::umma_desc_sw128(dev::smem_u32(sBh + s * 32));
                const uint64_t bl = dev::umma_desc_sw128(dev::smem_u32(sBl + s * 32));
                dev::umma_bf16(tmem, ah, bh, idesc, (p | s) ? 1u : 0u);
                dev::umma_bf16(tmem, al, bh, idesc, 1u);
                if (w_has_lo)
                    dev::umma_bf16(tmem, ah, bl, idesc, 1u);
            }
            dev::umma_commit(p == 0 ? &bar_mma0 : &bar_mma1);
            ++issued;
        }
        if (!ok)
            abort_flag = 1;
    }
    __syncthreads();
    bool ok = abort_flag == 0;
    if (ok)
        ok = dev::mbar_wait_bounded(&bar_mma1, 0);
    ok = __syncthreads_and(ok) != 0;
    dev::tc_fence_after();

    if (ok) {
        // The operand stage is dead now: it holds the output tile and the queue.
        uint32_t *out_tile = reinterpret_cast<uint32_t *>(smem);                 // [128][BN/32], 2 KB
        uint16_t *queue = reinterpret_cast<uint16_t *>(smem + 2048);             // <= 128*BN entries, 32 KB
        const int quad = warp & 3, half = warp >> 2;
        const int row = quad * 32 + lane;
        const int kp = m0 + row;
        const bool valid = kp < n && (kps == nullptr || dev::kp_valid(kps[kp]));
#pragma unroll 1
        for (int cc = 0; cc < BN / 64; ++cc) {
            const int c = half * (BN / 64) + cc;  // 32-column chunk of this warp
            uint32_t r[32];
            dev::tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 32), r);
            uint32_t word = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float m = __uint_as_float(r[j]) + bias_s[c * 32 + j];
                word |= (m > 0.0f) ? (1u << j) : 0u;
                if (valid && fabsf(m) < band_s[c * 32 + j]) {
                    const int q = atomicAdd(&list_n, 1);
                    queue[q] = (uint16_t)((row << 7) | (c * 32 + j));
                }
            }
            out_tile[row * (BN / 32) + c] = valid ? word : 0u;
        }
        __syncthreads();
        // FP32 re-check: four threads per queued bit, one 32-term chunk each
        const int total = list_n;
        const int qq = t & 3;
#pragma unroll 1
        for (int base = 0; base < total; base += NTH / 4) {
            const int e = base + (t >> 2);
            const bool act = e < total;
            const int ent = act ? queue[e] : 0;
            const int rr = ent >> 7, cc = ent & 127;
            float part = 0.0f;
            if (act) {
                const float4 *hv = reinterpret_cast<const float4 *>(hist32 + (size_t)(m0 + rr) * kHistDim) + 8 * qq;
                const float4 *wv = reinterpret_cast<const float4 *>(Wt32 + (size_t)(n0 + cc) * kHistDim) + 8 * qq;
                float4 a[8], b[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    a[i] = __ldg(hv + i);
                    b[i] = __ldg(wv + i);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    part = fmaf(a[i].x, b[i].x, part);
                    part = fmaf(a[i].y, b[i].y, part);
                    part = fmaf(a[i].z, b[i].z, part);
                    part = fmaf(a[i].w, b[i].w, part);
                }
            }
            const float c1 = __shfl_down_sync(0xffffffffu, part, 1, 4);
            const float c2 = __shfl_down_sync(0xffffffffu, part, 2, 4);
            const float c3 = __shfl_down_sync(0xffffffffu, part, 3, 4);
            if (act && qq == 0) {
                const float m32 = ((part + c1) + c2) + c3 + bias_s[cc];
                if (m32 > 0.0f)
                    atomicOr(&out_tile[rr * (BN / 32) + (cc >> 5)], 1u << (cc & 31));
                else
                    atomicAnd(&out_tile[rr * (BN / 32) + (cc >> 5)], ~(1u << (cc & 31)));
            }
        }
        __syncthreads();
        if (t == 0 && total)
            atomicAdd(&status->rescued, (unsigned long long)total);
        if (t < BM && m0 + t < n) {
            uint32_t *dst = out + (size_t)(m0 + t) * (K / 32) + n0 / 32;
#pragma unroll
            for (int c = 0; c < BN / 32; ++c)
                dst[c] = out_tile[t * (BN / 32) + c];
        }
    } else if (t == 0) {
        dev::raise_flag(status, BD_FLAG_TIMEOUT);
        if (issued >= 1)
            dev::mbar_wait_bounded(&bar_mma0, 0);  // let issued MMAs drain before freeing TMEM
        if (issued >= 2)
            dev::mbar_wait_bounded(&bar_mma1, 0);
    }
    dev::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        dev::tmem_dealloc(tmem, BN);
}

}  // namespace

cudaError_t prepare_hs_proj_tc()
{
    return cudaFuncSetAttribute(hs_proj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES);
}

cudaError_t launch_hs_proj_tc(const bd_hs_params *p, const CUtensorMap &tm_hi,
                              const CUtensorMap &tm_lo, const float *hist, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st, const bd_keypoint *kps)
{
    dim3 grid(p->nbits / BN, (n + BM - 1) / BM);
    cudaError_t e = launch_pdl(hs_proj_tc_kernel, grid, dim3(NTH), SMEM_BYTES, st, tm_hi, tm_lo,
                               p->tmap_w_hi, p->tmap_w_lo, p->w_has_lo ? 1 : 0, hist,
                               (const float *)p->d_Wt, (const float *)p->d_bias,
                               (const float *)p->d_band, kps, n, p->nbits, out, status);
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "hs_proj_tc");
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
