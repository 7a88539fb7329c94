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
// phases:
//  - thread 0 loads the W^T head / tail tiles with TMA (128-byte swizzle):
//    both phases at the start when the grid is one wave or less (BothB,
//    96 KB of shared memory, lowest latency), else one phase at a time
//    through one stage (64 KB; two CTAs per SM either way, by registers,
//    and three measured slower: less of the SM's memory is left as L1);
//  - every thread loads its share of the FP32 histogram rows for both
//    phases at once (row t/2, half t%2 of the phase's 64 values), splits
//    them into BF16 head and tail in registers and writes the phase's A
//    operands into shared memory in the same 128-byte-swizzled K-major
//    layout TMA would produce (no separate conversion pass and no BF16 copy
//    of the histograms in global memory);
//  - thread 0 issues 4 x (2 or 3) MMAs of K = 16 per phase, committed to an
//    mbarrier; the A stage is refilled for phase 1 once phase 0's MMAs are done;
//  - warps w and w+4 read TMEM lane quadrant w%4 (= 32 keypoints), each half
//    of the columns, add the FP32 bias, take the sign and the band mask
//    without branches;
//  - a row of zeros (a patch without gradients) projects to exactly the bias
//    on both paths (every product is zero), so its bits are never queued;
//  - band bits go to a list in shared memory and are re-evaluated in FP32
//    64 at a time, four lanes per bit: lane q sums terms [32q, 32q + 32) as a
//    chain from zero (histogram row and FP32 W row from L2), and the partials
//    are combined in the FP32 projection kernel's order ((c0 + c1) + c2) + c3.
// Waits on mbarriers are bounded; on a timeout the CTA raises
// BD_FLAG_TIMEOUT, waits once more for its MMAs, frees TMEM and returns.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int TILE = BM * 128;              // bytes of one 64-wide BF16 K chunk of a 128-row operand
constexpr int NTH = 256;                    // threads per CTA
// A hi/lo (one phase) + B hi/lo (both phases, or one stage)
constexpr int smem_bytes(bool both_b) { return (both_b ? 6 : 4) * TILE + 1024; }
static_assert(2048 + 2 * BM * BN <= 4 * TILE, "output tile and band list do not fit the operand area");

// Offset of 16-byte chunk c (0..7) of row r in a 128-row x 128-byte operand
// tile with the 128-byte swizzle: chunk positions are XORed with r mod 8.
__device__ __forceinline__ uint32_t sw128_offset(int r, int c)
{
    return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// Splits 8 FP32 values into BF16 head and tail (x = hi + lo + O(2^-16 |x|))
// and stores both 16-byte chunks.
__device__ __forceinline__ void split_store8(const float4 &a, const float4 &b, uint8_t *hi_dst,
                                             uint8_t *lo_dst)
{
    const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hv = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
        const float2 hf = __bfloat1622float2(hv);
        const __nv_bfloat162 lv = __floats2bfloat162_rn(x[2 * q] - hf.x, x[2 * q + 1] - hf.y);
        h[q] = *reinterpret_cast<const uint32_t *>(&hv);
        l[q] = *reinterpret_cast<const uint32_t *>(&lv);
    }
    *reinterpret_cast<uint4 *>(hi_dst) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo_dst) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <bool BothB>
__global__ void __launch_bounds__(NTH, 2) hs_proj_tc_kernel(
    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int w_has_lo,
    const float *__restrict__ hist32, const float *__restrict__ Wt32,
    const float *__restrict__ bias, const float *__restrict__ band,
    const bd_keypoint *__restrict__ kps, int n, int K, uint32_t *__restrict__ out,
    DeviceStatus *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sAh = smem, *sAl = smem + TILE;
    uint8_t *sB = smem + 2 * TILE;  // phase p: head at tile 2p, tail at 2p + 1 (BothB; else p = 0)
    __shared__ uint64_t bar_b0, bar_b1, bar_mma0, bar_mma1;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int list_n;
    __shared__ float bias_s[BN], band_s[BN];
    __shared__ int row_nz[BM];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // the bit tiles of one keypoint tile are neighbours in launch order, so they
    // read the same histogram rows while those are still in L2
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    if (t == 0) {
        dev::mbar_init(&bar_b0, 1);
        dev::mbar_init(&bar_b1, 1);
        dev::mbar_init(&bar_mma0, 1);
        dev::mbar_init(&bar_mma1, 1);
        dev::fence_mbar_init();
        abort_flag = 0;
        list_n = 0;
    }
    if (t < BN) {
        bias_s[t] = __ldg(bias + n0 + t);
        band_s[t] = __ldg(band + n0 + t);
    }
    static_assert(BN <= NTH, "one thread per bias entry");
    // W is a parameter, not written by earlier kernels: load it right away
    auto load_b = [&](int p) {
        uint8_t *dst = BothB ? sB + 2 * p * TILE : sB;
        uint64_t *bar = p == 0 ? &bar_b0 : &bar_b1;
        dev::mbar_arrive_expect_tx(bar, (w_has_lo ? 2 : 1) * TILE);
        dev::tma_load_2d(dst, &tmBh, 64 * p, n0, bar);
        if (w_has_lo)
            dev::tma_load_2d(dst + TILE, &tmBl, 64 * p, n0, bar);
    };
    if (t == 0) {
        load_b(0);
        if (BothB)
            load_b(1);
    }
    // programmatic launch: the prologue above overlaps the previous kernel
    // (which writes the histograms read below)
    dev::griddep_wait();
    dev::griddep_launch_dependents();

    // this thread's histogram values: row ar, values [64p + 32 ah, + 32) of phase p
    const int ar = t >> 1, ah = t & 1;
    float4 av[2][8];
    {
        const bool in = m0 + ar < n;
        const float4 *src = reinterpret_cast<const float4 *>(hist32 + (size_t)(m0 + ar) * kHistDim);
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int v = 0; v < 8; ++v)
                av[p][v] = in ? __ldg(src + 16 * p + 8 * ah + v) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // A row of zeros projects to exactly the bias on either path: no re-check
    {
        uint32_t nz = 0;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int v = 0; v < 8; ++v)
                nz |= (__float_as_uint(av[p][v].x) | __float_as_uint(av[p][v].y) |
                       __float_as_uint(av[p][v].z) | __float_as_uint(av[p][v].w)) & 0x7fffffffu;
        nz |= __shfl_xor_sync(0xffffffffu, nz, 1);
        if (ah == 0)
            row_nz[ar] = nz != 0u;
    }
    // epilogue row and its validity, fetched early
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const int kp = m0 + row;
    const bool valid = kp < n && (kps == nullptr || dev::kp_valid(kps[kp]));

    if (warp == 0)
        dev::tmem_alloc(&tmem_slot, BN);
    // phase 0 A operands
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint32_t off = sw128_offset(ar, 4 * ah + c);
        split_store8(av[0][2 * c], av[0][2 * c + 1], sAh + off, sAl + off);
    }
    dev::fence_proxy_async_smem();
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = dev::umma_idesc_bf16_f32(BM, BN);

    int issued = 0;  // commits issued (thread 0)
    auto issue = [&](int p) {
        const uint8_t *bh = BothB ? sB + 2 * p * TILE : sB, *bl = bh + TILE;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const uint64_t ahd = dev::umma_desc_sw128(dev::smem_u32(sAh + s * 32));
            const uint64_t ald = dev::umma_desc_sw128(dev::smem_u32(sAl + s * 32));
            const uint64_t bhd = dev::umma_desc_sw128(dev::smem_u32(bh + s * 32));
            const uint64_t bld = dev::umma_desc_sw128(dev::smem_u32(bl + s * 32));
            dev::umma_bf16(tmem, ahd, bhd, idesc, (p | s) ? 1u : 0u);
            dev::umma_bf16(tmem, ald, bhd, idesc, 1u);
            if (w_has_lo)
                dev::umma_bf16(tmem, ahd, bld, idesc, 1u);
        }
        dev::umma_commit(p == 0 ? &bar_mma0 : &bar_mma1);
        ++issued;
    };
    int b_loads = BothB ? 2 : 1;  // W loads issued (thread 0)
    if (t == 0) {
        if (dev::mbar_wait_bounded(&bar_b0, 0)) {
            dev::tc_fence_after();
            issue(0);
        } else {
            abort_flag = 1;
        }
    }
    // phase 1 A operands, once phase 0's MMAs have read the stage
    __syncthreads();
    bool ok = abort_flag == 0;
    if (ok)
        ok = dev::mbar_wait_bounded(&bar_mma0, 0);
    if (ok) {
        if (!BothB && t == 0) {  // the W stage is free too: its phase-1 tiles
            load_b(1);
            b_loads = 2;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t off = sw128_offset(ar, 4 * ah + c);
            split_store8(av[1][2 * c], av[1][2 * c + 1], sAh + off, sAl + off);
        }
        dev::fence_proxy_async_smem();
    }
    dev::tc_fence_before();
    ok = __syncthreads_and(ok) != 0;
    dev::tc_fence_after();
    if (ok && t == 0) {
        if (dev::mbar_wait_bounded(&bar_b1, 0)) {
            dev::tc_fence_after();
            issue(1);
        } else {
            abort_flag = 1;
        }
    }
    ok = __syncthreads_and(ok && abort_flag == 0) != 0;
    if (ok)
        ok = dev::mbar_wait_bounded(&bar_mma1, 0);
    ok = __syncthreads_and(ok) != 0;
    dev::tc_fence_after();

    if (ok) {
        // The operand area is dead now: it holds the output tile and the list
        // of band bits (row << 7 | column, at most 128 x 128 entries).
        uint32_t *out_tile = reinterpret_cast<uint32_t *>(smem);           // [128][BN/32], 2 KB
        uint16_t *list = reinterpret_cast<uint16_t *>(smem + 2048);        // up to 32 KB
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
            const int c = half * 2 + cc;  // 32-column chunk of this warp
            uint32_t r[32];
            dev::tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 32), r);
            uint32_t word = 0, near = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float m = __uint_as_float(r[j]) + bias_s[c * 32 + j];
                word |= (m > 0.0f ? 1u : 0u) << j;
                near |= (fabsf(m) < band_s[c * 32 + j] ? 1u : 0u) << j;
            }
            if (!valid || !row_nz[row])
                near = 0u;
            out_tile[row * (BN / 32) + c] = valid ? word : 0u;
            if (near) {
                int e = atomicAdd(&list_n, __popc(near));
                for (uint32_t m = near; m; m &= m - 1, ++e)
                    list[e] = (uint16_t)((row << 7) | (c * 32 + __ffs(m) - 1));
            }
        }
        __syncthreads();
        // FP32 re-check of the listed bits, 64 at a time: the four lanes of a
        // group sum one 32-term chunk each as a chain from zero (histogram row
        // and W row from L2), and the group's first lane combines them in the
        // FP32 projection kernel's order ((c0 + c1) + c2) + c3 + b.
        const int total = list_n;
        const int g = t >> 2, q = t & 3;
#pragma unroll 1
        for (int e0 = 0; e0 < total; e0 += NTH / 4) {
            const int e = e0 + g;
            const bool act = e < total;
            const uint32_t v = act ? (uint32_t)list[e] : 0u;
            const int er = (int)(v >> 7), ec = (int)(v & 127u);
            float part = 0.0f;
            if (act) {
                const float4 *fr = reinterpret_cast<const float4 *>(hist32 + (size_t)(m0 + er) * kHistDim) + 8 * q;
                const float4 *wr = reinterpret_cast<const float4 *>(Wt32 + (size_t)(n0 + ec) * kHistDim) + 8 * q;
                float4 fv[8], wv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    fv[i] = __ldg(fr + i);
                    wv[i] = __ldg(wr + i);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    part = fmaf(fv[i].x, wv[i].x, part);
                    part = fmaf(fv[i].y, wv[i].y, part);
                    part = fmaf(fv[i].z, wv[i].z, part);
                    part = fmaf(fv[i].w, wv[i].w, part);
                }
            }
            const float c1 = __shfl_down_sync(0xffffffffu, part, 1);
            const float c2 = __shfl_down_sync(0xffffffffu, part, 2);
            const float c3 = __shfl_down_sync(0xffffffffu, part, 3);
            if (act && q == 0) {
                const float m32 = ((part + c1) + c2) + c3 + bias_s[ec];
                uint32_t *o = &out_tile[er * (BN / 32) + (ec >> 5)];
                if (m32 > 0.0f)
                    atomicOr(o, 1u << (ec & 31));
                else
                    atomicAnd(o, ~(1u << (ec & 31)));
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
        // the W loads land before the CTA leaves
        dev::mbar_wait_bounded(&bar_b0, 0);
        if (b_loads >= 2)
            dev::mbar_wait_bounded(&bar_b1, 0);
    }
    dev::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        dev::tmem_dealloc(tmem, BN);
}

}  // namespace

cudaError_t prepare_hs_proj_tc()
{
    cudaError_t e = cudaFuncSetAttribute(hs_proj_tc_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes(true));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hs_proj_tc_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(false));
    return e;
}

cudaError_t launch_hs_proj_tc(const bd_hs_params *p, const float *hist, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st, const bd_keypoint *kps)
{
    dim3 grid(p->nbits / BN, (n + BM - 1) / BM);
    // one wave or less (two CTAs per SM): both W phases resident, lowest
    // latency; more: the single-stage variant, with more shared memory left
    // to L1
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool both_b = (long long)grid.x * grid.y <= 2LL * sms;
    cudaError_t e = launch_pdl(both_b ? hs_proj_tc_kernel<true> : hs_proj_tc_kernel<false>, grid,
                               dim3(NTH), (size_t)smem_bytes(both_b), st, p->tmap_w_hi,
                               p->tmap_w_lo, p->w_has_lo ? 1 : 0, hist, (const float *)p->d_Wt,
                               (const float *)p->d_bias, (const float *)p->d_band, kps, n,
                               p->nbits, out, status);
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "hs_proj_tc");
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
