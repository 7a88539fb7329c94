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
// Persistent, warp-specialised kernel, one CTA per SM.  CTA c works on the
// 128-bit chunk c / cpc of the hash (its W^T head and tail tiles stay in
// shared memory for the whole launch, loaded once by TMA) and on a
// contiguous range of 128-keypoint blocks; per block:
//  - 7 converter warps (rows w, w + 7, ...: one coalesced 512-byte row per
//    warp load, all of a warp's rows in flight) split the FP32 rows into BF16
//    head and tail in registers and write them into one of two operand
//    stages in the 128-byte-swizzled K-major layout TMA would produce (no
//    BF16 copy of the histograms in global memory);
//  - one thread issues 8 K-steps x (2 or 3) MMAs into one of two TMEM
//    accumulators and commits them to the stage's "empty" barrier and the
//    accumulator's "full" barrier;
//  - 8 epilogue warps (TMEM lane quadrant = warp mod 4, two warps per
//    quadrant, 64 columns each) read the accumulator, add the bias, take
//    the sign and the band mask, release the
//    accumulator, then re-check their rows' band bits in FP32 from the
//    histogram row and the FP32 W^T row (L2), in the FP32 projection
//    kernel's order: four 32-term chains from zero, ((c0 + c1) + c2) + c3,
//    plus the bias; a row of zeros (a patch without gradients) projects to
//    exactly the bias on both paths and is never re-checked.
// So the conversion of block j + 1, the MMAs of block j and the epilogue of
// block j - 1 overlap.  When the histogram producer has already written the
// rows in that operand image (the batched kernel does, as it finishes each
// histogram), one thread copies each block's 64 KB stage with bulk copies
// instead, and the zero-row flags come with it: no conversion remains.  The
// other six converter warps then take over the re-check: the epilogue warps
// hand the block's words and band bits over in shared memory (two buffers),
// and those warps re-check the bits while the epilogue goes on with the next
// block, then store the words (a block with more than RLCAP band bits keeps
// the rest for the epilogue warps' own re-check); from 16384 keypoints, where
// each CTA has several blocks.  Every mbarrier wait is bounded; a wait that gives up
// raises BD_FLAG_TIMEOUT and stops every role at its next block; the CTA
// then waits (bounded) for the MMAs it issued and the W loads before it
// frees TMEM and returns.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int BM = 128;          // keypoints per block
constexpr int BN = 128;          // bits per chunk (one CTA's W slice)
constexpr int TILE = BM * 128;   // bytes of one 64-wide BF16 K half of a 128-row operand
constexpr int NCONV = 7;         // converter warps: rows cw, cw + 7, ... (16 warps in all:
                                 // registers are granted for whole groups of 4 warps)
constexpr int CROWS = (128 + NCONV - 1) / NCONV;  // rows per converter warp, at most
constexpr int CBATCH = CROWS;    // rows a converter lane has in flight (all of them)
constexpr int NZSLOTS = 8;       // zero-row flags, by block: a converter reaches block
                                 // j + 8 only after the epilogue finished block j
constexpr int LCAP = 256;        // band bits an epilogue warp re-checks per round
constexpr int NEPI = 8;          // epilogue warps: TMEM lane quadrant warp mod 4, 64 columns each
constexpr int ECOLS = BN * 4 / NEPI;  // columns per epilogue warp
constexpr int NTH = 32 * (1 + NCONV + NEPI);
constexpr int NRES = NCONV - 1;  // with the pre-split operand image: warps 2 .. NCONV re-check
constexpr int RLCAP = 1024;      // band bits of one block handed to them (two buffers)
constexpr int STAGES = 2;        // A operand stages
constexpr int ACCS = 2;          // TMEM accumulators of BN columns
// W (head K0, head K1, tail K0, tail K1) + STAGES x A (same four tiles)
constexpr int smem_bytes() { return (4 + 4 * STAGES) * TILE + 1024; }

// Offset of 16-byte chunk c (0..7) of row r in a 128-row x 128-byte operand
// tile with the 128-byte swizzle: chunk positions are XORed with r mod 8.
__device__ __forceinline__ uint32_t sw128_offset(int r, int c)
{
    return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// BF16 head and tail of 4 FP32 values (x = hi + lo + O(2^-16 |x|)).
__device__ __forceinline__ void split4(const float4 &a, uint2 &hi, uint2 &lo)
{
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(a.z, a.w);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(a.x - f0.x, a.y - f0.y);
    const __nv_bfloat162 l1 = __floats2bfloat162_rn(a.z - f1.x, a.w - f1.y);
    hi = make_uint2(*reinterpret_cast<const uint32_t *>(&h0), *reinterpret_cast<const uint32_t *>(&h1));
    lo = make_uint2(*reinterpret_cast<const uint32_t *>(&l0), *reinterpret_cast<const uint32_t *>(&l1));
}

// Chunk q (terms 32 q .. 32 q + 31, one fmaf chain from zero) of the FP32
// margin of keypoint row kp for bit n0 + ec: the histogram row from global
// memory (band_rows, issued first so that several rows are in flight), W from
// the head tile in shared memory when W is exactly BF16, else the FP32 W^T
// row (L2).
__device__ __forceinline__ void band_rows(const float *__restrict__ hist32, size_t kp, int q, float4 (&fv)[8])
{
    const float4 *fr = reinterpret_cast<const float4 *>(hist32 + kp * kHistDim) + 8 * q;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        fv[i] = __ldg(fr + i);
}

__device__ __forceinline__ float band_dot(const float4 (&fv)[8], const float *__restrict__ Wt32,
                                          const uint8_t *sW, int w_has_lo, int n0, int ec, int q)
{
    float w[32];
    if (!w_has_lo) {
        // W is exactly BF16: its head tile in shared memory is W
        // (row ec, K values 32 q .. 32 q + 31: chunks 4 (q & 1) .. + 3)
        const uint8_t *wrow = sW + (q >> 1) * TILE + ec * 128;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = 4 * (q & 1) + i;
            const uint4 u = *reinterpret_cast<const uint4 *>(wrow + ((c ^ (ec & 7)) << 4));
            const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                w[8 * i + 2 * e] = __uint_as_float(uw[e] << 16);
                w[8 * i + 2 * e + 1] = __uint_as_float(uw[e] & 0xffff0000u);
            }
        }
    } else {
        const float4 *wr = reinterpret_cast<const float4 *>(Wt32 + (size_t)(n0 + ec) * kHistDim) + 8 * q;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 x = __ldg(wr + i);
            w[4 * i] = x.x;
            w[4 * i + 1] = x.y;
            w[4 * i + 2] = x.z;
            w[4 * i + 3] = x.w;
        }
    }
    float part = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        part = fmaf(fv[i].x, w[4 * i], part);
        part = fmaf(fv[i].y, w[4 * i + 1], part);
        part = fmaf(fv[i].z, w[4 * i + 2], part);
        part = fmaf(fv[i].w, w[4 * i + 3], part);
    }
    return part;
}

__global__ void __launch_bounds__(NTH, 1) hs_proj_tc_kernel(
    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int w_has_lo,
    const float *__restrict__ hist32, const float *__restrict__ Wt32,
    const float *__restrict__ bias, const float *__restrict__ band,
    const bd_keypoint *__restrict__ kps, int n, int K, uint32_t *__restrict__ out,
    DeviceStatus *status, int nblocks, int cpc, const uint8_t *__restrict__ a16,
    const uint8_t *__restrict__ nzg, float *__restrict__ relaxed, float inv_t)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sW = smem;              // head K0, head K1, tail K0, tail K1
    uint8_t *sA = smem + 4 * TILE;   // stage s at s * 4 TILE: head K0, head K1, tail K0, tail K1
    __shared__ uint64_t bar_w, bar_afull[STAGES], bar_aempty[STAGES], bar_accfull[ACCS],
        bar_accempty[ACCS], bar_nz[NZSLOTS];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_s, issued_s;
    __shared__ __align__(16) float bias_s[BN];
    __shared__ __align__(16) float band_s[BN];
    __shared__ uint8_t nz_s[NZSLOTS][BM];            // row has a nonzero histogram entry
    __shared__ uint16_t list_s[NEPI][LCAP];            // band bits: row in warp << 7 | column
    __shared__ uint32_t words_s[NEPI][32][ECOLS / 32]; // the warp's output words
    // with the pre-split image: block j's band bits (row << 7 | column) and
    // output words, buffer j % 2, the bits' count and the re-checking warps
    // done with them
    __shared__ uint32_t rl_s[2][RLCAP];
    __shared__ __align__(16) uint32_t wb_s[2][BM][BN / 32];
    __shared__ unsigned int rl_cnt[2], rl_done[2];
    __shared__ uint64_t bar_lfull[2], bar_lempty[2];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int chunk = blockIdx.x / cpc, part = blockIdx.x % cpc;
    const int n0 = chunk * BN;
    const int bb0 = (int)((long long)nblocks * part / cpc);
    // band bits handed to the re-checking warps when the CTAs have several
    // blocks to overlap (below that the hand-off only adds latency)
    const bool handoff = a16 != nullptr && n >= 16384;
    const int nb = (int)((long long)nblocks * (part + 1) / cpc) - bb0;

    if (t == 0) {
        dev::mbar_init(&bar_w, 1);
        for (int s = 0; s < STAGES; ++s) {
            // converter threads arrive, or the copying thread with the bytes
            dev::mbar_init(&bar_afull[s], a16 ? 1 : 32 * NCONV);
            dev::mbar_init(&bar_aempty[s], 1);
        }
        for (int a = 0; a < ACCS; ++a) {
            dev::mbar_init(&bar_accfull[a], 1);
            dev::mbar_init(&bar_accempty[a], 32 * NEPI);
        }
        for (int z = 0; z < NZSLOTS; ++z)
            dev::mbar_init(&bar_nz[z], NCONV);  // lane 0 of each converter warp
        for (int b = 0; b < 2; ++b) {
            dev::mbar_init(&bar_lfull[b], NEPI);   // lane 0 of each epilogue warp
            dev::mbar_init(&bar_lempty[b], NRES);  // lane 0 of each re-checking warp
            rl_cnt[b] = 0u;
            rl_done[b] = 0u;
        }
        dev::fence_mbar_init();
        abort_s = 0;
        issued_s = 0;
    }
    if (t < BN) {
        bias_s[t] = __ldg(bias + n0 + t);
        band_s[t] = __ldg(band + n0 + t);
    }
    if (warp == 0)
        dev::tmem_alloc(&tmem_slot, ACCS * BN);
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // W is a parameter, not written by earlier kernels: load it right away
    if (t == 0) {
        dev::mbar_arrive_expect_tx(&bar_w, (w_has_lo ? 4 : 2) * TILE);
        dev::tma_load_2d(sW, &tmBh, 0, n0, &bar_w);
        dev::tma_load_2d(sW + TILE, &tmBh, 64, n0, &bar_w);
        if (w_has_lo) {
            dev::tma_load_2d(sW + 2 * TILE, &tmBl, 0, n0, &bar_w);
            dev::tma_load_2d(sW + 3 * TILE, &tmBl, 64, n0, &bar_w);
        }
    }
    // programmatic launch: the prologue above overlaps the previous kernel
    // (which writes the histograms read below)
    dev::griddep_wait();
    dev::griddep_launch_dependents();

    auto give_up = [&]() {
        abort_s = 1;
        dev::raise_flag(status, BD_FLAG_TIMEOUT);
    };

    if (warp == 0) {
        // ---- MMA issue (one thread) ----
        if (lane == 0) {
            const uint32_t idesc = dev::umma_idesc_bf16_f32(BM, BN);
            int j = 0;
            bool ok = dev::mbar_wait_bounded(&bar_w, 0);
            for (; ok && j < nb; ++j) {
                const int s = j % STAGES, a = j % ACCS;
                const uint32_t ps = (uint32_t)(j / STAGES) & 1u, pa = (uint32_t)(j / ACCS) & 1u;
                if (*(volatile int *)&abort_s || !dev::mbar_wait_bounded(&bar_afull[s], ps) ||
                    !dev::mbar_wait_bounded(&bar_accempty[a], pa ^ 1u)) {
                    ok = false;
                    break;
                }
                dev::tc_fence_after();
                const uint8_t *Ah = sA + s * 4 * TILE, *Al = Ah + 2 * TILE;
                const uint32_t d = tmem + (uint32_t)(a * BN);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ahd = dev::umma_desc_sw128(dev::smem_u32(Ah + h * TILE + k * 32));
                        const uint64_t ald = dev::umma_desc_sw128(dev::smem_u32(Al + h * TILE + k * 32));
                        const uint64_t bhd = dev::umma_desc_sw128(dev::smem_u32(sW + h * TILE + k * 32));
                        dev::umma_bf16(d, ahd, bhd, idesc, (h | k) ? 1u : 0u);
                        dev::umma_bf16(d, ald, bhd, idesc, 1u);
                        if (w_has_lo) {
                            const uint64_t bld =
                                dev::umma_desc_sw128(dev::smem_u32(sW + (2 + h) * TILE + k * 32));
                            dev::umma_bf16(d, ahd, bld, idesc, 1u);
                        }
                    }
                dev::umma_commit(&bar_aempty[s]);
                dev::umma_commit(&bar_accfull[a]);
            }
            if (!ok)
                give_up();
            issued_s = j;
        }
        __syncwarp();
    } else if (warp <= NCONV && a16) {
        // ---- pre-split operands: bulk copies of each block's stage ----
        if (warp == 1 && lane == 0) {
            for (int j = 0; j < nb; ++j) {
                const int s = j % STAGES;
                const uint32_t ps = (uint32_t)(j / STAGES) & 1u;
                if (*(volatile int *)&abort_s)
                    break;
                if (!dev::mbar_wait_bounded(&bar_aempty[s], ps ^ 1u)) {
                    give_up();
                    break;
                }
                uint8_t *dst = sA + s * 4 * TILE;
                const uint8_t *src = a16 + (size_t)(bb0 + j) * (4 * TILE);
                dev::mbar_arrive_expect_tx(&bar_afull[s], 4 * TILE);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dev::bulk_load(dst + q * TILE, src + q * TILE, TILE, &bar_afull[s]);
            }
        } else if (warp >= 2 && handoff) {
            // ---- FP32 re-check of the band bits the epilogue handed over ----
            // block j's list (buffer j % 2): 16 bits per pass and warp, 4 lanes
            // per bit, in the FP32 projection kernel's order, the bit set or
            // cleared in the block's words in shared memory; the last warp
            // done with a block stores its words and clears the list's count
            // before the epilogue may fill that buffer again
            const int rw = warp - 2, g = lane >> 2, q = lane & 3;
            unsigned long long rescued = 0;
            for (int j = 0; j < nb; ++j) {
                const int b = j & 1;
                if (__any_sync(0xffffffffu, *(volatile int *)&abort_s != 0))
                    break;
                if (!__all_sync(0xffffffffu, dev::mbar_wait_bounded(&bar_lfull[b], (uint32_t)(j >> 1) & 1u))) {
                    give_up();
                    break;
                }
                const unsigned int cnt = *(volatile unsigned int *)&rl_cnt[b];
                const unsigned int ne = cnt < (unsigned int)RLCAP ? cnt : (unsigned int)RLCAP;
                const int m0 = (bb0 + j) * BM;
                // two bits per lane group and pass: both rows' loads in flight
#pragma unroll 1
                for (unsigned int e0 = (unsigned int)rw * 16u; e0 < ne; e0 += NRES * 16u) {
                    uint32_t v[2];
                    float4 fv[2][8];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const unsigned int e = e0 + 8u * (unsigned int)u + (unsigned int)g;
                        v[u] = e < ne ? rl_s[b][e] : 0xffffffffu;
                        if (v[u] != 0xffffffffu)
                            band_rows(hist32, (size_t)m0 + (v[u] >> 7), q, fv[u]);
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const bool act = v[u] != 0xffffffffu;
                        const int r = (int)(v[u] >> 7), ec = (int)(v[u] & 127u);
                        const float part = act ? band_dot(fv[u], Wt32, sW, w_has_lo, n0, ec, q) : 0.0f;
                        const float c1 = __shfl_down_sync(0xffffffffu, part, 1);
                        const float c2 = __shfl_down_sync(0xffffffffu, part, 2);
                        const float c3 = __shfl_down_sync(0xffffffffu, part, 3);
                        if (act && q == 0) {
                            const float m32 = ((part + c1) + c2) + c3 + bias_s[ec];
                            uint32_t *w = &wb_s[b][r][ec >> 5];
                            const uint32_t bit = 1u << (ec & 31);
                            if (m32 > 0.0f)
                                atomicOr(w, bit);
                            else
                                atomicAnd(w, ~bit);
                            ++rescued;
                        }
                    }
                }
                __syncwarp();
                __threadfence_block();
                unsigned int done = 0;
                if (lane == 0)
                    done = atomicAdd(&rl_done[b], 1u);
                done = __shfl_sync(0xffffffffu, done, 0);
                if (done == (unsigned int)NRES - 1u) {
                    // the other warps' corrections are in: store the block's words
                    __threadfence_block();
                    for (int r = lane; r < BM; r += 32) {
                        const int kp = m0 + r;
                        if (kp < n)
                            *reinterpret_cast<uint4 *>(out + (size_t)kp * (K / 32) + n0 / 32) =
                                *reinterpret_cast<const uint4 *>(&wb_s[b][r][0]);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        rl_cnt[b] = 0u;
                        rl_done[b] = 0u;
                    }
                }
                __syncwarp();
                if (lane == 0)
                    dev::mbar_arrive(&bar_lempty[b]);
                __syncwarp();
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                rescued += __shfl_xor_sync(0xffffffffu, rescued, o);
            if (lane == 0 && rescued)
                atomicAdd(&status->rescued, rescued);
        }
        __syncwarp();
    } else if (warp <= NCONV) {
        // ---- histogram rows -> BF16 head / tail operand stages ----
        const int cw = warp - 1;
        const int h = lane >> 4, c = (lane & 15) >> 1, sub = lane & 1;  // values 4 lane .. 4 lane + 3
        for (int j = 0; j < nb; ++j) {
            const int s = j % STAGES;
            const uint32_t ps = (uint32_t)(j / STAGES) & 1u;
            // warp-uniform decisions: the warp meets in shuffles below
            if (__any_sync(0xffffffffu, *(volatile int *)&abort_s != 0))
                break;
            // the MMAs of block j - STAGES have read this stage
            if (!__all_sync(0xffffffffu, dev::mbar_wait_bounded(&bar_aempty[s], ps ^ 1u))) {
                give_up();
                break;
            }
            const int m0 = (bb0 + j) * BM;
            uint8_t *Ah = sA + s * 4 * TILE, *Al = Ah + 2 * TILE;
#pragma unroll
            for (int q0 = 0; q0 < CROWS; q0 += CBATCH) {  // CBATCH rows in flight per lane
                float4 v[CBATCH];
#pragma unroll
                for (int q = 0; q < CBATCH; ++q) {
                    const int r = cw + NCONV * (q0 + q), row = m0 + r;
                    v[q] = (q0 + q < CROWS && r < BM && row < n)
                               ? __ldg(reinterpret_cast<const float4 *>(hist32 + (size_t)row * kHistDim) + lane)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < CBATCH; ++q) {
                    const int r = cw + NCONV * (q0 + q);
                    if (q0 + q >= CROWS || r >= BM)
                        break;
                    const uint32_t off = (uint32_t)(h * TILE) + sw128_offset(r, c) + (uint32_t)(sub * 8);
                    uint2 hi, lo;
                    split4(v[q], hi, lo);
                    *reinterpret_cast<uint2 *>(Ah + off) = hi;
                    *reinterpret_cast<uint2 *>(Al + off) = lo;
                    const uint32_t nzl = (__float_as_uint(v[q].x) | __float_as_uint(v[q].y) |
                                          __float_as_uint(v[q].z) | __float_as_uint(v[q].w)) & 0x7fffffffu;
                    const bool any = __any_sync(0xffffffffu, nzl != 0u);
                    if (lane == 0)
                        nz_s[j % NZSLOTS][r] = any ? 1 : 0;
                }
            }
            dev::fence_proxy_async_smem();
            dev::mbar_arrive(&bar_afull[s]);
            if (lane == 0)  // this warp's zero-row flags are written (release to the epilogue)
                dev::mbar_arrive(&bar_nz[j % NZSLOTS]);
        }
    } else {
        // ---- epilogue: TMEM -> bits, FP32 re-check of the band ----
        const int ew = warp - 1 - NCONV;
        const int qd = warp & 3, row = qd * 32 + lane, c0 = (ew >> 2) * ECOLS;
        static_assert(NEPI == 8 && ECOLS == 64, "two epilogue warps per TMEM lane quadrant");
        uint16_t *list = list_s[ew];
        uint32_t(*wds)[ECOLS / 32] = words_s[ew];
        unsigned long long rescued = 0;
        for (int j = 0; j < nb; ++j) {
            const int a = j % ACCS;
            const uint32_t pa = (uint32_t)(j / ACCS) & 1u;
            if (__any_sync(0xffffffffu, *(volatile int *)&abort_s != 0))
                break;
            // the row's keypoint and zero-row flag, loaded before the wait
            const int m0 = (bb0 + j) * BM, kp = m0 + row;
            const bool valid = kp < n && (kps == nullptr || dev::kp_valid(kps[kp]));
            const uint8_t nz_row = (a16 && kp < n) ? __ldg(nzg + kp) : (uint8_t)0;
            if (!__all_sync(0xffffffffu, dev::mbar_wait_bounded(&bar_accfull[a], pa))) {
                give_up();
                break;
            }
            dev::tc_fence_after();
            // the converters' zero-row flags of this block (already complete:
            // they were written before the MMAs could start), or the producer's
            if (!a16 && !__all_sync(0xffffffffu, dev::mbar_wait_bounded(&bar_nz[j % NZSLOTS],
                                                                       (uint32_t)(j / NZSLOTS) & 1u))) {
                give_up();
                break;
            }
            const bool row_nz = a16 ? nz_row != 0 : nz_s[j % NZSLOTS][row] != 0;
            uint32_t r[ECOLS];
            dev::tmem_ld64(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(a * BN + c0), r);
            uint32_t near[ECOLS / 32];
#pragma unroll
            for (int cc = 0; cc < ECOLS / 32; ++cc) {
                uint32_t wd = 0, nr = 0;
#pragma unroll
                for (int q4 = 0; q4 < 8; ++q4) {
                    const float4 bv = *reinterpret_cast<const float4 *>(&bias_s[c0 + cc * 32 + 4 * q4]);
                    const float4 dv = *reinterpret_cast<const float4 *>(&band_s[c0 + cc * 32 + 4 * q4]);
                    const float bb[4] = {bv.x, bv.y, bv.z, bv.w}, db[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = 4 * q4 + u;
                        const float m = __uint_as_float(r[cc * 32 + q]) + bb[u];
                        wd |= (m > 0.0f ? 1u : 0u) << q;
                        nr |= (fabsf(m) < db[u] ? 1u : 0u) << q;
                    }
                }
                wds[lane][cc] = valid ? wd : 0u;
                near[cc] = (valid && row_nz) ? nr : 0u;
            }
            dev::tc_fence_before();
            dev::mbar_arrive(&bar_accempty[a]);
            if (relaxed && kp < n) {
                // relaxed responses tanh(m / T) of these margins (training path)
                float4 *dst = reinterpret_cast<float4 *>(relaxed + (size_t)kp * K + n0 + c0);
#pragma unroll
                for (int i = 0; i < ECOLS / 4; ++i) {
                    const float4 bv = *reinterpret_cast<const float4 *>(&bias_s[c0 + 4 * i]);
                    float4 o;
                    o.x = dev::tanh_relaxed((__uint_as_float(r[4 * i]) + bv.x) * inv_t);
                    o.y = dev::tanh_relaxed((__uint_as_float(r[4 * i + 1]) + bv.y) * inv_t);
                    o.z = dev::tanh_relaxed((__uint_as_float(r[4 * i + 2]) + bv.z) * inv_t);
                    o.w = dev::tanh_relaxed((__uint_as_float(r[4 * i + 3]) + bv.w) * inv_t);
                    dst[i] = o;
                }
            }
            // with the pre-split image, the band bits go to the re-checking
            // warps (buffer j % 2, free once they are done with block j - 2);
            // a warp whose bits no longer fit marks the slots it reserved
            // unused and re-checks its bits itself below
            const int lb = j & 1;
            if (handoff) {
                if (!__all_sync(0xffffffffu, dev::mbar_wait_bounded(&bar_lempty[lb],
                                                                   ((uint32_t)(j >> 1) & 1u) ^ 1u))) {
                    give_up();
                    break;
                }
                const uint32_t cnt = __popc(near[0]) + __popc(near[1]);
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o)
                        incl += u;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
                if (total) {
                    uint32_t base = 0;
                    if (lane == 0)
                        base = atomicAdd(&rl_cnt[lb], total);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (base + total <= (uint32_t)RLCAP) {
                        uint32_t e = base + incl - cnt;
#pragma unroll
                        for (int cc = 0; cc < ECOLS / 32; ++cc) {
                            for (uint32_t m = near[cc]; m; m &= m - 1, ++e)
                                rl_s[lb][e] = ((uint32_t)row << 7) | (uint32_t)(c0 + cc * 32 + __ffs(m) - 1);
                            near[cc] = 0u;
                        }
                    } else {
                        for (uint32_t sl = base + lane; sl < (uint32_t)RLCAP && sl < base + total; sl += 32)
                            rl_s[lb][sl] = 0xffffffffu;
                    }
                }
            }
            // rounds: the lanes whose bits fit (a prefix of the warp) list
            // them; then 8 bits per pass, 4 lanes per bit (32-term chunk q of
            // the margin each, all loads in flight), combined in the FP32
            // projection kernel's order ((c0 + c1) + c2) + c3 + bias
            __syncwarp();
            for (;;) {
                const uint32_t cnt = __popc(near[0]) + __popc(near[1]);
                if (__all_sync(0xffffffffu, cnt == 0u))
                    break;
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o)
                        incl += u;
                }
                const bool fits = incl <= (uint32_t)LCAP;
                const uint32_t total = __shfl_sync(0xffffffffu, incl, 31 - __clz(__ballot_sync(0xffffffffu, fits)));
                if (fits) {
                    uint32_t e = incl - cnt;
#pragma unroll
                    for (int cc = 0; cc < ECOLS / 32; ++cc) {
                        for (uint32_t m = near[cc]; m; m &= m - 1, ++e)
                            list[e] = (uint16_t)((lane << 7) | (c0 + cc * 32 + __ffs(m) - 1));
                        near[cc] = 0u;
                    }
                }
                __syncwarp();
                const int g = lane >> 2, q = lane & 3;
#pragma unroll 1
                for (uint32_t e0 = 0; e0 < total; e0 += 8) {
                    const uint32_t e = e0 + (uint32_t)g;
                    const bool act = e < total;
                    const uint32_t v = act ? (uint32_t)list[e] : 0u;
                    const int er = (int)(v >> 7), ec = (int)(v & 127u);
                    float part = 0.0f;
                    if (act) {
                        float4 fv[8];
                        band_rows(hist32, (size_t)(m0 + qd * 32 + er), q, fv);
                        part = band_dot(fv, Wt32, sW, w_has_lo, n0, ec, q);
                    }
                    const float c1 = __shfl_down_sync(0xffffffffu, part, 1);
                    const float c2 = __shfl_down_sync(0xffffffffu, part, 2);
                    const float c3 = __shfl_down_sync(0xffffffffu, part, 3);
                    if (act && q == 0) {
                        const float m32 = ((part + c1) + c2) + c3 + bias_s[ec];
                        const uint32_t bit = 1u << (ec & 31);
                        if (m32 > 0.0f)
                            atomicOr(&wds[er][(ec - c0) >> 5], bit);
                        else
                            atomicAnd(&wds[er][(ec - c0) >> 5], ~bit);
                    }
                }
                rescued += total;  // counted on every lane; lane 0's copy is added below
                __syncwarp();
            }
            if (handoff) {
                // the block's words go to the re-checking warps with the list
#pragma unroll
                for (int cc = 0; cc < ECOLS / 32; ++cc)
                    wb_s[lb][row][c0 / 32 + cc] = wds[lane][cc];
                __syncwarp();
                if (lane == 0)
                    dev::mbar_arrive(&bar_lfull[lb]);
            } else if (kp < n) {
                uint32_t *dst = out + (size_t)kp * (K / 32) + (n0 + c0) / 32;
#pragma unroll
                for (int cc = 0; cc < ECOLS / 32; ++cc)
                    dst[cc] = wds[lane][cc];
            }
            __syncwarp();
        }
        if (lane == 0 && rescued)
            atomicAdd(&status->rescued, rescued);
    }

    // leave together; after a timeout, the MMAs issued and the W loads land
    // before TMEM is freed and the CTA exits
    __syncthreads();
    if (t == 0 && abort_s) {
        const int j = issued_s - 1;
        if (j >= 0)
            dev::mbar_wait_bounded(&bar_accfull[j % ACCS], (uint32_t)(j / ACCS) & 1u);
        dev::mbar_wait_bounded(&bar_w, 0);
    }
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    if (warp == 0)
        dev::tmem_dealloc(tmem, ACCS * BN);
}

}  // namespace

cudaError_t prepare_hs_proj_tc()
{
    return cudaFuncSetAttribute(hs_proj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes());
}

cudaError_t launch_hs_proj_tc(const bd_hs_params *p, const float *hist, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st, const bd_keypoint *kps,
                              const uint8_t *a16, const uint8_t *nz, float *relaxed, float inv_t)
{
    if (n <= 0)
        return cudaSuccess;
    // one CTA per SM: the 128-bit chunks share the SMs, each chunk's CTAs
    // split its 128-keypoint blocks into contiguous ranges
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int chunks = p->nbits / BN;
    const int nblocks = (n + BM - 1) / BM;
    if (a16 && !nz)
        return cudaErrorInvalidValue;
    int cpc = sms / chunks;
    if (cpc < 1)
        cpc = 1;
    if (cpc > nblocks)
        cpc = nblocks;
    cudaError_t e = launch_pdl(hs_proj_tc_kernel, dim3(chunks * cpc), dim3(NTH), (size_t)smem_bytes(),
                               st, p->tmap_w_hi, p->tmap_w_lo, p->w_has_lo ? 1 : 0, hist,
                               (const float *)p->d_Wt, (const float *)p->d_bias,
                               (const float *)p->d_band, kps, n, p->nbits, out, status, nblocks, cpc,
                               a16, nz, relaxed, inv_t);
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "hs_proj_tc");
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
