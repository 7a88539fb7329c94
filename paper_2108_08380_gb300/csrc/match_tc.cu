// Exact Hamming matching on the tensor cores.  With +-1 codes h(x) the
// paper's similarity is S = h(x)^T h(y) = K - 2 Hamming(x, y) (Sec. III-A), a
// dense contraction: the bits are expanded to FP8 E4M3 +-1 (exact), S is
// accumulated by tcgen05.mma kind::f8f6f4 in FP32 (exact: |S| <= 512), and the
// epilogue turns S into the distance (K - S)/2 and keeps a per-query top-2 of
// packed (distance << 22 | index) keys, exactly like the POPC kernel.
//
// Persistent grid (two CTAs per SM at K = 256), stream-K split: CTA c takes an
// equal contiguous range of the (128-query block, 128-entry train tile) pairs
// in query-block-major order.  CTA = 12 warps:
//  - warp 0 (one lane) loads a block's query tile when the block changes
//    (after the MMAs that read the previous one) and the train tiles into a
//    two-stage shared-memory ring with TMA (128-byte swizzle);
//  - warp 1 (one lane) issues K/32 MMAs per train tile into one of two TMEM
//    accumulators (128 x 128 FP32 each) and commits them to mbarriers;
//  - warps 4..11 drain the accumulators: warps w and w+4 share TMEM lane
//    quadrant w%4 (32 queries) and take 64 columns each, freeing the buffer
//    for the next MMA before they update their top-2 keys; at the end of the
//    CTA's part of a block they merge the halves and write the pair, and the
//    last CTA of the block (per-block arrival counter) merges the parts.
// Every wait is bounded by the GPU timer; on expiry the CTA raises
// BD_FLAG_TIMEOUT.
#include <algorithm>

#include "bd_internal.h"

namespace bd {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int NTHREADS = 384;
constexpr int EPI_WARPS = 8;
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    if (dev::mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = gtime();
    while (!dev::mbar_try_wait(bar, parity)) {
        if (*abort_flag || gtime() - t0 > kWaitNs)
            return false;
    }
    return true;
}

// Packed bits -> one byte per bit: +1.0 (E4M3 0x38) for a set bit, -1.0 (0xB8)
// otherwise; the query words [0, qwords) then the train words, in one launch.
__global__ void expand_pm1_kernel(const uint32_t *__restrict__ qbits, size_t qwords,
                                  uint4 *__restrict__ qout, const uint32_t *__restrict__ tbits,
                                  size_t twords, uint4 *__restrict__ tout)
{
    dev::griddep_wait();  // programmatic launch: the descriptors come from the previous kernel
    dev::griddep_launch_dependents();
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < qwords + twords;
         g += (size_t)gridDim.x * blockDim.x) {
        const bool isq = g < qwords;
        const size_t w = isq ? g : g - qwords;
        uint4 *out = isq ? qout : tout;
        const uint32_t v = __ldg((isq ? qbits : tbits) + w);
        uint32_t o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                x |= (((v >> (4 * q + b)) & 1u) ? 0x38u : 0xB8u) << (8 * b);
            o[q] = x;
        }
        out[2 * w] = make_uint4(o[0], o[1], o[2], o[3]);
        out[2 * w + 1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
}

__device__ __forceinline__ void top2_push(uint32_t key, uint32_t &k1, uint32_t &k2)
{
    k2 = min(k2, max(k1, key));
    k1 = min(k1, key);
}

__device__ __forceinline__ void top2_merge(uint32_t b1, uint32_t b2, uint32_t &k1, uint32_t &k2)
{
    const uint32_t m1 = min(k1, b1);
    const uint32_t m2 = min(max(k1, b1), min(k2, b2));
    k1 = m1;
    k2 = m2;
}

__device__ __forceinline__ void finalize(uint32_t k1, uint32_t k2, int nbits, int rnum, int rden,
                                         bd_match_result *o)
{
    const uint32_t d1 = k1 >> kMatchIdxBits, d2 = k2 >> kMatchIdxBits;
    const int32_t idx = (d1 > (uint32_t)nbits) ? -1 : (int32_t)(k1 & kMatchIdxMask);
    const uint32_t acc = ((long long)rden * d1 < (long long)rnum * d2) ? 1u : 0u;
    uint32_t *w = reinterpret_cast<uint32_t *>(o);
    w[0] = (uint32_t)idx;
    w[1] = d1 | (d2 << 16);
    w[2] = acc;
}

// Stream-K split of the (query block, train tile) pairs, query-block major:
// CTA c of G takes pairs [T c / G, T (c + 1) / G).  The CTA holding pair p is
// ((p + 1) G - 1) / T; the CTAs covering query block qb are first(qb) ..
// last(qb), and their partial top-2 pairs go to slots first(qb) + qb + (c -
// first(qb)) of a (G + #blocks) x 128 array (the slots of consecutive blocks
// never overlap).
__device__ __forceinline__ int cta_of(long long p, long long T, int G)
{
    return (int)(((p + 1) * G - 1) / T);
}

// Named barrier of the eight epilogue warps (threads 128..383).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// The same barrier, returning to every epilogue thread whether any of them
// passed v = true.
__device__ __forceinline__ bool epi_sync_or(bool v)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, 1, 256, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)v)
                 : "memory");
    return r != 0;
}

// MINB: resident CTAs per SM (2 for K = 256: 96 KB of shared memory each and
// at most 85 registers per thread; 1 for K = 512).
// MINE (hard-negative mining, nq == nt): the query's own column is left out
// when excl is set and only the nearest of the rest is kept, a maximum per
// score instead of a top-2 -- the same key that the top-2 with the own
// column skipped would give, since keys are unique.
template <int K, int MINB, bool MINE>
__global__ void __launch_bounds__(NTHREADS, MINB) match_tc_kernel(
    const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmT, int nq,
    int nt, int nbits, int rnum, int rden, uint2 *__restrict__ partial,
    bd_match_result *__restrict__ out, uint2 *__restrict__ raw_keys,
    unsigned int *__restrict__ arrivals, DeviceStatus *status)
{
    constexpr int CH = K / 128;          // 128-byte K chunks per row
    constexpr int A_BYTES = BM * K;
    constexpr int B_BYTES = BN * K;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB0 = smem + A_BYTES;
    __shared__ uint64_t bar_a, bar_ae, bar_bf[2], bar_be[2], bar_tf[2], bar_te[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int last_cta;
    __shared__ uint2 half_keys[BM];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int nqb = (nq + BM - 1) / BM;
    const int ntl = max(1, (nt + BN - 1) / BN);
    const long long T = (long long)nqb * ntl;
    const bool excl = MINE && nq == nt && nt > 1;  // the own column exists and is not the only one
    const int G = (int)gridDim.x, c = (int)blockIdx.x;
    const long long p0 = T * c / G, p1 = T * (c + 1) / G;

    if (t == 0) {
        dev::mbar_init(&bar_a, 1);
        dev::mbar_init(&bar_ae, 1);
        for (int s = 0; s < 2; ++s) {
            dev::mbar_init(&bar_bf[s], 1);
            dev::mbar_init(&bar_be[s], 1);
            dev::mbar_init(&bar_tf[s], 1);
            dev::mbar_init(&bar_te[s], EPI_WARPS);
        }
        dev::fence_mbar_init();
        abort_flag = 0;
    }
    // programmatic launch: the codes were written by the previous kernel
    dev::griddep_wait();
    dev::griddep_launch_dependents();
    if (warp == 0)
        dev::tmem_alloc(&tmem_slot, 2 * BN);
    dev::tc_fence_before();
    __syncthreads();
    dev::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t sentinel = ((uint32_t)(nbits + 1) << kMatchIdxBits) | kMatchIdxMask;

    int issued = 0;  // MMA commits (warp 1)
    if (warp == 0 && lane == 0) {
        // producer: the query tile at each new block, the train tiles through a
        // two-stage ring
        bool ok = true;
        int i = 0, seg = 0;
        for (long long p = p0; ok && p < p1; ++seg) {
            const int qb = (int)(p / ntl);
            const long long pend = min(p1, (long long)(qb + 1) * ntl);
            if (seg > 0)
                ok = wait_bar(&bar_ae, (seg - 1) & 1, &abort_flag);
            if (!ok)
                break;
            dev::mbar_arrive_expect_tx(&bar_a, A_BYTES);
            for (int ch = 0; ch < CH; ++ch)
                dev::tma_load_2d(sA + ch * BM * 128, &tmQ, ch * 128, qb * BM, &bar_a);
            for (; ok && p < pend; ++p, ++i) {
                const int s = i & 1;
                if (i >= 2)
                    ok = wait_bar(&bar_be[s], ((i >> 1) - 1) & 1, &abort_flag);
                if (!ok)
                    break;
                uint8_t *sB = sB0 + s * B_BYTES;
                dev::mbar_arrive_expect_tx(&bar_bf[s], B_BYTES);
                for (int ch = 0; ch < CH; ++ch)
                    dev::tma_load_2d(sB + ch * BN * 128, &tmT, ch * 128, (int)(p % ntl) * BN,
                                     &bar_bf[s]);
            }
        }
        if (!ok)
            abort_flag = 1;
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = dev::umma_idesc_e4m3_f32(BM, BN);
        bool ok = true;
        int i = 0, seg = 0;
        for (long long p = p0; ok && p < p1; ++seg) {
            const int qb = (int)(p / ntl);
            const long long pend = min(p1, (long long)(qb + 1) * ntl);
            ok = wait_bar(&bar_a, seg & 1, &abort_flag);
            for (; ok && p < pend; ++p, ++i) {
                const int s = i & 1;
                ok = wait_bar(&bar_bf[s], (i >> 1) & 1, &abort_flag);
                if (ok && i >= 2)
                    ok = wait_bar(&bar_te[s], ((i >> 1) - 1) & 1, &abort_flag);
                if (!ok)
                    break;
                dev::tc_fence_after();
                const uint8_t *sB = sB0 + s * B_BYTES;
#pragma unroll
                for (int ch = 0; ch < CH; ++ch)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint64_t a = dev::umma_desc_sw128(dev::smem_u32(sA + ch * BM * 128 + u * 32));
                        const uint64_t b = dev::umma_desc_sw128(dev::smem_u32(sB + ch * BN * 128 + u * 32));
                        dev::umma_e4m3(tmem + s * BN, a, b, idesc, (ch | u) ? 1u : 0u);
                    }
                dev::umma_commit(&bar_be[s]);
                dev::umma_commit(&bar_tf[s]);
                ++issued;
            }
            if (ok)
                dev::umma_commit(&bar_ae);  // the query tile may be replaced once these finish
        }
        if (!ok)
            abort_flag = 1;
    } else if (warp >= 4) {
        const int ew = warp - 4, quad = warp & 3, half = ew >> 2;
        const int row = quad * 32 + lane;
        const bool owner = half == 0;
        int i = 0;
        for (long long p = p0; p < p1;) {
            const int qb = (int)(p / ntl);
            const long long pend = min(p1, (long long)(qb + 1) * ntl);
            uint32_t k1 = sentinel, k2 = sentinel;
            for (; p < pend; ++p, ++i) {
                const int s = i & 1;
                // a failed wait skips the work but keeps the loop, so that all
                // eight warps reach the block's barriers below
                if (!wait_bar(&bar_tf[s], (i >> 1) & 1, &abort_flag)) {
                    abort_flag = 1;
                    continue;
                }
                dev::tc_fence_after();
                uint32_t r[32];
                const uint32_t col = (uint32_t)(s * BN + half * 64);
                const int j0 = (int)(p % ntl) * BN + half * 64;
                const int valid = nt - j0;
                // Tile-local keys in FP32: f = 256 S - jl (jl < 64) is exact and
                // larger f means larger S (smaller distance), then smaller jl.
                // The two best f of the 64 columns become global integer keys
                // once per tile.  Two 32-column loads; the buffer is released
                // after the second.  (Packing two 16-bit keys per register for
                // packed min/max measured slower.)
                float f1 = -INFINITY, f2 = -INFINITY;
                // MINE: the query's own column (row qb BM + row) is left out;
                // it falls in one tile of the block and there in the half
                // that holds the warp's 32 rows, so `own` is warp-uniform
                const int dcol = qb * BM + row - j0;
                const bool own = MINE && excl && dcol >= 0 && dcol < 64;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    dev::tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + col + 32 * hh, r);
                    if (hh == 1) {
                        dev::tc_fence_before();
                        __syncwarp();
                        if (lane == 0)
                            dev::mbar_arrive(&bar_te[s]);
                    }
                    if (valid >= 32 * hh + 32 && !own) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float f = fmaf(__uint_as_float(r[j]), 256.0f, -(float)(32 * hh + j));
                            if (!MINE)
                                f2 = fmaxf(f2, fminf(f1, f));
                            f1 = fmaxf(f1, f);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int c = 32 * hh + j;
                            const float f = c < valid && !(own && c == dcol)
                                                ? fmaf(__uint_as_float(r[j]), 256.0f, -(float)c)
                                                : -INFINITY;
                            if (!MINE)
                                f2 = fmaxf(f2, fminf(f1, f));
                            f1 = fmaxf(f1, f);
                        }
                    }
                }
#pragma unroll
                for (int bb = 0; bb < (MINE ? 1 : 2); ++bb) {
                    const float f = bb ? f2 : f1;
                    if (f == -INFINITY)
                        continue;
                    const int S = (int)ceilf(f * (1.0f / 256.0f));  // f = 256 S - jl, 0 <= jl < 64
                    const int jl = 256 * S - (int)f;
                    const uint32_t d = (uint32_t)((K - S) >> 1);
                    top2_push((d << kMatchIdxBits) | (uint32_t)(j0 + jl), k1, k2);
                }
            }
            // end of this CTA's part of query block qb: merge the two column
            // halves, then the CTAs' parts (last arriver), and write; on an
            // abort every epilogue warp leaves here together
            if (!owner)
                half_keys[row] = make_uint2(k1, k2);
            if (epi_sync_or(*(volatile int *)&abort_flag != 0))
                break;
            if (owner)
                top2_merge(half_keys[row].x, half_keys[row].y, k1, k2);
            const int query = qb * BM + row;
            const int first = cta_of((long long)qb * ntl, T, G);
            const int last = cta_of((long long)(qb + 1) * ntl - 1, T, G);
            if (first == last) {
                if (owner && query < nq) {
                    if (raw_keys)
                        raw_keys[query] = make_uint2(k1, k2);
                    else
                        finalize(k1, k2, nbits, rnum, rden, out + query);
                }
            } else {
                uint2 *slots = partial + (size_t)(first + qb) * BM;
                if (owner)
                    slots[(size_t)(c - first) * BM + row] = make_uint2(k1, k2);
                __threadfence();
                epi_sync();
                if (t == 128) {
                    const unsigned int prev = atomicAdd(arrivals + qb, 1u);
                    last_cta = prev == (unsigned)(last - first);
                    if (last_cta)
                        arrivals[qb] = 0u;
                }
                epi_sync();
                if (last_cta && owner && query < nq) {
                    __threadfence();
                    uint2 a = __ldcg(slots + row);
                    for (int sl = 1; sl <= last - first; ++sl) {
                        const uint2 b = __ldcg(slots + (size_t)sl * BM + row);
                        top2_merge(b.x, b.y, a.x, a.y);
                    }
                    if (raw_keys)
                        raw_keys[query] = a;
                    else
                        finalize(a.x, a.y, nbits, rnum, rden, out + query);
                }
            }
            epi_sync();  // half_keys and last_cta are reused by the next block
        }
    }
    __syncthreads();
    const bool aborted = abort_flag != 0;
    if (aborted && t == 0)
        dev::raise_flag(status, BD_FLAG_TIMEOUT);
    if (aborted && warp == 1 && lane == 0) {
        // let issued MMAs finish before TMEM is released
        for (int i = 0; i < issued; ++i) {
            uint64_t *b = &bar_tf[i & 1];
            const unsigned long long t0 = gtime();
            while (!dev::mbar_try_wait(b, (i >> 1) & 1) && gtime() - t0 < kWaitNs) {
            }
        }
    }
    dev::tc_fence_before();
    __syncthreads();
    if (warp == 0)
        dev::tmem_dealloc(tmem, 2 * BN);
}

// Persistent grid: as many CTAs as are resident (two per SM at K = 256, one
// at K = 512), at most one per (query block, train tile) pair.
int tc_grid(int nq, int nt, int nbits, int sm_count)
{
    const long long T = (long long)((nq + BM - 1) / BM) * (long long)std::max(1, (nt + BN - 1) / BN);
    const long long g = (long long)(nbits == 256 ? 2 : 1) * sm_count;
    return (int)std::max(1LL, std::min(T, g));
}

}  // namespace

int match_tc_query_blocks(int nq) { return (nq + BM - 1) / BM; }

size_t match_tc_scratch_bytes(int nq, int nt, int nbits, int sm_count)
{
    const int G = tc_grid(nq, nt, nbits, sm_count);
    return align_up((size_t)nq * nbits, 256) + align_up((size_t)(nt > 0 ? nt : 1) * nbits, 256) +
           align_up((size_t)(G + match_tc_query_blocks(nq)) * BM * sizeof(uint2), 256);
}

cudaError_t launch_match_tc_keys(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                                 int nbits, int ratio_num, int ratio_den, bd_match_result *out,
                                 uint2 *raw_keys, void *scratch, cudaStream_t st,
                                 unsigned int *arrivals, int mine)
{
    const int sm_count = ctx->sm_count;
    const int G = tc_grid(nq, nt, nbits, sm_count);
    uint8_t *qx = (uint8_t *)scratch;
    uint8_t *tx = qx + align_up((size_t)nq * nbits, 256);
    uint2 *partial = (uint2 *)(tx + align_up((size_t)(nt > 0 ? nt : 1) * nbits, 256));
    const size_t qw = (size_t)nq * (nbits / 32), tw = (size_t)nt * (nbits / 32);
    const size_t ew = qw + tw;
    cudaError_t e = launch_pdl(expand_pm1_kernel,
                               dim3((unsigned)((ew + 255) / 256 < 4096 ? (ew + 255) / 256 : 4096)),
                               dim3(256), 0, st, q, qw, reinterpret_cast<uint4 *>(qx),
                               nt > 0 ? t : q, tw, reinterpret_cast<uint4 *>(tx));
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "expand_pm1");
    CUtensorMap tmQ, tmT;
    if (!encode_tmap_2d_u8(&tmQ, qx, (uint64_t)nbits, (uint64_t)nq, (uint64_t)nbits, 128, 128) ||
        !encode_tmap_2d_u8(&tmT, tx, (uint64_t)nbits, (uint64_t)(nt > 0 ? nt : 1), (uint64_t)nbits,
                           128, 128))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)(BM + 2 * BN) * nbits + 1024;
    auto kern = mine ? (nbits == 256 ? match_tc_kernel<256, 2, true> : match_tc_kernel<512, 1, true>)
                     : (nbits == 256 ? match_tc_kernel<256, 2, false> : match_tc_kernel<512, 1, false>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    e = launch_pdl(kern, dim3(G), dim3(NTHREADS), smem, st, tmQ, tmT, nq, nt, nbits, ratio_num,
                   ratio_den, partial, out, raw_keys, arrivals, ctx->status);
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "match_tc");
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_match_tc(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                            int nbits, int ratio_num, int ratio_den, bd_match_result *out,
                            void *scratch, cudaStream_t st, unsigned int *arrivals)
{
    return launch_match_tc_keys(ctx, q, nq, t, nt, nbits, ratio_num, ratio_den, out, nullptr,
                                scratch, st, arrivals, 0);
}

}  // namespace bd
