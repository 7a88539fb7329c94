// Brute-force Hamming matching body (Sec. IV-C nearest-neighbour matching,
// Sec. III-A: S = K - 2 * Hamming for +-1 codes), shared by the matching
// kernels (match.cu) and the batched persistent kernel (batch.cu).
//
// A CTA of QB threads holds QB query descriptors, one per thread, in
// registers and streams a slice of the train set through shared memory in
// tiles of TT descriptors (every lane reads the same train descriptor: a
// broadcast).  Per query it keeps the two smallest packed keys
// (distance << 22 | train index): comparing keys orders by distance, then by
// lowest index, so the first key gives the nearest neighbour and the second
// key's distance is d2.  When the train set is split into S slices, each CTA
// publishes its per-slice top-2 pair and the last CTA of a query block
// (per-block arrival counter, reset by that CTA) merges them.
#pragma once

#include "bd_internal.h"

namespace bd {
namespace dev {

__device__ __forceinline__ void top2_push(uint32_t key, uint32_t &k1, uint32_t &k2)
{
    k2 = min(k2, max(k1, key));
    k1 = min(k1, key);
}

// The two smallest of two (smallest, second smallest) pairs.
__device__ __forceinline__ uint2 top2_merge(uint2 a, uint2 b)
{
    return make_uint2(min(a.x, b.x), min(max(a.x, b.x), min(a.y, b.y)));
}

// Merge of the S slice pairs of query qi (eight loads in flight at a time).
__device__ __forceinline__ uint2 merge_slices(const uint2 *__restrict__ partial, int nq, int qi,
                                              int S)
{
    uint2 a = __ldcg(partial + qi);
    int s = 1;
    for (; s + 8 <= S; s += 8) {
        uint2 b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            b[u] = __ldcg(partial + (size_t)(s + u) * nq + qi);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            a = top2_merge(a, b[u]);
    }
    for (; s < S; ++s)
        a = top2_merge(a, __ldcg(partial + (size_t)s * nq + qi));
    return a;
}

__device__ __forceinline__ void match_finalize(uint32_t k1, uint32_t k2, int nbits, int rnum,
                                               int rden, bd_match_result *o)
{
    const uint32_t d1 = k1 >> kMatchIdxBits, d2 = k2 >> kMatchIdxBits;
    const int32_t idx = (d1 > (uint32_t)nbits) ? -1 : (int32_t)(k1 & kMatchIdxMask);
    const uint32_t acc = ((long long)rden * d1 < (long long)rnum * d2) ? 1u : 0u;
    uint32_t *w = reinterpret_cast<uint32_t *>(o);
    w[0] = (uint32_t)idx;
    w[1] = d1 | (d2 << 16);
    w[2] = acc;
}

// Queries [bx QB, bx QB + QB) against train slice `by` of S (chunk entries
// each).  tile: TT * NW / 4 uint4 of shared memory.  Called by all QB
// threads; last_cta is a shared int.
template <int NW, int QB, int TT>
__device__ __forceinline__ void match_block(uint4 *tile, const uint32_t *__restrict__ q, int nq,
                                            const uint32_t *__restrict__ t, int nt, int chunk,
                                            int nbits, int rnum, int rden, int bx, int by, int S,
                                            uint2 *__restrict__ partial,
                                            bd_match_result *__restrict__ out,
                                            unsigned int *__restrict__ arrivals, int &last_cta)
{
    const int qi = bx * QB + (int)threadIdx.x;
    const int t0 = by * chunk;
    const int t1 = min(nt, t0 + chunk);

    // query descriptors may come from this launch (persistent kernel): L2 reads
    uint32_t qd[NW];
    if (qi < nq) {
        const uint4 *src = reinterpret_cast<const uint4 *>(q + (size_t)qi * NW);
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) {
            const uint4 x = __ldcg(src + v);
            qd[4 * v + 0] = x.x;
            qd[4 * v + 1] = x.y;
            qd[4 * v + 2] = x.z;
            qd[4 * v + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int v = 0; v < NW; ++v)
            qd[v] = 0;
    }
    const uint32_t sentinel = ((uint32_t)(nbits + 1) << kMatchIdxBits) | kMatchIdxMask;
    uint32_t k1 = sentinel, k2 = sentinel;

    for (int base = t0; base < t1; base += TT) {
        const int cnt = min(TT, t1 - base);
        __syncthreads();
        const uint4 *src = reinterpret_cast<const uint4 *>(t + (size_t)base * NW);
        for (int v = threadIdx.x; v < cnt * NW / 4; v += QB)
            tile[v] = __ldcg(src + v);
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
            uint32_t d = 0;
#pragma unroll
            for (int v = 0; v < NW / 4; ++v) {
                const uint4 x = tile[j * (NW / 4) + v];
                d += __popc(qd[4 * v + 0] ^ x.x) + __popc(qd[4 * v + 1] ^ x.y) +
                     __popc(qd[4 * v + 2] ^ x.z) + __popc(qd[4 * v + 3] ^ x.w);
            }
            top2_push((d << kMatchIdxBits) | (uint32_t)(base + j), k1, k2);
        }
    }
    if (S == 1) {
        if (qi < nq)
            match_finalize(k1, k2, nbits, rnum, rden, out + qi);
        return;
    }
    if (qi < nq)
        partial[(size_t)by * nq + qi] = make_uint2(k1, k2);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(arrivals + bx, 1u);
        last_cta = prev == (unsigned)S - 1;
        if (last_cta)
            arrivals[bx] = 0u;  // every slice has arrived: ready for the next call
    }
    __syncthreads();
    if (!last_cta || qi >= nq)
        return;
    __threadfence();
    // keys are unique, so the merge order does not matter
    const uint2 a = merge_slices(partial, nq, qi, S);
    match_finalize(a.x, a.y, nbits, rnum, rden, out + qi);
}

// A 128-thread CTA matches 32 queries [32 bx, 32 bx + 32) (one per lane)
// against train slice `by` of S: the slice is staged in shared memory TT
// descriptors at a time and warp w scans its entries w, w + 4, ...; the four
// warps' pairs are merged in shared memory, and with S > 1 the last CTA of the
// query block merges the slices.  Short chains for small problems (the
// batched kernel's matching items).  tile: TT * NW / 4 uint4; wpair: 128 uint2.
template <int NW, int TT>
__device__ __forceinline__ void match_block32(uint4 *tile, uint2 *wpair,
                                              const uint32_t *__restrict__ q, int nq,
                                              const uint32_t *__restrict__ t, int nt, int chunk,
                                              int nbits, int rnum, int rden, int bx, int by, int S,
                                              uint2 *__restrict__ partial,
                                              bd_match_result *__restrict__ out,
                                              unsigned int *__restrict__ arrivals, int &last_cta)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int qi = bx * 32 + lane;
    const int t0 = by * chunk;
    const int t1 = min(nt, t0 + chunk);
    uint32_t qd[NW];
    if (qi < nq) {
        const uint4 *src = reinterpret_cast<const uint4 *>(q + (size_t)qi * NW);
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) {
            const uint4 x = __ldcg(src + v);
            qd[4 * v + 0] = x.x;
            qd[4 * v + 1] = x.y;
            qd[4 * v + 2] = x.z;
            qd[4 * v + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int v = 0; v < NW; ++v)
            qd[v] = 0;
    }
    const uint32_t sentinel = ((uint32_t)(nbits + 1) << kMatchIdxBits) | kMatchIdxMask;
    uint32_t k1 = sentinel, k2 = sentinel;
    for (int base = t0; base < t1; base += TT) {
        const int cnt = min(TT, t1 - base);
        __syncthreads();
        const uint4 *src = reinterpret_cast<const uint4 *>(t + (size_t)base * NW);
        for (int v = threadIdx.x; v < cnt * NW / 4; v += 128)
            tile[v] = __ldcg(src + v);
        __syncthreads();
#pragma unroll 2
        for (int j = w; j < cnt; j += 4) {
            uint32_t d = 0;
#pragma unroll
            for (int v = 0; v < NW / 4; ++v) {
                const uint4 x = tile[j * (NW / 4) + v];
                d += __popc(qd[4 * v + 0] ^ x.x) + __popc(qd[4 * v + 1] ^ x.y) +
                     __popc(qd[4 * v + 2] ^ x.z) + __popc(qd[4 * v + 3] ^ x.w);
            }
            top2_push((d << kMatchIdxBits) | (uint32_t)(base + j), k1, k2);
        }
    }
    wpair[threadIdx.x] = make_uint2(k1, k2);
    __syncthreads();
    uint2 a = make_uint2(sentinel, sentinel);
    if (w == 0) {
        a = top2_merge(top2_merge(wpair[lane], wpair[32 + lane]),
                       top2_merge(wpair[64 + lane], wpair[96 + lane]));
        if (S == 1 && qi < nq)
            match_finalize(a.x, a.y, nbits, rnum, rden, out + qi);
        if (S > 1 && qi < nq)
            partial[(size_t)by * nq + qi] = a;
    }
    if (S == 1)
        return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(arrivals + bx, 1u);
        last_cta = prev == (unsigned)S - 1;
        if (last_cta)
            arrivals[bx] = 0u;  // every slice has arrived: ready for the next call
    }
    __syncthreads();
    if (!last_cta || w != 0 || qi >= nq)
        return;
    __threadfence();
    a = merge_slices(partial, nq, qi, S);
    match_finalize(a.x, a.y, nbits, rnum, rden, out + qi);
}

}  // namespace dev
}  // namespace bd
