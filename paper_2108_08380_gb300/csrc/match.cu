// Brute-force Hamming matching with a fused top-2 and ratio test (Sec. IV-C
// nearest-neighbour matching; Sec. III-A: S = K - 2 * Hamming for +-1 codes).
//
// Each thread keeps one query descriptor in registers; a CTA of 128 queries
// streams a slice of the train set through shared memory (all lanes read the
// same train descriptor, a broadcast) and keeps, per query, the two smallest
// packed keys (distance << 22 | train index).  Comparing packed keys orders
// by distance, then by lowest index, so the first key gives the nearest
// neighbour and the second key's distance is d2.  When the train set is split
// across CTAs, each CTA publishes its per-slice top-2 pairs and the last CTA of
// a query block (per-block arrival counter, reset by that CTA) merges them.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int QB = 128;   // queries per CTA (one per thread)
constexpr int TT = 256;   // train descriptors per shared-memory tile

__device__ __forceinline__ void top2_push(uint32_t key, uint32_t &k1, uint32_t &k2)
{
    k2 = min(k2, max(k1, key));
    k1 = min(k1, key);
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

template <int NW>
__global__ void __launch_bounds__(QB, 8) match_top2_kernel(const uint32_t *__restrict__ q, int nq,
                                                        const uint32_t *__restrict__ t, int nt,
                                                        int chunk, int nbits, int rnum, int rden,
                                                        uint2 *__restrict__ partial,
                                                        bd_match_result *__restrict__ out,
                                                        unsigned int *__restrict__ arrivals)
{
    __shared__ int last_cta;
    __shared__ uint4 tile[TT * NW / 4];
    const int qi = blockIdx.x * QB + threadIdx.x;
    const int t0 = blockIdx.y * chunk;
    const int t1 = min(nt, t0 + chunk);

    uint32_t qd[NW];
    if (qi < nq) {
        const uint4 *src = reinterpret_cast<const uint4 *>(q + (size_t)qi * NW);
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) {
            const uint4 x = __ldg(src + v);
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
            tile[v] = __ldg(src + v);
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
    if (gridDim.y == 1) {
        if (qi < nq)
            finalize(k1, k2, nbits, rnum, rden, out + qi);
        return;
    }
    if (qi < nq)
        partial[(size_t)blockIdx.y * nq + qi] = make_uint2(k1, k2);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(arrivals + blockIdx.x, 1u);
        last_cta = prev == gridDim.y - 1;
        if (last_cta)
            arrivals[blockIdx.x] = 0u;  // every slice has arrived: ready for the next call
    }
    __syncthreads();
    if (!last_cta || qi >= nq)
        return;
    __threadfence();
    uint2 a = __ldcg(partial + qi);
    for (int s = 1; s < (int)gridDim.y; ++s) {
        const uint2 b = __ldcg(partial + (size_t)s * nq + qi);
        const uint32_t m1 = min(a.x, b.x);
        const uint32_t m2 = min(max(a.x, b.x), min(a.y, b.y));
        a = make_uint2(m1, m2);
    }
    finalize(a.x, a.y, nbits, rnum, rden, out + qi);
}

void plan(int nq, int nt, int sm_count, int &S, int &chunk)
{
    const int qblocks = (nq + QB - 1) / QB;
    const int target = 8 * sm_count;
    S = (target + qblocks - 1) / qblocks;
    const int max_split = (nt + 31) / 32;
    if (S > max_split)
        S = max_split;
    if (S < 1)
        S = 1;
    chunk = (nt + S - 1) / S;
    if (chunk < 1)
        chunk = 1;
    S = (nt + chunk - 1) / chunk;
    if (S < 1)
        S = 1;
}

}  // namespace

size_t match_scratch_bytes(int nq, int nt, int nbits, int sm_count)
{
    (void)nbits;
    int S, chunk;
    plan(nq, nt, sm_count, S, chunk);
    return S > 1 ? align_up((size_t)S * nq * sizeof(uint2), 256) : 0;
}

int match_query_blocks(int nq) { return (nq + QB - 1) / QB; }

cudaError_t launch_match(const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits,
                         int ratio_num, int ratio_den, bd_match_result *out, void *scratch, int sm_count,
                         cudaStream_t st, unsigned int *arrivals)
{
    int S, chunk;
    plan(nq, nt, sm_count, S, chunk);
    dim3 grid((nq + QB - 1) / QB, S);
    uint2 *partial = (uint2 *)scratch;
    if (nbits == 256)
        match_top2_kernel<8><<<grid, QB, 0, st>>>(q, nq, t, nt, chunk, nbits, ratio_num, ratio_den,
                                                  partial, out, arrivals);
    else
        match_top2_kernel<16><<<grid, QB, 0, st>>>(q, nq, t, nt, chunk, nbits, ratio_num,
                                                   ratio_den, partial, out, arrivals);
    trace_kernel(st, "match_top2");
    note_launches(1);
    return cudaGetLastError();
}

namespace {

// Mutual check: query i keeps its nearest train entry j only if i is also
// the nearest query of j (both directions break ties to the lowest index).
__global__ void mnn_cross_kernel(const bd_match_result *__restrict__ fwd,
                                 const bd_match_result *__restrict__ rev, int nq,
                                 int32_t *__restrict__ mnn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq)
        return;
    const int j = fwd[i].idx;
    mnn[i] = (j >= 0 && rev[j].idx == i) ? j : -1;
}

}  // namespace

cudaError_t launch_mnn_cross(const bd_match_result *fwd, const bd_match_result *rev, int nq,
                             int32_t *mnn, cudaStream_t st)
{
    mnn_cross_kernel<<<(nq + 255) / 256, 256, 0, st>>>(fwd, rev, nq, mnn);
    trace_kernel(st, "mnn_cross");
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
