// One round of BAD feature selection (Algorithm 1) with the threshold search
// of Algorithm 2 in its integer-sorted form (Sec. III-A: thresholds on a 0.1
// grid over [-255, 255], 5102 values).
//
//  1. select_keys_kernel: 16 patches per CTA, each patch's summed-area table
//     in shared memory; for every candidate box pair j it writes the exact
//     key ceil(10 (sum1 - sum2) / s^2) of every patch, candidate-major
//     (keys[j][patch], int16), so that step 2 reads them coalesced.
//  2. select_threshold_kernel: one CTA per candidate.  Each triplet adds the
//     changes of its per-step loss term at its distinct keys into a 5102-bin
//     shared-memory histogram (integer, exact) and its term at the lowest
//     threshold into the base loss; a block-wide scan then gives the loss at
//     every threshold and the first minimum.  The best candidate is kept as
//     one 64-bit key (loss << 20 | j) with atomicMin; the last CTA to finish
//     writes its index.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int kQMin = BD_SELECT_QMIN;   // threshold numerator with h = -1 everywhere
constexpr int kBins = 2550 - kQMin + 1;  // thresholds q in [kQMin, 2550]
constexpr int SK_PATCHES = 16;           // patches per CTA of the key kernel
constexpr int ST_THREADS = 256;

struct SelectState {
    unsigned long long best_key;
    unsigned int arrived;
};

__global__ void __launch_bounds__(256) select_keys_kernel(const uint8_t *__restrict__ patches,
                                                          int rows, const int4 *__restrict__ cand,
                                                          const int *__restrict__ side, int j0,
                                                          int jn, int16_t *__restrict__ keys,
                                                          SelectState *state, int init)
{
    __shared__ uint32_t sat[SK_PATCHES][33 * 33];
    const int t = threadIdx.x;
    const int p0 = blockIdx.x * SK_PATCHES;
    if (init && blockIdx.x == 0 && t == 0) {
        state->best_key = ~0ull;
        state->arrived = 0u;
    }
    // summed-area tables: thread (patch t/16, row band t%16) builds rows by prefix sums
    {
        const int pi = t >> 4, lane16 = t & 15;
        uint32_t *S = sat[pi];
        const bool in = p0 + pi < rows;
        const uint8_t *src = patches + (size_t)(p0 + pi) * 1024;
        if (lane16 == 0)
            for (int x = 0; x <= 32; ++x)
                S[x] = 0u;
        // row y + 1 of the table = row y prefix sums (two rows per thread)
        for (int y = lane16; y < 32; y += 16) {
            uint32_t acc = 0;
            S[(y + 1) * 33] = 0u;
            for (int x = 0; x < 32; ++x) {
                acc += in ? (uint32_t)__ldg(src + y * 32 + x) : 0u;
                S[(y + 1) * 33 + x + 1] = acc;
            }
        }
        __syncthreads();
        // column sums down the table
        for (int x = lane16; x <= 32; x += 16) {
            uint32_t acc = 0;
            for (int y = 1; y <= 32; ++y) {
                acc += S[y * 33 + x];
                S[y * 33 + x] = acc;
            }
        }
    }
    __syncthreads();
    // keys: thread (patch t%16, candidate t/16 + 16 k)
    const int pi = t & 15, jj = t >> 4;
    const int p = p0 + pi;
    const uint32_t *S = sat[pi];
    for (int j = jj; j < jn; j += 16) {
        const int4 c = __ldg(cand + j0 + j);
        const int s = min(max(__ldg(side + j0 + j), 1), 32);  // validated on the host
        auto box = [&](int cx, int cy) -> int {
            const int xa = min(max(cx - s / 2, 0), 32), xb = min(max(cx - s / 2 + s, 0), 32);
            const int ya = min(max(cy - s / 2, 0), 32), yb = min(max(cy - s / 2 + s, 0), 32);
            return (int)(S[yb * 33 + xb] - S[ya * 33 + xb] - S[yb * 33 + xa] + S[ya * 33 + xa]);
        };
        const int num = 10 * (box(c.x, c.y) - box(c.z, c.w));
        const int den = s * s;
        // ceil(num / den) exactly: a float estimate, then integer corrections
        int q = __float2int_ru(__fdiv_rn((float)num, (float)den));
        q = min(max(q, -4096), 4096);  // |num / den| <= 2550
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            q += q * den < num ? 1 : 0;
            q -= (q - 1) * den >= num ? 1 : 0;
        }
        if (p < rows)
            keys[(size_t)j * rows + p] = (int16_t)q;
    }
}

__device__ __forceinline__ int sel_term(int tau, int sap, int san, int ha, int hp, int hn)
{
    const int v = tau - sap - ha * hp + san + ha * hn;
    return v > 0 ? v : 0;
}

__global__ void __launch_bounds__(ST_THREADS) select_threshold_kernel(
    const int16_t *__restrict__ keys, int n, const int *__restrict__ sap,
    const int *__restrict__ san, int tau, int j0, int32_t *__restrict__ theta_q,
    long long *__restrict__ loss, int32_t *__restrict__ best, int J, SelectState *state)
{
    __shared__ int hist[kBins];
    __shared__ long long red[ST_THREADS / 32];
    __shared__ long long wmin[ST_THREADS / 32];
    __shared__ int widx[ST_THREADS / 32];
    __shared__ long long chunk_pre[ST_THREADS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int j = j0 + blockIdx.x;
    const int16_t *kj = keys + (size_t)blockIdx.x * 3 * n;
    for (int b = t; b < kBins; b += ST_THREADS)
        hist[b] = 0;
    __syncthreads();
    long long base = 0;
    for (int i = t; i < n; i += ST_THREADS) {
        const int k0 = kj[i], k1 = kj[n + i], k2 = kj[2 * n + i];
        const int a = __ldg(sap + i), c = __ldg(san + i);
        base += sel_term(tau, a, c, -1, -1, -1);
        const int k[3] = {k0, k1, k2};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            bool dup = false;
#pragma unroll
            for (int q = 0; q < m; ++q)
                dup |= k[q] == k[m];
            if (dup)
                continue;
            const int key = k[m];
            const int at = sel_term(tau, a, c, k0 <= key ? 1 : -1, k1 <= key ? 1 : -1,
                                    k2 <= key ? 1 : -1);
            const int below = sel_term(tau, a, c, k0 < key ? 1 : -1, k1 < key ? 1 : -1,
                                       k2 < key ? 1 : -1);
            if (at != below)
                atomicAdd(&hist[key - kQMin], at - below);
        }
    }
    // base loss: block sum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        base += __shfl_xor_sync(0xffffffffu, base, o);
    if (lane == 0)
        red[warp] = base;
    __syncthreads();
    long long L0 = 0;
#pragma unroll
    for (int w = 0; w < ST_THREADS / 32; ++w)
        L0 += red[w];
    // loss at threshold kQMin + b = L0 + prefix sum of hist[0..b]: contiguous
    // chunks per thread, chunk totals scanned across the block
    constexpr int CH = (kBins + ST_THREADS - 1) / ST_THREADS;
    const int b0 = t * CH, b1 = min(kBins, b0 + CH);
    long long tot = 0;
    for (int b = b0; b < b1; ++b)
        tot += hist[b];
    chunk_pre[t] = tot;
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 256 chunk totals by one warp
        long long run = 0;
        for (int base_i = 0; base_i < ST_THREADS; base_i += 32) {
            long long v = chunk_pre[base_i + lane];
            long long incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += u;
            }
            chunk_pre[base_i + lane] = run + incl - v;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    long long cur = L0 + chunk_pre[t];
    long long mv = 0x7fffffffffffffffLL;
    int mi = kBins;
    for (int b = b0; b < b1; ++b) {
        cur += hist[b];
        if (cur < mv) {
            mv = cur;
            mi = b;
        }
    }
    // first minimum over the block: smaller loss, then smaller threshold
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, mv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
        if (ov < mv || (ov == mv && oi < mi)) {
            mv = ov;
            mi = oi;
        }
    }
    if (lane == 0) {
        wmin[warp] = mv;
        widx[warp] = mi;
    }
    __syncthreads();
    if (t == 0) {
        long long bv = wmin[0];
        int bi = widx[0];
        for (int w = 1; w < ST_THREADS / 32; ++w)
            if (wmin[w] < bv || (wmin[w] == bv && widx[w] < bi)) {
                bv = wmin[w];
                bi = widx[w];
            }
        theta_q[j] = kQMin + bi;
        loss[j] = bv;
        atomicMin(&state->best_key, ((unsigned long long)bv << 20) | (unsigned long long)j);
        __threadfence();
        if (atomicAdd(&state->arrived, 1u) == (unsigned)J - 1) {
            __threadfence();
            const unsigned long long bk = atomicAdd(&state->best_key, 0ull);
            *best = (int32_t)(bk & 0xFFFFFu);
        }
    }
}

}  // namespace

size_t select_scratch_bytes(int n, int J)
{
    return align_up(sizeof(SelectState), 256) + align_up((size_t)J * 3 * n * 2, 256);
}

cudaError_t launch_select_feature(const uint8_t *patches, int n, const int32_t *sap,
                                  const int32_t *san, int tau, const int32_t *cand_xy,
                                  const int32_t *cand_side, int J, int32_t *theta_q,
                                  int64_t *loss, int32_t *best, void *scratch, size_t scratch_bytes,
                                  cudaStream_t st)
{
    SelectState *state = (SelectState *)scratch;
    int16_t *keys = (int16_t *)((char *)scratch + align_up(sizeof(SelectState), 256));
    const int rows = 3 * n;
    // candidates per pass: as many as the scratch area holds
    const size_t per = (size_t)rows * 2;
    long long cap = (long long)((scratch_bytes - align_up(sizeof(SelectState), 256)) / per);
    if (cap < 1)
        return cudaErrorInvalidValue;
    for (int j0 = 0; j0 < J; j0 += (int)cap) {
        const int jn = (int)((long long)(J - j0) < cap ? J - j0 : cap);
        select_keys_kernel<<<(rows + SK_PATCHES - 1) / SK_PATCHES, 256, 0, st>>>(
            patches, rows, reinterpret_cast<const int4 *>(cand_xy), cand_side, j0, jn, keys, state,
            j0 == 0 ? 1 : 0);
        trace_kernel(st, "select_keys");
        select_threshold_kernel<<<jn, ST_THREADS, 0, st>>>(keys, n, sap, san, tau, j0, theta_q,
                                                           reinterpret_cast<long long *>(loss),
                                                           best, J, state);
        trace_kernel(st, "select_threshold");
        note_launches(2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace bd
