// One round of BAD feature selection (Algorithm 1) with the threshold search
// of Algorithm 2 in its integer-sorted form (Sec. III-A: thresholds on a 0.1
// grid over [-255, 255], 5102 values).
//
//  0. select_geom_kernel: per candidate box pair, the eight summed-area-table
//     offsets of the two boxes' corners (clamped to the patch), s^2 and
//     1/s^2, once per call (they do not depend on the patch).
//  1. select_keys_kernel: 16 patches per CTA, each patch's summed-area table
//     in shared memory (rows from 16-byte loads, prefix sums along rows, then
//     down columns); for every candidate box pair j it writes the exact key
//     ceil(10 (sum1 - sum2) / s^2) of every patch, candidate-major
//     (keys[j][patch], int16), so that step 2 reads them coalesced.  The
//     division is a reciprocal estimate corrected by one integer step each
//     way, which makes it exact.
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
constexpr int SAT = 33;                  // summed-area table row length (entries)

struct SelectState {
    unsigned long long best_key;
    unsigned int arrived;
};

// Corner offsets of candidate j: box b's table entries (ya, xa), (ya, xb),
// (yb, xa), (yb, xb) at off[4 b + 0..3]; sum = T[3] - T[1] - T[2] + T[0].
struct CandGeom {
    uint16_t off[8];
    int den;       // s^2
    float inv;     // 1 / s^2 (rounded)
    int pad[2];
};
static_assert(sizeof(CandGeom) == 32, "two 16-byte loads per candidate");

__global__ void select_geom_kernel(const int4 *__restrict__ cand, const int *__restrict__ side,
                                   int J, CandGeom *__restrict__ geom)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J)
        return;
    const int4 c = __ldg(cand + j);
    const int s = min(max(__ldg(side + j), 1), 32);  // validated on the host
    CandGeom g;
    const int cx[2] = {c.x, c.z}, cy[2] = {c.y, c.w};
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int xa = min(max(cx[b] - s / 2, 0), 32), xb = min(max(cx[b] - s / 2 + s, 0), 32);
        const int ya = min(max(cy[b] - s / 2, 0), 32), yb = min(max(cy[b] - s / 2 + s, 0), 32);
        g.off[4 * b + 0] = (uint16_t)(ya * SAT + xa);
        g.off[4 * b + 1] = (uint16_t)(ya * SAT + xb);
        g.off[4 * b + 2] = (uint16_t)(yb * SAT + xa);
        g.off[4 * b + 3] = (uint16_t)(yb * SAT + xb);
    }
    g.den = s * s;
    g.inv = 1.0f / (float)(s * s);
    g.pad[0] = g.pad[1] = 0;
    geom[j] = g;
}

__global__ void __launch_bounds__(256) select_keys_kernel(const uint8_t *__restrict__ patches,
                                                          int rows, const CandGeom *__restrict__ geom,
                                                          int j0, int jn, int16_t *__restrict__ keys,
                                                          SelectState *state, int init)
{
    __shared__ uint32_t sat[SK_PATCHES][SAT * SAT];
    const int t = threadIdx.x;
    const int p0 = blockIdx.x * SK_PATCHES;
    if (init && blockIdx.x == 0 && t == 0) {
        state->best_key = ~0ull;
        state->arrived = 0u;
    }
    // summed-area tables: thread (patch t/16, rows t%16 and t%16 + 16) loads
    // its two 32-byte rows with 16-byte loads and writes their prefix sums
    {
        const int pi = t >> 4, r0 = t & 15;
        uint32_t *S = sat[pi];
        const bool in = p0 + pi < rows;
        const uint4 *src = reinterpret_cast<const uint4 *>(patches + (size_t)(p0 + pi) * 1024);
        uint4 v[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            v[2 * h] = in ? __ldg(src + 2 * (r0 + 16 * h)) : make_uint4(0u, 0u, 0u, 0u);
            v[2 * h + 1] = in ? __ldg(src + 2 * (r0 + 16 * h) + 1) : make_uint4(0u, 0u, 0u, 0u);
        }
        if (r0 == 0)
            for (int x = 0; x <= 32; ++x)
                S[x] = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int y = r0 + 16 * h;
            uint32_t *R = S + (y + 1) * SAT;
            const uint32_t w[8] = {v[2 * h].x, v[2 * h].y, v[2 * h].z, v[2 * h].w,
                                   v[2 * h + 1].x, v[2 * h + 1].y, v[2 * h + 1].z, v[2 * h + 1].w};
            uint32_t acc = 0;
            R[0] = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    acc += (w[q] >> (8 * bb)) & 0xFFu;
                    R[4 * q + bb + 1] = acc;
                }
        }
        __syncthreads();
        // column sums down the table
        for (int x = r0; x <= 32; x += 16) {
            uint32_t acc = 0;
            for (int y = 1; y <= 32; ++y) {
                acc += S[y * SAT + x];
                S[y * SAT + x] = acc;
            }
        }
    }
    __syncthreads();
    // keys: thread (patch t%16, candidate t/16 + 16 k)
    const int pi = t & 15, jj = t >> 4;
    const int p = p0 + pi;
    const uint32_t *S = sat[pi];
    const uint4 *gq = reinterpret_cast<const uint4 *>(geom + j0);
#pragma unroll 2
    for (int j = jj; j < jn; j += 16) {
        const uint4 ga = __ldg(gq + 2 * j), gb = __ldg(gq + 2 * j + 1);
        const uint32_t o[4] = {ga.x, ga.y, ga.z, ga.w};  // two 16-bit offsets each
        uint32_t T[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T[2 * q] = S[o[q] & 0xFFFFu];
            T[2 * q + 1] = S[o[q] >> 16];
        }
        const int s1 = (int)(T[3] - T[1] - T[2] + T[0]);
        const int s2 = (int)(T[7] - T[5] - T[6] + T[4]);
        const int num = 10 * (s1 - s2);
        const int den = (int)gb.x;
        // ceil(num / den) exactly: |num| < 2^22, so the reciprocal estimate is
        // within one of it, and one integer step each way settles it
        int q = __float2int_ru((float)num * __uint_as_float(gb.y));
        q += q * den < num ? 1 : 0;
        q -= (q - 1) * den >= num ? 1 : 0;
        if (p < rows)
            keys[(size_t)j * rows + p] = (int16_t)q;
    }
}

// The same keys from 16-bit tables for candidates of side <= 16: a box sum is
// then below 2^16, so tables kept mod 2^16 give it exactly.  32 patches per
// CTA in the same shared memory; warp w takes candidates w, w + 8, ... for
// its 32 patches, one per lane, so the eight table reads of a key fall on 32
// distinct banks (patch tables 545 words apart) and the key stores are 64-byte
// runs.
constexpr int SK16_PATCHES = 32;
constexpr int SAT16 = 1090;  // halfwords per patch table (33 x 33, padded)

__global__ void __launch_bounds__(256) select_keys16_kernel(const uint8_t *__restrict__ patches,
                                                            int rows,
                                                            const CandGeom *__restrict__ geom,
                                                            int j0, int jn,
                                                            int16_t *__restrict__ keys,
                                                            SelectState *state, int init)
{
    __shared__ uint16_t sat[SK16_PATCHES * SAT16];
    const int t = threadIdx.x;
    const int p0 = blockIdx.x * SK16_PATCHES;
    if (init && blockIdx.x == 0 && t == 0) {
        state->best_key = ~0ull;
        state->arrived = 0u;
    }
    // row prefix sums: thread (patch t/8, rows t%8 + 8 h), 16-byte loads
    {
        const int pi = t >> 3, r0 = t & 7;
        uint16_t *S = sat + pi * SAT16;
        const bool in = p0 + pi < rows;
        const uint4 *src = reinterpret_cast<const uint4 *>(patches + (size_t)(p0 + pi) * 1024);
        uint4 v[8];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            v[2 * h] = in ? __ldg(src + 2 * (r0 + 8 * h)) : make_uint4(0u, 0u, 0u, 0u);
            v[2 * h + 1] = in ? __ldg(src + 2 * (r0 + 8 * h) + 1) : make_uint4(0u, 0u, 0u, 0u);
        }
        if (r0 == 0)
            for (int x = 0; x <= 32; ++x)
                S[x] = 0;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint16_t *R = S + (r0 + 8 * h + 1) * SAT;
            const uint32_t w[8] = {v[2 * h].x, v[2 * h].y, v[2 * h].z, v[2 * h].w,
                                   v[2 * h + 1].x, v[2 * h + 1].y, v[2 * h + 1].z, v[2 * h + 1].w};
            uint32_t acc = 0;
            R[0] = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    acc += (w[q] >> (8 * bb)) & 0xFFu;
                    R[4 * q + bb + 1] = (uint16_t)acc;
                }
        }
    }
    __syncthreads();
    // column sums: each thread one (patch, column), the 32 entries in registers
    for (int c = t; c < SK16_PATCHES * SAT; c += 256) {
        uint16_t *S = sat + (c / SAT) * SAT16 + c % SAT;
        uint32_t v[32];
#pragma unroll
        for (int y = 0; y < 32; ++y)
            v[y] = S[(y + 1) * SAT];
        uint32_t acc = 0;
#pragma unroll
        for (int y = 0; y < 32; ++y) {
            acc += v[y];
            S[(y + 1) * SAT] = (uint16_t)acc;
        }
    }
    __syncthreads();
    const int lane = t & 31, w = t >> 5;
    const int p = p0 + lane;
    const uint16_t *S = sat + lane * SAT16;
    const uint4 *gq = reinterpret_cast<const uint4 *>(geom + j0);
#pragma unroll 2
    for (int j = w; j < jn; j += 8) {
        const uint4 ga = __ldg(gq + 2 * j), gb = __ldg(gq + 2 * j + 1);
        const uint32_t o[4] = {ga.x, ga.y, ga.z, ga.w};
        uint32_t T[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T[2 * q] = S[o[q] & 0xFFFFu];
            T[2 * q + 1] = S[o[q] >> 16];
        }
        const int s1 = (int)((T[3] - T[1] - T[2] + T[0]) & 0xFFFFu);
        const int s2 = (int)((T[7] - T[5] - T[6] + T[4]) & 0xFFFFu);
        const int num = 10 * (s1 - s2);
        const int den = (int)gb.x;
        int q = __float2int_ru((float)num * __uint_as_float(gb.y));
        q += q * den < num ? 1 : 0;
        q -= (q - 1) * den >= num ? 1 : 0;
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
    auto triplet = [&](int k0, int k1, int k2, int a, int c) {
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
    };
    if ((n & 3) == 0) {
        // four triplets per iteration: 8-byte key loads, 16-byte similarity loads
        const short4 *k04 = reinterpret_cast<const short4 *>(kj);
        const short4 *k14 = reinterpret_cast<const short4 *>(kj + n);
        const short4 *k24 = reinterpret_cast<const short4 *>(kj + 2 * n);
        const int4 *a4 = reinterpret_cast<const int4 *>(sap), *c4 = reinterpret_cast<const int4 *>(san);
        for (int i = t; i < (n >> 2); i += ST_THREADS) {
            const short4 x = __ldg(k04 + i), y = __ldg(k14 + i), z = __ldg(k24 + i);
            const int4 a = __ldg(a4 + i), c = __ldg(c4 + i);
            triplet(x.x, y.x, z.x, a.x, c.x);
            triplet(x.y, y.y, z.y, a.y, c.y);
            triplet(x.z, y.z, z.z, a.z, c.z);
            triplet(x.w, y.w, z.w, a.w, c.w);
        }
    } else {
        for (int i = t; i < n; i += ST_THREADS)
            triplet(kj[i], kj[n + i], kj[2 * n + i], __ldg(sap + i), __ldg(san + i));
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

// Scratch for J candidates whose keys are made jn at a time (jn <= J).
size_t select_scratch_bytes_pass(int n, int J, int jn)
{
    return align_up(sizeof(SelectState), 256) + align_up((size_t)J * sizeof(CandGeom), 256) +
           align_up((size_t)jn * 3 * n * 2, 256);
}

size_t select_scratch_bytes(int n, int J) { return select_scratch_bytes_pass(n, J, J); }

cudaError_t launch_select_feature(const uint8_t *patches, int n, const int32_t *sap,
                                  const int32_t *san, int tau, const int32_t *cand_xy,
                                  const int32_t *cand_side, int max_side, int J, int32_t *theta_q,
                                  int64_t *loss, int32_t *best, void *scratch, size_t scratch_bytes,
                                  cudaStream_t st)
{
    SelectState *state = (SelectState *)scratch;
    const size_t head = align_up(sizeof(SelectState), 256);
    CandGeom *geom = (CandGeom *)((char *)scratch + head);
    const size_t head2 = head + align_up((size_t)J * sizeof(CandGeom), 256);
    int16_t *keys = (int16_t *)((char *)scratch + head2);
    const int rows = 3 * n;
    // candidates per pass: as many as the scratch area holds
    const size_t per = (size_t)rows * 2;
    if (scratch_bytes <= head2)
        return cudaErrorInvalidValue;
    long long cap = (long long)((scratch_bytes - head2) / per);
    if (cap < 1)
        return cudaErrorInvalidValue;
    select_geom_kernel<<<(J + 127) / 128, 128, 0, st>>>(reinterpret_cast<const int4 *>(cand_xy),
                                                        cand_side, J, geom);
    trace_kernel(st, "select_geom");
    note_launches(1);
    for (int j0 = 0; j0 < J; j0 += (int)cap) {
        const int jn = (int)((long long)(J - j0) < cap ? J - j0 : cap);
        if (max_side <= 16)
            select_keys16_kernel<<<(rows + SK16_PATCHES - 1) / SK16_PATCHES, 256, 0, st>>>(
                patches, rows, geom, j0, jn, keys, state, j0 == 0 ? 1 : 0);
        else
            select_keys_kernel<<<(rows + SK_PATCHES - 1) / SK_PATCHES, 256, 0, st>>>(
                patches, rows, geom, j0, jn, keys, state, j0 == 0 ? 1 : 0);
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
