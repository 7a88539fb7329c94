// Differentiable training step for BAD and HashSIFT (Sec. III-A Eq. 1 and
// Sec. III-B Eq. 3) on 32x32 patches, with a hand-written backward.
//
// Rows of the patch tensor: [0,n) anchors, [n,2n) positives, [2n,3n) negatives.
//  forward
//   - one pass over the patches (one warp per patch): the HashSIFT
//     histogram, then the relaxed BAD responses;
//   - relaxed BAD: the warp builds the patch's summed-area table in 64-bit
//     fixed point (value x 2^32, exact for |v| >= 2^-9), so box sums are exact
//     integer sums and the hard bit [f <= theta] is the exact comparison
//     D <= floor(theta s^2 2^32); r = tanh((theta - f)/(255 T)) in FP32;
//   - relaxed HashSIFT: the histogram from that pass, then the projection on
//     the tensor cores (W split into BF16 head and tail each step; three
//     MMAs, margins within about 4e-6 of FP32 at these sizes) with
//     r = tanh((W^T h + b)/T) from those margins, and hard bits [m > 0] equal
//     to the FP32 projection's (the bits within the rescue band 2^-13 ||W_k||
//     are recomputed in FP32);
//   - mining on hard codes: for anchor i the negative j != i with the smallest
//     min(Hamming(a_i,n_j), Hamming(p_i,n_j)) (= the largest similarity
//     K - 2 Hamming, Sec. III-A), lowest j on ties, from two exact
//     tensor-core nearest-neighbour searches that leave column i out
//     (match_tc.cu, a maximum per score); anchor swap keeps p_i when it
//     is closer to that negative than a_i;
//   - the hinge loss of each descriptor.
//  backward (mining held fixed)
//   - dL/dr from the active hinges; a negative collects one term per triplet
//     that mined it.  Hard-negative mining makes hubs (one negative can be
//     the hardest of ten thousand anchors, its dL/dr a sum of that many terms
//     near +-1, which FP32 atomics round to 1e-3), so the negatives mined more
//     than kHubMin times (at most n / kHubMin of them) collect the responses
//     r in [-1, 1] as 64-bit fixed point (r 2^40, exact for |r| >= 2^-16: an
//     exact, order-independent sum, |sum| <= n <= 2^20 far from overflow)
//     with integer atomics in a compact per-hub accumulator (kHubRep copies
//     each, summed at the end), converted and scaled by the loss weight at
//     the end (which also clears it); the others keep FP32 atomics;
//   - BAD: dtheta column sums, and the box adjoint as a 2-D difference array
//     per patch (the corner updates that fall inside the patch, then 2-D
//     prefix sums);
//   - the column sums over all 3n rows (dtheta, db) cancel heavily (anchors
//     and positives pull one way, negatives the other), so each thread sums
//     its rows with compensated (Kahan) FP32 additions and the partial sums
//     meet in FP64 accumulators, converted to FP32 at the end;
//   - HashSIFT: dW = H^T dM and db (split over rows); dh = W dm and the
//     normalisation adjoint as a tiled product over patches; the histogram
//     adjoint per pixel (recomputed from the patch), gathered into the patch
//     gradient together with the BAD box adjoint.
#include "hashsift_dev.cuh"

using namespace bd;

struct bd_train {
    bd_ctx *ctx = nullptr;
    const bd_bad_params *bad = nullptr;
    int n = 0, rows = 0, kb = 0, kh = 0;
    float T = 0.1f, tau_bad = 0.f, tau_hs = 0.f;
    float *r_bad = nullptr, *r_hs = nullptr, *h = nullptr, *norm = nullptr;
    uint32_t *bits_bad = nullptr, *bits_hs = nullptr;
    int32_t *mining = nullptr;  // [4][n]
    float *dr_bad = nullptr, *dr_hs = nullptr, *Wt = nullptr;
    float *dH = nullptr;         // [rows][128] adjoint of the normalised histograms
    // the tcgen05 projection's view of this step's W and b: W^T in FP32 and
    // as BF16 head and tail (their TMA maps encoded once), the per-bit band
    bd_hs_params hp;
    double *loss_acc = nullptr;  // [2] losses, then [Kb] dtheta and [Kh] db accumulators
    int *hub = nullptr;            // [2][n] times mined (zero between steps), then hub index or -1
    int *n_hubs = nullptr;         // [2]
    int *hub_list = nullptr;       // [2][max_hubs] the hubs' negatives
    long long *hub_acc = nullptr;  // [2][max_hubs][kHubRep][Kmax]: hubs' sum of r x 2^40, zero between steps
    int max_hubs = 0;
    void *tc_scratch = nullptr;       // FP8 codes and partials of the top-2 searches
    uint2 *keys = nullptr;            // [2][n] top-2 keys (anchors, positives)
    unsigned int *arrivals = nullptr; // zeroed per-block arrival counters
};

namespace bd {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kHubMin = 64;  // a negative mined more often than this is a hub
// Copies of each hub's accumulator (anchor i adds into copy i mod kHubRep):
// the thousands of anchors of one hub would otherwise queue on the same
// addresses; the copies' integer sums add up exactly in any order.
constexpr int kHubRep = 16;

// 2^32 (the fixed-point scale of the BAD summed-area tables).
constexpr double kFix = 4294967296.0;

__device__ __forceinline__ long long sat_box64(const long long (*S)[33], int x0, int y0, int s)
{
    const int xa = min(max(x0, 0), 32), xb = min(max(x0 + s, 0), 32);
    const int ya = min(max(y0, 0), 32), yb = min(max(y0 + s, 0), 32);
    return S[yb][xb] - S[ya][xb] - S[yb][xa] + S[ya][xa];
}

// Relaxed forward of both descriptors, one warp per patch (four per CTA, no
// CTA barrier in the patch loop); lane x holds column x of the patch in
// registers (the patch is read once, coalesced).
//  - HashSIFT: the orientation histogram, each row voted as the patch
//    histogram kernel votes it (same values, same order: the same histogram
//    and norm), into the warp's lane-private bins;
//  - BAD: then, over the same shared memory, the patch's 33 x 33 summed-area
//    table in 64-bit fixed point (column sums in registers, row sums in
//    shared memory: integer sums, the same table in any order), the box
//    differences D, the exact bit D <= floor(theta s^2 2^32) and r.
// Each CTA first turns the thresholds into their fixed-point bounds
// floor(theta_k s_k^2 2^32) and scales 2^-32 / s_k^2.  About 9 KB of shared
// memory per warp: five CTAs per SM.
template <int NW>
__global__ void __launch_bounds__(128) train_fwd_kernel(const float *__restrict__ patches, int rows,
                                                        const short4 *__restrict__ box,
                                                        const int *__restrict__ side,
                                                        const float *__restrict__ theta,
                                                        float inv_scale, float *__restrict__ r,
                                                        uint32_t *__restrict__ bits,
                                                        float *__restrict__ hist,
                                                        float *__restrict__ norm)
{
    constexpr int K = NW * 32;
    static_assert(sizeof(dev::WarpHist) >= sizeof(long long) * 33 * 33, "the table fits the histogram area");
    __shared__ dev::WarpHist H[4];
    __shared__ long long thr[K];
    __shared__ float fscale[K];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int k = t; k < K; k += 128) {
        const int sk = __ldg(side + k);
        const double s2 = (double)sk * (double)sk;
        thr[k] = (long long)floor((double)__ldg(theta + k) * s2 * kFix);  // exact product
        fscale[k] = (float)(1.0 / (s2 * kFix));
    }
    __syncthreads();
    dev::WarpHist &S = H[warp];
    long long (*Sw)[33] = reinterpret_cast<long long (*)[33]>(&S);
    const float g_half = 0.5f * dev::gauss16(lane);
    for (int row = blockIdx.x * 4 + warp; row < rows; row += gridDim.x * 4) {
        const float *p = patches + (size_t)row * 1024;
        float v[32];
#pragma unroll
        for (int y = 0; y < 32; ++y)
            v[y] = __ldg(p + y * 32 + lane);
        __syncwarp();  // the previous patch's table reads are done
        // HashSIFT: rows 0 .. 31 down this lane's column, row -1 and row 32
        // replicated
        dev::priv_zero_warp(S, lane);
        __syncwarp();
        {
            float up = v[0], here = v[0];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float down = v[i < 31 ? i + 1 : 31];
                dev::vote_px(S, lane, i, up, here, down, g_half);
                up = here;
                here = down;
            }
        }
        __syncwarp();
        dev::warp_finish(S, lane, true, hist, (size_t)row, norm, 0);
        // BAD: the table over the histogram's shared memory
        Sw[0][lane + 1] = 0;
        Sw[lane + 1][0] = 0;
        if (lane == 0)
            Sw[0][0] = 0;
        {
            long long acc = 0;
#pragma unroll
            for (int y = 0; y < 32; ++y) {
                acc += __float2ll_rn(v[y] * 4294967296.0f);
                Sw[y + 1][lane + 1] = acc;
            }
        }
        __syncwarp();
        // row y = lane + 1: prefix sums along x
        {
            long long acc = 0;
#pragma unroll 8
            for (int x = 1; x <= 32; ++x) {
                acc += Sw[lane + 1][x];
                Sw[lane + 1][x] = acc;
            }
        }
        __syncwarp();
#pragma unroll 2
        for (int j = 0; j < NW; ++j) {
            const int k = j * 32 + lane;
            const short4 b = __ldg(box + k);
            const int s = __ldg(side + k);
            const long long d = sat_box64(Sw, b.x, b.y, s) - sat_box64(Sw, b.z, b.w, s);
            const bool bit = d <= thr[k];  // f = d 2^-32 / s^2 <= theta, exactly
            const float f = (float)d * fscale[k];
            r[(size_t)row * K + k] = dev::tanh_relaxed((__ldg(theta + k) - f) * inv_scale);
            const uint32_t word = __ballot_sync(FULL, bit);
            if (lane == 0)
                bits[(size_t)row * NW + j] = word;
        }
    }
}

// Mining from the two searches (anchors vs negatives, positives vs
// negatives, keys = distance << 22 | index; the searches already leave
// column i out when n > 1, so .x is the nearest j != i and the .y fallback
// keeps the rule for a top-2 input): the first key of each pair whose index
// is not i (any index when n == 1), then the smaller of the two keys.
// Smaller key = smaller min(Hamming(a_i,n_j), Hamming(p_i,n_j)), lowest j on
// ties, i.e. the largest similarity K - 2 Hamming (Sec. III-A).
__global__ void train_mine_combine_kernel(const uint2 *__restrict__ keys_a,
                                          const uint2 *__restrict__ keys_p, int n,
                                          const uint32_t *__restrict__ bits, int NW,
                                          int32_t *__restrict__ nstar, int32_t *__restrict__ xsel)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint2 a = keys_a[i], p = keys_p[i];
    const bool any = n == 1;
    const uint32_t ca = (any || (int)(a.x & kMatchIdxMask) != i) ? a.x : a.y;
    const uint32_t cp = (any || (int)(p.x & kMatchIdxMask) != i) ? p.x : p.y;
    const int j = (int)(min(ca, cp) & kMatchIdxMask);
    uint32_t da = 0, dp = 0;
    for (int v = 0; v < NW; ++v) {
        const uint32_t nv = bits[(size_t)(2 * n + j) * NW + v];
        da += __popc(bits[(size_t)i * NW + v] ^ nv);
        dp += __popc(bits[(size_t)(n + i) * NW + v] ^ nv);
    }
    nstar[i] = j;
    xsel[i] = da <= dp ? 0 : 1;  // S(a,n*) >= S(p,n*) keeps the anchor
}

// Compensated FP32 summation: s + (-c) carries the sum, c the part the last
// addition lost (Kahan).  No products, so nothing is contracted into an FMA.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Warp per triplet: hinge term, loss accumulation and (backward) dL/dr.
// Lane l holds elements 4 (l + 32 q) .. 4 (l + 32 q) + 3 of each row (16-byte
// loads, stores and FP32 atomics); the CTA's 8 hinge terms meet in one FP64
// atomic.  Launched with 256 threads.
template <int K>
__global__ void __launch_bounds__(256) train_loss_kernel(const float *__restrict__ r, int n,
                                                         const int32_t *__restrict__ nstar,
                                                         const int32_t *__restrict__ xsel, float tau,
                                                         const float *__restrict__ gw,
                                                         double *__restrict__ loss_acc,
                                                         float *__restrict__ dr,
                                                         const int *__restrict__ hub,
                                                         long long *__restrict__ hub_acc)
{
    constexpr int Q = K / 128, K4 = K / 4;
    __shared__ float part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const bool valid = i < n;
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
    float4 ra[Q], rp[Q], rn[Q];
    int xs = 0, ns = 0;
    float term = 0.f;
    if (valid) {
        xs = xsel[i];
        ns = nstar[i];
        const size_t nrow = 2 * (size_t)n + ns;
        float sap = 0.f, sxn = 0.f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k4 = q * 32 + lane;
            ra[q] = r4[(size_t)i * K4 + k4];
            rp[q] = r4[(size_t)(n + i) * K4 + k4];
            rn[q] = r4[nrow * K4 + k4];
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float4 x = xs ? rp[q] : ra[q];
            sap = fmaf(ra[q].x, rp[q].x, sap);
            sap = fmaf(ra[q].y, rp[q].y, sap);
            sap = fmaf(ra[q].z, rp[q].z, sap);
            sap = fmaf(ra[q].w, rp[q].w, sap);
            sxn = fmaf(x.x, rn[q].x, sxn);
            sxn = fmaf(x.y, rn[q].y, sxn);
            sxn = fmaf(x.z, rn[q].z, sxn);
            sxn = fmaf(x.w, rn[q].w, sxn);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sap += __shfl_xor_sync(FULL, sap, o);
            sxn += __shfl_xor_sync(FULL, sxn, o);
        }
        term = tau - sap + sxn;
    }
    if (loss_acc) {
        if (lane == 0)
            part[warp] = valid && term > 0.f ? term : 0.f;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w)
                sum += (double)part[w];
            if (sum != 0.0)
                atomicAdd(loss_acc, sum);
        }
    }
    if (!dr || !valid)
        return;
    const float w = *gw;
    const bool on = term > 0.f;
    const int hb = on ? hub[ns] : -1;
    const size_t nrow = 2 * (size_t)n + ns;
    float4 *dr4 = reinterpret_cast<float4 *>(dr);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k4 = q * 32 + lane;
        const float4 a = ra[q], p = rp[q], ng = rn[q];
        const float4 x = xs ? p : a;
        float4 da = make_float4(0.f, 0.f, 0.f, 0.f), dp = da;
        if (on) {
            da = make_float4(w * (-p.x + (xs ? 0.f : ng.x)), w * (-p.y + (xs ? 0.f : ng.y)),
                             w * (-p.z + (xs ? 0.f : ng.z)), w * (-p.w + (xs ? 0.f : ng.w)));
            dp = make_float4(w * (-a.x + (xs ? ng.x : 0.f)), w * (-a.y + (xs ? ng.y : 0.f)),
                             w * (-a.z + (xs ? ng.z : 0.f)), w * (-a.w + (xs ? ng.w : 0.f)));
        }
        dr4[(size_t)i * K4 + k4] = da;
        dr4[(size_t)(n + i) * K4 + k4] = dp;
        if (on && hb < 0)
            atomicAdd(dr4 + nrow * K4 + k4, make_float4(w * x.x, w * x.y, w * x.z, w * x.w));
    }
    if (on && hb >= 0) {
        // a hub: r 2^40 into copy i mod kHubRep, element k = 32 q + lane (a
        // warp's 8-byte atomics on 256 contiguous bytes)
        const float *xr = r + (size_t)(xs ? n + i : i) * K;
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(
            hub_acc + ((size_t)hb * kHubRep + (i & (kHubRep - 1))) * K);
#pragma unroll
        for (int q = 0; q < K / 32; ++q)
            atomicAdd(acc + q * 32 + lane,
                      (unsigned long long)__float2ll_rn(xr[q * 32 + lane] * 1099511627776.0f));
    }
}

// Times each negative is mined, hub[d][nstar_d[i]] += 1 (d = i / n), as far
// as the threshold: only "more than kHubMin" matters, so a counter past it
// is not incremented further (a hub mined by ten thousand anchors would
// otherwise serialise them on one address); the lanes of a warp with the
// same negative add once, together.
__global__ void train_hub_count_kernel(const int32_t *__restrict__ mining, int n,
                                       int *__restrict__ hub)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < 2 * n;
    const int d = act ? i / n : 0;
    const int key = act ? d * n + mining[(size_t)(2 * d) * n + (i % n)] : -1;
    const unsigned same = __match_any_sync(FULL, key);
    if (act && (threadIdx.x & 31) == __ffs(same) - 1 &&
        *reinterpret_cast<volatile int *>(hub + key) <= kHubMin)
        atomicAdd(hub + key, __popc(same));
}

// The count becomes the hub index (in order of arrival) or -1; the hub's
// negative goes into the hub list.
__global__ void train_hub_assign_kernel(int n, int *__restrict__ hub, int *__restrict__ n_hubs,
                                        int *__restrict__ hub_list, int max_hubs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * n) {
        const int d = i / n;
        int hb = -1;
        if (hub[i] > kHubMin) {
            hb = atomicAdd(n_hubs + d, 1);
            hub_list[d * max_hubs + hb] = i - d * n;
        }
        hub[i] = hb;
    }
}

// Hub rows of dL/dr = w (sum of r 2^40) 2^-40: CTA (h, d) converts hub h of
// descriptor d (threads over the columns, the kHubRep copies summed in
// integers) and clears its accumulator; the grid also resets the marks to
// zero counts for the next step's mining.
__global__ void __launch_bounds__(256) train_hub_finish_kernel(int n, int kb, int kh, int *__restrict__ hub,
                                                               const int *__restrict__ hub_list,
                                                               const int *__restrict__ n_hubs,
                                                               long long *__restrict__ hub_acc, int max_hubs,
                                                               const float *__restrict__ gw,
                                                               float *__restrict__ dr_bad,
                                                               float *__restrict__ dr_hs)
{
    const int d = blockIdx.y, h = blockIdx.x, t = threadIdx.x;
    for (int i = (blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + t; i < 2 * n;
         i += gridDim.x * gridDim.y * blockDim.x)
        hub[i] = 0;
    if (h >= n_hubs[d])
        return;
    const int j = hub_list[d * max_hubs + h];
    const int K = d == 0 ? kb : kh, kmax = kb > kh ? kb : kh;
    // descriptor d's hubs start at d max_hubs kHubRep kmax, each kHubRep
    // copies of K entries (as train_loss writes them)
    long long *acc = hub_acc + ((size_t)d * max_hubs * kmax + (size_t)h * K) * kHubRep;
    float *row = d == 0 ? dr_bad + (size_t)(2 * n + j) * kb : dr_hs + (size_t)(2 * n + j) * kh;
    const float w = gw[d];
    for (int k = t; k < K; k += blockDim.x) {
        long long sum = 0;
#pragma unroll
        for (int c = 0; c < kHubRep; ++c) {
            sum += acc[(size_t)c * K + k];
            acc[(size_t)c * K + k] = 0;
        }
        row[k] = w * (float)((double)sum * 0x1p-40);
    }
}

__global__ void train_loss_finish_kernel(const double *__restrict__ acc, float *__restrict__ loss)
{
    if (threadIdx.x < 2)
        loss[threadIdx.x] = (float)acc[threadIdx.x];
}

// dtheta and db from their FP64 accumulators.
__global__ void train_grad_finish_kernel(const double *__restrict__ acc, int kb, int kh,
                                         float *__restrict__ dtheta, float *__restrict__ db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kb)
        dtheta[i] = (float)acc[i];
    else if (i < kb + kh)
        db[i - kb] = (float)acc[i];
}

// This step's W (128 x K, row-major) for the tcgen05 projection: W^T in FP32,
// its BF16 head and tail (W = hi + lo + O(2^-16 |W|)), and the rescue band
// 2^-13 ||W_k||_2 per bit (the bound the projection's FP32 re-check needs
// for normalised histograms).  One CTA of 128 threads per bit.
__global__ void __launch_bounds__(128) train_w_split_kernel(const float *__restrict__ W, int K,
                                                            float *__restrict__ Wt,
                                                            __nv_bfloat16 *__restrict__ hi,
                                                            __nv_bfloat16 *__restrict__ lo,
                                                            float *__restrict__ band)
{
    __shared__ float part[4];
    const int k = blockIdx.x, i = threadIdx.x;
    const float v = W[(size_t)i * K + k];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Wt[(size_t)k * 128 + i] = v;
    hi[(size_t)k * 128 + i] = h;
    lo[(size_t)k * 128 + i] = __float2bfloat16_rn(v - __bfloat162float(h));
    float ss = v * v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        ss += __shfl_xor_sync(FULL, ss, o);
    if ((i & 31) == 0)
        part[i >> 5] = ss;
    __syncthreads();
    if (i == 0)
        band[k] = 0x1p-13f * sqrtf(part[0] + part[1] + part[2] + part[3]);
}

__global__ void transpose_w_kernel(const float *__restrict__ W, int K, float *__restrict__ Wt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 128 * K) {
        const int q = e / K, k = e % K;
        Wt[(size_t)k * 128 + q] = W[e];
    }
}

// dW = H^T dM and db = colsum(dM), dM = dr (1 - r^2) / T.  CTA (x, y) takes
// rows [x R, x R + R) (R a multiple of DW_CHUNK) and columns 128 y .. 128 y +
// 127 of dW: 8 x 8 outputs per thread (dims 4 tq .. 4 tq + 3 and 64 + 4 tq ..,
// k likewise with tk, so that a warp's 16-byte shared loads are contiguous),
// DW_CHUNK rows at a time through shared memory with the next rows' loads in
// flight, each output one fmaf chain over the CTA's rows in order; the CTAs'
// sums meet in FP32 atomics.
constexpr int DW_CHUNK = 8;
__global__ void __launch_bounds__(256, 2) train_hs_dw_kernel(int rows, int K, int R,
                                                             const float *__restrict__ h,
                                                             const float *__restrict__ r,
                                                             const float *__restrict__ dr, float inv_t,
                                                             float *__restrict__ dW,
                                                             double *__restrict__ db_acc)
{
    __shared__ __align__(16) float Hs[DW_CHUNK][128];
    __shared__ __align__(16) float Ms[DW_CHUNK][128];
    const int t = threadIdx.x, tq = t >> 4, tk = t & 15;
    const int k0 = blockIdx.y * 128;
    const int r0 = blockIdx.x * R, r1 = min(rows, r0 + R);
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = 0.f;
    float dbs = 0.f, dbc = 0.f;
    // this thread's share of a chunk: entries t + 256 e of H and of the
    // (r, dr) pairs
    constexpr int E = DW_CHUNK * 128 / 256;
    float hv_n[E], rv_n[E], dv_n[E];
    auto fetch = [&](int base) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = t + 256 * e, rr = idx >> 7, c = idx & 127;
            const bool in = base + rr < r1;
            hv_n[e] = in ? h[(size_t)(base + rr) * 128 + c] : 0.f;
            rv_n[e] = in ? r[(size_t)(base + rr) * K + k0 + c] : 0.f;
            dv_n[e] = in ? dr[(size_t)(base + rr) * K + k0 + c] : 0.f;
        }
    };
    if (r0 < r1)
        fetch(r0);
    for (int base = r0; base < r1; base += DW_CHUNK) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int idx = t + 256 * e;
            Hs[idx >> 7][idx & 127] = hv_n[e];
            Ms[idx >> 7][idx & 127] = dv_n[e] * (1.f - rv_n[e] * rv_n[e]) * inv_t;
        }
        __syncthreads();
        if (base + DW_CHUNK < r1)
            fetch(base + DW_CHUNK);
#pragma unroll 4
        for (int rr = 0; rr < DW_CHUNK; ++rr) {
            const float4 h0 = *reinterpret_cast<const float4 *>(&Hs[rr][tq * 4]);
            const float4 h1 = *reinterpret_cast<const float4 *>(&Hs[rr][64 + tq * 4]);
            const float4 m0 = *reinterpret_cast<const float4 *>(&Ms[rr][tk * 4]);
            const float4 m1 = *reinterpret_cast<const float4 *>(&Ms[rr][64 + tk * 4]);
            const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
            const float mv[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    acc[a][b] = fmaf(hv[a], mv[b], acc[a][b]);
        }
        if (t < 128)
            for (int rr = 0; rr < DW_CHUNK; ++rr)
                kahan_add(dbs, dbc, Ms[rr][t]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int q = a < 4 ? tq * 4 + a : 64 + tq * 4 + a - 4;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            atomicAdd(dW + (size_t)q * K + k0 + (b < 4 ? tk * 4 + b : 64 + tk * 4 + b - 4), acc[a][b]);
    }
    if (t < 128)
        atomicAdd(db_acc + k0 + t, (double)dbs - (double)dbc);
}

// Adjoint of the normalised histogram, dH = (dh - h (h . dh)) / |h| with
// dh = W dm, dm = dr (1 - r^2) / T: a 64-patch x 128-dim tile per CTA, 4 x 8
// outputs per thread (columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3,
// so that a warp's 16-byte shared loads are contiguous), k in 32-deep chunks
// through shared memory with the next chunk's loads in flight.  Each dh is
// one fmaf chain over k = 0 .. K-1; h . dh sums the thread's 8 products, then
// the 16 threads of the row by a butterfly.  Rows of zero norm get dH = 0.
constexpr int DH_M = 64, DH_K = 32;
__global__ void __launch_bounds__(256) train_dh_kernel(int rows, int K, const float *__restrict__ Wt,
                                                       const float *__restrict__ h,
                                                       const float *__restrict__ norm,
                                                       const float *__restrict__ r,
                                                       const float *__restrict__ dr, float inv_t,
                                                       float *__restrict__ dH)
{
    __shared__ __align__(16) float Ds[DH_K][DH_M + 4];
    __shared__ __align__(16) float Ws[DH_K][128];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const int m0 = blockIdx.x * DH_M;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = 0.f;
    constexpr int DQ = DH_M * DH_K / 256, WQ = DH_K * 128 / 256;
    // raw (r, dr) pairs and W values, loaded a chunk ahead (dm is formed when
    // they are stored, so that the loads stay in flight during the FMAs)
    float rq[DQ], dq[DQ], wq[WQ];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < DQ; ++q) {
            const int e = t + 256 * q, row = m0 + e / DH_K, k = k0 + e % DH_K;
            const bool in = row < rows;
            rq[q] = in ? r[(size_t)row * K + k] : 0.f;
            dq[q] = in ? dr[(size_t)row * K + k] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            const int e = t + 256 * q;
            wq[q] = __ldg(Wt + (size_t)(k0 + e / 128) * 128 + e % 128);
        }
    };
    load(0);
    for (int k0 = 0; k0 < K; k0 += DH_K) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < DQ; ++q) {
            const int e = t + 256 * q;
            Ds[e % DH_K][e / DH_K] = dq[q] * (1.f - rq[q] * rq[q]) * inv_t;
        }
#pragma unroll
        for (int q = 0; q < WQ; ++q) {
            const int e = t + 256 * q;
            Ws[e / 128][e % 128] = wq[q];
        }
        __syncthreads();
        if (k0 + DH_K < K)
            load(k0 + DH_K);
#pragma unroll 8
        for (int kk = 0; kk < DH_K; ++kk) {
            const float4 dv = *reinterpret_cast<const float4 *>(&Ds[kk][ty * 4]);
            const float4 w0 = *reinterpret_cast<const float4 *>(&Ws[kk][tx * 4]);
            const float4 w1 = *reinterpret_cast<const float4 *>(&Ws[kk][64 + tx * 4]);
            const float d[4] = {dv.x, dv.y, dv.z, dv.w};
            const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    acc[a][b] = fmaf(w[b], d[a], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int row = m0 + ty * 4 + a;
        const bool in = row < rows;
        float hv[8];
        if (in) {
            const float4 h0 = *reinterpret_cast<const float4 *>(h + (size_t)row * 128 + tx * 4);
            const float4 h1 = *reinterpret_cast<const float4 *>(h + (size_t)row * 128 + 64 + tx * 4);
            hv[0] = h0.x; hv[1] = h0.y; hv[2] = h0.z; hv[3] = h0.w;
            hv[4] = h1.x; hv[5] = h1.y; hv[6] = h1.z; hv[7] = h1.w;
        } else {
#pragma unroll
            for (int b = 0; b < 8; ++b)
                hv[b] = 0.f;
        }
        float hd = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            hd = fmaf(hv[b], acc[a][b], hd);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1)
            hd += __shfl_xor_sync(FULL, hd, o);
        const float nrm = in ? norm[row] : 0.f;
        float o8[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            o8[b] = nrm > 0.f ? (acc[a][b] - hv[b] * hd) / nrm : 0.f;
        if (in) {
            *reinterpret_cast<float4 *>(dH + (size_t)row * 128 + tx * 4) = make_float4(o8[0], o8[1], o8[2], o8[3]);
            *reinterpret_cast<float4 *>(dH + (size_t)row * 128 + 64 + tx * 4) =
                make_float4(o8[4], o8[5], o8[6], o8[7]);
        }
    }
}

// Patch gradient of both losses and dtheta, written once per patch.  Warp w
// owns pixel rows 8w .. 8w + 7 of the patch; lane 8c + r takes row 8w + r,
// columns 8c .. 8c + 7 (the histogram's thread layout).  The patch comes in
// and its gradient goes out through shared memory with coalesced global
// accesses.  The HashSIFT adjoint per pixel (recomputed from the patch, with
// the patch's dH from train_dh_kernel) reads its gradient stencil from the
// staged patch; the adjoint of the central differences gathers by lane
// shuffles, with the warps' first and last rows through shared memory.  The
// BAD box adjoint is a 2-D difference array in shared memory (the corner
// updates that fall inside the patch, then prefix sums along x and y).  Both
// meet in one value per pixel, BAD + 0.5 * (HashSIFT gather).  The next
// patch's pixels and dH are in flight while the current patch is processed.
// dtheta columns are summed per thread with compensated additions over its
// rows and meet in the FP64 accumulators.
template <int KB>
__global__ void __launch_bounds__(128, 7) train_bwd_kernel(
    const float *__restrict__ patches, int rows, const float *__restrict__ dHg,
    const short4 *__restrict__ box, const int *__restrict__ side, const float *__restrict__ r_bad,
    const float *__restrict__ dr_bad, float inv_scale, double *__restrict__ dtheta_acc,
    float *__restrict__ dpatches)
{
    constexpr int QB = KB / 128;  // BAD bits per thread per patch
    __shared__ float D[32][33];  // odd row stride: the box corners spread over the banks
    __shared__ __align__(16) float P[32][36];                 // the patch
    __shared__ __align__(16) float O[32][36];                 // the previous patch's gradient
    __shared__ __align__(16) float gtop[4][32], gbot[4][32];  // dgy of rows 8w, 8w + 7
    __shared__ float ctot[4][32];                             // column sums of rows 8w .. 8w + 7
    __shared__ float dH[128];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r = lane & 7, c = lane >> 3;
    const int i = warp * 8 + r, j0 = c * 8;  // this thread's row and first column
    const dev::HistLane L = dev::hist_lane(t);
    float dth[QB], dthc[QB];
#pragma unroll
    for (int q = 0; q < QB; ++q)
        dth[q] = dthc[q] = 0.f;
    float pn[8];
    float hn = 0.f;
    int row = blockIdx.x, prev = -1;
    if (row < rows) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            pn[q] = __ldg(patches + (size_t)row * 1024 + t + q * 128);
        hn = dHg[(size_t)row * 128 + t];
    }
    for (; row < rows; row += gridDim.x) {
        // this patch's BAD responses and dL/dr (loads in flight meanwhile)
        float rb[QB], drb[QB];
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            rb[q] = r_bad[(size_t)row * KB + q * 128 + t];
            drb[q] = dr_bad[(size_t)row * KB + q * 128 + t];
        }
        __syncthreads();
        // the previous patch's gradient out (coalesced), this patch's pixels in
        if (prev >= 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = t + q * 128;
                dpatches[(size_t)prev * 1024 + e] = O[e >> 5][e & 31];
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = t + q * 128;
            P[e >> 5][e & 31] = pn[q];
        }
        dH[t] = hn;
        for (int e = t; e < 32 * 33; e += 128)
            (&D[0][0])[e] = 0.f;
        __syncthreads();
        // this thread's pixels and the stencil's neighbours: rows i -/+ 1 and
        // columns j0 - 1, j0 + 8, clamped to the patch
        float px[8], up[8], dn[8];
        {
            const int iu = max(i - 1, 0), id = min(i + 1, 31);
            const float4 a = *reinterpret_cast<const float4 *>(&P[i][j0]);
            const float4 b = *reinterpret_cast<const float4 *>(&P[i][j0 + 4]);
            const float4 ua = *reinterpret_cast<const float4 *>(&P[iu][j0]);
            const float4 ub = *reinterpret_cast<const float4 *>(&P[iu][j0 + 4]);
            const float4 da = *reinterpret_cast<const float4 *>(&P[id][j0]);
            const float4 db = *reinterpret_cast<const float4 *>(&P[id][j0 + 4]);
            px[0] = a.x; px[1] = a.y; px[2] = a.z; px[3] = a.w;
            px[4] = b.x; px[5] = b.y; px[6] = b.z; px[7] = b.w;
            up[0] = ua.x; up[1] = ua.y; up[2] = ua.z; up[3] = ua.w;
            up[4] = ub.x; up[5] = ub.y; up[6] = ub.z; up[7] = ub.w;
            dn[0] = da.x; dn[1] = da.y; dn[2] = da.z; dn[3] = da.w;
            dn[4] = db.x; dn[5] = db.y; dn[6] = db.z; dn[7] = db.w;
        }
        const float left = P[i][max(j0 - 1, 0)], right = P[i][min(j0 + 8, 31)];
        // per-pixel adjoint of the votes
        const int cell = t >> 3;
        float dgx[8], dgy[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float pl = q > 0 ? px[q - 1] : left, pr = q < 7 ? px[q + 1] : right;
            const float gx = 0.5f * (pr - pl);
            const float gy = 0.5f * (dn[q] - up[q]);
            const float m2 = gx * gx + gy * gy;
            dgx[q] = dgy[q] = 0.f;
            if (m2 > 0.f) {
                // 1/|g| and 1/|g|^2 from one reciprocal square root; the bin
                // pair from the forward's orient_bin, exact at multiples of 45
                // degrees (frequent on flat-sided patches), where the
                // histogram's derivative jumps
                const float im = rsqrtf(m2);
                const float m = m2 * im;
                float w1;
                int b0 = dev::orient_bin(gx, gy, w1);
                // on a bin edge the derivative in the angle is one-sided: take
                // the floor side (the bin that starts at the edge, w1 = 0), as
                // the exact definition floor(q) does; the votes are the same
                if (w1 >= 1.0f) {
                    b0 = (b0 + 1) & 7;
                    w1 = 0.0f;
                }
                const int b1 = (b0 + 1) & 7;
                const float d0 = dH[cell * 8 + b0], d1 = dH[cell * 8 + b1];
                const float g = L.g[q];
                const float dmag = g * ((1.f - w1) * d0 + w1 * d1);
                const float dphi = g * m * (d1 - d0) * 1.27323954473516268615f;
                const float im2 = im * im;
                dgx[q] = dmag * gx * im - dphi * gy * im2;
                dgy[q] = dmag * gy * im + dphi * gx * im2;
            }
        }
        // the next patch's pixels and dH, in flight from here
        const int next = row + gridDim.x;
        if (next < rows) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                pn[q] = __ldg(patches + (size_t)next * 1024 + t + q * 128);
            hn = dHg[(size_t)next * 128 + t];
        }
        if (r == 0) {
            *reinterpret_cast<float4 *>(&gtop[warp][j0]) = make_float4(dgy[0], dgy[1], dgy[2], dgy[3]);
            *reinterpret_cast<float4 *>(&gtop[warp][j0 + 4]) = make_float4(dgy[4], dgy[5], dgy[6], dgy[7]);
        }
        if (r == 7) {
            *reinterpret_cast<float4 *>(&gbot[warp][j0]) = make_float4(dgy[0], dgy[1], dgy[2], dgy[3]);
            *reinterpret_cast<float4 *>(&gbot[warp][j0 + 4]) = make_float4(dgy[4], dgy[5], dgy[6], dgy[7]);
        }
        // BAD: dtheta and the box adjoints of this patch (z = (theta - f) / (255 T))
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            const int k = q * 128 + t;
            const float dz = drb[q] * (1.f - rb[q] * rb[q]);
            kahan_add(dth[q], dthc[q], dz * inv_scale);
            if (dz == 0.f)
                continue;
            const int s = __ldg(side + k);
            const float g = -dz * inv_scale / (float)(s * s);
            const short4 b = __ldg(box + k);
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                const int x0 = bx ? b.z : b.x, y0 = bx ? b.w : b.y;
                const float sg = bx ? -g : g;
                const int xa = min(max(x0, 0), 32), xb = min(max(x0 + s, 0), 32);
                const int ya = min(max(y0, 0), 32), yb = min(max(y0 + s, 0), 32);
                // corners on row or column 32 lie outside the prefix sums' range
                if (xa < xb && ya < yb) {
                    atomicAdd(&D[ya][xa], sg);
                    if (xb < 32)
                        atomicAdd(&D[ya][xb], -sg);
                    if (yb < 32) {
                        atomicAdd(&D[yb][xa], -sg);
                        if (xb < 32)
                            atomicAdd(&D[yb][xb], sg);
                    }
                }
            }
        }
        __syncthreads();
        // prefix sums of the 32 x 32 difference array.  Along x: thread (y, u) = (t / 4, t % 4)
        // sums columns 8u .. 8u + 7 of row y in order, the four segments of
        // the row meet by a scan over their lanes.
        {
            const int y = t >> 2, u = t & 3;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                v[q] = D[y][8 * u + q];
#pragma unroll
            for (int q = 1; q < 8; ++q)
                v[q] += v[q - 1];
            float inc = v[7];
            float o = __shfl_up_sync(FULL, inc, 1);
            if (u >= 1) inc += o;
            o = __shfl_up_sync(FULL, inc, 2);
            if (u >= 2) inc += o;
            float ex = __shfl_up_sync(FULL, inc, 1);
            if (u == 0)
                ex = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                D[y][8 * u + q] = v[q] + ex;
        }
        __syncthreads();
        // along y: warp w sums rows 8w .. 8w + 7 of column lane in order, then
        // adds the column sums of the warps above
        float cv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            cv[u] = D[warp * 8 + u][lane];
#pragma unroll
        for (int u = 1; u < 8; ++u)
            cv[u] += cv[u - 1];
        ctot[warp][lane] = cv[7];
        __syncthreads();
        {
            float carry = 0.f;
            for (int w = 0; w < warp; ++w)
                carry += ctot[w][lane];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                D[warp * 8 + u][lane] = cv[u] + carry;
        }
        __syncthreads();
        // gather: gx(i, x) reads columns jr(x) (+) and jl(x) (-), gy likewise
        // for rows: pixel (y, x) collects dgx(y, x - 1), dgx(y, 31) at x = 31,
        // -dgx(y, x + 1), -dgx(y, 0) at x = 0, and the same in y; the patch
        // gradient is the BAD part plus half the HashSIFT sum
        float gl = __shfl_up_sync(FULL, dgx[7], 8), gr = __shfl_down_sync(FULL, dgx[0], 8);
        float gu[8], gd[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            gu[q] = __shfl_up_sync(FULL, dgy[q], 1);
            gd[q] = __shfl_down_sync(FULL, dgy[q], 1);
        }
        if (r == 0 && warp > 0) {
            const float4 a = *reinterpret_cast<const float4 *>(&gbot[warp - 1][j0]);
            const float4 b = *reinterpret_cast<const float4 *>(&gbot[warp - 1][j0 + 4]);
            gu[0] = a.x; gu[1] = a.y; gu[2] = a.z; gu[3] = a.w;
            gu[4] = b.x; gu[5] = b.y; gu[6] = b.z; gu[7] = b.w;
        }
        if (r == 7 && warp < 3) {
            const float4 a = *reinterpret_cast<const float4 *>(&gtop[warp + 1][j0]);
            const float4 b = *reinterpret_cast<const float4 *>(&gtop[warp + 1][j0 + 4]);
            gd[0] = a.x; gd[1] = a.y; gd[2] = a.z; gd[3] = a.w;
            gd[4] = b.x; gd[5] = b.y; gd[6] = b.z; gd[7] = b.w;
        }
        float dv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            dv[q] = D[i][j0 + q];
        float o8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int x = j0 + q;
            float v = 0.f;
            if (x >= 1) v += q > 0 ? dgx[q - 1] : gl;  // jr(x-1) = x
            if (x == 31) v += dgx[7];                  // jr(31) = 31
            if (x <= 30) v -= q < 7 ? dgx[q + 1] : gr; // jl(x+1) = x
            if (x == 0) v -= dgx[0];                   // jl(0) = 0
            if (i >= 1) v += gu[q];
            if (i == 31) v += dgy[q];
            if (i <= 30) v -= gd[q];
            if (i == 0) v -= dgy[q];
            o8[q] = dv[q] + 0.5f * v;
        }
        *reinterpret_cast<float4 *>(&O[i][j0]) = make_float4(o8[0], o8[1], o8[2], o8[3]);
        *reinterpret_cast<float4 *>(&O[i][j0 + 4]) = make_float4(o8[4], o8[5], o8[6], o8[7]);
        prev = row;
    }
    __syncthreads();
    if (prev >= 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = t + q * 128;
            dpatches[(size_t)prev * 1024 + e] = O[e >> 5][e & 31];
        }
    }
#pragma unroll
    for (int q = 0; q < QB; ++q)
        atomicAdd(dtheta_acc + q * 128 + t, (double)dth[q] - (double)dthc[q]);
}

int grid_rows(int rows, int sm_count, int per_sm)
{
    const long long g = (long long)sm_count * per_sm;
    return (int)(rows < g ? rows : g);
}

}  // namespace
}  // namespace bd

extern "C" {

bd_status bd_train_create(bd_ctx *ctx, const bd_bad_params *bad, int hs_bits, int n,
                          float temperature, float tau_bad, float tau_hs, bd_train **out)
{
    if (!ctx || !out)
        return BD_ERR_INVALID;
    *out = nullptr;
    if (!bad || (hs_bits != 256 && hs_bits != 512) || n < 1 || n > (1 << 20) ||
        !(temperature > 0.f) || !isfinite(tau_bad) || !isfinite(tau_hs))
        return set_err(ctx, BD_ERR_INVALID, "bd_train_create: bad arguments");
    bd_train *tr = new bd_train();
    tr->ctx = ctx;
    tr->bad = bad;
    tr->n = n;
    tr->rows = 3 * n;
    tr->kb = bad->nbits;
    tr->kh = hs_bits;
    tr->T = temperature;
    tr->tau_bad = tau_bad;
    tr->tau_hs = tau_hs;
    const size_t R = (size_t)tr->rows;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device)
        cudaSetDevice(ctx->device);
    cudaError_t e = cudaMalloc(&tr->r_bad, sizeof(float) * R * tr->kb);
    if (e == cudaSuccess) e = cudaMalloc(&tr->r_hs, sizeof(float) * R * tr->kh);
    if (e == cudaSuccess) e = cudaMalloc(&tr->h, sizeof(float) * R * 128);
    if (e == cudaSuccess) e = cudaMalloc(&tr->norm, sizeof(float) * R);
    if (e == cudaSuccess) e = cudaMalloc(&tr->bits_bad, sizeof(uint32_t) * R * (tr->kb / 32));
    if (e == cudaSuccess) e = cudaMalloc(&tr->bits_hs, sizeof(uint32_t) * R * (tr->kh / 32));
    const int kmax = tr->kb > tr->kh ? tr->kb : tr->kh;
    if (e == cudaSuccess) e = cudaMalloc(&tr->tc_scratch, match_tc_scratch_bytes(n, n, kmax, ctx->sm_count));
    if (e == cudaSuccess) e = cudaMalloc(&tr->keys, sizeof(uint2) * 2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&tr->arrivals, sizeof(unsigned int) * (size_t)match_tc_query_blocks(n));
    if (e == cudaSuccess) e = cudaMemset(tr->arrivals, 0, sizeof(unsigned int) * (size_t)match_tc_query_blocks(n));
    if (e == cudaSuccess) e = cudaMalloc(&tr->mining, sizeof(int32_t) * 4 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&tr->dr_bad, sizeof(float) * R * tr->kb);
    if (e == cudaSuccess) e = cudaMalloc(&tr->dr_hs, sizeof(float) * R * tr->kh);
    if (e == cudaSuccess) e = cudaMalloc(&tr->Wt, sizeof(float) * 128 * tr->kh);
    if (e == cudaSuccess) e = cudaMalloc(&tr->dH, sizeof(float) * R * 128);
    {
        bd_hs_params *hp = &tr->hp;
        hp->ctx = ctx;
        hp->nbits = tr->kh;
        hp->precision = BD_HS_BF16_RESCUE;
        hp->w_has_lo = true;
        if (e == cudaSuccess) e = cudaMalloc(&hp->d_Wt, sizeof(float) * 128 * tr->kh);
        if (e == cudaSuccess) e = cudaMalloc(&hp->d_Wt16_hi, sizeof(__nv_bfloat16) * 128 * tr->kh);
        if (e == cudaSuccess) e = cudaMalloc(&hp->d_Wt16_lo, sizeof(__nv_bfloat16) * 128 * tr->kh);
        if (e == cudaSuccess) e = cudaMalloc(&hp->d_band, sizeof(float) * tr->kh);
        if (e == cudaSuccess) {
            hp->tmap_ok = encode_tmap_2d_bf16(&hp->tmap_w_hi, hp->d_Wt16_hi, 128, (uint64_t)tr->kh, 256, 64, 128) &&
                          encode_tmap_2d_bf16(&hp->tmap_w_lo, hp->d_Wt16_lo, 128, (uint64_t)tr->kh, 256, 64, 128);
            if (!hp->tmap_ok)
                e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess)
            e = prepare_hs_proj_tc();
    }
    if (e == cudaSuccess) e = cudaMalloc(&tr->loss_acc, sizeof(double) * (2 + tr->kb + tr->kh));
    tr->max_hubs = n / (kHubMin + 1) + 1;
    const size_t hub_words = 2 * (size_t)tr->max_hubs * kHubRep * (size_t)std::max(tr->kb, tr->kh);
    if (e == cudaSuccess) e = cudaMalloc(&tr->hub, sizeof(int) * 2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemset(tr->hub, 0, sizeof(int) * 2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&tr->n_hubs, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&tr->hub_list, sizeof(int) * 2 * (size_t)tr->max_hubs);
    if (e == cudaSuccess) e = cudaMalloc(&tr->hub_acc, sizeof(long long) * hub_words);
    if (e == cudaSuccess) e = cudaMemset(tr->hub_acc, 0, sizeof(long long) * hub_words);
    if (prev >= 0 && prev != ctx->device)
        cudaSetDevice(prev);
    if (e != cudaSuccess) {
        bd_train_destroy(tr);
        return cuda_err(ctx, e, "bd_train_create");
    }
    *out = tr;
    return BD_OK;
}

void bd_train_destroy(bd_train *tr)
{
    if (!tr)
        return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != tr->ctx->device)
        cudaSetDevice(tr->ctx->device);
    cudaStreamSynchronize(tr->ctx->stream);
    for (void *p : {(void *)tr->r_bad, (void *)tr->r_hs, (void *)tr->h, (void *)tr->norm,
                    (void *)tr->bits_bad, (void *)tr->bits_hs, (void *)tr->tc_scratch,
                    (void *)tr->keys, (void *)tr->arrivals, (void *)tr->mining, (void *)tr->dr_bad,
                    (void *)tr->dr_hs, (void *)tr->Wt, (void *)tr->dH, (void *)tr->hp.d_Wt,
                    (void *)tr->hp.d_Wt16_hi, (void *)tr->hp.d_Wt16_lo, (void *)tr->hp.d_band,
                    (void *)tr->loss_acc, (void *)tr->hub,
                    (void *)tr->n_hubs, (void *)tr->hub_list, (void *)tr->hub_acc})
        if (p)
            cudaFree(p);
    if (prev >= 0 && prev != tr->ctx->device)
        cudaSetDevice(prev);
    delete tr;
}

bd_status bd_train_forward(bd_ctx *ctx, bd_train *tr, const float *patches, const float *theta,
                           const float *W, const float *b, const int32_t *fixed_mining,
                           float *loss, int32_t *mining_out)
{
    if (!ctx || !tr || tr->ctx != ctx || !patches || !theta || !W || !b || !loss)
        return BD_ERR_INVALID;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device)
        cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    TraceScope scope(ctx, st);
    const int n = tr->n, rows = tr->rows, sm = ctx->sm_count;
    const float inv_scale = 1.0f / (255.0f * tr->T);
    const bd_bad_params *bp = tr->bad;
    cudaError_t e = cudaSuccess;
    // relaxed BAD and the HashSIFT histograms in one pass over the patches
    if (tr->kb == 256)
        train_fwd_kernel<8><<<grid_rows((rows + 3) / 4, sm, 5), 128, 0, st>>>(
            patches, rows, bp->d_patch_box, bp->d_patch_side, theta, inv_scale, tr->r_bad, tr->bits_bad,
            tr->h, tr->norm);
    else
        train_fwd_kernel<16><<<grid_rows((rows + 3) / 4, sm, 5), 128, 0, st>>>(
            patches, rows, bp->d_patch_box, bp->d_patch_side, theta, inv_scale, tr->r_bad, tr->bits_bad,
            tr->h, tr->norm);
    trace_kernel(st, "train_fwd");
    e = cudaGetLastError();
    // relaxed HashSIFT projection
    if (e == cudaSuccess) {
        bd_hs_params *hp = &tr->hp;
        train_w_split_kernel<<<tr->kh, 128, 0, st>>>(W, tr->kh, hp->d_Wt, hp->d_Wt16_hi, hp->d_Wt16_lo,
                                                     hp->d_band);
        trace_kernel(st, "train_w_split");
        note_launches(1);
        hp->d_bias = const_cast<float *>(b);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = launch_hs_proj_tc(hp, tr->h, rows, tr->bits_hs, ctx->status, st, nullptr, nullptr, nullptr,
                                  tr->r_hs, 1.0f / tr->T);
    }
    // mining on hard codes, or the given mining
    if (e == cudaSuccess && fixed_mining) {
        e = cudaMemcpyAsync(tr->mining, fixed_mining, sizeof(int32_t) * 4 * (size_t)n,
                            cudaMemcpyDeviceToDevice, st);
    } else if (e == cudaSuccess) {
        for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
            const uint32_t *bits = d == 0 ? tr->bits_bad : tr->bits_hs;
            const int K = d == 0 ? tr->kb : tr->kh;
            const int nw = K / 32;
            const uint32_t *neg = bits + (size_t)2 * n * nw;
            e = launch_match_tc_keys(ctx, bits, n, neg, n, K, 1, 1, nullptr, tr->keys, tr->tc_scratch,
                                     st, tr->arrivals, 1);
            if (e == cudaSuccess)
                e = launch_match_tc_keys(ctx, bits + (size_t)n * nw, n, neg, n, K, 1, 1, nullptr,
                                         tr->keys + n, tr->tc_scratch, st, tr->arrivals, 1);
            if (e == cudaSuccess) {
                train_mine_combine_kernel<<<(n + 255) / 256, 256, 0, st>>>(
                    tr->keys, tr->keys + n, n, bits, nw, tr->mining + (size_t)(2 * d) * n,
                    tr->mining + (size_t)(2 * d + 1) * n);
                trace_kernel(st, "train_mine_combine");
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(tr->loss_acc, 0, sizeof(double) * 2, st);
    if (e == cudaSuccess) {
        const int blocks = (n * 32 + 255) / 256;
        for (int d = 0; d < 2; ++d) {
            const float *r = d == 0 ? tr->r_bad : tr->r_hs;
            const int K = d == 0 ? tr->kb : tr->kh;
            const float tau = d == 0 ? tr->tau_bad : tr->tau_hs;
            const int32_t *ns = tr->mining + (size_t)(2 * d) * n, *xs = ns + n;
            if (K == 256)
                train_loss_kernel<256><<<blocks, 256, 0, st>>>(r, n, ns, xs, tau, nullptr, tr->loss_acc + d,
                                                               nullptr, nullptr, nullptr);
            else
                train_loss_kernel<512><<<blocks, 256, 0, st>>>(r, n, ns, xs, tau, nullptr, tr->loss_acc + d,
                                                               nullptr, nullptr, nullptr);
            trace_kernel(st, "train_loss");
        }
        train_loss_finish_kernel<<<1, 32, 0, st>>>(tr->loss_acc, loss);
        trace_kernel(st, "train_loss_finish");
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && mining_out)
        e = cudaMemcpyAsync(mining_out, tr->mining, sizeof(int32_t) * 4 * (size_t)n,
                            cudaMemcpyDeviceToDevice, st);
    note_launches(fixed_mining ? 6 : 8);
    if (prev >= 0 && prev != ctx->device)
        cudaSetDevice(prev);
    return e == cudaSuccess ? BD_OK : cuda_err(ctx, e, "bd_train_forward");
}

bd_status bd_train_backward(bd_ctx *ctx, bd_train *tr, const float *patches, const float *W,
                            const float *grad_loss, float *dtheta, float *dW, float *db,
                            float *dpatches)
{
    if (!ctx || !tr || tr->ctx != ctx || !patches || !W || !grad_loss || !dtheta || !dW || !db ||
        !dpatches)
        return BD_ERR_INVALID;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device)
        cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    TraceScope scope(ctx, st);
    const int n = tr->n, rows = tr->rows, sm = ctx->sm_count;
    const size_t R = (size_t)rows;
    const float inv_scale = 1.0f / (255.0f * tr->T), inv_t = 1.0f / tr->T;
    const bd_bad_params *bp = tr->bad;
    cudaError_t e = cudaSuccess;
    // dL/dr: negatives' rows collect with atomics (FP32, or the hubs' fixed
    // point), so the FP32 rows start at zero; then the hubs of this mining
    e = cudaMemsetAsync(tr->dr_bad + (size_t)2 * n * tr->kb, 0, sizeof(float) * n * tr->kb, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(tr->dr_hs + (size_t)2 * n * tr->kh, 0, sizeof(float) * n * tr->kh, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(tr->n_hubs, 0, sizeof(int) * 2, st);
    if (e == cudaSuccess) {
        train_hub_count_kernel<<<(2 * n + 255) / 256, 256, 0, st>>>(tr->mining, n, tr->hub);
        trace_kernel(st, "train_hub_count");
        train_hub_assign_kernel<<<(2 * n + 255) / 256, 256, 0, st>>>(n, tr->hub, tr->n_hubs, tr->hub_list,
                                                                    tr->max_hubs);
        trace_kernel(st, "train_hub_assign");
        e = cudaGetLastError();
    }
    double *dth_acc = tr->loss_acc + 2, *db_acc = dth_acc + tr->kb;
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dth_acc, 0, sizeof(double) * (tr->kb + tr->kh), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dW, 0, sizeof(float) * 128 * tr->kh, st);
    if (e == cudaSuccess) {
        const int blocks = (n * 32 + 255) / 256;
        for (int d = 0; d < 2; ++d) {
            const float *r = d == 0 ? tr->r_bad : tr->r_hs;
            float *drp = d == 0 ? tr->dr_bad : tr->dr_hs;
            const int K = d == 0 ? tr->kb : tr->kh;
            const float tau = d == 0 ? tr->tau_bad : tr->tau_hs;
            const int32_t *ns = tr->mining + (size_t)(2 * d) * n, *xs = ns + n;
            const int *hub = tr->hub + (size_t)d * n;
            long long *hacc = tr->hub_acc + (size_t)d * tr->max_hubs * kHubRep * (size_t)std::max(tr->kb, tr->kh);
            if (K == 256)
                train_loss_kernel<256><<<blocks, 256, 0, st>>>(r, n, ns, xs, tau, grad_loss + d, nullptr,
                                                               drp, hub, hacc);
            else
                train_loss_kernel<512><<<blocks, 256, 0, st>>>(r, n, ns, xs, tau, grad_loss + d, nullptr,
                                                               drp, hub, hacc);
            trace_kernel(st, "train_dr");
        }
        train_hub_finish_kernel<<<dim3(tr->max_hubs, 2), 256, 0, st>>>(
            n, tr->kb, tr->kh, tr->hub, tr->hub_list, tr->n_hubs, tr->hub_acc, tr->max_hubs, grad_loss,
            tr->dr_bad, tr->dr_hs);
        trace_kernel(st, "train_hub_finish");
        // HashSIFT: dW and db; then both patch gradients and dtheta in one pass
        transpose_w_kernel<<<(128 * tr->kh + 255) / 256, 256, 0, st>>>(W, tr->kh, tr->Wt);
        {
            // one wave: 2 CTAs per SM over the K / 128 column tiles
            const int ktiles = tr->kh / 128;
            const int nx = std::max(1, 2 * sm / ktiles);
            const int R = ((rows + nx - 1) / nx + DW_CHUNK - 1) / DW_CHUNK * DW_CHUNK;
            dim3 g2((rows + R - 1) / R, ktiles);
            train_hs_dw_kernel<<<g2, 256, 0, st>>>(rows, tr->kh, R, tr->h, tr->r_hs, tr->dr_hs, inv_t, dW,
                                                   db_acc);
        }
        trace_kernel(st, "train_hs_dw");
        train_dh_kernel<<<(rows + DH_M - 1) / DH_M, 256, 0, st>>>(rows, tr->kh, tr->Wt, tr->h, tr->norm,
                                                                  tr->r_hs, tr->dr_hs, inv_t, tr->dH);
        trace_kernel(st, "train_dh");
        {
            auto kern = tr->kb == 256 ? train_bwd_kernel<256> : train_bwd_kernel<512>;
            kern<<<grid_rows(rows, sm, 7), 128, 0, st>>>(patches, rows, tr->dH, bp->d_patch_box,
                                                        bp->d_patch_side, tr->r_bad, tr->dr_bad, inv_scale,
                                                        dth_acc, dpatches);
            trace_kernel(st, "train_bwd");
        }
        train_grad_finish_kernel<<<(tr->kb + tr->kh + 255) / 256, 256, 0, st>>>(dth_acc, tr->kb, tr->kh,
                                                                               dtheta, db);
        trace_kernel(st, "train_grad_finish");
        e = cudaGetLastError();
    }
    note_launches(11);
    (void)R;
    if (prev >= 0 && prev != ctx->device)
        cudaSetDevice(prev);
    return e == cudaSuccess ? BD_OK : cuda_err(ctx, e, "bd_train_backward");
}

}  // extern "C"
