// Measurement probes: kernels that drive one hardware path close to its limit,
// so that each descriptor kernel's roofline is taken against a measured rate
// of the path that bounds it rather than a datasheet figure.
//
//  gather  random 4-byte loads through the read-only path, the access of the
//          BAD stump (eight integral-image corners per bit, Sec. III-A): each
//          warp draws a window of `window_words` words and its lanes load 64
//          independent random words of it per window, like one warp
//          describing one BAD-256 keypoint.  A window as large as the table
//          gives the L2 random-gather rate; a BAD-sized window (a few KB)
//          gives the L1-hit gather rate.
//  l1      the L1 data path's sector rate: every lane of a warp loads 16
//          consecutive bytes (a request = 512 contiguous bytes = 16 sectors
//          of 32 B) from a 16 KB window per CTA that stays in L1.  The
//          largest rate at which L1 can hand sectors to the SM's warps; the
//          BAD gathers' bound (the distinct sectors a keypoint's corner
//          reads touch, divided by this rate, is the least time they take).
//  popc    32-bit population counts (matching, S = K - 2 Hamming).
//  ffma    FP32 fused multiply-adds (histogram arithmetic).
//  mufu    ex2 on the special-function unit (exp / rsqrt of the histogram).
//
// Indices come from a per-lane linear congruential generator, so no load
// depends on another's value; every result is folded into one sink word.
#include "bd_internal.h"

namespace bd {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kLoadsPerWindow = 64;
constexpr int kChains = 8;

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ void fold(uint32_t v, uint32_t *sink)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(sink, v);
}

__global__ void __launch_bounds__(kProbeThreads) probe_gather_kernel(
    const uint32_t *__restrict__ table, uint32_t words_mask, uint32_t window_mask, int windows,
    uint32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t warp = tid >> 5;
    uint32_t x = mix32(tid * 0x9e3779b9u + 1u);
    uint32_t acc = 0;
#pragma unroll 1
    for (int wi = 0; wi < windows; ++wi) {
        const uint32_t base = (mix32(warp * 0x85ebca6bu + (uint32_t)wi) & words_mask) & ~window_mask;
        const uint32_t *win = table + base;
#pragma unroll 1
        for (int i = 0; i < kLoadsPerWindow; i += 16) {
            uint32_t v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                x = x * 1664525u + 1013904223u;
                v[u] = __ldg(win + ((x >> 7) & window_mask));
            }
#pragma unroll
            for (int u = 0; u < 16; ++u)
                acc += v[u];
        }
    }
    fold(acc, sink);
}

constexpr int kL1WindowVec = 1024;  // 16 KB window per CTA, in 16-byte vectors
constexpr int kL1Unroll = 8;        // requests in flight per warp

__global__ void __launch_bounds__(kProbeThreads) probe_l1_kernel(const uint4 *__restrict__ table,
                                                                 uint32_t vecs_mask, int reps,
                                                                 uint32_t *sink)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t base = (mix32(blockIdx.x * 0x9e3779b9u + 7u) & vecs_mask) & ~(uint32_t)(kL1WindowVec - 1);
    const uint4 *win = table + base;
    uint32_t off = warp * 32 * kL1Unroll;  // a multiple of 32 vectors: 512-byte aligned requests
    uint32_t acc = 0;
#pragma unroll 1
    for (int r = 0; r < reps; ++r) {
        uint4 v[kL1Unroll];
#pragma unroll
        for (int u = 0; u < kL1Unroll; ++u)
            v[u] = __ldg(win + ((off + 32 * u + lane) & (kL1WindowVec - 1)));
#pragma unroll
        for (int u = 0; u < kL1Unroll; ++u)
            acc += v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        off += 32 * (kL1Unroll + 1);
    }
    fold(acc, sink);
}

__global__ void __launch_bounds__(kProbeThreads) probe_popc_kernel(int iters, uint32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        a[c] = mix32(tid * kChains + c);
    const uint32_t k = mix32(tid ^ 0x5bd1e995u);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                a[c] = (uint32_t)__popc(a[c] ^ k) + a[c];
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += a[c];
    fold(s, sink);
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(int iters, uint32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        a[c] = (float)(mix32(tid * kChains + c) & 0xffff) * 1.0e-5f;
    const float m = 0.999f, k = 1.0e-3f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                a[c] = fmaf(a[c], m, k);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += a[c];
    fold(__float_as_uint(s), sink);
}

__device__ __forceinline__ float ex2_neg(float a)
{
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a));
    return r;
}

__global__ void __launch_bounds__(kProbeThreads) probe_mufu_kernel(int iters, uint32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        a[c] = (float)(mix32(tid * kChains + c) & 0xffff) * 1.0e-5f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                a[c] = ex2_neg(a[c]);  // stays in [0.5, 1]
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += a[c];
    fold(__float_as_uint(s), sink);
}

bool pow2(size_t v) { return v && !(v & (v - 1)); }

template <typename Kern>
int resident_blocks(Kern k)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kProbeThreads, 0) != cudaSuccess || b < 1)
        b = 1;
    return b;
}

}  // namespace

cudaError_t launch_probe(int kind, const uint32_t *table, size_t table_words, size_t window_words,
                         int reps, uint32_t *sink, int sm_count, cudaStream_t st,
                         unsigned long long *units, bool *bad_args)
{
    *bad_args = false;
    if (reps < 1 || reps > (1 << 20) || !sink) {
        *bad_args = true;
        return cudaSuccess;
    }
    int blocks = 0;
    const char *label = nullptr;
    switch (kind) {
    case BD_PROBE_GATHER:
        if (!table || !pow2(table_words) || !pow2(window_words) || window_words < 32 ||
            window_words > table_words || table_words > ((size_t)1 << 31)) {
            *bad_args = true;
            return cudaSuccess;
        }
        blocks = sm_count * resident_blocks(probe_gather_kernel);
        probe_gather_kernel<<<blocks, kProbeThreads, 0, st>>>(
            table, (uint32_t)(table_words - 1), (uint32_t)(window_words - 1), reps, sink);
        *units = (unsigned long long)blocks * kProbeThreads * reps * kLoadsPerWindow;
        label = "probe_gather";
        break;
    case BD_PROBE_L1_SECTORS:
        if (!table || !pow2(table_words) || table_words < 4 * (size_t)kL1WindowVec ||
            table_words > ((size_t)1 << 31) || (reinterpret_cast<uintptr_t>(table) & 15)) {
            *bad_args = true;
            return cudaSuccess;
        }
        blocks = sm_count * resident_blocks(probe_l1_kernel);
        probe_l1_kernel<<<blocks, kProbeThreads, 0, st>>>(
            reinterpret_cast<const uint4 *>(table), (uint32_t)(table_words / 4 - 1), reps, sink);
        // sectors: per warp and rep kL1Unroll requests of 512 B = 16 sectors
        *units = (unsigned long long)blocks * (kProbeThreads / 32) * reps * kL1Unroll * 16;
        label = "probe_l1";
        break;
    case BD_PROBE_POPC:
        blocks = sm_count * resident_blocks(probe_popc_kernel);
        probe_popc_kernel<<<blocks, kProbeThreads, 0, st>>>(reps, sink);
        label = "probe_popc";
        break;
    case BD_PROBE_FFMA:
        blocks = sm_count * resident_blocks(probe_ffma_kernel);
        probe_ffma_kernel<<<blocks, kProbeThreads, 0, st>>>(reps, sink);
        label = "probe_ffma";
        break;
    case BD_PROBE_MUFU:
        blocks = sm_count * resident_blocks(probe_mufu_kernel);
        probe_mufu_kernel<<<blocks, kProbeThreads, 0, st>>>(reps, sink);
        label = "probe_mufu";
        break;
    default:
        *bad_args = true;
        return cudaSuccess;
    }
    if (kind != BD_PROBE_GATHER && kind != BD_PROBE_L1_SECTORS)
        *units = (unsigned long long)blocks * kProbeThreads * reps * 8 * kChains;
    trace_kernel(st, label);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace bd
