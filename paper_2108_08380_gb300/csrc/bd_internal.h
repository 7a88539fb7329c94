// Internal declarations of the sm_103a descriptor library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bindesc.h"

// ---------------------------------------------------------------------------
// limits and constants
// ---------------------------------------------------------------------------
namespace bd {

constexpr int kPatch = 32;          // patch side (Sec. III-A: 32x32 patches)
constexpr int kHistDim = 128;       // 4x4 cells x 8 orientation bins
constexpr int kMaxImageSide = 32767;
constexpr int kMaxAngleBins = 64;
constexpr int kMaxLevels = 16;
constexpr int kMatchIdxBits = 22;   // train index bits in a packed (distance, index) key
constexpr uint32_t kMatchIdxMask = (1u << kMatchIdxBits) - 1u;
// bounded spin-waits: iterations before a kernel gives up and raises BD_FLAG_TIMEOUT
constexpr uint32_t kSpinLimit = 1u << 26;

// integral-image tiling
constexpr int kIiTileRows = 32;
constexpr int kIiTileCols = 128;

// device status block: [0] flags (uint32 in a u64 slot), [1] rescued-bit counter
struct DeviceStatus {
    unsigned long long flags;
    unsigned long long rescued;
};

}  // namespace bd

// ---------------------------------------------------------------------------
// host-side objects behind the opaque ABI handles
// ---------------------------------------------------------------------------
namespace bd {
// one recorded CUDA event with the name of the kernel that ended before it
// ("begin" marks the start of an ABI call)
struct TraceMark {
    cudaEvent_t ev;
    const char *label;
};
}  // namespace bd

struct bd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    bd::DeviceStatus *status = nullptr;  // device
    void *scratch = nullptr;             // device, grows on demand
    size_t scratch_bytes = 0;
    unsigned int *arrivals = nullptr;    // device, zeroed per-block arrival counters (matching)
    int arrivals_cap = 0;
    std::string err;
    // tracing (bd_trace_*)
    bool trace = false;
    std::vector<cudaEvent_t> trace_pool;  // events owned by the context
    size_t trace_next = 0;
    std::vector<bd::TraceMark> marks;     // marks of the calls since the last reset
};

struct bd_bad_params {
    bd_ctx *ctx = nullptr;
    int nbits = 0, nbins = 0, nlevels = 0;
    int32_t thr_den = 1;
    float angle_scale = 0.f;  // float(NB / (2 pi)), applied in IEEE single precision
    float level_mid[bd::kMaxLevels] = {};  // float(sqrt(s_l s_{l+1}))
    // host copies (for bd_bad_params_table)
    int32_t *h_offsets = nullptr;  // [L][NB][K][4] centre offsets
    int32_t *h_sides = nullptr;    // [L][K]
    // device tables
    short4 *d_box = nullptr;       // [L][NB][2K] boxes (x, y, side, id), sorted by (y, side, x)
    int *d_thr = nullptr;          // [L][K] integer threshold on sum1 - sum2
    short4 *d_patch_box = nullptr; // [K] top-left corners in the 32x32 patch frame (training)
    int *d_patch_side = nullptr;   // [K] box sides in the patch frame
};

struct bd_hs_params {
    bd_ctx *ctx = nullptr;
    int nbits = 0;
    int precision = BD_HS_FP32;
    int variant = 0;  // BD_HS_VARIANT_* flags
    float spacing = 1.f;
    float *d_W = nullptr;           // [128][K] FP32 (row-major, as given)
    float *d_Wt = nullptr;          // [K][128] FP32 (per-bit rows, for the FP32 re-check)
    __nv_bfloat16 *d_Wt16_hi = nullptr;  // [K][128] BF16 head of W^T (tensor-core B operand, K-major)
    __nv_bfloat16 *d_Wt16_lo = nullptr;  // [K][128] BF16 tail: W - hi rounded to BF16
    bool w_has_lo = false;               // false when W is exactly BF16
    float *d_bias = nullptr;        // [K]
    float *d_band = nullptr;        // [K] rescue band per bit
    CUtensorMap tmap_w_hi, tmap_w_lo;  // TMA maps of the two BF16 parts, box 64 x 128
    bool tmap_ok = false;
};

// ---------------------------------------------------------------------------
// helpers shared by the .cu files
// ---------------------------------------------------------------------------
namespace bd {

bd_status set_err(bd_ctx *ctx, bd_status s, const char *fmt, ...);
bd_status cuda_err(bd_ctx *ctx, cudaError_t e, const char *what);
bd_status ensure_scratch(bd_ctx *ctx, size_t bytes);

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// process-wide count of kernels this library has launched (bd_kernel_launches)
void note_launches(int k);

// Tracing.  An ABI call opens a TraceScope on its thread; launch helpers call
// trace_kernel(stream, name) after each kernel.  With tracing on, each mark
// records a CUDA event on the stream.  Under graph capture the scope writes
// its marks (events it creates) into `captured` instead, and the owner replays
// them into the context's mark list at each graph launch.
struct TraceScope {
    TraceScope(bd_ctx *ctx, cudaStream_t st, std::vector<TraceMark> *captured = nullptr);
    ~TraceScope();
    bd_ctx *ctx;
    std::vector<TraceMark> *captured;
    TraceScope *prev;
};
void trace_kernel(cudaStream_t st, const char *label);

// TMA descriptor encoding through the driver entry point (no -lcuda needed).
bool encode_tmap_2d_bf16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer);
bool encode_tmap_2d_u8(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                       uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer);

// ---------------------------------------------------------------------------
// kernel launchers (each returns cudaGetLastError() of its launch)
// ---------------------------------------------------------------------------
struct IntegralScratch {
    uint32_t *colsum;   // [nty][w]
    uint32_t *rowsum;   // [h][ntx]
    uint32_t *tiletot;  // [nty][ntx]
};
size_t integral_scratch_bytes(int w, int h);
IntegralScratch integral_scratch_carve(void *base, int w, int h);
cudaError_t launch_integral(const uint8_t *img, int w, int h, int pitch, uint32_t *ii,
                            int ii_stride, const IntegralScratch &s, cudaStream_t st);

cudaError_t launch_bad_gather(const bd_bad_params *p, const uint32_t *ii, int ii_stride, int w,
                              int h, const bd_keypoint *kps, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st);

cudaError_t launch_hs_warp(const bd_hs_params *p, const uint8_t *img, int w, int h, int pitch,
                           const bd_keypoint *kps, int n, float *patches, DeviceStatus *status,
                           cudaStream_t st, int sm_count);
cudaError_t launch_hs_hist_patches(const float *patches, int n, float *hist, cudaStream_t st,
                                   int sm_count,
                                   float *norm_out = nullptr);
cudaError_t launch_hs_hist_image(const bd_hs_params *p, const uint8_t *img, int w, int h, int pitch,
                                 const bd_keypoint *kps, int n, float *hist,
                                 DeviceStatus *status, cudaStream_t st,
                                 int sm_count);
cudaError_t launch_hs_proj_fp32(const bd_hs_params *p, const float *hist, int n, uint32_t *out,
                                cudaStream_t st, const bd_keypoint *kps);
// raises the projection kernel's dynamic shared-memory limit (per device, at set-up)
cudaError_t prepare_hs_proj_tc();
// a16 (optional): the histograms already split into the BF16 operand image
// (split_offset), with nz[k] != 0 for rows that are not all zero; the kernel
// then copies each block's operands instead of converting the FP32 rows.
// relaxed (optional, [n][K] FP32): also writes tanh(m inv_t) of each margin
// m as the tensor cores give it (the training path's relaxed responses).
cudaError_t launch_hs_proj_tc(const bd_hs_params *p, const float *hist, int n, uint32_t *out,
                              DeviceStatus *status, cudaStream_t st, const bd_keypoint *kps,
                              const uint8_t *a16 = nullptr, const uint8_t *nz = nullptr,
                              float *relaxed = nullptr, float inv_t = 1.0f);

size_t match_scratch_bytes(int nq, int nt, int nbits, int sm_count);
// tensor-core matching: scratch for the FP8 codes and split partials
size_t match_tc_scratch_bytes(int nq, int nt, int nbits, int sm_count);
int match_tc_query_blocks(int nq);
cudaError_t launch_match_tc(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                            int nbits, int ratio_num, int ratio_den, bd_match_result *out,
                            void *scratch, cudaStream_t st, unsigned int *arrivals);
// same, returning the raw top-2 keys (distance << 22 | index) per query;
// mine != 0 (hard-negative mining, nq == nt > 1): the nearest key among the
// columns other than the query's own, in .x (.y is not the second nearest)
cudaError_t launch_match_tc_keys(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                                 int nbits, int ratio_num, int ratio_den, bd_match_result *out,
                                 uint2 *raw_keys, void *scratch, cudaStream_t st,
                                 unsigned int *arrivals, int mine);
// measurement probes (bd_probe); bad_args set when the geometry is refused
cudaError_t launch_probe(int kind, const uint32_t *table, size_t table_words, size_t window_words,
                         int reps, uint32_t *sink, int sm_count, cudaStream_t st,
                         unsigned long long *units, bool *bad_args);

// several POPC matchings in one launch (bd_match_batch); jobs already validated
size_t match_batch_scratch_bytes(const bd_match_job *jobs, int n, int sm_count);
int match_batch_query_blocks(const bd_match_job *jobs, int n);
cudaError_t launch_match_batch(const bd_match_job *jobs, int n, void *scratch, int sm_count,
                               cudaStream_t st, unsigned int *arrivals);
// mnn[i] = fwd[i].idx if rev[fwd[i].idx].idx == i, else -1 (rev: nearest queries of t)
cudaError_t launch_mnn_cross(const bd_match_result *fwd, const bd_match_result *rev, int nq,
                             int32_t *mnn, cudaStream_t st);

// feature selection round: scratch = state + candidate-major int16 keys (J x 3n)
size_t select_scratch_bytes_pass(int n, int J, int jn);
size_t select_scratch_bytes(int n, int J);
cudaError_t launch_select_feature(const uint8_t *patches, int n, const int32_t *sap,
                                  const int32_t *san, int tau, const int32_t *cand_xy,
                                  const int32_t *cand_side, int max_side, int J, int32_t *theta_q,
                                  int64_t *loss, int32_t *best, void *scratch, size_t scratch_bytes,
                                  cudaStream_t st);

int match_query_blocks(int nq);
// arrivals: one zero-initialised counter per query block (ctx-owned; each call leaves them zero)
cudaError_t launch_match(const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits,
                         int ratio_num, int ratio_den, bd_match_result *out, void *scratch,
                         int sm_count, cudaStream_t st, unsigned int *arrivals);

}  // namespace bd

// ---------------------------------------------------------------------------
// device-side PTX helpers (sm_100 family: mbarrier, TMA, tcgen05)
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
#include <utility>

namespace bd {

// Programmatic dependent launch: the kernel may be scheduled while the
// previous kernel of the stream is still running (its launch and prologue
// overlap that kernel's tail).  Such a kernel calls dev::griddep_wait()
// before it touches global memory that earlier work reads or writes; the
// wait returns once the previous grid has completed and its writes are
// visible, so stream order is kept.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace bd

namespace bd {
namespace dev {

// griddepcontrol (sm_90+): wait for the previous grid of the stream to
// complete and its memory to be visible; allow the next grid to launch.
// Relaxed response tanh(x) of the training path from its definition,
// (1 - u) / (1 + u) with u = e^(-2|x|) in (0, 1] and the sign of x: one
// exponential and one fast division.  The error is absolute (u's relative
// error, about 2^-21, times 2u / (1 + u)^2 <= 1/2: below 5e-7), far inside the
// training tolerances; near 0 it does not keep tanh(x) ~ x relatively.
__device__ __forceinline__ float tanh_relaxed(float x)
{
    const float u = __expf(-2.0f * fabsf(x));
    return copysignf(__fdividef(1.0f - u, 1.0f + u), x);
}

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void raise_flag(DeviceStatus *st, unsigned long long f)
{
    if (st)
        atomicOr(&st->flags, f);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; gives up after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int c0, int c1,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// Non-tensor bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing `bytes` of the mbarrier's transaction count.
__device__ __forceinline__ void bulk_load(void *smem_dst, const void *gsrc, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Byte offset of value v (0..127) of histogram row k in the pre-split BF16
// operand image the tcgen05 projection copies per block of 128 rows: block
// k / 128 at 64 KB steps holds [head K0][head K1][tail K0][tail K1] tiles of
// 128 rows x 128 bytes in the 128-byte-swizzled K-major layout (16-byte
// chunk c of row r at position c ^ (r mod 8)); add 32 KB for the tail.
__device__ __forceinline__ size_t split_offset(size_t k, int v)
{
    const int r = (int)(k & 127), h = v >> 6, c = (v & 63) >> 3, e = v & 7;
    return (k >> 7) * 65536 + (size_t)h * 16384 + (size_t)r * 128 + (size_t)(((c ^ (r & 7)) << 4) + e * 2);
}

// Writes value x of row k, v into the pre-split image: BF16 head and tail
// (x = hi + lo + O(2^-16 |x|)).
__device__ __forceinline__ void split_store(uint8_t *a16, size_t k, int v, float x)
{
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    const size_t o = split_offset(k, v);
    *reinterpret_cast<__nv_bfloat16 *>(a16 + o) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(a16 + o + 32768) = lo;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *smem_slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(smem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand stored in the 128-byte
// swizzled layout TMA writes (rows of 128 B, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, M x N tile.
__host__ __device__ constexpr uint32_t umma_idesc_bf16_f32(int M, int N)
{
    return (1u << 4)                       // D format: F32
           | (1u << 7)                     // A format: BF16
           | (1u << 10)                    // B format: BF16
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor: kind::f8f6f4 with E4M3 A and B, FP32 accumulator,
// both operands K-major, M x N tile.
__host__ __device__ constexpr uint32_t umma_idesc_e4m3_f32(int M, int N)
{
    return (1u << 4)                       // D format: F32
           | (0u << 7)                     // A format: E4M3
           | (0u << 10)                    // B format: E4M3
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Generic-proxy writes to shared memory made visible to the async proxy
// (tensor-core operand reads) of the CTA; then a barrier before the MMA.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 32 consecutive 32-bit TMEM columns: thread t of the warp gets
// lane (warp's lane base + t), columns [col, col+32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 lanes x 64 consecutive 32-bit TMEM columns in one load, then the wait
// (in the same statement, so no use of r can be scheduled before it).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
        "%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
}

// Keypoint validity and quantisation, in IEEE single precision with explicit
// round-to-nearest intrinsics so no multiply-add is contracted.
__device__ __forceinline__ bool kp_valid(const bd_keypoint &k)
{
    const float lim = 1048576.0f;
    if (!isfinite(k.x) || !isfinite(k.y) || !isfinite(k.scale) || !isfinite(k.angle))
        return false;
    if (fabsf(k.x) > lim || fabsf(k.y) > lim || fabsf(k.angle) > lim)
        return false;
    return k.scale > 0.0f && k.scale <= 1024.0f;
}

__device__ __forceinline__ int round_coord(float v) { return (int)floorf(__fadd_rn(v, 0.5f)); }

}  // namespace dev
}  // namespace bd
#endif
