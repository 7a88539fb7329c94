// Brute-force Hamming matching kernels with a fused top-2 and ratio test
// (Sec. IV-C nearest-neighbour matching): one query per thread, 128 queries
// per CTA, the train set split across CTAs into slices merged by the last
// CTA of each query block (the body is in match_dev.cuh).
#include <string.h>

#include "match_dev.cuh"

namespace bd {
namespace {

constexpr int QB = 128;   // queries per CTA (one per thread)
constexpr int TT = 256;   // train descriptors per shared-memory tile

// programmatic launch: wait for the kernel that wrote the descriptors
template <int NW>
__device__ __forceinline__ void match_cta(uint4 *tile, const uint32_t *__restrict__ q, int nq,
                                          const uint32_t *__restrict__ t, int nt, int chunk,
                                          int nbits, int rnum, int rden, int bx, int by, int S,
                                          uint2 *__restrict__ partial,
                                          bd_match_result *__restrict__ out,
                                          unsigned int *__restrict__ arrivals, int &last_cta)
{
    dev::griddep_wait();
    dev::griddep_launch_dependents();
    dev::match_block<NW, QB, TT>(tile, q, nq, t, nt, chunk, nbits, rnum, rden, bx, by, S, partial,
                                 out, arrivals, last_cta);
}

template <int NW>
__global__ void __launch_bounds__(QB, NW == 16 ? 6 : 8) match_top2_kernel(const uint32_t *__restrict__ q, int nq,
                                                        const uint32_t *__restrict__ t, int nt,
                                                        int chunk, int nbits, int rnum, int rden,
                                                        uint2 *__restrict__ partial,
                                                        bd_match_result *__restrict__ out,
                                                        unsigned int *__restrict__ arrivals)
{
    __shared__ int last_cta;
    __shared__ uint4 tile[TT * NW / 4];
    match_cta<NW>(tile, q, nq, t, nt, chunk, nbits, rnum, rden, blockIdx.x, blockIdx.y,
                  (int)gridDim.y, partial, out, arrivals, last_cta);
}

// Several matchings in one launch: job j owns CTAs [begin_j, begin_j +
// qblocks_j * S_j) of a 1-D grid.
struct MatchJobDev {
    const uint32_t *q, *t;
    bd_match_result *out;
    uint2 *partial;
    unsigned int *arrivals;
    int nq, nt, nbits, rnum, rden, S, chunk, qblocks, begin;
};

struct MatchJobsDev {
    int n;
    MatchJobDev j[BD_MATCH_MAX_JOBS];
};

__global__ void __launch_bounds__(QB, 6) match_multi_kernel(const __grid_constant__ MatchJobsDev J)
{
    __shared__ int last_cta;
    __shared__ uint4 tile[TT * 16 / 4];
    int k = 0;
    while (k + 1 < J.n && (int)blockIdx.x >= J.j[k + 1].begin)
        ++k;
    const MatchJobDev &b = J.j[k];
    const int local = (int)blockIdx.x - b.begin;
    const int bx = local % b.qblocks, by = local / b.qblocks;
    if (b.nbits == 256)
        match_cta<8>(tile, b.q, b.nq, b.t, b.nt, b.chunk, b.nbits, b.rnum, b.rden, bx, by, b.S,
                     b.partial, b.out, b.arrivals, last_cta);
    else
        match_cta<16>(tile, b.q, b.nq, b.t, b.nt, b.chunk, b.nbits, b.rnum, b.rden, bx, by, b.S,
                      b.partial, b.out, b.arrivals, last_cta);
}

void plan(int nq, int nt, int sm_count, int &S, int &chunk)
{
    const int qblocks = (nq + QB - 1) / QB;
    const int target = 8 * sm_count;
    S = (target + qblocks - 1) / qblocks;
    // slices of at least 16 train descriptors: small matchings spread over
    // more CTAs finish sooner (1000 x 1000: 16 -> 50.7 us plain step, 32 ->
    // 51.5, 128 -> 54.5)
    const int max_split = (nt + 15) / 16;
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
    cudaError_t e = launch_pdl(nbits == 256 ? match_top2_kernel<8> : match_top2_kernel<16>, grid,
                               dim3(QB), 0, st, q, nq, t, nt, chunk, nbits, ratio_num, ratio_den,
                               partial, out, arrivals);
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "match_top2");
    note_launches(1);
    return cudaGetLastError();
}

size_t match_batch_scratch_bytes(const bd_match_job *jobs, int n, int sm_count)
{
    size_t tot = 0;
    for (int k = 0; k < n; ++k)
        if (jobs[k].nq > 0)
            tot += match_scratch_bytes(jobs[k].nq, jobs[k].nt, jobs[k].nbits, sm_count);
    return tot;
}

int match_batch_query_blocks(const bd_match_job *jobs, int n)
{
    int tot = 0;
    for (int k = 0; k < n; ++k)
        tot += match_query_blocks(jobs[k].nq);
    return tot;
}

cudaError_t launch_match_batch(const bd_match_job *jobs, int n, void *scratch, int sm_count,
                               cudaStream_t st, unsigned int *arrivals)
{
    MatchJobsDev J;
    memset(&J, 0, sizeof(J));
    int blocks = 0, m = 0;
    char *sc = (char *)scratch;
    unsigned int *arr = arrivals;
    for (int k = 0; k < n; ++k) {
        const bd_match_job &a = jobs[k];
        if (a.nq <= 0)
            continue;
        MatchJobDev &b = J.j[m++];
        b.q = a.q;
        b.t = a.t;
        b.out = a.out;
        b.nq = a.nq;
        b.nt = a.nt;
        b.nbits = a.nbits;
        b.rnum = a.ratio_num;
        b.rden = a.ratio_den;
        plan(a.nq, a.nt, sm_count, b.S, b.chunk);
        b.qblocks = match_query_blocks(a.nq);
        b.begin = blocks;
        b.partial = (uint2 *)sc;
        b.arrivals = arr;
        sc += match_scratch_bytes(a.nq, a.nt, a.nbits, sm_count);
        arr += b.qblocks;
        blocks += b.qblocks * b.S;
    }
    J.n = m;
    if (m == 0)
        return cudaSuccess;
    cudaError_t e = launch_pdl(match_multi_kernel, dim3(blocks), dim3(QB), 0, st, J);
    if (e != cudaSuccess)
        return e;
    trace_kernel(st, "match_multi");
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
