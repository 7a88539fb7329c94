/*
 * bindesc.h -- C ABI of the GB300 (sm_103a) library for the BAD and HashSIFT
 * binary descriptors and brute-force Hamming matching of
 *   I. Suarez, J. M. Buenaposada, L. Baumela, "Revisiting Binary Local Image
 *   Description for Resource Limited Devices", IEEE RA-L 2021.
 *
 * The calls follow the paper's statement of the problem: an image, keypoints
 * (x, y, scale, angle) and learned descriptor parameters give packed binary
 * descriptors (Sec. III-A, Eq. 1 stumps h = +1 iff f <= theta; Sec. III-B,
 * D = sgn(B [f; 1])); two descriptor sets give nearest / second-nearest
 * matches (Sec. IV-C, Sec. IV-F pipeline table).
 *
 * Conventions shared by every call
 *  - Only plain pointers and sizes cross this boundary.  Pointers named
 *    "host" are CPU memory; every other data pointer is CUDA device memory
 *    owned by the caller, which must stay valid until the work completes.
 *  - Work is enqueued asynchronously on the context's stream; the caller
 *    synchronises (or calls bd_sync_status) before reading results.
 *  - Every call returns a bd_status; nothing is thrown across the ABI.  On an
 *    error nothing has been enqueued and bd_last_error() says why.
 *  - Descriptors are packed little-endian bit vectors: bit k of a descriptor
 *    is bit (k % 32) of 32-bit word k / 32; bit value 1 is the paper's +1.
 *  - Images are 8-bit grayscale, row-major with a row pitch in bytes;
 *    1 <= w, h <= 32767 and 255*w*h < 2^32.
 *  - A keypoint is valid iff its four fields are finite, |x|,|y| <= 2^20,
 *    0 < scale <= 1024 and |angle| <= 2^20.  Pixel centres sit at integer
 *    coordinates, angles are radians, the image y axis points down.  An
 *    invalid keypoint gets an all-zero descriptor and raises
 *    BD_FLAG_INVALID_KEYPOINT in the device status word.
 */
#ifndef BINDESC_H
#define BINDESC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bd_status {
    BD_OK = 0,
    BD_ERR_INVALID = 1,      /* bad argument; nothing was enqueued */
    BD_ERR_CUDA = 2,         /* a CUDA call failed */
    BD_ERR_NOMEM = 3,        /* device memory could not be allocated */
    BD_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    BD_ERR_DEVICE_CHECK = 5, /* a kernel flagged its input (see the flags) */
    BD_ERR_UNSUPPORTED = 6   /* device or feature not supported by this build */
} bd_status;

/* Bits of the device status word returned by bd_sync_status. */
#define BD_FLAG_INVALID_KEYPOINT 0x1u
#define BD_FLAG_TIMEOUT 0x2u

/* Keypoint: pixel position, scale (1 = the 32x32 patch frame covers 32 px)
 * and orientation in radians. */
typedef struct bd_keypoint {
    float x, y, scale, angle;
} bd_keypoint;

/* Most matchings of one bd_match_batch call or of one batch plan. */
#define BD_MATCH_MAX_JOBS 8

/* One query's result: train index of the nearest neighbour (-1 if the train
 * set is empty), its Hamming distance d1, the second-smallest distance d2
 * (nbits+1 when there is no second entry) and the ratio-test verdict. */
typedef struct bd_match_result {
    int32_t idx;
    uint16_t d1;
    uint16_t d2;
    uint8_t accept;
    uint8_t pad[3];
} bd_match_result;

typedef struct bd_ctx bd_ctx;
typedef struct bd_bad_params bd_bad_params;
typedef struct bd_hs_params bd_hs_params;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */

/* Creates a context on CUDA device `device` that enqueues on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The context owns a small
 * status block and a growable scratch area on that device.  Requires an
 * sm_103 device; otherwise BD_ERR_UNSUPPORTED. */
bd_status bd_create(int device, void *stream, bd_ctx **out);

/* Releases the context and its device memory (synchronising its stream).
 * Parameter sets and plans created from the context must be destroyed
 * first: they refer to it. */
void bd_destroy(bd_ctx *ctx);

/* Switches the stream later calls enqueue on. */
bd_status bd_set_stream(bd_ctx *ctx, void *stream);

/* Message of the last failed call on this context (static storage owned by
 * the context; valid until the next call). */
const char *bd_last_error(const bd_ctx *ctx);

/* Synchronises the context's stream, returns the device status flags
 * (BD_FLAG_*) raised since the last call in *flags (may be NULL) and clears
 * them.  Returns BD_ERR_TIMEOUT if BD_FLAG_TIMEOUT was raised,
 * BD_ERR_DEVICE_CHECK if any other flag was, else BD_OK. */
bd_status bd_sync_status(bd_ctx *ctx, uint32_t *flags);

/* Number of HashSIFT bits re-evaluated in FP32 since the last reset
 * (synchronises the stream).  reset != 0 zeroes the counter afterwards. */
bd_status bd_rescued_count(bd_ctx *ctx, uint64_t *count, int reset);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t bd_kernel_launches(void);

/* Tracing: with tracing on, every call records a CUDA event on its stream
 * when it starts and after each kernel it launches (a graph captured while
 * tracing is on records them at each replay).  bd_trace_read synchronises on
 * the last event and returns, for up to max consecutive mark pairs since the
 * last bd_trace_reset, the elapsed ms and the name of the kernel that ended
 * at the later mark ("begin" for the gap before a call).  Returns the number
 * of intervals written, or -1 on error. */
bd_status bd_trace_enable(bd_ctx *ctx, int on);
bd_status bd_trace_reset(bd_ctx *ctx);
int bd_trace_read(bd_ctx *ctx, int max, float *ms, const char **labels);

/* Grows the scratch area to at least `bytes` now, so that later calls of
 * that size allocate nothing (needed before capturing them in a CUDA graph). */
bd_status bd_reserve(bd_ctx *ctx, size_t bytes);

/* Scratch bytes the calls below need for the given sizes (host-side query). */
size_t bd_scratch_bytes_bad(int w, int h);
size_t bd_scratch_bytes_hashsift(int n);
size_t bd_scratch_bytes_match(int nq, int nt, int nbits);

/* ------------------------------------------------------------------------ */
/* BAD parameters (Sec. III-A)                                               */

/* Learned BAD parameters, copied from host memory and owned by the handle.
 *  nbits        256 or 512 (K weak descriptors).
 *  centres      host, nbits x 2 x 2 uint8: box centre (x, y) of box 1 and 2
 *               of pair k in the 32x32 patch frame (values 0..31; the frame
 *               centre is (16,16)).
 *  sides        host, nbits uint8 box sides s (1..64); both boxes of a pair
 *               share s (Sec. III-A: the two boxes of a pair have one size).
 *  thr_num      host, nbits int32; threshold theta_k = thr_num[k] / thr_den.
 *  thr_den      > 0 (1 for integer thresholds; 10 for the 0.1 grid of
 *               Sec. III-A, Alg. 2 discussion).
 *  n_angle_bins 1..64 orientation bins (32 in the benchmarks).
 *  level_scales host, n_levels strictly increasing pyramid scales in
 *               (0, 32]; a keypoint uses the level whose geometric-mean
 *               neighbourhood contains its scale.
 * The library builds, on the host, an integer table of every box's rotated
 * and scaled corner offsets per (level, angle bin) and uploads it. */
bd_status bd_bad_params_create(bd_ctx *ctx, int nbits, const uint8_t *centres,
                               const uint8_t *sides, const int32_t *thr_num, int32_t thr_den,
                               int n_angle_bins, const float *level_scales, int n_levels,
                               bd_bad_params **out);
void bd_bad_params_destroy(bd_bad_params *p);

/* Copies the host-side table out (for checking): for each level l, angle
 * bin b and bit k, offsets[((l*NB + b)*nbits + k)*4 + {0..3}] = centre offset
 * (dx1, dy1, dx2, dy2) of the two boxes from the keypoint's pixel, and
 * sides_out[l*nbits + k] = scaled side.  Buffers are host memory of
 * n_levels*NB*nbits*4 and n_levels*nbits int32. */
bd_status bd_bad_params_table(const bd_bad_params *p, int32_t *offsets, int32_t *sides_out);

/* ------------------------------------------------------------------------ */
/* HashSIFT parameters (Sec. III-B)                                          */

#define BD_HS_FP32 0        /* projection on CUDA cores in FP32 */
#define BD_HS_BF16_RESCUE 1 /* tcgen05 BF16 x BF16 -> FP32 (split head/tail), FP32 re-check near 0 */
/* SIFT variants of the histogram before hashing (bd_hs_params_set_variant) */
#define BD_HS_VARIANT_TRILINEAR 1 /* votes shared by the 2 x 2 nearest cells */
#define BD_HS_VARIANT_CLIP 2      /* L2-normalise, clip at 0.2, renormalise */
#define BD_HS_VARIANT_ROOT 4      /* RootSIFT: L1-normalise, square roots */

/* Learned hash B = [W^T | b], copied from host memory.
 *  nbits     256 or 512.
 *  W         host, 128 x nbits float, row-major (W[i*nbits + k]).
 *  bias      host, nbits float (the last column of B).
 *  spacing   patch pixel step in units of the keypoint scale (> 0, <= 16).
 *  precision BD_HS_FP32 or BD_HS_BF16_RESCUE.
 *  band      BF16 mode: f and W are split into BF16 head + tail and the
 *            tensor cores accumulate f_hi W_hi + f_lo W_hi + f_hi W_lo in FP32;
 *            bits whose margin |W_k.f + b_k| falls below the band are
 *            recomputed in FP32 exactly as the FP32 mode computes them.
 *            band < 0 selects the per-bit bound 2^-13 * ||W_k||_2, which covers
 *            the split's rounding and both FP32 accumulations for unit-norm f,
 *            so the two modes give identical bits; band >= 0 is used as given
 *            for every bit (a smaller band may differ from FP32 mode). */
bd_status bd_hs_params_create(bd_ctx *ctx, int nbits, const float *W, const float *bias,
                              float spacing, int precision, float band, bd_hs_params **out);
/* Selects SIFT variants of the histogram for the descriptor calls that use
 * p (the paper's HashSIFT hashes the plain histogram; it names RootSIFT as
 * the key improvement of histogram descriptors, Sec. II): any OR of
 * BD_HS_VARIANT_TRILINEAR (each vote shared by the two nearest cell rows and
 * cell columns, cell c centred at pixel 8c + 3.5 with weight 1 - |d| / 8),
 * BD_HS_VARIANT_CLIP (Lowe's 0.2 clip with renormalisation) and
 * BD_HS_VARIANT_ROOT (L1 normalisation and square roots); applied in that
 * order.  0 restores the plain histogram.  bd_hashsift_describe supports all
 * of them; bd_batch_create refuses parameters with TRILINEAR
 * (BD_ERR_UNSUPPORTED).  Errors: BD_ERR_INVALID for other bits. */
bd_status bd_hs_params_set_variant(bd_hs_params *p, int flags);

void bd_hs_params_destroy(bd_hs_params *p);

/* ------------------------------------------------------------------------ */
/* Work                                                                      */

/* Integral image (Sec. III-A): ii[y*ii_stride + x] = sum of img over
 * [0,y) x [0,x), for 0 <= y <= h, 0 <= x <= w; ii_stride >= w+1 entries. */
bd_status bd_integral(bd_ctx *ctx, const uint8_t *img, int w, int h, int pitch, uint32_t *ii,
                      int ii_stride);

/* BAD descriptors (Sec. III-A) of n keypoints: out is n x nbits/32 words.
 * Builds the integral image in scratch, then one warp per keypoint gathers
 * the box sums of every pair and packs the stump outputs. */
bd_status bd_bad_describe(bd_ctx *ctx, const bd_bad_params *p, const uint8_t *img, int w, int h,
                          int pitch, const bd_keypoint *kps, int n, uint32_t *out);

/* 32x32 FP32 patches of n keypoints (Sec. III-A/III-B: patches normalised to
 * 32x32): patches is n x 1024 floats, pixel (i, j) at [i*32 + j], sampled
 * bilinearly (clamp to edge) at (x,y) + scale*spacing*R(angle)(j-15.5, i-15.5). */
bd_status bd_hashsift_warp(bd_ctx *ctx, const bd_hs_params *p, const uint8_t *img, int w, int h,
                           int pitch, const bd_keypoint *kps, int n, float *patches);

/* L2-normalised 128-bin gradient-orientation histograms (Sec. III-B, "SIFT
 * features") of n FP32 patches (n x 1024): hist is n x 128 floats, index
 * (cell_row*4 + cell_col)*8 + orientation_bin. */
bd_status bd_hashsift_hist(bd_ctx *ctx, const float *patches, int n, float *hist);

/* Hash bits D = sgn(W^T f + b) (Sec. III-B) of n FP32 histograms (n x 128):
 * out is n x nbits/32 words.  Uses the precision chosen in p; the BF16 path
 * needs hist 16-byte aligned. */
bd_status bd_hashsift_project(bd_ctx *ctx, const bd_hs_params *p, const float *hist, int n,
                              uint32_t *out);

/* Whole HashSIFT descriptor of n keypoints: warp + histogram fused in one
 * kernel, then the projection.  hist_out (n x 128 floats, 16-byte aligned)
 * may be NULL. */
bd_status bd_hashsift_describe(bd_ctx *ctx, const bd_hs_params *p, const uint8_t *img, int w,
                               int h, int pitch, const bd_keypoint *kps, int n, uint32_t *out,
                               float *hist_out);

/* Brute-force Hamming matching (Sec. IV-C nearest neighbour): for each of the
 * nq query descriptors, the nearest train descriptor (lowest index among
 * equal distances), its distance d1, the second-smallest distance d2 over
 * the remaining train entries, and accept = ratio_den*d1 < ratio_num*d2.
 * q: nq x nbits/32 words; t: nt x nbits/32 words (both 16-byte aligned);
 * out: nq entries (4-byte aligned).
 * nbits 256 or 512; 0 <= nt < 2^22; 0 < ratio_num <= ratio_den. */
bd_status bd_match(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits,
                   int ratio_num, int ratio_den, bd_match_result *out);

/* ------------------------------------------------------------------------ */
/* Batched description (many images in one persistent launch)               */

typedef struct bd_batch bd_batch;

/* Launch shape of the batched kernel (picked by bd_batch_autotune).
 *  bad_kp_per_item  keypoints per BAD work item (multiple of 4, 4..256)
 *  ctas_per_sm      resident CTAs per SM of the persistent grid (0 = the most
 *                   that fit)
 *  hs_first         where the HashSIFT items (which depend on nothing) sit in
 *                   the queue: 0 after the BAD items, 1 between the integral
 *                   tiles and the BAD items, 2 one grid's worth there and the
 *                   rest after the BAD items, 3 spread evenly among the BAD
 *                   items, 4 before the integral tiles, 5 spread evenly among
 *                   the integral tiles and the BAD items.
 *  hs_kp_per_item   HashSIFT keypoints per work item: 1 = the CTA's four warps
 *                   share each keypoint (lower latency, for few keypoints),
 *                   4 = one keypoint per warp (higher throughput).
 *  proj_fused       0: the tcgen05 projection kernel hashes the histograms
 *                   after the persistent kernel (the parameters' precision);
 *                   1: the persistent kernel projects them itself, 32 x 32
 *                   tiles in FP32 in the FP32 path's summation order (the
 *                   same bits as both paths; no rescue, one launch fewer, for
 *                   small batches).
 *  bad_shared       0: one BAD keypoint per warp; 1: the CTA's four warps share
 *                   each keypoint, a quarter of its words each (one
 *                   integral-image window per CTA in L1 instead of four);
 *                   2: warp pairs share a keypoint, half its words each (two
 *                   keypoints at a time, two windows per CTA).
 *  proj_half        with proj_fused = 1: 0 projects 32 keypoints x 32 bits
 *                   per work item, 1 32 keypoints x 16 bits (twice the items,
 *                   half the chain each; the same bits). */
typedef struct bd_batch_config {
    int bad_kp_per_item;
    int ctas_per_sm;
    int hs_first;
    int hs_kp_per_item;
    int proj_fused;
    int bad_shared;
    int proj_half;
} bd_batch_config;

/* Plans the description of n_img images with BAD and/or HashSIFT (either
 * params may be NULL, not both).  w, h, pitch: host arrays of n_img image
 * sizes; kp_offsets: host array of n_img+1 non-decreasing keypoint offsets
 * (keypoints of image i are kps[kp_offsets[i] .. kp_offsets[i+1])).  The
 * plan allocates, once, the integral tables of all images, their carries,
 * the histograms and the work-queue counters. */
bd_status bd_batch_create(bd_ctx *ctx, const bd_bad_params *bad, const bd_hs_params *hs,
                          int n_img, const int *w, const int *h, const int *pitch,
                          const int *kp_offsets, bd_batch **out);
void bd_batch_destroy(bd_batch *b);
bd_status bd_batch_set_config(bd_batch *b, const bd_batch_config *cfg);
bd_status bd_batch_get_config(const bd_batch *b, bd_batch_config *cfg);

/* Describes the whole batch: one persistent kernel builds every integral
 * image (one pass over each image: a tile publishes its column sums, row
 * sums and total, waits for those of the tiles to its left and above, then
 * writes its table entries) and computes every BAD descriptor and HashSIFT
 * histogram from one work queue, then the projection kernel hashes all
 * histograms.
 *  imgs     host array of n_img device pointers to the images
 *  kps      device, all keypoints (kp_offsets[n_img] of them)
 *  bad_out  device, n x bad_nbits/32 words, or NULL to skip BAD
 *  hs_out   device, n x hs_nbits/32 words, or NULL to skip HashSIFT
 *  use_graph != 0: the launches are captured once into a CUDA graph (per set
 *           of pointers) and replayed on later calls. */
bd_status bd_describe_batch(bd_ctx *ctx, bd_batch *b, const uint8_t *const *imgs,
                            const bd_keypoint *kps, uint32_t *bad_out, uint32_t *hs_out,
                            int use_graph);

/* Times every candidate launch shape (reps launches each after a warm-up
 * launch, CUDA events on the context's stream), re-times the four fastest
 * with 3 x reps launches, keeps the fastest of those in the plan and returns
 * it (best_ms: its mean time per launch). */
bd_status bd_batch_autotune(bd_ctx *ctx, bd_batch *b, const uint8_t *const *imgs,
                            const bd_keypoint *kps, uint32_t *bad_out, uint32_t *hs_out,
                            int reps, bd_batch_config *best, float *best_ms);

/* Item timeline of the persistent kernel (tracing aid).  One record per work
 * item of the last bd_describe_batch, indexed by queue position; times are
 * the GPU's global nanosecond timer read by the CTA's thread 0:
 *  t_claim  the item was taken from the queue
 *  t_ready  its dependency counters were complete (= t_claim without a wait)
 *  t_end    its work was done, before it published its own completion
 * so an item's t_ready is never below the t_end of an item it waited on,
 * except that an integral tile waits for what the tiles to its left and
 * above publish early in their work (after their t_claim, before their
 * t_end). */
enum {
    BD_ITEM_II_TILE = 0,    /* integral tile (one pass: aggregates, wait, table) */
    BD_ITEM_HASHSIFT = 1,   /* HashSIFT histogram(s) */
                            /* 2: not used */
    BD_ITEM_BAD = 3,        /* BAD descriptors of a keypoint group */
    BD_ITEM_PROJ = 4,       /* fused projection tile (proj_fused) */
    BD_ITEM_MATCH = 5       /* matching of a query block against a train slice */
};
typedef struct bd_batch_event {
    int32_t kind;    /* BD_ITEM_* */
    int32_t index;   /* index among the items of its kind */
    int32_t sm;      /* SM that ran it */
    int32_t cta;     /* CTA of the persistent grid */
    uint64_t t_claim, t_ready, t_end;
} bd_batch_event;

/* Matchings done by the batched launch itself (Sec. IV-C nearest-neighbour
 * matching with the ratio test): after describing, the descriptors of
 * query_image are matched against those of train_image, read from the same
 * call's outputs; each job writes n_kp(query_image) records to out, exactly
 * the records bd_match returns on those descriptors (nbits = the plan's BAD
 * or HashSIFT length).  A job whose query image has no keypoints writes
 * nothing. */
enum { BD_DESC_BAD = 0, BD_DESC_HASHSIFT = 1 };
typedef struct bd_batch_match {
    int desc;                  /* BD_DESC_BAD or BD_DESC_HASHSIFT */
    int query_image, train_image;
    int ratio_num, ratio_den;  /* 0 < ratio_num <= ratio_den */
    bd_match_result *out;      /* device, n_kp(query_image) records, 4-byte aligned */
} bd_batch_match;

/* Sets the plan's matchings (host array, copied; 0 <= n_jobs <=
 * BD_MATCH_MAX_JOBS, 0 clears them).  BAD jobs need BAD parameters in the
 * plan, HashSIFT jobs HashSIFT parameters; bd_describe_batch then refuses a
 * call without the outputs the jobs read (BD_ERR_INVALID).  When the
 * persistent kernel holds every descriptor the jobs read (BAD jobs only, or
 * proj_fused = 1), the matchings are its last work items, each waiting for
 * the descriptors of its two images; otherwise one matching launch follows
 * the projection. */
bd_status bd_batch_set_matches(bd_batch *b, const bd_batch_match *jobs, int n_jobs);

/* Limit, in nanoseconds of the GPU timer, of each dependency wait of the
 * persistent kernel (an item waiting for the items it reads: integral tiles,
 * histograms, descriptors of a matching); 0 restores the default of 2 s.
 * A wait that runs out raises BD_FLAG_TIMEOUT (bd_sync_status then returns
 * BD_ERR_TIMEOUT), the item skips its work, every CTA still leaves the
 * queue, and the last one out resets the plan's counters, so the next call
 * starts clean; the outputs of the call that timed out are undefined.  A
 * short limit makes waits run out on purpose (a test of this error path).
 * Takes effect at the next bd_describe_batch (a captured graph is
 * re-captured). */
bd_status bd_batch_set_wait_limit(bd_batch *b, uint64_t ns);

/* enable != 0: later launches of the plan record the timeline (device buffer
 * owned by the plan; the graph is re-captured); 0 turns it off. */
bd_status bd_batch_set_timeline(bd_batch *b, int enable);
/* Waits for the context's stream and copies up to cap records of the last
 * launch to host memory `out`; *n = the number of items of that launch
 * (records past cap are not copied).  BD_ERR_INVALID when the timeline is off
 * or no launch recorded one. */
bd_status bd_batch_get_timeline(bd_batch *b, bd_batch_event *out, int cap, int *n);

/* ------------------------------------------------------------------------ */
/* Differentiable training step (relaxed descriptors, Sec. III-A Eq. 1,      */
/* Sec. III-B Eq. 3)                                                         */

typedef struct bd_train bd_train;

/* Plans a training step over n triplets of 32x32 FP32 patches.
 *  bad          BAD parameters: their box centres and sides, read in the
 *               32x32 patch frame, define the relaxed BAD responses (its
 *               integer thresholds are not used; theta is an input below).
 *  hs_bits      256 or 512 HashSIFT bits.
 *  temperature  T of the relaxations r = tanh(z / T), with z = (theta - f)/255
 *               for BAD (f a difference of box means, in intensity units) and
 *               z = W^T h + b for HashSIFT.
 *  tau_bad, tau_hs  margins of the two triplet ranking losses.
 * The plan owns the responses, hard codes, histograms and mining of the last
 * forward call, which the backward call reuses. */
bd_status bd_train_create(bd_ctx *ctx, const bd_bad_params *bad, int hs_bits, int n,
                          float temperature, float tau_bad, float tau_hs, bd_train **out);
void bd_train_destroy(bd_train *tr);

/* Forward: patches [3][n][32][32] FP32 (anchors, positives, negatives);
 * theta [Kb], W [128][Kh] row-major, b [Kh] FP32.  Hard-negative mining on
 * the hard codes (S = K - 2 Hamming, Sec. III-A): for anchor i the negative
 * j != i most similar to a_i or p_i (lowest j on ties); anchor swap uses p_i
 * when it is the more similar one.  loss (device, 2 floats) receives
 * L = sum_i [tau - r(a_i).r(p_i) + r(x*_i).r(n*_i)]_+ for BAD and HashSIFT;
 * mining_out (device, nullable) receives [4][n] int32: n*_bad, swap_bad,
 * n*_hs, swap_hs; fixed_mining (device, nullable) replaces the mining.
 * The HashSIFT margins come from the tensor cores (W split into a BF16 head
 * and tail each call, three products per term: within a few 1e-6 of the FP32
 * sum for unit histograms and ||W_k|| near 1); the hard HashSIFT codes equal
 * the FP32 projection's (bits within 2^-13 ||W_k|| are recomputed in FP32). */
bd_status bd_train_forward(bd_ctx *ctx, bd_train *tr, const float *patches, const float *theta,
                           const float *W, const float *b, const int32_t *fixed_mining,
                           float *loss, int32_t *mining_out);

/* Backward of grad_loss[0] * L_bad + grad_loss[1] * L_hs (grad_loss: device,
 * 2 floats) through the last forward's state, mining held fixed.  Writes
 * dtheta [Kb], dW [128][Kh], db [Kh] and dpatches [3][n][32][32] (device).
 * Conventions at the non-differentiable points: a pixel with zero gradient
 * contributes nothing, a zero histogram has zero gradient, an inactive hinge
 * has zero gradient. */
bd_status bd_train_backward(bd_ctx *ctx, bd_train *tr, const float *patches, const float *W,
                            const float *grad_loss, float *dtheta, float *dW, float *db,
                            float *dpatches);

/* ------------------------------------------------------------------------ */
/* Allocation-free variant (the paper has no counterpart: this is a          */
/* deployment aid of this library)                                           */

/* Bytes of the static device area bd_bad_describe_noalloc works in. */
#define BD_BAD_NOALLOC_SCRATCH_BYTES ((size_t)9 << 20)

/* BAD descriptors like bd_bad_describe, for callers that cannot call
 * cudaMalloc: processes whose device memory is all reserved up front by
 * another allocator (a framework's caching pool), where a fresh cudaMalloc
 * fails or fragments the pool; real-time loops that cannot take the
 * device-wide synchronisation cudaFree implies; plug-ins run inside a host
 * program that forbids allocation once it is up.  The call allocates
 * nothing: the integral image and its tile carries live in a file-scope
 * static device array of BD_BAD_NOALLOC_SCRATCH_BYTES (held by every GPU
 * that loads the library until the process exits).  Parameters come from
 * bd_bad_params_create, done once at set-up.  The paper has no counterpart:
 * this is a deployment aid of this library.
 *  - Same arguments and outputs as bd_bad_describe, plus the cudaStream_t to
 *    enqueue on (NULL = legacy default stream); the parameters' device must be
 *    the current device.
 *  - Images whose table needs more than BD_BAD_NOALLOC_SCRATCH_BYTES
 *    ((h+1)(w+1) 4-byte entries plus carries; about 2.3 megapixels, e.g.
 *    1920x1088) are rejected with BD_ERR_INVALID and a message in the
 *    parameters' context; nothing is enqueued then.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it per
 *    device context (a context made after cudaDeviceReset gets a lookup of
 *    its own); make that first call before any stream capture.
 *  - Every call on a device shares the one array, which keeps the last call's
 *    contents (each call overwrites all it reads); calls that overlap on the
 *    GPU (other streams, or graph nodes not ordered after each other) race.
 *  - Invalid keypoints get all-zero descriptors but raise no status flag:
 *    the call has no context status word. */
bd_status bd_bad_describe_noalloc(const bd_bad_params *p, const uint8_t *img, int w, int h,
                                  int pitch, const bd_keypoint *kps, int n, uint32_t *out,
                                  void *stream);

/* ------------------------------------------------------------------------ */
/* Tensor-core matching                                                      */

/* Same contract and results as bd_match, computed on the tensor cores: the
 * codes are expanded to +-1 in FP8 E4M3 and the similarity S = h(q)^T h(t)
 * = nbits - 2 Hamming (Sec. III-A) is accumulated exactly in FP32 by
 * tcgen05 MMAs, with the top-2 and ratio test fused into the epilogue.
 * Needs (nq + nt) * nbits bytes of scratch; nq <= 65535 * 128. */
bd_status bd_match_tc(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                      int nbits, int ratio_num, int ratio_den, bd_match_result *out);

/* ------------------------------------------------------------------------ */
/* Several matchings in one launch                                           */

/* One matching of a bd_match_batch call: the arguments of bd_match. */
typedef struct {
    const uint32_t *q;      /* device, nq x nbits/32 words, 16-byte aligned */
    const uint32_t *t;      /* device, nt x nbits/32 words, 16-byte aligned */
    bd_match_result *out;   /* device, nq records, 4-byte aligned */
    int nq, nt, nbits, ratio_num, ratio_den;
} bd_match_job;

/* Runs up to BD_MATCH_MAX_JOBS independent bd_match problems (Sec. IV-C NN
 * matching with the top-2 ratio test; Sec. III-A S = K - 2 Hamming) as one
 * kernel launch on the POPC path, e.g. the BAD and the HashSIFT descriptors
 * of an image pair, or several image pairs.  Every job gets exactly the
 * records bd_match would return.  jobs is a host array, read during the
 * call.  Jobs may mix nbits 256 and 512; a job with nq = 0 is skipped.
 * Scratch: the sum of the jobs' bd_match scratch.  Errors: BD_ERR_INVALID for
 * n_jobs outside [0, BD_MATCH_MAX_JOBS] or any job that bd_match would
 * refuse (nothing is enqueued then). */
bd_status bd_match_batch(bd_ctx *ctx, const bd_match_job *jobs, int n_jobs);

/* ------------------------------------------------------------------------ */
/* Mutual nearest neighbours                                                 */

/* Hamming mutual-nearest-neighbour matching, the matching step of the
 * paper's pipeline-timing experiment (Sec. V: ORB detection, Hamming MNN
 * matching, PROSAC).  Query i and train entry j are a mutual pair iff j is
 * the nearest train entry of i and i is the nearest query of j, each
 * direction breaking equal distances to the lowest index.
 *  - out (device, nq records): the bd_match records of q against t, exactly
 *    as bd_match / bd_match_tc return them (ratio test ratio_num/ratio_den).
 *  - mnn (device, nq int32): out[i].idx when the pair is mutual, else -1.
 *  - tensor_cores: 0 runs both directions on the POPC kernel, 1 on the
 *    tensor-core kernel; the results are identical.
 *  - Scratch: nt * 12 bytes (rounded up to 256) for the reverse records plus
 *    the larger of the two directions' matching scratch.
 *  - Errors: BD_ERR_INVALID as for bd_match, and also when nq > 2^22 - 1, mnn is
 *    null or misaligned, or (tensor cores) nt > 65535 * 128.  nq = 0 is a
 *    no-op; nt = 0 gives out as bd_match does and mnn = -1 everywhere. */
bd_status bd_match_mnn(bd_ctx *ctx, const uint32_t *q, int nq, const uint32_t *t, int nt,
                       int nbits, int ratio_num, int ratio_den, int tensor_cores,
                       bd_match_result *out, int32_t *mnn);

/* ------------------------------------------------------------------------ */
/* BAD feature selection (Algorithm 1 with Algorithm 2)                      */

/* Threshold numerator with h = -1 for every patch (theta = -255.1). */
#define BD_SELECT_QMIN (-2551)

/* One round of the greedy BAD learning of Algorithm 1: for each of J
 * candidate box pairs, the threshold with the lowest per-step triplet loss
 *   L_h = sum_i [tau - S_ap[i] - h(a_i) h(p_i) + S_an[i] + h(a_i) h(n_i)]_+
 * (Sec. III-A; S_ap, S_an: similarities of the bits chosen before) found by
 * Algorithm 2 in its integer-sorted form, and the best candidate.
 *  - patches  device, 3 x n uint8 32x32 patches: anchors [0, n), positives
 *             [n, 2n), negatives [2n, 3n) (the triplets, already mined).
 *  - sim_ap, sim_an  device, n int32 each.
 *  - centres  host, J x 4 int32 (x1, y1, x2, y2) box centres in the patch
 *             frame; sides host, J int32 in [1, 32]; a box covers
 *             [c - floor(s/2), c - floor(s/2) + s) and pixels outside the patch
 *             count as 0; |centre| < 2^15.
 *  - f = (sum1 - sum2) / s^2 is compared with thresholds theta = q / 10 on
 *    the 0.1 grid: h = +1 iff 10 f <= q, i.e. iff ceil(10 f) <= q, for q in
 *    [BD_SELECT_QMIN, 2550]; the result is a BAD stump with thr_num = q and
 *    thr_den = 10.
 *  - theta_q (device, J int32): the lowest q with the minimal loss of each
 *    candidate; loss (device, J int64, 8-byte aligned): that loss; best
 *    (device, one int32): the first candidate with the minimal loss.
 *  - Scratch: 256 bytes + J x 3n x 2 bytes of keys (processed in passes of
 *    fewer candidates when that exceeds 1 GiB), plus the candidates.
 *  - Errors: BD_ERR_INVALID for n < 1 or n > 2^20, J < 1 or J >= 2^20, a side
 *    outside [1, 32], a centre out of range, null or misaligned pointers,
 *    or tau outside [-2^20, 2^20]. */
bd_status bd_select_feature(bd_ctx *ctx, const uint8_t *patches, int n, const int32_t *sim_ap,
                            const int32_t *sim_an, int tau, const int32_t *centres,
                            const int32_t *sides, int J, int32_t *theta_q, int64_t *loss,
                            int32_t *best);

/* ------------------------------------------------------------------------ */
/* Measurement probes (the paper has no counterpart: they give each kernel's  */
/* roofline a measured denominator)                                          */

typedef enum {
    BD_PROBE_GATHER = 0, /* random 4-byte loads, read-only path (BAD stump access) */
    BD_PROBE_POPC = 1,   /* 32-bit population counts (Hamming matching) */
    BD_PROBE_FFMA = 2,   /* FP32 fused multiply-adds (histogram arithmetic) */
    BD_PROBE_MUFU = 3,   /* ex2 on the special-function unit */
    BD_PROBE_L1_SECTORS = 4 /* 32-byte sectors handed out by L1 (BAD gather bound) */
} bd_probe_kind;

/* Enqueues one probe kernel on the context's stream, sized to fill every SM
 * (a multiple of the SM count at full occupancy), and stores in *units the
 * operations (loads or instructions) it performs; time it with events on the
 * same stream and divide.
 *  - BD_PROBE_GATHER: table (device, table_words uint32, contents irrelevant)
 *    with table_words and window_words powers of two, 32 <= window_words <=
 *    table_words <= 2^31.  Each warp draws reps windows of window_words
 *    words; per window every lane loads 64 random words of it, independent
 *    of each other.  window_words = table_words measures L2 random gathers
 *    once the table is larger than L1; a window of a few KB measures L1 hits.
 *  - BD_PROBE_L1_SECTORS: table (device, 16-byte aligned, table_words a
 *    power of two >= 4096) holds one 16 KB window per CTA; every lane loads
 *    16 consecutive bytes per request (512 contiguous bytes per warp), reps
 *    x 8 requests per warp; window_words is ignored.  *units = 32-byte
 *    sectors delivered (16 per request).
 *  - The other kinds ignore table and window_words; each thread runs
 *    reps x 64 instructions of the kind in eight independent chains.
 *  - sink: one device uint32 that the results are added to (keeps the work
 *    live); its value means nothing.
 *  - Errors: BD_ERR_INVALID for an unknown kind, reps outside [1, 2^20], a
 *    null sink or units, or a gather geometry that breaks the rules above. */
bd_status bd_probe(bd_ctx *ctx, int kind, const uint32_t *table, size_t table_words,
                   size_t window_words, int reps, uint32_t *sink, uint64_t *units);

#ifdef __cplusplus
}
#endif

#endif /* BINDESC_H */
