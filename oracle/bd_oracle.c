/*
 * Plain, slow, single-threaded CPU oracle for the BAD and HashSIFT binary
 * descriptors and their brute-force Hamming matching, after Suarez,
 * Buenaposada and Baumela, "Revisiting Binary Local Image Description for
 * Resource Limited Devices" (IEEE RA-L 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA library: every step is
 * written out here from the paper's definitions, in integers for BAD and the
 * Hamming distances and in double precision for HashSIFT.
 *
 * Readings of the paper (where it is silent the choice is stated once, here):
 *  - Box pairs live in a 32x32 patch frame (Sec. III-A: patches re-scaled to
 *    32x32) whose centre is the integer point (16,16).  A keypoint
 *    (x, y, scale, angle) maps frame offset d = u - (16,16) to the image
 *    offset round(sigma_l * R(theta_b) d), R the rotation in image
 *    coordinates (y down), theta_b = 2*pi*b/NB the centre of angle bin b and
 *    sigma_l the scale of the pyramid level chosen for the keypoint; the box
 *    side becomes max(1, round(s * sigma_l)).  round() is half away from zero.
 *  - A box of side s centred on pixel c covers [c - floor(s/2), c - floor(s/2) + s)
 *    in x and y; pixels outside the image count as 0 and the mean always
 *    divides by s^2.
 *  - BAD weak descriptor (Sec. III-A): h = +1 iff f <= theta, f the
 *    difference of the two box means.  With theta = num/den (den > 0) the
 *    test den*(sum1 - sum2) <= num*s^2 is exact in 64-bit integers.  h = +1
 *    is stored as bit 1; bit k goes to word k/32, bit position k%32.
 *  - Keypoint quantisation, in IEEE single precision without contraction:
 *    ix = floor(x + 0.5), iy = floor(y + 0.5),
 *    b = floor(angle * float(NB/(2 pi)) + 0.5) mod NB,
 *    level = number of midpoints float(sqrt(sigma_i sigma_{i+1})) below scale.
 *  - A keypoint is valid iff x, y, scale, angle are finite, |x|,|y| <= 2^20,
 *    0 < scale <= 1024 and |angle| <= 2^20; an invalid one gets an all-zero
 *    descriptor (and histogram) and is counted.
 *  - HashSIFT (Sec. III-B): f is the SIFT-style gradient orientation
 *    histogram of the 32x32 patch: 4x4 cells of 8x8 pixels, 8 orientation
 *    bins, central differences with replicated edges, Gaussian weight
 *    sigma = 16 about the patch centre (15.5, 15.5), linear (soft) voting
 *    between the two nearest orientation bins, L2 normalisation (a zero
 *    histogram stays zero).  No spatial interpolation or clipping.
 *  - Patch pixel (i, j) samples the image at
 *    (x, y) + scale*spacing*R(angle) (j - 15.5, i - 15.5), bilinear with
 *    clamp-to-edge taps; the angle is not binned for HashSIFT.
 *  - D = sgn(B [f; 1]) with B = [W^T | b]: bit k = 1 iff W_k . f + b_k > 0
 *    (a zero margin gives bit 0).
 *  - Matching (Sec. IV-C nearest neighbour; Lowe-style ratio test): per
 *    query, the train entries sorted by (distance, index); idx/d1 from the
 *    first, d2 from the second (nbits+1 when there is none, and idx = -1,
 *    d1 = nbits+1 for an empty train set); accept iff den*d1 < num*d2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Integral image (Sec. III-A: box means from an integral image; Sec. IV-F). */
/* ii has (h+1) rows of (w+1) entries; ii[y][x] = sum of img over [0,y)x[0,x). */
void or_integral(const uint8_t *img, int w, int h, int pitch, uint32_t *ii)
{
    const size_t W1 = (size_t)w + 1;
    for (int x = 0; x <= w; ++x)
        ii[x] = 0;
    for (int y = 0; y < h; ++y) {
        uint32_t row = 0; /* sum of img[y][0..x] */
        ii[(size_t)(y + 1) * W1] = 0;
        for (int x = 0; x < w; ++x) {
            row += img[(size_t)y * pitch + x];
            ii[(size_t)(y + 1) * W1 + x + 1] = ii[(size_t)y * W1 + x + 1] + row;
        }
    }
}

/* Sum of the image over the square [x0, x0+side) x [y0, y0+side), zero outside. */
int64_t or_box_sum(const uint8_t *img, int w, int h, int pitch, int x0, int y0, int side)
{
    int64_t s = 0;
    for (int y = y0; y < y0 + side; ++y) {
        if (y < 0 || y >= h)
            continue;
        for (int x = x0; x < x0 + side; ++x) {
            if (x < 0 || x >= w)
                continue;
            s += img[(size_t)y * pitch + x];
        }
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Keypoint handling.                                                        */

int or_kp_valid(const float *kp)
{
    for (int i = 0; i < 4; ++i)
        if (!isfinite(kp[i]))
            return 0;
    if (fabsf(kp[0]) > 1048576.0f || fabsf(kp[1]) > 1048576.0f)
        return 0;
    if (!(kp[2] > 0.0f) || kp[2] > 1024.0f)
        return 0;
    if (fabsf(kp[3]) > 1048576.0f)
        return 0;
    return 1;
}

int or_round_coord(float v)
{
    volatile float t = v + 0.5f; /* one single-precision add */
    return (int)floorf(t);
}

int or_angle_bin(float angle, int nbins)
{
    const float c = (float)((double)nbins / (2.0 * OR_PI));
    volatile float t = angle * c; /* single-precision multiply, then add */
    volatile float u = t + 0.5f;
    int b = (int)floorf(u);
    b %= nbins;
    if (b < 0)
        b += nbins;
    return b;
}

int or_scale_level(float scale, const float *level_scales, int nlevels)
{
    int l = 0;
    for (int i = 0; i + 1 < nlevels; ++i) {
        const float mid = (float)sqrt((double)level_scales[i] * (double)level_scales[i + 1]);
        if (mid < scale)
            ++l;
    }
    return l;
}

/* Box geometry of all K pairs at pyramid scale sigma and angle theta:
 * centre offsets off[(k*2+j)*2 + {0,1}] (x, y) and sides sp[k]. */
void or_bad_geometry(int K, const uint8_t *centres, const uint8_t *sides, double sigma,
                     double theta, int *off, int *sp)
{
    const double c = cos(theta), s = sin(theta);
    for (int k = 0; k < K; ++k) {
        int side = (int)round((double)sides[k] * sigma);
        sp[k] = side < 1 ? 1 : side;
        for (int j = 0; j < 2; ++j) {
            const double dx = (double)centres[(k * 2 + j) * 2 + 0] - 16.0;
            const double dy = (double)centres[(k * 2 + j) * 2 + 1] - 16.0;
            off[(k * 2 + j) * 2 + 0] = (int)round(sigma * (c * dx - s * dy));
            off[(k * 2 + j) * 2 + 1] = (int)round(sigma * (s * dx + c * dy));
        }
    }
}

/* ------------------------------------------------------------------------ */
/* BAD descriptor (Sec. III-A).  out: n x (K/32) words.  Returns the number
 * of invalid keypoints. */
int or_bad_describe(const uint8_t *img, int w, int h, int pitch, const float *kps, int n, int K,
                    const uint8_t *centres, const uint8_t *sides, const int32_t *thr_num,
                    int32_t thr_den, int nbins, const float *level_scales, int nlevels,
                    uint32_t *out)
{
    const int nw = K / 32;
    int *off = (int *)malloc(sizeof(int) * 4 * (size_t)K);
    int *sp = (int *)malloc(sizeof(int) * (size_t)K);
    int invalid = 0;
    for (int i = 0; i < n; ++i) {
        const float *kp = kps + 4 * (size_t)i;
        uint32_t *d = out + (size_t)i * nw;
        memset(d, 0, sizeof(uint32_t) * nw);
        if (!or_kp_valid(kp)) {
            ++invalid;
            continue;
        }
        const int ix = or_round_coord(kp[0]);
        const int iy = or_round_coord(kp[1]);
        const int l = or_scale_level(kp[2], level_scales, nlevels);
        const int b = or_angle_bin(kp[3], nbins);
        const double theta = 2.0 * OR_PI * (double)b / (double)nbins;
        or_bad_geometry(K, centres, sides, (double)level_scales[l], theta, off, sp);
        for (int k = 0; k < K; ++k) {
            const int s = sp[k];
            int64_t sum[2];
            for (int j = 0; j < 2; ++j) {
                const int cx = ix + off[(k * 2 + j) * 2 + 0];
                const int cy = iy + off[(k * 2 + j) * 2 + 1];
                sum[j] = or_box_sum(img, w, h, pitch, cx - s / 2, cy - s / 2, s);
            }
            const int64_t lhs = (int64_t)thr_den * (sum[0] - sum[1]);
            const int64_t rhs = (int64_t)thr_num[k] * (int64_t)s * (int64_t)s;
            if (lhs <= rhs)
                d[k / 32] |= 1u << (k % 32);
        }
    }
    free(off);
    free(sp);
    return invalid;
}

/* ------------------------------------------------------------------------ */
/* HashSIFT (Sec. III-B).                                                     */

static double or_pix(const uint8_t *img, int w, int h, int pitch, double xf, double yf)
{
    /* clamp-to-edge tap at integer-valued coordinates xf, yf */
    double xc = xf < 0.0 ? 0.0 : (xf > (double)(w - 1) ? (double)(w - 1) : xf);
    double yc = yf < 0.0 ? 0.0 : (yf > (double)(h - 1) ? (double)(h - 1) : yf);
    return (double)img[(size_t)(int)yc * pitch + (int)xc];
}

/* 32x32 patch P[i*32 + j] around the keypoint. */
void or_hs_patch(const uint8_t *img, int w, int h, int pitch, const float *kp, double spacing,
                 double *P)
{
    const double x = kp[0], y = kp[1], sg = (double)kp[2] * spacing;
    const double c = cos((double)kp[3]), s = sin((double)kp[3]);
    for (int i = 0; i < 32; ++i) {
        for (int j = 0; j < 32; ++j) {
            const double u = (double)j - 15.5, v = (double)i - 15.5;
            const double sx = x + sg * (c * u - s * v);
            const double sy = y + sg * (s * u + c * v);
            const double x0 = floor(sx), y0 = floor(sy);
            const double fx = sx - x0, fy = sy - y0;
            const double i00 = or_pix(img, w, h, pitch, x0, y0);
            const double i01 = or_pix(img, w, h, pitch, x0 + 1.0, y0);
            const double i10 = or_pix(img, w, h, pitch, x0, y0 + 1.0);
            const double i11 = or_pix(img, w, h, pitch, x0 + 1.0, y0 + 1.0);
            P[i * 32 + j] = (1.0 - fy) * ((1.0 - fx) * i00 + fx * i01) + fy * ((1.0 - fx) * i10 + fx * i11);
        }
    }
}

/* Unnormalised 128-bin histogram H of a 32x32 patch; returns ||H||_2. */
double or_hs_hist_raw(const double *P, double *H)
{
    for (int q = 0; q < 128; ++q)
        H[q] = 0.0;
    for (int i = 0; i < 32; ++i) {
        for (int j = 0; j < 32; ++j) {
            const int jl = j > 0 ? j - 1 : 0, jr = j < 31 ? j + 1 : 31;
            const int iu = i > 0 ? i - 1 : 0, id = i < 31 ? i + 1 : 31;
            const double gx = 0.5 * (P[i * 32 + jr] - P[i * 32 + jl]);
            const double gy = 0.5 * (P[id * 32 + j] - P[iu * 32 + j]);
            const double m = sqrt(gx * gx + gy * gy);
            double phi = atan2(gy, gx);
            if (phi < 0.0)
                phi += 2.0 * OR_PI;
            const double t = phi * 8.0 / (2.0 * OR_PI);
            const double fl = floor(t);
            const double w1 = t - fl;
            const int b0 = ((int)fl) % 8;
            const int b1 = (b0 + 1) % 8;
            const double di = (double)i - 15.5, dj = (double)j - 15.5;
            const double g = exp(-(di * di + dj * dj) / (2.0 * 16.0 * 16.0));
            const int cell = (i / 8) * 4 + (j / 8);
            H[cell * 8 + b0] += g * m * (1.0 - w1);
            H[cell * 8 + b1] += g * m * w1;
        }
    }
    double nn = 0.0;
    for (int q = 0; q < 128; ++q)
        nn += H[q] * H[q];
    return sqrt(nn);
}

/* SIFT variants of the histogram before hashing (the paper names RootSIFT,
 * Sec. II; SIFT's trilinear binning and 0.2 clip are Lowe's).  flags:
 *   1 trilinear: each vote is shared by the two nearest cell rows and cell
 *     columns (cell c's centre at pixel 8c + 3.5, weight 1 - |x - centre| / 8,
 *     cells outside the 4x4 grid dropped) instead of going to the pixel's cell;
 *   2 clip: L2-normalise, clip every entry at 0.2, L2-normalise again;
 *   4 root (RootSIFT): divide by the L1 norm, take square roots (unit L2 norm).
 * Applied in the order binning, clip, root; a zero histogram stays zero. */
void or_hs_hist_variant(const double *P, int flags, double *h)
{
    double H[128];
    if (flags & 1) {
        for (int q = 0; q < 128; ++q)
            H[q] = 0.0;
        for (int i = 0; i < 32; ++i) {
            for (int j = 0; j < 32; ++j) {
                const int jl = j > 0 ? j - 1 : 0, jr = j < 31 ? j + 1 : 31;
                const int iu = i > 0 ? i - 1 : 0, id = i < 31 ? i + 1 : 31;
                const double gx = 0.5 * (P[i * 32 + jr] - P[i * 32 + jl]);
                const double gy = 0.5 * (P[id * 32 + j] - P[iu * 32 + j]);
                const double m = sqrt(gx * gx + gy * gy);
                double phi = atan2(gy, gx);
                if (phi < 0.0)
                    phi += 2.0 * OR_PI;
                const double t = phi * 8.0 / (2.0 * OR_PI);
                const double w1 = t - floor(t);
                const int b0 = ((int)floor(t)) % 8, b1 = (b0 + 1) % 8;
                const double di = (double)i - 15.5, dj = (double)j - 15.5;
                const double g = exp(-(di * di + dj * dj) / (2.0 * 16.0 * 16.0));
                for (int ci = 0; ci < 4; ++ci) {
                    const double wy = 1.0 - fabs((double)i - (8.0 * ci + 3.5)) / 8.0;
                    if (wy <= 0.0)
                        continue;
                    for (int cj = 0; cj < 4; ++cj) {
                        const double wx = 1.0 - fabs((double)j - (8.0 * cj + 3.5)) / 8.0;
                        if (wx <= 0.0)
                            continue;
                        const int cell = ci * 4 + cj;
                        H[cell * 8 + b0] += g * m * wy * wx * (1.0 - w1);
                        H[cell * 8 + b1] += g * m * wy * wx * w1;
                    }
                }
            }
        }
    } else {
        or_hs_hist_raw(P, H);
    }
    double n2 = 0.0;
    for (int q = 0; q < 128; ++q)
        n2 += H[q] * H[q];
    double nrm = sqrt(n2);
    for (int q = 0; q < 128; ++q)
        h[q] = nrm > 0.0 ? H[q] / nrm : 0.0;
    if ((flags & 2) && nrm > 0.0) {
        n2 = 0.0;
        for (int q = 0; q < 128; ++q) {
            if (h[q] > 0.2)
                h[q] = 0.2;
            n2 += h[q] * h[q];
        }
        nrm = sqrt(n2);
        for (int q = 0; q < 128; ++q)
            h[q] /= nrm;
    }
    if (flags & 4) {
        double l1 = 0.0;
        for (int q = 0; q < 128; ++q)
            l1 += h[q];
        for (int q = 0; q < 128; ++q)
            h[q] = l1 > 0.0 ? sqrt(h[q] / l1) : 0.0;
    }
}

/* L2-normalised histogram h of n patches (patches: n x 1024, hist: n x 128). */
void or_hs_hist(const double *patches, int n, double *hist)
{
    for (int p = 0; p < n; ++p) {
        double *hh = hist + (size_t)p * 128;
        const double nrm = or_hs_hist_raw(patches + (size_t)p * 1024, hh);
        for (int q = 0; q < 128; ++q)
            hh[q] = nrm > 0.0 ? hh[q] / nrm : 0.0;
    }
}

/* margins m = W^T h + b (W: 128 x K row-major) and bits [m > 0]. */
void or_hs_project(const double *hist, int n, const float *W, const float *bias, int K,
                   double *margins, uint32_t *bits)
{
    const int nw = K / 32;
    for (int p = 0; p < n; ++p) {
        uint32_t *d = bits + (size_t)p * nw;
        for (int q = 0; q < nw; ++q)
            d[q] = 0;
        for (int k = 0; k < K; ++k) {
            double m = (double)bias[k];
            for (int i = 0; i < 128; ++i)
                m += (double)W[(size_t)i * K + k] * hist[(size_t)p * 128 + i];
            if (margins)
                margins[(size_t)p * K + k] = m;
            if (m > 0.0)
                d[k / 32] |= 1u << (k % 32);
        }
    }
}

/* Whole HashSIFT descriptor of n keypoints; patches/hist/margins optional. */
int or_hs_describe(const uint8_t *img, int w, int h, int pitch, const float *kps, int n,
                   double spacing, const float *W, const float *bias, int K, uint32_t *bits,
                   double *hist_out, double *margins_out, double *patches_out)
{
    double P[1024], hh[128];
    double *mg = (double *)malloc(sizeof(double) * (size_t)K);
    int invalid = 0;
    const int nw = K / 32;
    for (int p = 0; p < n; ++p) {
        const float *kp = kps + 4 * (size_t)p;
        if (!or_kp_valid(kp)) {
            ++invalid;
            for (int q = 0; q < nw; ++q)
                bits[(size_t)p * nw + q] = 0;
            if (hist_out)
                memset(hist_out + (size_t)p * 128, 0, sizeof(double) * 128);
            if (margins_out)
                memset(margins_out + (size_t)p * K, 0, sizeof(double) * K);
            if (patches_out)
                memset(patches_out + (size_t)p * 1024, 0, sizeof(double) * 1024);
            continue;
        }
        or_hs_patch(img, w, h, pitch, kp, spacing, P);
        or_hs_hist(P, 1, hh);
        or_hs_project(hh, 1, W, bias, K, mg, bits + (size_t)p * nw);
        if (hist_out)
            memcpy(hist_out + (size_t)p * 128, hh, sizeof(double) * 128);
        if (margins_out)
            memcpy(margins_out + (size_t)p * K, mg, sizeof(double) * K);
        if (patches_out)
            memcpy(patches_out + (size_t)p * 1024, P, sizeof(double) * 1024);
    }
    free(mg);
    return invalid;
}

/* ------------------------------------------------------------------------ */
/* Hamming distance and brute-force nearest / second-nearest matching.       */

static int or_popcount32(uint32_t x)
{
    int c = 0;
    while (x) {
        x &= x - 1u;
        ++c;
    }
    return c;
}

int or_hamming(const uint32_t *a, const uint32_t *b, int nwords)
{
    int d = 0;
    for (int q = 0; q < nwords; ++q)
        d += or_popcount32(a[q] ^ b[q]);
    return d;
}

typedef struct {
    int d;
    int idx;
} or_pair;

static int or_pair_cmp(const void *pa, const void *pb)
{
    const or_pair *a = (const or_pair *)pa, *b = (const or_pair *)pb;
    if (a->d != b->d)
        return a->d < b->d ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

void or_match(const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits, int ratio_num,
              int ratio_den, int32_t *idx, int32_t *d1, int32_t *d2, uint8_t *accept)
{
    const int nw = nbits / 32;
    or_pair *pr = (or_pair *)malloc(sizeof(or_pair) * (size_t)(nt > 0 ? nt : 1));
    for (int i = 0; i < nq; ++i) {
        for (int j = 0; j < nt; ++j) {
            pr[j].d = or_hamming(q + (size_t)i * nw, t + (size_t)j * nw, nw);
            pr[j].idx = j;
        }
        qsort(pr, (size_t)nt, sizeof(or_pair), or_pair_cmp);
        const int a = nt > 0 ? pr[0].d : nbits + 1;
        const int b = nt > 1 ? pr[1].d : nbits + 1;
        idx[i] = nt > 0 ? pr[0].idx : -1;
        d1[i] = a;
        d2[i] = b;
        accept[i] = ((int64_t)ratio_den * a < (int64_t)ratio_num * b) ? 1 : 0;
    }
    free(pr);
}

/* Nearest entry of set b for one descriptor a (lowest index among equal
 * distances); -1 when b is empty. */
static int or_nearest(const uint32_t *a, const uint32_t *b, int nb, int nw)
{
    int best = -1, bd = 0;
    for (int j = 0; j < nb; ++j) {
        const int d = or_hamming(a, b + (size_t)j * nw, nw);
        if (best < 0 || d < bd) {
            best = j;
            bd = d;
        }
    }
    return best;
}

/* Mutual nearest neighbours (the Hamming MNN matching of the pipeline-timing
 * experiment, Sec. V): query i and train entry j match iff j is the nearest
 * train entry of i and i is the nearest query of j, each side breaking ties
 * to the lowest index.  mnn[i] = j, or -1 when i has no mutual partner. */
void or_match_mnn(const uint32_t *q, int nq, const uint32_t *t, int nt, int nbits, int32_t *mnn)
{
    const int nw = nbits / 32;
    int *back = (int *)malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
    for (int j = 0; j < nt; ++j)
        back[j] = or_nearest(t + (size_t)j * nw, q, nq, nw);
    for (int i = 0; i < nq; ++i) {
        const int j = or_nearest(q + (size_t)i * nw, t, nt, nw);
        mnn[i] = (j >= 0 && back[j] == i) ? j : -1;
    }
    free(back);
}
