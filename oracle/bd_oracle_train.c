/*
 * Plain CPU oracle of the differentiable training step: relaxed BAD and
 * HashSIFT responses on 32x32 patches, the triplet ranking loss with
 * hard-negative mining and anchor swap, and its analytic gradient.
 *
 * TEST INFRASTRUCTURE ONLY (see bd_oracle.c); double precision throughout.
 *
 * Definitions (paper: Sec. III-A Eq. 1 for BAD, Sec. III-B Eq. 3 for HashSIFT;
 * hard-negative mining after HardNet and anchor swap after TFeat, Sec. III):
 *  - patches: 3n rows of 32x32, rows [0,n) anchors a_i, [n,2n) positives p_i,
 *    [2n,3n) negatives n_j;
 *  - BAD on a patch: f_k = (sum box1 - sum box2) / s_k^2 with boxes of side s_k
 *    centred on the pair's frame points (top-left = u - floor(s/2), zero outside
 *    the patch); hard bit = [f_k <= theta_k]; relaxed r_k = tanh((theta_k - f_k) / (255 T))
 *    (the 1/255 maps intensity differences to the unit range before the
 *    temperature T);
 *  - HashSIFT on a patch: h = the L2-normalised 128-bin histogram of
 *    or_hs_hist_raw, m = W^T h + b, hard bit = [m > 0], relaxed r = tanh(m / T);
 *  - similarity of hard codes S(x,y) = K - 2 Hamming(x,y) (Sec. III-A);
 *    mining: n*_i = argmax_{j != i} max(S(a_i,n_j), S(p_i,n_j)), lowest j on
 *    ties (with a single triplet, n*_0 = 0); anchor swap: x*_i = a_i if
 *    S(a_i,n*) >= S(p_i,n*) else p_i;
 *  - loss L = sum_i [tau - r(a_i).r(p_i) + r(x*_i).r(n*_i)]_+ , one loss per
 *    descriptor; the mining is held fixed when differentiating.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

double or_hs_hist_raw(const double *P, double *H);  /* bd_oracle.c */
int or_hamming(const uint32_t *a, const uint32_t *b, int nwords);

static const double ORT_PI = 3.14159265358979323846;

static double ort_box(const double *P, int x0, int y0, int s)
{
    double acc = 0.0;
    for (int y = y0; y < y0 + s; ++y) {
        if (y < 0 || y >= 32)
            continue;
        for (int x = x0; x < x0 + s; ++x) {
            if (x < 0 || x >= 32)
                continue;
            acc += P[y * 32 + x];
        }
    }
    return acc;
}

/* BAD feature values f[row][k] of `rows` patches. */
void or_bad_patch_features(const double *P, int rows, int K, const uint8_t *centres,
                           const uint8_t *sides, double *f)
{
    for (int r = 0; r < rows; ++r) {
        const double *p = P + (size_t)r * 1024;
        for (int k = 0; k < K; ++k) {
            const int s = sides[k];
            const double s1 = ort_box(p, centres[k * 4 + 0] - s / 2, centres[k * 4 + 1] - s / 2, s);
            const double s2 = ort_box(p, centres[k * 4 + 2] - s / 2, centres[k * 4 + 3] - s / 2, s);
            f[(size_t)r * K + k] = (s1 - s2) / ((double)s * (double)s);
        }
    }
}

static void pack_bit(uint32_t *bits, int K, int row, int k, int v)
{
    if (v)
        bits[(size_t)row * (K / 32) + k / 32] |= 1u << (k % 32);
}

/* Relaxed and hard BAD codes: r[row][k], bits[row][K/32]. */
void or_bad_relaxed(const double *P, int rows, int K, const uint8_t *centres, const uint8_t *sides,
                    const double *theta, double T, double *f, double *r, uint32_t *bits)
{
    or_bad_patch_features(P, rows, K, centres, sides, f);
    memset(bits, 0, sizeof(uint32_t) * (size_t)rows * (K / 32));
    for (int row = 0; row < rows; ++row)
        for (int k = 0; k < K; ++k) {
            const double fv = f[(size_t)row * K + k];
            r[(size_t)row * K + k] = tanh((theta[k] - fv) / (255.0 * T));
            pack_bit(bits, K, row, k, fv <= theta[k]);
        }
}

/* Relaxed and hard HashSIFT codes; h[row][128] and m[row][K] are returned too. */
void or_hs_relaxed(const double *P, int rows, int K, const double *W, const double *b, double T,
                   double *h, double *m, double *r, uint32_t *bits)
{
    memset(bits, 0, sizeof(uint32_t) * (size_t)rows * (K / 32));
    for (int row = 0; row < rows; ++row) {
        double H[128];
        const double nrm = or_hs_hist_raw(P + (size_t)row * 1024, H);
        double *hh = h + (size_t)row * 128;
        for (int q = 0; q < 128; ++q)
            hh[q] = nrm > 0.0 ? H[q] / nrm : 0.0;
        for (int k = 0; k < K; ++k) {
            double acc = b[k];
            for (int q = 0; q < 128; ++q)
                acc += W[(size_t)q * K + k] * hh[q];
            m[(size_t)row * K + k] = acc;
            r[(size_t)row * K + k] = tanh(acc / T);
            pack_bit(bits, K, row, k, acc > 0.0);
        }
    }
}

/* Hard-negative mining with anchor swap on hard codes (3n rows). */
void or_mine(const uint32_t *bits, int n, int K, int32_t *nstar, int32_t *xsel)
{
    const int nw = K / 32;
    for (int i = 0; i < n; ++i) {
        const uint32_t *a = bits + (size_t)i * nw;
        const uint32_t *p = bits + (size_t)(n + i) * nw;
        int best = -1, arg = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i && n > 1)
                continue;
            const uint32_t *ng = bits + (size_t)(2 * n + j) * nw;
            const int sa = K - 2 * or_hamming(a, ng, nw);
            const int sp = K - 2 * or_hamming(p, ng, nw);
            const int s = sa > sp ? sa : sp;
            if (best < 0 || s + K > best) { /* scores shifted by K are >= 0 */
                best = s + K;
                arg = j;
            }
        }
        nstar[i] = arg;
        const uint32_t *ng = bits + (size_t)(2 * n + arg) * nw;
        const int sa = K - 2 * or_hamming(a, ng, nw);
        const int sp = K - 2 * or_hamming(p, ng, nw);
        xsel[i] = sa >= sp ? 0 : 1;
    }
}

/* Triplet ranking loss; adds dL/dr into dr (3n x K) when dr != NULL. */
double or_trl(const double *r, int n, int K, const int32_t *nstar, const int32_t *xsel, double tau,
              double w, double *dr)
{
    double L = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *ra = r + (size_t)i * K;
        const double *rp = r + (size_t)(n + i) * K;
        const int xrow = xsel[i] ? n + i : i;
        const double *rx = r + (size_t)xrow * K;
        const int nrow = 2 * n + nstar[i];
        const double *rn = r + (size_t)nrow * K;
        double sap = 0.0, sxn = 0.0;
        for (int k = 0; k < K; ++k) {
            sap += ra[k] * rp[k];
            sxn += rx[k] * rn[k];
        }
        const double term = tau - sap + sxn;
        if (term > 0.0) {
            L += term;
            if (dr) {
                for (int k = 0; k < K; ++k) {
                    dr[(size_t)i * K + k] -= w * rp[k];
                    dr[(size_t)(n + i) * K + k] -= w * ra[k];
                    dr[(size_t)xrow * K + k] += w * rn[k];
                    dr[(size_t)nrow * K + k] += w * rx[k];
                }
            }
        }
    }
    return L;
}

/* BAD backward: dtheta (K) and dP (rows x 1024), both accumulated. */
void or_bad_backward(int rows, int K, const uint8_t *centres, const uint8_t *sides, double T,
                     const double *r, const double *dr, double *dtheta, double *dP)
{
    const double c = 1.0 / (255.0 * T);
    for (int row = 0; row < rows; ++row) {
        double *dp = dP + (size_t)row * 1024;
        for (int k = 0; k < K; ++k) {
            const double rv = r[(size_t)row * K + k];
            const double dz = dr[(size_t)row * K + k] * (1.0 - rv * rv);
            dtheta[k] += dz * c;
            const double df = -dz * c;  /* z = (theta - f) c */
            const int s = sides[k];
            const double g = df / ((double)s * (double)s);
            for (int j = 0; j < 2; ++j) {
                const int x0 = centres[k * 4 + 2 * j] - s / 2, y0 = centres[k * 4 + 2 * j + 1] - s / 2;
                const double sg = j == 0 ? g : -g;
                for (int y = y0; y < y0 + s; ++y) {
                    if (y < 0 || y >= 32)
                        continue;
                    for (int x = x0; x < x0 + s; ++x) {
                        if (x < 0 || x >= 32)
                            continue;
                        dp[y * 32 + x] += sg;
                    }
                }
            }
        }
    }
}

/* HashSIFT backward: dW (128 x K), db (K), dP (rows x 1024), all accumulated. */
void or_hs_backward(const double *P, int rows, int K, const double *W, double T, const double *h,
                    const double *r, const double *dr, double *dW, double *db, double *dP)
{
    double *dm = (double *)malloc(sizeof(double) * (size_t)K);
    for (int row = 0; row < rows; ++row) {
        const double *hh = h + (size_t)row * 128;
        for (int k = 0; k < K; ++k) {
            const double rv = r[(size_t)row * K + k];
            dm[k] = dr[(size_t)row * K + k] * (1.0 - rv * rv) / T;
            db[k] += dm[k];
            for (int q = 0; q < 128; ++q)
                dW[(size_t)q * K + k] += hh[q] * dm[k];
        }
        double dh[128];
        for (int q = 0; q < 128; ++q) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k)
                acc += W[(size_t)q * K + k] * dm[k];
            dh[q] = acc;
        }
        /* h = H / ||H||  ->  dH = (dh - h (h . dh)) / ||H|| */
        const double *p = P + (size_t)row * 1024;
        double H[128];
        const double nrm = or_hs_hist_raw(p, H);
        if (!(nrm > 0.0))
            continue;
        double hd = 0.0;
        for (int q = 0; q < 128; ++q)
            hd += hh[q] * dh[q];
        double dH[128];
        for (int q = 0; q < 128; ++q)
            dH[q] = (dh[q] - hh[q] * hd) / nrm;
        double *dp = dP + (size_t)row * 1024;
        for (int i = 0; i < 32; ++i) {
            for (int j = 0; j < 32; ++j) {
                const int jl = j > 0 ? j - 1 : 0, jr = j < 31 ? j + 1 : 31;
                const int iu = i > 0 ? i - 1 : 0, id = i < 31 ? i + 1 : 31;
                const double gx = 0.5 * (p[i * 32 + jr] - p[i * 32 + jl]);
                const double gy = 0.5 * (p[id * 32 + j] - p[iu * 32 + j]);
                const double m2 = gx * gx + gy * gy;
                if (!(m2 > 0.0))
                    continue;
                const double mag = sqrt(m2);
                double phi = atan2(gy, gx);
                if (phi < 0.0)
                    phi += 2.0 * ORT_PI;
                const double t = phi * 8.0 / (2.0 * ORT_PI);
                const double fl = floor(t);
                const double w1 = t - fl;
                const int b0 = ((int)fl) % 8, b1 = (b0 + 1) % 8;
                const double di = (double)i - 15.5, dj = (double)j - 15.5;
                const double g = exp(-(di * di + dj * dj) / (2.0 * 16.0 * 16.0));
                const int cell = (i / 8) * 4 + (j / 8);
                const double d0 = dH[cell * 8 + b0], d1 = dH[cell * 8 + b1];
                const double dmag = g * ((1.0 - w1) * d0 + w1 * d1);
                const double dphi = g * mag * (d1 - d0) * 8.0 / (2.0 * ORT_PI);
                const double dgx = dmag * gx / mag - dphi * gy / m2;
                const double dgy = dmag * gy / mag + dphi * gx / m2;
                dp[i * 32 + jr] += 0.5 * dgx;
                dp[i * 32 + jl] -= 0.5 * dgx;
                dp[id * 32 + j] += 0.5 * dgy;
                dp[iu * 32 + j] -= 0.5 * dgy;
            }
        }
    }
    free(dm);
}

/*
 * One training step.  patches: 3n x 1024; theta: Kb; W: 128 x Kh; b: Kh.  fixed_mining (4n int32: nstar_bad, xsel_bad, nstar_hs,
 * xsel_hs) replaces the mining when non-NULL; mining_out receives the mining
 * used.  Gradients are of w_bad * L_bad + w_hs * L_hs; any output may be NULL.
 */
void or_train_step(const double *patches, int n, int Kb, const uint8_t *centres,
                   const uint8_t *sides, const double *theta, int Kh, const double *W, const double *b,
                   double T, double tau_bad, double tau_hs, double w_bad, double w_hs,
                   const int32_t *fixed_mining, double *loss, int32_t *mining_out, double *dtheta,
                   double *dW, double *db, double *dpatches, double *r_bad_out, double *r_hs_out)
{
    const int rows = 3 * n;
    double *P = (double *)malloc(sizeof(double) * (size_t)rows * 1024);
    for (size_t q = 0; q < (size_t)rows * 1024; ++q)
        P[q] = (double)patches[q];
    double *th = (double *)malloc(sizeof(double) * (size_t)Kb);
    for (int k = 0; k < Kb; ++k)
        th[k] = (double)theta[k];
    double *Wd = (double *)malloc(sizeof(double) * 128 * (size_t)Kh);
    double *bd = (double *)malloc(sizeof(double) * (size_t)Kh);
    for (size_t q = 0; q < 128 * (size_t)Kh; ++q)
        Wd[q] = (double)W[q];
    for (int k = 0; k < Kh; ++k)
        bd[k] = (double)b[k];

    double *fb = (double *)malloc(sizeof(double) * (size_t)rows * Kb);
    double *rb = (double *)malloc(sizeof(double) * (size_t)rows * Kb);
    uint32_t *bb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)rows * (Kb / 32));
    double *hh = (double *)malloc(sizeof(double) * (size_t)rows * 128);
    double *mh = (double *)malloc(sizeof(double) * (size_t)rows * Kh);
    double *rh = (double *)malloc(sizeof(double) * (size_t)rows * Kh);
    uint32_t *bh = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)rows * (Kh / 32));
    int32_t *mine = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)n);

    or_bad_relaxed(P, rows, Kb, centres, sides, th, T, fb, rb, bb);
    or_hs_relaxed(P, rows, Kh, Wd, bd, T, hh, mh, rh, bh);
    if (fixed_mining) {
        memcpy(mine, fixed_mining, sizeof(int32_t) * 4 * (size_t)n);
    } else {
        or_mine(bb, n, Kb, mine, mine + n);
        or_mine(bh, n, Kh, mine + 2 * n, mine + 3 * n);
    }
    if (mining_out)
        memcpy(mining_out, mine, sizeof(int32_t) * 4 * (size_t)n);

    double *drb = (double *)calloc((size_t)rows * Kb, sizeof(double));
    double *drh = (double *)calloc((size_t)rows * Kh, sizeof(double));
    const double Lb = or_trl(rb, n, Kb, mine, mine + n, tau_bad, w_bad, drb);
    const double Lh = or_trl(rh, n, Kh, mine + 2 * n, mine + 3 * n, tau_hs, w_hs, drh);
    if (loss) {
        loss[0] = Lb;
        loss[1] = Lh;
    }
    double *dth = (double *)calloc((size_t)Kb, sizeof(double));
    double *dWd = (double *)calloc(128 * (size_t)Kh, sizeof(double));
    double *dbd = (double *)calloc((size_t)Kh, sizeof(double));
    double *dP = (double *)calloc((size_t)rows * 1024, sizeof(double));
    if (dtheta || dW || db || dpatches) {
        or_bad_backward(rows, Kb, centres, sides, T, rb, drb, dth, dP);
        or_hs_backward(P, rows, Kh, Wd, T, hh, rh, drh, dWd, dbd, dP);
    }
    if (dtheta)
        memcpy(dtheta, dth, sizeof(double) * (size_t)Kb);
    if (dW)
        memcpy(dW, dWd, sizeof(double) * 128 * (size_t)Kh);
    if (db)
        memcpy(db, dbd, sizeof(double) * (size_t)Kh);
    if (dpatches)
        memcpy(dpatches, dP, sizeof(double) * (size_t)rows * 1024);
    if (r_bad_out)
        memcpy(r_bad_out, rb, sizeof(double) * (size_t)rows * Kb);
    if (r_hs_out)
        memcpy(r_hs_out, rh, sizeof(double) * (size_t)rows * Kh);
    free(P); free(th); free(Wd); free(bd); free(fb); free(rb); free(bb); free(hh); free(mh);
    free(rh); free(bh); free(mine); free(drb); free(drh); free(dth); free(dWd); free(dbd); free(dP);
}

/* Hard codes of all 3n patches (for the mining pins). */
void or_train_codes(const double *patches, int n, int Kb, const uint8_t *centres,
                    const uint8_t *sides, const double *theta, int Kh, const double *W, const double *b,
                    uint32_t *bits_bad, uint32_t *bits_hs, double *f_bad, double *m_hs)
{
    const int rows = 3 * n;
    double *P = (double *)malloc(sizeof(double) * (size_t)rows * 1024);
    for (size_t q = 0; q < (size_t)rows * 1024; ++q)
        P[q] = (double)patches[q];
    double *th = (double *)malloc(sizeof(double) * (size_t)Kb);
    for (int k = 0; k < Kb; ++k)
        th[k] = (double)theta[k];
    double *Wd = (double *)malloc(sizeof(double) * 128 * (size_t)Kh);
    double *bd = (double *)malloc(sizeof(double) * (size_t)Kh);
    for (size_t q = 0; q < 128 * (size_t)Kh; ++q)
        Wd[q] = (double)W[q];
    for (int k = 0; k < Kh; ++k)
        bd[k] = (double)b[k];
    double *rb = (double *)malloc(sizeof(double) * (size_t)rows * Kb);
    double *hh = (double *)malloc(sizeof(double) * (size_t)rows * 128);
    double *rh = (double *)malloc(sizeof(double) * (size_t)rows * Kh);
    or_bad_relaxed(P, rows, Kb, centres, sides, th, 1.0, f_bad, rb, bits_bad);
    or_hs_relaxed(P, rows, Kh, Wd, bd, 1.0, hh, m_hs, rh, bits_hs);
    free(P); free(th); free(Wd); free(bd); free(rb); free(hh); free(rh);
}
