/* Oracle (test infrastructure only) of one round of BAD feature selection:
 * Algorithm 1 (choose, among J candidate box pairs, the weak descriptor with
 * the lowest per-step triplet loss L_h) with Algorithm 2 (find the threshold
 * with the lowest L_h of one candidate), in the integer-sorted variant of
 * Sec. III-A (thresholds on a 0.1 grid over [-255, 255]).
 *
 * Definitions (readings stated in the design notes):
 *  - patch: uint8 32x32; a candidate is two boxes of side s with centres
 *    (x1, y1), (x2, y2) in the patch frame, top-left at centre - floor(s/2),
 *    pixels outside the patch count as 0 (as for BAD on images);
 *  - f(x) = (sum1 - sum2) / s^2 and its key ceil(10 f), an integer in
 *    [-2550, 2550]; a threshold is an integer q with theta = q / 10, and
 *    h(x) = +1 iff f(x) <= theta, i.e. iff key(x) <= q; q = -2551 gives h = -1
 *    everywhere;
 *  - per-step loss (Sec. III-A): sum over triplets of
 *      [tau - S_ap - h(a)h(p) + S_an + h(a)h(n)]_+
 *    with S_ap, S_an the similarities of the bits chosen before;
 *  - the loss changes only at the keys of the triplets' patches; the change
 *    of a triplet at key k is its term at q = k minus its term at q = k - 1
 *    (equal keys of one triplet give one change, not two);
 *  - theta* is the lowest q with the minimal loss (scanning upwards and
 *    taking strictly smaller values), starting from L(q = -2551);
 *  - the selected candidate is the first with the minimal loss.
 * Plain loops: box sums by double loops, events sorted with qsort. */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OS_QMIN (-2551)

static int64_t os_box(const uint8_t *p, int cx, int cy, int s)
{
    const int x0 = cx - s / 2, y0 = cy - s / 2;
    int64_t acc = 0;
    for (int y = y0; y < y0 + s; ++y)
        for (int x = x0; x < x0 + s; ++x)
            if (x >= 0 && x < 32 && y >= 0 && y < 32)
                acc += p[y * 32 + x];
    return acc;
}

static int64_t os_ceil_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if (q * b < a)
        ++q;
    return q;
}

/* key = ceil(10 (sum1 - sum2) / s^2); cand = {x1, y1, x2, y2, s}. */
int or_select_key(const uint8_t *patch, const int32_t *cand)
{
    const int s = cand[4];
    const int64_t d = os_box(patch, cand[0], cand[1], s) - os_box(patch, cand[2], cand[3], s);
    return (int)os_ceil_div(10 * d, (int64_t)s * s);
}

static int64_t os_term(int tau, int sap, int san, int ha, int hp, int hn)
{
    const int64_t v = (int64_t)tau - sap - ha * hp + san + ha * hn;
    return v > 0 ? v : 0;
}

typedef struct {
    int key;
    int64_t dl;
} os_event;

static int os_cmp(const void *a, const void *b)
{
    const int ka = ((const os_event *)a)->key, kb = ((const os_event *)b)->key;
    return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

/* Algorithm 2 for one candidate.  patches: 3n patches (anchors, positives,
 * negatives); sap, san: n similarities.  Outputs the threshold numerator q
 * (theta = q / 10) and the loss. */
void or_find_threshold(const uint8_t *patches, int n, const int32_t *cand, const int32_t *sap,
                       const int32_t *san, int tau, int32_t *theta_q, int64_t *loss)
{
    os_event *ev = (os_event *)malloc(sizeof(os_event) * (size_t)(3 * n > 0 ? 3 * n : 1));
    int ne = 0;
    int64_t base = 0;
    for (int i = 0; i < n; ++i) {
        const int k[3] = {or_select_key(patches + (size_t)i * 1024, cand),
                          or_select_key(patches + (size_t)(n + i) * 1024, cand),
                          or_select_key(patches + (size_t)(2 * n + i) * 1024, cand)};
        base += os_term(tau, sap[i], san[i], -1, -1, -1);
        for (int m = 0; m < 3; ++m) {
            int dup = 0;
            for (int q = 0; q < m; ++q)
                dup |= k[q] == k[m];
            if (dup)
                continue;
            /* term just at q = k[m] and just below it */
            const int key = k[m];
            const int64_t at = os_term(tau, sap[i], san[i], k[0] <= key ? 1 : -1,
                                       k[1] <= key ? 1 : -1, k[2] <= key ? 1 : -1);
            const int64_t below = os_term(tau, sap[i], san[i], k[0] <= key - 1 ? 1 : -1,
                                          k[1] <= key - 1 ? 1 : -1, k[2] <= key - 1 ? 1 : -1);
            ev[ne].key = key;
            ev[ne].dl = at - below;
            ++ne;
        }
    }
    qsort(ev, (size_t)ne, sizeof(os_event), os_cmp);
    int64_t cur = base, best = base;
    int bestq = OS_QMIN;
    for (int e = 0; e < ne;) {
        const int key = ev[e].key;
        while (e < ne && ev[e].key == key)
            cur += ev[e++].dl;
        if (cur < best) {
            best = cur;
            bestq = key;
        }
    }
    *theta_q = bestq;
    *loss = best;
    free(ev);
}

/* Algorithm 1, one round: the best of J candidates (cands: J x 5). */
void or_select_feature(const uint8_t *patches, int n, const int32_t *cands, int J,
                       const int32_t *sap, const int32_t *san, int tau, int32_t *theta_q,
                       int64_t *loss, int32_t *best)
{
    int b = -1;
    for (int j = 0; j < J; ++j) {
        or_find_threshold(patches, n, cands + (size_t)j * 5, sap, san, tau, theta_q + j, loss + j);
        if (b < 0 || loss[j] < loss[b])
            b = j;
    }
    *best = b;
}
