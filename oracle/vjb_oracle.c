/*
 * CPU oracle for one Viola-Jones AdaBoost training round (and the loop of
 * rounds) over the full Haar feature set.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path calls this code; it is
 * loaded by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg.  It is deliberately plain and slow: loops over pixels, a merge sort per
 * feature, FP64 sums.  It shares no code, header or table with the CUDA path.
 *
 * What each part follows (Abualkibash, ElSayed, Mahmood, arXiv 1306.1467):
 *   - integral image i(x,y) = sum of o(x',y') for x'<=x, y'<=y      Sec. 2.1
 *   - rectangle sum from four integral-image corners "4 + 1 - (2 + 3)" Sec. 2.1
 *   - five Haar types, value = dark sum minus white sum, enumerated over
 *     every position and every integer scale of the base shape     Sec. 2.2
 *   - decision stump h(x,f,p,theta) = 1 iff p f(x) < p theta          Sec. 2.2
 *   - initial weights 1/(2l) for faces, 1/(2m) for non-faces          Sec. 2.3, Table 2
 *   - per round: normalise; eps = min over (f,p,theta) of
 *     sum_i w_i |h(x_i) - y_i|; beta = eps/(1-eps);
 *     w <- w beta^(1-e_i); alpha = log(1/beta)                      Sec. 2.3 steps 1-4
 *   - strong classifier C(x) = 1 iff sum alpha h >= 1/2 sum alpha     Sec. 2.3
 *
 * Readings where the paper is silent (its Fig. 3 is missing):
 *   - feature geometry: "H" types place their rectangles side by side along x
 *     (base 2x1 or 3x1, width x height), "V" types are the transpose, the
 *     four-rectangle type has base 2x2; every multiple of the base that fits
 *     the window is used at every position.
 *   - sign: two-rectangle value = S(right|bottom) - S(left|top);
 *     three-rectangle value = S(middle) - S(first) - S(last) (no weight 2);
 *     four-rectangle value = S(top-right) + S(bottom-left) - S(top-left)
 *     - S(bottom-right).
 *   - canonical feature order: types 3H, 3V, 2H, 2V, 4 (the order the paper
 *     lists them in); inside a type: width, then height, then y, then x,
 *     all ascending.
 *   - threshold canonical form: a split after the first s samples in value
 *     order is written p=+1, theta = value at position s (max+1 if s = N),
 *     or p=-1, theta = value at position s-1 (min-1 if s = 0).
 *   - ties in error are broken by lowest feature index, then lowest split s,
 *     then p=+1 before p=-1.
 *   - eps == 0 stops training after keeping the stump (alpha = +inf);
 *     eps >= 1/2 stops training without keeping it.
 *
 * Two independent ways to find the per-feature minimum are provided:
 *   tier (a) brute force: every candidate threshold, error summed directly
 *            over all samples, O(N^2) per feature;
 *   tier (b) sorted scan: samples ordered by value (stable), FP64 prefix sums
 *            of positive and of negative weight.
 * Tier (a) pins tier (b) on small inputs; tier (b) is what the GPU path is
 * compared with.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Haar type codes in canonical order. */
enum { ORC_3H = 0, ORC_3V = 1, ORC_2H = 2, ORC_2V = 3, ORC_4 = 4 };
static const int kBaseW[5] = {3, 1, 2, 1, 2};
static const int kBaseH[5] = {1, 3, 1, 2, 2};

typedef struct {
    int64_t feature;
    int32_t split;      /* number of samples on the "below" side in value order */
    int32_t polarity;   /* +1 or -1 */
    int32_t threshold;
    int32_t pad;
    double err;         /* weighted error of this stump */
    double second_err;  /* best error among all other (feature, split, polarity) */
} orc_choice;

typedef struct {
    int64_t feature;
    int32_t threshold;
    int32_t polarity;
    int32_t split;
    int32_t pad;
    double err;
    double beta;
    double alpha;
    double second_err;
} orc_stump;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel loops (the benchmark times 1 and all). */
void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* ---------------------------------------------------------------- Sec. 2.2 */

/* Enumerate every feature of a W x H window in canonical order.  desc may be
 * NULL (count only); otherwise it receives nf rows of (type, x, y, w, h). */
int64_t orc_haar_enumerate(int W, int H, int32_t *desc, int64_t *per_type)
{
    int64_t n = 0;
    for (int t = 0; t < 5; ++t) {
        int64_t cnt = 0;
        for (int w = kBaseW[t]; w <= W; w += kBaseW[t])
            for (int h = kBaseH[t]; h <= H; h += kBaseH[t])
                for (int y = 0; y + h <= H; ++y)
                    for (int x = 0; x + w <= W; ++x) {
                        if (desc) {
                            int32_t *d = desc + 5 * n;
                            d[0] = t; d[1] = x; d[2] = y; d[3] = w; d[4] = h;
                        }
                        ++n;
                        ++cnt;
                    }
        if (per_type) per_type[t] = cnt;
    }
    return n;
}

/* ---------------------------------------------------------------- Sec. 2.1 */

/* Integral image with a zero first row and column:
 * ii[y][x] = sum of px[y'][x'] over y' < y, x' < x, for 0 <= y <= H, 0 <= x <= W. */
void orc_integral(const uint8_t *px, int64_t n, int H, int W, int32_t *ii)
{
    const int64_t S = (int64_t)(H + 1) * (W + 1);
    for (int64_t i = 0; i < n; ++i) {
        const uint8_t *img = px + i * H * W;
        int32_t *o = ii + i * S;
        for (int x = 0; x <= W; ++x) o[x] = 0;
        for (int y = 1; y <= H; ++y) {
            o[y * (W + 1)] = 0;
            for (int x = 1; x <= W; ++x)
                o[y * (W + 1) + x] = img[(y - 1) * W + (x - 1)]
                                   + o[(y - 1) * (W + 1) + x]
                                   + o[y * (W + 1) + x - 1]
                                   - o[(y - 1) * (W + 1) + x - 1];
        }
    }
}

/* Rectangle sum by adding up pixels. */
static int32_t rect_direct(const uint8_t *img, int W, int x, int y, int w, int h)
{
    int32_t s = 0;
    for (int yy = y; yy < y + h; ++yy)
        for (int xx = x; xx < x + w; ++xx) s += img[yy * W + xx];
    return s;
}

/* Rectangle sum from the four corners of the integral image (points 1..4 of
 * the paper's Fig. 2: 4 + 1 - (2 + 3)). */
static int32_t rect_ii(const int32_t *ii, int W, int x, int y, int w, int h)
{
    const int s = W + 1;
    int32_t p1 = ii[y * s + x], p2 = ii[y * s + x + w];
    int32_t p3 = ii[(y + h) * s + x], p4 = ii[(y + h) * s + x + w];
    return p4 + p1 - (p2 + p3);
}

/* Value of one feature given a rectangle-sum function. */
#define FEATURE_VALUE(RECT, SRC)                                                  \
    do {                                                                          \
        switch (t) {                                                              \
        case ORC_2H: { int a = w / 2;                                             \
            v = RECT(SRC, W, x + a, y, a, h) - RECT(SRC, W, x, y, a, h); } break;  \
        case ORC_2V: { int b = h / 2;                                             \
            v = RECT(SRC, W, x, y + b, w, b) - RECT(SRC, W, x, y, w, b); } break;  \
        case ORC_3H: { int a = w / 3;                                             \
            v = RECT(SRC, W, x + a, y, a, h) - RECT(SRC, W, x, y, a, h)            \
              - RECT(SRC, W, x + 2 * a, y, a, h); } break;                         \
        case ORC_3V: { int b = h / 3;                                             \
            v = RECT(SRC, W, x, y + b, w, b) - RECT(SRC, W, x, y, w, b)            \
              - RECT(SRC, W, x, y + 2 * b, w, b); } break;                         \
        default: { int a = w / 2, b = h / 2;                                      \
            v = RECT(SRC, W, x + a, y, a, b) + RECT(SRC, W, x, y + b, a, b)        \
              - RECT(SRC, W, x, y, a, b) - RECT(SRC, W, x + a, y + b, a, b); }     \
        }                                                                         \
    } while (0)

/* Tier (a) feature values: rectangle sums by pixel loops.  out is [nf][n]. */
void orc_feature_values_direct(const uint8_t *px, int64_t n, int H, int W,
                               const int32_t *desc, int64_t nf, int32_t *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t f = 0; f < nf; ++f) {
        const int t = desc[5 * f], x = desc[5 * f + 1], y = desc[5 * f + 2];
        const int w = desc[5 * f + 3], h = desc[5 * f + 4];
        for (int64_t i = 0; i < n; ++i) {
            const uint8_t *img = px + i * H * W;
            int32_t v;
            FEATURE_VALUE(rect_direct, img);
            out[f * n + i] = v;
        }
    }
}

/* Tier (b) feature values: rectangle sums from the integral images. */
void orc_feature_values_integral(const int32_t *ii, int64_t n, int H, int W,
                                 const int32_t *desc, int64_t nf, int32_t *out)
{
    const int64_t S = (int64_t)(H + 1) * (W + 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t f = 0; f < nf; ++f) {
        const int t = desc[5 * f], x = desc[5 * f + 1], y = desc[5 * f + 2];
        const int w = desc[5 * f + 3], h = desc[5 * f + 4];
        for (int64_t i = 0; i < n; ++i) {
            const int32_t *img = ii + i * S;
            int32_t v;
            FEATURE_VALUE(rect_ii, img);
            out[f * n + i] = v;
        }
    }
}

/* ------------------------------------------------------- ordering by value */

/* Stable merge sort of sample indices by value (equal values keep index order). */
static void merge_sort(int32_t *a, int32_t *tmp, int64_t n, const int32_t *val)
{
    for (int64_t i = 0; i < n; ++i) a[i] = (int32_t)i;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = (val[a[j]] < val[a[i]]) ? a[j++] : a[i++];
            while (i < mid) tmp[k++] = a[i++];
            while (j < hi) tmp[k++] = a[j++];
        }
        memcpy(a, tmp, (size_t)n * sizeof(int32_t));
    }
}

/* order[f][k] = index of the sample at position k when feature f's values are
 * sorted ascending, ties by ascending sample index. */
void orc_sort_rows(const int32_t *vals, int64_t nf, int64_t n, int32_t *order)
{
#pragma omp parallel
    {
        int32_t *tmp = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t f = 0; f < nf; ++f) merge_sort(order + f * n, tmp, n, vals + f * n);
        free(tmp);
    }
}

/* -------------------------------------------------- per-feature best stump */

/* Candidate ordering: error, then split, then +1 before -1 (inside a feature). */
static int cand_less(double e1, int s1, int p1, double e2, int s2, int p2)
{
    if (e1 != e2) return e1 < e2;
    if (s1 != s2) return s1 < s2;
    return p1 > p2;
}

typedef struct { double e1; int s1, p1; double e2; } best2;

static void consider(best2 *b, double e, int s, int p)
{
    if (cand_less(e, s, p, b->e1, b->s1, b->p1)) {
        b->e2 = b->e1;
        b->e1 = e; b->s1 = s; b->p1 = p;
    } else if (e < b->e2) {
        b->e2 = e;
    }
}

static int32_t canonical_theta(const int32_t *val, const int32_t *ord, int64_t n, int s, int p)
{
    if (p > 0) return s < n ? val[ord[s]] : val[ord[n - 1]] + 1;
    return s > 0 ? val[ord[s - 1]] : val[ord[0]] - 1;
}

/* Tier (b): per feature, scan samples in value order keeping FP64 prefix sums
 * S+ (faces) and S- (non-faces) of the weights.  A split after s samples is a
 * threshold only where the values at positions s-1 and s differ (or s = 0, N).
 *   p = +1 ("below" is a face):  err = S-(s) + (T+ - S+(s))
 *   p = -1 ("above" is a face):  err = S+(s) + (T- - S-(s))
 * Writes the feature's best (err, split, polarity, theta) and its second-best
 * error among the feature's other candidates. */
void orc_feature_best_sorted(const int32_t *vals, const int32_t *order, int64_t nf, int64_t n,
                             const uint8_t *y, const double *w,
                             double *err, int32_t *split, int32_t *pol, int32_t *theta,
                             double *err2)
{
    double Tp = 0.0, Tm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (y[i]) Tp += w[i]; else Tm += w[i];
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t *val = vals + f * n;
        const int32_t *ord = order + f * n;
        best2 b = {INFINITY, 0, 1, INFINITY};
        double Sp = 0.0, Sm = 0.0;
        consider(&b, Tp, 0, +1);
        consider(&b, Tm, 0, -1);
        for (int64_t k = 0; k < n; ++k) {
            const int32_t i = ord[k];
            if (y[i]) Sp += w[i]; else Sm += w[i];
            const int64_t s = k + 1;
            if (s == n || val[ord[k]] < val[ord[k + 1]]) {
                consider(&b, Sm + (Tp - Sp), (int)s, +1);
                consider(&b, Sp + (Tm - Sm), (int)s, -1);
            }
        }
        err[f] = b.e1; split[f] = b.s1; pol[f] = b.p1;
        theta[f] = canonical_theta(val, ord, n, b.s1, b.p1);
        if (err2) err2[f] = b.e2;
    }
}

static int cmp_int32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Tier (a): brute force.  For p = +1 every distinct value and max+1 is tried as
 * theta, for p = -1 every distinct value and min-1; the error of each
 * candidate is summed over all samples straight from the stump definition.
 * The split s of a candidate is the number of samples it puts "below"
 * (value < theta for p=+1, value <= theta for p=-1). */
void orc_feature_best_brute(const int32_t *vals, int64_t nf, int64_t n,
                            const uint8_t *y, const double *w,
                            double *err, int32_t *split, int32_t *pol, int32_t *theta,
                            double *err2)
{
#pragma omp parallel
    {
        int32_t *u = (int32_t *)malloc((size_t)(n + 2) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 4)
        for (int64_t f = 0; f < nf; ++f) {
            const int32_t *val = vals + f * n;
            memcpy(u, val, (size_t)n * sizeof(int32_t));
            qsort(u, (size_t)n, sizeof(int32_t), cmp_int32);
            int64_t nd = 0;
            for (int64_t k = 0; k < n; ++k)
                if (k == 0 || u[k] != u[nd - 1]) u[nd++] = u[k];
            best2 b = {INFINITY, 0, 1, INFINITY};
            int32_t bt = 0;
            for (int p = 1; p >= -1; p -= 2) {
                for (int64_t c = 0; c <= nd; ++c) {
                    int32_t th;
                    if (p > 0) th = c < nd ? u[c] : u[nd - 1] + 1;
                    else th = c == 0 ? u[0] - 1 : u[c - 1];
                    double e = 0.0;
                    int s = 0;
                    for (int64_t i = 0; i < n; ++i) {
                        int h = (p > 0) ? (val[i] < th) : (val[i] > th);
                        int below = (p > 0) ? (val[i] < th) : (val[i] <= th);
                        s += below;
                        if (h != (int)y[i]) e += w[i];
                    }
                    double old = b.e1; int os = b.s1, op = b.p1;
                    consider(&b, e, s, p);
                    if (b.e1 != old || b.s1 != os || b.p1 != op) bt = th;
                }
            }
            err[f] = b.e1; split[f] = b.s1; pol[f] = b.p1; theta[f] = bt;
            if (err2) err2[f] = b.e2;
        }
        free(u);
    }
}

/* Across features: the lowest (err, feature, split, polarity) and the best
 * error of every other candidate (its own second best or another feature's best). */
void orc_select(const double *err, const int32_t *split, const int32_t *pol,
                const int32_t *theta, const double *err2, int64_t nf, orc_choice *out)
{
    int64_t bf = -1;
    for (int64_t f = 0; f < nf; ++f) {
        if (bf < 0 || err[f] < err[bf]) bf = f;   /* first lowest = lowest index on ties */
    }
    double sec = err2 ? err2[bf] : INFINITY;
    for (int64_t f = 0; f < nf; ++f)
        if (f != bf && err[f] < sec) sec = err[f];
    out->feature = bf; out->split = split[bf]; out->polarity = pol[bf];
    out->threshold = theta[bf]; out->err = err[bf]; out->second_err = sec; out->pad = 0;
}

/* ------------------------------------------------------------- Sec. 2.3 */

/* Initial weights of Table 2: 1/(2l) for each of the l faces, 1/(2m) for each
 * of the m non-faces. */
void orc_initial_weights(const uint8_t *y, int64_t n, double *w)
{
    int64_t l = 0, m = 0;
    for (int64_t i = 0; i < n; ++i) { if (y[i]) ++l; else ++m; }
    for (int64_t i = 0; i < n; ++i) w[i] = y[i] ? 1.0 / (2.0 * (double)l) : 1.0 / (2.0 * (double)m);
}

/* Step 1: w_i <- w_i / sum_j w_j. */
void orc_normalize(double *w, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += w[i];
    for (int64_t i = 0; i < n; ++i) w[i] /= s;
}

/* h(x_i) of a stump on one feature's values. */
static int stump_h(int32_t v, int32_t theta, int p)
{
    return p > 0 ? (v < theta) : (v > theta);
}

/* Weighted error of a given stump, summed straight from the definition. */
double orc_stump_error(const int32_t *val, int64_t n, const uint8_t *y, const double *w,
                       int32_t theta, int32_t p)
{
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (stump_h(val[i], theta, p) != (int)y[i]) e += w[i];
    return e;
}

/* Step 4: w_i <- w_i beta^(1 - e_i), e_i = 1 if x_i is misclassified. */
void orc_update(const int32_t *val, int64_t n, const uint8_t *y, double *w,
                int32_t theta, int32_t p, double beta)
{
    for (int64_t i = 0; i < n; ++i)
        if (stump_h(val[i], theta, p) == (int)y[i]) w[i] *= beta;
}

/* One boosting round (steps 1-4) on prepared values/orders.  w is updated in
 * place.  Returns 0 for a normal round, 1 if eps == 0 (stump kept, training
 * over), 2 if eps >= 1/2 (stump not kept, training over). */
int orc_round(const int32_t *vals, const int32_t *order, int64_t nf, int64_t n,
              const uint8_t *y, double *w, orc_stump *out)
{
    orc_normalize(w, n);
    double *err = (double *)malloc((size_t)nf * sizeof(double));
    double *err2 = (double *)malloc((size_t)nf * sizeof(double));
    int32_t *split = (int32_t *)malloc((size_t)nf * sizeof(int32_t));
    int32_t *pol = (int32_t *)malloc((size_t)nf * sizeof(int32_t));
    int32_t *theta = (int32_t *)malloc((size_t)nf * sizeof(int32_t));
    orc_feature_best_sorted(vals, order, nf, n, y, w, err, split, pol, theta, err2);
    orc_choice c;
    orc_select(err, split, pol, theta, err2, nf, &c);
    free(err); free(err2); free(split); free(pol); free(theta);

    const int32_t *val = vals + c.feature * n;
    const double eps = orc_stump_error(val, n, y, w, c.threshold, c.polarity);
    out->feature = c.feature; out->threshold = c.threshold; out->polarity = c.polarity;
    out->split = c.split; out->pad = 0; out->err = eps; out->second_err = c.second_err;
    if (eps == 0.0) {
        out->beta = 0.0; out->alpha = INFINITY;
        return 1;
    }
    if (eps >= 0.5) {
        out->beta = eps / (1.0 - eps); out->alpha = log(1.0 / out->beta);
        return 2;
    }
    out->beta = eps / (1.0 - eps);
    out->alpha = log(1.0 / out->beta);
    orc_update(val, n, y, w, c.threshold, c.polarity, out->beta);
    return 0;
}

/* T rounds.  Stumps of kept rounds go to out[0 .. *rounds_done). */
int orc_train(const int32_t *vals, const int32_t *order, int64_t nf, int64_t n,
              const uint8_t *y, double *w, int32_t T, orc_stump *out, int32_t *rounds_done)
{
    int32_t done = 0;
    int status = 0;
    for (int32_t t = 0; t < T; ++t) {
        orc_stump s;
        status = orc_round(vals, order, nf, n, y, w, &s);
        if (status == 2) break;
        out[done++] = s;
        if (status == 1) break;
    }
    *rounds_done = done;
    return status;
}

/* Strong classifier: C(x) = 1 iff sum_t alpha_t h_t(x) >= 1/2 sum_t alpha_t.
 * fval is [T][n]: the value of stump t's feature on each sample. */
void orc_strong_classify(const int32_t *fval, int64_t n, const orc_stump *st, int32_t T,
                         uint8_t *out)
{
    double half = 0.0;
    for (int32_t t = 0; t < T; ++t) half += st[t].alpha;
    half *= 0.5;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t t = 0; t < T; ++t)
            if (stump_h(fval[(int64_t)t * n + i], st[t].threshold, st[t].polarity)) s += st[t].alpha;
        out[i] = s >= half;
    }
}
