// Weight kernels of a boosting round (Sec. 2.3):
//  * k_init_weights: the initial weights of Table 2 (1/(2l) per face, 1/(2m)
//    per non-face) or caller-given weights, normalised (step 1).  One CTA.
//  * k_update_a: the round's stump applied to every sample: e_i (misclassified
//    or not) and FP64 partial sums of the misclassified and of all weight.
//    The last CTA to finish forms the error (step 2, exact given the FP32
//    weights), the threshold, beta and alpha (step 3), records the stump, and
//    derives the two factors of the update and renormalisation:
//        w_i <- w_i beta^(1 - e_i) / Z,   Z = M + beta (T - M),
//    M the misclassified weight and T the total (steps 4 and 1).
//  * k_update_b: applies those factors in FP64 and stores the FP32 weights in
//    both copies of the weight array; its last CTA forms the class totals of
//    the stored weights for the next search.
// FP64 is used only for the sums, the error, beta, alpha and the one multiply
// per sample of the renormalisation.
#include <math.h>

#include "vjb_device.cuh"
#include "vjb_internal.cuh"

namespace vjb {

constexpr int kOneCta = 1024;

// Sum of one double per thread over the CTA (every thread gets the result,
// added in a fixed order so that runs are reproducible).
__device__ __forceinline__ double cta_sum(double x, double *red) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    x = warp_sum_d(x);
    __syncthreads();
    if (lane == 0) red[wp] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

__device__ __forceinline__ void store_v(float *v, const WeightLayout &L, int i, float x) {
    v[i] = x;
    if (L.dual) v[L.off_b + rot_b(i)] = x;
}

__global__ void __launch_bounds__(kOneCta)
    k_init_weights(const uint8_t *__restrict__ y, WeightLayout L, const float *__restrict__ w_in,
                   float *__restrict__ w, float *__restrict__ v, RoundState *rs) {
    __shared__ double red[32];
    const int n = L.n;
    double l = 0.0, m = 0.0;
    if (!w_in) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            if (y[i]) l += 1.0; else m += 1.0;
        }
        l = cta_sum(l, red);
        m = cta_sum(m, red);
    }
    // Table 2: 1/(2l) for faces, 1/(2m) for non-faces
    const double wf = w_in ? 0.0 : 1.0 / (2.0 * l), wn = w_in ? 0.0 : 1.0 / (2.0 * m);
    double tot = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        tot += w_in ? (double)w_in[i] : (y[i] ? wf : wn);
    tot = cta_sum(tot, red);
    const double r = 1.0 / tot;
    double tp = 0.0, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double wi = w_in ? (double)w_in[i] : (y[i] ? wf : wn);
        const float f = __double2float_rn(wi * r);
        w[i] = f;
        store_v(v, L, i, y[i] ? f : -f);
        if (y[i]) tp += (double)f; else tn += (double)f;
    }
    tp = cta_sum(tp, red);
    tn = cta_sum(tn, red);
    if (threadIdx.x == 0) {
        v[n] = 0.f;
        rs->t_pos = tp;
        rs->t_neg = tn;
        rs->weight_sum = tp + tn;
        rs->status = VJB_OK;
        rs->cand_count = 0;
        rs->forced = 0;
        rs->done_rescan = rs->done_update_a = rs->done_update_b = 0u;
        if (!(tot > 0.0) || !isfinite(tot)) rs->flags |= kFlagBadWeights;
    }
}

cudaError_t launch_init_weights(const uint8_t *y, const WeightLayout &L, const float *w_in,
                                float *w, float *v, RoundState *rs, cudaStream_t st) {
    k_init_weights<<<1, kOneCta, 0, st>>>(y, L, w_in, w, v, rs);
    return cudaGetLastError();
}

int update_grid(int n) {
    const int g = (n + kUpdateThreads - 1) / kUpdateThreads;
    return g < 1 ? 1 : (g > kUpdateMaxCtas ? kUpdateMaxCtas : g);
}

// Per-CTA reduction of three doubles into partials[3 * blockIdx.x + k].
__device__ __forceinline__ void cta_partials(double a, double b, double c, double *partials) {
    __shared__ double red[3][kUpdateThreads / 32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    c = warp_sum_d(c);
    if (lane == 0) { red[0][wp] = a; red[1][wp] = b; red[2][wp] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < kUpdateThreads / 32; ++k) { s0 += red[0][k]; s1 += red[1][k]; s2 += red[2][k]; }
        partials[3 * blockIdx.x + 0] = s0;
        partials[3 * blockIdx.x + 1] = s1;
        partials[3 * blockIdx.x + 2] = s2;
    }
}

// True in the one CTA that finishes last (thread 0 decides, all threads learn).
__device__ __forceinline__ bool last_cta_done(uint32_t *counter) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__global__ void __launch_bounds__(kUpdateThreads)
    k_update_a(const uint16_t *__restrict__ rows, int npad, WeightLayout L,
               const int32_t *__restrict__ ii_t, int ii_stride, int w, const DevFeature *__restrict__ feat,
               const uint8_t *__restrict__ y, const float *__restrict__ wts, uint8_t *__restrict__ miss,
               double *partials, RoundState *rs, vjb_stump *stumps, vjb_round_diag *diag,
               int stump_cap, vjb_stump *last, const float *__restrict__ ferr) {
    if (rs->status != VJB_OK) return;
    const int n = L.n;
    const bool forced = rs->forced != 0;
    const int32_t f = forced ? rs->forced_feature : rs->win_feature;
    const int32_t p = forced ? rs->forced_polarity : rs->win_polarity;
    const int32_t s = forced ? 0 : rs->win_split;
    const int32_t theta_f = rs->forced_threshold;
    const DevFeature d = feat[f];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double mw = 0.0, tw = 0.0, below = 0.0;
    if (k < n) {
        int i;
        bool h;
        if (!forced) {
            // sorted position k: the first s positions are "below" the threshold
            i = word_to_sample(rows[(size_t)f * npad + phys_of(k, npad / 32)] & kIndexMask, L);
            const bool bl = k < s;
            h = (p > 0) ? bl : !bl;
        } else {
            i = k;
            const int32_t val = haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, i);
            h = (p > 0) ? (val < theta_f) : (val > theta_f);
            below = (p > 0) ? (val < theta_f) : (val <= theta_f);
        }
        const bool m = h != (y[i] != 0);
        miss[i] = m;
        const double wi = (double)wts[i];
        tw = wi;
        if (m) mw = wi;
    }
    cta_partials(mw, tw, below, partials);
    if (!last_cta_done(&rs->done_update_a)) return;
    if (threadIdx.x != 0) return;
    double M = 0.0, T = 0.0, B = 0.0;
    for (unsigned c = 0; c < gridDim.x; ++c) {
        M += ((volatile double *)partials)[3 * c + 0];
        T += ((volatile double *)partials)[3 * c + 1];
        B += ((volatile double *)partials)[3 * c + 2];
    }
    const double eps = M / T;
    int32_t theta, split = s;
    if (forced) {
        theta = theta_f;
        split = (int32_t)B;
    } else {
        // canonical threshold: p=+1 -> value at position s (max+1 at s = n);
        // p=-1 -> value at position s-1 (min-1 at s = 0)
        const uint16_t *row = rows + (size_t)f * npad;
        auto val_at = [&](int pos) {
            const int i = word_to_sample(row[phys_of(pos, npad / 32)] & kIndexMask, L);
            return haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, i);
        };
        if (p > 0) theta = (s < n) ? val_at(s) : val_at(n - 1) + 1;
        else theta = (s > 0) ? val_at(s - 1) : val_at(0) - 1;
    }
    vjb_stump st;
    st.feature = f;
    st.threshold = theta;
    st.polarity = p;
    st.split = split;
    st.error = eps;
    // what the search saw of this stump, next to its FP64 error; the search
    // works in units of the current weight total T, so divide by it
    vjb_round_diag dg;
    dg.search_error = forced ? eps : ((double)rs->win_err_hi + (double)rs->win_err_lo) / T;
    dg.screen_error = forced ? (float)eps : (float)((double)ferr[f] / T);
    dg.screen_min = forced ? (float)eps : (float)((double)rs->screen_min / T);
    dg.candidates = forced ? 0 : rs->cand_count;
    dg.forced = forced ? 1 : 0;
    if (rs->rounds < stump_cap) diag[rs->rounds] = dg;
    rs->last_cands = rs->cand_count;
    rs->cand_count = 0;
    rs->forced = 0;
    rs->done_update_a = 0u;
    if (eps == 0.0) {
        // perfect stump: kept with alpha = +inf, training is over
        st.beta = 0.0;
        st.alpha = INFINITY;
        if (rs->rounds < stump_cap) stumps[rs->rounds] = st;
        rs->rounds += 1;
        *last = st;
        rs->status = VJB_DONE_PERFECT;
        return;
    }
    const double beta = eps / (1.0 - eps);
    st.beta = beta;
    st.alpha = log((1.0 - eps) / eps);  // log(1 / beta)
    *last = st;
    if (eps >= 0.5) {
        // no stump does better than chance: not kept, training is over
        rs->status = VJB_DONE_NOGAIN;
        return;
    }
    if (rs->rounds < stump_cap) stumps[rs->rounds] = st;
    rs->rounds += 1;
    const double Z = M + beta * (T - M);
    rs->scale_hit = beta / Z;
    rs->scale_miss = 1.0 / Z;
}

__global__ void __launch_bounds__(kUpdateThreads)
    k_update_b(WeightLayout L, const uint8_t *__restrict__ y, float *__restrict__ wts,
               float *__restrict__ v, const uint8_t *__restrict__ miss, double *partials,
               RoundState *rs) {
    if (rs->status != VJB_OK) return;
    const int n = L.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double tp = 0.0, tn = 0.0;
    if (i < n) {
        const double scale = miss[i] ? rs->scale_miss : rs->scale_hit;
        const float fw = __double2float_rn((double)wts[i] * scale);
        wts[i] = fw;
        const bool face = y[i] != 0;
        store_v(v, L, i, face ? fw : -fw);
        if (face) tp = (double)fw; else tn = (double)fw;
    }
    cta_partials(tp, tn, 0.0, partials);
    if (!last_cta_done(&rs->done_update_b)) return;
    if (threadIdx.x != 0) return;
    double P = 0.0, Q = 0.0;
    for (unsigned c = 0; c < gridDim.x; ++c) {
        P += ((volatile double *)partials)[3 * c + 0];
        Q += ((volatile double *)partials)[3 * c + 1];
    }
    rs->t_pos = P;
    rs->t_neg = Q;
    rs->weight_sum = P + Q;
    rs->done_update_b = 0u;
}

cudaError_t launch_update_a(const uint16_t *rows, int npad, const WeightLayout &L,
                            const int32_t *ii_t, int ii_stride, int w, const DevFeature *feat,
                            const uint8_t *y, const float *wts, uint8_t *miss, double *partials,
                            RoundState *rs, vjb_stump *stumps, vjb_round_diag *diag, int stump_cap,
                            vjb_stump *last, const float *ferr, cudaStream_t st) {
    k_update_a<<<update_grid(L.n), kUpdateThreads, 0, st>>>(rows, npad, L, ii_t, ii_stride, w, feat, y,
                                                            wts, miss, partials, rs, stumps, diag,
                                                            stump_cap, last, ferr);
    return cudaGetLastError();
}

cudaError_t launch_update_b(const WeightLayout &L, const uint8_t *y, float *wts, float *v,
                            const uint8_t *miss, double *partials, RoundState *rs,
                            cudaStream_t st) {
    k_update_b<<<update_grid(L.n), kUpdateThreads, 0, st>>>(L, y, wts, v, miss, partials, rs);
    return cudaGetLastError();
}

}  // namespace vjb
