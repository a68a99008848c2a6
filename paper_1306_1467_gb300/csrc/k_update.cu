// Weight kernels of a boosting round (Sec. 2.3):
//  * k_init_weights: the initial weights of Table 2 (1/(2l) per face, 1/(2m)
//    per non-face) or caller-given weights, normalised (step 1).
//  * k_finalize: picks the winning stump from the shortlist (step 3), computes
//    its error exactly in FP64 from the FP32 weights, its threshold, beta and
//    alpha, then reweights w <- w beta^(1 - e) (step 4) and normalises for the
//    next round (step 1).
// Both run as one CTA: their work is O(N) against the O(F N) search.
#include <math.h>

#include "vjb_device.cuh"
#include "vjb_internal.cuh"

namespace vjb {

constexpr int kOneCta = 1024;

// Sum of one double per thread over the CTA (all threads get the result).
__device__ __forceinline__ double cta_sum(double x, double *red) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    x = warp_sum_d(x);
    __syncthreads();
    if (lane == 0) red[wp] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];  // fixed order: deterministic
    return s;
}

__global__ void __launch_bounds__(kOneCta)
    k_init_weights(const uint8_t *__restrict__ y, int n, const float *__restrict__ w_in,
                   float *__restrict__ w, float *__restrict__ v, RoundState *rs) {
    __shared__ double red[32];
    double l = 0.0, m = 0.0;
    if (!w_in) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            if (y[i]) l += 1.0; else m += 1.0;
        }
        l = cta_sum(l, red);
        m = cta_sum(m, red);
    }
    // Table 2: 1/(2l) for faces, 1/(2m) for non-faces
    const double wp_ = w_in ? 0.0 : 1.0 / (2.0 * l), wn_ = w_in ? 0.0 : 1.0 / (2.0 * m);
    double tot = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        tot += w_in ? (double)w_in[i] : (y[i] ? wp_ : wn_);
    tot = cta_sum(tot, red);
    double tp = 0.0, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double wi = w_in ? (double)w_in[i] : (y[i] ? wp_ : wn_);
        const float f = __double2float_rn(wi / tot);
        w[i] = f;
        v[i] = y[i] ? f : -f;
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
        if (!(tot > 0.0) || !isfinite(tot)) rs->flags |= kFlagBadWeights;
    }
}

cudaError_t launch_init_weights(const uint8_t *y, int n, const float *w_in, float *w, float *v,
                                RoundState *rs, cudaStream_t st) {
    k_init_weights<<<1, kOneCta, 0, st>>>(y, n, w_in, w, v, rs);
    return cudaGetLastError();
}

// Candidate order: error (double-float), then feature, split, +1 before -1.
__device__ __forceinline__ bool cand_less(const Candidate &a, const Candidate &b) {
    if (a.err_hi != b.err_hi) return a.err_hi < b.err_hi;
    if (a.err_lo != b.err_lo) return a.err_lo < b.err_lo;
    if (a.feature != b.feature) return a.feature < b.feature;
    if (a.split != b.split) return a.split < b.split;
    return a.polarity > b.polarity;
}

__device__ __forceinline__ Candidate cand_shfl_xor(const Candidate &c, int d) {
    Candidate o;
    o.err_hi = __shfl_xor_sync(0xffffffffu, c.err_hi, d);
    o.err_lo = __shfl_xor_sync(0xffffffffu, c.err_lo, d);
    o.feature = __shfl_xor_sync(0xffffffffu, c.feature, d);
    o.split = __shfl_xor_sync(0xffffffffu, c.split, d);
    o.polarity = __shfl_xor_sync(0xffffffffu, c.polarity, d);
    o.pad = 0;
    return o;
}

__global__ void __launch_bounds__(kOneCta)
    k_finalize(const uint16_t *__restrict__ rows, int npad, int n, const int32_t *__restrict__ ii_t,
               int ii_stride, int w, const DevFeature *__restrict__ feat, int64_t nfeat,
               const uint8_t *__restrict__ y, float *__restrict__ wts, float *__restrict__ v,
               RoundState *rs, const Candidate *__restrict__ cands, vjb_stump *stumps,
               int stump_cap, vjb_stump *last) {
    __shared__ double red[32];
    __shared__ Candidate wc[32];
    __shared__ uint8_t miss[VJB_MAX_SAMPLES + 2];
    __shared__ int32_t s_theta;
    if (rs->status != VJB_OK) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const bool forced = rs->forced != 0;

    // ---- step 3: the chosen stump
    int32_t f, s = 0, p, theta = 0;
    if (!forced) {
        const int cnt = rs->cand_count;
        Candidate b;
        b.err_hi = INFINITY; b.err_lo = 0.f; b.feature = 0x7fffffff; b.split = 0x7fffffff;
        b.polarity = 1; b.pad = 0;
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const Candidate c = cands[k];
            if (cand_less(c, b)) b = c;
        }
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            const Candidate o = cand_shfl_xor(b, d);
            if (cand_less(o, b)) b = o;
        }
        if (lane == 0) wc[wp] = b;
        __syncthreads();
        b = wc[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            if (cand_less(wc[k], b)) b = wc[k];
        if (cnt == 0 || b.feature < 0 || b.feature >= nfeat) {
            if (threadIdx.x == 0) rs->flags |= kFlagNoCandidate;
            return;
        }
        f = b.feature;
        s = b.split;
        p = b.polarity;
    } else {
        f = rs->forced_feature;
        p = rs->forced_polarity;
        theta = rs->forced_threshold;
    }
    const DevFeature d = feat[f];

    // error of the stump on the current weights, FP64 (Sec. 2.3 step 2), and e_i
    double eacc = 0.0, tacc = 0.0, below = 0.0;
    if (!forced) {
        const uint16_t *row = rows + (size_t)f * npad;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int i = row[k] & kIndexMask;
            const bool bl = k < s;
            const bool h = (p > 0) ? bl : !bl;
            const bool m = h != (y[i] != 0);
            miss[i] = m;
            const double wi = (double)wts[i];
            tacc += wi;
            if (m) eacc += wi;
        }
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int32_t val = haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, i);
            const bool h = (p > 0) ? (val < theta) : (val > theta);
            below += (p > 0) ? (val < theta) : (val <= theta);
            const bool m = h != (y[i] != 0);
            miss[i] = m;
            const double wi = (double)wts[i];
            tacc += wi;
            if (m) eacc += wi;
        }
    }
    eacc = cta_sum(eacc, red);
    tacc = cta_sum(tacc, red);
    if (forced) {
        s = (int32_t)cta_sum(below, red);
    } else if (threadIdx.x == 0) {
        // canonical threshold: p=+1 -> value at position s (max+1 at s = n);
        // p=-1 -> value at position s-1 (min-1 at s = 0)
        const uint16_t *row = rows + (size_t)f * npad;
        int32_t th;
        if (p > 0) {
            th = (s < n) ? haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, row[s] & kIndexMask)
                         : haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, row[n - 1] & kIndexMask) + 1;
        } else {
            th = (s > 0) ? haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, row[s - 1] & kIndexMask)
                         : haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, row[0] & kIndexMask) - 1;
        }
        s_theta = th;
    }
    __syncthreads();
    if (!forced) theta = s_theta;

    const double eps = eacc / tacc;
    vjb_stump st;
    st.feature = f;
    st.threshold = theta;
    st.polarity = p;
    st.split = s;
    st.error = eps;
    if (eps == 0.0) {
        st.beta = 0.0;
        st.alpha = INFINITY;
        if (threadIdx.x == 0) {
            if (rs->rounds < stump_cap) stumps[rs->rounds] = st;
            rs->rounds += 1;
            *last = st;
            rs->status = VJB_DONE_PERFECT;
            rs->last_cands = rs->cand_count;
            rs->cand_count = 0;
            rs->forced = 0;
        }
        return;
    }
    const double beta = eps / (1.0 - eps);
    st.beta = beta;
    st.alpha = log((1.0 - eps) / eps);  // log(1 / beta)
    if (eps >= 0.5) {
        if (threadIdx.x == 0) {
            *last = st;
            rs->status = VJB_DONE_NOGAIN;
            rs->last_cands = rs->cand_count;
            rs->cand_count = 0;
            rs->forced = 0;
        }
        return;
    }

    // ---- step 4: w <- w beta^(1 - e), then step 1 of the next round: w <- w / sum w
    double uacc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double wi = (double)wts[i];
        uacc += miss[i] ? wi : wi * beta;
    }
    const double utot = cta_sum(uacc, red);
    double tp = 0.0, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double wi = (double)wts[i];
        const double wn = miss[i] ? wi : wi * beta;
        const float fw = __double2float_rn(wn / utot);
        wts[i] = fw;
        const bool face = y[i] != 0;
        v[i] = face ? fw : -fw;
        if (face) tp += (double)fw; else tn += (double)fw;
    }
    tp = cta_sum(tp, red);
    tn = cta_sum(tn, red);
    if (threadIdx.x == 0) {
        if (rs->rounds < stump_cap) stumps[rs->rounds] = st;
        rs->rounds += 1;
        *last = st;
        rs->t_pos = tp;
        rs->t_neg = tn;
        rs->weight_sum = tp + tn;
        rs->last_cands = rs->cand_count;
        rs->cand_count = 0;
        rs->forced = 0;
    }
}

cudaError_t launch_finalize(const uint16_t *rows, int npad, int n, const int32_t *ii_t,
                            int ii_stride, int w, const DevFeature *feat, int64_t nfeat,
                            const uint8_t *y, float *wts, float *v, RoundState *rs,
                            const Candidate *cands, vjb_stump *stumps, int stump_cap,
                            vjb_stump *last, cudaStream_t st) {
    k_finalize<<<1, kOneCta, 0, st>>>(rows, npad, n, ii_t, ii_stride, w, feat, nfeat, y, wts, v, rs,
                                      cands, stumps, stump_cap, last);
    return cudaGetLastError();
}

}  // namespace vjb
