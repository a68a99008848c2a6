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
#include "vjb_haar.cuh"
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
    if (L.dual && i < L.nb) v[L.off_b + rot_b(i)] = x;
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
        rs->screen_min_bits = 0x7f800000u;
        rs->in_round = 0;
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

// Per-CTA reduction of three doubles into partials[3 * blk + k].  FP64 runs
// at a couple of lanes per clock per SM on this GPU, so a warp-wide FP64 add
// takes the FP64 pipe of its scheduler for tens of cycles: each value is
// summed by a warp of its own (warps 0, 1, 2 sit on different schedulers),
// lane l adding the threads l, l + 32, ... in order and the lanes then by a
// butterfly, 13 warp-wide adds a value instead of 40 spread over the CTA.
// The third value is reduced only where it can be non-zero (`third`, uniform
// over the launch), and its slot is 0 otherwise.
__device__ __forceinline__ void cta_partials(double a, double b, double c, bool third, double *partials, int blk) {
    __shared__ double red[3][kUpdateThreads];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    if (third) red[2][threadIdx.x] = c;
    __syncthreads();
    if (wp < 3) {
        double x = 0.0;
        if (wp < 2 || third) {
#pragma unroll
            for (int k = 0; k < kUpdateThreads / 32; ++k) x += red[wp][lane + 32 * k];
            x = warp_sum_d(x);
        }
        if (lane == 0) partials[3 * blk + wp] = x;
    }
}

// True in the CTA that finishes the last of `nblocks` blocks counted on
// `counter` (thread 0 decides, all threads learn).
__device__ __forceinline__ bool last_block_done(uint32_t *counter, int nblocks) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == (uint32_t)nblocks - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Step 3-4, part 1, for the 256 samples (or sorted positions) of block `blk`:
// e_i and the block's FP64 sums of misclassified weight, of all weight and (for
// a host-given stump) of samples below the threshold.  The round state's
// fields are read in one trip with the status; false (nothing done, uniform
// over the CTA) when the job has stopped or, in a batch, sits this round out.
__device__ bool update_a_block(const JobDesc &J, int blk, bool batched) {
    const int n = J.lay.n;
    const RoundState *rs = J.rs;
    const int32_t status = rs->status, in_round = rs->in_round, forced_i = rs->forced;
    const int32_t ff = rs->forced_feature, wf = rs->win_feature;
    const int32_t fp = rs->forced_polarity, wp = rs->win_polarity, ws = rs->win_split;
    const int32_t theta_f = rs->forced_threshold;
    if (status != VJB_OK || (batched && !in_round)) return false;
    const bool forced = forced_i != 0;
    const int32_t f = forced ? ff : wf;
    const int32_t p = forced ? fp : wp;
    const int32_t s = forced ? 0 : ws;
    const int k = blk * kUpdateThreads + threadIdx.x;
    double mw = 0.0, tw = 0.0, below = 0.0;
    if (k < n) {
        int i;
        bool h;
        if (!forced) {
            // sorted position k: the first s positions are "below" the threshold
            const int P = phys_of(k, J.npad / 32);
            i = word_to_sample(entry_word(J.rows[(size_t)f * J.npad + P], P), J.lay);
            const bool bl = k < s;
            h = (p > 0) ? bl : !bl;
        } else {
            i = k;
            const DevFeature d = J.feat[f];
            const int32_t val = haar_value(J.ii, J.ii_stride, J.win_w, d.type, d.x, d.y, d.w, d.h, i);
            h = (p > 0) ? (val < theta_f) : (val > theta_f);
            below = (p > 0) ? (val < theta_f) : (val <= theta_f);
        }
        const bool m = h != (J.y[i] != 0);
        J.miss[i] = m;
        const double wi = (double)J.w[i];
        tw = wi;
        if (m) mw = wi;
    }
    cta_partials(mw, tw, below, forced, J.partials, blk);
    return true;
}

// Sums of the three per-block partials over `nblocks` blocks by the finishing
// CTA in a fixed order, each value by a warp of its own (lane l adds blocks
// l, l + 32, ... in order, then the lanes by a butterfly); every thread gets
// them.  The third only where it can be non-zero (`third`), as in
// cta_partials.
__device__ __forceinline__ void sum_partials(const double *partials, int nblocks, bool third, double &a,
                                             double &b, double &c) {
    __shared__ double tot[3];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (wp < 3) {
        double x = 0.0;
        if (wp < 2 || third) {
            for (int k = lane; k < nblocks; k += 32) x += ((volatile const double *)partials)[3 * k + wp];
            x = warp_sum_d(x);
        }
        if (lane == 0) tot[wp] = x;
    }
    __syncthreads();
    a = tot[0];
    b = tot[1];
    c = tot[2];
}

// The searched stump's canonical threshold: p=+1 -> value at position s
// (max+1 at s = n); p=-1 -> value at position s-1 (min-1 at s = 0).  One
// thread of the update's first block stores it in the round state before
// that block is counted, off the finishing block's path.
__device__ void store_threshold(const JobDesc &J) {
    RoundState *rs = J.rs;
    if (rs->forced) return;
    const int n = J.lay.n;
    const int32_t f = rs->win_feature, p = rs->win_polarity, s = rs->win_split;
    const DevFeature d = J.feat[f];
    const uint16_t *row = J.rows + (size_t)f * J.npad;
    auto val_at = [&](int pos) {
        const int P = phys_of(pos, J.npad / 32);
        const int i = word_to_sample(entry_word(row[P], P), J.lay);
        return haar_value(J.ii, J.ii_stride, J.win_w, d.type, d.x, d.y, d.w, d.h, i);
    };
    int32_t theta;
    if (p > 0) theta = (s < n) ? val_at(s) : val_at(n - 1) + 1;
    else theta = (s > 0) ? val_at(s - 1) : val_at(0) - 1;
    rs->win_theta = theta;
}

// Step 3-4, part 1, finish (after every block; the CTA's threads have summed
// the partials): the stump's FP64 error, threshold, beta and alpha, its
// record, and the update factors.  Three warps share the scalar work, so that
// the factors update b waits for do not queue behind the logarithm, the
// divisions of the diagnostics and their memory traffic (one thread did all of
// it in 7.5 us of a 13.3 us update at 24x24 / 15k): warp 0 the factors and
// the round state, warp 1 alpha and the stump record, warp 2 the diagnostics.
// Each value is computed exactly as one thread would.
__device__ void update_a_finish(const JobDesc &J, double M, double T, double B) {
    RoundState *rs = J.rs;
    // the round state the parts read, taken before any part writes it
    const bool forced = rs->forced != 0;
    const int32_t f = forced ? rs->forced_feature : rs->win_feature;
    const int32_t p = forced ? rs->forced_polarity : rs->win_polarity;
    const int32_t s = forced ? 0 : rs->win_split;
    const int32_t r0 = rs->rounds;
    const int32_t cands = rs->cand_count;
    __syncthreads();
    const double eps = M / T;
    if (threadIdx.x == 0) {
        rs->last_cands = cands;
        rs->cand_count = 0;
        rs->forced = 0;
        rs->done_update_a = 0u;
        if (eps == 0.0) {
            // perfect stump: kept with alpha = +inf, training is over
            rs->rounds = r0 + 1;
            rs->status = VJB_DONE_PERFECT;
        } else if (eps >= 0.5) {
            // no stump does better than chance: not kept, training is over
            rs->status = VJB_DONE_NOGAIN;
        } else {
            const double beta = eps / (1.0 - eps);
            rs->rounds = r0 + 1;
            const double Z = M + beta * (T - M);
            rs->scale_hit = beta / Z;
            rs->scale_miss = 1.0 / Z;
        }
    } else if (threadIdx.x == 32) {
        int32_t theta, split = s;
        if (forced) {
            theta = rs->forced_threshold;
            split = (int32_t)B;
        } else {
            // written by another CTA in this launch: read past this SM's L1
            theta = *reinterpret_cast<volatile int32_t *>(&rs->win_theta);
        }
        vjb_stump st;
        st.feature = f;
        st.threshold = theta;
        st.polarity = p;
        st.split = split;
        st.error = eps;
        if (eps == 0.0) {
            st.beta = 0.0;
            st.alpha = INFINITY;
        } else {
            st.beta = eps / (1.0 - eps);
            st.alpha = log((1.0 - eps) / eps);  // log(1 / beta)
        }
        *J.last = st;
        if (eps < 0.5 && r0 < J.stump_cap) J.stumps[r0] = st;
    } else if (threadIdx.x == 64) {
        // what the search saw of this stump, next to its FP64 error; the search
        // works in units of the current weight total T, so divide by it
        vjb_round_diag dg;
        dg.search_error = forced ? eps : ((double)rs->win_err_hi + (double)rs->win_err_lo) / T;
        dg.screen_error = forced ? (float)eps : (float)((double)J.ferr[f] / T);
        dg.screen_min = forced ? (float)eps : (float)((double)rs->screen_min / T);
        dg.candidates = forced ? 0 : cands;
        dg.forced = forced ? 1 : 0;
        if (r0 < J.stump_cap) J.diag[r0] = dg;
    }
}

// Step 4 and step 1 of the next round for the 256 samples of block `blk`.  The
// samples' miss flags, weights and labels are read in the same trip as the
// round state; false as for update_a_block.
__device__ bool update_b_block(const JobDesc &J, int blk, bool batched) {
    const int i = blk * kUpdateThreads + threadIdx.x;
    const bool in = i < J.lay.n;
    const bool miss = in && J.miss[i];
    const float w0 = in ? J.w[i] : 0.f;
    const bool face = in && J.y[i] != 0;
    const RoundState *rs = J.rs;
    const int32_t status = rs->status, in_round = rs->in_round;
    const double scale_miss = rs->scale_miss, scale_hit = rs->scale_hit;
    if (status != VJB_OK || (batched && !in_round)) return false;
    double tp = 0.0, tn = 0.0;
    if (in) {
        const double scale = miss ? scale_miss : scale_hit;
        const float fw = __double2float_rn((double)w0 * scale);
        J.w[i] = fw;
        store_v(J.v, J.lay, i, face ? fw : -fw);
        if (face) tp = (double)fw; else tn = (double)fw;
    }
    cta_partials(tp, tn, 0.0, false, J.partials, blk);
    return true;
}

__device__ void update_b_finish(const JobDesc &J, double P, double Q) {
    RoundState *rs = J.rs;
    rs->t_pos = P;
    rs->t_neg = Q;
    rs->weight_sum = P + Q;
    rs->done_update_b = 0u;
}

// The finishing CTA of update a / update b (all its threads).
__device__ void finish_a(const JobDesc &J, int nblocks) {
    double M, T, B;
    // (the count below the threshold only for a host-given stump; read before
    // any part of the finish resets `forced`)
    sum_partials(J.partials, nblocks, J.rs->forced != 0, M, T, B);
    update_a_finish(J, M, T, B);
}

__device__ void finish_b(const JobDesc &J, int nblocks) {
    double P, Q, unused;
    sum_partials(J.partials, nblocks, false, P, Q, unused);
    if (threadIdx.x == 0) update_b_finish(J, P, Q);
}

__global__ void __launch_bounds__(kUpdateThreads) k_update_a(const JobDesc J) {
    if (!update_a_block(J, blockIdx.x, false)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) store_threshold(J);
    if (!last_block_done(&J.rs->done_update_a, gridDim.x)) return;
    finish_a(J, gridDim.x);
}

__global__ void __launch_bounds__(kUpdateThreads) k_update_b(const JobDesc J) {
    if (!update_b_block(J, blockIdx.x, false)) return;
    if (!last_block_done(&J.rs->done_update_b, gridDim.x)) return;
    finish_b(J, gridDim.x);
}

cudaError_t launch_update_a(const JobDesc &J, cudaStream_t st) {
    k_update_a<<<update_grid(J.lay.n), kUpdateThreads, 0, st>>>(J);
    return cudaGetLastError();
}

cudaError_t launch_update_b(const JobDesc &J, cudaStream_t st) {
    k_update_b<<<update_grid(J.lay.n), kUpdateThreads, 0, st>>>(J);
    return cudaGetLastError();
}

// Batched: the blocks of all jobs in the round, flattened (job j owns blocks
// [ublock_base_j, ublock_base_j + update_grid(n_j))), each job's last block
// finishing it.  The same blocks and the same order of partial sums as the
// plain kernels, so a job's results do not depend on its batch.
template <bool A>
__global__ void __launch_bounds__(kUpdateThreads) k_bupdate(const JobDesc *__restrict__ jobs, BatchMeta *meta) {
    __shared__ int base[kMaxBatchJobs + 1];
    const int nj = meta->njobs;
    for (int j = threadIdx.x; j < nj; j += blockDim.x) base[j] = jobs[j].ublock_base;
    if (threadIdx.x == 0) base[nj] = meta->total_ublocks;
    __syncthreads();
    const int total = base[nj];
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (base[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const JobDesc &J = jobs[lo];
        const int blk = g - base[lo], nblocks = base[lo + 1] - base[lo];
        if (A) {
            if (!update_a_block(J, blk, true)) continue;
            if (blk == 0 && threadIdx.x == 0) store_threshold(J);
        } else {
            if (!update_b_block(J, blk, true)) continue;
        }
        if (last_block_done(A ? &J.rs->done_update_a : &J.rs->done_update_b, nblocks)) {
            if (A) finish_a(J, nblocks);
            else finish_b(J, nblocks);
        }
        __syncthreads();
    }
}

cudaError_t launch_bupdate_a(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st) {
    k_bupdate<true><<<grid, kUpdateThreads, 0, st>>>(jobs, meta);
    return cudaGetLastError();
}

cudaError_t launch_bupdate_b(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st) {
    k_bupdate<false><<<grid, kUpdateThreads, 0, st>>>(jobs, meta);
    return cudaGetLastError();
}

}  // namespace vjb
