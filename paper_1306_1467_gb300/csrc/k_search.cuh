// Device pieces shared by the plain search kernels (k_search.cu) and the
// batched ones (k_bsearch.cu): the FP32 scan of a stage of table entries and
// the end of a row, the shortlist threshold, and the double-float re-scan of a
// shortlisted feature with the choice of the round's stump.
#pragma once

#include <limits.h>
#include <math.h>

#include "vjb_device.cuh"
#include "vjb_internal.cuh"

namespace vjb {

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The signed weights (`words` floats, a multiple of 4; a device allocation)
// into shared memory by the whole CTA: 16-byte loads, eight in flight per
// thread.  Scalar loads one after another took 12.7 us per CTA at 15,000
// samples, in every search and at every job switch of a batched one.
__device__ __forceinline__ void stage_weights(float *sv, const float *v, int words) {
    const float4 *__restrict__ v4 = reinterpret_cast<const float4 *>(v);
    float4 *sv4 = reinterpret_cast<float4 *>(sv);
    const int n4 = words >> 2;
#pragma unroll 8
    for (int i = threadIdx.x; i < n4; i += blockDim.x) sv4[i] = __ldg(v4 + i);
}

// Predicated running max/min: update only where `flag` is set (a valid split).
__device__ __forceinline__ void minmax_if(uint32_t flag, float a, float &mx, float &mn) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %2, 0;\n\t"
        "@p max.f32 %0, %0, %3;\n\t"
        "@p min.f32 %1, %1, %3;\n\t}"
        : "+f"(mx), "+f"(mn)
        : "r"(flag), "f"(a));
}

// U pieces of CR chunk rows of a stage (8 entries per lane per chunk row),
// worked on together for instruction-level parallelism.  Lane k reads chunk
// t * 32 + k: its own run, in order, 16 bytes at a time, the 32 lanes covering
// 512 contiguous bytes (no bank conflict).  Each piece is summed in FP32 from
// zero; its largest and smallest prefix at a valid split, offset by the
// lane's compensated running total (ahi + alo), update the lane's best
// (bmx, bmn); then the piece total enters the running total through TwoSum.
template <int U, int CR>
__device__ __forceinline__ void scan_pieces(uint32_t sbase, int t0, int lane, const float *sv,
                                            float &ahi, float &alo, float &bmx, float &bmn) {
    constexpr int E = CR * kChunkElems;
    uint32_t wd[U][CR * 4];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < CR; ++c) {
            const uint4 q = lds128(sbase + (uint32_t)(((t0 + u * CR + c) * 32 + lane) * 16));
            wd[u][4 * c + 0] = q.x;
            wd[u][4 * c + 1] = q.y;
            wd[u][4 * c + 2] = q.z;
            wd[u][4 * c + 3] = q.w;
        }
    float g[U][E];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < E / 2; ++j) {
            g[u][2 * j] = sv[wd[u][j] & kIndexMask];  // even position: word | flag << 15
            g[u][2 * j + 1] = sv[wd[u][j] >> 17];      // odd position: (word << 1 | flag) << 16
        }
    float a[U], mx[U], mn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        a[u] = 0.f;
        mx[u] = -INFINITY;
        mn[u] = INFINITY;
    }
#pragma unroll
    for (int j = 0; j < E; ++j)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] += g[u][j];
            const uint32_t fl = (j & 1) ? (wd[u][j >> 1] & 0x10000u) : (wd[u][j >> 1] & 0x8000u);
            minmax_if(fl, a[u], mx[u], mn[u]);
        }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        bmx = fmaxf(bmx, ahi + (alo + mx[u]));
        bmn = fminf(bmn, ahi + (alo + mn[u]));
        float sum, err;
        two_sum(ahi, a[u], sum, err);
        ahi = sum;
        alo += err;
    }
}

// ---- shared pieces of the search kernels -----------------------------------------------

// All chunk rows of one stage, 2U chunk rows (16U entries per lane) at a
// time: U pieces of 16 entries, or with U = 3 two pieces of 24 (fewer piece
// ends to fold in; 24 terms keep the screening bound of k_search.cu).  A full
// stage of 2U chunk rows -- all but a row's last stage -- takes a path of its
// own with no loop around it (3.4% of the search time at 24x24 / 15k).
template <int U>
__device__ __forceinline__ void scan_stage(uint32_t sbase, int crs, int lane, const float *sv,
                                           float &ahi, float &alo, float &bmx, float &bmn) {
    if (crs == 2 * U) {
        if constexpr (U == 3) scan_pieces<2, 3>(sbase, 0, lane, sv, ahi, alo, bmx, bmn);
        else scan_pieces<U, 2>(sbase, 0, lane, sv, ahi, alo, bmx, bmn);
        return;
    }
    int t = 0;
    if constexpr (U == 3) {
        for (; t + 6 <= crs; t += 6) scan_pieces<2, 3>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
    } else {
        for (; t + 2 * U <= crs; t += 2 * U) scan_pieces<U, 2>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
    }
    // what is left of a row's last stage: two 16-entry pieces at a time, then
    // one piece of 24, 16 or 8 (0.7589 -> 0.7554 ms at 24x24 / 15k, +1% at
    // 4,000 samples, against single pieces of 16)
    for (; t + 4 <= crs; t += 4) scan_pieces<2, 2>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
    if (t + 3 <= crs) {
        scan_pieces<1, 3>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
        t += 3;
    } else if (t + 2 <= crs) {
        scan_pieces<1, 2>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
        t += 2;
    }
    if (t < crs) scan_pieces<1, 1>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
}

// End of a row: the runs of the lanes below come first, so an exclusive
// scan of the run totals offsets each lane's best prefixes; the feature's
// error is min(T+ - max D, T- + min D), split 0 (D = 0) included.  The scan is
// plain FP32 over the run totals rounded once (it adds at most 6u of the
// weight total to the screening bound of k_search.cu; a double-float scan
// here cost about 2% of the search at 15,000 samples and 13% at 2,500).
//
// The row's error is min over lanes of min(Tp - x_l, Tm + y_l), x_l and y_l the
// lane's best prefixes placed on its offset, and of Tp and Tm (split 0): the
// same floats as Tp - max x_l and Tm + min y_l, since a min does not round.
// So each lane forms its own candidate and one integer min reduction
// (redux.sync on an order-preserving key of the float) ends the row: a
// shorter chain at every row end than a max and a min of five shuffles each.
__device__ __forceinline__ int32_t float_order_key(float f) {
    const int32_t b = __float_as_int(f);
    return b ^ ((b >> 31) & 0x7fffffff);  // negative floats: reverse their magnitude order
}
__device__ __forceinline__ float float_from_order_key(int32_t k) {
    return __int_as_float(k ^ ((k >> 31) & 0x7fffffff));
}

__device__ __forceinline__ float finish_row(float ahi, float alo, float bmx, float bmn, float Tp,
                                            float Tm, int lane) {
    float x = ahi + alo;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    float excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) excl = 0.f;
    const float e = fminf(fminf(Tp - (excl + bmx), Tm + (excl + bmn)), fminf(Tp, Tm));
    return float_from_order_key(__reduce_min_sync(0xffffffffu, float_order_key(e)));
}

// The screened error within which a feature must lie of the smallest one
// (twice the screening bound, in units of the weight total).
__device__ __forceinline__ float shortlist_threshold(float m, const RoundState *rs) {
    return m + kScreenMarginUlps * 5.9604644775390625e-8f * (float)(rs->t_pos + rs->t_neg);
}

// ---- compensated re-scan of shortlisted features --------------------------------------

__device__ __forceinline__ bool df_eq(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }

// Lexicographic candidate order: error (double-float), feature, split, +1 first.
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

constexpr int kRescanWarps = 32;  // one warp per lane run of the row (select_stump relies on 32)

struct RunResult {
    DF total, mx, mn;
    int smx, smn;
};

// One warp scans lane run k of a row in double-float: 32 chunks of 8 entries
// at a time, lane i holding chunk u0 + i of the run.  Returns (in every lane)
// the run total and its largest / smallest prefix at a valid split, relative
// to the run start, with the split position (number of entries before it in
// the whole value order) and the lowest position on ties (INT_MAX if none).
static __device__ RunResult rescan_run(const uint16_t *__restrict__ row, int run, int k,
                                const float *__restrict__ v, int lane) {
    DF carry{0.f, 0.f}, bmax{-INFINITY, 0.f}, bmn{INFINITY, 0.f};
    int smax = INT_MAX, smn = INT_MAX;
    const int nch = run / kChunkElems;
    auto load_chunk = [&](int t) {
        return t < nch ? __ldg(reinterpret_cast<const uint4 *>(row + (size_t)(t * 32 + k) * kChunkElems))
                       : make_uint4(0u, 0u, 0u, 0u);
    };
    uint4 qn = load_chunk(lane);  // the next 32 chunks load while these are scanned
    for (int u0 = 0; u0 < nch; u0 += 32) {
        const int t = u0 + lane;
        const uint4 q = qn;
        if (u0 + 32 < nch) qn = load_chunk(t + 32);
        const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
        const bool have = t < nch;
        DF a{0.f, 0.f}, lmx{-INFINITY, 0.f}, lmn{INFINITY, 0.f};
        int lsx = INT_MAX, lsn = INT_MAX;
        if (have) {
#pragma unroll
            for (int j = 0; j < kChunkElems; ++j) {
                const uint32_t e = (j & 1) ? (wd[j >> 1] >> 16) : (wd[j >> 1] & 0xffffu);
                a = df_add_f(a, __ldg(v + entry_word(e, j)));
                if (entry_flag(e, j)) {
                    const int pos = k * run + t * kChunkElems + j + 1;
                    if (df_less(lmx, a)) { lmx = a; lsx = pos; }
                    if (df_less(a, lmn)) { lmn = a; lsn = pos; }
                }
            }
        }
        DF x = a;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const DF y = df_shfl_up(x, d);
            if (lane >= d) x = df_add(y, x);
        }
        DF excl = df_shfl_up(x, 1);
        if (lane == 0) excl = DF{0.f, 0.f};
        const DF tot = df_shfl(x, 31);
        const DF offs = df_add(carry, excl);
        if (lsx != INT_MAX) {
            const DF c = df_add(offs, lmx);
            if (df_less(bmax, c)) { bmax = c; smax = lsx; }
        }
        if (lsn != INT_MAX) {
            const DF c = df_add(offs, lmn);
            if (df_less(c, bmn)) { bmn = c; smn = lsn; }
        }
        carry = df_add(carry, tot);
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        const DF om = df_shfl_xor(bmax, d);
        const int os = __shfl_xor_sync(0xffffffffu, smax, d);
        if (df_less(bmax, om) || (df_eq(om, bmax) && os < smax)) { bmax = om; smax = os; }
        const DF on = df_shfl_xor(bmn, d);
        const int on_s = __shfl_xor_sync(0xffffffffu, smn, d);
        if (df_less(on, bmn) || (df_eq(on, bmn) && on_s < smn)) { bmn = on; smn = on_s; }
    }
    RunResult r;
    r.total = carry;
    r.mx = bmax;
    r.mn = bmn;
    r.smx = smax;
    r.smn = smn;
    return r;
}

// One warp combines a row's 32 lane runs (lane k holds run k's result q):
// runs in value order, an exclusive double-float scan of their totals places
// each run's extremes in the row; then the largest and the smallest prefix
// over the row (lowest split on ties), split 0 (D = 0) included, give the
// feature's best error, split and polarity.  The result is valid in lane 0.
__device__ __forceinline__ Candidate combine_runs(const JobDesc &J, int32_t f, const RunResult &q, int lane) {
    Candidate cd;
    cd.err_hi = INFINITY; cd.err_lo = 0.f; cd.feature = f; cd.split = 0; cd.polarity = 1; cd.pad = 0;
    DF x = q.total;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const DF y = df_shfl_up(x, d);
        if (lane >= d) x = df_add(y, x);
    }
    DF offs = df_shfl_up(x, 1);
    if (lane == 0) offs = DF{0.f, 0.f};
    DF bmax = q.smx != INT_MAX ? df_add(offs, q.mx) : DF{-INFINITY, 0.f};
    DF bmn = q.smn != INT_MAX ? df_add(offs, q.mn) : DF{INFINITY, 0.f};
    int smax = q.smx, smn = q.smn;
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        const DF om = df_shfl_xor(bmax, d);
        const int os = __shfl_xor_sync(0xffffffffu, smax, d);
        if (df_less(bmax, om) || (df_eq(om, bmax) && os < smax)) { bmax = om; smax = os; }
        const DF on = df_shfl_xor(bmn, d);
        const int on_s = __shfl_xor_sync(0xffffffffu, smn, d);
        if (df_less(on, bmn) || (df_eq(on, bmn) && on_s < smn)) { bmn = on; smn = on_s; }
    }
    if (!df_less(DF{0.f, 0.f}, bmax)) { bmax = DF{0.f, 0.f}; smax = 0; }
    if (!df_less(bmn, DF{0.f, 0.f})) { bmn = DF{0.f, 0.f}; smn = 0; }
    if (lane == 0) {
        const DF Tp = df_from_double(J.rs->t_pos), Tm = df_from_double(J.rs->t_neg);
        const DF ep = df_add(Tp, df_neg(bmax));
        const DF em = df_add(Tm, bmn);
        const bool minus = df_less(em, ep) || (df_eq(em, ep) && smn < smax);
        cd.err_hi = minus ? em.hi : ep.hi;
        cd.err_lo = minus ? em.lo : ep.lo;
        cd.split = minus ? smn : smax;
        cd.polarity = minus ? -1 : 1;
    }
    return cd;
}

// The whole CTA re-scans feature f of job J, its warps taking the row's 32
// lane runs in turn; thread 0 returns its best (error, split, polarity).
// `rres` is 32 slots of shared memory.
static __device__ Candidate rescan_feature(const JobDesc &J, int32_t f, RunResult *rres) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int run = J.npad / 32;
    const uint16_t *row = J.rows + (size_t)f * J.npad;
    for (int k = warp; k < 32; k += nw) {
        const RunResult r = rescan_run(row, run, k, J.v, lane);
        if (lane == 0) rres[k] = r;
    }
    __syncthreads();
    Candidate cd;
    cd.err_hi = INFINITY; cd.err_lo = 0.f; cd.feature = f; cd.split = 0; cd.polarity = 1; cd.pad = 0;
    if (warp == 0) cd = combine_runs(J, f, rres[lane], lane);
    __syncthreads();
    return cd;
}

// The round's stump from the best of `cnt` re-scanned candidates, `b` (one
// thread); no candidate stops the job with an error flag.
__device__ __forceinline__ void record_stump(const JobDesc &J, int cnt, const Candidate &b) {
    RoundState *rs = J.rs;
    if (cnt == 0 || b.feature == INT_MAX) {
        rs->flags |= kFlagNoCandidate;
        rs->status = VJB_EDEVICE;
    } else {
        rs->win_feature = b.feature;
        rs->win_split = b.split;
        rs->win_polarity = b.polarity;
        rs->win_err_hi = b.err_hi;
        rs->win_err_lo = b.err_lo;
    }
    rs->done_rescan = 0u;
}

__device__ __forceinline__ Candidate load_candidate(const Candidate *p) {
    Candidate c;
    const volatile Candidate *vc = p;
    c.err_hi = vc->err_hi; c.err_lo = vc->err_lo; c.feature = vc->feature;
    c.split = vc->split; c.polarity = vc->polarity; c.pad = 0;
    return c;
}

// One warp picks job J's stump among its `cnt` re-scanned candidates.
__device__ __forceinline__ void select_stump_warp(const JobDesc &J, int cnt, int lane) {
    Candidate b;
    b.err_hi = INFINITY; b.err_lo = 0.f; b.feature = INT_MAX; b.split = INT_MAX; b.polarity = 1; b.pad = 0;
    for (int k = lane; k < cnt; k += 32) {
        const Candidate c = load_candidate(J.cands + k);
        if (cand_less(c, b)) b = c;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        const Candidate o = cand_shfl_xor(b, d);
        if (cand_less(o, b)) b = o;
    }
    if (lane == 0) record_stump(J, cnt, b);
}

// The whole CTA picks job J's stump among its `cnt` re-scanned candidates.
static __device__ void select_stump(const JobDesc &J, int cnt) {
    __shared__ Candidate wc[kRescanWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    Candidate b;
    b.err_hi = INFINITY; b.err_lo = 0.f; b.feature = INT_MAX; b.split = INT_MAX; b.polarity = 1; b.pad = 0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const Candidate c = load_candidate(J.cands + k);
        if (cand_less(c, b)) b = c;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        const Candidate o = cand_shfl_xor(b, d);
        if (cand_less(o, b)) b = o;
    }
    if (lane == 0) wc[warp] = b;
    __syncthreads();
    if (warp == 0) {
        if (lane < nw) b = wc[lane];
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            const Candidate o = cand_shfl_xor(b, d);
            if (cand_less(o, b)) b = o;
        }
    }
    if (threadIdx.x == 0) record_stump(J, cnt, b);
    __syncthreads();
}

}  // namespace vjb
