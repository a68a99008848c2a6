// Per-round search for the least-error decision stump over every Haar feature
// (Sec. 2.3 step 2: eps_t = min over f, p, theta of sum_i w_i |h(x_i) - y_i|).
//
// For one feature, let the samples be taken in value order (the sorted table)
// and let D(s) = sum over the first s samples of v_i, v_i = +w_i for a face and
// -w_i for a non-face.  With T+ and T- the face and non-face weight totals, the
// stump that puts the first s samples "below" the threshold errs by
//     T+ - D(s)   for p = +1 (below is a face),
//     T- + D(s)   for p = -1 (above is a face),
// and only splits between two different values are thresholds (bit 15 of the
// entry before the split; s = 0 is always one).  So the feature's least error
// is min(T+ - max D, T- + min D) over valid splits.
//
// Three kernels per search:
//  * k_screen (the hot kernel): streams the whole uint16 table once per round
//    with TMA, gathers v from shared memory, and forms D with FP32 prefix sums.
//    A warp scans one row: lane k walks its own run of the value order (the
//    row layout interleaves 32 runs), summing 16 entries at a time in FP32 and
//    folding each piece into a compensated (TwoSum) running total; one
//    double-float warp scan of the 32 run totals per row places every lane's
//    best prefix in the row.  It writes each feature's FP32 error and each
//    CTA's minimum.
//  * k_shortlist: lists every feature whose screened error is within a margin
//    of the smallest one.
//  * k_rescan: one CTA per listed feature scans its row again in double-float
//    (compensated FP32) arithmetic throughout, giving the feature's best split,
//    polarity and an error to about 1e-14 relative; the last CTA to finish
//    picks the round's stump: lowest error, then feature, split, +1 before -1.
//
// Screening error bound (u = 2^-24, sum |v| = T+ + T- = 1 after normalising):
// a piece's partial sums of at most 16 terms err by at most 16u times the
// piece's |v| mass; the compensated run total and the double-float scan of run
// totals add O(u^2); placing the piece's extreme on the run total, and that on
// the run offset, adds 4u |D|; forming T+- -/+ D in FP32 adds 2u.  So
// |screened - exact| <= 22u.  A margin of 64u (twice 32u) keeps every
// feature that could beat the best one.
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "vjb_device.cuh"
#include "vjb_internal.cuh"

namespace vjb {

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Dynamic shared memory of k_screen: the weight array at the base, then (from
// the next 1 KiB boundary) the per-warp TMA rings, their mbarriers and the
// per-warp minima.
size_t search_smem_bytes(const SearchShape &s, int words) {
    size_t b = align_up((size_t)words * 4, 16);
    b += 1024;  // alignment of the rings to 1 KiB
    b += (size_t)s.warps * s.stages * s.box_lines * kLineBytes;
    b += (size_t)s.warps * s.stages * 8;
    b += (size_t)s.warps * 4 + 16;
    return b;
}

WeightLayout make_layout(int n, bool allow_dual) {
    WeightLayout L;
    L.n = n;
    const int off_b = (int)align_up((size_t)n + 1, 32);
    // table entries hold 15-bit word offsets: copy B takes what is left of the
    // 32,768 words after copy A, whole 32-sample blocks (all n while n <= 16,351)
    const int room = off_b < 32768 ? (32768 - off_b) / 32 * 32 : 0;
    L.nb = allow_dual ? (n < room ? n : room) : 0;
    L.dual = L.nb > 0 ? 1 : 0;
    L.off_b = L.dual ? off_b : 0;
    L.words = L.dual ? off_b + (int)align_up((size_t)L.nb, 32) : (int)align_up((size_t)n + 1, 4);
    return L;
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

// All chunk rows of one stage.
template <int U>
__device__ __forceinline__ void scan_stage(uint32_t sbase, int crs, int lane, const float *sv,
                                           float &ahi, float &alo, float &bmx, float &bmn) {
    int t = 0;
    for (; t + 2 * U <= crs; t += 2 * U) scan_pieces<U, 2>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
    for (; t + 2 <= crs; t += 2) scan_pieces<1, 2>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
    if (t < crs) scan_pieces<1, 1>(sbase, t, lane, sv, ahi, alo, bmx, bmn);
}

// End of a row: the runs of the lanes below come first, so an exclusive
// double-float scan of the run totals offsets each lane's best prefixes; the
// feature's error is min(T+ - max D, T- + min D), split 0 (D = 0) included.
__device__ __forceinline__ float finish_row(float ahi, float alo, float bmx, float bmn, float Tp,
                                            float Tm, int lane) {
    DF x{ahi, alo};
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const DF y = df_shfl_up(x, d);
        if (lane >= d) x = df_add(y, x);
    }
    DF excl = df_shfl_up(x, 1);
    if (lane == 0) excl = DF{0.f, 0.f};
    float MX = warp_max(excl.hi + (excl.lo + bmx));
    float MN = warp_min(excl.hi + (excl.lo + bmn));
    MX = fmaxf(MX, 0.f);
    MN = fminf(MN, 0.f);
    return fminf(Tp - MX, Tm + MN);
}

template <int U>
__global__ void __launch_bounds__(U >= 4 ? 384 : (U == 3 ? 512 : 640), 1)
    k_screen(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ v, int words,
             int lines_per_row, int box_lines, int stage_lines, int64_t nfeat,
             int stages, RoundState *rs, float *__restrict__ ferr, float *__restrict__ bmin) {
    if (rs->status != VJB_OK) return;
    extern __shared__ __align__(16) float sv[];  // weights at the base of dynamic shared memory
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sv32 = smem_u32(sv);
    const uint32_t stage_bytes = (uint32_t)stage_lines * kLineBytes;  // a multiple of 1 KiB
    const uint32_t ring0 = (uint32_t)align_up(sv32 + (uint32_t)words * 4u, 1024);
    const uint32_t bars0 = ring0 + (uint32_t)nw * stages * stage_bytes;
    float *wbest = reinterpret_cast<float *>(reinterpret_cast<char *>(sv) + (bars0 + nw * stages * 8 - sv32));

    for (int i = threadIdx.x; i < words; i += blockDim.x) sv[i] = v[i];
    const uint32_t ring_w = ring0 + (uint32_t)warp * stages * stage_bytes;
    const uint32_t bar_w = bars0 + (uint32_t)(warp * stages * 8);
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(bar_w + 8 * s, 1);
        fence_barrier_init();
    }
    __syncthreads();

    const int64_t gw = (int64_t)blockIdx.x * nw + warp;
    const int64_t G = (int64_t)gridDim.x * nw;
    const int64_t nf_w = gw < nfeat ? (nfeat - 1 - gw) / G + 1 : 0;
    const int nc = (lines_per_row + box_lines - 1) / box_lines;
    const int64_t total = nf_w * nc;
    const uint32_t tx = (uint32_t)box_lines * kLineBytes;

    // producer state (lane 0): the next chunk to load, in this warp's order
    int64_t pk = 0, issued = 0;
    int pc = 0, pstage = 0;
    auto issue_next = [&]() {
        if (issued >= total) return;
        const uint32_t bar = bar_w + 8u * (uint32_t)pstage;
        mbar_arrive_expect_tx(bar, tx);
        tma_load_3d(ring_w + (uint32_t)pstage * stage_bytes, &tmap, 0, pc * box_lines,
                    (int32_t)(gw + pk * G), bar);
        if (++pc == nc) { pc = 0; ++pk; }
        if (++pstage == stages) pstage = 0;
        ++issued;
    };
    if (lane == 0)
        for (int s = 0; s < stages; ++s) issue_next();
    __syncwarp();

    const float Tp = (float)rs->t_pos, Tm = (float)rs->t_neg;
    float best = INFINITY;
    int cstage = 0;
    uint32_t cpar = 0;  // consumer ring position and mbarrier phase
    int64_t consumed = 0;
    bool ok = true;
    for (int64_t k = 0; k < nf_w && ok; ++k) {
        const int64_t f = gw + k * G;
        float ahi = 0.f, alo = 0.f, bmx = -INFINITY, bmn = INFINITY;
        for (int c = 0; c < nc; ++c) {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar))) {
                ok = false;
                break;
            }
            const int lines_here = min(box_lines, lines_per_row - c * box_lines);
            const int crs = lines_here >> 2;  // chunk rows (a line is a quarter of one)
            const uint32_t sbase = ring_w + (uint32_t)cstage * stage_bytes;
            scan_stage<U>(sbase, crs, lane, sv, ahi, alo, bmx, bmn);
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async_smem();
                issue_next();
            }
            if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
            ++consumed;
        }
        if (!ok) break;
        const float e = finish_row(ahi, alo, bmx, bmn, Tp, Tm, lane);
        if (lane == 0) {
            ferr[f] = e;
            best = fminf(best, e);
        }
    }
    if (!ok) {
        // stop: record the failure and wait (bounded) for this warp's copies in flight
        if (lane == 0) {
            atomicOr(&rs->flags, kFlagWaitTimeout);
            // chunks issued but not consumed sit in the ring from the current stage on
            int st = cstage;
            uint32_t ph = cpar;
            const int64_t pending = issued - consumed;
            for (int64_t s = 0; s < pending; ++s) {
                mbar_wait_bounded(bar_w + 8u * (uint32_t)st, ph, 100000000ull);
                if (++st == stages) { st = 0; ph ^= 1u; }
            }
        }
        __syncwarp();
    }
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = INFINITY;
        for (int w = 0; w < nw; ++w) m = fminf(m, wbest[w]);
        bmin[blockIdx.x] = m;
    }
}

cudaError_t launch_screen(const CUtensorMap *tmap, const float *v, const WeightLayout &L,
                          int lines_per_row, int box_lines, int64_t nfeat, const SearchShape &shape,
                          int grid, RoundState *rs, float *ferr, float *bmin, cudaStream_t st) {
    const size_t sm = search_smem_bytes(shape, L.words);
    const int threads = shape.warps * 32;
    switch (shape.unroll) {
    case 1:
        k_screen<1><<<grid, threads, sm, st>>>(*tmap, v, L.words, lines_per_row, box_lines,
                                               shape.box_lines, nfeat, shape.stages, rs, ferr, bmin);
        break;
    case 4:
        k_screen<4><<<grid, threads, sm, st>>>(*tmap, v, L.words, lines_per_row, box_lines,
                                               shape.box_lines, nfeat, shape.stages, rs, ferr, bmin);
        break;
    case 3:
        k_screen<3><<<grid, threads, sm, st>>>(*tmap, v, L.words, lines_per_row, box_lines,
                                               shape.box_lines, nfeat, shape.stages, rs, ferr, bmin);
        break;
    default:
        k_screen<2><<<grid, threads, sm, st>>>(*tmap, v, L.words, lines_per_row, box_lines,
                                               shape.box_lines, nfeat, shape.stages, rs, ferr, bmin);
    }
    return cudaGetLastError();
}

cudaError_t set_screen_smem_limit(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_screen<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_screen<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_screen<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_screen<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

int screen_max_warps(int unroll) { return unroll >= 4 ? 12 : (unroll == 3 ? 16 : 20); }

int screen_occupancy(const SearchShape &s, int words) {
    int blocks = 0;
    cudaError_t e;
    const size_t sm = search_smem_bytes(s, words);
    if (s.unroll == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_screen<1>, s.warps * 32, sm);
    else if (s.unroll == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_screen<4>, s.warps * 32, sm);
    else if (s.unroll == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_screen<3>, s.warps * 32, sm);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_screen<2>, s.warps * 32, sm);
    return e == cudaSuccess ? blocks : 0;
}

// ---- shortlist ------------------------------------------------------------------------

// The screened error within which a feature must lie of the smallest one
// (twice the screening bound, in units of the weight total).
__device__ __forceinline__ float shortlist_threshold(float m, const RoundState *rs) {
    return m + kScreenMarginUlps * 5.9604644775390625e-8f * (float)(rs->t_pos + rs->t_neg);
}

__global__ void __launch_bounds__(256)
    k_shortlist(const JobDesc J, const float *__restrict__ bmin, int nbmin) {
    RoundState *rs = J.rs;
    if (rs->status != VJB_OK || rs->forced) return;
    __shared__ float red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float m = INFINITY;
    for (int i = threadIdx.x; i < nbmin; i += blockDim.x) m = fminf(m, bmin[i]);
    m = warp_min(m);
    if (lane == 0) red[warp] = m;
    __syncthreads();
    m = INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fminf(m, red[w]);
    const float thr = shortlist_threshold(m, rs);
    if (blockIdx.x == 0 && threadIdx.x == 0) rs->screen_min = m;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < J.nfeat; base += stride) {
        const int64_t f = base + lane;
        const bool take = f < J.nfeat && J.ferr[f] <= thr;
        const uint32_t mask = __ballot_sync(0xffffffffu, take);
        if (!mask) continue;
        int slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(&rs->cand_count, __popc(mask));
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        if (take) J.cand_ids[slot0 + __popc(mask & ((1u << lane) - 1u))] = (int32_t)f;
    }
}

cudaError_t launch_shortlist(const JobDesc &J, const float *bmin, int nbmin, int grid, cudaStream_t st) {
    k_shortlist<<<grid, 256, 0, st>>>(J, bmin, nbmin);
    return cudaGetLastError();
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

constexpr int kRescanWarps = 32;  // one warp per lane run of the row

struct RunResult {
    DF total, mx, mn;
    int smx, smn;
};

// One warp scans lane run k of a row in double-float: 32 chunks of 8 entries
// at a time, lane i holding chunk u0 + i of the run.  Returns (in every lane)
// the run total and its largest / smallest prefix at a valid split, relative
// to the run start, with the split position (number of entries before it in
// the whole value order) and the lowest position on ties (INT_MAX if none).
__device__ RunResult rescan_run(const uint16_t *__restrict__ row, int run, int k,
                                const float *__restrict__ v, int lane) {
    DF carry{0.f, 0.f}, bmax{-INFINITY, 0.f}, bmn{INFINITY, 0.f};
    int smax = INT_MAX, smn = INT_MAX;
    const int nch = run / kChunkElems;
    for (int u0 = 0; u0 < nch; u0 += 32) {
        const int t = u0 + lane;
        uint32_t wd[4] = {0u, 0u, 0u, 0u};
        const bool have = t < nch;
        if (have) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(row + (size_t)(t * 32 + k) * kChunkElems));
            wd[0] = q.x; wd[1] = q.y; wd[2] = q.z; wd[3] = q.w;
        }
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

// The whole CTA (kRescanWarps warps) re-scans feature f of job J; thread 0
// returns its best (error, split, polarity).  `rres` is 32 slots of shared memory.
__device__ Candidate rescan_feature(const JobDesc &J, int32_t f, RunResult *rres) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int run = J.npad / 32;
    const uint16_t *row = J.rows + (size_t)f * J.npad;
    for (int k = warp; k < 32; k += kRescanWarps) {
        const RunResult r = rescan_run(row, run, k, J.v, lane);
        if (lane == 0) rres[k] = r;
    }
    __syncthreads();
    Candidate cd;
    cd.err_hi = INFINITY; cd.err_lo = 0.f; cd.feature = f; cd.split = 0; cd.polarity = 1; cd.pad = 0;
    if (threadIdx.x == 0) {
        const DF Tp = df_from_double(J.rs->t_pos), Tm = df_from_double(J.rs->t_neg);
        DF offs{0.f, 0.f}, bmax{0.f, 0.f}, bmn{0.f, 0.f};  // split 0: D = 0
        int smax = 0, smn = 0;
        for (int k = 0; k < 32; ++k) {  // runs in value order
            const RunResult &q = rres[k];
            if (q.smx != INT_MAX) {
                const DF cc = df_add(offs, q.mx);
                if (df_less(bmax, cc)) { bmax = cc; smax = q.smx; }
            }
            if (q.smn != INT_MAX) {
                const DF cc = df_add(offs, q.mn);
                if (df_less(cc, bmn)) { bmn = cc; smn = q.smn; }
            }
            offs = df_add(offs, q.total);
        }
        const DF ep = df_add(Tp, df_neg(bmax));
        const DF em = df_add(Tm, bmn);
        const bool minus = df_less(em, ep) || (df_eq(em, ep) && smn < smax);
        cd.err_hi = minus ? em.hi : ep.hi;
        cd.err_lo = minus ? em.lo : ep.lo;
        cd.split = minus ? smn : smax;
        cd.polarity = minus ? -1 : 1;
    }
    __syncthreads();
    return cd;
}

// The whole CTA picks job J's stump among its `cnt` re-scanned candidates.
__device__ void select_stump(const JobDesc &J, int cnt) {
    __shared__ Candidate wc[kRescanWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Candidate b;
    b.err_hi = INFINITY; b.err_lo = 0.f; b.feature = INT_MAX; b.split = INT_MAX; b.polarity = 1; b.pad = 0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        Candidate c;
        const volatile Candidate *vc = J.cands + k;
        c.err_hi = vc->err_hi; c.err_lo = vc->err_lo; c.feature = vc->feature;
        c.split = vc->split; c.polarity = vc->polarity; c.pad = 0;
        if (cand_less(c, b)) b = c;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        const Candidate o = cand_shfl_xor(b, d);
        if (cand_less(o, b)) b = o;
    }
    if (lane == 0) wc[warp] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kRescanWarps; ++w)
            if (cand_less(wc[w], b)) b = wc[w];
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
    __syncthreads();
}

__global__ void __launch_bounds__(kRescanWarps * 32) k_rescan(const JobDesc J) {
    if (J.rs->status != VJB_OK || J.rs->forced) return;
    __shared__ RunResult rres[32];
    __shared__ bool last_cta;
    const int cnt = J.rs->cand_count;
    for (int c = blockIdx.x; c < cnt; c += gridDim.x) {
        const Candidate cd = rescan_feature(J, J.cand_ids[c], rres);
        if (threadIdx.x == 0) J.cands[c] = cd;
    }
    // the last CTA to finish picks the round's stump
    if (threadIdx.x == 0) {
        __threadfence();
        last_cta = atomicAdd(&J.rs->done_rescan, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_cta) return;
    __threadfence();
    select_stump(J, cnt);
}

cudaError_t launch_rescan(const JobDesc &J, int grid, cudaStream_t st) {
    k_rescan<<<grid, kRescanWarps * 32, 0, st>>>(J);
    return cudaGetLastError();
}

// ---- batched rounds --------------------------------------------------------------------
// A batch trains many jobs at once: one launch of each round kernel covers all
// of them.  The job table and the counters live in device memory, so a round
// replays as one CUDA graph however the set of jobs changes between rounds.

// Index of the job whose range [base_j, base_{j+1}) holds g (bases ascending).
template <class F>
__device__ __forceinline__ int find_job(int nj, int64_t g, F base) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Which jobs take part in this round; per-job search minimum reset; the
// partitioned search's row ranges.
__global__ void k_bbegin(JobDesc *jobs, BatchMeta *meta) {
    __shared__ int64_t cum[kMaxBatchJobs + 1];  // table lines (+1 per row) before each job
    __shared__ int32_t rw[kMaxBatchJobs];       // lines + 1 of a row of each job taking part
    const int nj = meta->njobs;
    for (int j = threadIdx.x; j < nj; j += blockDim.x) {
        RoundState *rs = jobs[j].rs;
        const int in = jobs[j].active && rs->status == VJB_OK && rs->forced == 0 &&
                       rs->rounds < jobs[j].round_target;
        rs->in_round = in;
        rs->screen_min_bits = 0x7f800000u;  // +inf
        rw[j] = in ? jobs[j].lines + 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int j = 0; j < nj; ++j) {
            cum[j] = acc;
            acc += (int64_t)rw[j] * jobs[j].nfeat;
        }
        cum[nj] = acc;
    }
    __syncthreads();
    // CTA c starts at the row where the running count of lines reaches c / G
    // of the whole; jobs that do not take part weigh nothing
    const int G = meta->screen_ctas;
    const int64_t W = cum[nj];
    for (int c = threadIdx.x; c <= G; c += blockDim.x) {
        int64_t g = meta->total_feat;
        const int64_t target = W * c / G;
        if (c < G && target < W) {
            int lo = 0, hi = nj - 1;  // last job whose start is at or before the target
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cum[mid] <= target) lo = mid;
                else hi = mid - 1;
            }
            g = jobs[lo].feat_base + (target - cum[lo]) / rw[lo];
        }
        meta->cta_start[c] = g;
    }
}

cudaError_t launch_bbegin(JobDesc *jobs, BatchMeta *meta, cudaStream_t st) {
    k_bbegin<<<1, 256, 0, st>>>(jobs, meta);
    return cudaGetLastError();
}

size_t bscreen_smem_bytes(const SearchShape &s, int max_words) {
    return search_smem_bytes(s, max_words);  // stages of s.box_lines lines
}

// One stage of the batched search: `lh` lines (a multiple of 4, at most the
// stage height S) at arena line `line`, with one copy from the map whose box
// is exactly that height, completing on `bar`.
__device__ __forceinline__ void tma_stage(const BatchMaps &maps, uint32_t dst, int32_t line, int lh, int S,
                                          uint32_t bar) {
    mbar_arrive_expect_tx(bar, (uint32_t)lh * kLineBytes);
    const CUtensorMap *m = &maps.m[lh == S ? 0 : (lh >> 2)];
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(0), "r"(line), "r"(bar)
        : "memory");
}

template <int U>
__global__ void __launch_bounds__(U >= 4 ? 384 : (U == 3 ? 512 : 640), 1)
    k_bscreen(const __grid_constant__ BatchMaps maps, const JobDesc *__restrict__ jobs,
              const WorkItem *__restrict__ items, BatchMeta *meta, int max_words, int stages, int stage_lines) {
    extern __shared__ __align__(16) float sv[];
    __shared__ int s_item;
    __shared__ float s_min[32];
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t stage_bytes = (uint32_t)stage_lines * kLineBytes;
    const uint32_t sv32 = smem_u32(sv);
    const uint32_t ring0 = (uint32_t)align_up(sv32 + (uint32_t)max_words * 4u, 1024);
    const uint32_t bars0 = ring0 + (uint32_t)nw * stages * stage_bytes;
    const uint32_t ring_w = ring0 + (uint32_t)warp * stages * stage_bytes;
    const uint32_t bar_w = bars0 + (uint32_t)(warp * stages * 8);
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(bar_w + 8 * s, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int n_items = meta->n_items;
    int cur_job = -1;
    int pstage = 0, cstage = 0;
    uint32_t cpar = 0;
    bool ok = true;  // false once one of this warp's waits timed out
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&meta->item_next, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const WorkItem W = items[it];
        const JobDesc &J = jobs[W.job];
        if (!J.rs->in_round) continue;
        if (W.job != cur_job) {  // this job's weights into shared memory
            for (int i = threadIdx.x; i < J.lay.words; i += blockDim.x) sv[i] = J.v[i];
            __syncthreads();
            cur_job = W.job;
        }
        const int lines = J.lines;
        const int nc = (lines + stage_lines - 1) / stage_lines;
        const int nrows = W.f1 - W.f0 > warp ? (W.f1 - W.f0 - warp + nw - 1) / nw : 0;
        const int total = ok ? nrows * nc : 0;
        const float Tp = (float)J.rs->t_pos, Tm = (float)J.rs->t_neg;
        // producer (lane 0): the arena line of the next stage and the lines left in its row
        int issued = 0, p_left = lines;
        int64_t p_row = J.line_base + (W.f0 + warp) * (int64_t)lines, p_cur = p_row;
        const int64_t p_step = (int64_t)nw * lines;
        auto issue_next = [&]() {
            if (issued >= total) return;
            const int lh = min(stage_lines, p_left);
            tma_stage(maps, ring_w + (uint32_t)pstage * stage_bytes, (int32_t)p_cur, lh, stage_lines,
                      bar_w + 8u * (uint32_t)pstage);
            p_cur += lh;
            if ((p_left -= lh) == 0) {
                p_row += p_step;
                p_cur = p_row;
                p_left = lines;
            }
            if (++pstage == stages) pstage = 0;
            ++issued;
        };
        if (lane == 0)
            for (int s = 0; s < stages; ++s) issue_next();
        __syncwarp();
        float wmin = INFINITY;
        int consumed = 0;
        for (int k = 0; k < nrows && ok; ++k) {
            const int64_t f = W.f0 + warp + (int64_t)k * nw;
            float ahi = 0.f, alo = 0.f, bmx = -INFINITY, bmn = INFINITY;
            for (int c = 0; c < nc; ++c) {
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar))) {
                    ok = false;
                    break;
                }
                const int lh = min(stage_lines, lines - c * stage_lines);
                scan_stage<U>(ring_w + (uint32_t)cstage * stage_bytes, lh >> 2, lane, sv, ahi, alo, bmx, bmn);
                __syncwarp();
                if (lane == 0) {
                    fence_proxy_async_smem();
                    issue_next();
                }
                if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
                ++consumed;
            }
            if (!ok) break;
            const float e = finish_row(ahi, alo, bmx, bmn, Tp, Tm, lane);
            if (lane == 0) J.ferr[f] = e;
            wmin = fminf(wmin, e);
        }
        if (!ok) {
            // record the failure, wait (bounded) for this warp's copies in flight, stop working
            if (lane == 0) {
                atomicOr(&meta->flags, kFlagWaitTimeout);
                atomicOr(&J.rs->flags, kFlagWaitTimeout);
                const int pending = __shfl_sync(1u, issued, 0) - consumed;
                for (int s = 0; s < pending; ++s) {
                    mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar, 100000000ull);
                    if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
                }
            }
            __syncwarp();
        }
        if (lane == 0) s_min[warp] = wmin;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = INFINITY;
            for (int w = 0; w < nw; ++w) m = fminf(m, s_min[w]);
            if (m < INFINITY) atomicMin(&J.rs->screen_min_bits, __float_as_uint(fmaxf(m, 0.f)));
        }
        __syncthreads();
    }
    // the last CTA resets the work queue for the next round
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&meta->screen_done, 1u) == gridDim.x - 1) {
            meta->item_next = 0u;
            meta->screen_done = 0u;
        }
    }
}

// Partitioned schedule: CTA c takes one contiguous range of all jobs' rows
// (job after job), sized by k_bbegin so that every CTA streams the same number
// of table lines; inside it, warp w takes every nw-th row of each job, and its
// producer lane runs ahead across job boundaries so the TMA ring never drains.
// The CTA synchronises only when it moves to the next job (to swap the weights
// in shared memory), which with ranges this long happens once or twice a round.
template <int U>
__global__ void __launch_bounds__(U >= 4 ? 384 : (U == 3 ? 512 : 640), 1)
    k_bscreen_pt(const __grid_constant__ BatchMaps maps, const JobDesc *__restrict__ jobs,
                 BatchMeta *meta, int max_words, int stages, int stage_lines) {
    extern __shared__ __align__(16) float sv[];
    __shared__ float s_min[32];
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t stage_bytes = (uint32_t)stage_lines * kLineBytes;
    const uint32_t sv32 = smem_u32(sv);
    const uint32_t ring0 = (uint32_t)align_up(sv32 + (uint32_t)max_words * 4u, 1024);
    const uint32_t bars0 = ring0 + (uint32_t)nw * stages * stage_bytes;
    const uint32_t ring_w = ring0 + (uint32_t)warp * stages * stage_bytes;
    const uint32_t bar_w = bars0 + (uint32_t)(warp * stages * 8);
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(bar_w + 8 * s, 1);
        fence_barrier_init();
    }
    const int nj = meta->njobs;
    const int64_t g0 = meta->cta_start[blockIdx.x], g1 = meta->cta_start[blockIdx.x + 1];
    // first job of the range
    const int j0 = find_job(nj, g0, [&](int i) { return jobs[i].feat_base; });
    // the CTA's rows of job J: [a, b); this warp's: a + warp, a + warp + nw, ...
    auto range_of = [&](const JobDesc &J, int64_t &a, int64_t &b) {
        a = max(g0 - J.feat_base, (int64_t)0);
        b = min(g1 - J.feat_base, J.nfeat);
        if (!J.rs->in_round || a >= b) a = b = 0;
    };
    auto rows_of = [&](int64_t a, int64_t b) -> int {
        return b - a > warp ? (int)((b - a - warp + nw - 1) / nw) : 0;
    };
    // producer (lane 0): job of the next load, the arena line of its stage, the
    // lines left in its row and the rows left in the job, in this warp's order
    int pj = j0 - 1, pstage = 0, p_lines = 0, p_left = 0, p_rows = 0, issued = 0;
    int32_t p_row = 0, p_cur = 0, p_step = 0;
    auto next_job = [&]() {
        for (++pj; pj < nj && jobs[pj].feat_base < g1; ++pj) {
            const JobDesc &J = jobs[pj];
            int64_t a, b;
            range_of(J, a, b);
            p_rows = rows_of(a, b);
            if (p_rows) {
                p_lines = J.lines;
                p_left = p_lines;
                p_row = (int32_t)(J.line_base + (a + warp) * (int64_t)p_lines);
                p_cur = p_row;
                p_step = nw * p_lines;
                return;
            }
        }
        pj = nj;
    };
    auto issue_next = [&]() {
        if (pj >= nj) return;
        const int lh = min(stage_lines, p_left);
        tma_stage(maps, ring_w + (uint32_t)pstage * stage_bytes, p_cur, lh, stage_lines,
                  bar_w + 8u * (uint32_t)pstage);
        if (++pstage == stages) pstage = 0;
        ++issued;
        p_cur += lh;
        if ((p_left -= lh) == 0) {
            if (--p_rows == 0) {
                next_job();
            } else {
                p_row += p_step;
                p_cur = p_row;
                p_left = p_lines;
            }
        }
    };
    if (lane == 0) {
        next_job();
        for (int s = 0; s < stages; ++s) issue_next();
    }
    __syncwarp();
    int cstage = 0, prev = -1;
    uint32_t cpar = 0;
    int consumed = 0;
    bool ok = true;  // false once one of this warp's waits timed out
    for (int j = j0; j < nj && jobs[j].feat_base < g1; ++j) {
        const JobDesc &J = jobs[j];
        int64_t a, b;
        range_of(J, a, b);
        if (a >= b) continue;  // uniform over the CTA
        __syncthreads();  // every warp is done with the previous job's weights and minima
        if (prev >= 0 && threadIdx.x == 0) {
            float m = INFINITY;
            for (int w = 0; w < nw; ++w) m = fminf(m, s_min[w]);
            if (m < INFINITY) atomicMin(&jobs[prev].rs->screen_min_bits, __float_as_uint(fmaxf(m, 0.f)));
        }
        for (int i = threadIdx.x; i < J.lay.words; i += blockDim.x) sv[i] = J.v[i];
        __syncthreads();
        prev = j;
        const int lines = J.lines;
        const int nc = (lines + stage_lines - 1) / stage_lines;
        const int nrows = ok ? rows_of(a, b) : 0;
        const float Tp = (float)J.rs->t_pos, Tm = (float)J.rs->t_neg;
        float *ferr = J.ferr;
        float wmin = INFINITY;
        const int f0 = (int)a + warp;
        for (int k = 0; k < nrows && ok; ++k) {
            const int f = f0 + k * nw;
            float ahi = 0.f, alo = 0.f, bmx = -INFINITY, bmn = INFINITY;
            for (int c = 0; c < nc; ++c) {
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar))) {
                    ok = false;
                    break;
                }
                const int lh = min(stage_lines, lines - c * stage_lines);
                scan_stage<U>(ring_w + (uint32_t)cstage * stage_bytes, lh >> 2, lane, sv, ahi, alo, bmx, bmn);
                __syncwarp();
                if (lane == 0) {
                    fence_proxy_async_smem();
                    issue_next();
                }
                if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
                ++consumed;
            }
            if (!ok) break;
            const float e = finish_row(ahi, alo, bmx, bmn, Tp, Tm, lane);
            if (lane == 0) ferr[f] = e;
            wmin = fminf(wmin, e);
        }
        if (!ok && lane == 0) {
            atomicOr(&meta->flags, kFlagWaitTimeout);
            atomicOr(&J.rs->flags, kFlagWaitTimeout);
        }
        if (lane == 0) s_min[warp] = wmin;
    }
    __syncthreads();
    if (prev >= 0 && threadIdx.x == 0) {
        float m = INFINITY;
        for (int w = 0; w < nw; ++w) m = fminf(m, s_min[w]);
        if (m < INFINITY) atomicMin(&jobs[prev].rs->screen_min_bits, __float_as_uint(fmaxf(m, 0.f)));
    }
    if (!ok && lane == 0) {
        // wait (bounded) for this warp's copies still in flight before the CTA exits
        const int pending = issued - consumed;
        for (int s = 0; s < pending; ++s) {
            mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar, 100000000ull);
            if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
        }
    }
}

// Interleaved schedule: the plain search's row order applied to each job in
// turn.  Warp w of the grid (G warps) takes rows w, w + G, w + 2G, ... of job
// 0, then of job 1, and so on, so at any time the whole GPU streams one compact
// window of consecutive rows, as the plain search does; the producer lane runs
// ahead across job boundaries.  The CTA synchronises at every job (to swap the
// weights), and skips jobs in which none of its warps has a row.
template <int U>
__global__ void __launch_bounds__(U >= 4 ? 384 : (U == 3 ? 512 : 640), 1)
    k_bscreen_il(const __grid_constant__ BatchMaps maps, const JobDesc *__restrict__ jobs,
                 BatchMeta *meta, int max_words, int stages, int stage_lines) {
    extern __shared__ __align__(16) float sv[];
    __shared__ float s_min[32];
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t stage_bytes = (uint32_t)stage_lines * kLineBytes;
    const uint32_t sv32 = smem_u32(sv);
    const uint32_t ring0 = (uint32_t)align_up(sv32 + (uint32_t)max_words * 4u, 1024);
    const uint32_t bars0 = ring0 + (uint32_t)nw * stages * stage_bytes;
    const uint32_t ring_w = ring0 + (uint32_t)warp * stages * stage_bytes;
    const uint32_t bar_w = bars0 + (uint32_t)(warp * stages * 8);
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(bar_w + 8 * s, 1);
        fence_barrier_init();
    }
    const int nj = meta->njobs;
    // 32-bit state: rows, lines of the arena and counts fit, and the scan
    // below needs the registers
    const int gw = blockIdx.x * nw + warp;
    const int G = gridDim.x * nw;
    auto rows_of = [&](const JobDesc &J) -> int {
        return (J.rs->in_round && gw < J.nfeat) ? (int)((J.nfeat - 1 - gw) / G + 1) : 0;
    };
    // producer (lane 0): job of the next load, the arena line of its stage, the
    // lines left in its row and the rows left in the job
    int pj = -1, pstage = 0, p_lines = 0, p_left = 0, p_rows = 0, issued = 0;
    int32_t p_row = 0, p_cur = 0, p_step = 0;
    auto next_job = [&]() {
        for (++pj; pj < nj; ++pj) {
            const JobDesc &J = jobs[pj];
            p_rows = rows_of(J);
            if (p_rows) {
                p_lines = J.lines;
                p_left = p_lines;
                p_row = (int32_t)(J.line_base + (int64_t)gw * p_lines);
                p_cur = p_row;
                p_step = G * p_lines;
                return;
            }
        }
    };
    auto issue_next = [&]() {
        if (pj >= nj) return;
        const int lh = min(stage_lines, p_left);
        tma_stage(maps, ring_w + (uint32_t)pstage * stage_bytes, p_cur, lh, stage_lines,
                  bar_w + 8u * (uint32_t)pstage);
        if (++pstage == stages) pstage = 0;
        ++issued;
        p_cur += lh;
        if ((p_left -= lh) == 0) {
            if (--p_rows == 0) {
                next_job();
            } else {
                p_row += p_step;
                p_cur = p_row;
                p_left = p_lines;
            }
        }
    };
    if (lane == 0) {
        next_job();
        for (int s = 0; s < stages; ++s) issue_next();
    }
    __syncwarp();
    int cstage = 0, prev = -1;
    uint32_t cpar = 0;
    int consumed = 0;
    bool ok = true;  // false once one of this warp's waits timed out
    for (int j = 0; j < nj; ++j) {
        const JobDesc &J = jobs[j];
        if (!J.rs->in_round || (int64_t)blockIdx.x * nw >= J.nfeat) continue;  // uniform over the CTA
        __syncthreads();  // every warp is done with the previous job's weights and minima
        if (prev >= 0 && threadIdx.x == 0) {
            float m = INFINITY;
            for (int w = 0; w < nw; ++w) m = fminf(m, s_min[w]);
            if (m < INFINITY) atomicMin(&jobs[prev].rs->screen_min_bits, __float_as_uint(fmaxf(m, 0.f)));
        }
        for (int i = threadIdx.x; i < J.lay.words; i += blockDim.x) sv[i] = J.v[i];
        __syncthreads();
        prev = j;
        const int lines = J.lines;
        const int nc = (lines + stage_lines - 1) / stage_lines;
        const int nrows = ok ? rows_of(J) : 0;
        const float Tp = (float)J.rs->t_pos, Tm = (float)J.rs->t_neg;
        float *ferr = J.ferr;
        float wmin = INFINITY;
        for (int k = 0; k < nrows && ok; ++k) {
            const int f = gw + k * G;
            float ahi = 0.f, alo = 0.f, bmx = -INFINITY, bmn = INFINITY;
            for (int c = 0; c < nc; ++c) {
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar))) {
                    ok = false;
                    break;
                }
                const int lh = min(stage_lines, lines - c * stage_lines);
                scan_stage<U>(ring_w + (uint32_t)cstage * stage_bytes, lh >> 2, lane, sv, ahi, alo, bmx, bmn);
                __syncwarp();
                if (lane == 0) {
                    fence_proxy_async_smem();
                    issue_next();
                }
                if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
                ++consumed;
            }
            if (!ok) break;
            const float e = finish_row(ahi, alo, bmx, bmn, Tp, Tm, lane);
            if (lane == 0) ferr[f] = e;
            wmin = fminf(wmin, e);
        }
        if (!ok && lane == 0) {
            atomicOr(&meta->flags, kFlagWaitTimeout);
            atomicOr(&J.rs->flags, kFlagWaitTimeout);
        }
        if (lane == 0) s_min[warp] = wmin;
    }
    __syncthreads();
    if (prev >= 0 && threadIdx.x == 0) {
        float m = INFINITY;
        for (int w = 0; w < nw; ++w) m = fminf(m, s_min[w]);
        if (m < INFINITY) atomicMin(&jobs[prev].rs->screen_min_bits, __float_as_uint(fmaxf(m, 0.f)));
    }
    if (!ok && lane == 0) {
        // wait (bounded) for this warp's copies still in flight before the CTA exits
        const int pending = issued - consumed;
        for (int s = 0; s < pending; ++s) {
            mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar, 100000000ull);
            if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
        }
    }
}

cudaError_t launch_bscreen(const BatchMaps &maps, const JobDesc *jobs, const WorkItem *items,
                           BatchMeta *meta, int max_words, const SearchShape &shape, int schedule,
                           int grid, cudaStream_t st) {
    const size_t sm = bscreen_smem_bytes(shape, max_words);
    const int threads = shape.warps * 32;
    const int sl = shape.box_lines;
    if (schedule == VJB_BATCH_INTERLEAVED) {
        switch (shape.unroll) {
        case 1: k_bscreen_il<1><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl); break;
        case 3: k_bscreen_il<3><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl); break;
        case 4: k_bscreen_il<4><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl); break;
        default: k_bscreen_il<2><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl);
        }
        return cudaGetLastError();
    }
    if (schedule == VJB_BATCH_PARTITIONED) {
        switch (shape.unroll) {
        case 1: k_bscreen_pt<1><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl); break;
        case 3: k_bscreen_pt<3><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl); break;
        case 4: k_bscreen_pt<4><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl); break;
        default: k_bscreen_pt<2><<<grid, threads, sm, st>>>(maps, jobs, meta, max_words, shape.stages, sl);
        }
        return cudaGetLastError();
    }
    switch (shape.unroll) {
    case 1: k_bscreen<1><<<grid, threads, sm, st>>>(maps, jobs, items, meta, max_words, shape.stages, sl); break;
    case 3: k_bscreen<3><<<grid, threads, sm, st>>>(maps, jobs, items, meta, max_words, shape.stages, sl); break;
    case 4: k_bscreen<4><<<grid, threads, sm, st>>>(maps, jobs, items, meta, max_words, shape.stages, sl); break;
    default: k_bscreen<2><<<grid, threads, sm, st>>>(maps, jobs, items, meta, max_words, shape.stages, sl);
    }
    return cudaGetLastError();
}

cudaError_t set_bscreen_smem_limit(int bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void *)k_bscreen<1>);
    set((const void *)k_bscreen<2>);
    set((const void *)k_bscreen<3>);
    set((const void *)k_bscreen<4>);
    set((const void *)k_bscreen_pt<1>);
    set((const void *)k_bscreen_pt<2>);
    set((const void *)k_bscreen_pt<3>);
    set((const void *)k_bscreen_pt<4>);
    set((const void *)k_bscreen_il<1>);
    set((const void *)k_bscreen_il<2>);
    set((const void *)k_bscreen_il<3>);
    set((const void *)k_bscreen_il<4>);
    return e;
}


__global__ void __launch_bounds__(256) k_bshortlist(const JobDesc *__restrict__ jobs, BatchMeta *meta) {
    __shared__ int64_t base[kMaxBatchJobs];
    const int nj = meta->njobs;
    const int64_t total = meta->total_feat;
    for (int j = threadIdx.x; j < nj; j += blockDim.x) base[j] = jobs[j].feat_base;
    __syncthreads();
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < nj; j += blockDim.x)
            if (jobs[j].rs->in_round) jobs[j].rs->screen_min = __uint_as_float(jobs[j].rs->screen_min_bits);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const int j = find_job(nj, g, [&](int i) { return base[i]; });
        const JobDesc &J = jobs[j];
        RoundState *rs = J.rs;
        if (!rs->in_round) continue;
        const int64_t f = g - J.feat_base;
        if (f >= J.nfeat) continue;
        const float thr = shortlist_threshold(__uint_as_float(rs->screen_min_bits), rs);
        if (J.ferr[f] <= thr) J.cand_ids[atomicAdd(&rs->cand_count, 1)] = (int32_t)f;
    }
}

cudaError_t launch_bshortlist(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st) {
    k_bshortlist<<<grid, 256, 0, st>>>(jobs, meta);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kRescanWarps * 32) k_brescan(const JobDesc *__restrict__ jobs, BatchMeta *meta) {
    __shared__ RunResult rres[32];
    __shared__ int pref[kMaxBatchJobs + 1];
    __shared__ bool s_last;
    const int nj = meta->njobs;
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int j = 0; j < nj; ++j) {
            pref[j] = acc;
            const RoundState *rs = jobs[j].rs;
            if (rs->in_round && rs->status == VJB_OK) {
                if (rs->cand_count == 0 && blockIdx.x == 0) {  // nothing to pick from: stop the job
                    jobs[j].rs->flags |= kFlagNoCandidate;
                    jobs[j].rs->status = VJB_EDEVICE;
                } else {
                    acc += rs->cand_count;
                }
            }
        }
        pref[nj] = acc;
    }
    __syncthreads();
    const int total = pref[nj];
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        int j = 0;
        while (pref[j + 1] <= p) ++j;
        const JobDesc &J = jobs[j];
        const int c = p - pref[j];
        const Candidate cd = rescan_feature(J, J.cand_ids[c], rres);
        if (threadIdx.x == 0) {
            J.cands[c] = cd;
            __threadfence();
            s_last = atomicAdd(&J.rs->done_rescan, 1u) == (uint32_t)(pref[j + 1] - pref[j]) - 1;
        }
        __syncthreads();
        if (s_last) {  // the job's last candidate: pick its stump
            __threadfence();
            select_stump(J, pref[j + 1] - pref[j]);
        }
        __syncthreads();
    }
}

cudaError_t launch_brescan(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st) {
    k_brescan<<<grid, kRescanWarps * 32, 0, st>>>(jobs, meta);
    return cudaGetLastError();
}

}  // namespace vjb

namespace vjb {

// ---- allocation-free variant of the search kernel --------------------------------------
// Some callers cannot call cudaMalloc at the moment they want a search: a host
// that is stream-capturing its own CUDA graph, a real-time loop whose memory
// is fixed up front, or a framework that hands all device memory to its own
// pool.  vjb_screen_noalloc serves them: the caller passes the sorted table,
// the signed weights and the outputs, and the only scratch the search needs --
// one (error, feature) partial per CTA plus a completion counter for the
// last-CTA reduction -- lives in the file-scope array below.  Every GPU that
// loads this library holds the array (8.4 KiB) until the process exits, and
// every call shares it.
constexpr int kNoAllocMaxCtas = 1024;
constexpr int kNoAllocWords = 2 * kNoAllocMaxCtas + 64;
constexpr int kNoAllocDone = 2 * kNoAllocMaxCtas;      // completion counter
constexpr int kNoAllocFlags = 2 * kNoAllocMaxCtas + 1; // error flags of the call
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// Dynamic shared memory of k_screen_noalloc: the TMA rings first (1 KiB
// aligned), then the n + 1 weights, the mbarriers and the per-warp minima.
static size_t noalloc_smem_bytes(const SearchShape &s, int n) {
    size_t b = 1024;
    b += (size_t)s.warps * s.stages * kStageBytes;
    b += align_up((size_t)(n + 1) * 4, 16);
    b += (size_t)s.warps * s.stages * 8;
    b += (size_t)s.warps * 4;
    return b;
}

// Same unit as screen_unit, with every gathered index clamped to n: the table
// comes straight from the caller, so an entry above n reads as padding.
__device__ __forceinline__ void screen_unit_clamped(uint32_t sbase, int unit, int lane,
                                                    int lines_here, uint32_t n,
                                                    const float *__restrict__ sv, float &chi,
                                                    float &clo, float &MX, float &MN) {
    const uint32_t line = (uint32_t)unit * 8u + ((uint32_t)lane >> 2);
    const uint32_t sw = ((uint32_t)lane >> 2) & 7u;
    const uint32_t c0 = ((2u * ((uint32_t)lane & 3u)) ^ sw) << 4;
    const uint32_t c1 = ((2u * ((uint32_t)lane & 3u) + 1u) ^ sw) << 4;
    const uint32_t pad2 = n | (n << 16);
    uint4 q0 = make_uint4(pad2, pad2, pad2, pad2), q1 = q0;
    if (line < (uint32_t)lines_here) {
        q0 = lds128(sbase + line * kLineBytes + c0);
        q1 = lds128(sbase + line * kLineBytes + c1);
    }
    const uint32_t wd[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
    float g[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        g[2 * j] = sv[min(wd[j] & kIndexMask, n)];
        g[2 * j + 1] = sv[min((wd[j] >> 16) & kIndexMask, n)];
    }
    float a = 0.f, mx = -INFINITY, mn = INFINITY;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        a += g[j];
        const uint32_t fl = (j & 1) ? (wd[j >> 1] & 0x80000000u) : (wd[j >> 1] & 0x8000u);
        if (fl) {
            mx = fmaxf(mx, a);
            mn = fminf(mn, a);
        }
    }
    float x = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    float excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) excl = 0.f;
    const float tot = __shfl_sync(0xffffffffu, x, 31);
    const float base = chi + (clo + excl);
    MX = fmaxf(MX, base + mx);
    MN = fminf(MN, base + mn);
    float s, e;
    two_sum(chi, tot, s, e);
    chi = s;
    clo += e;
}

__global__ void __launch_bounds__(512, 1)
    k_screen_noalloc(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ v, int n,
                     int lines_per_row, int box_lines, int64_t nfeat, int stages, float Tp,
                     float Tm, float *__restrict__ ferr, float *__restrict__ best_err,
                     int32_t *__restrict__ best_feature, uint32_t *__restrict__ scratch) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(align_up(reinterpret_cast<size_t>(smem_raw), 1024));
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *rings = base;
    float *sv = reinterpret_cast<float *>(rings + (size_t)nw * stages * kStageBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sv + align_up((size_t)(n + 1), 4));
    float *wbest = reinterpret_cast<float *>(bars + nw * stages);
    __shared__ int32_t wfeat[16];
    __shared__ bool last_cta;

    for (int i = threadIdx.x; i <= n; i += blockDim.x) sv[i] = (i < n) ? v[i] : 0.f;
    const uint32_t ring_w = smem_u32(rings + (size_t)warp * stages * kStageBytes);
    const uint32_t bar_w = smem_u32(bars + warp * stages);
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(bar_w + 8 * s, 1);
        fence_barrier_init();
    }
    __syncthreads();

    const int64_t gw = (int64_t)blockIdx.x * nw + warp;
    const int64_t G = (int64_t)gridDim.x * nw;
    const int64_t nf_w = gw < nfeat ? (nfeat - 1 - gw) / G + 1 : 0;
    const int nc = (lines_per_row + box_lines - 1) / box_lines;
    const int64_t total = nf_w * nc;
    const uint32_t tx = (uint32_t)box_lines * kLineBytes;
    auto issue = [&](int64_t seq) {
        const int64_t k = seq / nc;
        const int c = (int)(seq - k * nc);
        const int64_t f = gw + k * G;
        const int stage = (int)(seq % stages);
        const uint32_t bar = bar_w + 8u * stage;
        mbar_arrive_expect_tx(bar, tx);
        tma_load_3d(ring_w + (uint32_t)stage * kStageBytes, &tmap, 0, c * box_lines, (int32_t)f, bar);
    };
    if (lane == 0) {
        const int64_t pro = total < stages ? total : stages;
        for (int64_t s = 0; s < pro; ++s) issue(s);
    }
    __syncwarp();

    float best = INFINITY;
    int32_t bestf = 0x7fffffff;
    int64_t seq = 0;
    bool ok = true;
    for (int64_t k = 0; k < nf_w && ok; ++k) {
        const int64_t f = gw + k * G;
        float chi = 0.f, clo = 0.f, MX = 0.f, MN = 0.f;
        for (int c = 0; c < nc; ++c) {
            const int stage = (int)(seq % stages);
            const uint32_t par = (uint32_t)((seq / stages) & 1);
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_w + 8u * stage, par))) {
                ok = false;
                break;
            }
            const int lines_here = min(box_lines, lines_per_row - c * box_lines);
            const int units = (lines_here + 7) >> 3;
            const uint32_t sbase = ring_w + (uint32_t)stage * kStageBytes;
            for (int u = 0; u < units; ++u)
                screen_unit_clamped(sbase, u, lane, lines_here, (uint32_t)n, sv, chi, clo, MX, MN);
            __syncwarp();
            if (lane == 0 && seq + stages < total) {
                fence_proxy_async_smem();
                issue(seq + stages);
            }
            ++seq;
        }
        if (!ok) break;
        MX = warp_max(MX);
        MN = warp_min(MN);
        const float e = fminf(Tp - MX, Tm + MN);
        if (lane == 0) {
            ferr[f] = e;
            if (e < best) { best = e; bestf = (int32_t)f; }
        }
    }
    if (!ok && lane == 0) {
        atomicOr(&scratch[kNoAllocFlags], (uint32_t)kFlagWaitTimeout);
        const int64_t issued = (seq + stages < total) ? seq + stages : total;
        for (int64_t s = seq; s < issued; ++s)
            mbar_wait_bounded(bar_w + 8u * (uint32_t)(s % stages), (uint32_t)((s / stages) & 1), 100000000ull);
    }
    __syncwarp();
    if (lane == 0) { wbest[warp] = best; wfeat[warp] = bestf; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = INFINITY;
        int32_t mf = 0x7fffffff;
        for (int w = 0; w < nw; ++w)
            if (wbest[w] < m || (wbest[w] == m && wfeat[w] < mf)) { m = wbest[w]; mf = wfeat[w]; }
        scratch[blockIdx.x] = __float_as_uint(m);
        scratch[kNoAllocMaxCtas + blockIdx.x] = (uint32_t)mf;
        __threadfence();
        last_cta = atomicAdd(&scratch[kNoAllocDone], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last_cta && threadIdx.x == 0) {
        __threadfence();
        float m = INFINITY;
        int32_t mf = -1;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            const float e = __uint_as_float(((volatile uint32_t *)scratch)[b]);
            const int32_t f = (int32_t)((volatile uint32_t *)scratch)[kNoAllocMaxCtas + b];
            if (e < m || (e == m && f < mf)) { m = e; mf = f; }
        }
        const bool failed = ((volatile uint32_t *)scratch)[kNoAllocFlags] != 0u;
        *best_err = m;
        *best_feature = failed ? -1 : mf;
        scratch[kNoAllocDone] = 0u;  // the next call starts from zero
    }
}

}  // namespace vjb

namespace {

typedef CUresult (*NoAllocEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct NoAllocDevice {
    bool ready = false;
    uint32_t *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int num_sms = 0;
    int max_smem = 0;             // dynamic shared memory the kernel may use
};
constexpr int kNoAllocDevices = 64;
NoAllocDevice g_noalloc_dev[kNoAllocDevices];
NoAllocEncodeFn g_noalloc_encode = nullptr;
std::mutex g_noalloc_mu;

}  // namespace

namespace vjb {
int report_error(int code, const char *msg);
}

extern "C" int vjb_screen_noalloc(const uint16_t *rows, const float *v, int32_t n, int32_t npad,
                                  int64_t nfeat, double t_pos, double t_neg, int32_t ctas,
                                  float *feature_err, float *best_err, int32_t *best_feature,
                                  void *cuda_stream) {
    using namespace vjb;
    if (!rows || !v || !feature_err || !best_err || !best_feature)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: NULL pointer argument");
    if (n < 1 || n > VJB_MAX_SAMPLES)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: n outside [1, VJB_MAX_SAMPLES]");
    if (npad < n || npad % kLineElems != 0)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: npad must be >= n and a multiple of 64");
    if (nfeat < 1 || nfeat > 0x7fffffffLL)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: nfeat outside [1, 2^31 - 1]");
    if ((reinterpret_cast<uintptr_t>(rows) & 15u) != 0)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: rows must be 16-byte aligned");
    if (!(t_pos >= 0.0) || !(t_neg >= 0.0) || !std::isfinite(t_pos) || !std::isfinite(t_neg))
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: class totals must be finite and >= 0");
    if (ctas < 0 || ctas > kNoAllocMaxCtas)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: ctas outside [0, 1024] (the scratch array holds 1024 partials)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocDevices)
        return report_error(VJB_ECUDA, "vjb_screen_noalloc: no usable current device");
    NoAllocDevice &D = g_noalloc_dev[dev];
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!D.ready) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return report_error(VJB_ECUDA, "vjb_screen_noalloc: cudaGetSymbolAddress of the scratch array failed");
            int optin = 0;
            cudaFuncAttributes fa;
            if (cudaDeviceGetAttribute(&D.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, k_screen_noalloc) != cudaSuccess)
                return report_error(VJB_ECUDA, "vjb_screen_noalloc: device attribute query failed");
            // the kernel's own static shared memory comes out of the same per-CTA limit
            D.max_smem = optin - (int)fa.sharedSizeBytes;
            if (cudaFuncSetAttribute(k_screen_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, D.max_smem) != cudaSuccess)
                return report_error(VJB_ECUDA, "vjb_screen_noalloc: setting the kernel's shared-memory limit failed");
            if (!g_noalloc_encode) {
                void *fn = nullptr;
                cudaDriverEntryPointQueryResult q;
                if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
                    q != cudaDriverEntryPointSuccess || !fn)
                    return report_error(VJB_ECUDA, "vjb_screen_noalloc: cuTensorMapEncodeTiled unavailable");
                g_noalloc_encode = reinterpret_cast<NoAllocEncodeFn>(fn);
            }
            D.scratch = static_cast<uint32_t *>(p);
            D.ready = true;
        }
    }
    const int grid = ctas ? ctas : std::min(D.num_sms, kNoAllocMaxCtas);
    const SearchShape tries[] = {{8, 4, 1, 1, 32}, {8, 3, 1, 1, 32}, {4, 4, 1, 1, 32}, {4, 2, 1, 1, 32},
                                 {2, 2, 1, 1, 32}};
    const SearchShape *shape = nullptr;
    for (const auto &s : tries)
        if (noalloc_smem_bytes(s, n) <= (size_t)D.max_smem) { shape = &s; break; }
    if (!shape) return report_error(VJB_EINVAL, "vjb_screen_noalloc: n too large for shared memory");
    const int lines = npad / kLineElems;
    const int box_lines = std::min(kBoxLinesMax, lines);
    CUtensorMap tmap;
    cuuint64_t dims[3] = {(cuuint64_t)kLineElems, (cuuint64_t)lines, (cuuint64_t)nfeat};
    cuuint64_t strides[2] = {(cuuint64_t)kLineBytes, (cuuint64_t)lines * kLineBytes};
    cuuint32_t box[3] = {(cuuint32_t)kLineElems, (cuuint32_t)box_lines, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (g_noalloc_encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t *>(rows), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return report_error(VJB_EINVAL, "vjb_screen_noalloc: the table cannot be described by a tensor map");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the counter and the flags must start at zero; the partials are all overwritten
    if (cudaMemsetAsync(D.scratch + kNoAllocDone, 0, 2 * sizeof(uint32_t), st) != cudaSuccess)
        return report_error(VJB_ECUDA, "vjb_screen_noalloc: clearing the scratch counter failed");
    k_screen_noalloc<<<grid, shape->warps * 32, noalloc_smem_bytes(*shape, n), st>>>(
        tmap, v, n, lines, box_lines, nfeat, shape->stages, (float)t_pos, (float)t_neg, feature_err,
        best_err, best_feature, D.scratch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(VJB_ECUDA, cudaGetErrorString(e));
    return VJB_OK;
}
