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
//    row layout interleaves 32 runs), summing 16 or 24 entries at a time in
//    FP32 and folding each piece into a compensated (TwoSum) running total; one
//    FP32 warp scan of the 32 run totals per row places every lane's best
//    prefix in the row.  It writes each feature's FP32 error and each CTA's
//    minimum.
//  * k_shortlist: lists every feature whose screened error is within a margin
//    of the smallest one.
//  * k_rescan: one CTA per listed feature scans its row again in double-float
//    (compensated FP32) arithmetic throughout, giving the feature's best split,
//    polarity and an error to about 1e-14 relative; the last CTA to finish
//    picks the round's stump: lowest error, then feature, split, +1 before -1.
//
// Screening error bound (u = 2^-24, sum |v| = T+ + T- = 1 after normalising):
// a piece's partial sums of at most 24 terms err by at most 24u times the
// piece's |v| mass; the compensated run total adds O(u^2); placing the
// piece's extreme on the run total adds 2u |D|; rounding the 32 run totals
// to FP32 adds u, their five-level FP32 scan 5u (each total passes through
// at most five additions, sum |run totals| <= 1), and placing a lane's
// extreme on its run offset u |D|; forming T+- -/+ D in FP32 adds 2u.  So
// |screened - exact| <= 35u.  A margin of 72u (twice 36u) keeps every
// feature that could beat the best one.
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "k_search.cuh"

namespace vjb {

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

    const uint32_t ring_w = ring0 + (uint32_t)warp * stages * stage_bytes;
    const uint32_t bar_w = bars0 + (uint32_t)(warp * stages * 8);
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(bar_w + 8 * s, 1);
        fence_barrier_init();
    }

    // rows gw, gw + G, ... of this warp; feature indices fit int32 (nfeat <
    // 2^31), and so does the warp's chunk count (G >= 152 warps, at most 128
    // chunks per row)
    const int gw = blockIdx.x * nw + warp;
    const int G = gridDim.x * nw;
    const int nf_w = gw < nfeat ? (int)((nfeat - 1 - gw) / G) + 1 : 0;
    const int nc = (lines_per_row + box_lines - 1) / box_lines;
    const int total = nf_w * nc;
    const uint32_t tx = (uint32_t)box_lines * kLineBytes;

    // producer state (lane 0): the next chunk to load, in this warp's order
    int issued = 0, prow = gw, pline = 0, pstage = 0;
    const int last_line = (nc - 1) * box_lines;
    auto issue_next = [&]() {
        if (issued >= total) return;
        const uint32_t bar = bar_w + 8u * (uint32_t)pstage;
        mbar_arrive_expect_tx(bar, tx);
        tma_load_3d(ring_w + (uint32_t)pstage * stage_bytes, &tmap, 0, pline, prow, bar);
        if (pline == last_line) { pline = 0; prow += G; } else { pline += box_lines; }
        if (++pstage == stages) pstage = 0;
        ++issued;
    };
    if (lane == 0)
        for (int s = 0; s < stages; ++s) issue_next();
    __syncwarp();
    // the weights, staged while the first copies of the table are in flight
    stage_weights(sv, v, words);
    __syncthreads();

    const float Tp = (float)rs->t_pos, Tm = (float)rs->t_neg;
    float best = INFINITY;
    int cstage = 0;
    uint32_t cpar = 0;  // consumer ring position and mbarrier phase
    int consumed = 0;
    bool ok = true;
    const int crs_full = box_lines >> 2;                          // chunk rows of a full stage
    const int crs_last = (lines_per_row - (nc - 1) * box_lines) >> 2;  // and of a row's last one
    for (int k = 0; k < nf_w && ok; ++k) {
        const int f = gw + k * G;
        float ahi = 0.f, alo = 0.f, bmx = -INFINITY, bmn = INFINITY;
        // one stage: wait for its copy, scan it, give the slot its next copy
        auto stage_step = [&](auto scan) -> bool {
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_w + 8u * (uint32_t)cstage, cpar))) return false;
            scan(ring_w + (uint32_t)cstage * stage_bytes);
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async_smem();
                issue_next();
            }
            if (++cstage == stages) { cstage = 0; cpar ^= 1u; }
            ++consumed;
            return true;
        };
        if (U == 3 && crs_full == 6) {
            // the default shape: the full stages in a loop of their own around
            // one call that the compiler schedules apart from the general stage
            // (0.787 -> 0.759 ms at 24x24 / 15k), then the row's last stage
            for (int c = 0; c < nc - 1 && ok; ++c)
                ok = stage_step([&](uint32_t sb) { scan_pieces<2, 3>(sb, 0, lane, sv, ahi, alo, bmx, bmn); });
            if (ok) ok = stage_step([&](uint32_t sb) { scan_stage<U>(sb, crs_last, lane, sv, ahi, alo, bmx, bmn); });
        } else {
            for (int c = 0; c < nc && ok; ++c)
                ok = stage_step([&](uint32_t sb) {
                    scan_stage<U>(sb, c == nc - 1 ? crs_last : crs_full, lane, sv, ahi, alo, bmx, bmn);
                });
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
            const int pending = issued - consumed;
            for (int s = 0; s < pending; ++s) {
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

__global__ void __launch_bounds__(256)
    k_shortlist(const JobDesc J, const float *__restrict__ bmin, int nbmin) {
    RoundState *rs = J.rs;
    __shared__ float red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * blockDim.x + warp * 32;
    // every load this kernel needs before it can decide, issued together: the
    // thread's first screened errors, the per-CTA minima and the round state
    // (one trip to memory instead of three in a row: 4.2 instead of 5.5 us a
    // launch at 24x24 / 15k under ncu, with the updates' same change)
    constexpr int kPre = 3;
    float fe[kPre];
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
        const int64_t f = b0 + q * stride + lane;
        fe[q] = f < J.nfeat ? J.ferr[f] : INFINITY;
    }
    float m = INFINITY;
    for (int i = threadIdx.x; i < nbmin; i += blockDim.x) m = fminf(m, bmin[i]);
    if (rs->status != VJB_OK || rs->forced) return;
    m = warp_min(m);
    if (lane == 0) red[warp] = m;
    __syncthreads();
    m = INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fminf(m, red[w]);
    const float thr = shortlist_threshold(m, rs);
    if (blockIdx.x == 0 && threadIdx.x == 0) rs->screen_min = m;
    auto step = [&](int64_t base, float e) {  // base: uniform over the warp
        const int64_t f = base + lane;
        const bool take = f < J.nfeat && e <= thr;
        const uint32_t mask = __ballot_sync(0xffffffffu, take);
        if (!mask) return;
        int slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(&rs->cand_count, __popc(mask));
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        if (take) J.cand_ids[slot0 + __popc(mask & ((1u << lane) - 1u))] = (int32_t)f;
    };
#pragma unroll
    for (int q = 0; q < kPre; ++q)
        if (b0 + q * stride < J.nfeat) step(b0 + q * stride, fe[q]);
    for (int64_t base = b0 + kPre * stride; base < J.nfeat; base += stride)
        step(base, base + lane < J.nfeat ? J.ferr[base + lane] : INFINITY);
}

cudaError_t launch_shortlist(const JobDesc &J, const float *bmin, int nbmin, int grid, cudaStream_t st) {
    k_shortlist<<<grid, 256, 0, st>>>(J, bmin, nbmin);
    return cudaGetLastError();
}

// The compensated re-scan of the shortlist, spread over the SMs: work item i
// is lane run i % 32 of shortlisted feature i / 32, taken by warp (i / G) % W
// of CTA i % G (G CTAs of W warps), so that a feature's 32 runs land on 32
// SMs (one SM doing all 32 was issue-bound: 11.6 us at 24x24 / 15k).  The
// warp that finishes a feature's last run combines its 32 run results; the
// warp that completes the last feature picks the round's stump.  Features
// beyond kRescanSplitCap (only a plateau of ties lists that many) are
// re-scanned whole, one CTA each.
constexpr int kRescanCtas = 32;
constexpr int kRescanCtaWarps = 16;
static_assert(sizeof(RunResult) == kRunResultBytes, "run result layout");

__device__ __forceinline__ RunResult load_run_result(const RunResult *p) {
    const volatile uint32_t *w = reinterpret_cast<const volatile uint32_t *>(p);
    RunResult r;
    r.total.hi = __uint_as_float(w[0]); r.total.lo = __uint_as_float(w[1]);
    r.mx.hi = __uint_as_float(w[2]);    r.mx.lo = __uint_as_float(w[3]);
    r.mn.hi = __uint_as_float(w[4]);    r.mn.lo = __uint_as_float(w[5]);
    r.smx = (int)w[6];                  r.smn = (int)w[7];
    return r;
}

__global__ void __launch_bounds__(kRescanCtaWarps * 32) k_rescan(const JobDesc J) {
    RoundState *rs = J.rs;
    if (rs->status != VJB_OK || rs->forced) return;
    __shared__ RunResult rres[32];
    __shared__ int last_cta;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cnt = rs->cand_count;
    if (cnt == 0) {  // nothing was listed: stop the job with an error flag
        if (blockIdx.x == 0 && warp == 0) select_stump_warp(J, 0, lane);
        return;
    }
    const int run = J.npad / 32;
    const int items = min(cnt, kRescanSplitCap) * 32;
    for (int i = (int)blockIdx.x + (int)gridDim.x * warp; i < items; i += (int)gridDim.x * kRescanCtaWarps) {
        const int c = i >> 5;
        const int32_t f = J.cand_ids[c];
        const RunResult r = rescan_run(J.rows + (size_t)f * J.npad, run, i & 31, J.v, lane);
        uint32_t prev = 0;
        if (lane == 0) {
            J.runres[i] = r;
            __threadfence();
            prev = atomicAdd(&J.cand_runs[c], 1u);
        }
        if (__shfl_sync(0xffffffffu, prev, 0) != 31u) continue;
        // this feature's last run: combine its 32 runs
        __threadfence();
        const Candidate cd = combine_runs(J, f, load_run_result(J.runres + c * 32 + lane), lane);
        if (cnt == 1) {
            // the only listed feature (most rounds): the stump, picked as the
            // list would pick it, without the trip through the list
            if (lane == 0) {
                J.cand_runs[c] = 0u;
                Candidate b;
                b.err_hi = INFINITY; b.err_lo = 0.f; b.feature = INT_MAX; b.split = INT_MAX; b.polarity = 1;
                b.pad = 0;
                if (cand_less(cd, b)) b = cd;
                record_stump(J, 1, b);
            }
            continue;
        }
        uint32_t done = 0;
        if (lane == 0) {
            J.cand_runs[c] = 0u;
            J.cands[c] = cd;
            __threadfence();
            done = atomicAdd(&rs->done_rescan, 1u);
        }
        if (__shfl_sync(0xffffffffu, done, 0) == (uint32_t)cnt - 1) {
            __threadfence();
            select_stump_warp(J, cnt, lane);
        }
    }
    for (int c = kRescanSplitCap + (int)blockIdx.x; c < cnt; c += (int)gridDim.x) {
        const Candidate cd = rescan_feature(J, J.cand_ids[c], rres);
        if (threadIdx.x == 0) {
            J.cands[c] = cd;
            __threadfence();
            last_cta = atomicAdd(&rs->done_rescan, 1u) == (uint32_t)cnt - 1;
        }
        __syncthreads();
        if (last_cta && warp == 0) {
            __threadfence();
            select_stump_warp(J, cnt, lane);
        }
        __syncthreads();
    }
}

cudaError_t launch_rescan(const JobDesc &J, int grid, cudaStream_t st) {
    (void)grid;
    k_rescan<<<kRescanCtas, kRescanCtaWarps * 32, 0, st>>>(J);
    return cudaGetLastError();
}

}  // namespace vjb

namespace vjb {

// ---- allocation-free variant of the search kernel --------------------------------------
// Some callers cannot call cudaMalloc at the moment they want a search: a
// real-time loop whose memory is fixed up front, or a framework that hands all
// device memory to its own pool.  vjb_screen_noalloc serves them: the caller passes the sorted table,
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
        // a wait that gave up leaves rows unscanned: no minimum to report
        const bool failed = ((volatile uint32_t *)scratch)[kNoAllocFlags] != 0u;
        *best_err = failed ? __int_as_float(0x7fc00000) : m;
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
