// Batched round kernels: one launch of each covers every job of a batch (the
// per-job arithmetic is the plain kernels', so a job's results do not depend
// on its batch).  The job table and the counters live in device memory, so a
// round replays as one CUDA graph however the set of jobs changes.
#include "k_search.cuh"

namespace vjb {

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
            stage_weights(sv, J.v, J.lay.words);
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
            const int last_crs = (lines - (nc - 1) * stage_lines) >> 2;
            if (U == 3 && stage_lines == 24) {
                // the default shape: full stages in a loop of their own, then the row's last
                for (int c = 0; c < nc - 1 && ok; ++c)
                    ok = stage_step([&](uint32_t sb) { scan_pieces<2, 3>(sb, 0, lane, sv, ahi, alo, bmx, bmn); });
                if (ok) ok = stage_step([&](uint32_t sb) { scan_stage<U>(sb, last_crs, lane, sv, ahi, alo, bmx, bmn); });
            } else {
                for (int c = 0; c < nc && ok; ++c)
                    ok = stage_step([&](uint32_t sb) {
                        scan_stage<U>(sb, c == nc - 1 ? last_crs : stage_lines >> 2, lane, sv, ahi, alo, bmx, bmn);
                    });
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
        stage_weights(sv, J.v, J.lay.words);
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
            const int last_crs = (lines - (nc - 1) * stage_lines) >> 2;
            if (U == 3 && stage_lines == 24) {
                // the default shape: full stages in a loop of their own, then the row's last
                for (int c = 0; c < nc - 1 && ok; ++c)
                    ok = stage_step([&](uint32_t sb) { scan_pieces<2, 3>(sb, 0, lane, sv, ahi, alo, bmx, bmn); });
                if (ok) ok = stage_step([&](uint32_t sb) { scan_stage<U>(sb, last_crs, lane, sv, ahi, alo, bmx, bmn); });
            } else {
                for (int c = 0; c < nc && ok; ++c)
                    ok = stage_step([&](uint32_t sb) {
                        scan_stage<U>(sb, c == nc - 1 ? last_crs : stage_lines >> 2, lane, sv, ahi, alo, bmx, bmn);
                    });
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
        stage_weights(sv, J.v, J.lay.words);
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
            const int last_crs = (lines - (nc - 1) * stage_lines) >> 2;
            if (U == 3 && stage_lines == 24) {
                // the default shape: full stages in a loop of their own, then the row's last
                for (int c = 0; c < nc - 1 && ok; ++c)
                    ok = stage_step([&](uint32_t sb) { scan_pieces<2, 3>(sb, 0, lane, sv, ahi, alo, bmx, bmn); });
                if (ok) ok = stage_step([&](uint32_t sb) { scan_stage<U>(sb, last_crs, lane, sv, ahi, alo, bmx, bmn); });
            } else {
                for (int c = 0; c < nc && ok; ++c)
                    ok = stage_step([&](uint32_t sb) {
                        scan_stage<U>(sb, c == nc - 1 ? last_crs : stage_lines >> 2, lane, sv, ahi, alo, bmx, bmn);
                    });
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
