// C ABI of batches (many jobs per launch) and of the serving loop (continuous
// batching of training requests); declared in include/vjb.h.
#include "vjb_host.h"

using namespace vjb;

// ---- batches of jobs ------------------------------------------------------------------
// A batch trains many jobs with one launch of each round kernel.  It owns an
// HBM arena for the jobs' sorted tables (the budget given at creation; jobs are
// placed first-fit and rejected with VJB_EFULL when their table does not fit)
// and, per job, a context that owns everything else.

namespace {

struct BatchSlot {
    vjb_ctx *ctx = nullptr;
    int32_t id = -1;
    int64_t line_base = 0, line_count = 0;
    int32_t round_target = 0;
};

constexpr int kBatchMaxWords = 32768;  // weights of any job fit the search kernel's shared memory

}  // namespace

struct vjb_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0, max_smem = 0;
    uint16_t *arena = nullptr;
    int64_t arena_lines = 0;
    BatchMaps maps;
    std::vector<std::pair<int64_t, int64_t>> free_list;  // (first line, line count), by first line
    std::vector<BatchSlot> slots;                        // jobs, in the order of the job table
    int32_t next_id = 0;
    JobDesc *d_jobs = nullptr;
    BatchMeta *d_meta = nullptr;
    WorkItem *d_items = nullptr;
    int items_cap = 0;
    bool dirty = true;  // the device job table must be rebuilt
    SearchShape shape{16, 2, 1, 3, 24};
    int rows_per_warp = VJB_BATCH_INTERLEAVED;  // the schedule; > 0: work queue of that many rows per warp
    // the round graph; with timing on, the search (graph) and the rest
    // (graph2), launched with the timing events (round start, search end,
    // round end) recorded on the stream between them
    cudaGraph_t graph = nullptr, graph2 = nullptr;
    cudaGraphExec_t gexec = nullptr, gexec2 = nullptr;
    int64_t launches = 0;
    bool timing = false, graph_timed = false;
    std::vector<EventTriple> ev_free, ev_pending;
    vjb_timing tacc{};

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gexec2) cudaGraphExecDestroy(gexec2);
        if (graph) cudaGraphDestroy(graph);
        if (graph2) cudaGraphDestroy(graph2);
        gexec = gexec2 = nullptr;
        graph = graph2 = nullptr;
    }
};

namespace {

int batch_encode_maps(vjb_batch *b) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn)
            return fail(VJB_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    const int S = b->shape.box_lines;  // stage height of the batched search
    memset(&b->maps, 0, sizeof b->maps);
    for (int k = 0; k < S / 4; ++k) {
        cuuint64_t dims[2] = {(cuuint64_t)kLineElems, (cuuint64_t)b->arena_lines};
        cuuint64_t strides[1] = {(cuuint64_t)kLineBytes};
        cuuint32_t box[2] = {(cuuint32_t)kLineElems, (cuuint32_t)(k == 0 ? S : 4 * k)};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&b->maps.m[k], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, b->arena, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(VJB_ECUDA, "cuTensorMapEncodeTiled (arena) failed (%d)", (int)r);
    }
    return VJB_OK;
}

int64_t table_lines(int n, int h, int w) {
    std::vector<vjb_feature> f;
    enumerate_host(w, h, f);
    const int64_t npad = (n + kRowAlign - 1) / kRowAlign * kRowAlign;
    return (int64_t)f.size() * (npad / kLineElems);
}

bool arena_take(vjb_batch *b, int64_t count, int64_t *first) {
    for (size_t k = 0; k < b->free_list.size(); ++k) {
        auto &fr = b->free_list[k];
        if (fr.second >= count) {
            *first = fr.first;
            fr.first += count;
            fr.second -= count;
            if (fr.second == 0) b->free_list.erase(b->free_list.begin() + (long)k);
            return true;
        }
    }
    return false;
}

void arena_give(vjb_batch *b, int64_t first, int64_t count) {
    b->free_list.emplace_back(first, count);
    std::sort(b->free_list.begin(), b->free_list.end());
    std::vector<std::pair<int64_t, int64_t>> merged;
    for (const auto &fr : b->free_list) {
        if (!merged.empty() && merged.back().first + merged.back().second == fr.first) merged.back().second += fr.second;
        else merged.push_back(fr);
    }
    b->free_list.swap(merged);
}

BatchSlot *find_slot(vjb_batch *b, int32_t id) {
    for (auto &s : b->slots)
        if (s.id == id) return &s;
    return nullptr;
}

// Rebuild the device job table, the work items and the counters.
int batch_sync(vjb_batch *b) {
    if (!b->dirty) return VJB_OK;
    const int nj = (int)b->slots.size();
    std::vector<JobDesc> jd((size_t)nj);
    std::vector<WorkItem> items;
    const int rows_per_item = std::max(1, b->rows_per_warp) * b->shape.warps;
    int64_t fbase = 0;
    int ubase = 0;
    for (int j = 0; j < nj; ++j) {
        const BatchSlot &s = b->slots[j];
        JobDesc J = job_desc(s.ctx);
        J.active = 1;
        J.round_target = s.round_target;
        J.feat_base = fbase;
        J.ublock_base = ubase;
        jd[j] = J;
        fbase += J.nfeat;
        ubase += update_grid(J.lay.n);
        if (b->rows_per_warp > 0)
            for (int64_t f0 = 0; f0 < J.nfeat; f0 += rows_per_item)
                items.push_back(WorkItem{j, (int32_t)f0, (int32_t)std::min<int64_t>(J.nfeat, f0 + rows_per_item), 0});
    }
    if ((int)items.size() > b->items_cap) {
        dfree(b->d_items);
        const int cap = std::max<int>((int)items.size(), 1024);
        CK(cudaMalloc(&b->d_items, sizeof(WorkItem) * cap));
        b->items_cap = cap;
        b->drop_graph();
    }
    if (nj) CK(cudaMemcpyAsync(b->d_jobs, jd.data(), sizeof(JobDesc) * nj, cudaMemcpyHostToDevice, b->stream));
    if (!items.empty())
        CK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, b->stream));
    BatchMeta m{};
    m.screen_ctas = b->num_sms * b->shape.ctas_per_sm;
    m.njobs = nj;
    m.n_items = (int32_t)items.size();
    m.total_feat = fbase;
    m.total_ublocks = ubase;
    CK(cudaMemcpyAsync(b->d_meta, &m, sizeof m, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    b->dirty = false;
    return VJB_OK;
}

// Part 1 of a batched round (begin + search), part 2 (shortlist, re-scan,
// update), or 0 for both.
int batch_enqueue_round(vjb_batch *b, int part) {
    const int g = b->num_sms;
    if (part != 2) {
        CK(launch_bbegin(b->d_jobs, b->d_meta, b->stream));
        CK(launch_bscreen(b->maps, b->d_jobs, b->d_items, b->d_meta, kBatchMaxWords, b->shape,
                          b->rows_per_warp, g * b->shape.ctas_per_sm, b->stream));
    }
    if (part != 1) {
        CK(launch_bshortlist(b->d_jobs, b->d_meta, g * 4, b->stream));
        CK(launch_brescan(b->d_jobs, b->d_meta, std::min(g, 128), b->stream));
        CK(launch_bupdate_a(b->d_jobs, b->d_meta, g * 4, b->stream));
        CK(launch_bupdate_b(b->d_jobs, b->d_meta, g * 4, b->stream));
    }
    return VJB_OK;
}

int batch_take_events(vjb_batch *b, EventTriple &t) {
    if (b->ev_free.empty()) {
        for (auto &e : t) CK(cudaEventCreate(&e));
    } else {
        t = b->ev_free.back();
        b->ev_free.pop_back();
    }
    return VJB_OK;
}

// Fold finished event triples into the batch's timing totals (stream idle).
int batch_collect_timing(vjb_batch *b) {
    for (auto &t : b->ev_pending) {
        float s = 0.f, r = 0.f;
        CK(cudaEventElapsedTime(&s, t[0], t[1]));
        CK(cudaEventElapsedTime(&r, t[0], t[2]));
        vjb_timing &a = b->tacc;
        a.search_ms_min = a.rounds ? std::min(a.search_ms_min, (double)s) : s;
        a.search_ms_max = a.rounds ? std::max(a.search_ms_max, (double)s) : s;
        a.rounds += 1;
        a.search_ms_total += s;
        a.round_ms_total += r;
        b->ev_free.push_back(t);
    }
    b->ev_pending.clear();
    return VJB_OK;
}

int batch_capture(vjb_batch *b, int part, cudaGraph_t *graph, cudaGraphExec_t *exec) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_enqueue_round(b, part);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(VJB_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        *exec = nullptr;
        return fail(VJB_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    }
    *graph = g;
    return VJB_OK;
}

int batch_ensure_graph(vjb_batch *b) {
    if (b->gexec && b->graph_timed == b->timing) return VJB_OK;
    b->drop_graph();
    int rc = batch_capture(b, b->timing ? 1 : 0, &b->graph, &b->gexec);
    if (rc == VJB_OK && b->timing) rc = batch_capture(b, 2, &b->graph2, &b->gexec2);
    if (rc) {
        b->drop_graph();
        return rc;
    }
    b->graph_timed = b->timing;
    return VJB_OK;
}

bool batch_shape_ok(const vjb_batch *b, const SearchShape &s) {
    return s.warps >= 1 && s.warps <= screen_max_warps(s.unroll) && s.stages >= 1 && s.stages <= 8 &&
           s.ctas_per_sm == 1 && s.unroll >= 1 && s.unroll <= 4 && s.box_lines >= 4 &&
           s.box_lines <= kBoxLinesMax && s.box_lines % 4 == 0 &&
           bscreen_smem_bytes(s, kBatchMaxWords) + 256 <= (size_t)b->max_smem;
}

// Largest number of rounds a job of the batch still wants (0 when all are
// done); grows the jobs' stump records to their targets.
int batch_rounds_wanted(vjb_batch *b, int *want, std::vector<RoundState> *states = nullptr) {
    *want = 0;
    std::vector<RoundState> st(b->slots.size());
    for (size_t k = 0; k < st.size(); ++k)
        CK(cudaMemcpyAsync(&st[k], b->slots[k].ctx->d_rs, sizeof(RoundState), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k < st.size(); ++k) {
        BatchSlot &s = b->slots[k];
        if (st[k].status == VJB_OK && !st[k].flags) *want = std::max(*want, s.round_target - st[k].rounds);
        if (s.round_target > s.ctx->stump_cap) {
            const int rc = ensure_stump_cap(s.ctx, s.round_target);
            if (rc) return rc;
            b->dirty = true;
        }
    }
    if (states) states->swap(st);
    return VJB_OK;
}

// R batched rounds (graph replays); `ms` (may be NULL) receives their device time.
int batch_run(vjb_batch *b, int R, float *ms) {
    int rc = batch_sync(b);
    if (rc) return rc;
    if (R > 0 && !b->slots.empty()) {
        rc = batch_ensure_graph(b);
        if (rc) return rc;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ms) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, b->stream));
        }
        for (int r = 0; r < R; ++r) {
            if (b->timing) {
                EventTriple ev;
                rc = batch_take_events(b, ev);
                if (rc) return rc;
                CK(cudaEventRecord(ev[0], b->stream));
                CK(cudaGraphLaunch(b->gexec, b->stream));
                CK(cudaEventRecord(ev[1], b->stream));
                CK(cudaGraphLaunch(b->gexec2, b->stream));
                CK(cudaEventRecord(ev[2], b->stream));
                b->ev_pending.push_back(ev);
            } else {
                CK(cudaGraphLaunch(b->gexec, b->stream));
            }
            b->launches += 6;
        }
        if (ms) {
            CK(cudaEventRecord(e1, b->stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(ms, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
    } else if (ms) {
        *ms = 0.f;
    }
    CK(cudaStreamSynchronize(b->stream));
    BatchMeta m;
    CK(cudaMemcpy(&m, b->d_meta, sizeof m, cudaMemcpyDeviceToHost));
    if (m.flags) return fail(VJB_EDEVICE, "batched kernel error flags 0x%x", m.flags);
    return VJB_OK;
}

}  // namespace

extern "C" {

int vjb_batch_create(vjb_batch **out, int device, void *cuda_stream, int64_t table_budget_bytes) {
    g_err[0] = 0;
    if (!out) return fail(VJB_EINVAL, "out is NULL");
    *out = nullptr;
    if (table_budget_bytes < kLineBytes) return fail(VJB_EINVAL, "table budget below one line");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(VJB_EINVAL, "device %d outside [0, %d)", device, ndev);
    CK(cudaSetDevice(device));
    vjb_batch *b = new vjb_batch();
    b->device = device;
    auto bail = [&](int rc) {
        if (b->arena) cudaFree(b->arena);
        if (b->d_jobs) cudaFree(b->d_jobs);
        if (b->d_meta) cudaFree(b->d_meta);
        if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
        delete b;
        return rc;
    };
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return bail(fail(VJB_ECUDA, "device query failed"));
    b->num_sms = prop.multiProcessorCount;
    b->max_smem = (int)prop.sharedMemPerBlockOptin;
    if (set_bscreen_smem_limit(b->max_smem - 256) != cudaSuccess || set_screen_smem_limit(b->max_smem) != cudaSuccess)
        return bail(fail(VJB_ECUDA, "shared-memory limit of the search kernels"));
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(VJB_ECUDA, "stream creation failed"));
        b->own_stream = true;
    }
    // the search addresses arena lines with 32-bit coordinates
    b->arena_lines = std::min<int64_t>(table_budget_bytes / kLineBytes, INT32_MAX);
    cudaError_t e = cudaMalloc(&b->arena, (size_t)b->arena_lines * kLineBytes);
    if (e != cudaSuccess) return bail(fail(VJB_ENOMEM, "table arena of %lld bytes: %s", (long long)table_budget_bytes, cudaGetErrorString(e)));
    if (cudaMalloc(&b->d_jobs, sizeof(JobDesc) * kMaxBatchJobs) != cudaSuccess ||
        cudaMalloc(&b->d_meta, sizeof(BatchMeta)) != cudaSuccess)
        return bail(fail(VJB_ENOMEM, "batch job table"));
    cudaMemset(b->d_meta, 0, sizeof(BatchMeta));
    const int rc = batch_encode_maps(b);
    if (rc) return bail(rc);
    b->free_list.emplace_back(0, b->arena_lines);
    *out = b;
    return VJB_OK;
}

void vjb_batch_destroy(vjb_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->drop_graph();
    for (auto &s : b->slots) vjb_destroy(s.ctx);
    dfree(b->arena);
    dfree(b->d_jobs);
    dfree(b->d_meta);
    dfree(b->d_items);
    for (auto &t : b->ev_pending) b->ev_free.push_back(t);
    for (auto &t : b->ev_free)
        for (auto e : t) cudaEventDestroy(e);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int vjb_batch_set_timing(vjb_batch *b, int32_t enable) {
    g_err[0] = 0;
    if (!b) return fail(VJB_EINVAL, "batch is NULL");
    CK(cudaSetDevice(b->device));
    CK(cudaStreamSynchronize(b->stream));
    for (auto &t : b->ev_pending) b->ev_free.push_back(t);
    b->ev_pending.clear();
    b->tacc = vjb_timing{};
    b->timing = enable != 0;
    return VJB_OK;
}

int vjb_batch_get_timing(vjb_batch *b, vjb_timing *out) {
    g_err[0] = 0;
    if (!b || !out) return fail(VJB_EINVAL, "NULL argument");
    CK(cudaSetDevice(b->device));
    CK(cudaStreamSynchronize(b->stream));
    const int rc = batch_collect_timing(b);
    if (rc) return rc;
    *out = b->tacc;
    return VJB_OK;
}

int vjb_batch_table_bytes(int32_t n, int32_t h, int32_t w, int64_t *bytes) {
    g_err[0] = 0;
    if (!bytes) return fail(VJB_EINVAL, "bytes is NULL");
    if (n < 2 || n > VJB_MAX_SAMPLES || h < 1 || w < 1 || h > VJB_MAX_WINDOW || w > VJB_MAX_WINDOW)
        return fail(VJB_EINVAL, "sizes outside the limits");
    *bytes = table_lines(n, h, w) * kLineBytes;
    return VJB_OK;
}

int vjb_batch_add_job(vjb_batch *b, const uint8_t *pixels, const uint8_t *labels, int32_t n, int32_t h,
                      int32_t w, int32_t rounds, int32_t *job_id) {
    g_err[0] = 0;
    if (!b || !job_id) return fail(VJB_EINVAL, "NULL argument");
    if ((int)b->slots.size() >= kMaxBatchJobs) return fail(VJB_EFULL, "batch holds %d jobs already", kMaxBatchJobs);
    if (rounds < 0) return fail(VJB_EINVAL, "rounds < 0");
    if (n < 2 || n > VJB_MAX_SAMPLES || h < 1 || w < 1 || h > VJB_MAX_WINDOW || w > VJB_MAX_WINDOW)
        return fail(VJB_EINVAL, "sizes outside the limits");
    CK(cudaSetDevice(b->device));
    const int64_t need = table_lines(n, h, w);
    int64_t first = 0;
    if (need == 0) return fail(VJB_EINVAL, "window %dx%d has no feature", w, h);
    if (!arena_take(b, need, &first))
        return fail(VJB_EFULL, "table of %lld bytes does not fit the remaining budget", (long long)(need * kLineBytes));
    vjb_ctx *c = nullptr;
    int rc = vjb_create(&c, b->device, b->stream);
    if (rc == VJB_OK) rc = vjb_load_windows(c, pixels, labels, n, h, w);
    if (rc == VJB_OK && make_layout(n, true).words > kBatchMaxWords) rc = fail(VJB_EINVAL, "n too large for a batch");
    if (rc == VJB_OK) {
        c->rows_external = true;
        c->d_rows = b->arena + first * kLineElems;
        c->line_base = first;
        rc = vjb_build_integral(c);
    }
    int64_t cnt = 0;
    if (rc == VJB_OK) rc = vjb_enumerate_haar(c, &cnt, nullptr);
    if (rc != VJB_OK) {
        const std::string msg = vjb_last_error();
        if (c) vjb_destroy(c);
        arena_give(b, first, need);
        return fail(rc, "%s", msg.c_str());
    }
    BatchSlot s;
    s.ctx = c;
    s.id = b->next_id++;
    s.line_base = first;
    s.line_count = need;
    s.round_target = rounds;
    b->slots.push_back(s);
    b->dirty = true;
    *job_id = s.id;
    return VJB_OK;
}

int vjb_batch_remove_job(vjb_batch *b, int32_t job_id) {
    g_err[0] = 0;
    if (!b) return fail(VJB_EINVAL, "batch is NULL");
    CK(cudaSetDevice(b->device));
    for (size_t k = 0; k < b->slots.size(); ++k)
        if (b->slots[k].id == job_id) {
            CK(cudaStreamSynchronize(b->stream));
            vjb_destroy(b->slots[k].ctx);
            arena_give(b, b->slots[k].line_base, b->slots[k].line_count);
            b->slots.erase(b->slots.begin() + (long)k);
            b->dirty = true;
            return VJB_OK;
        }
    return fail(VJB_EINVAL, "no job %d in the batch", job_id);
}

int vjb_batch_train(vjb_batch *b, int32_t max_rounds, int32_t *rounds_run) {
    g_err[0] = 0;
    if (!b || max_rounds < 0) return fail(VJB_EINVAL, "bad argument");
    CK(cudaSetDevice(b->device));
    int want = 0;
    int rc = batch_rounds_wanted(b, &want);
    if (rc) return rc;
    const int R = std::min(want, max_rounds);
    rc = batch_run(b, R, nullptr);
    if (rounds_run) *rounds_run = rc ? 0 : R;
    return rc;
}

int vjb_batch_autotune(vjb_batch *b, int32_t trial_rounds, int32_t *rounds_run, vjb_batch_trial *trials,
                       int32_t max_trials, int32_t *n_trials) {
    g_err[0] = 0;
    if (!b || trial_rounds < 1) return fail(VJB_EINVAL, "bad argument");
    CK(cudaSetDevice(b->device));
    // (warps, stages, unroll, features per warp and work item); results do not
    // depend on the shape, so every trial round is a real round of the jobs
    // (rows: VJB_BATCH_INTERLEAVED / VJB_BATCH_PARTITIONED schedules, else the work queue)
    constexpr int IL = VJB_BATCH_INTERLEAVED;
    constexpr int PT = VJB_BATCH_PARTITIONED;
    static const int kTries[][5] = {{16, 2, 3, 24, IL}, {16, 2, 3, 24, PT}, {16, 2, 3, 24, 16}, {16, 2, 3, 24, 32},
                                    {12, 2, 4, 32, IL}, {12, 2, 4, 32, PT}, {12, 2, 4, 32, 32}, {16, 2, 3, 24, 64}};
    const SearchShape keep = b->shape;
    const int keep_rpw = b->rows_per_warp;
    double best = -1.0;
    SearchShape best_s = keep;
    int best_rpw = keep_rpw, ran = 0, ntr = 0;
    for (const auto &t : kTries) {
        int want = 0;
        int rc = batch_rounds_wanted(b, &want);
        if (rc) return rc;
        if (want < trial_rounds + 1) break;
        const SearchShape s{t[0], t[1], 1, t[2], t[3]};
        if (!batch_shape_ok(b, s)) continue;
        b->shape = s;
        b->rows_per_warp = t[4];
        b->dirty = true;
        b->drop_graph();
        rc = batch_encode_maps(b);
        if (rc) return rc;
        float ms = 0.f;
        rc = batch_run(b, 1, nullptr);  // first round of a shape: graph set-up, not timed
        if (rc == VJB_OK) rc = batch_run(b, trial_rounds, &ms);
        if (rc) return rc;
        ran += 1 + trial_rounds;
        if (trials && ntr < max_trials)
            trials[ntr] = vjb_batch_trial{s.warps, s.stages, s.unroll, t[4], s.box_lines, ms / (float)trial_rounds};
        ++ntr;
        if (best < 0.0 || ms < best) {
            best = ms;
            best_s = s;
            best_rpw = t[4];
        }
    }
    b->shape = best_s;
    b->rows_per_warp = best_rpw;
    b->dirty = true;
    b->drop_graph();
    const int rce = batch_encode_maps(b);
    if (rce) return rce;
    if (rounds_run) *rounds_run = ran;
    if (n_trials) *n_trials = std::min(ntr, std::max(max_trials, 0));
    return VJB_OK;
}

int vjb_batch_job_state(vjb_batch *b, int32_t job_id, int32_t *rounds_done, int32_t *status) {
    g_err[0] = 0;
    if (!b) return fail(VJB_EINVAL, "batch is NULL");
    BatchSlot *s = find_slot(b, job_id);
    if (!s) return fail(VJB_EINVAL, "no job %d in the batch", job_id);
    vjb_info info;
    int rc = vjb_get_info(s->ctx, &info);
    if (rc) return rc;
    if (rounds_done) *rounds_done = info.rounds_done;
    if (status) *status = info.device_flags ? VJB_EDEVICE : info.status;
    return VJB_OK;
}

int vjb_batch_get_stumps(vjb_batch *b, int32_t job_id, int32_t first, int32_t count, vjb_stump *out) {
    g_err[0] = 0;
    if (!b || !out) return fail(VJB_EINVAL, "NULL argument");
    BatchSlot *s = find_slot(b, job_id);
    if (!s) return fail(VJB_EINVAL, "no job %d in the batch", job_id);
    vjb_info info;
    int rc = vjb_get_info(s->ctx, &info);
    if (rc) return rc;
    if (first < 0 || count < 0 || first + count > info.rounds_done)
        return fail(VJB_EINVAL, "stumps [%d, %d) outside the %d kept", first, first + count, info.rounds_done);
    if (count == 0) return VJB_OK;
    CK(cudaSetDevice(b->device));
    CK(cudaMemcpy(out, s->ctx->d_stumps + first, sizeof(vjb_stump) * count, cudaMemcpyDeviceToHost));
    return VJB_OK;
}

int vjb_batch_get_weights(vjb_batch *b, int32_t job_id, float *out) {
    g_err[0] = 0;
    if (!b) return fail(VJB_EINVAL, "batch is NULL");
    BatchSlot *s = find_slot(b, job_id);
    if (!s) return fail(VJB_EINVAL, "no job %d in the batch", job_id);
    return vjb_get_weights(s->ctx, out);
}

int vjb_batch_set_search_shape(vjb_batch *b, const vjb_search_shape *in, int32_t rows_per_warp) {
    g_err[0] = 0;
    if (!b) return fail(VJB_EINVAL, "batch is NULL");
    SearchShape s = b->shape;
    if (in) {
        if (in->warps) s.warps = in->warps;
        if (in->stages) s.stages = in->stages;
        if (in->unroll) s.unroll = in->unroll;
        if (in->ctas_per_sm) s.ctas_per_sm = in->ctas_per_sm;
        if (in->box_lines) s.box_lines = in->box_lines;
    }
    if (!batch_shape_ok(b, s) || rows_per_warp < VJB_BATCH_INTERLEAVED || rows_per_warp > 4096)
        return fail(VJB_EINVAL, "batch search shape (%d warps, %d stages, unroll %d, %d rows per warp) not usable",
                    s.warps, s.stages, s.unroll, rows_per_warp);
    b->shape = s;
    if (rows_per_warp) b->rows_per_warp = rows_per_warp;
    b->dirty = true;
    b->drop_graph();
    return batch_encode_maps(b);
}

int vjb_batch_get_info(vjb_batch *b, vjb_batch_info *out) {
    g_err[0] = 0;
    if (!b || !out) return fail(VJB_EINVAL, "NULL argument");
    memset(out, 0, sizeof *out);
    out->jobs = (int32_t)b->slots.size();
    out->warps = b->shape.warps;
    out->stages = b->shape.stages;
    out->unroll = b->shape.unroll;
    out->box_lines = b->shape.box_lines;
    out->rows_per_warp = b->rows_per_warp;
    out->budget_bytes = b->arena_lines * kLineBytes;
    int64_t free_lines = 0, largest = 0;
    for (const auto &fr : b->free_list) {
        free_lines += fr.second;
        largest = std::max(largest, fr.second);
    }
    out->free_bytes = free_lines * kLineBytes;
    out->largest_free_bytes = largest * kLineBytes;
    double bytes = 0.0;
    for (const auto &s : b->slots) bytes += 2.0 * (double)s.ctx->nfeat * s.ctx->n;
    out->search_bytes = bytes;
    out->launches = b->launches;
    return VJB_OK;
}

}  // extern "C"

// ---- serving: continuous batching of training requests ---------------------------------
// A server keeps one batch on the device.  Requests wait in arrival order
// until their sorted table fits the free part of the batch's arena (and a job
// slot is free); a worker thread then prepares each admitted request on its
// low-priority stream -- windows, integral images, features, sorted table
// written into the arena -- while the main thread keeps running batched
// rounds for the jobs already training, on a high-priority stream.  A prepared request joins the batch at the next round;
// a job that reaches its round count (or stops early) leaves it, its stumps
// and weights are copied to the host and its table space is freed for the
// requests still waiting.

namespace {

enum { kReqQueued = 0, kReqPreparing = 1, kReqTraining = 2, kReqDone = 3, kReqFailed = 4 };
constexpr int kMaxBypass = 8;  // later requests may overtake a waiting one this often

struct ServerReq {
    int64_t id = 0;
    std::vector<uint8_t> px, y;
    int32_t n = 0, h = 0, w = 0, rounds = 0;
    int state = kReqQueued;
    int status = VJB_OK;
    int64_t line_first = 0, line_count = 0;
    vjb_ctx *ctx = nullptr;
    int32_t slot = -1;
    double t_submit = 0, t_admit = -1, t_ready = -1, t_done = -1;
    double round_ms_sum = 0;
    int32_t rounds_timed = 0;
    int bypassed = 0;
    std::vector<vjb_stump> stumps;
    std::vector<float> weights;
    std::string error;
};

}  // namespace

struct vjb_server {
    vjb_batch *b = nullptr;
    int device = 0;
    int max_jobs = 0;
    std::chrono::steady_clock::time_point t0;
    std::map<int64_t, std::unique_ptr<ServerReq>> reqs;
    std::deque<ServerReq *> queue;  // waiting for admission, in arrival order
    int64_t next_id = 1;
    // worker thread and what it shares with the main thread (under mu)
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerReq *> to_prepare;
    std::vector<ServerReq *> prepared;
    std::vector<vjb_ctx *> to_destroy;  // retired jobs' contexts: their cudaFree waits for the device
    bool stop = false;
    // rounds run on a high-priority stream, preparation on a low-priority one,
    // so that a round's CTAs go ahead of a running sort's as SMs free up
    cudaStream_t hi = nullptr, lo = nullptr;
    int preparing = 0;  // admitted, not yet collected (main thread only)
    std::vector<float> round_ms;
    std::vector<int32_t> round_jobs;
    int64_t job_rounds = 0;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Worker side: build a request's context with its table in the arena.
int server_prepare(vjb_server *s, ServerReq *r) {
    vjb_ctx *c = nullptr;
    int rc = vjb_create(&c, s->device, s->lo);
    if (rc == VJB_OK) rc = vjb_load_windows(c, r->px.data(), r->y.data(), r->n, r->h, r->w);
    if (rc == VJB_OK) {
        c->rows_external = true;
        c->d_rows = s->b->arena + r->line_first * kLineElems;
        c->line_base = r->line_first;
        rc = vjb_build_integral(c);
    }
    int64_t cnt = 0;
    if (rc == VJB_OK) rc = vjb_enumerate_haar(c, &cnt, nullptr);
    if (rc == VJB_OK) rc = ensure_stump_cap(c, std::max(r->rounds, 1));
    if (rc != VJB_OK) {
        r->error = vjb_last_error();
        if (c) vjb_destroy(c);
        return rc;
    }
    r->ctx = c;
    return VJB_OK;
}

void server_worker(vjb_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        ServerReq *r = nullptr;
        std::vector<vjb_ctx *> dead;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->to_prepare.empty() || !s->to_destroy.empty(); });
            dead.swap(s->to_destroy);
            if (!s->to_prepare.empty()) {
                r = s->to_prepare.front();
                s->to_prepare.pop_front();
            }
        }
        // freeing device memory waits for the whole device: here, not on the
        // thread that runs the rounds
        for (vjb_ctx *c : dead) vjb_destroy(c);
        if (!r) {
            if (s->stop) return;  // stop requested and nothing left
            continue;
        }
        const int rc = s->stop ? VJB_ESTATE : server_prepare(s, r);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (rc != VJB_OK) {
                r->status = rc;
                if (r->error.empty()) r->error = "server stopped before the request was prepared";
            }
            s->prepared.push_back(r);
        }
        s->cv_done.notify_all();
    }
}

// Main side: move prepared requests into the batch (or to failed).
void server_collect(vjb_server *s, bool wait) {
    std::vector<ServerReq *> got;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (wait && s->prepared.empty() && s->preparing > 0)
            s->cv_done.wait_for(lk, std::chrono::milliseconds(5), [&] { return !s->prepared.empty(); });
        got.swap(s->prepared);
    }
    for (ServerReq *r : got) {
        s->preparing -= 1;
        r->t_ready = s->now_ms();
        if (r->status != VJB_OK) {
            arena_give(s->b, r->line_first, r->line_count);
            r->state = kReqFailed;
            r->t_done = r->t_ready;
            continue;
        }
        BatchSlot sl;
        sl.ctx = r->ctx;
        sl.id = s->b->next_id++;
        sl.line_base = r->line_first;
        sl.line_count = r->line_count;
        sl.round_target = r->rounds;
        s->b->slots.push_back(sl);
        s->b->dirty = true;
        r->slot = sl.id;
        r->state = kReqTraining;
    }
}

ServerReq *req_of_slot(vjb_server *s, int32_t slot) {
    for (auto &kv : s->reqs)
        if (kv.second->state == kReqTraining && kv.second->slot == slot) return kv.second.get();
    return nullptr;
}

// Jobs that reached their round count or stopped leave the batch.
int server_retire(vjb_server *s, const std::vector<RoundState> &st) {
    vjb_batch *b = s->b;
    std::vector<BatchSlot> keep;
    for (size_t k = 0; k < b->slots.size(); ++k) {
        const BatchSlot &sl = b->slots[k];
        const RoundState &rs = st[k];
        const bool done = rs.flags || rs.status != VJB_OK || rs.rounds >= sl.round_target;
        if (!done) {
            keep.push_back(sl);
            continue;
        }
        ServerReq *r = req_of_slot(s, sl.id);
        if (r) {
            r->status = rs.flags ? VJB_EDEVICE : rs.status;
            r->stumps.resize((size_t)rs.rounds);
            if (rs.rounds) CK(cudaMemcpy(r->stumps.data(), sl.ctx->d_stumps, sizeof(vjb_stump) * rs.rounds, cudaMemcpyDeviceToHost));
            r->weights.resize((size_t)r->n);
            CK(cudaMemcpy(r->weights.data(), sl.ctx->d_w, sizeof(float) * r->n, cudaMemcpyDeviceToHost));
            r->state = kReqDone;
            r->t_done = s->now_ms();
            r->ctx = nullptr;
            r->px.clear();
            r->px.shrink_to_fit();
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->to_destroy.push_back(sl.ctx);
        }
        s->cv_work.notify_all();
        arena_give(b, sl.line_base, sl.line_count);
        b->dirty = true;
    }
    b->slots.swap(keep);
    return VJB_OK;
}

// Waiting requests whose tables fit the free arena are handed to the worker,
// in arrival order; later ones may overtake one that does not fit, at most
// kMaxBypass times, so that a large table is not starved.
void server_admit(vjb_server *s) {
    int active = (int)s->b->slots.size() + s->preparing;
    bool blocked = false;
    for (auto it = s->queue.begin(); it != s->queue.end() && active < s->max_jobs;) {
        ServerReq *r = *it;
        int64_t first = 0;
        if (arena_take(s->b, r->line_count, &first)) {
            r->line_first = first;
            r->state = kReqPreparing;
            r->t_admit = s->now_ms();
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->to_prepare.push_back(r);
            }
            s->cv_work.notify_one();
            s->preparing += 1;
            active += 1;
            it = s->queue.erase(it);
            // the requests this one overtook
            for (auto jt = s->queue.begin(); jt != it; ++jt) (*jt)->bypassed += 1;
        } else {
            if (r->bypassed >= kMaxBypass) blocked = true;
            if (blocked) break;
            ++it;
        }
    }
}

}  // namespace

extern "C" {

int vjb_server_create(vjb_server **out, int device, int64_t table_budget_bytes, int32_t max_jobs) {
    g_err[0] = 0;
    if (!out) return fail(VJB_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_jobs < 1 || max_jobs > kMaxBatchJobs)
        return fail(VJB_EINVAL, "max_jobs = %d outside [1, %d]", max_jobs, kMaxBatchJobs);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(VJB_EINVAL, "device %d out of range", device);
    CK(cudaSetDevice(device));
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    cudaStream_t hi = nullptr, lo = nullptr;
    CK(cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, greatest));
    if (cudaStreamCreateWithPriority(&lo, cudaStreamNonBlocking, least) != cudaSuccess) {
        cudaStreamDestroy(hi);
        return fail(VJB_ECUDA, "stream creation failed");
    }
    vjb_batch *b = nullptr;
    int rc = vjb_batch_create(&b, device, hi, table_budget_bytes);
    if (rc) {
        cudaStreamDestroy(hi);
        cudaStreamDestroy(lo);
        return rc;
    }
    vjb_server *s = new vjb_server();
    s->b = b;
    s->hi = hi;
    s->lo = lo;
    s->device = device;
    s->max_jobs = max_jobs;
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread(server_worker, s);
    *out = s;
    return VJB_OK;
}

void vjb_server_destroy(vjb_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (ServerReq *r : s->prepared)
        if (r->ctx) vjb_destroy(r->ctx);
    for (vjb_ctx *c : s->to_destroy) vjb_destroy(c);
    vjb_batch_destroy(s->b);  // destroys the contexts of the training jobs
    cudaStreamDestroy(s->hi);
    cudaStreamDestroy(s->lo);
    delete s;
}

int vjb_server_submit(vjb_server *s, const uint8_t *pixels, const uint8_t *labels, int32_t n, int32_t h,
                      int32_t w, int32_t rounds, int64_t *request_id) {
    g_err[0] = 0;
    if (!s || !pixels || !labels || !request_id) return fail(VJB_EINVAL, "NULL argument");
    if (rounds < 1) return fail(VJB_EINVAL, "rounds = %d < 1", rounds);
    if (n < 2 || n > VJB_MAX_SAMPLES || h < 1 || w < 1 || h > VJB_MAX_WINDOW || w > VJB_MAX_WINDOW)
        return fail(VJB_EINVAL, "sizes outside the limits");
    int rc = validate_labels(labels, n);
    if (rc) return rc;
    const int64_t need = table_lines(n, h, w);
    if (need == 0) return fail(VJB_EINVAL, "window %dx%d has no feature", w, h);
    if (need > s->b->arena_lines)
        return fail(VJB_EFULL, "table of %lld bytes exceeds the whole budget of %lld", (long long)(need * kLineBytes),
                    (long long)(s->b->arena_lines * kLineBytes));
    auto r = std::make_unique<ServerReq>();
    r->id = s->next_id++;
    r->px.assign(pixels, pixels + (size_t)n * h * w);
    r->y.assign(labels, labels + n);
    r->n = n;
    r->h = h;
    r->w = w;
    r->rounds = rounds;
    r->line_count = need;
    r->t_submit = s->now_ms();
    s->queue.push_back(r.get());
    *request_id = r->id;
    s->reqs[r->id] = std::move(r);
    return VJB_OK;
}

int vjb_server_step(vjb_server *s, int32_t max_rounds, int32_t *rounds_run) {
    g_err[0] = 0;
    if (!s || max_rounds < 0) return fail(VJB_EINVAL, "bad argument");
    if (rounds_run) *rounds_run = 0;
    CK(cudaSetDevice(s->device));
    vjb_batch *b = s->b;
    server_admit(s);
    server_collect(s, b->slots.empty());
    int ran = 0;
    for (; ran < max_rounds; ++ran) {
        int want = 0;
        std::vector<RoundState> st;
        int rc = batch_rounds_wanted(b, &want, &st);
        if (rc) return rc;
        rc = server_retire(s, st);
        if (rc) return rc;
        if (want == 0) break;
        int in_round = 0;
        for (size_t k = 0; k < st.size(); ++k)
            if (st[k].status == VJB_OK && !st[k].flags && st[k].rounds < b->slots[k].round_target) ++in_round;
        std::vector<ServerReq *> members;
        for (auto &sl : b->slots) {
            ServerReq *r = req_of_slot(s, sl.id);
            if (r) members.push_back(r);
        }
        float ms = 0.f;
        rc = batch_run(b, 1, &ms);
        if (rc) return rc;
        s->round_ms.push_back(ms);
        s->round_jobs.push_back(in_round);
        s->job_rounds += in_round;
        for (ServerReq *r : members) {
            r->round_ms_sum += ms;
            r->rounds_timed += 1;
        }
        server_admit(s);
        server_collect(s, false);
    }
    // retire what the last round finished
    {
        int want = 0;
        std::vector<RoundState> st;
        int rc = batch_rounds_wanted(b, &want, &st);
        if (rc) return rc;
        rc = server_retire(s, st);
        if (rc) return rc;
        server_admit(s);
    }
    if (rounds_run) *rounds_run = ran;
    return VJB_OK;
}

int vjb_server_request(vjb_server *s, int64_t request_id, vjb_request_info *out) {
    g_err[0] = 0;
    if (!s || !out) return fail(VJB_EINVAL, "NULL argument");
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(VJB_EINVAL, "no request %lld", (long long)request_id);
    const ServerReq &r = *it->second;
    memset(out, 0, sizeof *out);
    out->request_id = r.id;
    out->state = r.state;
    out->status = r.status;
    out->rounds_done = (int32_t)r.stumps.size();
    out->rounds_target = r.rounds;
    out->n = r.n;
    out->h = r.h;
    out->w = r.w;
    out->rounds_timed = r.rounds_timed;
    out->table_bytes = r.line_count * kLineBytes;
    out->t_submit_ms = r.t_submit;
    out->t_admit_ms = r.t_admit;
    out->t_ready_ms = r.t_ready;
    out->t_done_ms = r.t_done;
    out->round_ms_sum = r.round_ms_sum;
    if (r.state == kReqTraining) {
        RoundState rs;
        CK(cudaMemcpy(&rs, r.ctx->d_rs, sizeof rs, cudaMemcpyDeviceToHost));
        out->rounds_done = rs.rounds;
    }
    if (r.state == kReqFailed) fail(r.status, "%s", r.error.c_str());
    return VJB_OK;
}

int vjb_server_result(vjb_server *s, int64_t request_id, vjb_stump *stumps, int32_t cap, float *weights) {
    g_err[0] = 0;
    if (!s) return fail(VJB_EINVAL, "server is NULL");
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(VJB_EINVAL, "no request %lld", (long long)request_id);
    const ServerReq &r = *it->second;
    if (r.state == kReqFailed) return fail(r.status, "%s", r.error.c_str());
    if (r.state != kReqDone) return fail(VJB_ESTATE, "request %lld is not finished", (long long)request_id);
    if (stumps) {
        if (cap < (int32_t)r.stumps.size()) return fail(VJB_EINVAL, "cap %d < %zu stumps", cap, r.stumps.size());
        if (!r.stumps.empty()) memcpy(stumps, r.stumps.data(), sizeof(vjb_stump) * r.stumps.size());
    }
    if (weights) memcpy(weights, r.weights.data(), sizeof(float) * r.weights.size());
    return r.status;
}

int vjb_server_release(vjb_server *s, int64_t request_id) {
    g_err[0] = 0;
    if (!s) return fail(VJB_EINVAL, "server is NULL");
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(VJB_EINVAL, "no request %lld", (long long)request_id);
    if (it->second->state != kReqDone && it->second->state != kReqFailed)
        return fail(VJB_ESTATE, "request %lld is not finished", (long long)request_id);
    s->reqs.erase(it);
    return VJB_OK;
}

int vjb_server_stats(vjb_server *s, vjb_server_summary *out) {
    g_err[0] = 0;
    if (!s || !out) return fail(VJB_EINVAL, "NULL argument");
    memset(out, 0, sizeof *out);
    for (auto &kv : s->reqs) {
        switch (kv.second->state) {
        case kReqQueued: out->queued += 1; break;
        case kReqPreparing: out->preparing += 1; break;
        case kReqTraining: out->training += 1; break;
        case kReqDone: out->done += 1; break;
        default: out->failed += 1;
        }
    }
    out->rounds = (int64_t)s->round_ms.size();
    out->job_rounds = s->job_rounds;
    int64_t free_lines = 0;
    for (const auto &fr : s->b->free_list) free_lines += fr.second;
    out->budget_bytes = s->b->arena_lines * kLineBytes;
    out->free_bytes = free_lines * kLineBytes;
    double busy = 0.0;
    for (float m : s->round_ms) busy += m;
    out->round_ms_total = busy;
    out->clock_ms = s->now_ms();
    return VJB_OK;
}

int vjb_server_round_times(vjb_server *s, int64_t first, int32_t count, float *ms, int32_t *jobs) {
    g_err[0] = 0;
    if (!s) return fail(VJB_EINVAL, "server is NULL");
    if (first < 0 || count < 0 || first + count > (int64_t)s->round_ms.size())
        return fail(VJB_EINVAL, "rounds [%lld, %lld) outside the %zu run", (long long)first,
                    (long long)(first + count), s->round_ms.size());
    for (int32_t k = 0; k < count; ++k) {
        if (ms) ms[k] = s->round_ms[(size_t)(first + k)];
        if (jobs) jobs[k] = s->round_jobs[(size_t)(first + k)];
    }
    return VJB_OK;
}

}  // extern "C"
