// C ABI of the library (declared in include/vjb.h): context ownership,
// argument checking, the order of the training steps, and the launch sequence
// of a boosting round (search -> refine -> finalize), replayed as a CUDA graph
// by vjb_train_strong.
#include "vjb_host.h"

using namespace vjb;

namespace vjb {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace vjb


// Context internals (external: the batch and serving code reuses a few).
namespace vjb {

int set_dev(vjb_ctx *c) {
    CK(cudaSetDevice(c->device));
    return VJB_OK;
}

int32_t *flags_ptr(vjb_ctx *c) {
    return reinterpret_cast<int32_t *>(reinterpret_cast<char *>(c->d_rs) + offsetof(RoundState, flags));
}

// Canonical enumeration (types 3H, 3V, 2H, 2V, 4; then width, height, y, x).
void enumerate_host(int W, int H, std::vector<vjb_feature> &out) {
    static const int bw[5] = {3, 1, 2, 1, 2}, bh[5] = {1, 3, 1, 2, 2};
    out.clear();
    for (int t = 0; t < 5; ++t)
        for (int fw = bw[t]; fw <= W; fw += bw[t])
            for (int fh = bh[t]; fh <= H; fh += bh[t])
                for (int y = 0; y + fh <= H; ++y)
                    for (int x = 0; x + fw <= W; ++x)
                        out.push_back(vjb_feature{(uint8_t)t, (uint8_t)x, (uint8_t)y, (uint8_t)fw, (uint8_t)fh});
}

int make_tensor_map(vjb_ctx *c) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn)
            return fail(VJB_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    // rows of the sorted table as [feature][line][64 entries]
    cuuint64_t dims[3] = {(cuuint64_t)kLineElems, (cuuint64_t)c->lines, (cuuint64_t)c->nfeat};
    cuuint64_t strides[2] = {(cuuint64_t)kLineBytes, (cuuint64_t)c->lines * kLineBytes};
    cuuint32_t box[3] = {(cuuint32_t)kLineElems, (cuuint32_t)c->box_lines, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(&c->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, c->d_rows, dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(VJB_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    c->tmap_ok = true;
    return VJB_OK;
}

bool shape_fits(const vjb_ctx *c, const SearchShape &s) {
    return s.warps <= screen_max_warps(s.unroll) && search_smem_bytes(s, c->lay.words) <= (size_t)c->max_smem;
}

int make_tensor_map(vjb_ctx *c);

int apply_shape(vjb_ctx *c) {
    c->screen_grid = c->num_sms * c->shape.ctas_per_sm;
    const int box = std::min(c->shape.box_lines, c->lines);
    if (box != c->box_lines || !c->tmap_ok) {
        c->box_lines = box;
        if (c->d_rows) {
            const int rc = make_tensor_map(c);
            if (rc) return rc;
        }
    }
    if (c->screen_grid > c->bmin_cap) {
        dfree(c->d_bmin);
        CK(cudaMalloc(&c->d_bmin, sizeof(float) * c->screen_grid));
        c->bmin_cap = c->screen_grid;
    }
    c->shortlist_grid = c->num_sms * 2;
    // a round shortlists a handful of features: a few CTAs (each takes every
    // grid-th candidate) launch and hand over to the last one faster than two per SM
    c->rescan_grid = 16;
    c->shape_set = true;
    c->drop_graph();
    return VJB_OK;
}

int choose_default_shape(vjb_ctx *c) {
    if (c->shape_set && shape_fits(c, c->shape)) return apply_shape(c);
    // measured on the 24x24 / 15k workload: 16 warps (four per scheduler), two
    // stages of 24 lines, three pieces in flight per lane; then smaller shapes.
    // Rows whose lines divide into whole 32-line stages (npad a multiple of
    // 2,048: 4,000 or 8,000 samples) go faster with 32-line stages where they
    // fit (24x24: 82.9 -> 85.9% of the measured peak at 4,000 samples, 90.2 ->
    // 90.8% at 8,000); otherwise a short last stage costs more than the
    // 24-line fast path saves (12,000 samples: 94.2 against 95.9%).
    const SearchShape whole32{16, 2, 1, 3, 32};
    if (c->lines % 32 == 0 && shape_fits(c, whole32)) {
        c->shape = whole32;
        return apply_shape(c);
    }
    const SearchShape tries[] = {{16, 2, 1, 3, 24}, {12, 2, 1, 4, 32}, {12, 2, 1, 2, 32}, {8, 3, 1, 4, 32},
                                 {8, 2, 1, 4, 32}, {6, 3, 1, 2, 32}, {4, 4, 1, 2, 32}, {4, 2, 1, 2, 32},
                                 {2, 2, 1, 2, 16}, {2, 2, 1, 1, 8}};
    for (const auto &s : tries)
        if (shape_fits(c, s)) {
            c->shape = s;
            return apply_shape(c);
        }
    return fail(VJB_EINVAL, "no search shape fits shared memory for n = %d", c->n);
}

int ensure_stump_cap(vjb_ctx *c, int need) {
    if (need <= c->stump_cap) return VJB_OK;
    int cap = std::max(1024, c->stump_cap);
    while (cap < need) cap *= 2;
    vjb_stump *p = nullptr;
    vjb_round_diag *q = nullptr;
    CK(cudaMalloc(&p, sizeof(vjb_stump) * cap));
    CK(cudaMalloc(&q, sizeof(vjb_round_diag) * cap));
    if (c->d_stumps && c->stump_cap) {
        CK(cudaMemcpyAsync(p, c->d_stumps, sizeof(vjb_stump) * c->stump_cap, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(q, c->d_diag, sizeof(vjb_round_diag) * c->stump_cap, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    dfree(c->d_stumps);
    dfree(c->d_diag);
    c->d_stumps = p;
    c->d_diag = q;
    c->stump_cap = cap;
    c->drop_graph();
    return VJB_OK;
}

int take_events(vjb_ctx *c, EventTriple &t) {
    if (c->ev_free.empty()) {
        for (auto &e : t) CK(cudaEventCreate(&e));
    } else {
        t = c->ev_free.back();
        c->ev_free.pop_back();
    }
    return VJB_OK;
}

// Fold finished event triples into the timing totals (the stream must be idle).
int collect_timing(vjb_ctx *c) {
    for (auto &p : c->ev_pending) {
        const EventTriple &t = p.ev;
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, t[0], t[1]));
        CK(cudaEventElapsedTime(&b, t[0], p.end));
        if (c->tacc.rounds == 0) {
            c->tacc.search_ms_min = a;
            c->tacc.search_ms_max = a;
        } else {
            c->tacc.search_ms_min = std::min(c->tacc.search_ms_min, (double)a);
            c->tacc.search_ms_max = std::max(c->tacc.search_ms_max, (double)a);
        }
        c->tacc.rounds += 1;
        c->tacc.search_ms_total += a;
        c->tacc.round_ms_total += b;
        c->ev_free.push_back(t);
    }
    c->ev_pending.clear();
    return VJB_OK;
}

// The launches of one round (Sec. 2.3 steps 2-4, with step 1 of the next
// round).  `ev` (may be NULL) brackets the search kernel and the round.
JobDesc job_desc(const vjb_ctx *c) {
    JobDesc J{};
    J.rows = c->d_rows;
    J.npad = c->npad;
    J.lines = c->lines;
    J.nfeat = c->nfeat;
    J.line_base = c->line_base;
    J.lay = c->lay;
    J.v = c->d_v;
    J.w = c->d_w;
    J.y = c->d_y;
    J.miss = c->d_miss;
    J.partials = c->d_partials;
    J.rs = c->d_rs;
    J.ferr = c->d_ferr;
    J.cand_ids = c->d_cand_ids;
    J.runres = static_cast<RunResult *>(c->d_runres);
    J.cand_runs = c->d_cand_runs;
    J.cands = c->d_cand;
    J.stumps = c->d_stumps;
    J.diag = c->d_diag;
    J.last = c->d_last;
    J.stump_cap = c->stump_cap;
    J.ii_stride = c->ii_stride;
    J.ii = c->d_ii;
    J.feat = c->d_feat;
    J.win_w = c->w;
    return J;
}

int enqueue_update(vjb_ctx *c) {
    const JobDesc J = job_desc(c);
    CK(launch_update_a(J, c->stream));
    CK(launch_update_b(J, c->stream));
    return VJB_OK;
}

// The search kernel of a round, then the rest (shortlist, re-scan, update).
int enqueue_search(vjb_ctx *c) {
    CK(launch_screen(&c->tmap, c->d_v, c->lay, c->lines, c->box_lines, c->nfeat, c->shape,
                     c->screen_grid, c->d_rs, c->d_ferr, c->d_bmin, c->stream));
    return VJB_OK;
}

int enqueue_tail(vjb_ctx *c) {
    const JobDesc J = job_desc(c);
    CK(launch_shortlist(J, c->d_bmin, c->screen_grid, c->shortlist_grid, c->stream));
    CK(launch_rescan(J, c->rescan_grid, c->stream));
    return enqueue_update(c);
}

int enqueue_round(vjb_ctx *c, const EventTriple *ev) {
    if (ev) CK(cudaEventRecord((*ev)[0], c->stream));
    int rc = enqueue_search(c);
    if (rc) return rc;
    if (ev) CK(cudaEventRecord((*ev)[1], c->stream));
    rc = enqueue_tail(c);
    if (rc) return rc;
    if (ev) CK(cudaEventRecord((*ev)[2], c->stream));
    return VJB_OK;
}

// Capture `part` of a round (0 the whole round, 1 the search, 2 the rest) as
// an instantiated graph.
int capture_round(vjb_ctx *c, int part, cudaGraph_t *graph, cudaGraphExec_t *exec) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = part == 1 ? enqueue_search(c) : (part == 2 ? enqueue_tail(c) : enqueue_round(c, nullptr));
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != VJB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(VJB_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        *exec = nullptr;
        return fail(VJB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    *graph = g;
    return VJB_OK;
}

// The round as one graph; with timing on, as two (the search and the rest)
// with the timing events recorded on the stream around them, so that no
// graph is updated between replays.
int ensure_graph(vjb_ctx *c) {
    if (c->gexec && c->graph_timed == c->timing) return VJB_OK;
    c->drop_graph();
    int rc = capture_round(c, c->timing ? 1 : 0, &c->graph, &c->gexec);
    if (rc == VJB_OK && c->timing) rc = capture_round(c, 2, &c->graph2, &c->gexec2);
    if (rc != VJB_OK) {
        c->drop_graph();
        return rc;
    }
    c->graph_timed = c->timing;
    return VJB_OK;
}

int read_state(vjb_ctx *c, RoundState *rs) {
    CK(cudaMemcpyAsync(rs, c->d_rs, sizeof(RoundState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return VJB_OK;
}

int device_flags_error(const RoundState &rs) {
    return fail(VJB_EDEVICE, "kernel error flags 0x%x (1 = wait timeout, 2 = no candidate, 4 = bad weights, 8 = bad table)",
                rs.flags | 0);
}

int validate_labels(const uint8_t *y, int n) {
    int l = 0, m = 0;
    for (int i = 0; i < n; ++i) {
        if (y[i] > 1) return fail(VJB_EINVAL, "label %d of sample %d is not 0 or 1", (int)y[i], i);
        if (y[i]) ++l; else ++m;
    }
    if (!l || !m) return fail(VJB_EINVAL, "need at least one face and one non-face (got %d, %d)", l, m);
    return VJB_OK;
}

int load_common(vjb_ctx *c, const uint8_t *pixels, const uint8_t *labels, int32_t n, int32_t h,
                int32_t w, bool on_device) {
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    if (!pixels || !labels) return fail(VJB_EINVAL, "pixels or labels is NULL");
    if (n < 2 || n > VJB_MAX_SAMPLES) return fail(VJB_EINVAL, "n = %d outside [2, %d]", n, VJB_MAX_SAMPLES);
    if (h < 1 || w < 1 || h > VJB_MAX_WINDOW || w > VJB_MAX_WINDOW)
        return fail(VJB_EINVAL, "window %dx%d outside [1, %d]", w, h, VJB_MAX_WINDOW);
    int rc = set_dev(c);
    if (rc) return rc;
    std::vector<uint8_t> hy((size_t)n);
    if (on_device) {
        CK(cudaMemcpy(hy.data(), labels, (size_t)n, cudaMemcpyDeviceToHost));
    } else {
        memcpy(hy.data(), labels, (size_t)n);
    }
    rc = validate_labels(hy.data(), n);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    const bool same_shape = c->d_px && c->n == n && c->h == h && c->w == w;
    if (!same_shape) {
        // a new shape: release everything sized by the old one
        c->free_all();
        c->n = n;
        c->h = h;
        c->w = w;
        const size_t npx = (size_t)n * h * w;
        CK(cudaMalloc(&c->d_px, npx));
        CK(cudaMalloc(&c->d_y, (size_t)n));
        CK(cudaMalloc(&c->d_w, sizeof(float) * n));
        CK(cudaMalloc(&c->d_wtmp, sizeof(float) * n));
        c->lay = make_layout(n, true);
        CK(cudaMalloc(&c->d_v, sizeof(float) * c->lay.words));
        CK(cudaMemset(c->d_v, 0, sizeof(float) * c->lay.words));
        CK(cudaMalloc(&c->d_miss, (size_t)n));
        CK(cudaMalloc(&c->d_partials, sizeof(double) * 3 * kUpdateMaxCtas));
        CK(cudaMalloc(&c->d_rs, sizeof(RoundState)));
        CK(cudaMalloc(&c->d_last, sizeof(vjb_stump)));
        rc = ensure_stump_cap(c, 1024);
        if (rc) return rc;
    }
    // same shape: buffers, tables and the round graph are reused; contents are rebuilt
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(c->d_px, pixels, (size_t)n * h * w, kind, c->stream));
    CK(cudaMemcpyAsync(c->d_y, hy.data(), (size_t)n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->d_rs, 0, sizeof(RoundState), c->stream));
    CK(cudaMemsetAsync(c->d_last, 0, sizeof(vjb_stump), c->stream));
    CK(launch_init_weights(c->d_y, c->lay, nullptr, c->d_w, c->d_v, c->d_rs, c->stream));
    c->launches += 1;
    CK(cudaStreamSynchronize(c->stream));
    c->stage = kStageLoaded;
    return VJB_OK;
}

int copy_stump_out(vjb_ctx *c, vjb_stump *out) {
    if (!out) return VJB_OK;
    CK(cudaMemcpyAsync(out, c->d_last, sizeof(vjb_stump), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return VJB_OK;
}

// Feature values (K2) and sort (K3) a tile of features at a time, then a check
// of the finished table.
int prepare_tables(vjb_ctx *c) {
    if (c->feats.empty()) {
        enumerate_host(c->w, c->h, c->feats);
        c->nfeat = (int64_t)c->feats.size();
        if (c->nfeat == 0 || c->nfeat > 0x7fffffffLL)
            return fail(VJB_EINVAL, "window %dx%d has %lld features", c->w, c->h, (long long)c->nfeat);
        std::vector<DevFeature> df((size_t)c->nfeat);
        for (size_t k = 0; k < df.size(); ++k) {
            const vjb_feature &f = c->feats[k];
            df[k] = DevFeature{f.type, f.x, f.y, f.w, f.h, 0, 0, 0};
        }
        CK(cudaMalloc(&c->d_feat, sizeof(DevFeature) * df.size()));
        CK(cudaMemcpy(c->d_feat, df.data(), sizeof(DevFeature) * df.size(), cudaMemcpyHostToDevice));
        c->npad = (c->n + kRowAlign - 1) / kRowAlign * kRowAlign;
        c->lines = c->npad / kLineElems;
        c->box_lines = 0;  // set with the search shape
    }
    if (!c->d_rows) {
        if (c->rows_external) return fail(VJB_ESTATE, "external table not set");
        CK(cudaMalloc(&c->d_rows, sizeof(uint16_t) * (size_t)c->nfeat * c->npad));
    }
    // feature values (the K2 arithmetic, fused into the sort) and sort, a tile
    // of rows per launch (one launch up to 2^22 rows: 24x24 windows take one,
    // so no SM idles at a tile's end); the sort kernels check every entry they
    // write (the search kernels gather through the table without bounds
    // checks) and count the rows they write
    const int64_t tile = std::max<int64_t>(1, std::min<int64_t>(c->nfeat, int64_t(1) << 22));
    // (kept with the context: a cudaFree here would wait for the whole device,
    // other contexts' rounds included, when a server prepares a request)
    if (!c->d_scratch) CK(cudaMalloc(&c->d_scratch, sizeof(int32_t) * (size_t)(3 + tile)));
    int32_t *d_scratch = c->d_scratch;  // check state, then the rows the packed sort hands to the two-word sort
    cudaError_t e = cudaMemsetAsync(d_scratch, 0, 2 * sizeof(int32_t), c->stream);
    for (int64_t f0 = 0; f0 < c->nfeat && e == cudaSuccess; f0 += tile) {
        const int64_t nf = std::min(tile, c->nfeat - f0);
        e = launch_sort_rows(c->d_ii, c->ii16(), c->ii_stride, c->w, c->d_feat, f0, nf, c->lay,
                             c->d_rows + (size_t)f0 * c->npad, c->npad, d_scratch, c->stream);
        c->launches += 1;
    }
    int32_t stat[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(stat, d_scratch, sizeof stat, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(VJB_ECUDA, "sort of the feature rows: %s", cudaGetErrorString(e));
    if (stat[0] || stat[1] != c->nfeat)
        return fail(VJB_EDEVICE, "sorted table check failed: flags 0x%x, %d of %lld rows written", stat[0],
                    stat[1], (long long)c->nfeat);
    RoundState rs;
    int rc = read_state(c, &rs);
    if (rc) return rc;
    if (rs.flags) return device_flags_error(rs);
    if (!c->d_ferr) CK(cudaMalloc(&c->d_ferr, sizeof(float) * c->nfeat));
    if (!c->d_cand) CK(cudaMalloc(&c->d_cand, sizeof(Candidate) * c->nfeat));
    if (!c->d_cand_ids) CK(cudaMalloc(&c->d_cand_ids, sizeof(int32_t) * c->nfeat));
    if (!c->d_runres) CK(cudaMalloc(&c->d_runres, (size_t)kRunResultBytes * 32 * kRescanSplitCap));
    if (!c->d_cand_runs) {
        CK(cudaMalloc(&c->d_cand_runs, sizeof(uint32_t) * kRescanSplitCap));
        CK(cudaMemset(c->d_cand_runs, 0, sizeof(uint32_t) * kRescanSplitCap));
    }
    if (!c->d_bmin || !c->tmap_ok) {
        rc = choose_default_shape(c);
        if (rc) return rc;
    }
    return VJB_OK;
}

}  // namespace vjb

namespace vjb {
// Error reporting for entry points defined in other translation units.
int report_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace vjb

extern "C" {

const char *vjb_last_error(void) { return g_err; }

int vjb_create(vjb_ctx **out, int device, void *cuda_stream) {
    g_err[0] = 0;
    if (!out) return fail(VJB_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(VJB_EINVAL, "device %d outside [0, %d)", device, ndev);
    CK(cudaSetDevice(device));
    vjb_ctx *c = new vjb_ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess && prop.major < 10) {
        delete c;
        return fail(VJB_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a", device,
                    prop.major, prop.minor);
    }
    if (e == cudaSuccess) {
        c->num_sms = prop.multiProcessorCount;
        c->max_smem = (int)prop.sharedMemPerBlockOptin;
    }
    if (e == cudaSuccess) e = set_screen_smem_limit(c->max_smem);
    if (e == cudaSuccess && cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    if (e != cudaSuccess) {
        delete c;
        return fail(VJB_ECUDA, "context setup failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return VJB_OK;
}

void vjb_destroy(vjb_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->free_all();
    c->free_events();
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int vjb_load_windows(vjb_ctx *c, const uint8_t *pixels, const uint8_t *labels, int32_t n,
                     int32_t h, int32_t w) {
    g_err[0] = 0;
    return load_common(c, pixels, labels, n, h, w, false);
}

int vjb_load_windows_device(vjb_ctx *c, const uint8_t *pixels, const uint8_t *labels, int32_t n,
                            int32_t h, int32_t w) {
    g_err[0] = 0;
    return load_common(c, pixels, labels, n, h, w, true);
}

int vjb_build_integral(vjb_ctx *c) {
    g_err[0] = 0;
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    if (c->stage < kStageLoaded) return fail(VJB_ESTATE, "vjb_build_integral before vjb_load_windows");
    int rc = set_dev(c);
    if (rc) return rc;
    // the int32 integral images, then the same modulo 2^16 (ii16())
    if (!c->d_ii) {
        c->ii_stride = (c->n + 31) / 32 * 32;
        CK(cudaMalloc(&c->d_ii, (sizeof(int32_t) + sizeof(uint16_t)) * (size_t)(c->h + 1) * (c->w + 1) *
                                    c->ii_stride));
    }
    CK(launch_integral(c->d_px, c->n, c->h, c->w, c->d_ii, c->ii16(), c->ii_stride, c->stream));
    c->launches += 1;
    CK(cudaStreamSynchronize(c->stream));
    c->stage = kStageIntegral;
    return VJB_OK;
}

int vjb_enumerate_haar(vjb_ctx *c, int64_t *count, vjb_feature *out) {
    g_err[0] = 0;
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    if (!count) return fail(VJB_EINVAL, "count is NULL");
    if (c->stage < kStageIntegral) return fail(VJB_ESTATE, "vjb_enumerate_haar before vjb_build_integral");
    int rc = set_dev(c);
    if (rc) return rc;
    if (c->stage < kStagePrepared) {
        rc = prepare_tables(c);
        if (rc) return rc;
        c->stage = kStagePrepared;
    }
    *count = c->nfeat;
    if (out) memcpy(out, c->feats.data(), sizeof(vjb_feature) * c->feats.size());
    return VJB_OK;
}

int vjb_train_round(vjb_ctx *c, vjb_stump *out) {
    g_err[0] = 0;
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "vjb_train_round before vjb_enumerate_haar");
    int rc = set_dev(c);
    if (rc) return rc;
    RoundState rs;
    rc = read_state(c, &rs);
    if (rc) return rc;
    if (rs.status == VJB_OK) {
        rc = ensure_stump_cap(c, rs.rounds + 1);
        if (rc) return rc;
        EventTriple ev{};
        if (c->timing) {
            rc = take_events(c, ev);
            if (rc) return rc;
        }
        rc = enqueue_round(c, c->timing ? &ev : nullptr);
        if (rc) return rc;
        c->launches += kRoundLaunches;
        if (c->timing) c->ev_pending.push_back(PendingRound{ev, ev[2]});
        rc = read_state(c, &rs);
        if (rc) return rc;
    }
    if (rs.flags) return device_flags_error(rs);
    rc = copy_stump_out(c, out);
    if (rc) return rc;
    return rs.status;
}

int vjb_train_strong(vjb_ctx *c, int32_t T, vjb_stump *out, int32_t *rounds_done) {
    g_err[0] = 0;
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    if (T < 0) return fail(VJB_EINVAL, "T = %d < 0", T);
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "vjb_train_strong before vjb_enumerate_haar");
    int rc = set_dev(c);
    if (rc) return rc;
    RoundState rs;
    rc = read_state(c, &rs);
    if (rc) return rc;
    const int r0 = rs.rounds;
    if (rs.status == VJB_OK && T > 0) {
        rc = ensure_stump_cap(c, r0 + T);
        if (rc) return rc;
        rc = ensure_graph(c);
        if (rc) return rc;
        for (int32_t t = 0; t < T; ++t) {
            if (c->timing) {
                // two events per round: a round ends where the next one
                // starts; the last one records its own end
                EventTriple ev{};
                rc = take_events(c, ev);
                if (rc) return rc;
                CK(cudaEventRecord(ev[0], c->stream));
                if (t > 0) c->ev_pending.back().end = ev[0];
                CK(cudaGraphLaunch(c->gexec, c->stream));
                CK(cudaEventRecord(ev[1], c->stream));
                CK(cudaGraphLaunch(c->gexec2, c->stream));
                if (t == T - 1) CK(cudaEventRecord(ev[2], c->stream));
                c->ev_pending.push_back(PendingRound{ev, ev[2]});
            } else {
                CK(cudaGraphLaunch(c->gexec, c->stream));
            }
            c->launches += kRoundLaunches;
        }
        rc = read_state(c, &rs);
        if (rc) return rc;
    }
    if (rs.flags) return device_flags_error(rs);
    const int kept = rs.rounds - r0;
    if (out && kept > 0) {
        CK(cudaMemcpyAsync(out, c->d_stumps + r0, sizeof(vjb_stump) * kept, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (rounds_done) *rounds_done = kept;
    return rs.status;
}

int vjb_get_weights(vjb_ctx *c, float *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStageLoaded) return fail(VJB_ESTATE, "no training set loaded");
    int rc = set_dev(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out, c->d_w, sizeof(float) * c->n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return VJB_OK;
}

int vjb_set_weights(vjb_ctx *c, const float *wts) {
    g_err[0] = 0;
    if (!c || !wts) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStageLoaded) return fail(VJB_ESTATE, "no training set loaded");
    double s = 0.0;
    for (int i = 0; i < c->n; ++i) {
        if (!std::isfinite(wts[i]) || wts[i] < 0.f) return fail(VJB_EINVAL, "weight %d is negative or not finite", i);
        s += wts[i];
    }
    if (!(s > 0.0)) return fail(VJB_EINVAL, "weights sum to zero");
    int rc = set_dev(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->d_wtmp, wts, sizeof(float) * c->n, cudaMemcpyHostToDevice, c->stream));
    CK(launch_init_weights(c->d_y, c->lay, c->d_wtmp, c->d_w, c->d_v, c->d_rs, c->stream));
    c->launches += 1;
    CK(cudaStreamSynchronize(c->stream));
    return VJB_OK;
}

int vjb_force_stump(vjb_ctx *c, int32_t feature, int32_t threshold, int32_t polarity, vjb_stump *out) {
    g_err[0] = 0;
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "vjb_force_stump before vjb_enumerate_haar");
    if (feature < 0 || feature >= c->nfeat) return fail(VJB_EINVAL, "feature %d out of range", feature);
    if (polarity != 1 && polarity != -1) return fail(VJB_EINVAL, "polarity %d is not +-1", polarity);
    int rc = set_dev(c);
    if (rc) return rc;
    RoundState rs;
    rc = read_state(c, &rs);
    if (rc) return rc;
    if (rs.status == VJB_OK) {
        rc = ensure_stump_cap(c, rs.rounds + 1);
        if (rc) return rc;
        int32_t f4[4] = {1, feature, threshold, polarity};
        char *dst = reinterpret_cast<char *>(c->d_rs) + offsetof(RoundState, forced);
        CK(cudaMemcpyAsync(dst, f4, sizeof f4, cudaMemcpyHostToDevice, c->stream));
        rc = enqueue_update(c);
        if (rc) return rc;
        c->launches += 2;
        rc = read_state(c, &rs);
        if (rc) return rc;
    }
    if (rs.flags) return device_flags_error(rs);
    rc = copy_stump_out(c, out);
    if (rc) return rc;
    return rs.status;
}

int vjb_get_info(vjb_ctx *c, vjb_info *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    memset(out, 0, sizeof *out);
    out->n = c->n;
    out->h = c->h;
    out->w = c->w;
    out->npad = c->npad;
    out->features = c->nfeat;
    out->kernel_warps = c->shape.warps;
    out->kernel_stages = c->shape.stages;
    out->kernel_ctas = c->screen_grid;
    out->kernel_unroll = c->shape.unroll;
    out->kernel_box_lines = c->box_lines;
    out->dual_weights = c->lay.dual;
    out->search_bytes = 2.0 * (double)c->nfeat * (double)c->n;
    out->launches = c->launches;
    if (c->stage >= kStageLoaded) {
        int rc = set_dev(c);
        if (rc) return rc;
        RoundState rs;
        rc = read_state(c, &rs);
        if (rc) return rc;
        out->rounds_done = rs.rounds;
        out->status = rs.status;
        out->t_pos = rs.t_pos;
        out->t_neg = rs.t_neg;
        out->weight_sum = rs.weight_sum;
        out->screen_min = rs.screen_min;
        out->candidates = rs.last_cands;
        out->device_flags = rs.flags;
    }
    return VJB_OK;
}

int vjb_classify(vjb_ctx *c, const uint8_t *pixels, int32_t n, const vjb_stump *stumps, int32_t T,
                 uint8_t *labels, double *scores) {
    g_err[0] = 0;
    if (!c || !pixels || !labels || (T > 0 && !stumps)) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "vjb_classify before vjb_enumerate_haar");
    if (n < 1 || n > (1 << 26)) return fail(VJB_EINVAL, "n = %d outside [1, 2^26]", n);
    if (T < 0) return fail(VJB_EINVAL, "T < 0");
    double half = 0.0;
    for (int t = 0; t < T; ++t) {
        const vjb_stump &s = stumps[t];
        if (s.feature < 0 || s.feature >= c->nfeat || (s.polarity != 1 && s.polarity != -1) || std::isnan(s.alpha))
            return fail(VJB_EINVAL, "stump %d is not a stump of this window size", t);
        half += s.alpha;
    }
    half *= 0.5;  // C(x) = 1 iff sum alpha_t h_t(x) >= 1/2 sum alpha_t
    int rc = set_dev(c);
    if (rc) return rc;
    const size_t px_bytes = (size_t)n * c->h * c->w;
    const int stride = (n + 31) / 32 * 32;
    uint8_t *d_px = nullptr, *d_lab = nullptr;
    int32_t *d_ii = nullptr;
    vjb_stump *d_st = nullptr;
    double *d_sc = nullptr;
    auto cleanup = [&]() {
        dfree(d_px); dfree(d_lab); dfree(d_ii); dfree(d_st); dfree(d_sc);
    };
    cudaError_t e = cudaMalloc(&d_px, px_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_ii, sizeof(int32_t) * (size_t)(c->h + 1) * (c->w + 1) * stride);
    if (e == cudaSuccess) e = cudaMalloc(&d_lab, (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d_st, sizeof(vjb_stump) * (size_t)std::max(T, 1));
    if (e == cudaSuccess && scores) e = cudaMalloc(&d_sc, sizeof(double) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_px, pixels, px_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && T > 0) e = cudaMemcpyAsync(d_st, stumps, sizeof(vjb_stump) * T, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_integral(d_px, n, c->h, c->w, d_ii, nullptr, stride, c->stream);
    if (e == cudaSuccess)
        e = launch_strong_classify(d_ii, stride, n, c->w, c->d_feat, d_st, T, half, d_lab, d_sc, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels, d_lab, (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && scores)
        e = cudaMemcpyAsync(scores, d_sc, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->launches += 2;
    cleanup();
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? VJB_ENOMEM : VJB_ECUDA, "classify: %s", cudaGetErrorString(e));
    return VJB_OK;
}

int vjb_get_integral(vjb_ctx *c, int32_t *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStageIntegral) return fail(VJB_ESTATE, "integral images not built");
    int rc = set_dev(c);
    if (rc) return rc;
    const int P = (c->h + 1) * (c->w + 1);
    std::vector<int32_t> t((size_t)P * c->ii_stride);
    CK(cudaMemcpyAsync(t.data(), c->d_ii, sizeof(int32_t) * t.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->n; ++i)
        for (int p = 0; p < P; ++p) out[(size_t)i * P + p] = t[(size_t)p * c->ii_stride + i];
    return VJB_OK;
}

int vjb_feature_values(vjb_ctx *c, int64_t f0, int64_t nf, int32_t *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "features not enumerated");
    if (f0 < 0 || nf < 0 || f0 + nf > c->nfeat) return fail(VJB_EINVAL, "feature range outside [0, F)");
    if (nf == 0) return VJB_OK;
    int rc = set_dev(c);
    if (rc) return rc;
    int32_t *d = nullptr;
    CK(cudaMalloc(&d, sizeof(int32_t) * (size_t)nf * c->n));
    cudaError_t e = launch_feature_values(c->d_ii, c->ii_stride, c->n, c->w, c->d_feat, f0, nf, d, c->stream);
    c->launches += 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(int32_t) * (size_t)nf * c->n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(VJB_ECUDA, "feature values failed: %s", cudaGetErrorString(e));
    return VJB_OK;
}

int vjb_sorted_rows(vjb_ctx *c, int64_t f0, int64_t nf, uint16_t *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "features not enumerated");
    if (f0 < 0 || nf < 0 || f0 + nf > c->nfeat) return fail(VJB_EINVAL, "feature range outside [0, F)");
    if (nf == 0) return VJB_OK;
    int rc = set_dev(c);
    if (rc) return rc;
    // rows in value order: undo the lane-run interleave and name samples, not weight words
    std::vector<uint16_t> raw((size_t)nf * c->npad);
    CK(cudaMemcpyAsync(raw.data(), c->d_rows + (size_t)f0 * c->npad, sizeof(uint16_t) * raw.size(),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int run = c->npad / 32;
    for (int64_t r = 0; r < nf; ++r)
        for (int e = 0; e < c->n; ++e) {
            const int P = phys_of(e, run);
            const uint16_t x = raw[(size_t)r * c->npad + P];
            out[(size_t)r * c->n + e] =
                (uint16_t)((entry_flag(x, P) ? kFlagBit : 0) | word_to_sample(entry_word(x, P), c->lay));
        }
    return VJB_OK;
}

int vjb_screen_errors(vjb_ctx *c, float *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStagePrepared) return fail(VJB_ESTATE, "features not enumerated");
    int rc = set_dev(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out, c->d_ferr, sizeof(float) * c->nfeat, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return VJB_OK;
}

int vjb_set_search_shape(vjb_ctx *c, const vjb_search_shape *in) {
    g_err[0] = 0;
    if (!c || !in) return fail(VJB_EINVAL, "NULL argument");
    SearchShape s = c->shape;
    if (in->warps) s.warps = in->warps;
    if (in->stages) s.stages = in->stages;
    if (in->ctas_per_sm) s.ctas_per_sm = in->ctas_per_sm;
    if (in->unroll) s.unroll = in->unroll;
    if (in->box_lines) s.box_lines = in->box_lines;
    if (s.warps < 1 || s.warps > 20 || s.stages < 1 || s.stages > 8 || s.ctas_per_sm < 1 || s.ctas_per_sm > 4 ||
        (s.unroll < 1 || s.unroll > 4) || s.warps > screen_max_warps(s.unroll) ||
        s.box_lines < 4 || s.box_lines > 32 || s.box_lines % 4 != 0)
        return fail(VJB_EINVAL, "search shape (%d warps, %d stages, %d CTAs/SM, unroll %d, box %d lines) out of range",
                    s.warps, s.stages, s.ctas_per_sm, s.unroll, s.box_lines);
    if (c->n > 0 && !shape_fits(c, s))
        return fail(VJB_EINVAL, "search shape needs %zu bytes of shared memory (limit %d)",
                    search_smem_bytes(s, c->lay.words), c->max_smem);
    if (c->n > 0 && screen_occupancy(s, c->lay.words) < s.ctas_per_sm)
        return fail(VJB_EINVAL, "%d CTAs per SM of this shape do not fit one SM", s.ctas_per_sm);
    int rc = set_dev(c);
    if (rc) return rc;
    c->shape = s;
    c->shape_set = true;
    if (c->stage >= kStagePrepared) return apply_shape(c);
    return VJB_OK;
}

int vjb_get_search_shape(vjb_ctx *c, vjb_search_shape *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    out->warps = c->shape.warps;
    out->stages = c->shape.stages;
    out->ctas_per_sm = c->shape.ctas_per_sm;
    out->unroll = c->shape.unroll;
    out->box_lines = c->shape.box_lines;
    return VJB_OK;
}

int vjb_get_round_diag(vjb_ctx *c, int32_t first, int32_t count, vjb_round_diag *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    if (c->stage < kStageLoaded) return fail(VJB_ESTATE, "no training set loaded");
    int rc = set_dev(c);
    if (rc) return rc;
    RoundState rs;
    rc = read_state(c, &rs);
    if (rc) return rc;
    if (first < 0 || count < 0 || first + count > rs.rounds || first + count > c->stump_cap)
        return fail(VJB_EINVAL, "rounds [%d, %d) outside the %d kept", first, first + count, rs.rounds);
    if (count == 0) return VJB_OK;
    CK(cudaMemcpyAsync(out, c->d_diag + first, sizeof(vjb_round_diag) * count, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return VJB_OK;
}

int vjb_set_timing(vjb_ctx *c, int32_t enable) {
    g_err[0] = 0;
    if (!c) return fail(VJB_EINVAL, "context is NULL");
    int rc = set_dev(c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    for (auto &t : c->ev_pending) c->ev_free.push_back(t.ev);
    c->ev_pending.clear();
    c->tacc = vjb_timing{};
    c->timing = enable != 0;
    return VJB_OK;
}

int vjb_get_timing(vjb_ctx *c, vjb_timing *out) {
    g_err[0] = 0;
    if (!c || !out) return fail(VJB_EINVAL, "NULL argument");
    int rc = set_dev(c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    rc = collect_timing(c);
    if (rc) return rc;
    *out = c->tacc;
    return VJB_OK;
}

}  // extern "C"
