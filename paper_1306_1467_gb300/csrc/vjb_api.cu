// C ABI of the library (declared in include/vjb.h): context ownership,
// argument checking, the order of the training steps, and the launch sequence
// of a boosting round (search -> refine -> finalize), replayed as a CUDA graph
// by vjb_train_strong.
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "vjb_internal.cuh"

namespace vjb {
cudaError_t set_screen_smem_limit(int bytes);
int screen_occupancy(const SearchShape &s, int words);
int screen_max_warps(int unroll);
}  // namespace vjb

using namespace vjb;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? VJB_ENOMEM : VJB_ECUDA,       \
                        "%s failed: %s", #call, cudaGetErrorString(e_));               \
    } while (0)

template <class T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

constexpr int kStageNone = 0, kStageLoaded = 1, kStageIntegral = 2, kStagePrepared = 3;
constexpr int kRoundLaunches = 5;  // screen, shortlist, rescan, update a, update b

using EventTriple = std::array<cudaEvent_t, 3>;  // round start, search end, round end

}  // namespace

struct vjb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int max_smem = 0;
    int stage = kStageNone;
    int64_t launches = 0;

    int n = 0, h = 0, w = 0;
    int ii_stride = 0, npad = 0, lines = 0, box_lines = 0;
    int64_t nfeat = 0;
    WeightLayout lay{};

    uint8_t *d_px = nullptr, *d_y = nullptr;
    int32_t *d_ii = nullptr;
    DevFeature *d_feat = nullptr;
    uint16_t *d_rows = nullptr;
    bool rows_external = false;  // the table lives in a batch's arena
    int64_t line_base = 0;       // its first line there
    float *d_w = nullptr, *d_v = nullptr, *d_wtmp = nullptr;
    float *d_ferr = nullptr, *d_bmin = nullptr;
    Candidate *d_cand = nullptr;
    int32_t *d_cand_ids = nullptr;
    uint8_t *d_miss = nullptr;
    double *d_partials = nullptr;
    RoundState *d_rs = nullptr;
    vjb_stump *d_stumps = nullptr, *d_last = nullptr;
    vjb_round_diag *d_diag = nullptr;
    int stump_cap = 0;
    int bmin_cap = 0;

    std::vector<vjb_feature> feats;
    CUtensorMap tmap;
    bool tmap_ok = false;
    SearchShape shape{12, 2, 1, 4, 32};
    bool shape_set = false;
    int screen_grid = 0, shortlist_grid = 0, rescan_grid = 0;

    // graph of one round; with timing on it holds three event-record nodes
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_timed = false;
    cudaGraphNode_t ev_nodes[3] = {nullptr, nullptr, nullptr};

    bool timing = false;
    std::vector<EventTriple> ev_free, ev_pending;
    vjb_timing tacc{};

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
    }
    void free_all() {
        drop_graph();
        dfree(d_px); dfree(d_y); dfree(d_ii); dfree(d_feat);
        if (rows_external) d_rows = nullptr;
        dfree(d_rows);
        rows_external = false;
        dfree(d_w); dfree(d_v); dfree(d_wtmp); dfree(d_ferr); dfree(d_bmin); dfree(d_cand);
        dfree(d_cand_ids); dfree(d_miss); dfree(d_partials);
        dfree(d_rs); dfree(d_stumps); dfree(d_last); dfree(d_diag);
        stump_cap = bmin_cap = 0;
        feats.clear();
        stage = kStageNone;
        tmap_ok = false;
        n = h = w = ii_stride = npad = lines = box_lines = 0;
        nfeat = 0;
        lay = WeightLayout{};
    }
    void free_events() {
        for (auto &t : ev_free) for (auto e : t) cudaEventDestroy(e);
        for (auto &t : ev_pending) for (auto e : t) cudaEventDestroy(e);
        ev_free.clear();
        ev_pending.clear();
    }
};

namespace {

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
    // stages of 24 lines, three pieces in flight per lane; then smaller shapes
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
    for (auto &t : c->ev_pending) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, t[0], t[1]));
        CK(cudaEventElapsedTime(&b, t[0], t[2]));
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

int enqueue_round(vjb_ctx *c, const EventTriple *ev, unsigned rec_flags) {
    if (ev) CK(cudaEventRecordWithFlags((*ev)[0], c->stream, rec_flags));
    CK(launch_screen(&c->tmap, c->d_v, c->lay, c->lines, c->box_lines, c->nfeat, c->shape,
                     c->screen_grid, c->d_rs, c->d_ferr, c->d_bmin, c->stream));
    if (ev) CK(cudaEventRecordWithFlags((*ev)[1], c->stream, rec_flags));
    const JobDesc J = job_desc(c);
    CK(launch_shortlist(J, c->d_bmin, c->screen_grid, c->shortlist_grid, c->stream));
    CK(launch_rescan(J, c->rescan_grid, c->stream));
    int rc = enqueue_update(c);
    if (rc) return rc;
    if (ev) CK(cudaEventRecordWithFlags((*ev)[2], c->stream, rec_flags));
    return VJB_OK;
}

int ensure_graph(vjb_ctx *c) {
    if (c->gexec && c->graph_timed == c->timing) return VJB_OK;
    c->drop_graph();
    EventTriple cap{};
    if (c->timing) {
        int rc = take_events(c, cap);
        if (rc) return rc;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_round(c, c->timing ? &cap : nullptr, cudaEventRecordExternal);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (c->timing) c->ev_free.push_back(cap);
    if (rc != VJB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(VJB_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    if (c->timing) {
        size_t nn = 0;
        CK(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(g, nodes.data(), &nn));
        int found = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nd, &ty));
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < 3; ++k)
                if (ev == cap[k]) { c->ev_nodes[k] = nd; ++found; }
        }
        if (found != 3) {
            cudaGraphDestroy(g);
            return fail(VJB_ECUDA, "timed graph has %d of 3 event nodes", found);
        }
    }
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        c->gexec = nullptr;
        return fail(VJB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    c->graph = g;
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
    // feature values (the K2 arithmetic, fused into the sort) and sort, a tile of rows per launch
    const int64_t tile = std::max<int64_t>(1, std::min<int64_t>(c->nfeat, 65535));
    int32_t *d_ovf = nullptr;  // rows the packed sort hands to the two-word sort
    CK(cudaMalloc(&d_ovf, sizeof(int32_t) * (size_t)(1 + tile)));
    for (int64_t f0 = 0; f0 < c->nfeat; f0 += tile) {
        const int64_t nf = std::min(tile, c->nfeat - f0);
        const cudaError_t e = launch_sort_rows(c->d_ii, c->ii_stride, c->w, c->h, c->d_feat, f0, nf, c->lay,
                                               c->d_rows + (size_t)f0 * c->npad, c->npad, d_ovf, c->stream);
        if (e != cudaSuccess) {
            cudaFree(d_ovf);
            return fail(VJB_ECUDA, "sort of rows %lld..: %s", (long long)f0, cudaGetErrorString(e));
        }
        c->launches += 1;
    }
    CK(cudaStreamSynchronize(c->stream));
    dfree(d_ovf);
    // the search kernels gather through the table without bounds checks: validate it once
    CK(launch_check_rows(c->d_rows, c->nfeat, c->lay, c->npad, flags_ptr(c), c->num_sms * 8, c->stream));
    c->launches += 1;
    RoundState rs;
    int rc = read_state(c, &rs);
    if (rc) return rc;
    if (rs.flags) return device_flags_error(rs);
    if (!c->d_ferr) CK(cudaMalloc(&c->d_ferr, sizeof(float) * c->nfeat));
    if (!c->d_cand) CK(cudaMalloc(&c->d_cand, sizeof(Candidate) * c->nfeat));
    if (!c->d_cand_ids) CK(cudaMalloc(&c->d_cand_ids, sizeof(int32_t) * c->nfeat));
    if (!c->d_bmin || !c->tmap_ok) {
        rc = choose_default_shape(c);
        if (rc) return rc;
    }
    return VJB_OK;
}

}  // namespace

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
    if (!c->d_ii) {
        c->ii_stride = (c->n + 31) / 32 * 32;
        CK(cudaMalloc(&c->d_ii, sizeof(int32_t) * (size_t)(c->h + 1) * (c->w + 1) * c->ii_stride));
    }
    CK(launch_integral(c->d_px, c->n, c->h, c->w, c->d_ii, c->ii_stride, c->stream));
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
        rc = enqueue_round(c, c->timing ? &ev : nullptr, cudaEventRecordDefault);
        if (rc) return rc;
        c->launches += kRoundLaunches;
        if (c->timing) c->ev_pending.push_back(ev);
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
                EventTriple ev{};
                rc = take_events(c, ev);
                if (rc) return rc;
                for (int k = 0; k < 3; ++k)
                    CK(cudaGraphExecEventRecordNodeSetEvent(c->gexec, c->ev_nodes[k], ev[k]));
                c->ev_pending.push_back(ev);
            }
            CK(cudaGraphLaunch(c->gexec, c->stream));
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
    if (e == cudaSuccess) e = launch_integral(d_px, n, c->h, c->w, d_ii, stride, c->stream);
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
    for (auto &t : c->ev_pending) c->ev_free.push_back(t);
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
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0;
    // with timing on, the round graph holds three event-record nodes (round
    // start, search end, round end) given fresh events at every replay
    bool timing = false, graph_timed = false;
    cudaGraphNode_t ev_nodes[3] = {nullptr, nullptr, nullptr};
    std::vector<EventTriple> ev_free, ev_pending;
    vjb_timing tacc{};

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
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

int batch_enqueue_round(vjb_batch *b, const EventTriple *ev) {
    const int g = b->num_sms;
    if (ev) CK(cudaEventRecordWithFlags((*ev)[0], b->stream, cudaEventRecordExternal));
    CK(launch_bbegin(b->d_jobs, b->d_meta, b->stream));
    CK(launch_bscreen(b->maps, b->d_jobs, b->d_items, b->d_meta, kBatchMaxWords, b->shape,
                      b->rows_per_warp, g * b->shape.ctas_per_sm, b->stream));
    if (ev) CK(cudaEventRecordWithFlags((*ev)[1], b->stream, cudaEventRecordExternal));
    CK(launch_bshortlist(b->d_jobs, b->d_meta, g * 4, b->stream));
    CK(launch_brescan(b->d_jobs, b->d_meta, std::min(g, 128), b->stream));
    CK(launch_bupdate_a(b->d_jobs, b->d_meta, g * 4, b->stream));
    CK(launch_bupdate_b(b->d_jobs, b->d_meta, g * 4, b->stream));
    if (ev) CK(cudaEventRecordWithFlags((*ev)[2], b->stream, cudaEventRecordExternal));
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

int batch_ensure_graph(vjb_batch *b) {
    if (b->gexec && b->graph_timed == b->timing) return VJB_OK;
    b->drop_graph();
    EventTriple cap{};
    if (b->timing) {
        const int rc = batch_take_events(b, cap);
        if (rc) return rc;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_enqueue_round(b, b->timing ? &cap : nullptr);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (b->timing) b->ev_free.push_back(cap);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(VJB_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    if (b->timing) {
        size_t nn = 0;
        CK(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        CK(cudaGraphGetNodes(g, nodes.data(), &nn));
        int found = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            CK(cudaGraphNodeGetType(nd, &ty));
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < 3; ++k)
                if (ev == cap[k]) { b->ev_nodes[k] = nd; ++found; }
        }
        if (found != 3) {
            cudaGraphDestroy(g);
            return fail(VJB_ECUDA, "timed batch graph has %d of 3 event nodes", found);
        }
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        b->gexec = nullptr;
        return fail(VJB_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    }
    b->graph = g;
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
                for (int k = 0; k < 3; ++k) CK(cudaGraphExecEventRecordNodeSetEvent(b->gexec, b->ev_nodes[k], ev[k]));
                b->ev_pending.push_back(ev);
            }
            CK(cudaGraphLaunch(b->gexec, b->stream));
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
// own stream -- windows, integral images, features, sorted table written into
// the arena -- while the main thread keeps running batched rounds for the jobs
// already training.  A prepared request joins the batch at the next round;
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
    bool stop = false;
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
    int rc = vjb_create(&c, s->device, nullptr);
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
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->to_prepare.empty(); });
            if (s->to_prepare.empty()) return;  // stop requested and nothing left
            r = s->to_prepare.front();
            s->to_prepare.pop_front();
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
        vjb_destroy(sl.ctx);
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
    vjb_batch *b = nullptr;
    int rc = vjb_batch_create(&b, device, nullptr, table_budget_bytes);
    if (rc) return rc;
    vjb_server *s = new vjb_server();
    s->b = b;
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
    vjb_batch_destroy(s->b);  // destroys the contexts of the training jobs
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
