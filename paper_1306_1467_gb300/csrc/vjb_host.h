// Host-side internals shared by the library's C ABI translation units
// (vjb_api.cu: contexts; vjb_batch.cu: batches and serving): error reporting,
// the context structure and the context helpers the batch code reuses.
#pragma once

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

// The calling thread's last error message (vjb_last_error) and the helper
// that sets it and returns `code`.
extern thread_local char g_err[512];
int fail(int code, const char *fmt, ...);

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
// A timed round: its events and the one that ends it (its own third event, or
// the next round's start when rounds follow each other in one call).
struct PendingRound {
    EventTriple ev;
    cudaEvent_t end;
};

}  // namespace vjb

// Both library units work in the vjb names.
using namespace vjb;

// One training context (the C ABI's vjb_ctx): its device buffers and state.
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
    void *d_runres = nullptr;        // re-scan: lane-run results of the split features
    uint32_t *d_cand_runs = nullptr;  // re-scan: runs done per split feature (kept at zero between rounds)
    uint8_t *d_miss = nullptr;
    int32_t *d_scratch = nullptr;  // table preparation: check state and listed rows
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

    // graph of one round; with timing on, of its search (graph) and of the
    // rest (graph2), launched with the timing events between them
    cudaGraph_t graph = nullptr, graph2 = nullptr;
    cudaGraphExec_t gexec = nullptr, gexec2 = nullptr;
    bool graph_timed = false;

    bool timing = false;
    std::vector<EventTriple> ev_free;
    std::vector<PendingRound> ev_pending;
    vjb_timing tacc{};

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gexec2) cudaGraphExecDestroy(gexec2);
        if (graph) cudaGraphDestroy(graph);
        if (graph2) cudaGraphDestroy(graph2);
        gexec = gexec2 = nullptr;
        graph = graph2 = nullptr;
    }
    void free_all() {
        drop_graph();
        dfree(d_px); dfree(d_y); dfree(d_ii); dfree(d_feat);
        if (rows_external) d_rows = nullptr;
        dfree(d_rows);
        rows_external = false;
        dfree(d_w); dfree(d_v); dfree(d_wtmp); dfree(d_ferr); dfree(d_bmin); dfree(d_cand);
        dfree(d_cand_ids); dfree(d_runres); dfree(d_cand_runs); dfree(d_miss); dfree(d_partials); dfree(d_scratch);
        dfree(d_rs); dfree(d_stumps); dfree(d_last); dfree(d_diag);
        stump_cap = bmin_cap = 0;
        feats.clear();
        stage = kStageNone;
        tmap_ok = false;
        n = h = w = ii_stride = npad = lines = box_lines = 0;
        nfeat = 0;
        lay = WeightLayout{};
    }
    // the integral images modulo 2^16, stored after the int32 ones in d_ii
    uint16_t *ii16() const {
        return d_ii ? reinterpret_cast<uint16_t *>(d_ii + (size_t)(h + 1) * (w + 1) * ii_stride) : nullptr;
    }
    void free_events() {
        for (auto &t : ev_free) for (auto e : t) cudaEventDestroy(e);
        for (auto &t : ev_pending) for (auto e : t.ev) cudaEventDestroy(e);
        ev_free.clear();
        ev_pending.clear();
    }
};

namespace vjb {

// Context helpers (vjb_api.cu) that the batch and serving code reuse.
void enumerate_host(int w, int h, std::vector<vjb_feature> &out);
int ensure_stump_cap(vjb_ctx *c, int need);
JobDesc job_desc(const vjb_ctx *c);
int validate_labels(const uint8_t *y, int n);

}  // namespace vjb
