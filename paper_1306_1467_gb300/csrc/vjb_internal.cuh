// Internal declarations shared by the library's translation units: device
// data layouts, the per-round state record and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vjb.h"

namespace vjb {

// Feature descriptor as the kernels read it (8 bytes, one load).
struct DevFeature {
    uint8_t type, x, y, w, h, pad0, pad1, pad2;
};

// Where the signed weights v_i (+w_i for a face, -w_i for a non-face) live.
// Table entries are word offsets into this array.  With two copies, copy A
// holds v_i at word i and copy B at word off_b + rot(i), where rot rotates
// each aligned block of 32 samples by 13 * (block number): the two copies put
// a sample in unrelated shared-memory banks, and the sort kernel picks, for
// every group of 32 entries one gather instruction reads, the copy of each
// entry that balances the banks.  Word n holds 0 and is the padding entry.
struct WeightLayout {
    int n;
    int dual;    // 1: a copy B exists, 0: copy A only
    int off_b;   // first word of copy B (a multiple of 32), 0 without it
    int words;   // array length in floats
    int nb;      // samples 0 .. nb-1 have a copy B (nb = n unless 15-bit offsets run out)
};

__host__ __device__ __forceinline__ int rot_b(int i) {
    return (i & ~31) | ((i + 13 * (i >> 5)) & 31);
}
__host__ __device__ __forceinline__ int unrot_b(int r) {
    return (r & ~31) | ((r - 13 * (r >> 5)) & 31);
}
// Sample named by a table word (n for the padding word).
__host__ __device__ __forceinline__ int word_to_sample(int word, const WeightLayout &L) {
    if (L.dual && word >= L.off_b) return unrot_b(word - L.off_b);
    return word;
}

// Round state that lives on the device between the kernels of a round.
struct RoundState {
    double t_pos;        // FP64 sum of the FP32 weights of faces
    double t_neg;        // same for non-faces
    double weight_sum;   // t_pos + t_neg
    double scale_hit;    // beta / updated total: factor for correctly classified samples
    double scale_miss;   // 1 / updated total: factor for misclassified samples
    int32_t status;      // VJB_OK or VJB_DONE_*
    int32_t rounds;      // stumps kept so far
    int32_t cand_count;  // shortlisted features of the current search
    int32_t last_cands;  // shortlist size of the last finished search
    int32_t flags;       // error flags (kFlag*)
    float screen_min;    // smallest screened error of the last search
    int32_t forced;      // 1 while a host-given stump replaces the search
    int32_t forced_feature, forced_threshold, forced_polarity;
    int32_t win_feature, win_split, win_polarity;  // the round's stump
    uint32_t done_rescan, done_update_a, done_update_b;  // last-CTA counters
    float win_err_hi, win_err_lo;  // the stump's error from the compensated re-scan
    uint32_t screen_min_bits;  // batched search: smallest screened error (bits of a float >= 0)
    int32_t in_round;          // batched rounds: 1 if the job takes part in the current round
    int32_t win_theta;         // the searched stump's threshold (set by the update's first block)
};

// Device error flags.
constexpr int32_t kFlagWaitTimeout = 1;   // an mbarrier wait gave up
constexpr int32_t kFlagNoCandidate = 2;   // the shortlist was empty
constexpr int32_t kFlagBadWeights = 4;    // weight total not positive / finite
constexpr int32_t kFlagBadTable = 8;      // a sorted-table entry out of range

// One shortlisted feature after the compensated re-scan.
struct Candidate {
    float err_hi, err_lo;  // double-float weighted error
    int32_t feature;
    int32_t split;
    int32_t polarity;
    int32_t pad;
};

// Search-kernel geometry: rows of the sorted table are viewed as 128-byte
// lines of 64 uint16 entries; a TMA box is up to 32 lines (4 KiB).
constexpr int kLineElems = 64;
constexpr int kLineBytes = 128;
constexpr int kBoxLinesMax = 32;
constexpr int kStageBytes = kBoxLinesMax * kLineBytes;  // 4096
constexpr int kUnitElems = 512;                         // 32 lanes x 16 entries

// Row layout of the sorted table.  A row holds npad entries (n rounded up to
// a multiple of 256; entries from n on are padding).  The value order is cut
// into 32 runs of npad / 32 entries, one per lane of the warp that scans the
// row, and the runs are interleaved in 16-byte chunks of 8 entries: chunk t of
// run k is chunk t * 32 + k of the row.  A 512-byte "chunk row" thus holds the
// next 8 entries of every run, and a lane reading chunk t * 32 + lane walks its
// own run in order.
constexpr int kRowAlign = 256;
constexpr int kChunkElems = 8;
__host__ __device__ __forceinline__ int phys_of(int e, int run) {
    const int k = e / run, r = e - k * run;
    return ((r >> 3) * 32 + k) * kChunkElems + (r & 7);
}
__host__ __device__ __forceinline__ int logical_of(int phys, int run) {
    const int c = phys >> 3;
    return (c & 31) * run + (c >> 5) * kChunkElems + (phys & 7);
}
constexpr uint16_t kFlagBit = 0x8000u;
constexpr uint16_t kIndexMask = 0x7FFFu;
// Table entries are 15-bit weight-word offsets with a split flag, packed by
// physical position: an entry at an even position is word | flag << 15, one at
// an odd position (the high half of a 32-bit word) word << 1 | flag, so that a
// 32-bit pair gives its high word with one shift.  Padding: word n, no flag.
__host__ __device__ __forceinline__ uint16_t make_entry(int word, bool flag, int phys) {
    return (phys & 1) ? (uint16_t)((word << 1) | (flag ? 1 : 0)) : (uint16_t)(word | (flag ? kFlagBit : 0));
}
__host__ __device__ __forceinline__ int entry_word(uint32_t e, int phys) {
    return (phys & 1) ? (int)((e & 0xffffu) >> 1) : (int)(e & kIndexMask);
}
__host__ __device__ __forceinline__ bool entry_flag(uint32_t e, int phys) {
    return (phys & 1) ? (e & 1u) != 0 : (e & kFlagBit) != 0;
}

// Margin (in units of 2^-24 times the weight total) within which a feature's
// FP32 screened error must lie of the smallest one to be re-scanned
// compensated.  It is twice a bound on the screening error (see k_search.cu).
constexpr float kScreenMarginUlps = 72.0f;

// The plain re-scan spreads the first kRescanSplitCap shortlisted features'
// lane runs over the grid, one run per warp; later ones (a tie plateau) are
// re-scanned whole by one CTA each.  A run result is 32 bytes.
constexpr int kRescanSplitCap = 256;
constexpr int kRunResultBytes = 32;

// Partials of the multi-CTA update kernels (one slot per CTA).
constexpr int kUpdateThreads = 256;
constexpr int kUpdateMaxCtas = 4096;

// Everything the round kernels need about one training job.  The plain
// kernels get it by value; a batch keeps one per job in device memory.
struct JobDesc {
    const uint16_t *rows;  // sorted table [nfeat][npad], lane-run layout
    int npad, lines;       // row length in entries and in 128-byte lines
    int64_t nfeat;
    int64_t line_base;     // batch: first line of the table in the batch's table arena
    WeightLayout lay;
    float *v;              // signed weights, lay.words floats
    float *w;              // FP32 weights [n]
    const uint8_t *y;
    uint8_t *miss;
    double *partials;      // 3 * kUpdateMaxCtas
    RoundState *rs;
    float *ferr;
    int32_t *cand_ids;
    struct Candidate *cands;
    struct RunResult *runres;  // plain re-scan: lane-run results [kRescanSplitCap][32]
    uint32_t *cand_runs;       // plain re-scan: runs done per candidate [kRescanSplitCap]
    vjb_stump *stumps;
    vjb_round_diag *diag;
    vjb_stump *last;
    int32_t stump_cap;
    int32_t ii_stride;
    const int32_t *ii;
    const DevFeature *feat;
    int32_t win_w;         // window width
    int32_t active;        // batch: 1 if the job is trained by the batch
    int32_t round_target;  // batch: train while rounds < round_target
    int32_t ublock_base;   // batch: update blocks of the jobs before this one
    int64_t feat_base;     // batch: features of the jobs before this one
};

// Batch-wide counters in device memory.
constexpr int kMaxScreenCtas = 1024;
struct BatchMeta {
    int32_t njobs;          // job slots in use
    int32_t n_items;        // search work items
    uint32_t item_next;     // next work item (reset by the last CTA of the search)
    uint32_t screen_done;   // CTAs done with the search
    int64_t total_feat;     // sum of nfeat over the job slots
    int32_t total_ublocks;  // sum of update blocks over the job slots
    int32_t flags;          // error flags of batched kernels
    int32_t screen_ctas;    // CTAs of the partitioned search
    int32_t pad;
    // partitioned search: CTA c takes rows [cta_start[c], cta_start[c + 1]) of
    // the jobs' rows in job order (row g of job j is g - feat_base_j), set each
    // round by k_bbegin so that every CTA gets the same share of table lines
    int64_t cta_start[kMaxScreenCtas + 1];
};

// A search work item: features [f0, f1) of one job.
struct WorkItem {
    int32_t job, f0, f1, pad;
};

constexpr int kMaxBatchJobs = 256;

struct SearchShape {
    int warps;        // consumer warps per CTA
    int stages;       // TMA stages per warp
    int ctas_per_sm;
    int unroll;       // 512-entry units a warp works on together (1, 2 or 4)
    int box_lines;    // 128-byte lines per TMA box (8, 16 or 32)
};

size_t search_smem_bytes(const SearchShape &s, int words);
WeightLayout make_layout(int n, bool allow_dual);

// Launchers (each returns the launch error).
cudaError_t launch_integral(const uint8_t *px, int n, int h, int w, int32_t *ii_t, uint16_t *ii16,
                            int ii_stride, cudaStream_t st);
cudaError_t launch_strong_classify(const int32_t *ii_t, int ii_stride, int n, int win_w, const DevFeature *feat,
                                   const vjb_stump *stumps, int T, double half_alpha, uint8_t *labels,
                                   double *scores, cudaStream_t st);
cudaError_t launch_feature_values(const int32_t *ii_t, int ii_stride, int n, int w,
                                  const DevFeature *feat, int64_t f0, int64_t nf, int32_t *out,
                                  cudaStream_t st);
cudaError_t launch_sort_rows(const int32_t *ii_t, const uint16_t *ii16, int ii_stride, int w,
                             const DevFeature *feat, int64_t f0, int64_t nf, const WeightLayout &L, uint16_t *rows,
                             int npad, int32_t *scratch, cudaStream_t st);
cudaError_t launch_init_weights(const uint8_t *y, const WeightLayout &L, const float *w_in,
                                float *w, float *v, RoundState *rs, cudaStream_t st);
cudaError_t launch_screen(const CUtensorMap *tmap, const float *v, const WeightLayout &L,
                          int lines_per_row, int box_lines, int64_t nfeat, const SearchShape &shape,
                          int grid, RoundState *rs, float *ferr, float *bmin, cudaStream_t st);
cudaError_t launch_shortlist(const JobDesc &J, const float *bmin, int nbmin, int grid, cudaStream_t st);
cudaError_t launch_rescan(const JobDesc &J, int grid, cudaStream_t st);
cudaError_t launch_update_a(const JobDesc &J, cudaStream_t st);
cudaError_t launch_update_b(const JobDesc &J, cudaStream_t st);
// batched rounds over the jobs of a device job table
// The table arena as [lines][64 entries]: m[0] loads a whole stage of the
// batched search (its box is the stage height S); m[k], 0 < k < S / 4, loads
// 4k lines (the tail of a row).  One copy per stage either way.
constexpr int kBatchMaps = kBoxLinesMax / 4;
struct BatchMaps {
    CUtensorMap m[kBatchMaps];
};
cudaError_t launch_bbegin(JobDesc *jobs, BatchMeta *meta, cudaStream_t st);
cudaError_t launch_bscreen(const BatchMaps &maps, const JobDesc *jobs, const WorkItem *items,
                           BatchMeta *meta, int max_words, const SearchShape &shape, int schedule,
                           int grid, cudaStream_t st);
cudaError_t launch_bshortlist(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st);
cudaError_t launch_brescan(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st);
cudaError_t launch_bupdate_a(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st);
cudaError_t launch_bupdate_b(const JobDesc *jobs, BatchMeta *meta, int grid, cudaStream_t st);
size_t bscreen_smem_bytes(const SearchShape &s, int max_words);
cudaError_t set_bscreen_smem_limit(int bytes);
int update_grid(int n);

}  // namespace vjb
