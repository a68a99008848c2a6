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
    int dual;    // 1: two copies, 0: copy A only
    int off_b;   // first word of copy B (a multiple of 32), 0 without it
    int words;   // array length in floats
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
    int32_t pad;
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

// Margin (in units of 2^-24 times the weight total) within which a feature's
// FP32 screened error must lie of the smallest one to be re-scanned
// compensated.  It is twice a bound on the screening error (see k_search.cu).
constexpr float kScreenMarginUlps = 64.0f;

// Partials of the multi-CTA update kernels (one slot per CTA).
constexpr int kUpdateThreads = 256;
constexpr int kUpdateMaxCtas = 4096;

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
cudaError_t launch_integral(const uint8_t *px, int n, int h, int w, int32_t *ii_t, int ii_stride,
                            cudaStream_t st);
cudaError_t launch_feature_values(const int32_t *ii_t, int ii_stride, int n, int w,
                                  const DevFeature *feat, int64_t f0, int64_t nf, int32_t *out,
                                  cudaStream_t st);
cudaError_t launch_sort_rows(const int32_t *ii_t, int ii_stride, int w, int h, const DevFeature *feat,
                             int64_t f0, int64_t nf, const WeightLayout &L, uint16_t *rows, int npad,
                             int32_t *flags, cudaStream_t st);
cudaError_t launch_check_rows(const uint16_t *rows, int64_t nfeat, const WeightLayout &L, int npad,
                              int32_t *flags, int grid, cudaStream_t st);
cudaError_t launch_init_weights(const uint8_t *y, const WeightLayout &L, const float *w_in,
                                float *w, float *v, RoundState *rs, cudaStream_t st);
cudaError_t launch_screen(const CUtensorMap *tmap, const float *v, const WeightLayout &L,
                          int lines_per_row, int box_lines, int64_t nfeat, const SearchShape &shape,
                          int grid, RoundState *rs, float *ferr, float *bmin, cudaStream_t st);
cudaError_t launch_shortlist(int64_t nfeat, RoundState *rs, const float *ferr, const float *bmin,
                             int nbmin, int32_t *cand_ids, int grid, cudaStream_t st);
cudaError_t launch_rescan(const uint16_t *rows, int npad, const float *v, const WeightLayout &L,
                          RoundState *rs, const int32_t *cand_ids, Candidate *cands, int grid,
                          cudaStream_t st);
cudaError_t launch_update_a(const uint16_t *rows, int npad, const WeightLayout &L,
                            const int32_t *ii_t, int ii_stride, int w, const DevFeature *feat,
                            const uint8_t *y, const float *wts, uint8_t *miss, double *partials,
                            RoundState *rs, vjb_stump *stumps, vjb_round_diag *diag, int stump_cap,
                            vjb_stump *last, const float *ferr, cudaStream_t st);
cudaError_t launch_update_b(const WeightLayout &L, const uint8_t *y, float *wts, float *v,
                            const uint8_t *miss, double *partials, RoundState *rs,
                            cudaStream_t st);
int update_grid(int n);

}  // namespace vjb
