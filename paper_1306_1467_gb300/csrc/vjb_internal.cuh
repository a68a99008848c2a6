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

// Round state that lives on the device between the kernels of a round.
struct RoundState {
    double t_pos;        // FP64 sum of the FP32 weights of faces
    double t_neg;        // same for non-faces
    double weight_sum;   // t_pos + t_neg
    int32_t status;      // VJB_OK or VJB_DONE_*
    int32_t rounds;      // stumps kept so far
    int32_t cand_count;  // shortlist entries written by the refine kernel
    int32_t last_cands;  // shortlist size of the last finished search
    int32_t flags;       // error flags (kFlag*)
    float screen_min;    // smallest screened error of the last search
    int32_t forced;      // 1 while a host-given stump replaces the search
    int32_t forced_feature, forced_threshold, forced_polarity;
    int32_t pad;
};

// Device error flags.
constexpr int32_t kFlagWaitTimeout = 1;   // an mbarrier wait gave up
constexpr int32_t kFlagNoCandidate = 2;   // the refine kernel found no feature
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
constexpr uint16_t kFlagBit = 0x8000u;
constexpr uint16_t kIndexMask = 0x7FFFu;

// Margin (in units of 2^-24 times the weight total) within which a feature's
// FP32 screened error must lie of the smallest one to be re-scanned
// compensated.  It is twice a bound on the screening error (see k_search.cu).
constexpr float kScreenMarginUlps = 64.0f;

struct SearchShape {
    int warps;        // consumer warps per CTA
    int stages;       // TMA stages per warp
    int ctas_per_sm;
};

size_t search_smem_bytes(const SearchShape &s, int n);

// Launchers (each returns the launch error).
cudaError_t launch_integral(const uint8_t *px, int n, int h, int w, int32_t *ii_t, int ii_stride,
                            cudaStream_t st);
cudaError_t launch_feature_values(const int32_t *ii_t, int ii_stride, int n, int w,
                                  const DevFeature *feat, int64_t f0, int64_t nf, int32_t *out,
                                  cudaStream_t st);
cudaError_t launch_sort_rows(const int32_t *vals, int n, int64_t nf, uint16_t *rows, int npad,
                             cudaStream_t st);
cudaError_t launch_check_rows(const uint16_t *rows, int64_t nfeat, int n, int npad, int32_t *flags,
                              int grid, cudaStream_t st);
cudaError_t launch_init_weights(const uint8_t *y, int n, const float *w_in, float *w, float *v,
                                RoundState *rs, cudaStream_t st);
cudaError_t launch_screen(const CUtensorMap *tmap, const float *v, int n, int lines_per_row,
                          int box_lines, int64_t nfeat, const SearchShape &shape, int grid,
                          RoundState *rs, float *ferr, float *bmin, cudaStream_t st);
cudaError_t launch_refine(const uint16_t *rows, int npad, int n, int64_t nfeat, const float *v,
                          RoundState *rs, const float *ferr, const float *bmin, int nbmin,
                          Candidate *cands, int grid, cudaStream_t st);
cudaError_t launch_finalize(const uint16_t *rows, int npad, int n, const int32_t *ii_t,
                            int ii_stride, int w, const DevFeature *feat, int64_t nfeat,
                            const uint8_t *y, float *wts, float *v, RoundState *rs,
                            const Candidate *cands, vjb_stump *stumps, int stump_cap,
                            vjb_stump *last, cudaStream_t st);

}  // namespace vjb
