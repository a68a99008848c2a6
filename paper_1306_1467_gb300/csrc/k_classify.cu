// The strong classifier of Sec. 2.3 (the final hypothesis) applied to windows:
//     C(x) = 1  iff  sum_t alpha_t h_t(x) >= 1/2 sum_t alpha_t,
// h_t(x) = 1 iff p_t f_t(x) < p_t theta_t.  One thread per window; the stumps
// (feature geometry, threshold, polarity, alpha) are staged in shared memory
// a block at a time and every thread adds its alpha_t in FP64 in stump order,
// so the score of a window does not depend on the launch shape.
#include <math.h>

#include "vjb_device.cuh"
#include "vjb_haar.cuh"
#include "vjb_internal.cuh"

namespace vjb {

constexpr int kClassifyThreads = 256;
constexpr int kClassifyStage = 256;  // stumps per shared-memory block

struct ClassStump {
    DevFeature f;
    int32_t threshold, polarity;
    double alpha;
};

__global__ void __launch_bounds__(kClassifyThreads)
    k_strong_classify(const int32_t *__restrict__ ii_t, int ii_stride, int n, int win_w,
                      const DevFeature *__restrict__ feat, const vjb_stump *__restrict__ stumps, int T,
                      double half_alpha, uint8_t *__restrict__ labels, double *__restrict__ scores) {
    __shared__ ClassStump sst[kClassifyStage];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    for (int t0 = 0; t0 < T; t0 += kClassifyStage) {
        const int m = min(kClassifyStage, T - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const vjb_stump st = stumps[t0 + k];
            sst[k] = ClassStump{feat[st.feature], st.threshold, st.polarity, st.alpha};
        }
        __syncthreads();
        if (i < n)
            for (int k = 0; k < m; ++k) {
                const ClassStump &c = sst[k];
                const int32_t v = haar_value(ii_t, ii_stride, win_w, c.f.type, c.f.x, c.f.y, c.f.w, c.f.h, i);
                const bool h = c.polarity > 0 ? (v < c.threshold) : (v > c.threshold);
                if (h) s += c.alpha;
            }
    }
    if (i < n) {
        labels[i] = s >= half_alpha ? 1 : 0;
        if (scores) scores[i] = s;
    }
}

cudaError_t launch_strong_classify(const int32_t *ii_t, int ii_stride, int n, int win_w, const DevFeature *feat,
                                   const vjb_stump *stumps, int T, double half_alpha, uint8_t *labels,
                                   double *scores, cudaStream_t st) {
    const int grid = (n + kClassifyThreads - 1) / kClassifyThreads;
    k_strong_classify<<<grid, kClassifyThreads, 0, st>>>(ii_t, ii_stride, n, win_w, feat, stumps, T, half_alpha,
                                                         labels, scores);
    return cudaGetLastError();
}

}  // namespace vjb
