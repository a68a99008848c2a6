// One-time preparation kernels: integral images (Sec. 2.1), int32 Haar feature
// values (Sec. 2.2) and the per-feature stable sample order that the round
// search scans (the threshold search of Sec. 2.2-2.3 needs the samples of a
// feature in value order).
#include <limits.h>

#include <type_traits>

#include "vjb_device.cuh"
#include "vjb_haar.cuh"
#include "vjb_internal.cuh"

namespace vjb {

// ---- K1: integral images --------------------------------------------------------
// One thread per window.  Output is point-major, ii_t[(y * (w + 1) + x) * stride + i],
// so that the feature kernel reads consecutive windows with coalesced loads.
// ii(x, y) = sum of pixels with x' < x and y' < y (zero first row and column),
// built row by row: ii(x, y) = ii(x, y - 1) + (sum of row y - 1 up to x - 1).
// With ii16 non-null, also the values modulo 2^16 in the same layout (the
// sort evaluates features of small boxes from these).
__global__ void k_integral(const uint8_t *__restrict__ px, int n, int h, int w,
                           int32_t *__restrict__ ii_t, uint16_t *__restrict__ ii16, int stride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int W1 = w + 1;
    const uint8_t *img = px + (size_t)i * h * w;
    for (int x = 0; x <= w; ++x) {
        ii_t[(size_t)x * stride + i] = 0;
        if (ii16) ii16[(size_t)x * stride + i] = 0;
    }
    for (int y = 1; y <= h; ++y) {
        ii_t[(size_t)(y * W1) * stride + i] = 0;
        if (ii16) ii16[(size_t)(y * W1) * stride + i] = 0;
        int32_t row = 0;
        for (int x = 1; x <= w; ++x) {
            row += img[(y - 1) * w + (x - 1)];
            const int32_t up = ii_t[(size_t)((y - 1) * W1 + x) * stride + i];
            ii_t[(size_t)(y * W1 + x) * stride + i] = up + row;
            if (ii16) ii16[(size_t)(y * W1 + x) * stride + i] = (uint16_t)(up + row);
        }
    }
}

cudaError_t launch_integral(const uint8_t *px, int n, int h, int w, int32_t *ii_t, uint16_t *ii16,
                            int ii_stride, cudaStream_t st) {
    const int b = 128;
    k_integral<<<(n + b - 1) / b, b, 0, st>>>(px, n, h, w, ii_t, ii16, ii_stride);
    return cudaGetLastError();
}

// ---- K2: feature values ------------------------------------------------------------
// One CTA per feature; threads stride over windows.  out[(f - f0) * n + i].
__global__ void k_feature_values(const int32_t *__restrict__ ii_t, int stride, int n, int w,
                                 const DevFeature *__restrict__ feat, int64_t f0,
                                 int32_t *__restrict__ out) {
    const DevFeature d = feat[f0 + blockIdx.x];
    int32_t *o = out + (size_t)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        o[i] = haar_value(ii_t, stride, w, d.type, d.x, d.y, d.w, d.h, i);
}

cudaError_t launch_feature_values(const int32_t *ii_t, int ii_stride, int n, int w,
                                  const DevFeature *feat, int64_t f0, int64_t nf, int32_t *out,
                                  cudaStream_t st) {
    if (nf <= 0) return cudaSuccess;
    k_feature_values<<<(unsigned)nf, 256, 0, st>>>(ii_t, ii_stride, n, w, feat, f0, out);
    return cudaGetLastError();
}

// ---- K3: segmented stable sort ---------------------------------------------------------
// One 1024-thread CTA per feature row.  The CTA first evaluates its feature on
// every window (the K2 arithmetic, fused here so the int32 values never leave
// the SM), then sorts keys value - min (non-negative) by an LSD radix sort with
// 8-bit digits over only the bits the row's value span needs.  Each pass ranks
// digits stably: items are held in registers in a "warp-striped" layout (warp
// wp, column j, lane l -> position wp*32*IPT + j*32 + l), a warp walks its
// columns in position order and ranks equal digits inside a column, and the
// per-(digit, warp) counts are scanned digit-major.  Equal keys therefore keep
// their order, and since items start in sample order, ties end up ordered by
// sample index.  Output entry = weight word | (value < next value) << 15,
// written in the lane-run row layout; positions n .. npad-1 hold the padding
// word n (weight 0, no flag).
constexpr int kSortThreads = 1024;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadix = 256;
constexpr int kHistStride = kSortWarps + 1;  // (digit, warp) counters, padded against bank conflicts
constexpr int kHistWords = kRadix * kHistStride;
// Gather groups of a row with two weight copies (n <= 16352): one per entry
// of a lane run, at most 16384 / 32.  Their masks sit after the histogram and
// the per-thread bank loads (32 bytes each) reuse the histogram space.
constexpr int kMaxGroups = 512;
static_assert(kSortThreads * 32 / 4 <= kHistWords, "histogram space too small for bank loads");

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// End of a row's write (all threads of the CTA): count the row and flag an
// entry before position n whose word lies outside the weight array or is the
// padding word.  The search kernels gather weights through the table without
// bounds checks; the host accepts a table only if no entry was flagged and
// every row was counted.  stat[0]: kFlagBadTable or 0, stat[1]: rows written.
__device__ __forceinline__ void row_written(bool bad, int32_t *stat) {
    const int any_bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        if (any_bad) atomicOr(&stat[0], kFlagBadTable);
        atomicAdd(&stat[1], 1);
    }
}

// Lanes of the warp holding the same BITS-bit digit `d` as this lane: one
// ballot per digit bit, each narrowing the set to the lanes that agree on that
// bit.  On this GPU BITS ballots (four instructions a bit) rank a sort pass
// faster than one __match_any_sync: 29.8 vs 31.7 ms for the 24x24 / 15k
// tables.
template <int BITS>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
    uint32_t eq = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        uint32_t m;
        asm("{\n\t.reg .pred p;\n\t"
            "and.b32 %0, %1, %2;\n\t"
            "setp.ne.u32 p, %0, 0;\n\t"
            "vote.sync.ballot.b32 %0, p, 0xffffffff;\n\t"
            "@!p not.b32 %0, %0;\n\t}"
            : "=r"(m)
            : "r"(d), "r"(1u << b));
        eq &= m;
    }
    return eq;
}

// Exclusive scan of one int per thread over the CTA; returns the thread's
// exclusive prefix.  `ws` holds kSortWarps ints.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *ws) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) ws[wp] = inc;
    __syncthreads();
    if (wp == 0) {
        uint32_t t = ws[lane];
        uint32_t ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, d);
            if (lane >= d) ti += y;
        }
        ws[lane] = ti - t;
    }
    __syncthreads();
    const uint32_t r = ws[wp] + inc - x;
    __syncthreads();
    return r;
}

template <int IPT>
__global__ void __launch_bounds__(kSortThreads, 1)
    k_sort_rows(const int32_t *__restrict__ ii_t, int ii_stride, int w,
                const DevFeature *__restrict__ feat, int64_t f0, WeightLayout L,
                uint16_t *__restrict__ rows, int npad, const int32_t *__restrict__ row_list, int32_t *stat) {
    const int row = row_list ? row_list[blockIdx.x] : (int)blockIdx.x;  // row of the tile
    constexpr int NP = kSortThreads * IPT;
    const int n = L.n;
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *skey = reinterpret_cast<uint32_t *>(smem);
    uint32_t *hist = skey + NP;                                            // kHistWords (+ kMaxGroups)
    uint32_t *ws = hist + kHistWords + (IPT <= 16 ? kMaxGroups : 0);        // kSortWarps
    int32_t *mm = reinterpret_cast<int32_t *>(ws + kSortWarps);             // 2
    uint16_t *sidx = reinterpret_cast<uint16_t *>(mm + 2);                  // NP

    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int pos0 = wp * 32 * IPT + lane;
    const DevFeature d = feat[f0 + row];

    // the feature on every window, into shared memory (K2's arithmetic)
    int32_t lo = INT_MAX, hi = INT_MIN;
    for (int p = threadIdx.x; p < n; p += kSortThreads) {
        const int32_t x = haar_value(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, p);
        skey[p] = static_cast<uint32_t>(x);
        lo = min(lo, x);
        hi = max(hi, x);
    }
    __syncthreads();
    uint32_t key[IPT];
    uint32_t ipk[(IPT + 1) / 2];  // two 16-bit sample indices per register
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int p = pos0 + j * 32;
        key[j] = p < n ? skey[p] : 0u;
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if (threadIdx.x == 0) { mm[0] = INT_MAX; mm[1] = INT_MIN; }
    __syncthreads();
    if (lane == 0) { atomicMin(&mm[0], lo); atomicMax(&mm[1], hi); }
    __syncthreads();
    lo = mm[0];
    hi = mm[1];
    const uint32_t span = static_cast<uint32_t>(hi) - static_cast<uint32_t>(lo);
    const int bits = span ? 32 - __clz(span) : 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int p = pos0 + j * 32;
        // padding items take the all-ones key: they sort after every real item
        key[j] = (p < n) ? key[j] - static_cast<uint32_t>(lo) : 0xffffffffu;
        if (j & 1) ipk[j >> 1] |= static_cast<uint32_t>(p) << 16;
        else ipk[j >> 1] = static_cast<uint32_t>(p) & 0xffffu;
    }

    const uint32_t lt = lanemask_lt();
    for (int shift = 0; shift < bits; shift += 8) {
        for (int k = threadIdx.x; k < kHistWords; k += kSortThreads) hist[k] = 0;
        __syncthreads();
        // count digits per (digit, warp)
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t dg = (key[j] >> shift) & (kRadix - 1);
            const uint32_t peers = digit_peers<8>(dg);
            if (lane == __ffs(peers) - 1) hist[dg * kHistStride + wp] += __popc(peers);
        }
        __syncthreads();
        // exclusive scan, digit-major then warp: thread t owns 8 consecutive counters
        {
            constexpr int PER = kRadix * kSortWarps / kSortThreads;  // 8
            uint32_t c[PER];
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int lin = threadIdx.x * PER + q;
                c[q] = hist[(lin >> 5) * kHistStride + (lin & 31)];
                s += c[q];
            }
            uint32_t off = block_exclusive_scan(s, ws);
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int lin = threadIdx.x * PER + q;
                hist[(lin >> 5) * kHistStride + (lin & 31)] = off;
                off += c[q];
            }
        }
        __syncthreads();
        // scatter in position order
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t dg = (key[j] >> shift) & (kRadix - 1);
            const uint32_t peers = digit_peers<8>(dg);
            const uint32_t base = hist[dg * kHistStride + wp];
            __syncwarp();
            if (lane == __ffs(peers) - 1) hist[dg * kHistStride + wp] = base + __popc(peers);
            __syncwarp();
            const uint32_t dst = base + __popc(peers & lt);
            skey[dst] = key[j];
            sidx[dst] = static_cast<uint16_t>((j & 1) ? (ipk[j >> 1] >> 16) : (ipk[j >> 1] & 0xffffu));
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int p = pos0 + j * 32;
            key[j] = skey[p];
            const uint32_t ix = sidx[p];
            if (j & 1) ipk[j >> 1] = (ipk[j >> 1] & 0xffffu) | (ix << 16);
            else ipk[j >> 1] = ix;
        }
        __syncthreads();
    }
    // make the final order visible in shared memory (also when no pass ran)
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int p = pos0 + j * 32;
        skey[p] = key[j];
        sidx[p] = static_cast<uint16_t>((j & 1) ? (ipk[j >> 1] >> 16) : (ipk[j >> 1] & 0xffffu));
    }
    __syncthreads();
    uint16_t *out = rows + (size_t)row * npad;
    const int run = npad / 32;  // entries per lane run (see phys_of)
    if (L.dual) {
        // With two weight copies, choose per entry which copy the search
        // gathers from.  One gather instruction of the search kernel reads
        // entry r of every lane run: the 32 entries k * run + r, k = 0..31.
        // For each such group, greedily put each entry that has a copy B
        // (samples below L.nb) in the less loaded of its two banks (copy A:
        // i mod 32, copy B: rot(i) mod 32), then let such entries move to a
        // lighter bank.  Bank loads are kept per thread, bank-major so that
        // the threads do not share banks.  The split flags first go into bit 15
        // of the sample indices (n <= 32767), which frees the keys' space for
        // the choices of the 32-item variant.
        for (int p = threadIdx.x; p < n; p += kSortThreads)
            if (p == n - 1 || skey[p] < skey[p + 1]) sidx[p] |= 0x8000u;
        __syncthreads();
        uint32_t *gchoice = IPT <= 16 ? hist + kRadix * kSortWarps : skey;  // one mask per group
        uint8_t *ld = reinterpret_cast<uint8_t *>(hist) + threadIdx.x;
        for (int g = threadIdx.x; g < run; g += kSortThreads) {
#pragma unroll
            for (int b = 0; b < 32; ++b) ld[b * kSortThreads] = 0;
            uint32_t mask = 0;
            bool pad_seen = false;
            for (int k = 0; k < 32; ++k) {
                const int p = k * run + g;
                if (p >= n) {
                    if (!pad_seen) ld[(n & 31) * kSortThreads]++;  // padding: one broadcast read
                    pad_seen = true;
                    continue;
                }
                const int i = sidx[p] & 0x7fff;
                const int ba = i & 31, bb = rot_b(i) & 31;
                if (i < L.nb && ld[bb * kSortThreads] < ld[ba * kSortThreads]) {
                    ld[bb * kSortThreads]++;
                    mask |= 1u << k;
                } else {
                    ld[ba * kSortThreads]++;
                }
            }
            // two passes of single moves: an entry leaves its bank when the
            // other one is at least two entries lighter
            for (int pass = 0; pass < 2; ++pass)
                for (int k = 0; k < 32; ++k) {
                    const int p = k * run + g;
                    if (p >= n) break;
                    const int i = sidx[p] & 0x7fff;
                    if (i >= L.nb) continue;
                    const int ba = i & 31, bb = rot_b(i) & 31;
                    const bool onb = (mask >> k) & 1u;
                    const int cur = onb ? bb : ba, oth = onb ? ba : bb;
                    if (ld[cur * kSortThreads] > ld[oth * kSortThreads] + 1) {
                        ld[cur * kSortThreads]--;
                        ld[oth * kSortThreads]++;
                        mask ^= 1u << k;
                    }
                }
            gchoice[g] = mask;
        }
        __syncthreads();
        bool bad = false;
        for (int P = threadIdx.x; P < npad; P += kSortThreads) {
            const int p = logical_of(P, run);
            uint16_t e;
            if (p < n) {
                const uint32_t x = sidx[p];
                int word = (int)(x & 0x7fffu);
                const int k = (P >> 3) & 31, g = (P >> 8) * kChunkElems + (P & 7);  // p = k * run + g
                if ((gchoice[g] >> k) & 1u) word = L.off_b + rot_b(word);
                bad |= word >= L.words || word == n;
                e = make_entry(word, (x & 0x8000u) != 0, P);
            } else {
                e = make_entry(n, false, P);
            }
            out[P] = e;
        }
        row_written(bad, stat);
        return;
    }
    bool bad = false;
    for (int P = threadIdx.x; P < npad; P += kSortThreads) {
        const int p = logical_of(P, run);
        uint16_t e;
        if (p < n) {
            const bool step = (p == n - 1) || (skey[p] < skey[p + 1]);
            bad |= (int)sidx[p] >= L.words || (int)sidx[p] == n;
            e = make_entry(sidx[p], step, P);
        } else {
            e = make_entry(n, false, P);
        }
        out[P] = e;
    }
    row_written(bad, stat);
}

template <int IPT>
static size_t sort_smem() {
    const size_t hist_words = kHistWords + (IPT <= 16 ? kMaxGroups : 0);
    return (size_t)kSortThreads * IPT * 4 + hist_words * 4 + kSortWarps * 4 + 8 +
           (size_t)kSortThreads * IPT * 2;
}

template <int IPT>
static cudaError_t launch_sort_ipt(const int32_t *ii_t, int ii_stride, int w, const DevFeature *feat,
                                   int64_t f0, int64_t nf, const WeightLayout &L, uint16_t *rows,
                                   int npad, const int32_t *row_list, int32_t *stat, cudaStream_t st) {
    const size_t sm = sort_smem<IPT>();
    cudaError_t e = cudaFuncSetAttribute(k_sort_rows<IPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_sort_rows<IPT><<<(unsigned)nf, kSortThreads, sm, st>>>(ii_t, ii_stride, w, feat, f0, L, rows, npad,
                                                            row_list, stat);
    return cudaGetLastError();
}

// ---- K3, packed variant (the one every row goes through first) ---------------------------
// The same stable sort for rows whose items fit one 32-bit word: value - min
// in the high bits above a sample index of ib bits (ib = 14 up to 16,384
// samples with 512-thread CTAs, two per SM; 15 above, with 1024-thread CTAs).
// A row whose value span does not fit next to its index is listed for the
// two-word sort above.  Only the value bits are sorted, in one pass when the
// span has at most 9 bits and in two passes over digits of half the span's
// bits (5 to 9) otherwise; the starting index order and stable passes order
// ties by sample index.  A pass ranks each item once: while the warps count
// their digits (the lanes holding the same digit come from one ballot per
// digit bit), every item records its rank among its warp's earlier items of
// the same digit (in shared memory, or two 16-bit ranks per register), so the
// scatter after the CTA-wide scan needs only the scanned offsets.  Then the
// bank choice of the two weight copies and the run-interleaved write, one
// 16-byte chunk per thread.
constexpr int kPkThreads = 512;
constexpr int kPkRefinePasses = 1;  // a second pass buys no search time
constexpr int kPkDigitBits = 9;
constexpr int kPkRadix = 1 << kPkDigitBits;

__host__ __device__ constexpr bool packed_ranks_in_smem(int ipt, int th) { return th <= 512 && ipt >= 20 && ipt <= 30; }

template <int IPT, int TH>
__global__ void __launch_bounds__(TH, TH <= 512 ? 2 : 1)
    k_sort_rows_packed(const int32_t *__restrict__ ii_t, const uint16_t *__restrict__ ii16, int ii_stride, int w,
                       const DevFeature *__restrict__ feat, int64_t f0, WeightLayout L,
                       uint16_t *__restrict__ rows, int npad, int32_t *ovf, int32_t *stat) {
    constexpr int NP = TH * IPT;
    constexpr int WARPS = TH / 32, HSTRIDE = WARPS + 1, HWORDS = kPkRadix * HSTRIDE;
    constexpr int GROUPS = NP / 32;  // lane-run groups of the longest row
    static_assert(3 * GROUPS * 4 <= HWORDS * (packed_ranks_in_smem(IPT, TH) ? 2 : 4),
                  "histogram space too small for the refine list");
    // 512-thread CTAs of 20 to 30 items keep the items' ranks in shared memory
    // (registers would spill) and count in 16 bits (counts and offsets stay
    // below 2^16) so that two CTAs still fit an SM; the others keep them in
    // registers
    constexpr bool RS = packed_ranks_in_smem(IPT, TH);
    using HT = typename std::conditional<RS, uint16_t, uint32_t>::type;
    const int n = L.n;
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *skey = reinterpret_cast<uint32_t *>(smem);                        // NP items
    uint16_t *rks = reinterpret_cast<uint16_t *>(skey + NP);                   // NP ranks (RS)
    HT *hist = reinterpret_cast<HT *>(RS ? (uint8_t *)(rks + NP) : (uint8_t *)(skey + NP));  // HWORDS
    uint32_t *gchoice = reinterpret_cast<uint32_t *>(
        reinterpret_cast<uint8_t *>(hist) + (((size_t)HWORDS * sizeof(HT) + 15) & ~(size_t)15));  // GROUPS
    uint32_t *ws = gchoice + GROUPS;                                            // WARPS
    int32_t *mm = reinterpret_cast<int32_t *>(ws + WARPS);                      // 2

    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int pos0 = wp * 32 * IPT + lane;
    const DevFeature d = feat[f0 + blockIdx.x];

    // the feature on every window (K2's arithmetic), four windows per thread
    // and corner load; boxes of at most kNarrowArea pixels from the integral
    // images modulo 2^16 (half the bytes)
    int32_t lo = INT_MAX, hi = INT_MIN;
    auto values = [&](auto value4) {
        for (int q = threadIdx.x; 4 * q < n; q += TH) {
            const int p = 4 * q;
            const int4 x = value4(p);
            reinterpret_cast<uint4 *>(skey)[q] = make_uint4((uint32_t)x.x, (uint32_t)x.y, (uint32_t)x.z, (uint32_t)x.w);
            lo = min(lo, x.x);
            hi = max(hi, x.x);
            if (p + 1 < n) { lo = min(lo, x.y); hi = max(hi, x.y); }
            if (p + 2 < n) { lo = min(lo, x.z); hi = max(hi, x.z); }
            if (p + 3 < n) { lo = min(lo, x.w); hi = max(hi, x.w); }
        }
    };
    if (ii16 && d.w * d.h <= kNarrowArea)
        values([&](int p) { return haar_value4_narrow(ii16, ii_stride, w, d.type, d.x, d.y, d.w, d.h, p); });
    else
        values([&](int p) { return haar_value4(ii_t, ii_stride, w, d.type, d.x, d.y, d.w, d.h, p); });
#pragma unroll
    for (int s = 16; s; s >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if (threadIdx.x == 0) { mm[0] = INT_MAX; mm[1] = INT_MIN; }
    __syncthreads();
    if (lane == 0) { atomicMin(&mm[0], lo); atomicMax(&mm[1], hi); }
    __syncthreads();
    lo = mm[0];
    hi = mm[1];
    const uint32_t span = static_cast<uint32_t>(hi) - static_cast<uint32_t>(lo);
    const int bits = span ? 32 - __clz(span) : 0;
    const int ib = 32 - __clz((uint32_t)(n - 1));  // bits of a sample index
    const uint32_t imask = (1u << ib) - 1u;
    if (bits + ib > 32) {  // value and index do not fit one word: the two-word sort takes the row
        if (threadIdx.x == 0) ovf[1 + atomicAdd(ovf, 1)] = (int32_t)blockIdx.x;
        return;
    }
    uint32_t c[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int p = pos0 + j * 32;
        // padding items take the all-ones word: they sort after every real item
        c[j] = (p < n) ? (((skey[p] - static_cast<uint32_t>(lo)) << ib) | (uint32_t)p) : 0xffffffffu;
    }
    __syncthreads();

    const uint32_t lt = lanemask_lt();
    // one stable pass over the D-bit digit at value bit `shift`; the sorted
    // items end in skey and in c
    auto radix_pass = [&](auto dbits, int shift) {
        constexpr int D = decltype(dbits)::value;
        constexpr uint32_t DMASK = (1u << D) - 1u;
        // counts warp-major (warp w's digit d at w * R + d): the lanes of a
        // warp touch neighbouring words, whatever their digits
        constexpr int R = (1 << D) + (sizeof(HT) == 2 ? 2 : 1);
        static_assert(WARPS * R <= HWORDS, "histogram space too small");
        const int sh = ib + shift;
        for (int k = threadIdx.x; k < WARPS * R; k += TH) hist[k] = 0;
        __syncthreads();
        // each item's rank among the warp's earlier items of its digit, in
        // position order (item j before item j + 1, lanes in order): in shared
        // memory at the item's position (RS), else two per register
        uint32_t rk[RS ? 1 : (IPT + 1) / 2];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t dg = (c[j] >> sh) & DMASK;
            const uint32_t peers = digit_peers<D>(dg);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (lane == leader) {
                old = hist[wp * R + dg];
                hist[wp * R + dg] = (HT)(old + __popc(peers));
            }
            old = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
            if constexpr (RS) {
                rks[pos0 + j * 32] = (uint16_t)old;
            } else {
                if (j & 1) rk[j >> 1] |= old << 16;
                else rk[j >> 1] = old;
            }
        }
        __syncthreads();
        {
            constexpr int PER = (1 << D) * WARPS / TH;
            static_assert(PER >= 1, "digit too narrow for the scan");
            uint32_t cnt[PER];
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int lin = threadIdx.x * PER + q;
                cnt[q] = hist[(lin % WARPS) * R + lin / WARPS];
                s += cnt[q];
            }
            // CTA-wide exclusive scan of the per-thread sums
            uint32_t inc = s;
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, dd);
                if (lane >= dd) inc += y;
            }
            if (lane == 31) ws[wp] = inc;
            __syncthreads();
            if (wp == 0) {
                const uint32_t t = lane < WARPS ? ws[lane] : 0u;
                uint32_t ti = t;
#pragma unroll
                for (int dd = 1; dd < 32; dd <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, ti, dd);
                    if (lane >= dd) ti += y;
                }
                if (lane < WARPS) ws[lane] = ti - t;
            }
            __syncthreads();
            uint32_t off = ws[wp] + inc - s;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int lin = threadIdx.x * PER + q;
                hist[(lin % WARPS) * R + lin / WARPS] = (HT)off;
                off += cnt[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint32_t dg = (c[j] >> sh) & DMASK;
            const uint32_t r = RS ? (uint32_t)rks[pos0 + j * 32] : ((rk[j >> 1] >> (16 * (j & 1))) & 0xffffu);
            skey[hist[wp * R + dg] + r] = c[j];
        }
        __syncthreads();
        // the next pass's first write to skey or hist follows two barriers
#pragma unroll
        for (int j = 0; j < IPT; ++j) c[j] = skey[pos0 + j * 32];
    };
    // Two passes at most (value bits <= 18); the digit is as narrow as that
    // allows (one ballot per digit bit), at least 5 bits.
    if (bits > 0) {
        const int passes = bits <= kPkDigitBits ? 1 : 2;
        const int D = max(5, (bits + passes - 1) / passes);
        for (int shift = 0; shift < bits; shift += D) {
            switch (D) {
                case 5: radix_pass(std::integral_constant<int, 5>{}, shift); break;
                case 6: radix_pass(std::integral_constant<int, 6>{}, shift); break;
                case 7: radix_pass(std::integral_constant<int, 7>{}, shift); break;
                case 8: radix_pass(std::integral_constant<int, 8>{}, shift); break;
                default: radix_pass(std::integral_constant<int, kPkDigitBits>{}, shift); break;
            }
        }
    } else {
        // one value: the items are already in order
#pragma unroll
        for (int j = 0; j < IPT; ++j) skey[pos0 + j * 32] = c[j];
        __syncthreads();
    }

    uint16_t *out = rows + (size_t)blockIdx.x * npad;
    const int run = npad / 32;
    if (L.dual) {
        // bank-balanced copy choice per gather group (see k_sort_rows); the
        // loads of the 32 banks as 2-bit counters in one 64-bit word (bank b
        // at bits 2b, 2b + 1; a load above 3 counts as 3).  Only the groups
        // left with a bank at 3 after the greedy pass get the pass of single
        // moves; they are listed first (in the free histogram space) so that
        // the threads share them evenly.
        auto level = [](uint64_t C, int b) { return (uint32_t)(C >> (2 * b)) & 3u; };
        auto inc = [&](uint64_t &C, int b) {
            if (level(C, b) != 3u) C += 1ull << (2 * b);
        };
        auto dec = [&](uint64_t &C, int b) {
            if (level(C, b) != 0u) C -= 1ull << (2 * b);
        };
        uint32_t *rlist = reinterpret_cast<uint32_t *>(hist);  // (group, counters lo, hi) of groups to refine
        if (threadIdx.x == 0) mm[0] = 0;
        __syncthreads();
        for (int g = threadIdx.x; g < run; g += TH) {
            uint64_t C = 0;
            uint32_t mask = 0;
            const int kend = min(32, (n - g + run - 1) / run);  // entries k * run + g < n
            for (int k = 0; k < kend; ++k) {
                const int i = (int)(skey[k * run + g] & imask);
                const int ba = i & 31, bb = rot_b(i) & 31;
                const uint32_t la = level(C, ba), lb = level(C, bb);
                const bool tob = i < L.nb && lb < la;
                const int c = tob ? bb : ba;
                if ((tob ? lb : la) != 3u) C += 1ull << (2 * c);
                mask |= (uint32_t)tob << k;
            }
            if (kend < 32) inc(C, n & 31);  // the padding word, read as a broadcast
            gchoice[g] = mask;
            if (kPkRefinePasses > 0 && ((C & (C >> 1)) & 0x5555555555555555ull)) {
                const int q = atomicAdd(&mm[0], 1);
                rlist[3 * q] = (uint32_t)g;
                rlist[3 * q + 1] = (uint32_t)C;
                rlist[3 * q + 2] = (uint32_t)(C >> 32);
            }
        }
        __syncthreads();
        const int nref = mm[0];
        for (int q = threadIdx.x; q < nref; q += TH) {
            const int g = (int)rlist[3 * q];
            uint64_t C = (uint64_t)rlist[3 * q + 1] | ((uint64_t)rlist[3 * q + 2] << 32);
            uint32_t mask = gchoice[g];
            const int kend = min(32, (n - g + run - 1) / run);
            for (int pass = 0; pass < kPkRefinePasses; ++pass)
                for (int k = 0; k < kend; ++k) {
                    const int i = (int)(skey[k * run + g] & imask);
                    if (i >= L.nb) continue;
                    const int ba = i & 31, bb = rot_b(i) & 31;
                    const bool onb = (mask >> k) & 1u;
                    const int cur = onb ? bb : ba, oth = onb ? ba : bb;
                    if (level(C, cur) > level(C, oth) + 1) {
                        dec(C, cur);
                        inc(C, oth);
                        mask ^= 1u << k;
                    }
                }
            gchoice[g] = mask;
        }
        __syncthreads();
    }
    // the run-interleaved write: one 16-byte chunk (8 entries) per thread;
    // chunk c holds entries t * 8 .. t * 8 + 7 of lane run k (c = t * 32 + k),
    // consecutive positions p0 .. p0 + 7 of the value order
    bool bad = false;
    for (int c = threadIdx.x; c < npad / kChunkElems; c += TH) {
        const int k = c & 31, t = c >> 5;
        const int p0 = k * run + t * kChunkElems;
        uint32_t cp[kChunkElems + 1];
        const uint4 lo4 = *reinterpret_cast<const uint4 *>(skey + p0);
        const uint4 hi4 = *reinterpret_cast<const uint4 *>(skey + p0 + 4);
        cp[0] = lo4.x; cp[1] = lo4.y; cp[2] = lo4.z; cp[3] = lo4.w;
        cp[4] = hi4.x; cp[5] = hi4.y; cp[6] = hi4.z; cp[7] = hi4.w;
        cp[8] = p0 + kChunkElems < n ? skey[p0 + kChunkElems] : 0u;
        uint32_t gc[kChunkElems] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        if (L.dual) {
            const uint4 g0 = *reinterpret_cast<const uint4 *>(gchoice + t * kChunkElems);
            const uint4 g1 = *reinterpret_cast<const uint4 *>(gchoice + t * kChunkElems + 4);
            gc[0] = g0.x; gc[1] = g0.y; gc[2] = g0.z; gc[3] = g0.w;
            gc[4] = g1.x; gc[5] = g1.y; gc[6] = g1.z; gc[7] = g1.w;
        }
        uint32_t wv[kChunkElems / 2];
#pragma unroll
        for (int j = 0; j < kChunkElems; ++j) {
            const int p = p0 + j;
            uint16_t e;
            if (p < n) {
                const bool step = (p == n - 1) || ((cp[j] >> ib) < (cp[j + 1] >> ib));
                int word = (int)(cp[j] & imask);
                if ((gc[j] >> k) & 1u) word = L.off_b + rot_b(word);
                bad |= word >= L.words || word == n;
                e = make_entry(word, step, j);
            } else {
                e = make_entry(n, false, j);
            }
            if (j & 1) wv[j >> 1] |= (uint32_t)e << 16;
            else wv[j >> 1] = e;
        }
        reinterpret_cast<uint4 *>(out)[c] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    row_written(bad, stat);
}

template <int IPT, int TH>
static size_t sort_packed_smem() {
    constexpr bool RS = packed_ranks_in_smem(IPT, TH);
    const size_t hist = (size_t)kPkRadix * (TH / 32 + 1) * (RS ? 2 : 4);
    return (size_t)TH * IPT * 4 + (RS ? (size_t)TH * IPT * 2 : 0) + ((hist + 15) & ~(size_t)15) +
           (size_t)(TH * IPT / 32 + TH / 32 + 2) * 4;
}

template <int IPT, int TH = kPkThreads>
static cudaError_t launch_sort_packed(const int32_t *ii_t, const uint16_t *ii16, int ii_stride, int w,
                                      const DevFeature *feat,
                                      int64_t f0, int64_t nf, const WeightLayout &L, uint16_t *rows,
                                      int npad, int32_t *ovf, int32_t *stat, cudaStream_t st) {
    const size_t sm = sort_packed_smem<IPT, TH>();
    cudaError_t e = cudaFuncSetAttribute(k_sort_rows_packed<IPT, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_sort_rows_packed<IPT, TH><<<(unsigned)nf, TH, sm, st>>>(ii_t, ii16, ii_stride, w, feat, f0, L, rows, npad,
                                                              ovf, stat);
    return cudaGetLastError();
}

// Two-word sort of `nf` rows of the tile (all of them, or those listed).
static cudaError_t launch_sort_wide(const int32_t *ii_t, int ii_stride, int w, const DevFeature *feat,
                                   int64_t f0, int64_t nf, const WeightLayout &L, uint16_t *rows, int npad,
                                   const int32_t *row_list, int32_t *stat, cudaStream_t st) {
    const int n = L.n;
#define VJB_SORT_CASE(I) launch_sort_ipt<I>(ii_t, ii_stride, w, feat, f0, nf, L, rows, npad, row_list, stat, st)
    if (n <= kSortThreads * 1) return VJB_SORT_CASE(1);
    if (n <= kSortThreads * 2) return VJB_SORT_CASE(2);
    if (n <= kSortThreads * 4) return VJB_SORT_CASE(4);
    if (n <= kSortThreads * 8) return VJB_SORT_CASE(8);
    if (n <= kSortThreads * 16) return VJB_SORT_CASE(16);
    return VJB_SORT_CASE(32);
#undef VJB_SORT_CASE
}

// Rows of a tile: the packed sort for every row (512 threads up to 16,384
// samples, 1024 above), then the two-word sort for the rows whose value span
// and sample index do not fit one word, which the packed sort lists.
// `ii16` (the integral images modulo 2^16, or null) serves the packed sort's
// features of small boxes.  `scratch` (3 + nf ints of device memory): [0] and [1] the table's check
// state (see row_written; zeroed by the caller once per table), [2] the
// tile's listed-row count, then the listed rows.  Waits for the stream when
// it reads the count.
cudaError_t launch_sort_rows(const int32_t *ii_t, const uint16_t *ii16, int ii_stride, int w,
                             const DevFeature *feat, int64_t f0, int64_t nf, const WeightLayout &L, uint16_t *rows,
                             int npad, int32_t *scratch, cudaStream_t st) {
    if (nf <= 0) return cudaSuccess;
    const int n = L.n;
    int32_t *stat = scratch, *ovf = scratch + 2;
    cudaError_t e = cudaMemsetAsync(ovf, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (n <= kPkThreads * 32) {
#define VJB_PK_CASE(I) launch_sort_packed<I>(ii_t, ii16, ii_stride, w, feat, f0, nf, L, rows, npad, ovf, stat, st)
        const int ipt = (n + kPkThreads - 1) / kPkThreads;
        if (ipt <= 4) e = VJB_PK_CASE(4);
        else if (ipt <= 8) e = VJB_PK_CASE(8);
        else if (ipt <= 12) e = VJB_PK_CASE(12);
        else if (ipt <= 16) e = VJB_PK_CASE(16);
        else if (ipt <= 20) e = VJB_PK_CASE(20);
        else if (ipt <= 24) e = VJB_PK_CASE(24);
        else if (ipt <= 28) e = VJB_PK_CASE(28);
        else if (ipt <= 30) e = VJB_PK_CASE(30);
        else e = VJB_PK_CASE(32);
#undef VJB_PK_CASE
    } else {
#define VJB_PK_WIDE(I) \
    launch_sort_packed<I, 1024>(ii_t, ii16, ii_stride, w, feat, f0, nf, L, rows, npad, ovf, stat, st)
        const int ipt = (n + 1023) / 1024;
        if (ipt <= 20) e = VJB_PK_WIDE(20);
        else if (ipt <= 24) e = VJB_PK_WIDE(24);
        else if (ipt <= 28) e = VJB_PK_WIDE(28);
        else e = VJB_PK_WIDE(32);
#undef VJB_PK_WIDE
    }
    if (e != cudaSuccess) return e;
    int32_t count = 0;
    e = cudaMemcpyAsync(&count, ovf, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || count == 0) return e;
    return launch_sort_wide(ii_t, ii_stride, w, feat, f0, count, L, rows, npad, ovf + 1, stat, st);
}

}  // namespace vjb
