// Haar feature values (Sec. 2.1-2.2) from the point-major integral images:
// one window, four windows per load, and the narrow-box form from the
// integral images modulo 2^16.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vjb.h"

namespace vjb {

// Haar feature value from integral images stored point-major: point (px, py)
// of sample i is at ii_t[(py * (w + 1) + px) * stride + i].  Rectangle sums use
// the four corners of Sec. 2.1 (4 + 1 - (2 + 3)); the combination per type is
// the dark-minus-white reading documented in vjb.h.
__device__ __forceinline__ int32_t haar_value(const int32_t *__restrict__ ii_t, int stride,
                                              int w, int type, int x, int y, int fw, int fh,
                                              int i) {
    const int W1 = w + 1;
    auto P = [&](int px, int py) -> int32_t { return __ldg(ii_t + (size_t)(py * W1 + px) * stride + i); };
    auto R = [&](int rx, int ry, int rw, int rh) -> int32_t {
        return P(rx + rw, ry + rh) + P(rx, ry) - (P(rx + rw, ry) + P(rx, ry + rh));
    };
    switch (type) {
    case VJB_HAAR_2H: {
        const int a = fw >> 1;
        return R(x + a, y, a, fh) - R(x, y, a, fh);
    }
    case VJB_HAAR_2V: {
        const int b = fh >> 1;
        return R(x, y + b, fw, b) - R(x, y, fw, b);
    }
    case VJB_HAAR_3H: {
        const int a = fw / 3;
        return R(x + a, y, a, fh) - R(x, y, a, fh) - R(x + 2 * a, y, a, fh);
    }
    case VJB_HAAR_3V: {
        const int b = fh / 3;
        return R(x, y + b, fw, b) - R(x, y, fw, b) - R(x, y + 2 * b, fw, b);
    }
    default: {
        const int a = fw >> 1, b = fh >> 1;
        return R(x + a, y, a, b) + R(x, y + b, a, b) - R(x, y, a, b) - R(x + a, y + b, a, b);
    }
    }
}

// The combination of haar_value for four windows at once, from a loader that
// returns the four windows' integral-image values at point (px, py).
template <class Load4>
__device__ __forceinline__ int4 haar_combine4(int type, int x, int y, int fw, int fh, Load4 P) {
    auto add = [](int4 a, int4 b) { return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); };
    auto sub = [](int4 a, int4 b) { return make_int4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); };
    auto R = [&](int rx, int ry, int rw, int rh) {
        return sub(add(P(rx + rw, ry + rh), P(rx, ry)), add(P(rx + rw, ry), P(rx, ry + rh)));
    };
    switch (type) {
    case VJB_HAAR_2H: {
        const int a = fw >> 1;
        return sub(R(x + a, y, a, fh), R(x, y, a, fh));
    }
    case VJB_HAAR_2V: {
        const int b = fh >> 1;
        return sub(R(x, y + b, fw, b), R(x, y, fw, b));
    }
    case VJB_HAAR_3H: {
        const int a = fw / 3;
        return sub(sub(R(x + a, y, a, fh), R(x, y, a, fh)), R(x + 2 * a, y, a, fh));
    }
    case VJB_HAAR_3V: {
        const int b = fh / 3;
        return sub(sub(R(x, y + b, fw, b), R(x, y, fw, b)), R(x, y + 2 * b, fw, b));
    }
    default: {
        const int a = fw >> 1, b = fh >> 1;
        return sub(add(R(x + a, y, a, b), R(x, y + b, a, b)), add(R(x, y, a, b), R(x + a, y + b, a, b)));
    }
    }
}

// haar_value for the four windows i .. i + 3 (i a multiple of 4, the row
// stride a multiple of 4): one 16-byte load per corner.
__device__ __forceinline__ int4 haar_value4(const int32_t *__restrict__ ii_t, int stride, int w, int type,
                                            int x, int y, int fw, int fh, int i) {
    const int W1 = w + 1;
    return haar_combine4(type, x, y, fw, fh, [&](int px, int py) -> int4 {
        return __ldg(reinterpret_cast<const int4 *>(ii_t + (size_t)(py * W1 + px) * stride + i));
    });
}

// Area of a feature's subtracted rectangles: its value lies in
// [-255 * neg, 255 * (fw * fh - neg)], a range 255 * fw * fh wide (the
// rectangles tile the fw x fh box; pixels are 0..255).
__device__ __forceinline__ int haar_neg_area(int type, int fw, int fh) {
    switch (type) {
    case VJB_HAAR_3H: return 2 * (fw / 3) * fh;
    case VJB_HAAR_3V: return 2 * fw * (fh / 3);
    default: return fw * fh / 2;  // 2H (fw even), 2V (fh even), four-rectangle (both even)
    }
}

// Largest box (fw * fh) whose values span at most 2^16 integers: 255 * 257 =
// 65535.
constexpr int kNarrowArea = 257;

// haar_value4 for a feature with fw * fh <= kNarrowArea from the integral
// images modulo 2^16 (ii16, same layout): one 8-byte load per corner.  The
// corner combination is exact modulo 2^16, and the value is the one integer
// of its residue class in [-255 * neg, -255 * neg + 65535].
__device__ __forceinline__ int4 haar_value4_narrow(const uint16_t *__restrict__ ii16, int stride, int w,
                                                   int type, int x, int y, int fw, int fh, int i) {
    const int W1 = w + 1;
    const int4 r = haar_combine4(type, x, y, fw, fh, [&](int px, int py) -> int4 {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(ii16 + (size_t)(py * W1 + px) * stride + i));
        return make_int4((int)(q.x & 0xffffu), (int)(q.x >> 16), (int)(q.y & 0xffffu), (int)(q.y >> 16));
    });
    const int lo = -255 * haar_neg_area(type, fw, fh);
    auto lift = [lo](int v) { return lo + (int)((uint32_t)(v - lo) & 0xffffu); };
    return make_int4(lift(r.x), lift(r.y), lift(r.z), lift(r.w));
}

}  // namespace vjb
