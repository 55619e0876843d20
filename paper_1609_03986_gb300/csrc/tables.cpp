// Sample-offset tables for the oriented, scaled LATCH window (Sec. 3.2, "Memory
// optimization": the window rotated to the keypoint's orientation is read as an
// upright square).  Built on the host once per scale table and uploaded.
//
// Reading of the rotation and rounding (the paper gives no formula):
//   theta_b = 2*pi*b/32 for bin b; the in-quadrant part r = b mod 8 uses libm
//   cos/sin of r*pi/16, and the b/8 quarter turns are applied exactly by swapping
//   and negating; window point (a, e) = (u - 24, v - 24) maps to the offset
//   (round(s*(c*a - sn*e)), round(s*(sn*a + c*e))), FP64, evaluated in exactly this
//   order (this file is compiled with -ffp-contract=off), round = half away from zero.
// With that rounding, the table of bin b+8 is the table of bin b turned by 90
// degrees at every scale, so nearest-pixel sampling commutes with quarter turns.
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace latch {

namespace {

struct Dir {
    double c, s;
};

Dir bin_direction(int bin) {
    const int b = bin & (kBins - 1);
    const int r = b & 7;
    Dir d{1.0, 0.0};
    if (r != 0) {
        const double ang = static_cast<double>(r) * M_PI / 16.0;
        d = Dir{std::cos(ang), std::sin(ang)};
    }
    switch (b >> 3) {
        case 1: return Dir{-d.s, d.c};   // +90 degrees
        case 2: return Dir{-d.c, -d.s};  // +180 degrees
        case 3: return Dir{d.s, -d.c};   // +270 degrees
        default: return d;
    }
}

}  // namespace

void build_offset_tables(const double* scales, int nscales, int8_t* out) {
    for (int si = 0; si < nscales; ++si) {
        const double s = scales[si];
        for (int b = 0; b < kBins; ++b) {
            const Dir d = bin_direction(b);
            int8_t* tab = out + (static_cast<size_t>(si) * kBins + b) * kWinPix * 2;
            for (int v = 0; v < kWin; ++v) {
                const double e = static_cast<double>(v - kHalf);
                for (int u = 0; u < kWin; ++u) {
                    const double a = static_cast<double>(u - kHalf);
                    const double x = s * (d.c * a - d.s * e);
                    const double y = s * (d.s * a + d.c * e);
                    tab[2 * (v * kWin + u) + 0] = static_cast<int8_t>(std::round(x));
                    tab[2 * (v * kWin + u) + 1] = static_cast<int8_t>(std::round(y));
                }
            }
        }
    }
}

int max_reach(const double* scales, int nscales) {
    double m = 0.0;
    for (int i = 0; i < nscales; ++i) m = scales[i] > m ? scales[i] : m;
    // corner of the window: |a|, |e| <= 24, so |offset| <= 24*sqrt(2)*s, then rounding
    return static_cast<int>(std::ceil(24.0 * std::sqrt(2.0) * m)) + 1;
}

}  // namespace latch
