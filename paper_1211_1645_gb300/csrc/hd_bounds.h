// hd_bounds.h -- host-side error bounds of the FP64 form's float pre-tests
// (pair_clear, k_hist_tile, k_psi6).  With t = 2^-20 (the relative error of
// approx_f32, a truncation of the double to the 20 mantissa bits of its high
// word) and u = 2^-24 (float rounding), a float estimate of a squared
// distance differs from the FP64 value by at most half the margin returned
// here; a float estimate farther than the margin from a threshold is on the
// same side of it as the FP64 value.
#pragma once

#include <cmath>

namespace hd {

// A pair of the colour pass: |q| < w, |cell offset| <= w, |np| < w + delta,
// so |rx| <= R = 2w + delta.  The float difference errs by at most
// E = t (2w + delta) + u (3w + R), the float square sum by
// 4 R E + 2 E^2 + 4 u (R + E)^2, and the FP64 square sum by less than
// 16 2^-53 R^2; the margin is twice their sum.
inline double pair_f32_margin(double w, double delta) {
    const double t = std::ldexp(1.0, -20), u = std::ldexp(1.0, -24);
    const double R = 2.0 * w + delta;
    const double E = t * (2.0 * w + delta) + u * (3.0 * w + R);
    return 2.0 * (4.0 * R * E + 2.0 * E * E + 4.0 * u * (R + E) * (R + E) + 16.0 * std::ldexp(1.0, -53) * R * R);
}

// A pair of a measurement H cells apart at most: both coordinates in [0, w),
// the offset dcx w added in float as dcx wf (rounded product), |rx| <= R =
// (H + 1) w; the float difference errs by at most E = 2 t w + u w (4H + 2).
inline double cells_f32_margin(double w, int H) {
    const double t = std::ldexp(1.0, -20), u = std::ldexp(1.0, -24);
    const double R = (double(H) + 1.0) * w;
    const double E = 2.0 * t * w + u * w * (4.0 * double(H) + 2.0);
    return 2.0 * (4.0 * R * E + 2.0 * E * E + 4.0 * u * (R + E) * (R + E) + 16.0 * std::ldexp(1.0, -53) * R * R);
}

}  // namespace hd
