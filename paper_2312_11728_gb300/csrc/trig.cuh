// Sine and cosine of an FP32 angle of moderate size, for the FP32 Kalman step.
//
// The angles the step takes (phi in (-pi, pi], theta in (0, pi), half turning angles) are all
// a few radians at most, so the general routine's reduction for huge arguments (and the stack
// frame and code it brings into every inlined call site) is not needed.  Method:
//  - reduction by pi/2 after Cody and Waite ("Software Manual for the Elementary Functions",
//    1980): k = rint(x * 2/pi), r = x - k*pi/2 with pi/2 split into three FP32 parts, each
//    product subtracted by one FMA (so k * part is exact for |k| < 2^24);
//  - the Taylor series of sin and cos on |r| <= pi/4, cut where the first dropped term is
//    below 2e-9 relative (sin through r^9, cos through r^10);
//  - the quadrant k mod 4 picks and signs the two results.
// Accuracy: within 2 ulp of the exact values for |x| <= 2^15 (checked against FP64 on the
// host over dense sweeps, including points next to multiples of pi/2).  Larger arguments lose
// accuracy gradually; NaN and infinity give NaN.  Compiles as host C++ too, for that check.
#pragma once

#if defined(__CUDACC__)
#define MK_TRIG_FN __host__ __device__ __forceinline__
#else
#include <cmath>
#define MK_TRIG_FN inline
#endif

namespace mk {

MK_TRIG_FN void sin_cos_cw(float x, float* s, float* c) {
    const float kTwoOverPi = 0.636619772f;
    const float kPio2a = 1.57079637f;        // pi/2 rounded to FP32
    const float kPio2b = -4.37113883e-8f;    // pi/2 - a, rounded
    const float kPio2c = -1.71512451e-15f;   // pi/2 - a - b, rounded
    const float k = rintf(x * kTwoOverPi);
    float r = fmaf(-k, kPio2a, x);
    r = fmaf(-k, kPio2b, r);
    r = fmaf(-k, kPio2c, r);
    const float r2 = r * r;
    const float ps = -1.0f / 6.0f + r2 * (1.0f / 120.0f + r2 * (-1.0f / 5040.0f + r2 * (1.0f / 362880.0f)));
    const float pc = 1.0f / 24.0f + r2 * (-1.0f / 720.0f + r2 * (1.0f / 40320.0f + r2 * (-1.0f / 3628800.0f)));
    const float sr = fmaf(r * r2, ps, r);
    const float cr = fmaf(r2, fmaf(r2, pc, -0.5f), 1.0f);
    const int q = static_cast<int>(k) & 3;
    const float a = (q & 1) ? cr : sr;   // sine up to sign
    const float b = (q & 1) ? sr : cr;   // cosine up to sign
    *s = (q & 2) ? -a : a;
    *c = ((q + 1) & 2) ? -b : b;
}

}  // namespace mk
