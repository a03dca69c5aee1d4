// Host build of the FP32 sine/cosine used by the Kalman step kernels, for the accuracy check.
#include "trig.cuh"

extern "C" void trig_sweep(const float* x, float* s, float* c, long n) {
    for (long i = 0; i < n; ++i) mk::sin_cos_cw(x[i], s + i, c + i);
}
