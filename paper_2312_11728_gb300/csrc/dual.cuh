// Forward-mode dual numbers for the derivative of the fit (growth row G1).
//
// Dual<T, K> carries a value and K directional derivatives.  The Kalman-step code is written
// once as templates on its scalar type, so instantiating it for Dual<float, K> propagates exact
// first derivatives through every operation of the fit: the Newton solution of the crossing
// (whose derivative converges with the value, as the implicit-function derivative -g_p/g_s of
// the surface constraint), the Jacobian, the covariance transport, the material terms, the
// Cholesky of S, the chi2 and the Joseph update.  Comparisons and branches act on values;
// rounding helpers (floor, rint) have zero derivative.
#pragma once

#include <math.h>

namespace mk {

template <class T, int K> struct Dual {
    T v;
    T d[K];

    __host__ __device__ constexpr Dual() : v(T(0)), d{} {}
    __host__ __device__ constexpr Dual(double x) : v(T(x)), d{} {}
    __host__ __device__ constexpr Dual(float x) : v(T(x)), d{} {}
    __host__ __device__ constexpr Dual(int x) : v(T(x)), d{} {}
    __host__ __device__ explicit operator float() const { return float(v); }
    __host__ __device__ explicit operator double() const { return double(v); }

    // ---- arithmetic
    friend __device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) {
        Dual r;
        r.v = a.v + b.v;
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) {
        Dual r;
        r.v = a.v - b.v;
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dual operator-(const Dual& a) {
        Dual r;
        r.v = -a.v;
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) {
        Dual r;
        r.v = a.v * b.v;
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
        return r;
    }
    friend __device__ __forceinline__ Dual operator/(const Dual& a, const Dual& b) {
        Dual r;
        r.v = a.v / b.v;
        const T ib = T(1) / b.v;
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
        return r;
    }
    __device__ __forceinline__ Dual& operator+=(const Dual& b) { return *this = *this + b; }
    __device__ __forceinline__ Dual& operator-=(const Dual& b) { return *this = *this - b; }
    __device__ __forceinline__ Dual& operator*=(const Dual& b) { return *this = *this * b; }
    __device__ __forceinline__ Dual& operator/=(const Dual& b) { return *this = *this / b; }

    // ---- comparisons act on values
    friend __device__ __forceinline__ bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
    friend __device__ __forceinline__ bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
    friend __device__ __forceinline__ bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
    friend __device__ __forceinline__ bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
    friend __device__ __forceinline__ bool operator==(const Dual& a, const Dual& b) { return a.v == b.v; }
    friend __device__ __forceinline__ bool operator!=(const Dual& a, const Dual& b) { return a.v != b.v; }

    // ---- elementary functions: f(a) with derivative f'(a) * da
    __device__ __forceinline__ Dual chain(T fv, T fp) const {
        Dual r;
        r.v = fv;
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = fp * d[k];
        return r;
    }
    friend __device__ __forceinline__ Dual sqrt(const Dual& a) {
        const T s = sqrt(a.v);
        return a.chain(s, s > T(0) ? T(0.5) / s : T(0));
    }
    friend __device__ __forceinline__ Dual fabs(const Dual& a) { return a.chain(fabs(a.v), a.v < T(0) ? T(-1) : T(1)); }
    friend __device__ __forceinline__ Dual floor(const Dual& a) { return Dual(floor(a.v)); }
    friend __device__ __forceinline__ Dual rint(const Dual& a) { return Dual(rint(a.v)); }
    friend __device__ __forceinline__ Dual asinh(const Dual& a) {
        return a.chain(asinh(a.v), T(1) / sqrt(T(1) + a.v * a.v));
    }
    friend __device__ __forceinline__ Dual atan2(const Dual& y, const Dual& x) {
        Dual r;
        r.v = atan2(y.v, x.v);
        const T den = T(1) / (x.v * x.v + y.v * y.v);
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * den;
        return r;
    }
    friend __device__ __forceinline__ Dual fmin(const Dual& a, const Dual& b) { return b.v < a.v ? b : a; }
    friend __device__ __forceinline__ Dual fmax(const Dual& a, const Dual& b) { return b.v > a.v ? b : a; }
    friend __device__ __forceinline__ Dual fma(const Dual& a, const Dual& b, const Dual& c) {
        Dual r;
        r.v = fma(a.v, b.v, c.v);
#pragma unroll
        for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k] + c.d[k];
        return r;
    }
};

template <class T> struct ScalarOf { using type = T; };
template <class T, int K> struct ScalarOf<Dual<T, K>> { using type = T; };

}  // namespace mk
