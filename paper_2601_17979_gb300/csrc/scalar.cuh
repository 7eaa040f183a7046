// scalar.cuh -- real and complex arithmetic for the batched Jacobi SVD kernels.
//
// T is float, double, float2 (complex float) or double2 (complex double),
// complex numbers stored interleaved (re, im).  R is the matching real type.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace bsvd {

template <class T> struct Traits;
template <> struct Traits<float>   { using R = float;  static constexpr bool kComplex = false; };
template <> struct Traits<double>  { using R = double; static constexpr bool kComplex = false; };
template <> struct Traits<float2>  { using R = float;  static constexpr bool kComplex = true; };
template <> struct Traits<double2> { using R = double; static constexpr bool kComplex = true; };

template <class T> using Real = typename Traits<T>::R;

// ---- construction -------------------------------------------------------
template <class T> __device__ __forceinline__ T make_s(Real<T> re);
template <> __device__ __forceinline__ float make_s<float>(float re) { return re; }
template <> __device__ __forceinline__ double make_s<double>(double re) { return re; }
template <> __device__ __forceinline__ float2 make_s<float2>(float re) { return make_float2(re, 0.f); }
template <> __device__ __forceinline__ double2 make_s<double2>(double re) { return make_double2(re, 0.0); }

// ---- parts ----------------------------------------------------------------
__device__ __forceinline__ float re(float x) { return x; }
__device__ __forceinline__ double re(double x) { return x; }
__device__ __forceinline__ float re(float2 x) { return x.x; }
__device__ __forceinline__ double re(double2 x) { return x.x; }

__device__ __forceinline__ float conj_s(float x) { return x; }
__device__ __forceinline__ double conj_s(double x) { return x; }
__device__ __forceinline__ float2 conj_s(float2 x) { return make_float2(x.x, -x.y); }
__device__ __forceinline__ double2 conj_s(double2 x) { return make_double2(x.x, -x.y); }

// |x|^2
__device__ __forceinline__ float abs2(float x) { return x * x; }
__device__ __forceinline__ double abs2(double x) { return x * x; }
__device__ __forceinline__ float abs2(float2 x) { return fmaf(x.x, x.x, x.y * x.y); }
__device__ __forceinline__ double abs2(double2 x) { return fma(x.x, x.x, x.y * x.y); }

// |x| without overflow
__device__ __forceinline__ float abs_s(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_s(double x) { return fabs(x); }
__device__ __forceinline__ float abs_s(float2 x) { return hypotf(x.x, x.y); }
__device__ __forceinline__ double abs_s(double2 x) { return hypot(x.x, x.y); }

// max(|re|, |im|)
__device__ __forceinline__ float maxabs(float x) { return fabsf(x); }
__device__ __forceinline__ double maxabs(double x) { return fabs(x); }
__device__ __forceinline__ float maxabs(float2 x) { return fmaxf(fabsf(x.x), fabsf(x.y)); }
__device__ __forceinline__ double maxabs(double2 x) { return fmax(fabs(x.x), fabs(x.y)); }

__device__ __forceinline__ bool finite_s(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_s(double x) { return isfinite(x); }
__device__ __forceinline__ bool finite_s(float2 x) { return isfinite(x.x) && isfinite(x.y); }
__device__ __forceinline__ bool finite_s(double2 x) { return isfinite(x.x) && isfinite(x.y); }

// ---- arithmetic -------------------------------------------------------------
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ float sub(float a, float b) { return a - b; }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 mul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// x * r (r real)
__device__ __forceinline__ float scale(float x, float r) { return x * r; }
__device__ __forceinline__ double scale(double x, double r) { return x * r; }
__device__ __forceinline__ float2 scale(float2 x, float r) { return make_float2(x.x * r, x.y * r); }
__device__ __forceinline__ double2 scale(double2 x, double r) { return make_double2(x.x * r, x.y * r); }

// x / r (r real), IEEE division
__device__ __forceinline__ float divr(float x, float r) { return x / r; }
__device__ __forceinline__ double divr(double x, double r) { return x / r; }
__device__ __forceinline__ float2 divr(float2 x, float r) { return make_float2(x.x / r, x.y / r); }
__device__ __forceinline__ double2 divr(double2 x, double r) { return make_double2(x.x / r, x.y / r); }

// a * b + c
__device__ __forceinline__ float fma_s(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_s(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 fma_s(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(-a.y, b.y, fmaf(a.x, b.x, c.x)), fmaf(a.y, b.x, fmaf(a.x, b.y, c.y)));
}
__device__ __forceinline__ double2 fma_s(double2 a, double2 b, double2 c) {
    return make_double2(fma(-a.y, b.y, fma(a.x, b.x, c.x)), fma(a.y, b.x, fma(a.x, b.y, c.y)));
}

// conj(a) * b + c
__device__ __forceinline__ float cfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double cfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.y, b.y, fmaf(a.x, b.x, c.x)), fmaf(-a.y, b.x, fmaf(a.x, b.y, c.y)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.y, b.y, fma(a.x, b.x, c.x)), fma(-a.y, b.x, fma(a.x, b.y, c.y)));
}

// x * 2^e, exact unless the result leaves the normal range
__device__ __forceinline__ float scalb_s(float x, int e) { return scalbnf(x, e); }
__device__ __forceinline__ double scalb_s(double x, int e) { return scalbn(x, e); }
__device__ __forceinline__ float2 scalb_s(float2 x, int e) { return make_float2(scalbnf(x.x, e), scalbnf(x.y, e)); }
__device__ __forceinline__ double2 scalb_s(double2 x, int e) { return make_double2(scalbn(x.x, e), scalbn(x.y, e)); }

template <class T> __device__ __forceinline__ T nan_s();
template <> __device__ __forceinline__ float nan_s<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double nan_s<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <> __device__ __forceinline__ float2 nan_s<float2>() { return make_float2(nan_s<float>(), nan_s<float>()); }
template <> __device__ __forceinline__ double2 nan_s<double2>() { return make_double2(nan_s<double>(), nan_s<double>()); }

// 1/sqrt(x): rsqrtf (within 2 ulp) for float, the double-precision rsqrt
// (within 1 ulp) for double -- a rotation only needs c^2 + s^2 = 1 to a few ulp.
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// e^{i arg(g)} given a = |g| > 0: the sign for real data
__device__ __forceinline__ float phase_s(float g, float) { return copysignf(1.0f, g); }
__device__ __forceinline__ double phase_s(double g, double) { return copysign(1.0, g); }
__device__ __forceinline__ float2 phase_s(float2 g, float a) { const float r = 1.0f / a; return make_float2(g.x * r, g.y * r); }
__device__ __forceinline__ double2 phase_s(double2 g, double a) { const double r = 1.0 / a; return make_double2(g.x * r, g.y * r); }

__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float hypot_r(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double hypot_r(double a, double b) { return hypot(a, b); }
__device__ __forceinline__ int ilogb_r(float x) { return ilogbf(x); }
__device__ __forceinline__ int ilogb_r(double x) { return ilogb(x); }
__device__ __forceinline__ float scalb_r(float x, int e) { return scalbnf(x, e); }
__device__ __forceinline__ double scalb_r(double x, int e) { return scalbn(x, e); }

}  // namespace bsvd
