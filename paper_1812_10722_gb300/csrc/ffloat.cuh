// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, about 48 significant bits.  Built on error-free
// transformations: Knuth's two-sum (the exact rounding error of an FP32 addition) and
// the FMA two-product (the exact rounding error of an FP32 product).  On this GPU the
// FP64 pipe runs at a small fraction of the FP32 rate, so the refinement residual of
// the iterative solver is evaluated in this arithmetic instead of native FP64.
//
// Additions use the "sloppy" form (one two-sum on the leading parts): its error is a
// few units of 2^-46 of the larger operand, which is what the residual needs.
#pragma once

#include <cuda_runtime.h>

struct ffloat {
    float hi, lo;

    ffloat() = default;   // trivial, so arrays can live in shared memory
    __host__ __device__ ffloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ ffloat(float v) : hi(v), lo(0.f) {}
    __host__ __device__ ffloat(int v) : hi((float)v), lo((float)(v - (int)(float)v)) {}
    __host__ __device__ ffloat(double v) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    __host__ __device__ operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// s + e = a + b exactly, assuming |a| >= |b| (or a == 0)
__device__ __forceinline__ void ff_quick_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ffloat operator+(const ffloat &x, const ffloat &y) {
    float s, e;
    ff_two_sum(x.hi, y.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    ffloat r;
    ff_quick_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ ffloat operator-(const ffloat &x) { return ffloat(-x.hi, -x.lo); }
__device__ __forceinline__ ffloat operator-(const ffloat &x, const ffloat &y) { return x + (-y); }

__device__ __forceinline__ ffloat operator*(const ffloat &x, const ffloat &y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);   // exact error of the leading product
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    ffloat r;
    ff_quick_two_sum(p, e, r.hi, r.lo);
    return r;
}

// acc += a * b for a running sum that is read once at the end as the exact (double) hi + lo: the
// product's leading part enters by a two-sum, its error and the two-sum's error go to lo, and the
// pair is not renormalised per step (lo stays within a few units of hi's last place times the
// number of terms, and its own rounding contributes ~2^-48 of hi per term).  12 FP32
// instructions against 16 for a multiply and a renormalising add.
__device__ __forceinline__ void ff_mac(ffloat &acc, const ffloat &a, const ffloat &b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, e;
    ff_two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ ffloat &operator+=(ffloat &x, const ffloat &y) { return x = x + y; }
__device__ __forceinline__ ffloat &operator-=(ffloat &x, const ffloat &y) { return x = x - y; }
__device__ __forceinline__ ffloat &operator*=(ffloat &x, const ffloat &y) { return x = x * y; }

// 1/sqrt(x): FP32 seed y0, then one Newton-Raphson step y0 (1 + h/2), h = 1 - x y0^2
// formed in float-float (1 - leading part is exact since x y0^2 is close to 1); the
// step leaves a relative error of about (3/8) h^2 ~ 1e-13.
__device__ __forceinline__ ffloat rsq(const ffloat &x) {
    const float y0 = rsqrtf(x.hi);
    const ffloat xy2 = x * (ffloat(y0) * ffloat(y0));
    const float h = __fsub_rn(__fsub_rn(1.f, xy2.hi), xy2.lo);
    ffloat r;
    ff_quick_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), h), r.hi, r.lo);
    return r;
}

// four float-float values (a source position + weight, a normal, four weight channels, ...)
struct __align__(16) ff4 {
    ffloat x, y, z, w;
};
