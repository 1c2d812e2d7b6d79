// arith.cuh -- the two arithmetics of the Krylov vectors, as policy types.
//   ArF64: IEEE binary64 on the FP64 pipe (the plain reference path).
//   ArDF:  double-float pairs on the FP32 pipe (see df64.cuh).
// Both store one value in 8 bytes (vec8), so buffers and layouts are shared.
#pragma once
#include "df64.cuh"
#include "irk_internal.h"

struct ArF64 {
    typedef double val;
    typedef double acc;
    static __device__ __forceinline__ val ld(const vec8 *p) { return __ldg(reinterpret_cast<const double *>(p)); }
    static __device__ __forceinline__ val ldv(const vec8 *p) { return *reinterpret_cast<const volatile double *>(p); }
    static __device__ __forceinline__ void st(vec8 *p, val v) { *reinterpret_cast<double *>(p) = v; }
    static __device__ __forceinline__ acc zero() { return 0.0; }
    static __device__ __forceinline__ void fma(acc &a, val x, val y) { a = ::fma(x, y, a); }
    static __device__ __forceinline__ void renorm(acc &) {}
    static __device__ __forceinline__ void add_to(acc &a, val x) { a += x; }
    static __device__ __forceinline__ val value(acc a) { return a; }
    static __device__ __forceinline__ val add(val a, val b) { return a + b; }
    static __device__ __forceinline__ val sub(val a, val b) { return a - b; }
    static __device__ __forceinline__ val neg(val a) { return -a; }
    static __device__ __forceinline__ val mul(val a, val b) { return a * b; }
    static __device__ __forceinline__ val ldcg(const vec8 *p) { return __ldcg(reinterpret_cast<const double *>(p)); }
    static __device__ __forceinline__ val from_double(double x) { return x; }
    static __device__ __forceinline__ val coef(double x, float, float) { return x; }
    static __device__ __forceinline__ double to_double(val v) { return v; }
    static __device__ __forceinline__ float to_float(val v) { return (float)v; }
    static __device__ __forceinline__ val from_float(float f) { return (double)f; }
    static __device__ __forceinline__ val shfl_down(val v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
    static __device__ __forceinline__ bool finite(val v) { return isfinite(v); }
};

struct ArDF {
    typedef df64 val;
    typedef df_acc acc;
    static __device__ __forceinline__ val ld(const vec8 *p) {
        float2 f = __ldg(reinterpret_cast<const float2 *>(p));
        return df_make(f.x, f.y);
    }
    static __device__ __forceinline__ val ldv(const vec8 *p) {
        const volatile float *q = reinterpret_cast<const volatile float *>(p);
        return df_make(q[0], q[1]);
    }
    static __device__ __forceinline__ void st(vec8 *p, val v) {
        *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
    }
    static __device__ __forceinline__ acc zero() { return df_acc_zero(); }
    static __device__ __forceinline__ void fma(acc &a, val x, val y) { df_acc_fma(a, x, y); }
    // fold the error term into the sum; the operator product does it after
    // every eighth column of a block and after its last column
    static __device__ __forceinline__ void renorm(acc &a) { df_acc_renorm(a); }
    static __device__ __forceinline__ void add_to(acc &a, val x) { df_acc_add(a, x); }
    static __device__ __forceinline__ val value(acc a) { return df_acc_value(a); }
    static __device__ __forceinline__ val add(val a, val b) { return df_add(a, b); }
    static __device__ __forceinline__ val sub(val a, val b) { return df_sub(a, b); }
    static __device__ __forceinline__ val neg(val a) { return df_neg(a); }
    static __device__ __forceinline__ val mul(val a, val b) { return df_mul(a, b); }
    static __device__ __forceinline__ val ldcg(const vec8 *p) {
        float2 f = __ldcg(reinterpret_cast<const float2 *>(p));
        return df_make(f.x, f.y);
    }
    static __device__ __forceinline__ val from_double(double x) { return df_from_double(x); }
    static __device__ __forceinline__ val coef(double, float hi, float lo) { return df_make(hi, lo); }
    static __device__ __forceinline__ double to_double(val v) { return df_to_double(v); }
    static __device__ __forceinline__ float to_float(val v) { return __fadd_rn(v.hi, v.lo); }
    static __device__ __forceinline__ val from_float(float f) { return df_make(f, 0.f); }
    static __device__ __forceinline__ val shfl_down(val v, int d) {
        return df_make(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
    }
    static __device__ __forceinline__ bool finite(val v) { return isfinite(v.hi) && isfinite(v.lo); }
};

// Scalar coefficient passed to kernels in both forms.
struct KCoef {
    double d;
    float hi, lo;
};

static inline KCoef make_kcoef(double x) {
    KCoef c;
    c.d = x;
    c.hi = (float)x;
    c.lo = (float)(x - (double)c.hi);
    return c;
}
