// df64.cuh -- double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 runs binary32 FMA about
// 60x faster than binary64, so the operator product, Gram-Schmidt and
// residuals of the Krylov solver use this type when the context selects
// IRK_KRYLOV_DF64.  The algorithms are the published error-free
// transformations:
//   TwoSum        Knuth (TAOCP vol. 2), Moller (1965)
//   FastTwoSum    Dekker (1971), valid when |a| >= |b| or a == 0
//   TwoProd       with a fused multiply-add (e.g. Muller et al., Handbook of
//                 Floating-Point Arithmetic, 2nd ed., Sec. 4.4)
//   DW + DW       "AccurateDWPlusDW", Joldes, Muller & Popescu, ACM TOMS 44
//                 (2017), Alg. 6 (relative error <= 3u^2)
//   DW x DW       "DWTimesDW3", ibid., Alg. 12 (relative error <= 4u^2)
//   dot products  the compensated scheme Dot2 of Ogita, Rump & Oishi, SISC 26
//                 (2005), extended with the cross terms of double-word inputs.
// Conversions to and from binary64 use the FP64 pipe and run only at the
// library boundary.
#pragma once
#include <cuda_runtime.h>

struct __align__(8) df64 {
    float hi, lo;
};

__device__ __forceinline__ df64 df_make(float h, float l) {
    df64 r;
    r.hi = h;
    r.lo = l;
    return r;
}

__device__ __forceinline__ df64 df_from_double(double x) {
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df_make(h, l);
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_add(df64 x, df64 y) {
    float sh, sl, th, tl, vh, vl;
    two_sum(x.hi, y.hi, sh, sl);
    two_sum(x.lo, y.lo, th, tl);
    float c = __fadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    float w = __fadd_rn(tl, vl);
    float zh, zl;
    fast_two_sum(vh, w, zh, zl);
    return df_make(zh, zl);
}

__device__ __forceinline__ df64 df_neg(df64 x) { return df_make(-x.hi, -x.lo); }

__device__ __forceinline__ df64 df_sub(df64 x, df64 y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df64 df_mul(df64 x, df64 y) {
    float ch = __fmul_rn(x.hi, y.hi);
    float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(cl1, cl2);
    float zh, zl;
    fast_two_sum(ch, cl3, zh, zl);
    return df_make(zh, zl);
}

// Dot-product accumulator: the running sum is s + c with c collecting the
// exact rounding errors of every addition and product (not renormalised per
// term); df_acc_value renormalises.
struct df_acc {
    float s, c;
};

__device__ __forceinline__ df_acc df_acc_zero() {
    df_acc a;
    a.s = 0.f;
    a.c = 0.f;
    return a;
}

// acc += x * y
__device__ __forceinline__ void df_acc_fma(df_acc &acc, df64 x, df64 y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    float s, t;
    two_sum(acc.s, p, s, t);
    float c = __fmaf_rn(x.hi, y.lo, acc.c);
    c = __fmaf_rn(x.lo, y.hi, c);
    acc.s = s;
    acc.c = __fadd_rn(c, __fadd_rn(t, e));
}

// acc += x * y for a binary32 y (a double-word value whose low word is 0):
// the same operations as df_acc_fma with the x.hi * y.lo term, which is
// exactly zero, left out.
__device__ __forceinline__ void df_acc_fma_f(df_acc &acc, df64 x, float y) {
    float p = __fmul_rn(x.hi, y);
    float e = __fmaf_rn(x.hi, y, -p);
    float s, t;
    two_sum(acc.s, p, s, t);
    float c = __fmaf_rn(x.lo, y, acc.c);
    acc.s = s;
    acc.c = __fadd_rn(c, __fadd_rn(t, e));
}

// Fold the error term into the running sum (s, c) <- FastTwoSum(s, c), so that
// c holds only what s cannot: without it c grows with every term and its own
// rounding errors (u |c| per addition, u = 2^-24) build up to about
// K u^2 |sum| over K terms; folding every few terms keeps |c| <= ulp(s) and the
// error near sqrt(K) u^2.  When |s| < |c| the fold is still within u min(|s|, |c|).
__device__ __forceinline__ void df_acc_renorm(df_acc &acc) {
    float s, c;
    fast_two_sum(acc.s, acc.c, s, c);
    acc.s = s;
    acc.c = c;
}

// acc += x (a double-word value)
__device__ __forceinline__ void df_acc_add(df_acc &acc, df64 x) {
    float s, t;
    two_sum(acc.s, x.hi, s, t);
    acc.s = s;
    acc.c = __fadd_rn(acc.c, __fadd_rn(t, x.lo));
}

__device__ __forceinline__ df64 df_acc_value(df_acc a) {
    float h, l;
    fast_two_sum(a.s, a.c, h, l);
    // fast_two_sum needs |s| >= |c|; when s is tiny against c (cancellation
    // to below the error term) fall back to the general two_sum.
    if (fabsf(a.s) < fabsf(a.c)) two_sum(a.s, a.c, h, l);
    return df_make(h, l);
}

__device__ __forceinline__ df64 df_sqrt(df64 a) {
    // one Newton step on the binary32 root (Karp & Markstein style):
    // r = sqrt(hi); result = r + (a - r*r) / (2 r)
    if (a.hi <= 0.f) return df_make(0.f, 0.f);
    float r = sqrtf(a.hi);
    float p = __fmul_rn(r, r);
    float pe = __fmaf_rn(r, r, -p);
    float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
    float corr = __fdiv_rn(d, __fmul_rn(2.f, r));
    float h, l;
    fast_two_sum(r, corr, h, l);
    return df_make(h, l);
}

__device__ __forceinline__ df64 df_div(df64 a, df64 b) {
    // q1 = a.hi / b.hi; remainder r = a - q1*b (double-word); q2 = r.hi / b.hi
    float q1 = __fdiv_rn(a.hi, b.hi);
    df64 r = df_sub(a, df_mul(b, df_make(q1, 0.f)));
    float q2 = __fdiv_rn(r.hi, b.hi);
    float h, l;
    fast_two_sum(q1, q2, h, l);
    return df_make(h, l);
}

// ---------------------------------------------------------------------------
// Two accumulators in one packed register pair.  The sm_100 family executes
// add/sub/mul/fma on two binary32 lanes per instruction (PTX .f32x2), each
// lane rounded as the scalar operation: the FP32 pipe does the same work,
// but one instruction issue covers both lanes, which leaves issue slots to
// the loads and the bookkeeping of an issue-bound loop.  df_acc2 holds two
// independent Dot2 accumulators (e.g. two rows of a block); every lane sees
// exactly the operations of df_acc_fma / df_acc_fma_f / df_acc_renorm above,
// so the results are theirs bit for bit.  A subtraction a - b is written as
// a - b or as a + (-b) where that saves a negation; binary32 negation and
// round-to-nearest are symmetric, so both give the scalar result exactly.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

struct df_acc2 {
    f32x2 s, c;
};

__device__ __forceinline__ df_acc2 df_acc2_zero() {
    df_acc2 a;
    a.s = f2_pack(0.f, 0.f);
    a.c = a.s;
    return a;
}

// Negation of both lanes (sign bits flipped: exact, on the integer pipe).
__device__ __forceinline__ f32x2 f2_neg(f32x2 a) { return a ^ 0x8000000080000000ull; }

// Lane k: acc_k += (bh_k + bl_k) * y for one binary32 y (df_acc_fma_f with
// x = (bh_k, bl_k)); bhn = -bh.
__device__ __forceinline__ void df_acc2_fma_f(df_acc2 &acc, f32x2 bh, f32x2 bhn, f32x2 bl, f32x2 y) {
    const f32x2 pn = f2_mul(bhn, y);          // -p, p = bh y
    const f32x2 e = f2_fma(bh, y, pn);        // bh y - p, exact
    const f32x2 s = f2_sub(acc.s, pn);        // TwoSum(acc.s, p): s = acc.s + p
    const f32x2 bb = f2_sub(s, acc.s);
    const f32x2 t = f2_sub(f2_sub(acc.s, f2_sub(s, bb)), f2_add(pn, bb));  // (acc.s - (s - bb)) + (p - bb)
    const f32x2 c = f2_fma(bl, y, acc.c);
    acc.s = s;
    acc.c = f2_add(c, f2_add(t, e));
}

// Lane k: acc_k += (bh_k + bl_k) * (yh + yl) (df_acc_fma); bhn = -bh.
__device__ __forceinline__ void df_acc2_fma(df_acc2 &acc, f32x2 bh, f32x2 bhn, f32x2 bl, f32x2 yh, f32x2 yl) {
    const f32x2 pn = f2_mul(bhn, yh);
    const f32x2 e = f2_fma(bh, yh, pn);
    const f32x2 s = f2_sub(acc.s, pn);
    const f32x2 bb = f2_sub(s, acc.s);
    const f32x2 t = f2_sub(f2_sub(acc.s, f2_sub(s, bb)), f2_add(pn, bb));
    f32x2 c = f2_fma(bh, yl, acc.c);
    c = f2_fma(bl, yh, c);
    acc.s = s;
    acc.c = f2_add(c, f2_add(t, e));
}

// df_acc_renorm on both lanes
__device__ __forceinline__ void df_acc2_renorm(df_acc2 &acc) {
    const f32x2 s = f2_add(acc.s, acc.c);
    acc.c = f2_sub(acc.c, f2_sub(s, acc.s));
    acc.s = s;
}

// lane 0 and lane 1 as scalar accumulators
__device__ __forceinline__ void df_acc2_split(df_acc2 a, df_acc &l0, df_acc &l1) {
    f2_unpack(a.s, l0.s, l1.s);
    f2_unpack(a.c, l0.c, l1.c);
}
