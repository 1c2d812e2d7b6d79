// matvec.cuh -- parameters and shared pieces of the operator-product kernels
// (Sec. 4.1): the launch parameters, the fold points of the double-float
// accumulators, the per-row mixing and store of the s stage sums, and the
// row-group shape of the compile-time block-size kernels.  Included by
// k_matvec.cu and k_matvec_tp.cu (the TMA-fed kernels, a translation unit of
// their own so that the two compile in parallel).
#pragma once
#include <mutex>

#include "arith.cuh"

namespace irk_mv {

struct MatvecParams {
    int T, m, form, mode;
    int xf32;  // 1: every x value is binary32 (double-float with a zero low word)
    const int *rp, *ci;
    const vec8 *J, *M, *x, *rhs;
    vec8 *y;
    KCoef C[IRK_MAX_S * IRK_MAX_S];  // A^{-1} (transformed) or A (untransformed)
    KCoef mdt;                       // -dt
    // one Jacobian per stage (k_matvec_ps): J_k = J + k * jstride; A for the
    // untransformed combination sum_l a_kl x_l
    long long jstride;
    KCoef Acomb[IRK_MAX_S * IRK_MAX_S];
    // row counter of the kernels that hand out element rows dynamically
    // (zeroed by their launcher before each launch)
    int *rowctr;
};

// Columns after which every double-float accumulator of the operator product
// folds its error term into its sum (df_acc_renorm): every eighth column of a
// block and its last one.  All launch variants fold at the same columns, so
// they stay bitwise identical.
__device__ __forceinline__ bool fold_after(int c, int m) { return (c & 7) == 7 || c == m - 1; }

// Mixes the per-stage sums of row i (t_l = sum_j J_ij x_{l,j},
// z_l = M_i x_{l,i}) into the s outputs of thread row a and stores them
// (mode 1: rhs - y).  IRK_FORM_JACOBIAN: y_k = t_k (the Jacobian alone).
template <class AR, int S>
__device__ __forceinline__ void store_row(const MatvecParams &P, long long i, int a, const typename AR::acc (&t)[S],
                                          const typename AR::acc (&z)[S]) {
    typedef typename AR::val val;
    typedef typename AR::acc acc;
    const int m = P.m;
    const long long sm = (long long)S * m;
    val tv[S], zv[S];
#pragma unroll
    for (int l = 0; l < S; ++l) {
        tv[l] = AR::value(t[l]);
        zv[l] = AR::value(z[l]);
    }
    const val mdt = AR::coef(P.mdt.d, P.mdt.hi, P.mdt.lo);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        acc o = AR::zero();
        if (P.form == IRK_FORM_JACOBIAN) {
            AR::add_to(o, tv[k]);
        } else if (P.form == IRK_TRANSFORMED) {
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const KCoef &cc = P.C[k * S + l];
                AR::fma(o, AR::coef(cc.d, cc.hi, cc.lo), zv[l]);
            }
            AR::fma(o, mdt, tv[k]);
        } else {
            AR::add_to(o, zv[k]);
            acc q = AR::zero();
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const KCoef &cc = P.C[k * S + l];
                AR::fma(q, AR::coef(cc.d, cc.hi, cc.lo), tv[l]);
            }
            AR::fma(o, mdt, AR::value(q));
        }
        val out = AR::value(o);
        vec8 *dst = P.y + i * sm + k * m + a;
        if (P.mode == 1) out = AR::sub(AR::ld(P.rhs + i * sm + k * m + a), out);
        AR::st(dst, out);
    }
}

// Element rows per CTA of the look-ahead kernel: as many as fill whole warps
// (G B a multiple of 32) within 256 threads, else 256 / B.
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int sp_groups(int B) {
    return (B * 32 / gcd_c(B, 32) <= 256) ? (256 / (B * 32 / gcd_c(B, 32))) * (32 / gcd_c(B, 32)) : 256 / B;
}
__host__ __device__ constexpr int sp_threads(int B) { return (sp_groups(B) * B + 31) / 32 * 32; }

// Device limits, cached per device.
struct DevLimits {
    int sms = 0, optin = 0, per_sm = 0;
};
inline DevLimits dev_limits() {
    static std::mutex mu;
    static DevLimits cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    DevLimits &L = cached[dev & 63];
    if (L.sms == 0) {
        cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&L.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&L.per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    return L;
}

// Operator product by the TMA-fed kernels (variant forms 5-10: k_matvec_tp
// with one or two rows per thread); false when the form does not apply to
// these sizes (the caller then runs the default variant).
bool run_matvec_tp_form(const MatvecParams &P, int s, int form, int *err, cudaStream_t st);

}  // namespace irk_mv
