// k_matvec.cu -- the stage-system operator product over all s stages in one
// pass (Sec. 4.1, Table 2), plus layout conversions at the boundary.
//
// Transformed (eq. big-irk):    y_k = sum_l A^{-1}_kl M_i x_{l,i} - dt sum_j J_ij x_{k,j}
// Untransformed (eq. newton-system-2, shared J):
//                               y_k = M_i x_{k,i} - dt sum_l a_kl sum_j J_ij x_{l,j}
// Both need the same per-element sums T_l = sum_j J_ij x_{l,j} and
// Z_l = M_i x_{l,i} for every stage l; they differ only in how the s sums are
// mixed.  Each J and M block is therefore read exactly once for all stages.
//
// Mapping: a group of m threads owns one element row i; thread a owns output
// row a of that block row for all s stages (s independent accumulators).
// Blocks are stored column-major on the device (element (a, c) at c*m + a),
// so the m threads of a group read consecutive words of every column:
// coalesced, and each J / M value is loaded by exactly one thread.  The
// stage vectors of the neighbour j (element-interleaved, s*m contiguous
// values) are read by all m threads of the group at the same address
// (a broadcast through L1).
#include "arith.cuh"

namespace {

struct MatvecParams {
    int T, m, form, mode;
    const int *rp, *ci;
    const vec8 *J, *M, *x, *rhs;
    vec8 *y;
    KCoef C[IRK_MAX_S * IRK_MAX_S];  // A^{-1} (transformed) or A (untransformed)
    KCoef mdt;                       // -dt
};

// dst[l] += sum_c B[c][a] x[l][c] for one column-major block (thread's row a
// pre-applied to B).  Chunks of CH columns: all loads of a chunk are issued
// before its arithmetic, so every thread keeps CH block loads in flight.
template <class AR, int S, int CH>
__device__ __forceinline__ void accum_block(typename AR::acc (&dst)[S], const vec8 *B, const vec8 *x, int m) {
    typedef typename AR::val val;
    for (int c0 = 0; c0 < m; c0 += CH) {
        val bv[CH], xv[S][CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) bv[u] = (c0 + u < m) ? AR::ld(B + (long long)(c0 + u) * m) : AR::from_float(0.f);
#pragma unroll
        for (int l = 0; l < S; ++l)
#pragma unroll
            for (int u = 0; u < CH; ++u) xv[l][u] = (c0 + u < m) ? AR::ld(x + l * m + c0 + u) : AR::from_float(0.f);
#pragma unroll
        for (int u = 0; u < CH; ++u)
#pragma unroll
            for (int l = 0; l < S; ++l) AR::fma(dst[l], bv[u], xv[l][u]);
    }
}

template <class AR, int S, int CH>
__global__ void __launch_bounds__(256) k_matvec(MatvecParams P) {
    typedef typename AR::val val;
    typedef typename AR::acc acc;
    const int m = P.m;
    const int groups = blockDim.x / m;
    const int g = threadIdx.x / m;
    const int a = threadIdx.x - g * m;
    if (g >= groups) return;
    const long long mm = (long long)m * m;
    const long long sm = (long long)S * m;
    for (long long i = (long long)blockIdx.x * groups + g; i < P.T; i += (long long)gridDim.x * groups) {
        acc t[S], z[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
            t[l] = AR::zero();
            z[l] = AR::zero();
        }
        const int p0 = P.rp[i], p1 = P.rp[i + 1];
        for (int p = p0; p < p1; ++p)
            accum_block<AR, S, CH>(t, P.J + (long long)p * mm + a, P.x + (long long)P.ci[p] * sm, m);
        accum_block<AR, S, CH>(z, P.M + i * mm + a, P.x + i * sm, m);
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
            if (P.form == IRK_TRANSFORMED) {
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
}

template <class AR>
__global__ void k_to_internal(long long N, int T, int m, int s, const double *__restrict__ src, vec8 *dst) {
    // dst[(i*s + k)*m + a] = src[(k*T + i)*m + a]
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        long long a = e % m;
        long long r = e / m;
        long long k = r % s;
        long long i = r / s;
        AR::st(dst + e, AR::from_double(src[(k * T + i) * m + a]));
    }
}

template <class AR>
__global__ void k_to_external(long long N, int T, int m, int s, const vec8 *__restrict__ src, double *dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        long long a = e % m;
        long long r = e / m;
        long long k = r % s;
        long long i = r / s;
        dst[(k * T + i) * m + a] = AR::to_double(AR::ld(src + e));
    }
}

template <class AR>
__global__ void k_convert_blocks(long long total, int m, const double *__restrict__ src, vec8 *dst) {
    // row-major source block element (a, c) -> column-major destination
    const long long mm = (long long)m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long blk = e / mm;
        long long r = e - blk * mm;
        long long c = r / m, a = r - c * m;
        AR::st(dst + e, AR::from_double(src[blk * mm + a * m + c]));
    }
}

int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    if (g > 152LL * 16) g = 152LL * 16;
    if (g < 1) g = 1;
    return (int)g;
}

template <class AR, int S>
void run_matvec(const MatvecParams &P, cudaStream_t st) {
    int groups = 256 / P.m;
    int threads = groups * P.m;
    threads = (threads + 31) / 32 * 32;
    long long g = (P.T + groups - 1) / groups;
    // chunk width: 8 columns for up to 3 stages, 4 beyond (register budget)
    if (S <= 3)
        k_matvec<AR, S, 8><<<(int)g, threads, 0, st>>>(P);
    else
        k_matvec<AR, S, 4><<<(int)g, threads, 0, st>>>(P);
}

template <class AR>
void dispatch_s(int s, const MatvecParams &P, cudaStream_t st) {
    switch (s) {
        case 1: run_matvec<AR, 1>(P, st); break;
        case 2: run_matvec<AR, 2>(P, st); break;
        case 3: run_matvec<AR, 3>(P, st); break;
        case 4: run_matvec<AR, 4>(P, st); break;
        case 5: run_matvec<AR, 5>(P, st); break;
        case 6: run_matvec<AR, 6>(P, st); break;
        case 7: run_matvec<AR, 7>(P, st); break;
        default: run_matvec<AR, 8>(P, st); break;
    }
}

}  // namespace

int launch_matvec(irk_ctx *c, const vec8 *x, vec8 *y, const vec8 *rhs, double dt, int mode) {
    MatvecParams P;
    P.T = c->T;
    P.m = c->m;
    P.form = c->opt.formulation;
    P.mode = mode;
    P.rp = c->d_rp;
    P.ci = c->d_ci;
    P.J = c->d_J;
    P.M = c->d_M;
    P.x = x;
    P.rhs = rhs;
    P.y = y;
    const double *C = (P.form == IRK_TRANSFORMED) ? c->Ainv : c->A;
    for (int q = 0; q < c->s * c->s; ++q) P.C[q] = make_kcoef(C[q]);
    P.mdt = make_kcoef(-dt);
    if (c->df)
        dispatch_s<ArDF>(c->s, P, c->stream);
    else
        dispatch_s<ArF64>(c->s, P, c->stream);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_to_internal(irk_ctx *c, const double *src, vec8 *dst) {
    int g = grid_for(c->N, 256);
    if (c->df)
        k_to_internal<ArDF><<<g, 256, 0, c->stream>>>(c->N, c->T, c->m, c->s, src, dst);
    else
        k_to_internal<ArF64><<<g, 256, 0, c->stream>>>(c->N, c->T, c->m, c->s, src, dst);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_to_external(irk_ctx *c, const vec8 *src, double *dst) {
    int g = grid_for(c->N, 256);
    if (c->df)
        k_to_external<ArDF><<<g, 256, 0, c->stream>>>(c->N, c->T, c->m, c->s, src, dst);
    else
        k_to_external<ArF64><<<g, 256, 0, c->stream>>>(c->N, c->T, c->m, c->s, src, dst);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_convert_blocks(irk_ctx *c, const double *src, vec8 *dst, long long nblocks) {
    long long total = nblocks * c->m * c->m;
    int g = grid_for(total, 256);
    if (c->df)
        k_convert_blocks<ArDF><<<g, 256, 0, c->stream>>>(total, c->m, src, dst);
    else
        k_convert_blocks<ArF64><<<g, 256, 0, c->stream>>>(total, c->m, src, dst);
    c->launches++;
    return cuda_status(cudaGetLastError());
}
