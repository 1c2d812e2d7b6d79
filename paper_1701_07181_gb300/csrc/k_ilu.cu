// k_ilu.cu -- block ILU(0) preconditioners (Sec. 4.2-4.3): assembly of the
// system blocks, level-scheduled factorisation and level-scheduled forward /
// backward block sweeps, all s stages in the same launches.
//
// One generic engine serves every preconditioner kind: the host assembles the
// block pattern of the matrix to factor (Sec. 4.3.2: s stage matrices
// (A^{-1}_kk + alpha_k) M - dt J side by side; Sec. 4.3.1 / Alg. 3: the whole
// stage-major system; or the element-major system with (s m)-blocks), and the
// device factorises it in the textbook row-by-row (IKJ) form of block ILU(0)
// (Alg. 1 with the i < k < j updates; equal to Alg. 2 / Alg. 3 when no two
// neighbours of an element are neighbours).  Rows with no dependency between
// them form a level; each level is one launch, one CTA per block row.
//
// Blocks are column-major on the device; the diagonal block of every row is
// stored as its explicit inverse D^{-1} (computed by Gauss-Jordan elimination
// with partial pivoting), so the backward sweep is two block products.
#include <cuda_bf16.h>

#include <stdlib.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "arith.cuh"
#include "tma.cuh"

#define IRK_MAX_GJ 256

namespace {


// Allow a kernel the device's full opt-in dynamic shared memory, once per
// kernel.  The attribute is per function and global to the process: setting
// it to each launch's own size would race between contexts / groups launching
// the same kernel from different threads with different block sizes.
int allow_max_smem(const void *func) {
    static std::mutex mu;
    static std::vector<const void *> done;
    std::lock_guard<std::mutex> g(mu);
    for (const void *f : done)
        if (f == func) return IRK_OK;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, func) != cudaSuccess)
        return IRK_ERR_CUDA;
    // the dynamic limit excludes the kernel's static shared memory
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
        return IRK_ERR_CUDA;
    done.push_back(func);
    return IRK_OK;
}

// Threads per inversion CTA (k_factor_diag) and the level width from which a
// level's inversions leave the product kernel (irk_kernel_options; 0 = the
// defaults 128 and 2048).
int gj_threads(const irk_ctx *c) {
    return c->ko.factor_gj_threads > 0 ? std::max(32, std::min(256, c->ko.factor_gj_threads)) : 128;
}
int gj_split_min(const irk_ctx *c) { return c->ko.factor_gj_split_min > 0 ? c->ko.factor_gj_split_min : 2048; }

// ---------------------------------------------------------------------------
// factor-storage loads (binary64, binary32 or bfloat16 storage)
__device__ __forceinline__ double ldfac(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldfac(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldfac(const __nv_bfloat16 *p) { return __bfloat162float(p[0]); }

template <class C>
struct CT;  // compute-type helpers
template <>
struct CT<double> {
    template <class AR>
    static __device__ __forceinline__ double from_vec(typename AR::val v) { return AR::to_double(v); }
    template <class AR>
    static __device__ __forceinline__ typename AR::val to_vec(double x) { return AR::from_double(x); }
    static __device__ __forceinline__ double from_store(vec8 raw, int df) {
        if (df) {
            float2 f = *reinterpret_cast<float2 *>(&raw);
            return (double)f.x + (double)f.y;
        }
        return __longlong_as_double((long long)raw);
    }
};
template <>
struct CT<float> {
    template <class AR>
    static __device__ __forceinline__ float from_vec(typename AR::val v) { return AR::to_float(v); }
    template <class AR>
    static __device__ __forceinline__ typename AR::val to_vec(float x) { return AR::from_float(x); }
    static __device__ __forceinline__ float from_store(vec8 raw, int df) {
        if (df) {
            float2 f = *reinterpret_cast<float2 *>(&raw);
            return f.x + f.y;
        }
        return (float)__longlong_as_double((long long)raw);
    }
};

// ---------------------------------------------------------------------------
// Assembly (stage-major kinds): value = cm[cm_id] * M[mi] + cj[cj_id] * J[jp]
struct AsmTables {
    double cm[IRK_MAX_S * IRK_MAX_S];
    double cj[IRK_MAX_S * IRK_MAX_S];
};

template <class C>
__global__ void __launch_bounds__(256) k_assemble(long long nnz, int m, const AsmEntry *ent, const vec8 *J,
                                                  const vec8 *M, int df, AsmTables tab, C *vals) {
    // one block per CTA iteration: the entry and its coefficients are
    // uniform, the threads stream the block's m*m values
    const int mm = m * m;
    for (long long q = blockIdx.x; q < nnz; q += gridDim.x) {
        const AsmEntry a = ent[q];
        const vec8 *Mb = a.mi >= 0 ? M + (long long)a.mi * mm : nullptr;
        const vec8 *Jb = a.jp >= 0 ? J + (long long)a.jp * mm : nullptr;
        const C cm = Mb ? (C)tab.cm[a.cm_id] : C(0);
        const C cj = Jb ? (C)tab.cj[a.cj_id] : C(0);
        C *out = vals + q * mm;
        for (int r = threadIdx.x; r < mm; r += blockDim.x) {
            C v = C(0);
            if (Mb) v += cm * CT<C>::from_store(Mb[r], df);
            if (Jb) v += cj * CT<C>::from_store(Jb[r], df);
            out[r] = v;
        }
    }
}

// Uncoupled kind with one shared J: the s stage systems list their blocks
// in the same order (stage k's entry q0 + k * per_stage has stage 0's J and
// M blocks), so one CTA reads a J block (and the mass block on the
// diagonal) once and writes all s assembled blocks d_k M - dt J, each with
// k_assemble's arithmetic.  Entries are read from stage 0's part of the table.
__device__ __forceinline__ void store_pair(float *p, const float (&v)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
__device__ __forceinline__ void store_pair(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

template <class C>
__global__ void __launch_bounds__(256, 4) k_assemble_stages(long long per_stage, int s, int m, const AsmEntry *ent,
                                                         const vec8 *J, const vec8 *M, int df, AsmTables tab,
                                                         C *vals) {
    const int mm = m * m;
    for (long long q = blockIdx.x; q < per_stage; q += gridDim.x) {
        const AsmEntry a = ent[q];
        const vec8 *Mb = a.mi >= 0 ? M + (long long)a.mi * mm : nullptr;
        const vec8 *Jb = a.jp >= 0 ? J + (long long)a.jp * mm : nullptr;
        const C cj = Jb ? (C)tab.cj[a.cj_id] : C(0);
        C cmk[IRK_MAX_S];
#pragma unroll
        for (int k = 0; k < IRK_MAX_S; ++k) cmk[k] = (Mb && k < s) ? (C)tab.cm[k * s + k] : C(0);
        if ((mm & 1) == 0) {
            // pairs of entries: 16-byte loads of J and M, two pairs per
            // thread with every load issued before the stores
            const int pairs = mm >> 1;
            const uint4 *J2 = reinterpret_cast<const uint4 *>(Jb), *M2 = reinterpret_cast<const uint4 *>(Mb);
            for (int e0 = threadIdx.x; e0 < pairs; e0 += 2 * blockDim.x) {
                uint4 jr[2], mr[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = e0 + u * blockDim.x;
                    const bool ok = e < pairs;
                    jr[u] = (ok && Jb) ? __ldg(J2 + e) : make_uint4(0, 0, 0, 0);
                    mr[u] = (ok && Mb) ? __ldg(M2 + e) : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e >= pairs) break;
                    C mv[2], jv[2];
                    const vec8 jraw[2] = {((vec8)jr[u].y << 32) | jr[u].x, ((vec8)jr[u].w << 32) | jr[u].z};
                    const vec8 mraw[2] = {((vec8)mr[u].y << 32) | mr[u].x, ((vec8)mr[u].w << 32) | mr[u].z};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        mv[h] = Mb ? CT<C>::from_store(mraw[h], df) : C(0);
                        jv[h] = Jb ? CT<C>::from_store(jraw[h], df) : C(0);
                    }
#pragma unroll
                    for (int k = 0; k < IRK_MAX_S; ++k) {
                        if (k >= s) break;
                        C v[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            v[h] = C(0);
                            if (Mb) v[h] += cmk[k] * mv[h];
                            if (Jb) v[h] += cj * jv[h];
                        }
                        store_pair(vals + (q + k * per_stage) * mm + 2 * e, v);
                    }
                }
            }
            continue;
        }
        for (int r = threadIdx.x; r < mm; r += blockDim.x) {
            const C mv = Mb ? CT<C>::from_store(Mb[r], df) : C(0);
            const C jv = Jb ? CT<C>::from_store(Jb[r], df) : C(0);
#pragma unroll
            for (int k = 0; k < IRK_MAX_S; ++k) {
                if (k >= s) break;
                C v = C(0);
                if (Mb) v += cmk[k] * mv;
                if (Jb) v += cj * jv;
                vals[(q + k * per_stage) * mm + r] = v;
            }
        }
    }
}

// Element-major assembly: one (s m) x (s m) block per J block p, entry
// ((k,a),(l,c)) at column-major index (l m + c) * sm + (k m + a).
//   form 0: C_kl M_i[a][c] [diag] - dt [k==l] J_p[a][c]
//   form 1: [k==l][diag] M_i[a][c] - dt C_kl J_p[a][c]
template <class C>
__global__ void k_assemble_elem(long long nnzb, int s, int m, int form, const int *rowof, const int *ci,
                                const vec8 *J, long long jstride, const vec8 *M, int df, AsmTables tab, double dt,
                                C *vals) {
    const long long sm = (long long)s * m, blk = sm * sm, mm = (long long)m * m;
    const long long total = nnzb * blk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long p = e / blk, r = e - p * blk;
        long long colbig = r / sm, rowbig = r - colbig * sm;
        int l = (int)(colbig / m), c = (int)(colbig - (long long)l * m);
        int k = (int)(rowbig / m), a = (int)(rowbig - (long long)k * m);
        int i = rowof[p];
        bool diag = (ci[p] == i);
        // stage k's rows use J_k (jstride = 0: one J shared by the stages)
        double Jv = (double)CT<C>::from_store(J[k * jstride + p * mm + (long long)c * m + a], df);
        double Mv = diag ? (double)CT<C>::from_store(M[(long long)i * mm + (long long)c * m + a], df) : 0.0;
        double coef = tab.cm[k * s + l];
        double v = (form == 0) ? coef * Mv - (k == l ? dt * Jv : 0.0) : (k == l ? Mv : 0.0) - dt * coef * Jv;
        vals[e] = (C)v;
    }
}

// ---------------------------------------------------------------------------
// Factorisation of one level: one CTA per block row R of the level.
//   for lower entries p of row R (increasing column i):
//       L_p = B_p D_i^{-1};  B_q -= L_p B_pos for the (q, pos) update pairs of p
//   D_R^{-1} = inverse(B_RR)
// Shared memory: two b x b buffers of the compute type.
template <class C>
__device__ void block_load(C *dst, const C *src, int bb) {
    for (int e = threadIdx.x; e < bb; e += blockDim.x) dst[e] = src[e];
}

// dst(b x b, global) = X (smem) * Y (smem), column-major
template <class C>
__device__ void block_mul_store(C *dst, const C *X, const C *Y, int b) {
    const int bb = b * b;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        int col = e / b, row = e - col * b;
        C acc = 0;
        for (int t = 0; t < b; ++t) acc += X[t * b + row] * Y[col * b + t];
        dst[e] = acc;
    }
}

// dst(global) -= X (smem) * Y (smem)
template <class C>
__device__ void block_mul_sub(C *dst, const C *X, const C *Y, int b) {
    const int bb = b * b;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        int col = e / b, row = e - col * b;
        C acc = 0;
        for (int t = 0; t < b; ++t) acc += X[t * b + row] * Y[col * b + t];
        dst[e] -= acc;
    }
}

// In-place Gauss-Jordan inversion with partial (row) pivoting of the b x b
// column-major matrix A in shared memory; the inverse is written to Out
// (shared memory).  Step k: pivot row p = argmax_{r >= k} |A(r,k)|, swap rows
// k and p, scale row k by 1/A(k,k) with A(k,k) replaced by 1, and eliminate
// column k from every other row with A(r,k) replaced by 0.  The in-place
// result is (P A)^{-1} for the row permutation P; the inverse of A is that
// matrix with its columns permuted back (swaps undone in reverse order).
// Thread layout: thread t updates row r = t % b for columns t / b, t / b + G,
// ... (G = blockDim / b groups): consecutive threads touch consecutive words
// of a column (no shared-memory bank conflicts).  Returns false on an exactly
// zero pivot.
template <class C>
__device__ bool gauss_jordan(C *A, C *Out, int b, C *fcol) {
    __shared__ int s_piv[IRK_MAX_GJ];
    __shared__ C s_pval;
    __shared__ int s_bad;
    const int G = blockDim.x / b;
    const int g = threadIdx.x / b, r = threadIdx.x - g * b;
    const bool act = g < G;
    if (threadIdx.x == 0) s_bad = 0;
    for (int k = 0; k < b; ++k) {
        if (threadIdx.x < 32) {
            C best = -1;
            int bi = k;
            for (int r = k + threadIdx.x; r < b; r += 32) {
                C v = fabs(A[k * b + r]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int d = 16; d > 0; d >>= 1) {
                C ob = __shfl_down_sync(0xffffffffu, best, d);
                int oi = __shfl_down_sync(0xffffffffu, bi, d);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (threadIdx.x == 0) {
                s_piv[k] = bi;
                s_pval = A[k * b + bi];
                if (!(best > C(0))) {
                    s_bad = 1;
                    s_pval = C(1);
                }
            }
        }
        __syncthreads();
        const int p = s_piv[k];
        const C pinv = C(1) / s_pval;
        // swap rows k and p; save column k (post-swap) for the elimination
        for (int cc = threadIdx.x; cc < b; cc += blockDim.x) {
            if (p != k) {
                C t = A[cc * b + k];
                A[cc * b + k] = A[cc * b + p];
                A[cc * b + p] = t;
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < b; r += blockDim.x) fcol[r] = A[k * b + r];
        __syncthreads();
        // scale row k (A(k,k) := 1 first)
        for (int cc = threadIdx.x; cc < b; cc += blockDim.x) A[cc * b + k] = (cc == k ? C(1) : A[cc * b + k]) * pinv;
        __syncthreads();
        if (act && r != k) {
            const C f = fcol[r];
            for (int cc = g; cc < b; cc += G) A[cc * b + r] = (cc == k ? C(0) : A[cc * b + r]) - f * A[cc * b + k];
        }
        __syncthreads();
    }
    // undo the row interchanges on the columns: Out(:, j) = A(:, idx[j])
    __shared__ int s_idx[IRK_MAX_GJ];
    if (threadIdx.x == 0) {
        for (int j = 0; j < b; ++j) s_idx[j] = j;
        for (int k = b - 1; k >= 0; --k) {
            int q = s_piv[k];
            int t = s_idx[k];
            s_idx[k] = s_idx[q];
            s_idx[q] = t;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        int j = e / b, r = e - j * b;
        Out[e] = A[s_idx[j] * b + r];
    }
    __syncthreads();
    return s_bad == 0;
}

template <class C>
__global__ void __launch_bounds__(256) k_factor_level(const int *rows, int b, const int *rp, const int *ci,
                                                      const int *diag, const int *upd_ptr, const int *upd,
                                                      C *vals, C *dinv, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *X = reinterpret_cast<C *>(smem_raw);
    C *Y = X + b * b;
    C *fcol = Y + b * b;
    const int R = rows[blockIdx.x];
    const long long bb = (long long)b * b;
    for (int p = rp[R]; p < rp[R + 1]; ++p) {
        const int i = ci[p];
        if (i >= R) break;
        // L_p = B_p D_i^{-1}
        block_load(X, vals + (long long)p * bb, (int)bb);
        block_load(Y, dinv + (long long)i * bb, (int)bb);
        __syncthreads();
        block_mul_store(vals + (long long)p * bb, X, Y, b);
        __syncthreads();
        block_load(X, vals + (long long)p * bb, (int)bb);  // X = L_p
        __syncthreads();
        for (int u = upd_ptr[p]; u < upd_ptr[p + 1]; ++u) {
            const int q = upd[2 * u], pos = upd[2 * u + 1];
            block_load(Y, vals + (long long)pos * bb, (int)bb);
            __syncthreads();
            block_mul_sub(vals + (long long)q * bb, X, Y, b);
            __syncthreads();
        }
    }
    block_load(X, vals + (long long)diag[R] * bb, (int)bb);
    __syncthreads();
    bool ok = gauss_jordan(X, Y, b, fcol);
    for (int e = threadIdx.x; e < bb; e += blockDim.x) dinv[(long long)R * bb + e] = Y[e];
    if (!ok && threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_SINGULAR);
}

// Gauss-Jordan with three barriers per pivot (the fast path of the
// factorisation).  Same algorithm and result as gauss_jordan above: phase 1
// finds the pivot; phase 2 performs the row interchange and the scaling of
// the pivot row together (each thread owns whole columns c != k) and saves
// the post-interchange pivot column; phase 3 eliminates, writing column k as
// -f_r / pivot (rows r != k) and 1 / pivot (row k).  A has leading dimension
// ld (an odd ld = b + 1 keeps the row accesses of phase 2 free of shared-
// memory bank conflicts); Out is b x b column-major.
template <class C>
__device__ bool gauss_jordan3(C *A, C *Out, int b, C *fcol, int ld) {
    __shared__ int s_piv[IRK_MAX_GJ];
    __shared__ C s_pinv;
    __shared__ int s_bad;
    const int G = blockDim.x / b;
    const int g = threadIdx.x / b, r = threadIdx.x - g * b;
    const bool act = g < G;
    if (threadIdx.x == 0) s_bad = 0;
    for (int k = 0; k < b; ++k) {
        if (threadIdx.x < 32) {
            C best = -1;
            int bi = k;
            for (int rr = k + threadIdx.x; rr < b; rr += 32) {
                C v = fabs(A[k * ld + rr]);
                if (v > best) {
                    best = v;
                    bi = rr;
                }
            }
            for (int d = 16; d > 0; d >>= 1) {
                C ob = __shfl_down_sync(0xffffffffu, best, d);
                int oi = __shfl_down_sync(0xffffffffu, bi, d);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (threadIdx.x == 0) {
                s_piv[k] = bi;
                C pv = A[k * ld + bi];
                if (!(best > C(0))) {
                    s_bad = 1;
                    pv = C(1);
                }
                s_pinv = C(1) / pv;
            }
        }
        __syncthreads();
        const int p = s_piv[k];
        const C pinv = s_pinv;
        for (int t = threadIdx.x; t < 2 * b; t += blockDim.x) {
            if (t < b) {
                // column save (post-interchange view of column k)
                const int rr = t;
                const int src = (rr == k) ? p : (rr == p ? k : rr);
                fcol[rr] = A[k * ld + src];
            } else {
                const int cc = t - b;
                if (cc == k) continue;
                const C ak = A[cc * ld + k], ap = A[cc * ld + p];
                A[cc * ld + k] = ap * pinv;
                if (p != k) A[cc * ld + p] = ak;
            }
        }
        __syncthreads();
        if (act) {
            if (r != k) {
                const C f = fcol[r];
                for (int cc = g; cc < b; cc += G)
                    A[cc * ld + r] = (cc == k) ? -f * pinv : A[cc * ld + r] - f * A[cc * ld + k];
            } else if (g == 0) {
                A[k * ld + k] = pinv;
            }
        }
        __syncthreads();
    }
    __shared__ int s_idx[IRK_MAX_GJ];
    if (threadIdx.x == 0) {
        for (int j = 0; j < b; ++j) s_idx[j] = j;
        for (int kk = b - 1; kk >= 0; --kk) {
            int q = s_piv[kk];
            int t = s_idx[kk];
            s_idx[kk] = s_idx[q];
            s_idx[q] = t;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        int j = e / b, rr = e - j * b;
        Out[e] = A[s_idx[j] * ld + rr];
    }
    __syncthreads();
    return s_bad == 0;
}

// Register-tiled block product on shared-memory operands (column-major):
// P = X Y, each thread owning a 4 x 2 tile of P (8 independent accumulation
// chains).  mode 0: dst1 = P (and dst2 = P when dst2 != nullptr);
// mode 1: dst1 -= P.
template <class C>
__device__ __forceinline__ void tile_gemm(C *dst1, C *dst2, const C *X, const C *Y, int b, int mode) {
    const int nrt = (b + 3) / 4, nct = (b + 1) / 2;
    for (int tile = threadIdx.x; tile < nrt * nct; tile += blockDim.x) {
        const int r0 = (tile % nrt) * 4, c0 = (tile / nrt) * 2;
        C acc[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = C(0);
        const bool c1ok = c0 + 1 < b;
        for (int t = 0; t < b; ++t) {
            C xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = (r0 + u < b) ? X[t * b + r0 + u] : C(0);
            const C y0 = Y[c0 * b + t];
            const C y1 = c1ok ? Y[(c0 + 1) * b + t] : C(0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[u][0] += xv[u] * y0;
                acc[u][1] += xv[u] * y1;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (r0 + u >= b) continue;
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                if (v == 1 && !c1ok) continue;
                const int e = (c0 + v) * b + r0 + u;
                if (mode == 0) {
                    dst1[e] = acc[u][v];
                    if (dst2) dst2[e] = acc[u][v];
                } else {
                    dst1[e] -= acc[u][v];
                }
            }
        }
    }
}

// Tensor-core block product for FP32 factors: P = X Y (column-major b x b in
// shared memory) with mma.sync m16n8k8 on TF32 operands, each operand split
// into a TF32 head and a TF32 tail so that P = Xh Yh + Xh Yt + Xt Yh keeps
// about FP32 accuracy (the "3xTF32" scheme).  Dimensions are padded with zeros
// to multiples of 16 (rows) and 8 (columns, inner).  Fragment layout of the
// m16n8k8 .tf32 shape (PTX ISA): with g = lane / 4, t = lane % 4,
//   A: a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
//   B: b0 (t, g), b1 (t+4, g)
//   C: c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1).
// mode 0: dst1 = P (dst2 too when non-null); mode 1: dst1 -= P.
__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 16 x 8 output tile of X * Y (column-major b x b operands in shared
// memory) accumulated into d with 3xTF32: each operand split into a TF32 high
// part and a TF32 remainder, three m16n8k8 products per k-step (the small
// terms first).
__device__ __forceinline__ void tc_tile(float (&d)[4], const float *X, const float *Y, int b, int r0, int c0) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int kt = (b + 7) / 8;
    for (int kk = 0; kk < kt; ++kk) {
        const int k0 = kk * 8;
        float av[4], bv[2];
        const int ar[4] = {r0 + g, r0 + g + 8, r0 + g, r0 + g + 8};
        const int ak[4] = {k0 + t, k0 + t, k0 + t + 4, k0 + t + 4};
#pragma unroll
        for (int q = 0; q < 4; ++q) av[q] = (ar[q] < b && ak[q] < b) ? X[ak[q] * b + ar[q]] : 0.f;
        const int bk[2] = {k0 + t, k0 + t + 4};
        const int bc = c0 + g;
#pragma unroll
        for (int q = 0; q < 2; ++q) bv[q] = (bk[q] < b && bc < b) ? Y[bc * b + bk[q]] : 0.f;
        unsigned ah[4], al[4], bh[2], bl[2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ah[q] = to_tf32(av[q]);
            al[q] = to_tf32(av[q] - __uint_as_float(ah[q]));
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            bh[q] = to_tf32(bv[q]);
            bl[q] = to_tf32(bv[q] - __uint_as_float(bh[q]));
        }
        mma_tf32(d, al, bh);  // small terms first
        mma_tf32(d, ah, bl);
        mma_tf32(d, ah, bh);
    }
}

// Writes (mode 0: dst1 = d, and dst2 = d when non-null) or subtracts
// (mode 1: dst1 -= d) a tile's accumulator.
__device__ __forceinline__ void tc_store(const float (&d)[4], float *dst1, float *dst2, int b, int r0, int c0,
                                         int mode) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int rr[4] = {r0 + g, r0 + g, r0 + g + 8, r0 + g + 8};
    const int cc[4] = {c0 + 2 * t, c0 + 2 * t + 1, c0 + 2 * t, c0 + 2 * t + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (rr[q] >= b || cc[q] >= b) continue;
        const int e = cc[q] * b + rr[q];
        if (mode == 0) {
            dst1[e] = d[q];
            if (dst2) dst2[e] = d[q];
        } else {
            dst1[e] -= d[q];
        }
    }
}

__device__ void tc_gemm(float *dst1, float *dst2, const float *X, const float *Y, int b, int mode) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int mt = (b + 15) / 16, nt = (b + 7) / 8;
    for (int tile = warp; tile < mt * nt; tile += nwarps) {
        const int r0 = (tile % mt) * 16, c0 = (tile / mt) * 8;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        tc_tile(d, X, Y, b, r0, c0);
        tc_store(d, dst1, dst2, b, r0, c0, mode);
    }
}

template <class C>
__device__ __forceinline__ void block_product(C *dst1, C *dst2, const C *X, const C *Y, int b, int mode);
template <>
__device__ __forceinline__ void block_product<float>(float *dst1, float *dst2, const float *X, const float *Y, int b,
                                                     int mode) {
    tc_gemm(dst1, dst2, X, Y, b, mode);
}
template <>
__device__ __forceinline__ void block_product<double>(double *dst1, double *dst2, const double *X, const double *Y,
                                                      int b, int mode) {
    tile_gemm<double>(dst1, dst2, X, Y, b, mode);
}

// Load two b x b blocks from global memory into shared memory with every
// thread's loads issued before its stores (one memory round trip).
template <class C>
__device__ __forceinline__ void load_pair(C *d1, const C *s1, C *d2, const C *s2, int bb) {
    for (int e0 = threadIdx.x; e0 < bb; e0 += 4 * blockDim.x) {
        C v1[4], v2[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            v1[u] = (e < bb) ? __ldg(s1 + e) : C(0);
            v2[u] = (s2 && e < bb) ? __ldg(s2 + e) : C(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < bb) {
                d1[e] = v1[u];
                if (s2) d2[e] = v2[u];
            }
        }
    }
}

// Factorisation of one level, fast path: four b x b shared buffers (X, Y, L,
// D) + b.  D (the row's diagonal block) stays in shared memory for the whole
// row; L_p = B_p D_i^{-1} is formed in shared memory and written once.
template <class C>
__global__ void __launch_bounds__(256) k_factor_level2(const int *rows, int b, const int *rp, const int *ci,
                                                       const int *diag, const int *upd_ptr, const int *upd,
                                                       C *vals, C *dinv, int *err, int do_inverse) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bb = b * b;
    C *X = reinterpret_cast<C *>(smem_raw);  // b * (b + 1): also the padded copy for Gauss-Jordan
    C *Y = X + bb + b;
    C *L = Y + bb;
    C *D = L + bb;
    C *fcol = D + bb;
    const int R = rows[blockIdx.x];
    const int dpos = diag[R];
    load_pair<C>(D, vals + (long long)dpos * bb, nullptr, nullptr, bb);
    for (int p = rp[R]; p < rp[R + 1]; ++p) {
        const int i = ci[p];
        if (i >= R) break;
        load_pair<C>(X, vals + (long long)p * bb, Y, dinv + (long long)i * bb, bb);
        __syncthreads();
        block_product<C>(L, vals + (long long)p * bb, X, Y, b, 0);  // L_p = B_p D_i^{-1}
        __syncthreads();
        for (int u = upd_ptr[p]; u < upd_ptr[p + 1]; ++u) {
            const int q = upd[2 * u], pos = upd[2 * u + 1];
            load_pair<C>(X, vals + (long long)pos * bb, nullptr, nullptr, bb);
            __syncthreads();
            block_product<C>((q == dpos) ? D : vals + (long long)q * bb, nullptr, L, X, b, 1);  // B_q -= L_p B_pos
            __syncthreads();
        }
    }
    // D to global (the U~ diagonal block) and to X with leading dimension b + 1
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const int col = e / b, row = e - col * b;
        vals[(long long)dpos * bb + e] = D[e];
        X[col * (b + 1) + row] = D[e];
    }
    if (!do_inverse) return;  // k_factor_diag inverts it
    __syncthreads();
    const bool ok = gauss_jordan3(X, Y, b, fcol, b + 1);
    for (int e = threadIdx.x; e < bb; e += blockDim.x) dinv[(long long)R * bb + e] = Y[e];
    if (!ok && threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_SINGULAR);
}

// Factorisation of one level (binary32 factors) when every update of a row
// lands on its own diagonal block: the lower neighbours i_1 < ... < i_r of a
// row are pairwise non-adjacent, so the only update of entry p is
// D -= L_p U_p with U_p the block (i_p, R).  The row's blocks are then
// independent of one another's products:
//   phase 1: L_p = B_p D_{i_p}^{-1} for all p at once, spread over the warps;
//   phase 2: D -= [L_1 ... L_r] [U_1; ...; U_r], one 3xTF32 product of inner
//            size r b accumulated per 16 x 8 tile of D.
// One thread stages the row by bulk copies (B_p and D_i^{-1} on one
// mbarrier, U_p and D on a second, waited for only before phase 2).  Phase-1
// accumulators stay in registers (at most IRK_FUSED_TPW tiles per warp) until
// every warp is past its reads of B_p, then overwrite B_p in shared memory.
// The diagonal blocks are inverted afterwards by the inversion kernel.
// Shared memory: 1 + 3 rmax block slots (128-byte aligned) + two barriers.
#define IRK_FUSED_TPW 8

__device__ __forceinline__ void copy_block_out(float *dst, const float *src, int bb) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int e = threadIdx.x; e < bb / 4; e += blockDim.x) d4[e] = s4[e];
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_factor_fused(const int *rows, int b, const int *rp, const int *ci,
                                                          const int *diag, const int *upd_ptr, const int *upd,
                                                          float *vals, const float *dinv, int rmax, int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int bb = b * b;
    const unsigned blk = (unsigned)bb * 4u;  // a multiple of 16 (b even)
    const size_t stride = ((size_t)blk + 127) / 128 * 128;
    auto slot = [&](int j) { return reinterpret_cast<float *>(smem_raw + stride * j); };
    float *D = slot(0);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem_raw + stride * (1 + 3 * rmax));
    const int R = rows[blockIdx.x];
    const int p0 = rp[R], pend = rp[R + 1];
    int r = 0;
    while (r < rmax && p0 + r < pend && ci[p0 + r] < R) ++r;
    const long long dpos = diag[R];
    if (threadIdx.x == 0) {
        mbar_init(bars);
        mbar_init(bars + 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_arrive(bars, 2u * r * blk);
        for (int p = 0; p < r; ++p) {
            tma_load_1d(slot(1 + p), vals + (long long)(p0 + p) * bb, blk, bars);
            tma_load_1d(slot(1 + rmax + p), dinv + (long long)ci[p0 + p] * bb, blk, bars);
        }
        mbar_expect_arrive(bars + 1, (unsigned)(r + 1) * blk);
        tma_load_1d(D, vals + dpos * bb, blk, bars + 1);
        for (int p = 0; p < r; ++p)
            tma_load_1d(slot(1 + 2 * rmax + p), vals + (long long)upd[2 * upd_ptr[p0 + p] + 1] * bb, blk, bars + 1);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int mt = (b + 15) / 16, nt = (b + 7) / 8, ntile = mt * nt;
    // a wait that gives up: every thread drains both barriers (bounded) and
    // the CTA leaves together
    const bool ok0 = mbar_wait(bars, 0);
    if (__syncthreads_or(!ok0)) {
        if (threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_TIMEOUT);
        mbar_wait(bars, 0);
        mbar_wait(bars + 1, 0);
        return;
    }
    // phase 1: L_p tiles, item = p * ntile + tile
    float acc[IRK_FUSED_TPW][4];
#pragma unroll
    for (int j = 0; j < IRK_FUSED_TPW; ++j) {
        acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        const int item = warp + j * NW;
        if (item < r * ntile) {
            const int p = item / ntile, t = item - p * ntile;
            tc_tile(acc[j], slot(1 + p), slot(1 + rmax + p), b, (t % mt) * 16, (t / mt) * 8);
        }
    }
    __syncthreads();  // every read of B_p done
#pragma unroll
    for (int j = 0; j < IRK_FUSED_TPW; ++j) {
        const int item = warp + j * NW;
        if (item < r * ntile) {
            const int p = item / ntile, t = item - p * ntile;
            tc_store(acc[j], slot(1 + p), nullptr, b, (t % mt) * 16, (t / mt) * 8, 0);
        }
    }
    const bool ok1 = mbar_wait(bars + 1, 0);
    if (__syncthreads_or(!ok1)) {  // also publishes the L_p tiles
        if (threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_TIMEOUT);
        mbar_wait(bars + 1, 0);
        return;
    }
    for (int p = 0; p < r; ++p) copy_block_out(vals + (long long)(p0 + p) * bb, slot(1 + p), bb);
    // phase 2: each warp owns tiles of D
    for (int t = warp; t < ntile; t += NW) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const int r0 = (t % mt) * 16, c0 = (t / mt) * 8;
        for (int p = 0; p < r; ++p) tc_tile(d, slot(1 + p), slot(1 + 2 * rmax + p), b, r0, c0);
        tc_store(d, D, nullptr, b, r0, c0, 1);
    }
    __syncthreads();
    copy_block_out(vals + dpos * bb, D, bb);
}

// The same staged-row factorisation with the block size known at compile
// time.  Work is cut into row strips instead of tiles: a warp computes the
// 16 x B strip X[r0:r0+16, :] Y of a product, so each A fragment is loaded
// and split into TF32 high / remainder parts once per k-step and used for
// all ceil(B/8) column tiles, and every index is a constant.
//   phase 1: item (p, strip): L_p's strip, written over the same rows of B_p
//            in shared memory (only this warp reads those rows);
//   phase 2: item (strip, p): the partial P_p = L_p U_p of the strip, written
//            into D_{i_p}^{-1}'s slot (free after phase 1);
//   then D - ((P_1 + P_2) + ...) in a fixed order, straight to global memory.
template <int B>
__device__ __forceinline__ void strip_product(float (&acc)[(B + 7) / 8][4], const float *X, const float *Y, int r0) {
    constexpr int NT = (B + 7) / 8, KT = (B + 7) / 8;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int ra = r0 + g, rb = r0 + g + 8;
    const bool oka = ra < B, okb = rb < B;
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
        const int ka = kk * 8 + t, kb = kk * 8 + t + 4;
        const bool ka_in = ka < B, kb_in = kb < B;
        float av[4];
        av[0] = (oka && ka_in) ? X[ka * B + ra] : 0.f;
        av[1] = (okb && ka_in) ? X[ka * B + rb] : 0.f;
        av[2] = (oka && kb_in) ? X[kb * B + ra] : 0.f;
        av[3] = (okb && kb_in) ? X[kb * B + rb] : 0.f;
        unsigned ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ah[q] = to_tf32(av[q]);
            al[q] = to_tf32(av[q] - __uint_as_float(ah[q]));
        }
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int col = n * 8 + g;
            const bool cin = col < B;
            const float b0 = (cin && ka_in) ? Y[col * B + ka] : 0.f;
            const float b1 = (cin && kb_in) ? Y[col * B + kb] : 0.f;
            unsigned bh[2], bl[2];
            bh[0] = to_tf32(b0);
            bl[0] = to_tf32(b0 - __uint_as_float(bh[0]));
            bh[1] = to_tf32(b1);
            bl[1] = to_tf32(b1 - __uint_as_float(bh[1]));
            mma_tf32(acc[n], al, bh);  // small terms first
            mma_tf32(acc[n], ah, bl);
            mma_tf32(acc[n], ah, bh);
        }
    }
}

template <int B>
__device__ __forceinline__ void strip_store(const float (&acc)[(B + 7) / 8][4], float *dst, int r0) {
    constexpr int NT = (B + 7) / 8;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        const int c = n * 8 + 2 * t;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = r0 + g + (q >> 1) * 8, col = c + (q & 1);
            if (row < B && col < B) dst[col * B + row] = acc[n][q];
        }
    }
}

template <int B>
__global__ void __launch_bounds__(512) k_factor_fused_b(const int *rows, const int *rp, const int *ci,
                                                        const int *diag, const int *upd_ptr, const int *upd,
                                                        float *vals, const float *dinv, int rmax, int *err) {
    constexpr int BB = B * B, MT = (B + 15) / 16, NT = (B + 7) / 8;
    constexpr unsigned BLK = BB * 4u;  // a multiple of 16 (B even)
    constexpr size_t STRIDE = ((size_t)BLK + 127) / 128 * 128;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto slot = [&](int j) { return reinterpret_cast<float *>(smem_raw + STRIDE * j); };
    float *D = slot(0);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem_raw + STRIDE * (1 + 3 * rmax));
    const int R = rows[blockIdx.x];
    const int p0 = rp[R], pend = rp[R + 1];
    int r = 0;
    while (r < rmax && p0 + r < pend && ci[p0 + r] < R) ++r;
    const long long dpos = diag[R];
    if (threadIdx.x == 0) {
        mbar_init(bars);
        mbar_init(bars + 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_arrive(bars, 2u * r * BLK);
        for (int p = 0; p < r; ++p) {
            tma_load_1d(slot(1 + p), vals + (long long)(p0 + p) * BB, BLK, bars);
            tma_load_1d(slot(1 + rmax + p), dinv + (long long)ci[p0 + p] * BB, BLK, bars);
        }
        mbar_expect_arrive(bars + 1, (unsigned)(r + 1) * BLK);
        tma_load_1d(D, vals + dpos * BB, BLK, bars + 1);
        for (int p = 0; p < r; ++p)
            tma_load_1d(slot(1 + 2 * rmax + p), vals + (long long)upd[2 * upd_ptr[p0 + p] + 1] * BB, BLK, bars + 1);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const bool ok0 = mbar_wait(bars, 0);
    if (__syncthreads_or(!ok0)) {
        if (threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_TIMEOUT);
        mbar_wait(bars, 0);
        mbar_wait(bars + 1, 0);
        return;
    }
    // phase 1: L_p = B_p D_{i_p}^{-1}, strip by strip, in place over B_p
    for (int it = warp; it < r * MT; it += nwarps) {
        const int p = it / MT, r0 = (it - p * MT) * 16;
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
        strip_product<B>(acc, slot(1 + p), slot(1 + rmax + p), r0);
        strip_store<B>(acc, slot(1 + p), r0);
    }
    const bool ok1 = mbar_wait(bars + 1, 0);
    if (__syncthreads_or(!ok1)) {  // also: every L_p complete, every D^{-1} read
        if (threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_TIMEOUT);
        mbar_wait(bars + 1, 0);
        return;
    }
    for (int p = 0; p < r; ++p) copy_block_out(vals + (long long)(p0 + p) * BB, slot(1 + p), BB);
    // phase 2: partial Schur products P_p = L_p U_p into the D^{-1} slots
    for (int it = warp; it < r * MT; it += nwarps) {
        const int p = it % r, r0 = (it / r) * 16;
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
        strip_product<B>(acc, slot(1 + p), slot(1 + 2 * rmax + p), r0);
        strip_store<B>(acc, slot(1 + rmax + p), r0);
    }
    __syncthreads();
    // D - sum_p P_p (fixed order), four elements per thread and step
    float4 *out = reinterpret_cast<float4 *>(vals + dpos * BB);
    for (int e = threadIdx.x; e < BB / 4; e += blockDim.x) {
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int p = 0; p < r; ++p) {
            const float4 v = reinterpret_cast<const float4 *>(slot(1 + rmax + p))[e];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        const float4 d = reinterpret_cast<const float4 *>(D)[e];
        out[e] = make_float4(d.x - s.x, d.y - s.y, d.z - s.z, d.w - s.w);
    }
}

// D_R^{-1} for a list of rows whose diagonal block is final (rows without
// lower entries, or rows whose updates k_factor_level2 applied): the same
// Gauss-Jordan (gauss_jordan3) by a small CTA.  The inversion is a chain of
// b barrier-separated pivot steps, so its throughput grows with the number of
// inversions an SM holds at once; the product kernel's 256-thread CTAs hold
// six, 128-thread CTAs with only the two b x b work arrays twice as many.
template <class C>
__global__ void __launch_bounds__(256) k_factor_diag(const int *rows, int b, const int *diag, const C *vals, C *dinv,
                                                     int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bb = b * b;
    C *X = reinterpret_cast<C *>(smem_raw);  // b * (b + 1), padded columns
    C *Y = X + bb + b;
    C *fcol = Y + bb;
    const int R = rows[blockIdx.x];
    const C *D = vals + (long long)diag[R] * bb;
    for (int e = threadIdx.x; e < bb; e += blockDim.x) {
        const int col = e / b, row = e - col * b;
        X[col * (b + 1) + row] = D[e];
    }
    __syncthreads();
    const bool ok = gauss_jordan3(X, Y, b, fcol, b + 1);
    for (int e = threadIdx.x; e < bb; e += blockDim.x) dinv[(long long)R * bb + e] = Y[e];
    if (!ok && threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_SINGULAR);
}

template <class C>
__global__ void k_to_bf16(long long n, const C *src, __nv_bfloat16 *dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16_rn((float)src[e]);
}

// Explicitly fused multiply-add: the sweeps' dot products round the same way
// in every kernel that computes them (the compiler may otherwise fuse a*b+c
// in one kernel and not in another).
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// sum_c B[c][a] x[c] for a column-major block (thread's row a pre-applied to
// B): chunks of 8 columns with every load of a chunk issued before its FMAs
// (two accumulators), so each thread keeps 8 block loads in flight.
template <class C, class F>
__device__ __forceinline__ C block_col_dot(const F *B, const C *x, int b) {
    C s0 = C(0), s1 = C(0);
    for (int c0 = 0; c0 < b; c0 += 8) {
        C bv[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const bool ok = c0 + u < b;
            bv[u] = ok ? (C)ldfac(B + (long long)(c0 + u) * b) : C(0);
            xv[u] = ok ? x[c0 + u] : C(0);
        }
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            s0 = fma_rn(bv[u], xv[u], s0);
            s1 = fma_rn(bv[u + 1], xv[u + 1], s1);
        }
    }
    return s0 + s1;
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inverses with the rows in registers (block sizes known at
// compile time).  One CTA of round_up(B, 32) threads per block; thread r
// keeps row r of the block in registers and the elimination is fully
// unrolled.  Pivoting is partial and implicit: at step k the pivot is the
// row not yet used as a pivot with the largest |A[r][k]| (lowest row on
// ties), found by a warp max of (|value|, row) keys plus a max over the
// warps' keys; the pivot row is scaled and broadcast through shared memory
// and every other row eliminates column k with it (in-place form: column k
// takes the inverse's column).  The rows are never swapped; with piv[c] the
// pivot row of step c, the inverse is inv[k][piv[c]] = S[piv[k]][c], so the
// thread whose row was step k's pivot writes inverse row k.  Two barriers
// per step (pivot keys, pivot row), each over one or two warps.
template <class C>
__device__ __forceinline__ unsigned long long gjr_key(C v, int r);
template <>
__device__ __forceinline__ unsigned long long gjr_key<float>(float v, int r) {
    const unsigned bits = v == v ? __float_as_uint(fabsf(v)) : 0u;  // NaN: magnitude 0
    return ((unsigned long long)bits << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)r);
}
template <>
__device__ __forceinline__ unsigned long long gjr_key<double>(double v, int r) {
    // magnitude's top 57 bits (rows < 128): values equal to 2^-45 relative tie
    const unsigned long long bits = v == v ? (unsigned long long)__double_as_longlong(fabs(v)) : 0ull;
    return (bits & ~127ull) | (unsigned long long)(127 - r);
}
template <class C>
__device__ __forceinline__ void gjr_decode(unsigned long long key, int &row, C &mag);
template <>
__device__ __forceinline__ void gjr_decode<float>(unsigned long long key, int &row, float &mag) {
    row = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
    mag = __uint_as_float((unsigned)(key >> 32));
}
template <>
__device__ __forceinline__ void gjr_decode<double>(unsigned long long key, int &row, double &mag) {
    row = 127 - (int)(key & 127ull);
    mag = __longlong_as_double((long long)(key & ~127ull));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
        v = o > v ? o : v;
    }
    return v;
}

// The warp's pivot key at a step: binary32 values take a 32-bit max of the
// magnitude bits over the unused rows (one redux.sync) and a ballot for the
// lowest such row; binary64 keys go through the 64-bit shuffle max.  Both
// give the key gjr_key would: largest magnitude, lowest row on ties, 0 when
// every row of the warp is used.
template <class C>
__device__ __forceinline__ unsigned long long warp_pivot_key(C v, bool used, int r);
template <>
__device__ __forceinline__ unsigned long long warp_pivot_key<float>(float v, bool used, int r) {
    const unsigned bits = used ? 0u : (v == v ? __float_as_uint(fabsf(v)) : 0u);
    const unsigned mx = __reduce_max_sync(0xffffffffu, bits);
    const unsigned bal = __ballot_sync(0xffffffffu, !used && bits == mx);
    if (!bal) return 0ull;
    const int row = (r & ~31) + __ffs(bal) - 1;
    return ((unsigned long long)mx << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)row);
}
template <>
__device__ __forceinline__ unsigned long long warp_pivot_key<double>(double v, bool used, int r) {
    return warp_max_u64(used ? 0ull : gjr_key<double>(v, r));
}

// 16-byte shared-memory moves of the pivot row (4 floats or 2 doubles).
template <class C>
struct Vec16;
template <>
struct Vec16<float> {
    static constexpr int W = 4;
    static __device__ __forceinline__ void ld(float (&d)[4], const float *p) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        d[0] = v.x, d[1] = v.y, d[2] = v.z, d[3] = v.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&d)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(d[0], d[1], d[2], d[3]);
    }
};
template <>
struct Vec16<double> {
    static constexpr int W = 2;
    static __device__ __forceinline__ void ld(double (&d)[2], const double *p) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        d[0] = v.x, d[1] = v.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&d)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(d[0], d[1]);
    }
};

template <class C, int B>
__global__ void __launch_bounds__((B + 31) / 32 * 32) k_factor_diag_rows(const int *rows, const int *diag,
                                                                          const C *vals, C *dinv, int *err) {
    constexpr int NW = (B + 31) / 32;
    constexpr int VW = Vec16<C>::W;
    constexpr int BP = (B + VW - 1) / VW * VW;  // pivot row padded to whole 16-byte moves
    __shared__ __align__(16) C s_prow[2][BP];
    __shared__ unsigned long long s_key[2][NW];
    __shared__ int s_piv[B];
    const int r = threadIdx.x, lane = r & 31, w = r >> 5;
    const bool act = r < B;
    const int R = rows[blockIdx.x];
    const C *D = vals + (long long)diag[R] * (B * B);
    C A[B];
#pragma unroll
    for (int c = 0; c < B; ++c) A[c] = act ? D[c * B + r] : C(0);
    bool used = !act;
    int mystep = 0;
    bool bad = false;
    {
        const unsigned long long key = warp_pivot_key<C>(A[0], used, r);
        if (lane == 0) s_key[0][w] = key;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < B; ++k) {
        const int buf = k & 1;
        unsigned long long kmax = 0ull;
#pragma unroll
        for (int q = 0; q < NW; ++q) kmax = s_key[buf][q] > kmax ? s_key[buf][q] : kmax;
        int p;
        C mag;
        gjr_decode<C>(kmax, p, mag);
        const bool zero = !(mag > C(0));
        bad |= zero;
        if (r == p) {
            const C pinv = C(1) / (zero ? C(1) : A[k]);
#pragma unroll
            for (int c0 = 0; c0 < BP; c0 += VW) {
                C pr[VW];
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    const int c = c0 + u;
                    if (c < B) {
                        const C v = c == k ? pinv : A[c] * pinv;
                        pr[u] = v;
                        A[c] = v;
                    } else {
                        pr[u] = C(0);
                    }
                }
                Vec16<C>::st(&s_prow[buf][c0], pr);
            }
            used = true;
            mystep = k;
            s_piv[k] = r;
        }
        __syncthreads();
        if (act && r != p) {
            const C f = A[k];
#pragma unroll
            for (int c0 = 0; c0 < BP; c0 += VW) {
                C pr[VW];
                Vec16<C>::ld(pr, &s_prow[buf][c0]);
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    const int c = c0 + u;
                    if (c < B && c != k) A[c] = fma_rn(-f, pr[u], A[c]);
                }
            }
            A[k] = -f * s_prow[buf][k];
        }
        if (k + 1 < B) {
            const unsigned long long key = warp_pivot_key<C>(A[k + 1], used, r);
            if (lane == 0) s_key[buf ^ 1][w] = key;
        }
        __syncthreads();
    }
    if (act) {
        C *out = dinv + (long long)R * (B * B);
#pragma unroll
        for (int c = 0; c < B; ++c) out[s_piv[c] * B + mystep] = A[c];
    }
    if (bad && r == 0) atomicOr(err, IRK_DEV_ERR_SINGULAR);
}

// ---------------------------------------------------------------------------
// Sweeps.  A group of b threads owns one block row; thread a owns row a.
//   forward (level of the lower DAG):  y_R = v_R - sum_{p lower} L_p y_col
//   backward (level of the upper DAG): z_R = D_R^{-1} (y_R - sum_{p upper} U_p z_col)
// y and z share one compute-precision buffer (a row's y is replaced by its z).
template <class AR, class C, class F>
__global__ void __launch_bounds__(256) k_sweep_fwd(const int *rows, int nrows, int b, const int *rp,
                                                   const int *ci, const int *voff, const F *vals,
                                                   const vec8 *v, C *y) {
    const int groups = blockDim.x / b;
    const int g = threadIdx.x / b, a = threadIdx.x - g * b;
    const int idx = blockIdx.x * groups + g;
    if (g >= groups || idx >= nrows) return;
    const int R = rows[idx];
    const long long bb = (long long)b * b;
    C acc = CT<C>::template from_vec<AR>(AR::ld(v + voff[R] + a));
    for (int p = rp[R]; p < rp[R + 1]; ++p) {
        const int col = ci[p];
        if (col >= R) break;
        acc -= block_col_dot<C>(vals + (long long)p * bb + a, y + voff[col], b);
    }
    y[voff[R] + a] = acc;
}

template <class AR, class C, class F>
__global__ void __launch_bounds__(256) k_sweep_bwd(const int *rows, int nrows, int b, const int *rp,
                                                   const int *ci, const int *voff, const F *vals,
                                                   const F *dinv, C *y, vec8 *z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *t = reinterpret_cast<C *>(smem_raw);
    const int groups = blockDim.x / b;
    const int g = threadIdx.x / b, a = threadIdx.x - g * b;
    const int idx = blockIdx.x * groups + g;
    const bool active = (g < groups) && (idx < nrows);
    const long long bb = (long long)b * b;
    int R = 0;
    if (active) {
        R = rows[idx];
        C acc = y[voff[R] + a];
        for (int p = rp[R + 1] - 1; p >= rp[R]; --p) {
            const int col = ci[p];
            if (col <= R) break;
            acc -= block_col_dot<C>(vals + (long long)p * bb + a, y + voff[col], b);
        }
        t[g * b + a] = acc;
    }
    __syncthreads();
    if (!active) return;
    C acc = block_col_dot<C>(dinv + (long long)R * bb + a, t + g * b, b);
    y[voff[R] + a] = acc;
    AR::st(z + voff[R] + a, CT<C>::template to_vec<AR>(acc));
}

// Backward sweep of the uncoupled preconditioner with the upper blocks read
// once for all stages.  Its s stage systems share the pattern, and where no
// factor update targets an upper block (no element with two mutually
// adjacent neighbours, checked at set-up) every stage's upper block is the
// same -dt J_ij; the item is an element row of stage 0, the block is loaded
// once and applied to the s stage vectors.  Per stage the sums run in
// block_col_dot's order (8-column chunks, two accumulators), so the result
// equals k_sweep_bwd's bit for bit.
template <class C, class F, int S>
__device__ __forceinline__ void block_col_dot_multi(const F *B, const C *const (&x)[S], int b, C (&out)[S]) {
    C s0[S], s1[S];
#pragma unroll
    for (int k = 0; k < S; ++k) s0[k] = s1[k] = C(0);
    for (int c0 = 0; c0 < b; c0 += 8) {
        C bv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) bv[u] = c0 + u < b ? (C)ldfac(B + (long long)(c0 + u) * b) : C(0);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            C xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) xv[u] = c0 + u < b ? x[k][c0 + u] : C(0);
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                s0[k] = fma_rn(bv[u], xv[u], s0[k]);
                s1[k] = fma_rn(bv[u + 1], xv[u + 1], s1[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < S; ++k) out[k] = s0[k] + s1[k];
}

template <class AR, class C, class F, int S>
__global__ void __launch_bounds__(256) k_sweep_bwd_shared(const int *rows0, int nrows, int b, int T,
                                                          const int *rp, const int *ci, const int *voff,
                                                          const F *vals, const F *dinv, C *y, vec8 *z) {
    constexpr int s = S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *t = reinterpret_cast<C *>(smem_raw);  // groups * s * b
    const int groups = blockDim.x / b;
    const int g = threadIdx.x / b, a = threadIdx.x - g * b;
    const int idx = blockIdx.x * groups + g;
    const bool active = (g < groups) && (idx < nrows);
    const long long bb = (long long)b * b;
    int R0 = 0;
    if (active) {
        R0 = rows0[idx];
        C acc[S];
#pragma unroll
        for (int k = 0; k < S; ++k) acc[k] = y[voff[k * T + R0] + a];
        for (int p = rp[R0 + 1] - 1; p >= rp[R0]; --p) {
            const int col = ci[p];
            if (col <= R0) break;
            const C *x[S];
#pragma unroll
            for (int k = 0; k < S; ++k) x[k] = y + voff[k * T + col];
            C d[S];
            block_col_dot_multi<C, F, S>(vals + (long long)p * bb + a, x, b, d);
#pragma unroll
            for (int k = 0; k < S; ++k) acc[k] -= d[k];
        }
#pragma unroll
        for (int k = 0; k < S; ++k) t[(g * s + k) * b + a] = acc[k];
    }
    __syncthreads();
    if (!active) return;
    for (int k = 0; k < s; ++k) {
        const int R = k * T + R0;
        const C v = block_col_dot<C>(dinv + (long long)R * bb + a, t + (g * s + k) * b, b);
        y[voff[R] + a] = v;
        AR::st(z + voff[R] + a, CT<C>::template to_vec<AR>(v));
    }
}

// ---------------------------------------------------------------------------
// Two-colour application (Sec. 4.2.1 sweeps on a bipartite block pattern):
// when the lower DAG has two levels, the rows of its second level have no
// upper entries and those of the first no lower entries, the two sweeps
// reduce to
//   K1, second-colour rows:  y_R = v_R - sum_p L_p v_col,  z_R = D_R^{-1} y_R
//   K2, first-colour rows:   z_R = D_R^{-1} (v_R - sum_p U_p z_col)
// since y = v on the first colour and z_R needs only y_R on the second.  Two
// launches instead of four, and neither y_A nor y_B goes through memory.  The
// block size is a compile-time constant: each block's B column loads are
// issued at once, and every dot product keeps block_col_dot's arithmetic
// (even columns into one accumulator, odd into the other, in column order,
// explicit fma), so the application is bitwise that of the level sweeps.
// RW consecutive rows of one block column (factor storage F, RW = 4 or 2;
// the caller keeps the address aligned to RW elements).
template <class F, int RW>
__device__ __forceinline__ void ld_rows(float (&o)[RW], const F *p);
template <>
__device__ __forceinline__ void ld_rows<float, 4>(float (&o)[4], const float *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
template <>
__device__ __forceinline__ void ld_rows<float, 2>(float (&o)[2], const float *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    o[0] = v.x, o[1] = v.y;
}
template <>
__device__ __forceinline__ void ld_rows<__nv_bfloat16, 4>(float (&o)[4], const __nv_bfloat16 *p) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    o[0] = __uint_as_float(v.x << 16), o[1] = __uint_as_float(v.x & 0xffff0000u);
    o[2] = __uint_as_float(v.y << 16), o[3] = __uint_as_float(v.y & 0xffff0000u);
}
template <>
__device__ __forceinline__ void ld_rows<__nv_bfloat16, 2>(float (&o)[2], const __nv_bfloat16 *p) {
    const unsigned v = __ldg(reinterpret_cast<const unsigned *>(p));
    o[0] = __uint_as_float(v << 16), o[1] = __uint_as_float(v & 0xffff0000u);
}

// rows a0 .. a0 + RW - 1 of sum_c B[a][c] x[c] (x from xf(c), c even: the
// pair c, c + 1 at once), with block_col_dot's arithmetic per row
template <class F, int B, int RW, class XF>
__device__ __forceinline__ void block_rows_dot(float (&out)[RW], const F *Bp, XF xf) {
    float s0[RW], s1[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) s0[r] = s1[r] = 0.f;
#pragma unroll
    for (int c = 0; c < B; c += 2) {
        float b0[RW], b1[RW], x0, x1;
        ld_rows<F, RW>(b0, Bp + c * B);
        ld_rows<F, RW>(b1, Bp + (c + 1) * B);
        xf(c, x0, x1);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            s0[r] = fma_rn(b0[r], x0, s0[r]);
            s1[r] = fma_rn(b1[r], x1, s1[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) out[r] = s0[r] + s1[r];
}

// K1: a group of B / RW threads per second-colour row, RW rows per thread.
template <class AR, class F, int B, int RW>
__global__ void __launch_bounds__(256) k_sweep_fd(const int *rows, int nrows, const int *rp, const int *ci,
                                                  const int *voff, const F *vals, const F *dinv, const vec8 *v,
                                                  float *y, vec8 *z) {
    constexpr int GT = B / RW, G = 256 / GT;
    constexpr long long BB = (long long)B * B;
    __shared__ __align__(16) float t[G * B];
    const int g = threadIdx.x / GT, a0 = (threadIdx.x - g * GT) * RW;
    const int idx = blockIdx.x * G + g;
    const bool active = (g < G) && (idx < nrows);
    int R = 0;
    if (active) {
        R = rows[idx];
        float acc[RW];
#pragma unroll
        for (int r = 0; r < RW; ++r) acc[r] = CT<float>::template from_vec<AR>(AR::ld(v + voff[R] + a0 + r));
        for (int p = rp[R]; p < rp[R + 1]; ++p) {
            const int col = ci[p];
            if (col >= R) break;
            const vec8 *xv = v + voff[col];  // y_col = v_col: a row without lower entries
            float d[RW];
            block_rows_dot<F, B, RW>(d, vals + p * BB + a0, [&](int c, float &x0, float &x1) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(xv + c));
                x0 = CT<float>::template from_vec<AR>(df_make(f.x, f.y));
                x1 = CT<float>::template from_vec<AR>(df_make(f.z, f.w));
            });
#pragma unroll
            for (int r = 0; r < RW; ++r) acc[r] -= d[r];
        }
#pragma unroll
        for (int r = 0; r < RW; ++r) t[g * B + a0 + r] = acc[r];
    }
    __syncthreads();
    if (!active) return;
    const float *tg = t + g * B;
    float zv[RW];
    block_rows_dot<F, B, RW>(zv, dinv + R * BB + a0, [&](int c, float &x0, float &x1) {
        x0 = tg[c];
        x1 = tg[c + 1];
    });
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        y[voff[R] + a0 + r] = zv[r];
        AR::st(z + voff[R] + a0 + r, CT<float>::template to_vec<AR>(zv[r]));
    }
}

// Forward level sweep with the block size at compile time (levels after the
// first in a multicolour order): y_R = v_R - sum_p L_p y_col, a group of
// B / RW threads per row, RW rows per thread, block_col_dot's arithmetic per
// row (bitwise the generic k_sweep_fwd).
template <class AR, class F, int B, int RW>
__global__ void __launch_bounds__(256) k_sweep_fl(const int *rows, int nrows, const int *rp, const int *ci,
                                                  const int *voff, const F *vals, const vec8 *v, float *y) {
    constexpr int GT = B / RW, G = 256 / GT;
    constexpr long long BB = (long long)B * B;
    const int g = threadIdx.x / GT, a0 = (threadIdx.x - g * GT) * RW;
    const int idx = blockIdx.x * G + g;
    if (g >= G || idx >= nrows) return;
    const int R = rows[idx];
    float acc[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) acc[r] = CT<float>::template from_vec<AR>(AR::ld(v + voff[R] + a0 + r));
    for (int p = rp[R]; p < rp[R + 1]; ++p) {
        const int col = ci[p];
        if (col >= R) break;
        const float *yc = y + voff[col];  // rows of earlier levels (earlier launches)
        float d[RW];
        block_rows_dot<F, B, RW>(d, vals + p * BB + a0, [&](int c, float &x0, float &x1) {
            const float2 f = __ldg(reinterpret_cast<const float2 *>(yc + c));
            x0 = f.x;
            x1 = f.y;
        });
#pragma unroll
        for (int r = 0; r < RW; ++r) acc[r] -= d[r];
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) y[voff[R] + a0 + r] = acc[r];
}

template <class C, class F, int B, class XF>
__device__ __forceinline__ C block_col_dot_b(const F *Bp, XF x) {
    C bv[B];
#pragma unroll
    for (int c = 0; c < B; ++c) bv[c] = (C)ldfac(Bp + c * B);
    C s0 = C(0), s1 = C(0);
#pragma unroll
    for (int c = 0; c < B; c += 2) {
        s0 = fma_rn(bv[c], x(c), s0);
        if (c + 1 < B) s1 = fma_rn(bv[c + 1], x(c + 1), s1);
    }
    return s0 + s1;
}

// K2 with the upper blocks shared by the S stages (-dt J_ij for every stage):
// one group per first-colour element, each upper block read once.  FY: the
// row's starting value is its forward result y_R (a backward level of a
// multicolour order) instead of v_R (the first colour of two, where y = v).
template <class AR, class C, class F, int S, int B, bool FY = false>
__global__ void __launch_bounds__(256) k_sweep_bu(const int *rows0, int nrows, int T, const int *rp, const int *ci,
                                                  const int *voff, const F *vals, const F *dinv, const vec8 *v,
                                                  C *y, vec8 *z) {
    constexpr int G = 256 / B;
    constexpr long long BB = (long long)B * B;
    __shared__ C t[G * S * B];
    const int g = threadIdx.x / B, a = threadIdx.x - g * B;
    const int idx = blockIdx.x * G + g;
    const bool active = (g < G) && (idx < nrows);
    int R0 = 0;
    if (active) {
        R0 = rows0[idx];
        C acc[S];
#pragma unroll
        for (int k = 0; k < S; ++k)
            acc[k] = FY ? y[voff[k * T + R0] + a] : CT<C>::template from_vec<AR>(AR::ld(v + voff[k * T + R0] + a));
        for (int p = rp[R0 + 1] - 1; p >= rp[R0]; --p) {
            const int col = ci[p];
            if (col <= R0) break;
            C bv[B];
#pragma unroll
            for (int c = 0; c < B; ++c) bv[c] = (C)ldfac(vals + p * BB + a + c * B);
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const C *x = y + voff[k * T + col];
                C s0 = C(0), s1 = C(0);
#pragma unroll
                for (int c = 0; c < B; c += 2) {
                    s0 = fma_rn(bv[c], x[c], s0);
                    if (c + 1 < B) s1 = fma_rn(bv[c + 1], x[c + 1], s1);
                }
                acc[k] -= s0 + s1;
            }
        }
#pragma unroll
        for (int k = 0; k < S; ++k) t[(g * S + k) * B + a] = acc[k];
    }
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int R = k * T + R0;
        const C *tk = t + (g * S + k) * B;
        const C zv = block_col_dot_b<C, F, B>(dinv + R * BB + a, [&](int c) { return tk[c]; });
        y[voff[R] + a] = zv;
        AR::st(z + voff[R] + a, CT<C>::template to_vec<AR>(zv));
    }
}

// ---------------------------------------------------------------------------
// Persistent sweeps: one launch applies the whole preconditioner.  The work
// list is the forward rows in lower-level order followed by the backward rows
// in upper-level order; warp w takes items w, w + W, w + 2W, ... (W warps in
// the grid, all resident: cooperative launch).  An item waits until the rows
// it reads are published (per-row flags set to this application's epoch),
// computes its row and publishes it.  Every dependency sits earlier in the
// list, so the lowest unfinished item can always proceed.  Waits are bounded:
// after `spin` polls (irk_options.spin_limit), or as soon as another warp
// reported an error, the warp records IRK_DEV_ERR_TIMEOUT (the first case),
// waits for its own bulk copies still in flight (bounded by the fixed
// IRK_SPIN_LIMIT of a copy's completion) and leaves.
#define IRK_PB 4  // values per lane: b <= 128

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float ldcg_c(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_c(const double *p) { return __ldcg(p); }

// Shared-memory staging of factor blocks: cp.async.bulk (TMA bulk copy, the
// helpers of tma.cuh) completing on an mbarrier; plain loads when the block is
// not 16-byte aligned / sized.
// Stage one block (nbytes, element type F) into a slot: TMA when possible.
template <class F>
__device__ __forceinline__ void stage_block(F *slot, const F *src, unsigned nbytes, bool tma,
                                            unsigned long long *bar) {
    const int lane = threadIdx.x & 31;
    if (tma) {
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_arrive(bar, nbytes);
            tma_load_1d(slot, src, nbytes, bar);
        }
    } else {
        const int n = nbytes / sizeof(F);
#pragma unroll 8
        for (int e = lane; e < n; e += 32) slot[e] = src[e];
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
}

// Self-validating vector words: a compute-precision value is published as
// sizeof(C)/4 64-bit words {32 value bits, epoch}.  A reader polls the words
// themselves (relaxed, L1-bypassing 64-bit loads) until every word carries the
// current epoch: one round trip per dependency and no flags or fences, since
// each word is written and read atomically.
template <class C>
struct LL;
template <>
struct LL<float> {
    static constexpr int W = 1;
    static __device__ __forceinline__ void put(unsigned long long *p, float v, int ep) {
        unsigned long long w = ((unsigned long long)(unsigned)ep << 32) | (unsigned)__float_as_uint(v);
        asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
    }
    // returns true and the value when the word carries epoch ep
    static __device__ __forceinline__ bool get(const unsigned long long *p, int ep, float &v) {
        unsigned long long w;
        asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
        v = __uint_as_float((unsigned)(w & 0xffffffffull));
        return (int)(w >> 32) == ep;
    }
};
template <>
struct LL<double> {
    static constexpr int W = 2;
    static __device__ __forceinline__ void put(unsigned long long *p, double v, int ep) {
        unsigned long long bits = (unsigned long long)__double_as_longlong(v);
        unsigned long long e = (unsigned long long)(unsigned)ep << 32;
        asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(e | (bits >> 32)) : "memory");
        asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p + 1), "l"(e | (bits & 0xffffffffull)) : "memory");
    }
    static __device__ __forceinline__ bool get(const unsigned long long *p, int ep, double &v) {
        unsigned long long w0, w1;
        asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w0) : "l"(p) : "memory");
        asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w1) : "l"(p + 1) : "memory");
        v = __longlong_as_double((long long)((w0 << 32) | (w1 & 0xffffffffull)));
        return (int)(w0 >> 32) == ep && (int)(w1 >> 32) == ep;
    }
};

// Poll the b published values of one row (lane holds entries lane + 32u);
// warp-uniform, bounded, abortable.  Returns false on timeout / abort.
template <class C>
__device__ __forceinline__ bool ll_wait_row(const unsigned long long *row, int b, int ep, int *err, int spin,
                                            C (&out)[IRK_PB]) {
    const int lane = threadIdx.x & 31;
    for (int spins = 0;; ++spins) {
        bool ok = true;
#pragma unroll
        for (int u = 0; u < IRK_PB; ++u) {
            const int cc = lane + 32 * u;
            if (cc < b) ok &= LL<C>::get(row + (long long)cc * LL<C>::W, ep, out[u]);
            else out[u] = C(0);
        }
        if (__all_sync(0xffffffffu, ok)) return true;
        if (spins > 64) __nanosleep(32);
        if ((spins & 255) == 255) {
            const int e = ld_acquire(err);
            if (__any_sync(0xffffffffu, e != 0)) return false;
        }
        if (spins >= spin) {
            if (lane == 0) atomicOr(err, IRK_DEV_ERR_TIMEOUT);
            return false;
        }
    }
}

// Persistent sweep with staged blocks.  Each warp owns NS slots of one block
// and NS mbarriers.  For an item it issues the copies of its first NS blocks
// at once (before waiting for any dependency), then consumes block k after
// the dependency of block k is published and the copy of block k landed,
// refilling the slot with block k + NS.  y (forward results) and zc
// (backward results) are published as self-validating words.
// Group mode (lane_of_row != nullptr): rows belong to independent requests
// ("lanes"); voff is lane-local and each lane's vectors and published words
// start at its own offsets (lane_vin < 0: the lane sits this launch out).
struct SweepLanes {
    const int *lane_of_row;
    const long long *vin, *zout, *yll, *zll;
};

template <class AR, class C, class F>
__global__ void __launch_bounds__(128) k_sweep_staged(int nb, int b, int NS, const int *lo_rows, const int *up_rows,
                                                      const int *rp, const int *ci, const int *voff, const F *vals,
                                                      const F *dinv, const vec8 *v, unsigned long long *yll,
                                                      unsigned long long *zll, vec8 *z, int ep, int *err,
                                                      SweepLanes lanes, int spin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int bb = b * b;
    const unsigned blk_bytes = (unsigned)(bb * sizeof(F));
    const size_t slot_stride = ((size_t)blk_bytes + 127) / 128 * 128;
    const size_t warp_bytes = slot_stride * NS + 128;
    unsigned char *base = smem_raw + wib * warp_bytes;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(base + slot_stride * NS);
    const bool tma = (blk_bytes % 16 == 0);
    if (lane == 0)
        for (int s = 0; s < NS; ++s) mbar_init(bars + s);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    unsigned phase = 0;    // bit s: parity of the next completion of slot s
    unsigned pending = 0;  // bit s: a copy into slot s is in flight
    // error exit: wait (bounded) for this warp's copies still in flight
    auto drain = [&]() {
        for (int s = 0; s < NS; ++s)
            if ((pending >> s) & 1u) mbar_wait(bars + s, (phase >> s) & 1u);
    };
    const int W = (gridDim.x * blockDim.x) >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned FULL = 0xffffffffu;
    constexpr int LW = LL<C>::W;
    const vec8 *v0 = v;
    vec8 *z0 = z;
    unsigned long long *y0 = yll, *zz0 = zll;
    for (int q = gw; q < 2 * nb; q += W) {
        const bool fwd = q < nb;
        const int R = fwd ? lo_rows[q] : up_rows[q - nb];
        const int vo = voff[R];
        if (lanes.lane_of_row) {
            const int ln = lanes.lane_of_row[R];
            const long long vb = lanes.vin[ln];
            if (vb < 0) continue;  // warp-uniform: the whole item is skipped
            v = v0 + vb;
            z = z0 + lanes.zout[ln];
            yll = y0 + lanes.yll[ln];
            zll = zz0 + lanes.zll[ln];
        }
        int pbeg, pend, nblk;
        if (fwd) {
            pbeg = rp[R];
            pend = pbeg;
            while (pend < rp[R + 1] && ci[pend] < R) ++pend;
            nblk = pend - pbeg;
        } else {
            pend = rp[R + 1];
            pbeg = pend;
            while (pbeg > rp[R] && ci[pbeg - 1] > R) --pbeg;
            nblk = pend - pbeg + 1;
        }
        auto block_ptr = [&](int kk) -> const F * {
            if (fwd) return vals + (long long)(pbeg + kk) * bb;
            if (kk < pend - pbeg) return vals + (long long)(pend - 1 - kk) * bb;
            return dinv + (long long)R * bb;
        };
        for (int kk = 0; kk < nblk && kk < NS; ++kk) {
            stage_block<F>(reinterpret_cast<F *>(base + slot_stride * kk), block_ptr(kk), blk_bytes, tma, bars + kk);
            pending |= 1u << kk;
        }
        C acc[IRK_PB];
        if (fwd) {
#pragma unroll
            for (int u = 0; u < IRK_PB; ++u) {
                int a = lane + 32 * u;
                acc[u] = (a < b) ? CT<C>::template from_vec<AR>(AR::ld(v + vo + a)) : C(0);
            }
        } else if (!ll_wait_row<C>(yll + (long long)vo * LW, b, ep, err, spin, acc)) {
            drain();
            return;
        }
        const int ndep = fwd ? nblk : nblk - 1;
        for (int kk = 0; kk < nblk; ++kk) {
            const int s = kk % NS;
            const bool is_dinv = !fwd && kk == ndep;
            C dep[IRK_PB];
            if (!is_dinv) {
                const int col = fwd ? ci[pbeg + kk] : ci[pend - 1 - kk];
                if (!ll_wait_row<C>((fwd ? yll : zll) + (long long)voff[col] * LW, b, ep, err, spin, dep)) {
                    drain();
                    return;
                }
            } else {
                // z_R = D^{-1} t with t = y_R - sum U z (held in acc)
#pragma unroll
                for (int u = 0; u < IRK_PB; ++u) {
                    dep[u] = acc[u];
                    acc[u] = C(0);
                }
            }
            if (!mbar_wait(bars + s, (phase >> s) & 1u)) {
                if (lane == 0) atomicOr(err, IRK_DEV_ERR_TIMEOUT);
                drain();
                return;
            }
            phase ^= (1u << s);
            pending &= ~(1u << s);
            const F *blk = reinterpret_cast<const F *>(base + slot_stride * s);
            const C sign = is_dinv ? C(1) : C(-1);
            // chunks of 8 columns: the 8 shuffles and 8 x IRK_PB shared loads of a
            // chunk are issued before its FMAs; two accumulator sets (even / odd
            // columns) halve the dependent chain
            C acc2[IRK_PB];
#pragma unroll
            for (int u = 0; u < IRK_PB; ++u) acc2[u] = C(0);
            for (int c0 = 0; c0 < b; c0 += 8) {
                const int uc = c0 >> 5;
                const C src = (uc == 0) ? dep[0] : (uc == 1) ? dep[1] : (uc == 2) ? dep[2] : dep[3];
                C dv[8];
                F cv[8][IRK_PB];
#pragma unroll
                for (int l = 0; l < 8; ++l) dv[l] = sign * __shfl_sync(FULL, src, (c0 + l) & 31);
#pragma unroll
                for (int l = 0; l < 8; ++l)
#pragma unroll
                    for (int u = 0; u < IRK_PB; ++u) {
                        const int a = lane + 32 * u;
                        cv[l][u] = (c0 + l < b && a < b) ? blk[(c0 + l) * b + a] : F(0);
                    }
#pragma unroll
                for (int l = 0; l < 8; ++l)
#pragma unroll
                    for (int u = 0; u < IRK_PB; ++u) {
                        if (c0 + l >= b) continue;
                        if (l & 1)
                            acc2[u] += (C)cv[l][u] * dv[l];
                        else
                            acc[u] += (C)cv[l][u] * dv[l];
                    }
            }
#pragma unroll
            for (int u = 0; u < IRK_PB; ++u) acc[u] += acc2[u];
            __syncwarp();
            if (kk + NS < nblk) {
                stage_block<F>(reinterpret_cast<F *>(base + slot_stride * s), block_ptr(kk + NS), blk_bytes, tma,
                               bars + s);
                pending |= 1u << s;
            }
        }
        unsigned long long *dst = (fwd ? yll : zll) + (long long)vo * LW;
#pragma unroll
        for (int u = 0; u < IRK_PB; ++u) {
            int a = lane + 32 * u;
            if (a < b) {
                LL<C>::put(dst + (long long)a * LW, acc[u], ep);
                if (!fwd) AR::st(z + vo + a, CT<C>::template to_vec<AR>(acc[u]));
            }
        }
    }
}

int grid_cap(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)std::max(1LL, g);
}

// ---------------------------------------------------------------------------
// Host-side construction of the pattern, levels and update lists.
struct HostPattern {
    int nb = 0, b = 0;
    std::vector<int> rp, ci, diag, voff, rowof;
    std::vector<AsmEntry> asmv;
    std::vector<int> upd_ptr, upd;
    std::vector<int> lo_rows, lo_ptr, up_rows, up_ptr;
};

void levels_lower(const HostPattern &h, std::vector<int> &rows, std::vector<int> &ptr) {
    std::vector<int> lev(h.nb, 0);
    int maxl = 0;
    for (int R = 0; R < h.nb; ++R) {
        int l = 0;
        for (int p = h.rp[R]; p < h.rp[R + 1]; ++p)
            if (h.ci[p] < R) l = std::max(l, lev[h.ci[p]] + 1);
        lev[R] = l;
        maxl = std::max(maxl, l);
    }
    ptr.assign(maxl + 2, 0);
    for (int R = 0; R < h.nb; ++R) ptr[lev[R] + 1]++;
    for (int l = 0; l <= maxl; ++l) ptr[l + 1] += ptr[l];
    rows.assign(h.nb, 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int R = 0; R < h.nb; ++R) rows[fill[lev[R]]++] = R;
}

void levels_upper(const HostPattern &h, std::vector<int> &rows, std::vector<int> &ptr) {
    std::vector<int> lev(h.nb, 0);
    int maxl = 0;
    for (int R = h.nb - 1; R >= 0; --R) {
        int l = 0;
        for (int p = h.rp[R]; p < h.rp[R + 1]; ++p)
            if (h.ci[p] > R) l = std::max(l, lev[h.ci[p]] + 1);
        lev[R] = l;
        maxl = std::max(maxl, l);
    }
    ptr.assign(maxl + 2, 0);
    for (int R = 0; R < h.nb; ++R) ptr[lev[R] + 1]++;
    for (int l = 0; l <= maxl; ++l) ptr[l + 1] += ptr[l];
    rows.assign(h.nb, 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int R = h.nb - 1; R >= 0; --R) rows[fill[lev[R]]++] = R;
}

int find_in_row(const HostPattern &h, int row, int col) {
    const int *b = h.ci.data() + h.rp[row], *e = h.ci.data() + h.rp[row + 1];
    const int *f = std::lower_bound(b, e, col);
    return (f != e && *f == col) ? (int)(f - h.ci.data()) : -1;
}

void build_updates(HostPattern &h) {
    h.upd_ptr.assign(h.ci.size() + 1, 0);
    h.upd.clear();
    for (int R = 0; R < h.nb; ++R)
        for (int p = h.rp[R]; p < h.rp[R + 1]; ++p) {
            h.upd_ptr[p] = (int)(h.upd.size() / 2);
            const int i = h.ci[p];
            if (i < R)
                for (int q = p + 1; q < h.rp[R + 1]; ++q) {
                    int pos = find_in_row(h, i, h.ci[q]);
                    if (pos >= 0) {
                        h.upd.push_back(q);
                        h.upd.push_back(pos);
                    }
                }
        }
    h.upd_ptr[h.ci.size()] = (int)(h.upd.size() / 2);
}

template <class Tv>
int upload(Tv **dst, const std::vector<Tv> &src) {
    size_t bytes = std::max<size_t>(1, src.size()) * sizeof(Tv);
    if (cudaMalloc((void **)dst, bytes) != cudaSuccess) return IRK_ERR_NOMEM;
    if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(Tv), cudaMemcpyHostToDevice) != cudaSuccess)
        return IRK_ERR_CUDA;
    return IRK_OK;
}

size_t csize(int fprec) { return fprec == IRK_FACTOR_FP64 ? 8 : 4; }

}  // namespace

// exported to the other translation units (operator product)
int irk_allow_max_smem(const void *func) { return allow_max_smem(func); }

// Build the block pattern of the matrix to factor for the context's
// preconditioner kind (see the file comment), its level schedules and the
// update lists of the IKJ factorisation, and allocate the factor storage.
int pc_build_pattern(irk_ctx *c) {
    PcSystem &P = c->pc;
    P.kind = c->opt.precond;
    if (P.kind == IRK_PC_NONE) return IRK_OK;
    const int s = c->s, T = c->T, m = c->m;
    const bool transformed = c->opt.formulation == IRK_TRANSFORMED;
    const std::vector<int> &rp = c->h_rp, &ci = c->h_ci;
    HostPattern h;
    // elimination order (perm[q] = element eliminated q-th) and partitions
    std::vector<int> perm(T), inv(T), part;
    for (int q = 0; q < T; ++q) perm[q] = q;
    if (c->opt.ordering == IRK_ORDER_MULTICOLOR) {
        std::vector<int> colour(T, -1);
        std::vector<char> used;
        for (int i = 0; i < T; ++i) {  // first-fit colouring in input order
            used.assign(rp[i + 1] - rp[i] + 2, 0);
            for (int p = rp[i]; p < rp[i + 1]; ++p) {
                int j = ci[p];
                if (j != i && colour[j] >= 0 && colour[j] < (int)used.size()) used[colour[j]] = 1;
            }
            int cc = 0;
            while (used[cc]) ++cc;
            colour[i] = cc;
        }
        std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return colour[x] < colour[y]; });
    }
    for (int q = 0; q < T; ++q) inv[perm[q]] = q;
    if (!c->h_part.empty()) {
        part = c->h_part;
    } else if (c->opt.partitions > 1) {
        part.resize(T);
        for (int i = 0; i < T; ++i) part[i] = (int)((long long)i * c->opt.partitions / T);
    }
    const bool reordered = c->opt.ordering != IRK_ORDER_NATURAL || !part.empty();
    if (P.kind == IRK_PC_UNCOUPLED || P.kind == IRK_PC_COUPLED) {
        if (P.kind == IRK_PC_UNCOUPLED && !transformed) return IRK_ERR_INVALID;
        h.nb = s * T;
        h.b = m;
        h.rp.push_back(0);
        std::vector<std::pair<int, int>> nb_new;  // (new index, J position) of kept neighbours
        for (int k = 0; k < s; ++k)
            for (int q = 0; q < T; ++q) {
                const int e = perm[q];
                nb_new.clear();
                for (int p = rp[e]; p < rp[e + 1]; ++p) {
                    const int j = ci[p];
                    if (!part.empty() && part[j] != part[e]) continue;
                    nb_new.push_back(std::make_pair(inv[j], p));
                }
                std::sort(nb_new.begin(), nb_new.end());
                auto mass = [&](int l) {  // block (k,e)-(l,e), mass coupling
                    h.ci.push_back(l * T + q);
                    h.asmv.push_back(AsmEntry{-1, e, k * s + l, 0});
                };
                if (P.kind == IRK_PC_COUPLED && transformed)
                    for (int l = 0; l < k; ++l) mass(l);
                int lfirst = (P.kind == IRK_PC_COUPLED && !transformed) ? 0 : k;
                int llast = (P.kind == IRK_PC_COUPLED && !transformed) ? s - 1 : k;
                // stage k's rows use J_k when the stages have their own Jacobians
                const int jk = c->nJ > 1 ? k * c->nnzb : 0;
                for (int l = lfirst; l <= llast; ++l)
                    for (const auto &nq : nb_new) {
                        const int p = nq.second, j = ci[p];
                        h.ci.push_back(l * T + nq.first);
                        if (transformed)  // d_k M - dt J_k  (uncoupled: d_k = A^{-1}_kk + alpha_k)
                            h.asmv.push_back(AsmEntry{jk + p, j == e ? e : -1, k * s + k, 0});
                        else  // [k==l][e==j] M - dt a_kl J_k
                            h.asmv.push_back(AsmEntry{jk + p, (j == e && l == k) ? e : -1, 0, k * s + l});
                    }
                if (P.kind == IRK_PC_COUPLED && transformed)
                    for (int l = k + 1; l < s; ++l) mass(l);
                h.rp.push_back((int)h.ci.size());
            }
        for (int R = 0; R < h.nb; ++R) {
            int k = R / T, q = R - k * T;
            h.voff.push_back((perm[q] * s + k) * m);
        }
    } else if (P.kind == IRK_PC_ELEMENT) {
        if (reordered) return IRK_ERR_INVALID;
        h.nb = T;
        h.b = s * m;
        h.rp = rp;
        h.ci = ci;
        for (int i = 0; i < T; ++i) {
            h.voff.push_back(i * s * m);
            for (int p = rp[i]; p < rp[i + 1]; ++p) h.rowof.push_back(i);
        }
        P.element_major = 1;
    } else {
        return IRK_ERR_INVALID;
    }
    const size_t cs = csize(c->fprec);
    if ((size_t)h.b * h.b * cs * 2 + h.b * cs + 64 > 227 * 1024) return IRK_ERR_INVALID;
    for (int R = 0; R < h.nb; ++R) {
        int d = find_in_row(h, R, R);
        if (d < 0) return IRK_ERR_INVALID;
        h.diag.push_back(d);
    }
    build_updates(h);
    P.max_item_blocks = 1;
    for (int R = 0; R < h.nb; ++R) {
        int lower = 0, upper = 0;
        for (int p = h.rp[R]; p < h.rp[R + 1]; ++p) {
            if (h.ci[p] < R) ++lower;
            if (h.ci[p] > R) ++upper;
        }
        P.max_item_blocks = std::max(P.max_item_blocks, std::max(lower, upper + 1));
    }
    levels_lower(h, h.lo_rows, h.lo_ptr);
    levels_upper(h, h.up_rows, h.up_ptr);
    // uncoupled kind: do all stages keep -dt J_ij as upper blocks (no factor
    // update targets an upper block)?  Then the backward sweep may read one
    // copy for all stages, and its items are the stage-0 rows of each level.
    std::vector<int> up0_rows, up0_ptr;
    P.shared_upper = 0;
    if (P.kind == IRK_PC_UNCOUPLED && s > 1) {
        bool upper_touched = false;
        for (int R = 0; R < h.nb && !upper_touched; ++R)
            for (int p = h.rp[R]; p < h.rp[R + 1] && !upper_touched; ++p)
                for (int u = h.upd_ptr[p]; u < h.upd_ptr[p + 1]; ++u)
                    if (h.ci[h.upd[2 * u]] > R) upper_touched = true;
        if (!upper_touched) {
            P.shared_upper = 1;
            up0_ptr.push_back(0);
            for (size_t l = 0; l + 1 < h.up_ptr.size(); ++l) {
                for (int q = h.up_ptr[l]; q < h.up_ptr[l + 1]; ++q)
                    if (h.up_rows[q] < T) up0_rows.push_back(h.up_rows[q]);
                up0_ptr.push_back((int)up0_rows.size());
            }
        }
    }
    P.two_colour = 0;
    if (h.lo_ptr.size() == 3 && h.up_ptr.size() == 3 &&
        (h.lo_ptr[2] - h.lo_ptr[1]) + (h.up_ptr[2] - h.up_ptr[1]) == h.nb) {
        bool ok = true;
        for (int q = h.lo_ptr[1]; q < h.lo_ptr[2] && ok; ++q) {
            const int R = h.lo_rows[q];
            if (h.ci[h.rp[R + 1] - 1] > R) ok = false;  // an upper entry
        }
        for (int q = h.up_ptr[1]; q < h.up_ptr[2] && ok; ++q) {
            const int R = h.up_rows[q];
            if (h.ci[h.rp[R]] < R) ok = false;  // a lower entry
        }
        P.two_colour = ok ? 1 : 0;
    }
    // does every update of a lower entry land on its row's diagonal block (a
    // single update each: no two lower neighbours of a row adjacent)?
    P.fused_r = 0;
    {
        bool diag_only = true;
        int rmax = 0;
        for (int R = 0; R < h.nb && diag_only; ++R) {
            int r = 0;
            for (int p = h.rp[R]; p < h.rp[R + 1] && h.ci[p] < R; ++p) {
                ++r;
                if (h.upd_ptr[p + 1] - h.upd_ptr[p] != 1 || h.upd[2 * h.upd_ptr[p]] != h.diag[R]) diag_only = false;
            }
            rmax = std::max(rmax, r);
        }
        if (diag_only) P.fused_r = rmax;
    }
    P.nb = h.nb;
    P.b = h.b;
    P.nnz = (long long)h.ci.size();
    P.lo_ptr = h.lo_ptr;
    P.up_ptr = h.up_ptr;
    P.up0_ptr = up0_ptr;
    int rc;
    if ((rc = upload(&P.d_rp, h.rp)) || (rc = upload(&P.d_ci, h.ci)) || (rc = upload(&P.d_diag, h.diag)) ||
        (rc = upload(&P.d_voff, h.voff)) || (rc = upload(&P.d_upd_ptr, h.upd_ptr)) ||
        (rc = upload(&P.d_upd, h.upd)) || (rc = upload(&P.d_lo_rows, h.lo_rows)) ||
        (rc = upload(&P.d_up_rows, h.up_rows)) || (P.shared_upper && (rc = upload(&P.d_up0_rows, up0_rows))))
        return rc;
    if (P.element_major) {
        if ((rc = upload(&P.d_rowof, h.rowof))) return rc;
    } else {
        if ((rc = upload(&P.d_asm, h.asmv))) return rc;
    }
    const long long bb = (long long)P.b * P.b;
    if (cudaMalloc(&P.d_vals, P.nnz * bb * cs) != cudaSuccess) return IRK_ERR_NOMEM;
    if (cudaMalloc(&P.d_dinv, (long long)P.nb * bb * cs) != cudaSuccess) return IRK_ERR_NOMEM;
    if (c->fprec == IRK_FACTOR_BF16) {
        if (cudaMalloc(&P.d_vals16, P.nnz * bb * 2) != cudaSuccess) return IRK_ERR_NOMEM;
        if (cudaMalloc(&P.d_dinv16, (long long)P.nb * bb * 2) != cudaSuccess) return IRK_ERR_NOMEM;
    }
    if (cudaMalloc(&P.d_y, (size_t)c->N * cs) != cudaSuccess) return IRK_ERR_NOMEM;
    // AUTO: one persistent launch when the levels are narrow (the sweep is
    // bound by the chain of levels); per-level launches when each level holds
    // enough rows to fill the GPU (few levels, e.g. a multicolour order)
    const int nlev_lo = (int)h.lo_ptr.size() - 1;
    const bool wide = nlev_lo > 0 && (long long)h.nb >= 4096LL * nlev_lo;
    P.persistent = (P.b <= 128) && c->opt.sweep != IRK_SWEEP_LEVELS && !wide;
    if (P.persistent) {
        // self-validating words: cs/4 words of 8 bytes per value, epoch 0 = never written
        const size_t words = (size_t)c->N * (cs / 4);
        if (cudaMalloc(&P.d_yll, words * 8) != cudaSuccess) return IRK_ERR_NOMEM;
        if (cudaMalloc(&P.d_zll, words * 8) != cudaSuccess) return IRK_ERR_NOMEM;
        cudaMemset(P.d_yll, 0, words * 8);
        cudaMemset(P.d_zll, 0, words * 8);
        P.epoch = 0;
    }
    return IRK_OK;
}

void pc_free(PcSystem &P) {
    cudaFree(P.d_rp);
    cudaFree(P.d_ci);
    cudaFree(P.d_diag);
    cudaFree(P.d_voff);
    cudaFree(P.d_asm);
    cudaFree(P.d_rowof);
    cudaFree(P.d_upd_ptr);
    cudaFree(P.d_upd);
    cudaFree(P.d_lo_rows);
    cudaFree(P.d_up_rows);
    cudaFree(P.d_up0_rows);
    cudaFree(P.d_vals);
    cudaFree(P.d_dinv);
    cudaFree(P.d_vals16);
    cudaFree(P.d_dinv16);
    cudaFree(P.d_y);
    cudaFree(P.d_yll);
    cudaFree(P.d_zll);
    P = PcSystem();
}

// The register-row inversion for the block sizes it is compiled for
// (on = irk_kernel_options.factor_gj_rows; 0 selects the shared-memory
// kernel); false otherwise.
template <class C>
static bool launch_diag_rows(cudaStream_t st, int n, int b, const int *rows, const int *diag, const C *vals, C *dinv,
                             int *err, bool on) {
    if (!on) return false;
    switch (b) {
        case 12: k_factor_diag_rows<C, 12><<<n, 32, 0, st>>>(rows, diag, vals, dinv, err); return true;
        case 20: k_factor_diag_rows<C, 20><<<n, 32, 0, st>>>(rows, diag, vals, dinv, err); return true;
        case 24: k_factor_diag_rows<C, 24><<<n, 32, 0, st>>>(rows, diag, vals, dinv, err); return true;
        case 40: k_factor_diag_rows<C, 40><<<n, 64, 0, st>>>(rows, diag, vals, dinv, err); return true;
        case 50: k_factor_diag_rows<C, 50><<<n, 64, 0, st>>>(rows, diag, vals, dinv, err); return true;
        default: return false;
    }
}

// Warps per CTA of k_factor_fused for this pattern (8 or 16), or 0 when it
// does not apply: updates not diagonal-only, odd block size (bulk copies want
// 16-byte multiples), more phase-1 tiles than the warps' registers hold, or
// the row's blocks do not fit in shared memory; irk_kernel_options
// factor_fused = 0 turns it off.
static size_t fused_smem(const PcSystem &P) {
    const size_t stride = ((size_t)P.b * P.b * 4 + 127) / 128 * 128;
    return stride * (1 + 3 * (size_t)P.fused_r) + 128;
}
static int fused_warps(const PcSystem &P, int mode) {
    if (P.fused_r <= 0 || (P.b & 1) || mode == 0) return 0;
    if (fused_smem(P) > 227 * 1024) return 0;
    const int items = P.fused_r * ((P.b + 15) / 16) * ((P.b + 7) / 8);
    if (items <= 8 * IRK_FUSED_TPW) return 8;
    if (items <= 16 * IRK_FUSED_TPW) return 16;
    return 0;
}
// Compile-time block sizes of k_factor_fused_b (the sizes of the workloads);
// other even sizes take the generic k_factor_fused.
template <int B>
static bool launch_fused_b(int n, size_t smem, cudaStream_t st, const int *rows, const PcSystem &P, float *vals,
                           const float *dinv, int *err) {
    if (P.b != B) return false;
    const int mt = (B + 15) / 16;
    const int nw = std::max(1, std::min(16, P.fused_r * mt));
    allow_max_smem((const void *)k_factor_fused_b<B>);
    k_factor_fused_b<B><<<n, 32 * nw, smem, st>>>(rows, P.d_rp, P.d_ci, P.d_diag, P.d_upd_ptr, P.d_upd, vals, dinv,
                                                 P.fused_r, err);
    return true;
}

static void launch_fused(int nw, int n, size_t smem, cudaStream_t st, const int *rows, const PcSystem &P,
                         float *vals, const float *dinv, int *err, int mode) {
    if (mode == 2 &&
        (launch_fused_b<40>(n, smem, st, rows, P, vals, dinv, err) ||
         launch_fused_b<50>(n, smem, st, rows, P, vals, dinv, err) ||
         launch_fused_b<24>(n, smem, st, rows, P, vals, dinv, err) ||
         launch_fused_b<20>(n, smem, st, rows, P, vals, dinv, err) ||
         launch_fused_b<12>(n, smem, st, rows, P, vals, dinv, err)))
        return;
    if (nw == 8) {
        allow_max_smem((const void *)k_factor_fused<8>);
        k_factor_fused<8><<<n, 256, smem, st>>>(rows, P.b, P.d_rp, P.d_ci, P.d_diag, P.d_upd_ptr, P.d_upd, vals,
                                                dinv, P.fused_r, err);
    } else {
        allow_max_smem((const void *)k_factor_fused<16>);
        k_factor_fused<16><<<n, 512, smem, st>>>(rows, P.b, P.d_rp, P.d_ci, P.d_diag, P.d_upd_ptr, P.d_upd, vals,
                                                 dinv, P.fused_r, err);
    }
}

template <class C>
static int factor_impl(irk_ctx *c, double dt) {
    PcSystem &P = c->pc;
    const int s = c->s;
    AsmTables tab;
    memset(&tab, 0, sizeof(tab));
    const bool transformed = c->opt.formulation == IRK_TRANSFORMED;
    int tm = tmark_begin(c);
    if (P.element_major) {
        const double *C0 = transformed ? c->Ainv : c->A;
        for (int q = 0; q < s * s; ++q) tab.cm[q] = C0[q];
        k_assemble_elem<C><<<grid_cap(P.nnz * P.b * P.b), 256, 0, c->stream>>>(
            P.nnz, s, c->m, transformed ? 0 : 1, P.d_rowof, P.d_ci, c->d_J,
            c->nJ > 1 ? (long long)c->nnzb * c->m * c->m : 0LL, c->d_M, c->dfop, tab, dt, (C *)P.d_vals);
    } else {
        if (P.kind == IRK_PC_UNCOUPLED) {
            for (int k = 0; k < s; ++k) tab.cm[k * s + k] = c->Ainv[k * s + k] + c->shift[k];
            tab.cj[0] = -dt;
        } else if (transformed) {
            for (int q = 0; q < s * s; ++q) tab.cm[q] = c->Ainv[q];
            tab.cj[0] = -dt;
        } else {
            tab.cm[0] = 1.0;
            for (int q = 0; q < s * s; ++q) tab.cj[q] = -dt * c->A[q];
        }
        if (P.kind == IRK_PC_UNCOUPLED && c->nJ == 1 && P.nnz % s == 0)
            k_assemble_stages<C><<<grid_cap(P.nnz / s * 256), 256, 0, c->stream>>>(
                P.nnz / s, s, c->m, P.d_asm, c->d_J, c->d_M, c->dfop, tab, (C *)P.d_vals);
        else
            k_assemble<C><<<grid_cap(P.nnz * 256), 256, 0, c->stream>>>(P.nnz, c->m, P.d_asm, c->d_J, c->d_M,
                                                                       c->dfop, tab, (C *)P.d_vals);
    }
    c->launches++;
    tmark_end(c, tm, 3);
    const int b = P.b;
    const size_t smem = (size_t)b * b * sizeof(C) * 2 + (size_t)b * sizeof(C);
    const size_t smem4 = (size_t)b * b * sizeof(C) * 4 + (size_t)2 * b * sizeof(C);
    const bool fast = smem4 <= 227 * 1024;
    allow_max_smem((const void *)k_factor_level2<C>);
    allow_max_smem((const void *)k_factor_level<C>);
    allow_max_smem((const void *)k_factor_diag<C>);
    const int nlev = (int)P.lo_ptr.size() - 1;
    c->stats.factor_fused_levels = 0;
    // staged whole-row products (binary32 factors, diagonal-only updates)
    const int fused_nw = std::is_same<C, float>::value ? fused_warps(P, c->ko.factor_fused) : 0;
    const size_t smem_f = fused_smem(P);
    // inversions in their own small CTAs: every row of level 0 (no lower
    // entries: nothing to update), and the rows of levels with at least
    // split_min rows after their products (one more launch per level)
    const int gjt = std::max(gj_threads(c), (b + 31) / 32 * 32);
    const int split_min = gj_split_min(c);
    const size_t smem_d = ((size_t)2 * b * b + (size_t)2 * b) * sizeof(C);
    for (int l = 0; l < nlev; ++l) {
        int n = P.lo_ptr[l + 1] - P.lo_ptr[l];
        if (n <= 0) continue;
        const int *lrows = P.d_lo_rows + P.lo_ptr[l];
        if (fast) {
            const bool split = l == 0 || n >= split_min;
            if (l > 0) {
                tm = tmark_begin(c);
                if (split && fused_nw > 0) {
                    launch_fused(fused_nw, n, smem_f, c->stream, lrows, P, (float *)P.d_vals, (const float *)P.d_dinv,
                                 c->d_err, c->ko.factor_fused);
                    c->stats.factor_fused_levels++;
                } else
                    k_factor_level2<C><<<n, 256, smem4, c->stream>>>(lrows, b, P.d_rp, P.d_ci, P.d_diag,
                                                                     P.d_upd_ptr, P.d_upd, (C *)P.d_vals,
                                                                     (C *)P.d_dinv, c->d_err, split ? 0 : 1);
                tmark_end(c, tm, 4);
            }
            if (split) {
                tm = tmark_begin(c);
                if (!launch_diag_rows<C>(c->stream, n, b, lrows, P.d_diag, (const C *)P.d_vals, (C *)P.d_dinv,
                                         c->d_err, c->ko.factor_gj_rows != 0))
                    k_factor_diag<C><<<n, gjt, smem_d, c->stream>>>(lrows, b, P.d_diag, (const C *)P.d_vals,
                                                                    (C *)P.d_dinv, c->d_err);
                tmark_end(c, tm, 5);
                c->launches++;
            }
        } else {
            tm = tmark_begin(c);
            k_factor_level<C><<<n, 256, smem, c->stream>>>(P.d_lo_rows + P.lo_ptr[l], b, P.d_rp, P.d_ci,
                                                           P.d_diag, P.d_upd_ptr, P.d_upd, (C *)P.d_vals,
                                                           (C *)P.d_dinv, c->d_err);
            tmark_end(c, tm, 4);
        }
        if (!fast || l > 0) c->launches++;
    }
    if (c->fprec == IRK_FACTOR_BF16) {
        const long long bb = (long long)b * b;
        k_to_bf16<C><<<grid_cap(P.nnz * bb), 256, 0, c->stream>>>(P.nnz * bb, (const C *)P.d_vals,
                                                                  (__nv_bfloat16 *)P.d_vals16);
        k_to_bf16<C><<<grid_cap(P.nb * bb), 256, 0, c->stream>>>(P.nb * bb, (const C *)P.d_dinv,
                                                                 (__nv_bfloat16 *)P.d_dinv16);
        c->launches += 2;
    }
    return cuda_status(cudaGetLastError());
}

int pc_factor(irk_ctx *c, double dt) {
    if (c->pc.kind == IRK_PC_NONE) return IRK_OK;
    return c->fprec == IRK_FACTOR_FP64 ? factor_impl<double>(c, dt) : factor_impl<float>(c, dt);
}

template <class AR, class C, class F>
static int apply_persistent(irk_ctx *c, const vec8 *v, vec8 *z, const F *vals, const F *dinv) {
    PcSystem &P = c->pc;
    auto kern = k_sweep_staged<AR, C, F>;
    const size_t blk_bytes = (size_t)P.b * P.b * sizeof(F);
    const size_t slot_stride = (blk_bytes + 127) / 128 * 128;
    // slots per warp: the longest item, within about 48 KB per warp; up to 4
    // warps per CTA, fewer when one slot is large
    int NS = std::max(1, std::min(std::min(P.max_item_blocks, 16), (int)((48 * 1024) / slot_stride)));
    const size_t warp_bytes = slot_stride * NS + 128;
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(227 * 1024) / warp_bytes));
    const int threads = 32 * warps;
    const size_t smem = warp_bytes * warps;
    if (smem > 227 * 1024) return IRK_ERR_INVALID;
    if (P.coop_blocks == 0 || P.coop_smem != smem) {
        allow_max_smem((const void *)kern);
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
        P.coop_blocks = per_sm * sms;
        P.coop_smem = smem;
        if (P.coop_blocks <= 0) return IRK_ERR_CUDA;
    }
    int nb = P.nb, b = P.b, ep = ++P.epoch;
    const int *lo = P.d_lo_rows, *up = P.d_up_rows, *rp = P.d_rp, *ci = P.d_ci, *vo = P.d_voff;
    unsigned long long *yll = P.d_yll, *zll = P.d_zll;
    int *err = c->d_err;
    SweepLanes none = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int spin = c->spin;
    void *args[] = {&nb, &b, &NS, &lo, &up, &rp, &ci, &vo, &vals, &dinv, &v, &yll, &zll, &z, &ep, &err, &none, &spin};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, P.coop_blocks, threads, args, smem, c->stream);
    c->launches++;
    return cuda_status(e);
}

// The two-colour application (k_sweep_fd, k_sweep_bu) for block size B:
// k_sweep_fd with four rows per thread (two when B is not a multiple of 4),
// k_sweep_bu with one (its accumulators grow as rows x stages; measured on
// the 20000-triangle workload: 0.084 ms per launch with one row, 0.105 and
// 0.115 ms with two and four).
template <class AR, class C, class F, int B>
static bool apply_two_colour(irk_ctx *c, const vec8 *v, vec8 *z, const F *vals, const F *dinv) {
    PcSystem &P = c->pc;
    if (P.b != B) return false;
    constexpr int RW = (B % 4 == 0) ? 4 : 2;
    constexpr int G = 256 / (B / RW);
    const int threads = (G * (B / RW) + 31) / 32 * 32;
    constexpr int G1 = 256 / B;
    const int threads1 = (G1 * B + 31) / 32 * 32;
    C *y = (C *)P.d_y;
    int tm = tmark_begin(c);
    const int n1 = P.lo_ptr[2] - P.lo_ptr[1];
    if (n1 > 0) {
        k_sweep_fd<AR, F, B, RW><<<(n1 + G - 1) / G, threads, 0, c->stream>>>(
            P.d_lo_rows + P.lo_ptr[1], n1, P.d_rp, P.d_ci, P.d_voff, vals, dinv, v, y, z);
        c->launches++;
    }
    tmark_end(c, tm, 6);
    tm = tmark_begin(c);
    const int s = c->s;
    if (P.shared_upper && s >= 2 && s <= 4 && c->ko.sweep_shared_upper) {
        const int n2 = P.up0_ptr[2] - P.up0_ptr[1];
        auto kern = s == 2 ? k_sweep_bu<AR, C, F, 2, B>
                           : (s == 3 ? k_sweep_bu<AR, C, F, 3, B> : k_sweep_bu<AR, C, F, 4, B>);
        if (n2 > 0) {
            kern<<<(n2 + G1 - 1) / G1, threads1, 0, c->stream>>>(P.d_up0_rows + P.up0_ptr[1], n2, c->T, P.d_rp,
                                                                 P.d_ci, P.d_voff, vals, dinv, v, y, z);
            c->launches++;
        }
    } else {
        const int n2 = P.up_ptr[2] - P.up_ptr[1];
        if (n2 > 0) {
            k_sweep_bu<AR, C, F, 1, B><<<(n2 + G1 - 1) / G1, threads1, 0, c->stream>>>(
                P.d_up_rows + P.up_ptr[1], n2, c->T, P.d_rp, P.d_ci, P.d_voff, vals, dinv, v, y, z);
            c->launches++;
        }
    }
    tmark_end(c, tm, 7);
    c->stats.sweep_two_colour = 1;
    return true;
}

// Level sweeps with the block size at compile time (binary32 compute,
// double-float vectors): the first forward level (rows without lower
// entries: y = v) by the generic kernel, the others by k_sweep_fl, every
// backward level by k_sweep_bu starting from y.  The same arithmetic as the
// generic level kernels, so the same bits.
template <class AR, class C, class F, int B>
static bool apply_levels_b(irk_ctx *c, const vec8 *v, vec8 *z, const F *vals, const F *dinv) {
    PcSystem &P = c->pc;
    if (P.b != B) return false;
    constexpr int RW = (B % 4 == 0) ? 4 : 2;
    constexpr int G = 256 / (B / RW);
    const int threads = (G * (B / RW) + 31) / 32 * 32;
    constexpr int G1 = 256 / B;
    const int threads1 = (G1 * B + 31) / 32 * 32;
    C *y = (C *)P.d_y;
    const int nlo = (int)P.lo_ptr.size() - 1;
    int tm = tmark_begin(c);
    for (int l = 0; l < nlo; ++l) {
        const int n = P.lo_ptr[l + 1] - P.lo_ptr[l];
        if (n <= 0) continue;
        if (l == 0) {
            const int groups = std::max(1, 256 / B);
            k_sweep_fwd<AR, C, F><<<(n + groups - 1) / groups, (groups * B + 31) / 32 * 32, 0, c->stream>>>(
                P.d_lo_rows + P.lo_ptr[l], n, B, P.d_rp, P.d_ci, P.d_voff, vals, v, y);
        } else {
            k_sweep_fl<AR, F, B, RW><<<(n + G - 1) / G, threads, 0, c->stream>>>(
                P.d_lo_rows + P.lo_ptr[l], n, P.d_rp, P.d_ci, P.d_voff, vals, v, y);
        }
        c->launches++;
    }
    tmark_end(c, tm, 6);
    tm = tmark_begin(c);
    const int s = c->s;
    const bool shared = P.shared_upper && s >= 2 && s <= 4 && c->ko.sweep_shared_upper;
    auto kern = !shared ? k_sweep_bu<AR, C, F, 1, B, true>
                        : (s == 2 ? k_sweep_bu<AR, C, F, 2, B, true>
                                  : (s == 3 ? k_sweep_bu<AR, C, F, 3, B, true> : k_sweep_bu<AR, C, F, 4, B, true>));
    const std::vector<int> &up = shared ? P.up0_ptr : P.up_ptr;
    const int *rows = shared ? P.d_up0_rows : P.d_up_rows;
    for (int l = 0; l + 1 < (int)up.size(); ++l) {
        const int n = up[l + 1] - up[l];
        if (n <= 0) continue;
        kern<<<(n + G1 - 1) / G1, threads1, 0, c->stream>>>(rows + up[l], n, c->T, P.d_rp, P.d_ci, P.d_voff, vals,
                                                          dinv, v, y, z);
        c->launches++;
    }
    tmark_end(c, tm, 7);
    return true;
}

template <class AR, class C, class F>
static int apply_impl(irk_ctx *c, const vec8 *v, vec8 *z, const F *vals, const F *dinv) {
    PcSystem &P = c->pc;
    const int b = P.b;
    c->stats.sweep_two_colour = 0;
    if (P.persistent) return apply_persistent<AR, C, F>(c, v, z, vals, dinv);
    if constexpr (std::is_same<C, float>::value && std::is_same<AR, ArDF>::value) {
        if (P.two_colour && c->ko.sweep_two_colour &&
            (apply_two_colour<AR, C, F, 40>(c, v, z, vals, dinv) ||
             apply_two_colour<AR, C, F, 50>(c, v, z, vals, dinv) ||
             apply_two_colour<AR, C, F, 24>(c, v, z, vals, dinv) ||
             apply_two_colour<AR, C, F, 20>(c, v, z, vals, dinv) ||
             apply_two_colour<AR, C, F, 12>(c, v, z, vals, dinv)))
            return cuda_status(cudaGetLastError());
        if (c->ko.sweep_compiled_levels &&
            (apply_levels_b<AR, C, F, 40>(c, v, z, vals, dinv) || apply_levels_b<AR, C, F, 50>(c, v, z, vals, dinv) ||
             apply_levels_b<AR, C, F, 24>(c, v, z, vals, dinv) || apply_levels_b<AR, C, F, 20>(c, v, z, vals, dinv) ||
             apply_levels_b<AR, C, F, 12>(c, v, z, vals, dinv)))
            return cuda_status(cudaGetLastError());
    }
    const int groups = std::max(1, 256 / b);
    const int threads = (groups * b + 31) / 32 * 32;
    C *y = (C *)P.d_y;
    const int nlo = (int)P.lo_ptr.size() - 1;
    int tm = tmark_begin(c);
    for (int l = 0; l < nlo; ++l) {
        int n = P.lo_ptr[l + 1] - P.lo_ptr[l];
        if (n <= 0) continue;
        k_sweep_fwd<AR, C, F><<<(n + groups - 1) / groups, threads, 0, c->stream>>>(
            P.d_lo_rows + P.lo_ptr[l], n, b, P.d_rp, P.d_ci, P.d_voff, vals, v, y);
        c->launches++;
    }
    tmark_end(c, tm, 6);
    tm = tmark_begin(c);
    const size_t smem = (size_t)groups * b * sizeof(C);
    const int s = c->s;
    if (P.shared_upper && s >= 2 && s <= 4 && c->ko.sweep_shared_upper) {
        auto kern = s == 2 ? k_sweep_bwd_shared<AR, C, F, 2>
                           : (s == 3 ? k_sweep_bwd_shared<AR, C, F, 3> : k_sweep_bwd_shared<AR, C, F, 4>);
        const int nup0 = (int)P.up0_ptr.size() - 1;
        for (int l = 0; l < nup0; ++l) {
            int n = P.up0_ptr[l + 1] - P.up0_ptr[l];
            if (n <= 0) continue;
            kern<<<(n + groups - 1) / groups, threads, smem * s, c->stream>>>(
                P.d_up0_rows + P.up0_ptr[l], n, b, c->T, P.d_rp, P.d_ci, P.d_voff, vals, dinv, y, z);
            c->launches++;
        }
        tmark_end(c, tm, 7);
        return cuda_status(cudaGetLastError());
    }
    const int nup = (int)P.up_ptr.size() - 1;
    for (int l = 0; l < nup; ++l) {
        int n = P.up_ptr[l + 1] - P.up_ptr[l];
        if (n <= 0) continue;
        k_sweep_bwd<AR, C, F><<<(n + groups - 1) / groups, threads, smem, c->stream>>>(
            P.d_up_rows + P.up_ptr[l], n, b, P.d_rp, P.d_ci, P.d_voff, vals, dinv, y, z);
        c->launches++;
    }
    tmark_end(c, tm, 7);
    return cuda_status(cudaGetLastError());
}

template <class AR>
static int apply_ar(irk_ctx *c, const vec8 *v, vec8 *z) {
    PcSystem &P = c->pc;
    if (c->fprec == IRK_FACTOR_FP64)
        return apply_impl<AR, double, double>(c, v, z, (const double *)P.d_vals, (const double *)P.d_dinv);
    if (c->fprec == IRK_FACTOR_FP32)
        return apply_impl<AR, float, float>(c, v, z, (const float *)P.d_vals, (const float *)P.d_dinv);
    return apply_impl<AR, float, __nv_bfloat16>(c, v, z, (const __nv_bfloat16 *)P.d_vals16,
                                                (const __nv_bfloat16 *)P.d_dinv16);
}

int pc_apply(irk_ctx *c, const vec8 *v, vec8 *z) {
    if (c->pc.kind == IRK_PC_NONE) {
        if (cudaMemcpyAsync(z, v, (size_t)c->N * sizeof(vec8), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return IRK_ERR_CUDA;
        return IRK_OK;
    }
    return c->df ? apply_ar<ArDF>(c, v, z) : apply_ar<ArF64>(c, v, z);
}

// ---------------------------------------------------------------------------
// irk_apply_precond_noalloc: the preconditioner application with its working
// vectors in a fixed device array instead of context-owned buffers, for
// callers that cannot allocate (see the header).  Layout of the array:
// [header | 256 B: error word at 0, |x| maximum at 64, scale pair at 128]
// [V internal | N vec8] [Z internal | N vec8]
// [forward words | N*w] [backward words | N*w], each region 256-byte aligned.
static __device__ __align__(256) unsigned char irk_noalloc_scratch[IRK_NOALLOC_SCRATCH_BYTES];

namespace {

#define IRK_NOALLOC_MAX_DEVICES 64
unsigned char *g_noalloc_base[IRK_NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mutex;

size_t na_align(size_t x) { return (x + 255) / 256 * 256; }

// Cooperative grid of the persistent sweep for one (kernel, CTA size, shared
// memory) on one device, computed once (the occupancy query is not free).
struct NaGrid {
    const void *kern;
    int dev, threads;
    size_t smem;
    int grid;
};
#define IRK_NOALLOC_GRIDS 256
NaGrid g_na_grids[IRK_NOALLOC_GRIDS];  // fixed table (no host allocation), guarded by g_noalloc_mutex
int g_na_ngrids = 0;

int na_grid(const void *kern, int dev, int threads, size_t smem) {
    std::lock_guard<std::mutex> g(g_noalloc_mutex);
    for (int q = 0; q < g_na_ngrids; ++q) {
        const NaGrid &e = g_na_grids[q];
        if (e.kern == kern && e.dev == dev && e.threads == threads && e.smem == smem) return e.grid;
    }
    if (allow_max_smem(kern)) return -1;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm <= 0)
        return -1;
    if (g_na_ngrids < IRK_NOALLOC_GRIDS) g_na_grids[g_na_ngrids++] = {kern, dev, threads, smem, per_sm * sms};
    return per_sm * sms;
}

template <class AR, class C, class F>
int na_sweep(irk_ctx *c, const vec8 *v, vec8 *z, const F *vals, const F *dinv, unsigned long long *yll,
             unsigned long long *zll, int *err, cudaStream_t st) {
    PcSystem &P = c->pc;
    auto kern = k_sweep_staged<AR, C, F>;
    const size_t blk_bytes = (size_t)P.b * P.b * sizeof(F);
    const size_t slot_stride = (blk_bytes + 127) / 128 * 128;
    int NS = std::max(1, std::min(std::min(P.max_item_blocks, 16), (int)((48 * 1024) / slot_stride)));
    const size_t warp_bytes = slot_stride * NS + 128;
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(227 * 1024) / warp_bytes));
    const int threads = 32 * warps;
    const size_t smem = warp_bytes * warps;
    if (smem > 227 * 1024) return IRK_ERR_INVALID;
    int grid = na_grid((const void *)kern, c->dev, threads, smem);
    if (grid <= 0) return IRK_ERR_CUDA;
    int nb = P.nb, b = P.b, ep = 1, spin = c->spin;
    const int *lo = P.d_lo_rows, *up = P.d_up_rows, *rp = P.d_rp, *ci = P.d_ci, *vo = P.d_voff;
    SweepLanes none = {nullptr, nullptr, nullptr, nullptr, nullptr};
    void *args[] = {&nb, &b, &NS, &lo, &up, &rp, &ci, &vo, &vals, &dinv, &v, &yll, &zll, &z, &ep, &err, &none, &spin};
    return cuda_status(cudaLaunchCooperativeKernel((const void *)kern, grid, threads, args, smem, st));
}

template <class AR>
int na_sweep_prec(irk_ctx *c, const vec8 *v, vec8 *z, unsigned long long *yll, unsigned long long *zll, int *err,
                  cudaStream_t st) {
    PcSystem &P = c->pc;
    if (c->fprec == IRK_FACTOR_FP64)
        return na_sweep<AR, double, double>(c, v, z, (const double *)P.d_vals, (const double *)P.d_dinv, yll, zll,
                                            err, st);
    if (c->fprec == IRK_FACTOR_FP32)
        return na_sweep<AR, float, float>(c, v, z, (const float *)P.d_vals, (const float *)P.d_dinv, yll, zll, err,
                                          st);
    return na_sweep<AR, float, __nv_bfloat16>(c, v, z, (const __nv_bfloat16 *)P.d_vals16,
                                              (const __nv_bfloat16 *)P.d_dinv16, yll, zll, err, st);
}

}  // namespace

extern "C" int irk_apply_precond_noalloc(irk_ctx *c, const double *V, double *Z, void *stream) {
    if (!c || !V || !Z || V == Z) return IRK_ERR_INVALID;
    if (c->pc.kind == IRK_PC_NONE || !c->pc.persistent) return IRK_ERR_INVALID;
    if (!c->factored) return IRK_ERR_STATE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->dev || dev < 0 || dev >= IRK_NOALLOC_MAX_DEVICES)
        return IRK_ERR_INVALID;
    const size_t N = (size_t)c->N;
    const size_t w = (c->fprec == IRK_FACTOR_FP64) ? 2 : 1;
    const size_t need = 256 + 2 * na_align(N * 8) + 2 * na_align(N * 8 * w);
    if (need > IRK_NOALLOC_SCRATCH_BYTES) return IRK_ERR_SCRATCH_LIMIT;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mutex);
        if (!g_noalloc_base[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, irk_noalloc_scratch);
            if (e != cudaSuccess || !p) return IRK_ERR_CUDA;
            g_noalloc_base[dev] = (unsigned char *)p;
        }
        base = g_noalloc_base[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int *err = reinterpret_cast<int *>(base);
    unsigned long long *amax = reinterpret_cast<unsigned long long *>(base + 64);
    double *scale = reinterpret_cast<double *>(base + 128);
    vec8 *vin = reinterpret_cast<vec8 *>(base + 256);
    vec8 *vout = reinterpret_cast<vec8 *>(base + 256 + na_align(N * 8));
    unsigned long long *yll = reinterpret_cast<unsigned long long *>(base + 256 + 2 * na_align(N * 8));
    unsigned long long *zll = reinterpret_cast<unsigned long long *>(base + 256 + 2 * na_align(N * 8) + na_align(N * 8 * w));
    // what must start at zero: the error word and the published words (epoch 0 = unwritten)
    if (cudaMemsetAsync(err, 0, 256, st) != cudaSuccess ||
        cudaMemsetAsync(yll, 0, 2 * na_align(N * 8 * w), st) != cudaSuccess)
        return IRK_ERR_CUDA;
    // double-float: the same power-of-two scaling as irk_apply_precond
    const double *sc = nullptr;
    int rc = IRK_OK;
    if (c->df) {
        rc = launch_pow2_scale(st, (long long)N, V, amax, scale);
        sc = scale;
    }
    if (!rc) rc = launch_to_internal_on(st, c, V, vin, sc);
    if (!rc) rc = c->df ? na_sweep_prec<ArDF>(c, vin, vout, yll, zll, err, st)
                        : na_sweep_prec<ArF64>(c, vin, vout, yll, zll, err, st);
    if (!rc) rc = launch_to_external_on(st, c, vout, Z, sc);
    int herr = 0;
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    if (!rc) {
        if (herr & IRK_DEV_ERR_SINGULAR) rc = IRK_ERR_SINGULAR;
        else if (herr & IRK_DEV_ERR_NONFINITE) rc = IRK_ERR_NONFINITE;
        else if (herr & IRK_DEV_ERR_TIMEOUT) rc = IRK_ERR_TIMEOUT;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// Launchers used by the multi-request engine (group.cu): the same kernels on
// caller-provided arrays.
int ilu_assemble(cudaStream_t st, int fprec, long long nnz, int m, const AsmEntry *ent, const vec8 *J,
                 const vec8 *M, int df, const double *cm, int ncm, const double *cj, int ncj, void *vals) {
    AsmTables tab;
    memset(&tab, 0, sizeof(tab));
    for (int q = 0; q < ncm && q < IRK_MAX_S * IRK_MAX_S; ++q) tab.cm[q] = cm[q];
    for (int q = 0; q < ncj && q < IRK_MAX_S * IRK_MAX_S; ++q) tab.cj[q] = cj[q];
    const int g = grid_cap(nnz * m * m);
    if (fprec == IRK_FACTOR_FP64)
        k_assemble<double><<<g, 256, 0, st>>>(nnz, m, ent, J, M, df, tab, (double *)vals);
    else
        k_assemble<float><<<g, 256, 0, st>>>(nnz, m, ent, J, M, df, tab, (float *)vals);
    return cuda_status(cudaGetLastError());
}

int ilu_factor_level(cudaStream_t st, int fprec, const int *rows, int nrows, int b, const int *rp, const int *ci,
                     const int *diag, const int *upd_ptr, const int *upd, void *vals, void *dinv, int *err) {
    if (nrows <= 0) return IRK_OK;
    if (fprec == IRK_FACTOR_FP64) {
        const size_t smem4 = (size_t)b * b * 8 * 4 + (size_t)2 * b * 8;
        if (smem4 > 227 * 1024) return IRK_ERR_INVALID;
        allow_max_smem((const void *)k_factor_level2<double>);
        k_factor_level2<double><<<nrows, 256, smem4, st>>>(rows, b, rp, ci, diag, upd_ptr, upd, (double *)vals,
                                                           (double *)dinv, err, 1);
    } else {
        const size_t smem4 = (size_t)b * b * 4 * 4 + (size_t)2 * b * 4;
        if (smem4 > 227 * 1024) return IRK_ERR_INVALID;
        allow_max_smem((const void *)k_factor_level2<float>);
        k_factor_level2<float><<<nrows, 256, smem4, st>>>(rows, b, rp, ci, diag, upd_ptr, upd, (float *)vals,
                                                          (float *)dinv, err, 1);
    }
    return cuda_status(cudaGetLastError());
}

template <class AR, class C>
static int sweep_group_impl(cudaStream_t st, int dev, int nitems, int b, int max_item_blocks, const int *lo,
                            const int *up, const int *rp, const int *ci, const int *voff, const void *vals,
                            const void *dinv, vec8 *vpool, unsigned long long *llpool, int ep, int *err,
                            SweepLanes lanes, int spin) {
    auto kern = k_sweep_staged<AR, C, C>;
    const size_t slot_stride = ((size_t)b * b * sizeof(C) + 127) / 128 * 128;
    int NS = std::max(1, std::min(std::min(max_item_blocks, 16), (int)((48 * 1024) / slot_stride)));
    const size_t warp_bytes = slot_stride * NS + 128;
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)(227 * 1024) / warp_bytes));
    const int threads = 32 * warps;
    const size_t smem = warp_bytes * warps;
    if (smem > 227 * 1024) return IRK_ERR_INVALID;
    allow_max_smem((const void *)kern);
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = per_sm * sms;
    if (grid <= 0) return IRK_ERR_CUDA;
    int nb = nitems;
    const C *vv = (const C *)vals, *dd = (const C *)dinv;
    const vec8 *v = vpool;
    vec8 *z = vpool;
    unsigned long long *yll = llpool, *zll = llpool;
    void *args[] = {&nb, &b, &NS, &lo, &up, &rp, &ci, &voff, &vv, &dd, &v, &yll, &zll, &z, &ep, &err, &lanes, &spin};
    return cuda_status(cudaLaunchCooperativeKernel((const void *)kern, grid, threads, args, smem, st));
}

// Cooperative sweep over a merged work list of several requests: lo / up hold
// nitems forward / backward rows; per-lane bases in vec8 (vectors) and word
// (published values) units relative to vpool / llpool.
int ilu_sweep_group(cudaStream_t st, int dev, int fprec, int df, int nitems, int b, int max_item_blocks,
                    const int *lo, const int *up, const int *rp, const int *ci, const int *voff, const void *vals,
                    const void *dinv, vec8 *vpool, unsigned long long *llpool, int ep, int *err,
                    const int *lane_of_row, const long long *vin, const long long *zout, const long long *yll,
                    const long long *zll, int spin) {
    SweepLanes L = {lane_of_row, vin, zout, yll, zll};
    if (df) {
        if (fprec == IRK_FACTOR_FP64)
            return sweep_group_impl<ArDF, double>(st, dev, nitems, b, max_item_blocks, lo, up, rp, ci, voff, vals,
                                                  dinv, vpool, llpool, ep, err, L, spin);
        return sweep_group_impl<ArDF, float>(st, dev, nitems, b, max_item_blocks, lo, up, rp, ci, voff, vals, dinv,
                                             vpool, llpool, ep, err, L, spin);
    }
    if (fprec == IRK_FACTOR_FP64)
        return sweep_group_impl<ArF64, double>(st, dev, nitems, b, max_item_blocks, lo, up, rp, ci, voff, vals, dinv,
                                               vpool, llpool, ep, err, L, spin);
    return sweep_group_impl<ArF64, float>(st, dev, nitems, b, max_item_blocks, lo, up, rp, ci, voff, vals, dinv,
                                          vpool, llpool, ep, err, L, spin);
}
