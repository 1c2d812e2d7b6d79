// k_krylov.cu -- Arnoldi (modified Gram-Schmidt), Givens rotations and the
// least-squares update of restarted flexible GMRES (Sec. 4: one operator
// product and one preconditioner application per iteration).
//
// Reductions are deterministic: every CTA writes one partial in a fixed
// order of work, and the last CTA to finish (ticket counter) sums the
// partials in index order with a fixed tree.  No floating-point atomics, so
// the same input gives bit-identical results.
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "arith.cuh"

namespace {

// Scalars written by the reductions: the binary64 value and its double-float
// split, so that double-float kernels never touch the FP64 pipe.
struct Scal {
    double d;      // value
    float hi, lo;  // value as a double-float pair
    double inv;    // 1 / value (0 when value == 0)
    float ihi, ilo;
};

template <class AR>
__device__ __forceinline__ typename AR::val block_reduce(typename AR::val v, typename AR::val *sh) {
    // warp tree, then the warp results in index order
    for (int d = 16; d > 0; d >>= 1) v = AR::add(v, AR::shfl_down(v, d));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        v = lane < nw ? sh[lane] : AR::from_float(0.f);
        for (int d = 16; d > 0; d >>= 1) v = AR::add(v, AR::shfl_down(v, d));
    }
    return v;  // valid in thread 0
}

// Sum of the n per-CTA partials of a reduction by one warp: lane l adds
// partials l, l + 32, ... in order, then a fixed shuffle tree; every CTA
// computes the same value in the same order.  Valid in lane 0 (the other
// lanes hold partial sums of the tree; only lane 0's result is used).
template <class AR>
__device__ __forceinline__ typename AR::val warp_sum_partials(const vec8 *pb, int n) {
    typename AR::acc a = AR::zero();
    for (int q = threadIdx.x & 31; q < n; q += 32) AR::add_to(a, AR::ldcg(pb + q));
    typename AR::val v = AR::value(a);
    for (int d = 16; d > 0; d >>= 1) v = AR::add(v, AR::shfl_down(v, d));
    return v;
}

template <class AR>
__device__ __forceinline__ typename AR::val scal_val(const Scal *s) {
    return AR::coef(s->d, s->hi, s->lo);
}

__device__ __forceinline__ void scal_store_d(Scal *s, double d) {
    s->d = d;
    float h = (float)d;
    s->hi = h;
    s->lo = (float)(d - (double)h);
    double inv = d != 0.0 ? 1.0 / d : 0.0;
    s->inv = inv;
    h = (float)inv;
    s->ihi = h;
    s->ilo = (float)(inv - (double)h);
}

template <class AR>
__device__ __forceinline__ void scal_store(Scal *s, typename AR::val v) {
    scal_store_d(s, AR::to_double(v));
}

// w <- w - hprev * vprev (if vprev), then out = <w, v> (or ||w|| if take_sqrt
// and v == w).  out is also copied into H_out (binary64) when non-null.
template <class AR>
__global__ void __launch_bounds__(256) k_axpy_dot(long long N, vec8 *w, const vec8 *vprev, const Scal *hprev,
                                                  const vec8 *v, int self, int take_sqrt, Scal *out,
                                                  double *H_out, vec8 *part,
                                                  unsigned int *ticket, int *err) {
    typedef typename AR::val val;
    __shared__ val sh[32];
    __shared__ int s_last;
    val nh = AR::from_float(0.f);
    if (vprev) nh = AR::neg(scal_val<AR>(hprev));
    typename AR::acc acc = AR::zero();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        val wv = AR::ld(w + e);
        if (vprev) {
            wv = AR::add(wv, AR::mul(nh, AR::ld(vprev + e)));
            AR::st(w + e, wv);
        }
        AR::fma(acc, wv, self ? wv : AR::ld(v + e));
    }
    val r = block_reduce<AR>(AR::value(acc), sh);
    if (threadIdx.x == 0) {
        AR::st(part + blockIdx.x, r);
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    typename AR::acc a2 = AR::zero();
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) AR::add_to(a2, AR::ldcg(part + q));
    __syncthreads();
    val tot = block_reduce<AR>(AR::value(a2), sh);
    if (threadIdx.x == 0) {
        double d = AR::to_double(tot);
        if (!isfinite(d)) {
            atomicOr(err, IRK_DEV_ERR_NONFINITE);
            d = 0.0;
        }
        if (take_sqrt) d = d > 0.0 ? sqrt(d) : 0.0;
        scal_store_d(out, d);
        if (H_out) *H_out = d;
        *ticket = 0u;
    }
}

// v_out = w / h, or zero when h == 0 (breakdown).
template <class AR>
__global__ void k_scale_inv(long long N, vec8 *w, const Scal *h) {
    typedef typename AR::val val;
    const val inv = AR::coef(h->inv, h->ihi, h->ilo);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
        AR::st(w + e, AR::mul(AR::ld(w + e), inv));
}

// Givens rotations on column j of H (binary64, one thread): the earlier
// rotations, then the new one that zeroes H[j+1][j]; est = |g[j+1]|.
__device__ void givens_col(int j, int R, double *H, double *cs, double *sn, double *g, double *est, int *err) {
    for (int i = 0; i < j; ++i) {
        double a = H[i * R + j], b = H[(i + 1) * R + j];
        H[i * R + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * R + j] = -sn[i] * a + cs[i] * b;
    }
    double a = H[j * R + j], b = H[(j + 1) * R + j];
    double rho = hypot(a, b);
    if (!isfinite(rho)) {
        atomicOr(err, IRK_DEV_ERR_NONFINITE);
        *est = 0.0;
        return;
    }
    double c = rho == 0.0 ? 1.0 : a / rho;
    double s = rho == 0.0 ? 0.0 : b / rho;
    cs[j] = c;
    sn[j] = s;
    H[j * R + j] = rho;
    H[(j + 1) * R + j] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    *est = fabs(g[j + 1]);
}

__global__ void k_givens(int j, int R, double *H, double *cs, double *sn, double *g, double *est,
                         int *err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    givens_col(j, R, H, cs, sn, g, est, err);
}

// The iteration's status for the host in one 24-byte block: residual
// estimate, h_{j+1,j} and the device error word (as a double), written by
// CTA 0 last (also when it leaves on a barrier timeout), so one copy replaces
// three.
__device__ __forceinline__ void arnoldi_status(double *status, double est, double hn, int *err) {
    status[0] = est;
    status[1] = hn;
    status[2] = (double)*reinterpret_cast<volatile int *>(err);
}

// Bounded grid-wide barrier of a cooperative launch (every CTA resident):
// bar[0] counts the arrivals of the current generation, bar[1] is the
// generation.  After `spin` polls (irk_options.spin_limit) a CTA records a
// timeout and the barrier returns false (the caller leaves; the host resets
// bar per solve).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *err, int *s_ok, int spin) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_u32(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            int spins = 0;
            while (ld_acquire_u32(bar + 1) == gen) {
                if (++spins >= spin) {
                    ok = 0;
                    atomicOr(err, IRK_DEV_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// One Arnoldi step of FGMRES after the operator product w = B z_j, in one
// cooperative launch: modified Gram-Schmidt against v_0..v_j (for i = 0..j:
// w -= h_{i-1,j} v_{i-1}, fused with h_{i,j} = <w, v_i>), then
// w -= h_{j,j} v_j with h_{j+1,j} = ||w||, w /= h_{j+1,j} (zero on
// breakdown), and the Givens rotations of column j.  The same element
// operations and scalar splits as k_axpy_dot / k_scale_inv; each reduction's
// per-CTA partials are summed in index order by every CTA (identical values
// everywhere, deterministic), in a buffer alternating between steps so that a
// CTA already in the next step never overwrites partials still being read.
template <class AR, int NT>
__global__ void __launch_bounds__(NT) k_arnoldi(long long N, int j, int R, vec8 *w, const vec8 *V, Scal *slots,
                                                 double *H, double *cs, double *sn, double *g, double *est,
                                                 vec8 *part, unsigned *bar, int *err, double *status, int spin) {
    typedef typename AR::val val;
    __shared__ val sh[32];
    __shared__ int s_ok;
    __shared__ double s_h;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double hprev = 0.0;
    for (int i = 0; i <= j + 1; ++i) {
        const bool last = i == j + 1;
        const vec8 *vp = i > 0 ? V + (long long)(i - 1) * N : nullptr;
        const vec8 *vi = last ? nullptr : V + (long long)i * N;
        const float hh = (float)hprev;
        const val nh = AR::neg(AR::coef(hprev, hh, (float)(hprev - (double)hh)));
        typename AR::acc acc = AR::zero();
        // U elements per thread and round, all loads issued before the
        // arithmetic; accumulation in the thread's element order
        constexpr int U = 4;
        for (long long e = e0; e < N; e += U * stride) {
            val wv[U], pv[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long ee = e + u * stride;
                const bool ok = ee < N;
                wv[u] = ok ? AR::ldcg(w + ee) : AR::from_float(0.f);  // written by this thread in the previous step
                pv[u] = (ok && vp) ? AR::ld(vp + ee) : AR::from_float(0.f);
                xv[u] = (ok && !last) ? AR::ld(vi + ee) : AR::from_float(0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long ee = e + u * stride;
                if (ee >= N) break;
                if (vp) {
                    wv[u] = AR::add(wv[u], AR::mul(nh, pv[u]));
                    AR::st(w + ee, wv[u]);
                }
                AR::fma(acc, wv[u], last ? wv[u] : xv[u]);
            }
        }
        vec8 *pb = part + (i & 1) * gridDim.x;
        const val r = block_reduce<AR>(AR::value(acc), sh);
        if (threadIdx.x == 0) AR::st(pb + blockIdx.x, r);
        if (!grid_sync(bar, err, &s_ok, spin)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) arnoldi_status(status, 0.0, 0.0, err);
            return;
        }
        if (threadIdx.x < 32) {
            const val tot = warp_sum_partials<AR>(pb, (int)gridDim.x);
            double d = AR::to_double(tot);
            if (!isfinite(d)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_NONFINITE);
                d = 0.0;
            }
            if (last) d = d > 0.0 ? sqrt(d) : 0.0;
            if (threadIdx.x == 0) {
                s_h = d;
                if (blockIdx.x == 0) {
                    scal_store_d(slots + 2 + i, d);
                    H[i * R + j] = d;
                }
            }
        }
        __syncthreads();
        hprev = s_h;
    }
    const double inv = hprev != 0.0 ? 1.0 / hprev : 0.0;
    const float ih = (float)inv;
    const val iv = AR::coef(inv, ih, (float)(inv - (double)ih));
    for (long long e = e0; e < N; e += 2 * stride) {
        const long long e2 = e + stride;
        const val a0 = AR::ldcg(w + e);
        const val a1 = e2 < N ? AR::ldcg(w + e2) : AR::from_float(0.f);
        AR::st(w + e, AR::mul(a0, iv));
        if (e2 < N) AR::st(w + e2, AR::mul(a1, iv));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        givens_col(j, R, H, cs, sn, g, est, err);
        arnoldi_status(status, *est, hprev, err);
    }
}

// y = H(0:jl, 0:jl)^{-1} g(0:jl) (one thread), stored as Scal for the update.
__global__ void k_backsolve(int jl, int R, const double *H, const double *g, double *y, Scal *ys) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = jl; i >= 0; --i) {
        double acc = g[i];
        for (int k = i + 1; k <= jl; ++k) acc -= H[i * R + k] * y[k];
        double d = H[i * R + i];
        y[i] = d != 0.0 ? acc / d : 0.0;
        scal_store_d(ys + i, y[i]);
    }
}

// x += sum_{i <= jl} y_i Z_i
template <class AR>
__global__ void k_update_x(long long N, int jl, vec8 *x, const vec8 *Z, const Scal *ys) {
    typedef typename AR::val val;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        typename AR::acc acc = AR::zero();
        AR::add_to(acc, AR::ld(x + e));
        for (int i = 0; i <= jl; ++i) AR::fma(acc, scal_val<AR>(ys + i), AR::ld(Z + (long long)i * N + e));
        AR::st(x + e, AR::value(acc));
    }
}

__global__ void k_cycle_start(int R, const Scal *beta, double *g) {
    int t = threadIdx.x;
    for (int q = t; q <= R; q += blockDim.x) g[q] = (q == 0) ? beta->d : 0.0;
}

__global__ void k_zero(long long n, vec8 *v) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) v[e] = 0ull;
}

int grid_stream(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// Scalar slots in c->d_scal (as Scal):
//   0: beta / norm results   1: residual estimate (binary64 in .d)
//   2 + i: h_{i,j} of the current column (i <= restart)
//   64 + i: y_i of the least-squares solution
// (slot size 32 bytes; c->d_scal holds 128 slots)
static Scal *scal(irk_ctx *c, int slot) { return reinterpret_cast<Scal *>(c->d_scal) + slot; }

double *irk_est_ptr(irk_ctx *c) { return &scal(c, 1)->d; }
// status block of k_arnoldi (last scalar slot: 4 doubles)
double *irk_status_ptr(irk_ctx *c) { return &scal(c, IRK_SCAL_SLOTS - 1)->d; }
double *irk_beta_ptr(irk_ctx *c) { return &scal(c, 0)->d; }

int launch_axpy_dot_slot(irk_ctx *c, vec8 *w, const vec8 *vprev, int hprev_slot, const vec8 *v,
                         int self, int take_sqrt, int out_slot, double *H_out) {
    const Scal *hp = vprev ? scal(c, hprev_slot) : nullptr;
    if (c->df)
        k_axpy_dot<ArDF><<<c->red_blocks, 256, 0, c->stream>>>(
            c->N, w, vprev, hp, v, self, take_sqrt, scal(c, out_slot), H_out,
            reinterpret_cast<vec8 *>(c->d_part), c->d_ticket, c->d_err);
    else
        k_axpy_dot<ArF64><<<c->red_blocks, 256, 0, c->stream>>>(
            c->N, w, vprev, hp, v, self, take_sqrt, scal(c, out_slot), H_out,
            reinterpret_cast<vec8 *>(c->d_part), c->d_ticket, c->d_err);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_scale_slot(irk_ctx *c, vec8 *w, int slot) {
    int g = grid_stream(c->N);
    if (c->df)
        k_scale_inv<ArDF><<<g, 256, 0, c->stream>>>(c->N, w, scal(c, slot));
    else
        k_scale_inv<ArF64><<<g, 256, 0, c->stream>>>(c->N, w, scal(c, slot));
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_givens(irk_ctx *c, int j, int restart) {
    k_givens<<<1, 32, 0, c->stream>>>(j, restart, c->d_H, c->d_cs, c->d_sn, c->d_g, &scal(c, 1)->d, c->d_err);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

// The same Arnoldi step with w kept in shared memory: CTA b owns the
// contiguous slice [b*chunk, (b+1)*chunk) of w for the whole step, so each
// Gram-Schmidt step streams only v_{i-1} (just read, mostly from L2) and v_i
// and never rewrites w in HBM until the normalised result.  One CTA per SM;
// used when a slice fits in shared memory.  Element operations as in
// k_arnoldi (the partition of the reductions differs).
template <class AR>
__global__ void __launch_bounds__(1024) k_arnoldi_smem(long long N, long long chunk, int j, int R, vec8 *w,
                                                       const vec8 *V, Scal *slots, double *H, double *cs,
                                                       double *sn, double *g, double *est, vec8 *part,
                                                       unsigned *bar, int *err, double *status, int spin) {
    typedef typename AR::val val;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec8 *ws = reinterpret_cast<vec8 *>(smem_raw);
    __shared__ val sh[32];
    __shared__ int s_ok;
    __shared__ double s_h;
    const long long c0 = (long long)blockIdx.x * chunk;
    const long long c1 = c0 + chunk < N ? c0 + chunk : N;
    const int len = c1 > c0 ? (int)(c1 - c0) : 0;
    for (int e = threadIdx.x; e < len; e += blockDim.x) ws[e] = w[c0 + e];
    __syncthreads();
    double hprev = 0.0;
    for (int i = 0; i <= j + 1; ++i) {
        const bool last = i == j + 1;
        const vec8 *vp = i > 0 ? V + (long long)(i - 1) * N + c0 : nullptr;
        const vec8 *vi = last ? nullptr : V + (long long)i * N + c0;
        const float hh = (float)hprev;
        const val nh = AR::neg(AR::coef(hprev, hh, (float)(hprev - (double)hh)));
        typename AR::acc acc = AR::zero();
        constexpr int U = 4;
        for (int e = threadIdx.x; e < len; e += U * blockDim.x) {
            val wv[U], pv[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int ee = e + u * blockDim.x;
                const bool ok = ee < len;
                wv[u] = ok ? AR::ldv(ws + ee) : AR::from_float(0.f);
                pv[u] = (ok && vp) ? AR::ld(vp + ee) : AR::from_float(0.f);
                xv[u] = (ok && !last) ? AR::ld(vi + ee) : AR::from_float(0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int ee = e + u * blockDim.x;
                if (ee >= len) break;
                if (vp) {
                    wv[u] = AR::add(wv[u], AR::mul(nh, pv[u]));
                    AR::st(ws + ee, wv[u]);
                }
                AR::fma(acc, wv[u], last ? wv[u] : xv[u]);
            }
        }
        vec8 *pb = part + (i & 1) * gridDim.x;
        const val r = block_reduce<AR>(AR::value(acc), sh);
        if (threadIdx.x == 0) AR::st(pb + blockIdx.x, r);
        if (!grid_sync(bar, err, &s_ok, spin)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) arnoldi_status(status, 0.0, 0.0, err);
            return;
        }
        if (threadIdx.x < 32) {
            const val tot = warp_sum_partials<AR>(pb, (int)gridDim.x);
            double d = AR::to_double(tot);
            if (!isfinite(d)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, IRK_DEV_ERR_NONFINITE);
                d = 0.0;
            }
            if (last) d = d > 0.0 ? sqrt(d) : 0.0;
            if (threadIdx.x == 0) {
                s_h = d;
                if (blockIdx.x == 0) {
                    scal_store_d(slots + 2 + i, d);
                    H[i * R + j] = d;
                }
            }
        }
        __syncthreads();
        hprev = s_h;
    }
    const double inv = hprev != 0.0 ? 1.0 / hprev : 0.0;
    const float ih = (float)inv;
    const val iv = AR::coef(inv, ih, (float)(inv - (double)ih));
    for (int e = threadIdx.x; e < len; e += blockDim.x) AR::st(w + c0 + e, AR::mul(AR::ldv(ws + e), iv));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        givens_col(j, R, H, cs, sn, g, est, err);
        arnoldi_status(status, *est, hprev, err);
    }
}

// ---------------------------------------------------------------------------
// The Arnoldi step by classical Gram-Schmidt applied twice (CGS2), in one
// cooperative launch with two grid-wide reductions instead of j + 2:
//   pass 1: h_i = <w, v_i>, i = 0..j                            (reduction 1)
//   pass 2: w' = w - sum_i h_i v_i; q_i = <w', v_i>; ||w'||^2    (reduction 2)
//   pass 3: v_{j+1} = (w' - sum_i q_i v_i) / h_{j+1,j},
// with H[i][j] = h_i + q_i and h_{j+1,j}^2 = ||w'||^2 - sum_i q_i^2: w' minus
// the final vector is V q, in the span of the orthonormal v_i, so the final
// norm follows without a third reduction (q is of the order of pass 2's
// rounding error: no cancellation).  Each CTA owns a contiguous slice of w,
// kept in shared memory when it fits (SM), else updated in place in global
// memory.  The basis is read three times (twice with MGS), in exchange for
// the j dependent grid-wide reductions MGS needs.  Every accumulator adds its
// elements in a fixed order, warps reduce with a fixed shuffle tree, and
// every CTA sums the CTAs' partials in the same order: deterministic.
// VM: the most basis vectors this instantiation handles (j + 1 <= VM); U:
// elements a thread works on at once.
template <class AR, int VM, int NT, int U, bool SM>
__global__ void __launch_bounds__(NT) k_arnoldi_cgs2(long long N, long long chunk, int j, int R, vec8 *w,
                                                     const vec8 *V, double *H, double *cs, double *sn, double *g,
                                                     double *est, vec8 *part, unsigned *bar, int *err,
                                                     double *status, int spin) {
    typedef typename AR::val val;
    typedef typename AR::acc acc;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ val s_w[NW][VM + 1];  // per-warp sums
    __shared__ double s_d[VM + 1];   // reduced values (binary64)
    __shared__ val s_c[VM];          // the current pass's coefficients, negated
    __shared__ int s_ok;
    const int nv = j + 1;
    const long long c0 = (long long)blockIdx.x * chunk;
    const long long c1 = c0 + chunk < N ? c0 + chunk : N;
    const int len = c1 > c0 ? (int)(c1 - c0) : 0;
    vec8 *ws = SM ? reinterpret_cast<vec8 *>(smem_raw) : w + c0;
    const vec8 *Vc = V + c0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (SM) {
        for (int e = threadIdx.x; e < len; e += NT) ws[e] = w[c0 + e];
        __syncthreads();
    }
    acc a[VM];
    acc an = AR::zero();
    // the CTA's sums of a[0..cnt) (and of an as value cnt when with_norm) into
    // part[base + i*grid + b]; after the grid barrier every CTA's totals in
    // s_d[0..cnt + with_norm); false on a timeout
    auto reduce = [&](int cnt, bool with_norm, long long base) -> bool {
        const int tot_n = cnt + (with_norm ? 1 : 0);
#pragma unroll
        for (int i = 0; i < VM + 1; ++i) {
            if (i >= tot_n) break;
            val v = (i < VM && i < cnt) ? AR::value(a[i < VM ? i : 0]) : AR::value(an);
            for (int d = 16; d > 0; d >>= 1) v = AR::add(v, AR::shfl_down(v, d));
            if (lane == 0) s_w[wid][i] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < tot_n; i += NT) {
            acc t = AR::zero();
            for (int q = 0; q < NW; ++q) AR::add_to(t, s_w[q][i]);
            AR::st(part + base + (long long)i * gridDim.x + blockIdx.x, AR::value(t));
        }
        if (!grid_sync(bar, err, &s_ok, spin)) return false;
        for (int i = wid; i < tot_n; i += NW) {
            const val tot = warp_sum_partials<AR>(part + base + (long long)i * gridDim.x, (int)gridDim.x);
            if (lane == 0) {
                double d = AR::to_double(tot);
                if (!isfinite(d)) {
                    if (blockIdx.x == 0) atomicOr(err, IRK_DEV_ERR_NONFINITE);
                    d = 0.0;
                }
                s_d[i] = d;
            }
        }
        __syncthreads();
        return true;
    };
    auto set_coefs = [&]() {
        for (int i = threadIdx.x; i < nv; i += NT) {
            const double d = s_d[i];
            const float hh = (float)d;
            s_c[i] = AR::neg(AR::coef(d, hh, (float)(d - (double)hh)));
        }
        __syncthreads();
    };
    // Each thread takes U elements at a time (e, e + NT, ...) and issues the
    // loads of all of them and all basis vectors before using any, so U (j+1)
    // loads are in flight per thread.
    // pass 1: h_i = <w, v_i>
#pragma unroll
    for (int i = 0; i < VM; ++i) a[i] = AR::zero();
    for (int e = threadIdx.x; e < len; e += U * NT) {
        val wv[U], v[U][VM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ee = e + u * NT;
            wv[u] = ee < len ? AR::ldv(ws + ee) : AR::from_float(0.f);
#pragma unroll
            for (int i = 0; i < VM; ++i)
                v[u][i] = (i < nv && ee < len) ? AR::ld(Vc + (long long)i * N + ee) : AR::from_float(0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < VM; ++i)
                if (i < nv && e + u * NT < len) AR::fma(a[i], wv[u], v[u][i]);
    }
    if (!reduce(nv, false, 0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) arnoldi_status(status, 0.0, 0.0, err);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int i = 0; i < nv; ++i) H[i * R + j] = s_d[i];
    set_coefs();
    // pass 2: w' = w - V h; q_i = <w', v_i>; ||w'||^2 (the basis values
    // loaded once serve both)
#pragma unroll
    for (int i = 0; i < VM; ++i) a[i] = AR::zero();
    for (int e = threadIdx.x; e < len; e += U * NT) {
        val wv[U], v[U][VM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ee = e + u * NT;
            wv[u] = ee < len ? AR::ldv(ws + ee) : AR::from_float(0.f);
#pragma unroll
            for (int i = 0; i < VM; ++i)
                v[u][i] = (i < nv && ee < len) ? AR::ld(Vc + (long long)i * N + ee) : AR::from_float(0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ee = e + u * NT;
            if (ee >= len) break;
            acc t = AR::zero();
            AR::add_to(t, wv[u]);
#pragma unroll
            for (int i = 0; i < VM; ++i)
                if (i < nv) AR::fma(t, s_c[i], v[u][i]);
            const val wn = AR::value(t);
            AR::st(ws + ee, wn);
#pragma unroll
            for (int i = 0; i < VM; ++i)
                if (i < nv) AR::fma(a[i], wn, v[u][i]);
            AR::fma(an, wn, wn);
        }
    }
    if (!reduce(nv, true, (long long)(VM + 1) * gridDim.x)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) arnoldi_status(status, 0.0, 0.0, err);
        return;
    }
    double qq = 0.0;
    for (int i = 0; i < nv; ++i) qq += s_d[i] * s_d[i];
    const double n2 = s_d[nv] - qq;
    const double hn = n2 > 0.0 ? sqrt(n2) : 0.0;
    const double inv = hn != 0.0 ? 1.0 / hn : 0.0;
    const float ih = (float)inv;
    const val iv = AR::coef(inv, ih, (float)(inv - (double)ih));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < nv; ++i) H[i * R + j] += s_d[i];
        H[(j + 1) * R + j] = hn;
    }
    set_coefs();
    // pass 3: v_{j+1} = (w' - V q) / h_{j+1,j}
    for (int e = threadIdx.x; e < len; e += U * NT) {
        val wv[U], v[U][VM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ee = e + u * NT;
            wv[u] = ee < len ? AR::ldv(ws + ee) : AR::from_float(0.f);
#pragma unroll
            for (int i = 0; i < VM; ++i)
                v[u][i] = (i < nv && ee < len) ? AR::ld(Vc + (long long)i * N + ee) : AR::from_float(0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int ee = e + u * NT;
            if (ee >= len) break;
            acc t = AR::zero();
            AR::add_to(t, wv[u]);
#pragma unroll
            for (int i = 0; i < VM; ++i)
                if (i < nv) AR::fma(t, s_c[i], v[u][i]);
            AR::st(w + c0 + ee, AR::mul(AR::value(t), iv));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        givens_col(j, R, H, cs, sn, g, est, err);
        arnoldi_status(status, *est, hn, err);
    }
}

// Launch shape of k_arnoldi: every CTA resident (cooperative launch).  Few
// large CTAs keep the grid barrier (one atomic per CTA on one counter) and
// the all-CTA reduction (every CTA reads every partial) short: one
// 1024-thread CTA per SM by default; irk_kernel_options.arnoldi_form = 2
// selects 256-thread CTAs, as many as fit.  At most IRK_PART_SLOTS / 2 CTAs
// (the partial buffer holds two steps).  grid 0: no cooperative launch.
struct ArnoldiShape {
    int grid = -1, threads = 0;
};

template <class AR>
static ArnoldiShape arnoldi_shape_for(int threads) {
    ArnoldiShape sh;
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sh.threads = threads;
    if (sh.threads == 256)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<AR, 256>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<AR, 1024>, 1024, 0);
    sh.grid = (coop && per_sm > 0) ? std::min(sms * per_sm, IRK_PART_SLOTS / 2) : 0;
    return sh;
}

static ArnoldiShape arnoldi_shape(irk_ctx *c) {
    static std::mutex mu;
    static ArnoldiShape cached[2][2];  // [arithmetic][256-thread CTAs]
    std::lock_guard<std::mutex> lk(mu);
    const int small = c->ko.arnoldi_form == 2 ? 1 : 0;
    ArnoldiShape &sh = cached[c->df ? 1 : 0][small];
    if (sh.grid < 0) sh = c->df ? arnoldi_shape_for<ArDF>(small ? 256 : 1024) : arnoldi_shape_for<ArF64>(small ? 256 : 1024);
    return sh;
}

// The whole Arnoldi step j (orthogonalisation, normalisation, Givens) in one
// launch; returns IRK_ERR_INVALID when the device cannot launch it (the
// caller then issues the step as separate launches).
// k_arnoldi_smem's launch, or false when its slices do not fit (or no
// cooperative launch): one 1024-thread CTA per SM, chunk = ceil(N / SMs).
static bool launch_arnoldi_smem(irk_ctx *c, int j, int restart, vec8 *w, int *rc) {
    if (c->ko.arnoldi_form != 0) return false;
    static std::mutex mu;
    static int sms = -1, optin = 0, coop = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (sms < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        }
    }
    if (!coop || sms <= 0 || sms * 2 > IRK_PART_SLOTS) return false;
    long long N = c->N;
    long long chunk = (N + sms - 1) / sms;
    chunk = (chunk + 1) / 2 * 2;  // even: 16-byte aligned slices
    const size_t smem = (size_t)chunk * sizeof(vec8);
    if (smem + 4096 > (size_t)optin) return false;
    const void *fn = c->df ? (const void *)k_arnoldi_smem<ArDF> : (const void *)k_arnoldi_smem<ArF64>;
    if (irk_allow_max_smem(fn)) return false;
    int jj = j, R = restart;
    const vec8 *V = c->d_V;
    Scal *slots = scal(c, 0);
    double *est = &scal(c, 1)->d;
    vec8 *part = reinterpret_cast<vec8 *>(c->d_part);
    double *status = irk_status_ptr(c);
    int spin = c->spin;
    void *args[] = {&N, &chunk, &jj, &R, &w, &V, &slots, &c->d_H, &c->d_cs, &c->d_sn, &c->d_g, &est, &part,
                    &c->d_gbar, &c->d_err, &status, &spin};
    *rc = cuda_status(cudaLaunchCooperativeKernel(fn, sms, 1024, args, smem, c->stream));
    c->launches++;
    return true;
}

// One CGS2 launch (k_arnoldi_cgs2): one CTA per SM, the w slice in shared
// memory when it fits; threads per CTA by the registers VM accumulators need.
// false when no cooperative launch is possible.
template <class AR, int VM, int NT, int U>
static bool launch_cgs2_vm(irk_ctx *c, int j, int restart, vec8 *w, int *rc) {
    static std::mutex mu;
    static int sms = -1, optin = 0, coop = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (sms < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        }
    }
    if (!coop || sms <= 0 || (long long)sms * 2 * (VM + 1) > IRK_PART_SLOTS) return false;
    long long N = c->N;
    long long chunk = (N + sms - 1) / sms;
    chunk = (chunk + 1) / 2 * 2;
    const size_t static_smem = sizeof(typename AR::val) * ((NT / 32) * (VM + 1) + VM) + 8 * (VM + 1) + 64;
    const bool fits = (size_t)chunk * sizeof(vec8) + static_smem + 1024 <= (size_t)optin;
    const void *fn = fits ? (const void *)k_arnoldi_cgs2<AR, VM, NT, U, true>
                          : (const void *)k_arnoldi_cgs2<AR, VM, NT, U, false>;
    const size_t smem = fits ? (size_t)chunk * sizeof(vec8) : 0;
    if (fits && irk_allow_max_smem(fn)) return false;
    int jj = j, R = restart, spin = c->spin;
    const vec8 *V = c->d_V;
    double *est = &scal(c, 1)->d;
    vec8 *part = reinterpret_cast<vec8 *>(c->d_part);
    double *status = irk_status_ptr(c);
    void *args[] = {&N, &chunk, &jj, &R, &w, &V, &c->d_H, &c->d_cs, &c->d_sn, &c->d_g, &est, &part, &c->d_gbar,
                    &c->d_err, &status, &spin};
    *rc = cuda_status(cudaLaunchCooperativeKernel(fn, sms, NT, args, smem, c->stream));
    c->launches++;
    return true;
}

template <class AR>
static bool launch_cgs2(irk_ctx *c, int j, int restart, vec8 *w, int *rc) {
    if (j + 1 <= 4) return launch_cgs2_vm<AR, 4, 1024, 4>(c, j, restart, w, rc);
    if (j + 1 <= 8) return launch_cgs2_vm<AR, 8, 512, 4>(c, j, restart, w, rc);
    if (j + 1 <= 16) return launch_cgs2_vm<AR, 16, 256, 2>(c, j, restart, w, rc);
    if (j + 1 <= 32) return launch_cgs2_vm<AR, 32, 256, 1>(c, j, restart, w, rc);
    return false;
}

int launch_arnoldi(irk_ctx *c, int j, int restart, vec8 *w) {
    int rc = IRK_OK;
    if (c->opt.orthogonalization == IRK_ORTHO_CGS2 &&
        (c->df ? launch_cgs2<ArDF>(c, j, restart, w, &rc) : launch_cgs2<ArF64>(c, j, restart, w, &rc)))
        return rc;
    if (launch_arnoldi_smem(c, j, restart, w, &rc)) return rc;
    const ArnoldiShape sh = arnoldi_shape(c);
    if (sh.grid <= 0) return IRK_ERR_INVALID;
    long long N = c->N;
    int jj = j, R = restart;
    const vec8 *V = c->d_V;
    Scal *slots = scal(c, 0);
    double *est = &scal(c, 1)->d;
    vec8 *part = reinterpret_cast<vec8 *>(c->d_part);
    double *status = irk_status_ptr(c);
    int spin = c->spin;
    void *args[] = {&N, &jj, &R, &w, &V, &slots, &c->d_H, &c->d_cs, &c->d_sn, &c->d_g, &est, &part, &c->d_gbar,
                    &c->d_err, &status, &spin};
    const void *fn;
    if (c->df)
        fn = sh.threads == 256 ? (const void *)k_arnoldi<ArDF, 256> : (const void *)k_arnoldi<ArDF, 1024>;
    else
        fn = sh.threads == 256 ? (const void *)k_arnoldi<ArF64, 256> : (const void *)k_arnoldi<ArF64, 1024>;
    const cudaError_t e = cudaLaunchCooperativeKernel(fn, sh.grid, sh.threads, args, 0, c->stream);
    c->launches++;
    return cuda_status(e);
}

int launch_lsq_update(irk_ctx *c, int jl, int restart) {
    k_backsolve<<<1, 32, 0, c->stream>>>(jl, restart, c->d_H, c->d_g, c->d_yls, scal(c, 64));
    c->launches++;
    int g = grid_stream(c->N);
    if (c->df)
        k_update_x<ArDF><<<g, 256, 0, c->stream>>>(c->N, jl, c->d_x, c->d_Z, scal(c, 64));
    else
        k_update_x<ArF64><<<g, 256, 0, c->stream>>>(c->N, jl, c->d_x, c->d_Z, scal(c, 64));
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_cycle_start(irk_ctx *c, int restart) {
    k_cycle_start<<<1, 64, 0, c->stream>>>(restart, scal(c, 0), c->d_g);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int launch_fill_zero(irk_ctx *c, vec8 *v, long long n) {
    k_zero<<<grid_stream(n), 256, 0, c->stream>>>(n, v);
    c->launches++;
    return cuda_status(cudaGetLastError());
}
