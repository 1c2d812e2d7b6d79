// group.cu -- the multi-request engine (irk_group_*, include/irk_gb300.h):
// many independent stage systems of one class (s, A, m, options) held in
// shared device pools and advanced together, one launch per phase:
//   - operator product of every request in one launch (k_g_matvec),
//   - one persistent cooperative sweep over the level-merged preconditioner
//     rows of every request (ilu_sweep_group, the kernel of k_ilu.cu),
//   - Gram-Schmidt with per-request deterministic reductions (k_g_axpy_dot),
//   - Givens rotations / least squares per request (one thread each).
// Each request runs restarted right-preconditioned FGMRES (Sec. 4) with its
// own inner iteration counter, so requests enter and leave between steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "arith.cuh"

namespace {

// First-fit allocator of integer ranges in [0, cap).
struct RangeAlloc {
    std::map<long long, long long> free_;  // start -> length
    void init(long long cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    long long alloc(long long n) {
        if (n <= 0) n = 1;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                long long s = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[s + n] = len - n;
                return s;
            }
        return -1;
    }
    void release(long long s, long long n) {
        if (s < 0) return;
        if (n <= 0) n = 1;
        auto it = free_.emplace(s, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// Scalar of one request (same layout as the single-request engine's).
struct GScal {
    double d;
    float hi, lo;
    double inv;
    float ihi, ilo;
};

__device__ __forceinline__ void gscal_store(GScal *s, double d) {
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

#define G_SLOTS 128  // per request: 0 = norm, 2 + i = h_{i,j}, 64 + i = y_i

// Per-request descriptor uploaded before every phase.
struct LaneDev {
    long long V, Z, X, B;  // vec8 offsets into the vector pool; V_k at V + k N
    long long N;           // s T m
    int e0;                // first element (global index)
    int j;                 // inner iteration of the current cycle
    int mv;                // operator role: 0 none, 1 V_{j+1} = B Z_j, 2 V_0 = b - B x
    int mgs;               // 1: Gram-Schmidt / Givens this step
    int res;               // 1: residual norm this step
    int upd;               // 1: least squares + x update this step
    int cyc;               // 1: starts a cycle (g = beta e_1, V_0 /= beta)
    int pad;
    KCoef mdt;  // -dt
};

struct GMatvec {
    int m, form;
    const int *elems;
    int n_elems;
    const int *lane_of_elem, *rp, *ci;
    const LaneDev *lanes;
    const vec8 *J, *M;
    vec8 *pool;
    KCoef C[IRK_MAX_S * IRK_MAX_S];
};

template <class AR, int S, int CH>
__device__ __forceinline__ void g_accum(typename AR::acc (&dst)[S], const vec8 *B, const vec8 *x, int m) {
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
        for (int u = 0; u < CH; ++u) {
#pragma unroll
            for (int l = 0; l < S; ++l) AR::fma(dst[l], bv[u], xv[l][u]);
            // the single-request product's fold points: after every eighth
            // column of a block and after its last column
            const int c = c0 + u;
            if (c < m && ((c & 7) == 7 || c == m - 1))
#pragma unroll
                for (int l = 0; l < S; ++l) AR::renorm(dst[l]);
        }
    }
}

// Operator product of every request (Sec. 4.1, eq. big-irk), element rows of
// all requests in one launch; same arithmetic as k_matvec per row.
template <class AR, int S, int CH>
__global__ void __launch_bounds__(256) k_g_matvec(GMatvec P) {
    typedef typename AR::val val;
    typedef typename AR::acc acc;
    const int m = P.m;
    const int groups = blockDim.x / m;
    const int g = threadIdx.x / m, a = threadIdx.x - g * m;
    if (g >= groups) return;
    const long long mm = (long long)m * m, sm = (long long)S * m;
    for (long long idx = (long long)blockIdx.x * groups + g; idx < P.n_elems; idx += (long long)gridDim.x * groups) {
        const int e = P.elems[idx];
        const LaneDev L = P.lanes[P.lane_of_elem[e]];
        if (L.mv == 0) continue;
        const vec8 *x = P.pool + (L.mv == 1 ? L.Z + (long long)L.j * L.N : L.X);
        vec8 *y = P.pool + (L.mv == 1 ? L.V + (long long)(L.j + 1) * L.N : L.V);
        const vec8 *rhs = P.pool + L.B;
        const long long off = (long long)(e - L.e0) * sm;
        acc t[S], z[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
            t[l] = AR::zero();
            z[l] = AR::zero();
        }
        for (int p = P.rp[e]; p < P.rp[e + 1]; ++p)
            g_accum<AR, S, CH>(t, P.J + (long long)p * mm + a, x + (long long)(P.ci[p] - L.e0) * sm, m);
        g_accum<AR, S, CH>(z, P.M + (long long)e * mm + a, x + off, m);
        val tv[S], zv[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
            tv[l] = AR::value(t[l]);
            zv[l] = AR::value(z[l]);
        }
        const val mdt = AR::coef(L.mdt.d, L.mdt.hi, L.mdt.lo);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            acc o = AR::zero();
#pragma unroll
            for (int l = 0; l < S; ++l) {
                const KCoef &cc = P.C[k * S + l];
                AR::fma(o, AR::coef(cc.d, cc.hi, cc.lo), zv[l]);
            }
            AR::fma(o, mdt, tv[k]);
            val out = AR::value(o);
            if (L.mv == 2) out = AR::sub(AR::ld(rhs + off + k * m + a), out);
            AR::st(y + off + k * m + a, out);
        }
    }
}

template <class AR>
__device__ __forceinline__ typename AR::val g_block_reduce(typename AR::val v, typename AR::val *sh) {
    for (int d = 16; d > 0; d >>= 1) v = AR::add(v, AR::shfl_down(v, d));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        v = lane < nw ? sh[lane] : AR::from_float(0.f);
        for (int d = 16; d > 0; d >>= 1) v = AR::add(v, AR::shfl_down(v, d));
    }
    return v;
}

// Work unit of the segmented vector kernels: a chunk of one request's vector.
struct Unit {
    int lane, start, len, pad;
};

struct GRed {
    const Unit *units;
    const int *lane_u0, *lane_nu;  // units of each lane: [u0, u0 + nu)
    const LaneDev *lanes;
    vec8 *pool;
    vec8 *part;
    unsigned *tickets;
    GScal *scal;  // G_SLOTS per lane
    double *H;    // (R+1) x R per lane
    double *hn;   // per lane: last h_{j+1,j} / norm
    int R, step, mode;  // mode 0: Gram-Schmidt step `step`; 1: residual norm of V_0
    int *err;
};

// mode 0, request at inner iteration j, step i:
//   i <= j : w = V_{j+1} - h_{i-1,j} V_{i-1} (i > 0); h_{i,j} = <w, V_i>
//   i == j+1: w = V_{j+1} - h_{j,j} V_j;         h_{j+1,j} = ||w||
//   i >  j+1: nothing.
// mode 1: slot 0 = ||V_0||.  One CTA per unit; per-request deterministic
// reduction by the last unit of the request.
template <class AR>
__global__ void __launch_bounds__(256) k_g_axpy_dot(GRed G) {
    typedef typename AR::val val;
    __shared__ val sh[32];
    __shared__ int s_last;
    const Unit U = G.units[blockIdx.x];
    const LaneDev L = G.lanes[U.lane];
    const int i = G.step;
    if (G.mode == 0 ? (!L.mgs || i > L.j + 1) : !L.res) return;  // uniform per CTA
    GScal *sc = G.scal + (long long)U.lane * G_SLOTS;
    vec8 *w;
    const vec8 *vprev = nullptr, *v = nullptr;
    int hprev_slot = 0, out_slot, take_sqrt = 0;
    if (G.mode == 1) {
        w = G.pool + L.V;
        out_slot = 0;
        take_sqrt = 1;
    } else {
        w = G.pool + L.V + (long long)(L.j + 1) * L.N;
        if (i <= L.j) {
            if (i > 0) {
                vprev = G.pool + L.V + (long long)(i - 1) * L.N;
                hprev_slot = 2 + i - 1;
            }
            v = G.pool + L.V + (long long)i * L.N;
            out_slot = 2 + i;
        } else {
            vprev = G.pool + L.V + (long long)L.j * L.N;
            hprev_slot = 2 + L.j;
            out_slot = 2 + L.j + 1;
            take_sqrt = 1;
        }
    }
    val nh = AR::from_float(0.f);
    if (vprev) nh = AR::neg(AR::coef(sc[hprev_slot].d, sc[hprev_slot].hi, sc[hprev_slot].lo));
    typename AR::acc acc = AR::zero();
    for (int e = U.start + threadIdx.x; e < U.start + U.len; e += blockDim.x) {
        val wv = AR::ld(w + e);
        if (vprev) {
            wv = AR::add(wv, AR::mul(nh, AR::ld(vprev + e)));
            AR::st(w + e, wv);
        }
        AR::fma(acc, wv, v ? AR::ld(v + e) : wv);
    }
    val r = g_block_reduce<AR>(AR::value(acc), sh);
    if (threadIdx.x == 0) {
        AR::st(G.part + blockIdx.x, r);
        __threadfence();
        unsigned t = atomicAdd(G.tickets + U.lane, 1u);
        s_last = (t == (unsigned)G.lane_nu[U.lane] - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int u0 = G.lane_u0[U.lane], nu = G.lane_nu[U.lane];
    typename AR::acc a2 = AR::zero();
    for (int q = threadIdx.x; q < nu; q += blockDim.x) AR::add_to(a2, AR::ldcg(G.part + u0 + q));
    __syncthreads();
    val tot = g_block_reduce<AR>(AR::value(a2), sh);
    if (threadIdx.x == 0) {
        double d = AR::to_double(tot);
        if (!isfinite(d)) {
            atomicOr(G.err, IRK_DEV_ERR_NONFINITE);
            d = 0.0;
        }
        if (take_sqrt) d = d > 0.0 ? sqrt(d) : 0.0;
        gscal_store(sc + out_slot, d);
        if (G.mode == 0) {
            double *H = G.H + (long long)U.lane * (G.R + 1) * G.R;
            const int row = (i <= L.j) ? i : L.j + 1;
            H[row * G.R + L.j] = d;
            if (i == L.j + 1) G.hn[U.lane] = d;
        } else {
            G.hn[U.lane] = d;
        }
        G.tickets[U.lane] = 0u;
    }
}

// mode 0: V_{j+1} /= h_{j+1,j} (requests with mgs); mode 1: V_0 /= beta
// (requests starting a cycle); mode 2: Z_j = V_j (no preconditioner);
// mode 3: x += sum_{i<=j} y_i Z_i (requests with upd).
template <class AR>
__global__ void __launch_bounds__(256) k_g_vec(const Unit *units, const LaneDev *lanes, vec8 *pool, const GScal *scal,
                                               int mode) {
    typedef typename AR::val val;
    const Unit U = units[blockIdx.x];
    const LaneDev L = lanes[U.lane];
    const GScal *sc = scal + (long long)U.lane * G_SLOTS;
    if (mode == 0 && L.mgs) {
        const GScal &h = sc[2 + L.j + 1];
        const val inv = AR::coef(h.inv, h.ihi, h.ilo);
        vec8 *w = pool + L.V + (long long)(L.j + 1) * L.N;
        for (int e = U.start + threadIdx.x; e < U.start + U.len; e += blockDim.x) AR::st(w + e, AR::mul(AR::ld(w + e), inv));
    } else if (mode == 1 && L.cyc) {
        const val inv = AR::coef(sc[0].inv, sc[0].ihi, sc[0].ilo);
        vec8 *w = pool + L.V;
        for (int e = U.start + threadIdx.x; e < U.start + U.len; e += blockDim.x) AR::st(w + e, AR::mul(AR::ld(w + e), inv));
    } else if (mode == 2 && L.mgs) {
        const vec8 *src = pool + L.V + (long long)L.j * L.N;
        vec8 *dst = pool + L.Z + (long long)L.j * L.N;
        for (int e = U.start + threadIdx.x; e < U.start + U.len; e += blockDim.x) dst[e] = src[e];
    } else if (mode == 3 && L.upd) {
        vec8 *x = pool + L.X;
        for (int e = U.start + threadIdx.x; e < U.start + U.len; e += blockDim.x) {
            typename AR::acc acc = AR::zero();
            AR::add_to(acc, AR::ld(x + e));
            for (int q = 0; q <= L.j; ++q) {
                const GScal &y = sc[64 + q];
                AR::fma(acc, AR::coef(y.d, y.hi, y.lo), AR::ld(pool + L.Z + (long long)q * L.N + e));
            }
            AR::st(x + e, AR::value(acc));
        }
    }
}

// One thread per request: Givens step on column j (mgs), cycle start (cyc:
// g = beta e_1), least squares (upd: y = H^{-1} g over columns 0..j).
__global__ void k_g_scalar(int nl, int R, const LaneDev *lanes, GScal *scal, double *H, double *cs, double *sn,
                           double *g, double *ybuf, double *est, int phase, int *err) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const LaneDev L = lanes[l];
    double *Hl = H + (long long)l * (R + 1) * R, *csl = cs + (long long)l * R, *snl = sn + (long long)l * R;
    double *gl = g + (long long)l * (R + 1), *yl = ybuf + (long long)l * R;
    GScal *sc = scal + (long long)l * G_SLOTS;
    if (phase == 0 && L.cyc) {
        for (int q = 0; q <= R; ++q) gl[q] = (q == 0) ? sc[0].d : 0.0;
    } else if (phase == 1 && L.mgs) {
        const int j = L.j;
        for (int i = 0; i < j; ++i) {
            double a = Hl[i * R + j], b = Hl[(i + 1) * R + j];
            Hl[i * R + j] = csl[i] * a + snl[i] * b;
            Hl[(i + 1) * R + j] = -snl[i] * a + csl[i] * b;
        }
        double a = Hl[j * R + j], b = Hl[(j + 1) * R + j];
        double rho = hypot(a, b);
        if (!isfinite(rho)) {
            atomicOr(err, IRK_DEV_ERR_NONFINITE);
            est[l] = 0.0;
            return;
        }
        double c = rho == 0.0 ? 1.0 : a / rho, s = rho == 0.0 ? 0.0 : b / rho;
        csl[j] = c;
        snl[j] = s;
        Hl[j * R + j] = rho;
        Hl[(j + 1) * R + j] = 0.0;
        gl[j + 1] = -s * gl[j];
        gl[j] = c * gl[j];
        est[l] = fabs(gl[j + 1]);
    } else if (phase == 2 && L.upd) {
        const int jl = L.j;
        for (int i = jl; i >= 0; --i) {
            double acc = gl[i];
            for (int k = i + 1; k <= jl; ++k) acc -= Hl[i * R + k] * yl[k];
            double d = Hl[i * R + i];
            yl[i] = d != 0.0 ? acc / d : 0.0;
            gscal_store(sc + 64 + i, yl[i]);
        }
    }
}

// Layout conversions of one request (stage-major binary64 <-> the request's
// element-interleaved vec8 vector) and block conversion into the pools.
template <class AR>
__global__ void k_g_in(long long N, int T, int m, int s, const double *__restrict__ src, vec8 *dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        long long a = e % m, r = e / m, k = r % s, i = r / s;
        AR::st(dst + e, AR::from_double(src[(k * T + i) * m + a]));
    }
}

template <class AR>
__global__ void k_g_out(long long N, int T, int m, int s, const vec8 *__restrict__ src, double *dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        long long a = e % m, r = e / m, k = r % s, i = r / s;
        dst[(k * T + i) * m + a] = AR::to_double(AR::ld(src + e));
    }
}

template <class AR>
__global__ void k_g_blocks(long long total, int m, const double *__restrict__ src, vec8 *dst) {
    const long long mm = (long long)m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        long long blk = e / mm, r = e - blk * mm, c = r / m, a = r - c * m;
        AR::st(dst + e, AR::from_double(src[blk * mm + a * m + c]));
    }
}

int g_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)std::max(1LL, g);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side.
namespace {

enum LaneState { L_FREE = 0, L_RESID = 1, L_ITER = 2, L_DONE = 3 };

struct Lane {
    int state = L_FREE;
    int T = 0, nnzb = 0;
    long long N = 0;
    long long e0 = -1, b0 = -1, r0 = -1, pb0 = -1, vo = -1, wo = -1, uo = -1;  // pool offsets
    long long n_e = 0, n_b = 0, n_r = 0, n_pb = 0, n_v = 0, n_w = 0, n_u = 0;  // their sizes
    int npb = 0;                  // preconditioner blocks actually used
    int max_item_blocks = 1;
    std::vector<std::vector<int>> lo_lv, up_lv;  // preconditioner rows (global) per level
    double dt = 0.0, rtol = 0.0, bnorm = -1.0, beta = 0.0, est = 0.0;
    int j = 0, total = 0, cycles = 0, status = IRK_OK;
    bool first = true;
};

}  // namespace

struct irk_group {
    int dev = 0;
    cudaStream_t stream = nullptr;
    irk_options opt;
    int s = 0, m = 0, R = 30, df = 0, fprec = IRK_FACTOR_FP32, pc = IRK_PC_UNCOUPLED;
    double A[IRK_MAX_S * IRK_MAX_S], Ainv[IRK_MAX_S * IRK_MAX_S], shift[IRK_MAX_S];
    long long Ecap = 0, Bcap = 0;
    int Lmax = 0;
    // pools and allocators
    RangeAlloc a_e, a_b, a_r, a_pb, a_v, a_w, a_u;
    int *d_rp = nullptr, *d_ci = nullptr, *d_lane_of_elem = nullptr;
    vec8 *d_J = nullptr, *d_M = nullptr, *d_pool = nullptr;
    unsigned long long *d_ll = nullptr;
    int *d_prp = nullptr, *d_pci = nullptr, *d_pdiag = nullptr, *d_pvoff = nullptr, *d_lane_of_prow = nullptr;
    AsmEntry *d_asm = nullptr;
    int *d_upd_ptr = nullptr, *d_upd = nullptr, *d_rows = nullptr, *d_lo = nullptr, *d_up = nullptr;
    void *d_vals = nullptr, *d_dinv = nullptr;
    int *d_elems = nullptr;
    Unit *d_units = nullptr;
    int *d_lane_u0 = nullptr, *d_lane_nu = nullptr;
    vec8 *d_part = nullptr;
    unsigned *d_tickets = nullptr;
    GScal *d_scal = nullptr;
    double *d_H = nullptr, *d_cs = nullptr, *d_sn = nullptr, *d_g = nullptr, *d_y = nullptr, *d_est = nullptr,
           *d_hn = nullptr;
    LaneDev *d_lanes = nullptr;
    long long *d_sw = nullptr;  // sweep bases: vin, zout, yll, zll (4 x Lmax)
    int *d_err = nullptr;
    // host mirrors
    std::vector<Lane> lanes;
    LaneDev *h_lanes = nullptr;  // pinned
    double *h_out = nullptr;     // pinned: est, hn (2 Lmax)
    long long *h_sw = nullptr;   // pinned
    int *h_err = nullptr;        // pinned
    bool dirty = true;           // membership changed: rebuild work lists
    int n_elems = 0, n_units = 0, n_items = 0, max_item_blocks = 1;
    long long unit_cap = 0, bytes = 0;
    int epoch = 0;
};

namespace {

int g_status(cudaError_t e) { return cuda_status(e); }

template <class Tv>
int g_malloc(irk_group *g, Tv **p, long long count) {
    size_t bytes = (size_t)std::max(1LL, count) * sizeof(Tv);
    if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return IRK_ERR_NOMEM;
    }
    g->bytes += (long long)bytes;
    return IRK_OK;
}

void g_free_all(irk_group *g) {
    void *ptrs[] = {g->d_rp, g->d_ci, g->d_lane_of_elem, g->d_J, g->d_M, g->d_pool, g->d_ll, g->d_prp, g->d_pci,
                    g->d_pdiag, g->d_pvoff, g->d_lane_of_prow, g->d_asm, g->d_upd_ptr, g->d_upd, g->d_rows,
                    g->d_lo, g->d_up, g->d_vals, g->d_dinv, g->d_elems, g->d_units, g->d_lane_u0, g->d_lane_nu,
                    g->d_part, g->d_tickets, g->d_scal, g->d_H, g->d_cs, g->d_sn, g->d_g, g->d_y, g->d_est,
                    g->d_hn, g->d_lanes, g->d_sw, g->d_err};
    for (void *p : ptrs) cudaFree(p);
    if (g->h_lanes) cudaFreeHost(g->h_lanes);
    if (g->h_out) cudaFreeHost(g->h_out);
    if (g->h_sw) cudaFreeHost(g->h_sw);
    if (g->h_err) cudaFreeHost(g->h_err);
}

const long long UNIT = 16384;  // values per unit of the segmented kernels

// Release every pool range of a lane.
void lane_release(irk_group *g, Lane &L) {
    g->a_e.release(L.e0, L.n_e);
    g->a_b.release(L.b0, L.n_b);
    g->a_r.release(L.r0, L.n_r);
    g->a_pb.release(L.pb0, L.n_pb);
    g->a_v.release(L.vo, L.n_v);
    g->a_w.release(L.wo, L.n_w);
    g->a_u.release(L.uo, L.n_u);
    L = Lane();
    g->dirty = true;
}

// Rebuild the work lists (active elements, units, level-merged sweep rows)
// after requests entered or left.
int rebuild_lists(irk_group *g) {
    std::vector<int> elems, lane_u0(g->Lmax, 0), lane_nu(g->Lmax, 0);
    std::vector<Unit> units;
    std::vector<int> lo, up;
    int maxlv = 0;
    g->max_item_blocks = 1;
    for (int l = 0; l < g->Lmax; ++l) {
        Lane &L = g->lanes[l];
        if (L.state == L_FREE || L.state == L_DONE) continue;
        for (int i = 0; i < L.T; ++i) elems.push_back((int)L.e0 + i);
        lane_u0[l] = (int)units.size();
        for (long long st = 0; st < L.N; st += UNIT) units.push_back(Unit{l, (int)st, (int)std::min(UNIT, L.N - st), 0});
        lane_nu[l] = (int)units.size() - lane_u0[l];
        maxlv = std::max(maxlv, (int)std::max(L.lo_lv.size(), L.up_lv.size()));
        g->max_item_blocks = std::max(g->max_item_blocks, L.max_item_blocks);
    }
    for (int lv = 0; lv < maxlv; ++lv)
        for (int l = 0; l < g->Lmax; ++l) {
            Lane &L = g->lanes[l];
            if (L.state == L_FREE || L.state == L_DONE) continue;
            if (lv < (int)L.lo_lv.size()) lo.insert(lo.end(), L.lo_lv[lv].begin(), L.lo_lv[lv].end());
            if (lv < (int)L.up_lv.size()) up.insert(up.end(), L.up_lv[lv].begin(), L.up_lv[lv].end());
        }
    if ((long long)units.size() > g->unit_cap) return IRK_ERR_NOMEM;
    g->n_elems = (int)elems.size();
    g->n_units = (int)units.size();
    g->n_items = (int)lo.size();
    cudaStream_t st = g->stream;
    if (!elems.empty() && cudaMemcpyAsync(g->d_elems, elems.data(), elems.size() * 4, cudaMemcpyHostToDevice, st))
        return IRK_ERR_CUDA;
    if (!units.empty() &&
        cudaMemcpyAsync(g->d_units, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice, st))
        return IRK_ERR_CUDA;
    if (cudaMemcpyAsync(g->d_lane_u0, lane_u0.data(), g->Lmax * 4, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(g->d_lane_nu, lane_nu.data(), g->Lmax * 4, cudaMemcpyHostToDevice, st))
        return IRK_ERR_CUDA;
    if (!lo.empty() && (cudaMemcpyAsync(g->d_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, st) ||
                        cudaMemcpyAsync(g->d_up, up.data(), up.size() * 4, cudaMemcpyHostToDevice, st)))
        return IRK_ERR_CUDA;
    // the host vectors above die at return: wait for the copies
    if (cudaStreamSynchronize(st) != cudaSuccess) return IRK_ERR_CUDA;
    g->dirty = false;
    return IRK_OK;
}

void fill_lane_dev(irk_group *g) {
    for (int l = 0; l < g->Lmax; ++l) {
        const Lane &L = g->lanes[l];
        LaneDev &D = g->h_lanes[l];
        memset(&D, 0, sizeof(D));
        if (L.state == L_FREE) continue;
        const long long N = L.N;
        D.V = L.vo;
        D.Z = L.vo + (long long)(g->R + 1) * N;
        D.X = D.Z + (long long)g->R * N;
        D.B = D.X + N;
        D.N = N;
        D.e0 = (int)L.e0;
        D.j = L.j;
        D.mdt = make_kcoef(-L.dt);
    }
}

int upload_lanes(irk_group *g) {
    return g_status(
        cudaMemcpyAsync(g->d_lanes, g->h_lanes, sizeof(LaneDev) * g->Lmax, cudaMemcpyHostToDevice, g->stream));
}

int sync_group(irk_group *g) {
    if (cudaMemcpyAsync(g->h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return IRK_ERR_CUDA;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return IRK_ERR_CUDA;
    int e = *g->h_err;
    if (e & IRK_DEV_ERR_SINGULAR) return IRK_ERR_SINGULAR;
    if (e & IRK_DEV_ERR_NONFINITE) return IRK_ERR_NONFINITE;
    if (e & IRK_DEV_ERR_TIMEOUT) return IRK_ERR_TIMEOUT;
    return IRK_OK;
}

// Launch shapes of the group operator product: (columns of loads in flight
// per thread, threads per CTA).  Every shape accumulates in the same order
// (columns ascending, the same fold points), so all give the same bits; the
// fastest per (m, s, arithmetic) is picked by timing them on a group's first
// product (the product only writes its output, so repeating it is harmless)
// and kept for the process.
struct GMvShape {
    int ch, threads;
};
const GMvShape kGMvShapes[] = {{8, 256}, {4, 256}, {2, 256}, {8, 128}, {4, 128}};
const int kNumGMvShapes = 5;
std::mutex g_gmv_mu;
std::map<long long, int> g_gmv_choice;

template <class AR, int S>
void run_g_matvec_shape(irk_group *g, const GMatvec &P, int v) {
    const GMvShape sh = kGMvShapes[v];
    const int groups = std::max(1, sh.threads / g->m);
    const int threads = (groups * g->m + 31) / 32 * 32;
    long long grid = (g->n_elems + groups - 1) / groups;
    if (grid < 1) grid = 1;
    if (sh.ch == 8)
        k_g_matvec<AR, S, 8><<<(int)grid, threads, 0, g->stream>>>(P);
    else if (sh.ch == 4)
        k_g_matvec<AR, S, 4><<<(int)grid, threads, 0, g->stream>>>(P);
    else
        k_g_matvec<AR, S, 2><<<(int)grid, threads, 0, g->stream>>>(P);
}

template <class AR, int S>
void launch_g_matvec_s(irk_group *g, GMatvec &P) {
    const long long key = ((long long)g->m << 20) | ((long long)S << 4) | g->df;
    int v = -1;
    {
        std::lock_guard<std::mutex> lk(g_gmv_mu);
        auto it = g_gmv_choice.find(key);
        if (it != g_gmv_choice.end()) v = it->second;
    }
    if (v < 0 && g->n_elems >= 256) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int q = 0; q < kNumGMvShapes; ++q) {
            if (kGMvShapes[q].threads < g->m) continue;
            float t[3] = {1e30f, 1e30f, 1e30f};
            bool launched = true;
            for (int rep = 0; rep < 4 && launched; ++rep) {
                cudaEventRecord(e0, g->stream);
                run_g_matvec_shape<AR, S>(g, P, q);
                launched = cudaGetLastError() == cudaSuccess;  // a shape that cannot launch is skipped
                cudaEventRecord(e1, g->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && launched) t[rep - 1] = ms;
            }
            std::sort(t, t + 3);
            if (t[1] < best) {
                best = t[1];
                v = q;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(g_gmv_mu);
        g_gmv_choice[key] = v;
    }
    if (v < 0) v = S <= 3 ? 0 : 1;  // small groups before a choice: the former default
    run_g_matvec_shape<AR, S>(g, P, v);
}

template <class AR>
void launch_g_matvec_ar(irk_group *g, GMatvec &P) {
    switch (g->s) {
        case 1: launch_g_matvec_s<AR, 1>(g, P); break;
        case 2: launch_g_matvec_s<AR, 2>(g, P); break;
        case 3: launch_g_matvec_s<AR, 3>(g, P); break;
        case 4: launch_g_matvec_s<AR, 4>(g, P); break;
        case 5: launch_g_matvec_s<AR, 5>(g, P); break;
        case 6: launch_g_matvec_s<AR, 6>(g, P); break;
        case 7: launch_g_matvec_s<AR, 7>(g, P); break;
        default: launch_g_matvec_s<AR, 8>(g, P); break;
    }
}

int launch_g_matvec(irk_group *g) {
    if (g->n_elems == 0) return IRK_OK;
    GMatvec P;
    P.m = g->m;
    P.form = IRK_TRANSFORMED;
    P.elems = g->d_elems;
    P.n_elems = g->n_elems;
    P.lane_of_elem = g->d_lane_of_elem;
    P.rp = g->d_rp;
    P.ci = g->d_ci;
    P.lanes = g->d_lanes;
    P.J = g->d_J;
    P.M = g->d_M;
    P.pool = g->d_pool;
    for (int q = 0; q < g->s * g->s; ++q) P.C[q] = make_kcoef(g->Ainv[q]);
    if (g->df)
        launch_g_matvec_ar<ArDF>(g, P);
    else
        launch_g_matvec_ar<ArF64>(g, P);
    return g_status(cudaGetLastError());
}

int launch_g_red(irk_group *g, int step, int mode) {
    if (g->n_units == 0) return IRK_OK;
    GRed G;
    G.units = g->d_units;
    G.lane_u0 = g->d_lane_u0;
    G.lane_nu = g->d_lane_nu;
    G.lanes = g->d_lanes;
    G.pool = g->d_pool;
    G.part = g->d_part;
    G.tickets = g->d_tickets;
    G.scal = g->d_scal;
    G.H = g->d_H;
    G.hn = g->d_hn;
    G.R = g->R;
    G.step = step;
    G.mode = mode;
    G.err = g->d_err;
    if (g->df)
        k_g_axpy_dot<ArDF><<<g->n_units, 256, 0, g->stream>>>(G);
    else
        k_g_axpy_dot<ArF64><<<g->n_units, 256, 0, g->stream>>>(G);
    return g_status(cudaGetLastError());
}

int launch_g_vec(irk_group *g, int mode) {
    if (g->n_units == 0) return IRK_OK;
    if (g->df)
        k_g_vec<ArDF><<<g->n_units, 256, 0, g->stream>>>(g->d_units, g->d_lanes, g->d_pool, g->d_scal, mode);
    else
        k_g_vec<ArF64><<<g->n_units, 256, 0, g->stream>>>(g->d_units, g->d_lanes, g->d_pool, g->d_scal, mode);
    return g_status(cudaGetLastError());
}

int launch_g_scalar(irk_group *g, int phase) {
    k_g_scalar<<<(g->Lmax + 127) / 128, 128, 0, g->stream>>>(g->Lmax, g->R, g->d_lanes, g->d_scal, g->d_H, g->d_cs,
                                                             g->d_sn, g->d_g, g->d_y, g->d_est, phase, g->d_err);
    return g_status(cudaGetLastError());
}

int launch_g_sweep(irk_group *g) {
    if (g->pc == IRK_PC_NONE) return launch_g_vec(g, 2);
    if (g->n_items == 0) return IRK_OK;
    // per-lane bases: V_j in, Z_j out, published words
    const int Lm = g->Lmax;
    long long *vin = g->h_sw, *zout = g->h_sw + Lm, *yll = g->h_sw + 2 * Lm, *zll = g->h_sw + 3 * Lm;
    const long long w = (g->fprec == IRK_FACTOR_FP64) ? 2 : 1;
    for (int l = 0; l < Lm; ++l) {
        const Lane &L = g->lanes[l];
        const LaneDev &D = g->h_lanes[l];
        if (L.state == L_FREE || !D.mgs) {
            vin[l] = -1;
            zout[l] = yll[l] = zll[l] = 0;
            continue;
        }
        vin[l] = D.V + (long long)D.j * D.N;
        zout[l] = D.Z + (long long)D.j * D.N;
        yll[l] = L.wo;
        zll[l] = L.wo + L.N * w;
    }
    if (cudaMemcpyAsync(g->d_sw, g->h_sw, sizeof(long long) * 4 * Lm, cudaMemcpyHostToDevice, g->stream))
        return IRK_ERR_CUDA;
    return ilu_sweep_group(g->stream, g->dev, g->fprec, g->df, g->n_items, g->m, g->max_item_blocks, g->d_lo,
                           g->d_up, g->d_prp, g->d_pci, g->d_pvoff, g->d_vals, g->d_dinv, g->d_pool, g->d_ll,
                           ++g->epoch, g->d_err, g->d_lane_of_prow, g->d_sw, g->d_sw + Lm, g->d_sw + 2 * Lm,
                           g->d_sw + 3 * Lm, g->opt.spin_limit > 0 ? g->opt.spin_limit : IRK_DEFAULT_SPIN_LIMIT);
}

}  // namespace

namespace {

// Radau IIA by collocation and small inverse live in api.cu; the group keeps
// its own copy of the tableau through these (declared there).
}  // namespace

bool irk_radau_iia_tableau(int s, double *A);
bool irk_invert_small(int n, const double *A, double *X);

namespace {

// Build one request's preconditioner pattern (stage-uncoupled, Sec. 4.3.2) in
// the group's global numbering: rows r0 + k T + q (q-th eliminated element),
// blocks at local positions (offset by pb0 at upload).  Mirrors the
// single-request construction in k_ilu.cu.
struct LanePattern {
    std::vector<int> rp, ci, diag, voff, upd_ptr, upd;
    std::vector<AsmEntry> asmv;
};

void build_lane_pattern(const irk_group *g, const std::vector<int> &rp, const std::vector<int> &ci, int T,
                        long long e0, long long b0, long long r0, LanePattern &P, Lane &L) {
    const int s = g->s, m = g->m;
    std::vector<int> perm(T), inv(T);
    for (int q = 0; q < T; ++q) perm[q] = q;
    if (g->opt.ordering == IRK_ORDER_MULTICOLOR) {
        std::vector<int> colour(T, -1);
        std::vector<char> used;
        for (int i = 0; i < T; ++i) {
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
    P.rp.assign(1, 0);
    std::vector<std::pair<int, int>> nb;
    for (int k = 0; k < s; ++k)
        for (int q = 0; q < T; ++q) {
            const int e = perm[q];
            nb.clear();
            for (int p = rp[e]; p < rp[e + 1]; ++p) nb.push_back(std::make_pair(inv[ci[p]], p));
            std::sort(nb.begin(), nb.end());
            for (const auto &x : nb) {
                const int p = x.second, j = ci[p];
                P.ci.push_back((int)r0 + k * T + x.first);
                P.asmv.push_back(AsmEntry{(int)b0 + p, j == e ? (int)e0 + e : -1, k * s + k, 0});
            }
            P.rp.push_back((int)P.ci.size());
            P.voff.push_back((e * s + k) * m);
        }
    const int nr = s * T;
    auto local_row = [&](int R) { return R - (int)r0; };
    // diagonal positions, IKJ update lists, levels (local rows -> global)
    P.diag.assign(nr, -1);
    for (int R = 0; R < nr; ++R)
        for (int p = P.rp[R]; p < P.rp[R + 1]; ++p)
            if (local_row(P.ci[p]) == R) P.diag[R] = p;
    P.upd_ptr.assign(P.ci.size() + 1, 0);
    P.upd.clear();
    for (int R = 0; R < nr; ++R)
        for (int p = P.rp[R]; p < P.rp[R + 1]; ++p) {
            P.upd_ptr[p] = (int)(P.upd.size() / 2);
            const int i = local_row(P.ci[p]);
            if (i < R)
                for (int q = p + 1; q < P.rp[R + 1]; ++q) {
                    const int col = P.ci[q];
                    const int *b = P.ci.data() + P.rp[i], *en = P.ci.data() + P.rp[i + 1];
                    const int *f = std::lower_bound(b, en, col);
                    if (f != en && *f == col) {
                        P.upd.push_back(q);
                        P.upd.push_back((int)(f - P.ci.data()));
                    }
                }
        }
    P.upd_ptr[P.ci.size()] = (int)(P.upd.size() / 2);
    std::vector<int> lev(nr, 0);
    int maxl = 0;
    L.max_item_blocks = 1;
    for (int R = 0; R < nr; ++R) {
        int l = 0, lower = 0, upper = 0;
        for (int p = P.rp[R]; p < P.rp[R + 1]; ++p) {
            const int c = local_row(P.ci[p]);
            if (c < R) {
                l = std::max(l, lev[c] + 1);
                ++lower;
            }
            if (c > R) ++upper;
        }
        lev[R] = l;
        maxl = std::max(maxl, l);
        L.max_item_blocks = std::max(L.max_item_blocks, std::max(lower, upper + 1));
    }
    L.lo_lv.assign(maxl + 1, std::vector<int>());
    for (int R = 0; R < nr; ++R) L.lo_lv[lev[R]].push_back((int)r0 + R);
    std::vector<int> ulev(nr, 0);
    int maxu = 0;
    for (int R = nr - 1; R >= 0; --R) {
        int l = 0;
        for (int p = P.rp[R]; p < P.rp[R + 1]; ++p) {
            const int c = local_row(P.ci[p]);
            if (c > R) l = std::max(l, ulev[c] + 1);
        }
        ulev[R] = l;
        maxu = std::max(maxu, l);
    }
    L.up_lv.assign(maxu + 1, std::vector<int>());
    for (int R = nr - 1; R >= 0; --R) L.up_lv[ulev[R]].push_back((int)r0 + R);
}

}  // namespace

extern "C" {

int irk_group_create(irk_group **out, int s, const double *A, int m, int max_elements, int max_blocks,
                     int max_requests, const irk_options *opt) {
    if (!out) return IRK_ERR_INVALID;
    *out = nullptr;
    if (s < 1 || s > IRK_MAX_S || m < 1 || m > IRK_MAX_M || max_elements < 1 || max_blocks < 1 || max_requests < 1)
        return IRK_ERR_INVALID;
    irk_group *g = new (std::nothrow) irk_group();
    if (!g) return IRK_ERR_NOMEM;
    irk_default_options(&g->opt);
    if (opt) g->opt = *opt;
    g->opt.shift = nullptr;
    g->opt.partition = nullptr;
    const irk_options &o = g->opt;
    if ((o.precond != IRK_PC_UNCOUPLED && o.precond != IRK_PC_NONE) || o.formulation != IRK_TRANSFORMED ||
        (o.factor_prec != IRK_FACTOR_FP32 && o.factor_prec != IRK_FACTOR_FP64) || o.krylov_arith < 0 ||
        o.krylov_arith > 1 || o.restart < 1 || o.restart > IRK_MAX_RESTART || o.partitions > 1 ||
        (opt && opt->partition) || o.ordering < 0 || o.ordering > 1 || m > 128 || o.stage_jacobians != 0 ||
        o.spin_limit < 0 || o.orthogonalization != IRK_ORTHO_MGS) {
        delete g;
        return IRK_ERR_INVALID;
    }
    g->s = s;
    g->m = m;
    g->R = o.restart;
    g->df = o.krylov_arith == IRK_KRYLOV_DF64;
    g->fprec = o.factor_prec;
    g->pc = o.precond;
    if (A)
        memcpy(g->A, A, sizeof(double) * s * s);
    else if (!irk_radau_iia_tableau(s, g->A)) {
        delete g;
        return IRK_ERR_INVALID;
    }
    if (!irk_invert_small(s, g->A, g->Ainv)) {
        delete g;
        return IRK_ERR_INVALID;
    }
    for (int k = 0; k < s; ++k) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j)
            if (j != k) acc += std::fabs(g->Ainv[j * s + k]);
        g->shift[k] = (opt && opt->shift) ? opt->shift[k] : acc;
    }
    cudaGetDevice(&g->dev);
    if (o.stream)
        g->stream = (cudaStream_t)o.stream;
    else if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete g;
        return IRK_ERR_CUDA;
    }
    const long long E = max_elements, B = max_blocks, Lm = max_requests, R = g->R;
    const long long mm = (long long)m * m, cs = (g->fprec == IRK_FACTOR_FP64) ? 8 : 4;
    const long long w = (g->fprec == IRK_FACTOR_FP64) ? 2 : 1;
    const long long Ncap = (long long)s * m * E;
    g->Ecap = E;
    g->Bcap = B;
    g->Lmax = (int)Lm;
    g->unit_cap = Ncap / UNIT + 2 * Lm + 1;
    g->a_e.init(E + Lm);
    g->a_b.init(B);
    g->a_r.init(s * E + Lm);
    g->a_pb.init(s * B + Lm);
    g->a_v.init((2 * R + 3) * Ncap);
    g->a_w.init(2 * Ncap * w);
    g->a_u.init(4 * s * B + 2 * Lm);
    int rc = IRK_OK;
    if ((rc = g_malloc(g, &g->d_rp, E + Lm + 1)) || (rc = g_malloc(g, &g->d_ci, B)) ||
        (rc = g_malloc(g, &g->d_lane_of_elem, E + Lm)) || (rc = g_malloc(g, &g->d_J, B * mm)) ||
        (rc = g_malloc(g, &g->d_M, (E + Lm) * mm)) || (rc = g_malloc(g, &g->d_pool, (2 * R + 3) * Ncap)) ||
        (rc = g_malloc(g, &g->d_ll, 2 * Ncap * w)) || (rc = g_malloc(g, &g->d_prp, s * E + Lm + 1)) ||
        (rc = g_malloc(g, &g->d_pci, s * B + Lm)) || (rc = g_malloc(g, &g->d_pdiag, s * E + Lm)) ||
        (rc = g_malloc(g, &g->d_pvoff, s * E + Lm)) || (rc = g_malloc(g, &g->d_lane_of_prow, s * E + Lm)) ||
        (rc = g_malloc(g, &g->d_asm, s * B + Lm)) || (rc = g_malloc(g, &g->d_upd_ptr, s * B + Lm + 1)) ||
        (rc = g_malloc(g, &g->d_upd, 4 * s * B + 2 * Lm)) || (rc = g_malloc(g, &g->d_rows, s * E + Lm)) ||
        (rc = g_malloc(g, &g->d_lo, s * E + Lm)) || (rc = g_malloc(g, &g->d_up, s * E + Lm)) ||
        (rc = g_malloc(g, (unsigned char **)&g->d_vals, (s * B + Lm) * mm * cs)) ||
        (rc = g_malloc(g, (unsigned char **)&g->d_dinv, (s * E + Lm) * mm * cs)) ||
        (rc = g_malloc(g, &g->d_elems, E + Lm)) || (rc = g_malloc(g, &g->d_units, g->unit_cap)) ||
        (rc = g_malloc(g, &g->d_lane_u0, Lm)) || (rc = g_malloc(g, &g->d_lane_nu, Lm)) ||
        (rc = g_malloc(g, &g->d_part, g->unit_cap)) || (rc = g_malloc(g, &g->d_tickets, Lm)) ||
        (rc = g_malloc(g, &g->d_scal, Lm * G_SLOTS)) || (rc = g_malloc(g, &g->d_H, Lm * (R + 1) * R)) ||
        (rc = g_malloc(g, &g->d_cs, Lm * R)) || (rc = g_malloc(g, &g->d_sn, Lm * R)) ||
        (rc = g_malloc(g, &g->d_g, Lm * (R + 1))) || (rc = g_malloc(g, &g->d_y, Lm * R)) ||
        (rc = g_malloc(g, &g->d_est, Lm)) || (rc = g_malloc(g, &g->d_hn, Lm)) ||
        (rc = g_malloc(g, &g->d_lanes, Lm)) || (rc = g_malloc(g, &g->d_sw, 4 * Lm)) ||
        (rc = g_malloc(g, &g->d_err, 1))) {
        g_free_all(g);
        if (!o.stream) cudaStreamDestroy(g->stream);
        delete g;
        return rc;
    }
    if (cudaMallocHost(&g->h_lanes, sizeof(LaneDev) * Lm) != cudaSuccess ||
        cudaMallocHost(&g->h_out, sizeof(double) * 2 * Lm) != cudaSuccess ||
        cudaMallocHost(&g->h_sw, sizeof(long long) * 4 * Lm) != cudaSuccess ||
        cudaMallocHost(&g->h_err, sizeof(int)) != cudaSuccess) {
        g_free_all(g);
        if (!o.stream) cudaStreamDestroy(g->stream);
        delete g;
        return IRK_ERR_NOMEM;
    }
    cudaMemsetAsync(g->d_tickets, 0, sizeof(unsigned) * Lm, g->stream);
    cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
    cudaMemsetAsync(g->d_H, 0, sizeof(double) * Lm * (R + 1) * R, g->stream);
    cudaMemsetAsync(g->d_ll, 0, sizeof(unsigned long long) * 2 * Ncap * w, g->stream);
    g->lanes.assign(Lm, Lane());
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
        g_free_all(g);
        if (!o.stream) cudaStreamDestroy(g->stream);
        delete g;
        return IRK_ERR_CUDA;
    }
    *out = g;
    return IRK_OK;
}

long long irk_group_device_bytes(const irk_group *g) { return g ? g->bytes : 0; }

void irk_group_destroy(irk_group *g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    g_free_all(g);
    if (!g->opt.stream) cudaStreamDestroy(g->stream);
    delete g;
}

}  // extern "C"

namespace {

int read_to_host(void *dst, const void *src, size_t bytes, int mem_space) {
    if (bytes == 0) return IRK_OK;
    if (mem_space == IRK_DEVICE) return cuda_status(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    memcpy(dst, src, bytes);
    return IRK_OK;
}

int stage_to_device(irk_group *g, double **tmp, const double *src, long long n, int mem_space) {
    if (cudaMalloc(tmp, sizeof(double) * std::max(1LL, n)) != cudaSuccess) {
        cudaGetLastError();
        return IRK_ERR_NOMEM;
    }
    return cuda_status(cudaMemcpyAsync(*tmp, src, sizeof(double) * n,
                                       mem_space == IRK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                       g->stream));
}

}  // namespace

extern "C" {

int irk_group_submit(irk_group *g, int T, const int32_t *row_ptr, const int32_t *col_idx, const double *J,
                     const double *M, const double *Rhs, double dt, double rtol, int mem_space, int *slot) {
    if (!g || T < 1 || !row_ptr || !col_idx || !J || !M || !Rhs || !slot || !(rtol >= 0.0) || !std::isfinite(dt))
        return IRK_ERR_INVALID;
    *slot = -1;
    const int s = g->s, m = g->m;
    std::vector<int> rp(T + 1), ci;
    int rc = read_to_host(rp.data(), row_ptr, sizeof(int) * (T + 1), mem_space);
    if (rc) return rc;
    if (rp[0] != 0) return IRK_ERR_INVALID;
    for (int i = 0; i < T; ++i)
        if (rp[i + 1] < rp[i]) return IRK_ERR_INVALID;
    const int nnzb = rp[T];
    ci.resize(std::max(1, nnzb));
    if ((rc = read_to_host(ci.data(), col_idx, sizeof(int) * nnzb, mem_space))) return rc;
    ci.resize(nnzb);
    for (int i = 0; i < T; ++i) {  // sorted, in range, diagonal, symmetric
        bool diag = false;
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const int j = ci[p];
            if (j < 0 || j >= T || (p > rp[i] && ci[p - 1] >= j)) return IRK_ERR_INVALID;
            diag |= (j == i);
            if (!std::binary_search(ci.begin() + rp[j], ci.begin() + rp[j + 1], i)) return IRK_ERR_INVALID;
        }
        if (!diag) return IRK_ERR_INVALID;
    }
    int lane = -1;
    for (int l = 0; l < g->Lmax; ++l)
        if (g->lanes[l].state == L_FREE) {
            lane = l;
            break;
        }
    if (lane < 0) return IRK_ERR_NOMEM;
    Lane L;
    L.T = T;
    L.nnzb = nnzb;
    L.N = (long long)s * T * m;
    const long long w = (g->fprec == IRK_FACTOR_FP64) ? 2 : 1;
    L.n_e = T + 1;
    L.n_b = nnzb;
    L.n_r = (long long)s * T + 1;
    L.n_v = (2LL * g->R + 3) * L.N;
    L.n_w = 2 * L.N * w;
    L.e0 = g->a_e.alloc(L.n_e);
    L.b0 = g->a_b.alloc(L.n_b);
    L.r0 = g->a_r.alloc(L.n_r);
    L.vo = g->a_v.alloc(L.n_v);
    L.wo = g->a_w.alloc(L.n_w);
    auto fail = [&](int code) {
        g->a_e.release(L.e0, L.n_e);
        g->a_b.release(L.b0, L.n_b);
        g->a_r.release(L.r0, L.n_r);
        g->a_pb.release(L.pb0, L.n_pb);
        g->a_v.release(L.vo, L.n_v);
        g->a_w.release(L.wo, L.n_w);
        g->a_u.release(L.uo, L.n_u);
        return code;
    };
    if (L.e0 < 0 || L.b0 < 0 || L.r0 < 0 || L.vo < 0 || L.wo < 0) return fail(IRK_ERR_NOMEM);
    const long long mm = (long long)m * m, cs = (g->fprec == IRK_FACTOR_FP64) ? 8 : 4;
    cudaStream_t st = g->stream;
    // pattern of J in the group's numbering
    std::vector<int> rpg(T + 1), cig(nnzb), lane_of(T + 1, lane);
    for (int i = 0; i <= T; ++i) rpg[i] = (int)L.b0 + rp[i];
    for (int p = 0; p < nnzb; ++p) cig[p] = (int)L.e0 + ci[p];
    LanePattern PP;
    std::vector<int> lane_of_prow;
    if (g->pc == IRK_PC_UNCOUPLED) {
        build_lane_pattern(g, rp, ci, T, L.e0, L.b0, L.r0, PP, L);
        L.npb = (int)PP.ci.size();
        L.n_pb = L.npb + 1;
        L.n_u = std::max<long long>(2, (long long)PP.upd.size());  // even: pairs stay aligned
        L.pb0 = g->a_pb.alloc(L.n_pb);
        L.uo = g->a_u.alloc(L.n_u);
        if (L.pb0 < 0 || L.uo < 0) return fail(IRK_ERR_NOMEM);
        for (auto &x : PP.rp) x += (int)L.pb0;
        for (auto &x : PP.diag) x += (int)L.pb0;
        for (size_t q = 0; q + 1 < PP.upd.size(); q += 2) {
            PP.upd[q] += (int)L.pb0;
            PP.upd[q + 1] += (int)L.pb0;
        }
        for (auto &x : PP.upd_ptr) x += (int)(L.uo / 2);
        lane_of_prow.assign(s * T + 1, lane);
    }
    double *tJ = nullptr, *tM = nullptr, *tR = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        cudaFree(tJ);
        cudaFree(tM);
        cudaFree(tR);
    };
    rc = IRK_OK;
#define G_TRY(x)                          \
    do {                                  \
        if ((rc = (x)) != IRK_OK) {       \
            cleanup();                    \
            return fail(rc);              \
        }                                 \
    } while (0)
#define G_CP(dst, src, bytes) G_TRY(cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)))
    G_CP(g->d_rp + L.e0, rpg.data(), sizeof(int) * (T + 1));
    if (nnzb) G_CP(g->d_ci + L.b0, cig.data(), sizeof(int) * nnzb);
    G_CP(g->d_lane_of_elem + L.e0, lane_of.data(), sizeof(int) * (T + 1));
    G_TRY(stage_to_device(g, &tJ, J, (long long)nnzb * mm, mem_space));
    G_TRY(stage_to_device(g, &tM, M, (long long)T * mm, mem_space));
    G_TRY(stage_to_device(g, &tR, Rhs, L.N, mem_space));
    const vec8 *dummy = nullptr;
    (void)dummy;
    const long long vB = L.vo + (2LL * g->R + 1) * L.N + L.N;  // B region (after V, Z, X)
    const long long vX = L.vo + (2LL * g->R + 1) * L.N;
    if (g->df) {
        if (nnzb) k_g_blocks<ArDF><<<g_grid((long long)nnzb * mm), 256, 0, st>>>((long long)nnzb * mm, m, tJ, g->d_J + L.b0 * mm);
        k_g_blocks<ArDF><<<g_grid((long long)T * mm), 256, 0, st>>>((long long)T * mm, m, tM, g->d_M + L.e0 * mm);
        k_g_in<ArDF><<<g_grid(L.N), 256, 0, st>>>(L.N, T, m, s, tR, g->d_pool + vB);
    } else {
        if (nnzb) k_g_blocks<ArF64><<<g_grid((long long)nnzb * mm), 256, 0, st>>>((long long)nnzb * mm, m, tJ, g->d_J + L.b0 * mm);
        k_g_blocks<ArF64><<<g_grid((long long)T * mm), 256, 0, st>>>((long long)T * mm, m, tM, g->d_M + L.e0 * mm);
        k_g_in<ArF64><<<g_grid(L.N), 256, 0, st>>>(L.N, T, m, s, tR, g->d_pool + vB);
    }
    G_TRY(cuda_status(cudaGetLastError()));
    G_TRY(cuda_status(cudaMemsetAsync(g->d_pool + vX, 0, sizeof(vec8) * L.N, st)));
    if (g->pc == IRK_PC_UNCOUPLED) {
        G_CP(g->d_prp + L.r0, PP.rp.data(), sizeof(int) * PP.rp.size());
        G_CP(g->d_pci + L.pb0, PP.ci.data(), sizeof(int) * PP.ci.size());
        G_CP(g->d_pdiag + L.r0, PP.diag.data(), sizeof(int) * PP.diag.size());
        G_CP(g->d_pvoff + L.r0, PP.voff.data(), sizeof(int) * PP.voff.size());
        G_CP(g->d_lane_of_prow + L.r0, lane_of_prow.data(), sizeof(int) * lane_of_prow.size());
        G_CP(g->d_asm + L.pb0, PP.asmv.data(), sizeof(AsmEntry) * PP.asmv.size());
        G_CP(g->d_upd_ptr + L.pb0, PP.upd_ptr.data(), sizeof(int) * PP.upd_ptr.size());
        if (!PP.upd.empty()) G_CP(g->d_upd + L.uo, PP.upd.data(), sizeof(int) * PP.upd.size());
        // assemble (d_k M - dt J) and factor, level by level
        double cm[IRK_MAX_S * IRK_MAX_S] = {0}, cj[1] = {-dt};
        for (int k = 0; k < s; ++k) cm[k * s + k] = g->Ainv[k * s + k] + g->shift[k];
        G_TRY(ilu_assemble(st, g->fprec, L.npb, m, g->d_asm + L.pb0, g->d_J, g->d_M, g->df, cm, s * s, cj, 1,
                           (char *)g->d_vals + L.pb0 * mm * cs));
        std::vector<int> rows;
        std::vector<int> lvp(1, 0);
        for (const auto &lv : L.lo_lv) {
            rows.insert(rows.end(), lv.begin(), lv.end());
            lvp.push_back((int)rows.size());
        }
        G_CP(g->d_rows + L.r0, rows.data(), sizeof(int) * rows.size());
        G_TRY(cuda_status(cudaMemsetAsync(g->d_err, 0, sizeof(int), st)));
        for (size_t l = 0; l + 1 < lvp.size(); ++l)
            G_TRY(ilu_factor_level(st, g->fprec, g->d_rows + L.r0 + lvp[l], lvp[l + 1] - lvp[l], m, g->d_prp,
                                   g->d_pci, g->d_pdiag, g->d_upd_ptr, g->d_upd, g->d_vals, g->d_dinv, g->d_err));
        G_TRY(sync_group(g));  // also keeps the host vectors alive until the copies ran
    } else {
        G_TRY(cuda_status(cudaStreamSynchronize(st)));
    }
#undef G_CP
#undef G_TRY
    cleanup();
    L.state = L_RESID;
    L.dt = dt;
    L.rtol = rtol;
    g->lanes[lane] = L;
    g->dirty = true;
    *slot = lane;
    return IRK_OK;
}

int irk_group_step(irk_group *g, int *n_active) {
    if (!g) return IRK_ERR_INVALID;
    int rc;
    if (g->dirty && (rc = rebuild_lists(g))) return rc;
    const int Lm = g->Lmax;
    fill_lane_dev(g);
    cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
    // phase A: true residual r = b - B x (into V_0) of requests at a cycle boundary
    bool any = false;
    for (int l = 0; l < Lm; ++l)
        if (g->lanes[l].state == L_RESID) {
            g->h_lanes[l].mv = 2;
            g->h_lanes[l].res = 1;
            any = true;
        }
    bool became_done = false;
    if (any) {
        if ((rc = upload_lanes(g)) || (rc = launch_g_matvec(g)) || (rc = launch_g_red(g, 0, 1))) return rc;
        cudaMemcpyAsync(g->h_out + Lm, g->d_hn, sizeof(double) * Lm, cudaMemcpyDeviceToHost, g->stream);
        if ((rc = sync_group(g))) return rc;
        bool start = false;
        for (int l = 0; l < Lm; ++l) {
            Lane &L = g->lanes[l];
            LaneDev &D = g->h_lanes[l];
            D.mv = 0;
            D.res = 0;
            if (L.state != L_RESID) continue;
            L.beta = g->h_out[Lm + l];
            if (L.first) {
                L.bnorm = L.beta;
                L.first = false;
            }
            if (!std::isfinite(L.beta)) {
                L.state = L_DONE;
                L.status = IRK_ERR_NONFINITE;
            } else if (L.bnorm == 0.0 || L.beta <= L.rtol * L.bnorm) {
                L.state = L_DONE;
                L.status = IRK_OK;
            } else if (L.total >= g->opt.max_iter) {
                L.state = L_DONE;
                L.status = IRK_NOT_CONVERGED;
            } else {
                L.state = L_ITER;
                L.j = 0;
                L.cycles++;
                D.cyc = 1;
                D.j = 0;
                start = true;
            }
            if (L.state == L_DONE) became_done = true;
        }
        if (start) {
            if ((rc = upload_lanes(g)) || (rc = launch_g_scalar(g, 0)) || (rc = launch_g_vec(g, 1))) return rc;
            for (int l = 0; l < Lm; ++l) g->h_lanes[l].cyc = 0;
        }
    }
    // phase B: one FGMRES iteration of every iterating request
    int maxj = -1;
    for (int l = 0; l < Lm; ++l)
        if (g->lanes[l].state == L_ITER) {
            g->h_lanes[l].mgs = 1;
            g->h_lanes[l].mv = 1;
            g->h_lanes[l].j = g->lanes[l].j;
            maxj = std::max(maxj, g->lanes[l].j);
        }
    if (maxj >= 0) {
        if ((rc = upload_lanes(g)) || (rc = launch_g_sweep(g)) || (rc = launch_g_matvec(g))) return rc;
        for (int i = 0; i <= maxj + 1; ++i)
            if ((rc = launch_g_red(g, i, 0))) return rc;
        if ((rc = launch_g_vec(g, 0)) || (rc = launch_g_scalar(g, 1))) return rc;
        cudaMemcpyAsync(g->h_out, g->d_est, sizeof(double) * Lm, cudaMemcpyDeviceToHost, g->stream);
        cudaMemcpyAsync(g->h_out + Lm, g->d_hn, sizeof(double) * Lm, cudaMemcpyDeviceToHost, g->stream);
        if ((rc = sync_group(g))) return rc;
        bool upd = false;
        for (int l = 0; l < Lm; ++l) {
            Lane &L = g->lanes[l];
            LaneDev &D = g->h_lanes[l];
            D.mv = 0;
            D.mgs = 0;
            if (L.state != L_ITER) continue;
            L.total++;
            L.est = g->h_out[l];
            const double hn = g->h_out[Lm + l];
            if (L.est <= L.rtol * L.bnorm || L.total >= g->opt.max_iter || L.j + 1 == g->R || hn == 0.0) {
                D.upd = 1;
                D.j = L.j;
                L.state = L_RESID;
                upd = true;
            } else {
                L.j++;
            }
        }
        if (upd && ((rc = upload_lanes(g)) || (rc = launch_g_scalar(g, 2)) || (rc = launch_g_vec(g, 3)))) return rc;
    }
    if (became_done) g->dirty = true;
    int na = 0;
    for (int l = 0; l < Lm; ++l)
        if (g->lanes[l].state == L_RESID || g->lanes[l].state == L_ITER) ++na;
    if (n_active) *n_active = na;
    return cuda_status(cudaGetLastError());
}

int irk_group_query(const irk_group *g, int slot, int *iters, double *relres, int *status) {
    if (!g || slot < 0 || slot >= g->Lmax || g->lanes[slot].state == L_FREE) return IRK_ERR_INVALID;
    const Lane &L = g->lanes[slot];
    if (iters) *iters = L.total;
    if (relres) *relres = L.bnorm > 0.0 ? L.beta / L.bnorm : 0.0;
    if (status) *status = L.status;
    return L.state == L_DONE ? 0 : 1;
}

int irk_group_collect(irk_group *g, int slot, double *W, int mem_space) {
    if (!g || !W || slot < 0 || slot >= g->Lmax) return IRK_ERR_INVALID;
    Lane &L = g->lanes[slot];
    if (L.state != L_DONE) return IRK_ERR_STATE;
    const long long vX = L.vo + (2LL * g->R + 1) * L.N;
    double *dst = W, *tmp = nullptr;
    if (mem_space != IRK_DEVICE) {
        if (cudaMalloc(&tmp, sizeof(double) * L.N) != cudaSuccess) {
            cudaGetLastError();
            return IRK_ERR_NOMEM;
        }
        dst = tmp;
    }
    if (g->df)
        k_g_out<ArDF><<<g_grid(L.N), 256, 0, g->stream>>>(L.N, L.T, g->m, g->s, g->d_pool + vX, dst);
    else
        k_g_out<ArF64><<<g_grid(L.N), 256, 0, g->stream>>>(L.N, L.T, g->m, g->s, g->d_pool + vX, dst);
    int rc = cuda_status(cudaGetLastError());
    if (!rc && tmp)
        rc = cuda_status(cudaMemcpyAsync(W, tmp, sizeof(double) * L.N, cudaMemcpyDeviceToHost, g->stream));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(g->stream));
    cudaFree(tmp);
    if (rc) return rc;
    lane_release(g, L);
    return IRK_OK;
}

}  // extern "C"
