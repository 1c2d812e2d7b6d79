// api.cu -- the C ABI (include/irk_gb300.h): context set-up, the Radau IIA
// tableau, and the host control of restarted flexible GMRES (Sec. 4), whose
// every vector operation runs in the kernels of k_matvec.cu, k_ilu.cu and
// k_krylov.cu.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "irk_internal.h"

// Map a CUDA runtime status to the library's codes.  With the environment
// variable IRK_DEBUG set, failures are also reported on stderr by name.
int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return IRK_OK;
    static const bool debug = getenv("IRK_DEBUG") != nullptr;
    if (debug) fprintf(stderr, "irk: CUDA error %s (%s)\n", cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return IRK_ERR_NOMEM;
    return IRK_ERR_CUDA;
}

namespace {

// ---------------------------------------------------------------------------
// Radau IIA tableau by collocation (App. A): c_k are the zeros of
// P_s(2x-1) - P_{s-1}(2x-1), a_ik = integral_0^{c_i} l_k(x) dx with l_k the
// Lagrange basis on the c's.  Polynomials as coefficient vectors (degree <= 8).
double legendre(int n, double y) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = y;
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * y * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

double radau_q(int s, double x) { return legendre(s, 2.0 * x - 1.0) - legendre(s - 1, 2.0 * x - 1.0); }

bool radau_iia(int s, double *A) {
    std::vector<double> c;
    const int NS = 20000;
    double xa = 0.0, fa = radau_q(s, 0.0);
    for (int q = 1; q <= NS && (int)c.size() < s - 1; ++q) {
        double xb = (double)q / NS, fb = radau_q(s, xb);
        if (fa == 0.0) {
            c.push_back(xa);
        } else if ((fa < 0) != (fb < 0) && xb < 1.0) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), fm = radau_q(s, mid);
                if ((fm < 0) == (flo < 0)) {
                    lo = mid;
                    flo = fm;
                } else {
                    hi = mid;
                }
            }
            c.push_back(0.5 * (lo + hi));
        }
        xa = xb;
        fa = fb;
    }
    c.push_back(1.0);
    if ((int)c.size() != s) return false;
    for (int k = 0; k < s; ++k) {
        // l_k(x) = prod_{q != k} (x - c_q) / (c_k - c_q)
        std::vector<double> poly(1, 1.0);
        double den = 1.0;
        for (int q = 0; q < s; ++q) {
            if (q == k) continue;
            std::vector<double> np(poly.size() + 1, 0.0);
            for (size_t d = 0; d < poly.size(); ++d) {
                np[d + 1] += poly[d];
                np[d] -= c[q] * poly[d];
            }
            poly.swap(np);
            den *= (c[k] - c[q]);
        }
        for (int i = 0; i < s; ++i) {
            double acc = 0.0, xp = c[i];
            for (size_t d = 0; d < poly.size(); ++d) {
                acc += poly[d] * xp / (double)(d + 1);
                xp *= c[i];
            }
            A[i * s + k] = acc / den;
        }
    }
    return true;
}

bool invert_small(int n, const double *A, double *X) {
    std::vector<double> a(A, A + n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) X[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (std::fabs(a[r * n + k]) > std::fabs(a[p * n + k])) p = r;
        if (a[p * n + k] == 0.0) return false;
        for (int j = 0; j < n; ++j) {
            std::swap(a[k * n + j], a[p * n + j]);
            std::swap(X[k * n + j], X[p * n + j]);
        }
        double ip = 1.0 / a[k * n + k];
        for (int j = 0; j < n; ++j) {
            a[k * n + j] *= ip;
            X[k * n + j] *= ip;
        }
        for (int r = 0; r < n; ++r) {
            if (r == k) continue;
            double f = a[r * n + k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                a[r * n + j] -= f * a[k * n + j];
                X[r * n + j] -= f * X[k * n + j];
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
int copy_in(void *dst, const void *src, size_t bytes, int mem_space, cudaStream_t st) {
    if (bytes == 0) return IRK_OK;
    cudaMemcpyKind kind = (mem_space == IRK_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    return cuda_status(cudaMemcpyAsync(dst, src, bytes, kind, st));
}

int copy_out(void *dst, const void *src, size_t bytes, int mem_space, cudaStream_t st) {
    if (bytes == 0) return IRK_OK;
    cudaMemcpyKind kind = (mem_space == IRK_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    return cuda_status(cudaMemcpyAsync(dst, src, bytes, kind, st));
}

int read_host(void *dst, const void *src, size_t bytes, int mem_space) {
    if (mem_space == IRK_DEVICE) return cuda_status(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    memcpy(dst, src, bytes);
    return IRK_OK;
}

// Wait for the context's stream and read the device error word (an ordered
// copy on the same stream into pinned memory: no device-wide synchronisation,
// so contexts on different streams do not serialise each other).
int err_code(int err) {
    if (err & IRK_DEV_ERR_SINGULAR) return IRK_ERR_SINGULAR;
    if (err & IRK_DEV_ERR_NONFINITE) return IRK_ERR_NONFINITE;
    if (err & IRK_DEV_ERR_TIMEOUT) return IRK_ERR_TIMEOUT;
    return IRK_OK;
}

int sync_err(irk_ctx *c) {
    int *herr = reinterpret_cast<int *>(c->h_scal + 3);
    cudaError_t e = cudaMemcpyAsync(herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return err_code(*herr);
}

// A largest magnitude the double-float arithmetic can carry: 0 or within
// [2^-100, 2^100] (include/irk_gb300.h).
bool df_range_ok(double amax) {
    return amax == 0.0 || (amax >= IRK_DF64_MIN_MAGNITUDE && amax <= IRK_DF64_MAX_MAGNITUDE);
}

// Load J and M (row-major binary64 in mem_space) into the context's
// column-major device blocks through a temporary device buffer.  The
// conversion records the largest magnitude of each and flags non-finite
// values: IRK_ERR_NONFINITE for a NaN or infinity, IRK_ERR_INVALID for
// double-float values out of range.
int load_values(irk_ctx *c, const double *J, const double *M, int mem_space) {
    const long long mm = (long long)c->m * c->m;
    const long long nJ = (long long)c->nJ * c->nnzb * mm, nM = (long long)c->T * mm;
    const long long need = nJ > nM ? nJ : nM;
    double *tmp = nullptr;
    int rc = cuda_status(cudaMalloc(&tmp, (size_t)need * sizeof(double)));
    if (rc) return rc;
    unsigned long long *amax = c->d_amax;  // [0] J, [1] M
    unsigned long long *hmax = reinterpret_cast<unsigned long long *>(c->h_scal + 4);
    int *herr = reinterpret_cast<int *>(c->h_scal + 3);
    if ((rc = cuda_status(cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned long long), c->stream))) == IRK_OK &&
        (rc = cuda_status(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream))) == IRK_OK &&
        (rc = copy_in(tmp, J, (size_t)nJ * sizeof(double), mem_space, c->stream)) == IRK_OK &&
        (rc = launch_convert_blocks(c, tmp, c->d_J, (long long)c->nJ * c->nnzb, amax, c->d_err)) == IRK_OK &&
        (rc = copy_in(tmp, M, (size_t)nM * sizeof(double), mem_space, c->stream)) == IRK_OK &&
        (rc = launch_convert_blocks(c, tmp, c->d_M, c->T, amax + 1, c->d_err)) == IRK_OK &&
        (rc = cuda_status(cudaMemcpyAsync(hmax, amax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                          c->stream))) == IRK_OK &&
        (rc = cuda_status(cudaMemcpyAsync(herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream))) == IRK_OK)
        rc = cuda_status(cudaStreamSynchronize(c->stream));
    cudaFree(tmp);
    if (rc) return rc;
    if (*herr & IRK_DEV_ERR_NONFINITE) return IRK_ERR_NONFINITE;
    double jm, mmx;
    memcpy(&jm, &hmax[0], sizeof(double));
    memcpy(&mmx, &hmax[1], sizeof(double));
    c->jmax = jm;
    c->mmax = mmx;
    if (c->dfop && (!df_range_ok(jm) || !df_range_ok(mmx))) return IRK_ERR_INVALID;
    return IRK_OK;
}

// dt admissible for the context's arithmetic: finite, and with double-float
// dt * max|J| within its range.
bool dt_ok(const irk_ctx *c, double dt) {
    if (!std::isfinite(dt)) return false;
    return !c->dfop || std::fabs(dt) * c->jmax <= IRK_DF64_MAX_MAGNITUDE;
}

// Power-of-two scale of a right-hand side in d_io when the operator product
// is double-float (see the header); null for binary64 (no scaling).
const double *rhs_scale(irk_ctx *c, int *rc) {
    if (!c->dfop) return nullptr;
    *rc = launch_pow2_scale(c->stream, c->N, c->d_io, c->d_amax + 2, c->d_vscale);
    c->launches += 2;
    return c->d_vscale;
}

}  // namespace

// Phase timing: tmark_begin / tmark_end record a pair of events around a
// phase of kind 0 (operator product), 1 (preconditioner), 2 (Gram-Schmidt),
// 3 (factor assembly), 4 (factor block products), 5 (factor inverses),
// 6 (forward sweep), 7 (backward sweep).
#define IRK_TMARK_FLUSH 32768

namespace {
void tflush(irk_ctx *c);
}

int tmark_begin(irk_ctx *c) {
    if (!c->opt.timing) return -1;
    if (c->opt.timing == 2 && c->tused >= 2 * IRK_TMARK_FLUSH) {
        // bound the pending marks of a caller that never asks for stats
        cudaStreamSynchronize(c->stream);
        tflush(c);
    }
    if (c->tused + 2 > (int)c->tev.size()) {
        for (int q = 0; q < 64; ++q) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            c->tev.push_back(e);
        }
        c->tkind.resize(c->tev.size() / 2);
    }
    int slot = c->tused;
    c->tused += 2;
    cudaEventRecord(c->tev[slot], c->stream);
    return slot;
}

void tmark_end(irk_ctx *c, int slot, int kind) {
    if (slot < 0) return;
    cudaEventRecord(c->tev[slot + 1], c->stream);
    c->tkind[slot / 2] = kind;
}

namespace {

void tcollect(irk_ctx *c) {
    c->stats.matvec_ms = c->stats.precond_ms = c->stats.ortho_ms = 0.0;
    c->stats.sweep_fwd_ms = c->stats.sweep_bwd_ms = 0.0;
    c->stats.n_matvec = c->stats.n_precond = c->stats.n_ortho = 0;
    for (int slot = 0; slot < c->tused; slot += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->tev[slot], c->tev[slot + 1]);
        switch (c->tkind[slot / 2]) {
            case 0: c->stats.matvec_ms += ms; c->stats.n_matvec++; break;
            case 1: c->stats.precond_ms += ms; c->stats.n_precond++; break;
            case 6: c->stats.sweep_fwd_ms += ms; break;
            case 7: c->stats.sweep_bwd_ms += ms; break;
            default: c->stats.ortho_ms += ms; c->stats.n_ortho++; break;
        }
    }
    c->tused = 0;
}

// timing = 2: read every pending mark into the running totals (by kind) and
// release the marks; the caller has synchronised the stream
void tflush(irk_ctx *c) {
    for (int slot = 0; slot < c->tused; slot += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->tev[slot], c->tev[slot + 1]);
        const int k = c->tkind[slot / 2] & 7;
        c->tacc_ms[k] += ms;
        c->tacc_n[k]++;
    }
    c->tused = 0;
}

// timing = 2: the totals since the last irk_get_stats into the phase fields
// (kind 0 operator product, 1 preconditioner, 2 orthogonalisation, 3-5
// factorisation kernels, 6-7 sweeps), then cleared
void treport(irk_ctx *c) {
    tflush(c);
    irk_stats &t = c->stats;
    t.matvec_ms = c->tacc_ms[0], t.n_matvec = c->tacc_n[0];
    t.precond_ms = c->tacc_ms[1], t.n_precond = c->tacc_n[1];
    t.ortho_ms = c->tacc_ms[2], t.n_ortho = c->tacc_n[2];
    t.factor_assemble_ms = c->tacc_ms[3];
    t.factor_products_ms = c->tacc_ms[4];
    t.factor_inverse_ms = c->tacc_ms[5];
    t.sweep_fwd_ms = c->tacc_ms[6];
    t.sweep_bwd_ms = c->tacc_ms[7];
    for (int k = 0; k < 8; ++k) c->tacc_ms[k] = 0.0, c->tacc_n[k] = 0;
}

// the factorisation's marks (kinds 3-5), collected after its synchronisation
static void tcollect_factor(irk_ctx *c) {
    c->stats.factor_assemble_ms = c->stats.factor_products_ms = c->stats.factor_inverse_ms = 0.0;
    for (int slot = 0; slot < c->tused; slot += 2) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->tev[slot], c->tev[slot + 1]);
        switch (c->tkind[slot / 2]) {
            case 3: c->stats.factor_assemble_ms += ms; break;
            case 4: c->stats.factor_products_ms += ms; break;
            case 5: c->stats.factor_inverse_ms += ms; break;
            default: break;
        }
    }
    c->tused = 0;
}

void free_ctx(irk_ctx *c) {
    if (!c) return;
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    pc_free(c->pc);
    cudaFree(c->d_rp);
    cudaFree(c->d_ci);
    cudaFree(c->d_J);
    cudaFree(c->d_M);
    cudaFree(c->d_V);
    cudaFree(c->d_Z);
    cudaFree(c->d_x);
    cudaFree(c->d_rowctr);
    cudaFree(c->d_xdf);
    cudaFree(c->d_ydf);
    cudaFree(c->d_b);
    cudaFree(c->d_io);
    cudaFree(c->d_H);
    cudaFree(c->d_cs);
    cudaFree(c->d_sn);
    cudaFree(c->d_g);
    cudaFree(c->d_yls);
    cudaFree(c->d_scal);
    cudaFree(c->d_part);
    cudaFree(c->d_ticket);
    cudaFree(c->d_err);
    cudaFree(c->d_vscale);
    cudaFree(c->d_amax);
    if (c->h_scal) cudaFreeHost(c->h_scal);
    delete c;
}

}  // namespace

// tableau helpers shared with the multi-request engine (group.cu)
bool irk_radau_iia_tableau(int s, double *A) { return radau_iia(s, A); }
bool irk_invert_small(int n, const double *A, double *X) { return invert_small(n, A, X); }

extern "C" {

void irk_default_options(irk_options *o) {
    if (!o) return;
    o->restart = 30;
    o->max_iter = 3000;
    o->precond = IRK_PC_UNCOUPLED;
    o->factor_prec = IRK_FACTOR_FP64;
    o->krylov_arith = IRK_KRYLOV_FP64;
    o->formulation = IRK_TRANSFORMED;
    o->shift = nullptr;
    o->stream = nullptr;
    o->timing = 0;
    o->sweep = IRK_SWEEP_AUTO;
    o->ordering = IRK_ORDER_NATURAL;
    o->partitions = 0;
    o->partition = nullptr;
    o->stage_jacobians = 0;
    o->spin_limit = 0;
    o->orthogonalization = IRK_ORTHO_MGS;
}

const char *irk_strerror(int code) {
    switch (code) {
        case IRK_OK: return "ok";
        case IRK_NOT_CONVERGED: return "not converged within max_iter";
        case IRK_ERR_INVALID: return "invalid argument or pattern";
        case IRK_ERR_NOMEM: return "out of memory";
        case IRK_ERR_SINGULAR: return "singular diagonal block in block ILU(0)";
        case IRK_ERR_NONFINITE: return "non-finite value in the Krylov iteration";
        case IRK_ERR_TIMEOUT: return "bounded device wait timed out";
        case IRK_ERR_CUDA: return "CUDA runtime error";
        case IRK_ERR_STATE: return "call out of order";
        case IRK_ERR_SCRATCH_LIMIT: return "system too large for the fixed scratch of irk_apply_precond_noalloc";
        default: return "unknown status";
    }
}

int irk_setup(irk_ctx **out, int s, const double *A, int T, int m, const int32_t *row_ptr,
              const int32_t *col_idx, const double *J, const double *M, int mem_space,
              const irk_options *opt) {
    if (!out) return IRK_ERR_INVALID;
    *out = nullptr;
    if (s < 1 || s > IRK_MAX_S || T < 1 || m < 1 || m > IRK_MAX_M || !row_ptr || !col_idx || !J || !M)
        return IRK_ERR_INVALID;
    if (mem_space != IRK_HOST && mem_space != IRK_DEVICE) return IRK_ERR_INVALID;
    irk_ctx *c = new (std::nothrow) irk_ctx();
    if (!c) return IRK_ERR_NOMEM;
    irk_default_options(&c->opt);
    if (opt) c->opt = *opt;
    c->opt.shift = nullptr;
    c->opt.partition = nullptr;
    int rc = IRK_OK;
    if (c->opt.restart < 1 || c->opt.restart > IRK_MAX_RESTART || c->opt.max_iter < 0 ||
        c->opt.precond < IRK_PC_NONE || c->opt.precond > IRK_PC_ELEMENT || c->opt.factor_prec < 0 ||
        c->opt.factor_prec > IRK_FACTOR_BF16 || c->opt.krylov_arith < 0 || c->opt.krylov_arith > IRK_KRYLOV_FP64_DFOP ||
        c->opt.formulation < 0 || c->opt.formulation > 1 || c->opt.sweep < 0 || c->opt.sweep > 1 ||
        c->opt.ordering < 0 || c->opt.ordering > 1 || c->opt.partitions < 0 || c->opt.stage_jacobians < 0 ||
        c->opt.stage_jacobians > 1 || c->opt.spin_limit < 0 || c->opt.orthogonalization < 0 ||
        c->opt.orthogonalization > IRK_ORTHO_CGS2 ||
        (c->opt.precond == IRK_PC_UNCOUPLED && c->opt.formulation != IRK_TRANSFORMED)) {
        delete c;
        return IRK_ERR_INVALID;
    }
    c->stream = (cudaStream_t)c->opt.stream;
    c->s = s;
    c->T = T;
    c->m = m;
    c->df = c->opt.krylov_arith == IRK_KRYLOV_DF64;
    c->dfop = c->opt.krylov_arith == IRK_KRYLOV_DF64 || c->opt.krylov_arith == IRK_KRYLOV_FP64_DFOP;
    c->fprec = c->opt.factor_prec;
    c->nJ = (c->opt.stage_jacobians && s > 1) ? s : 1;
    c->spin = c->opt.spin_limit > 0 ? c->opt.spin_limit : IRK_DEFAULT_SPIN_LIMIT;
    irk_default_kernel_options(&c->ko);
    cudaGetDevice(&c->dev);
    // pattern: host copy and validation
    c->h_rp.resize(T + 1);
    if ((rc = read_host(c->h_rp.data(), row_ptr, sizeof(int32_t) * (T + 1), mem_space))) {
        free_ctx(c);
        return rc;
    }
    if (c->h_rp[0] != 0) {
        free_ctx(c);
        return IRK_ERR_INVALID;
    }
    for (int i = 0; i < T; ++i)
        if (c->h_rp[i + 1] < c->h_rp[i]) {
            free_ctx(c);
            return IRK_ERR_INVALID;
        }
    c->nnzb = c->h_rp[T];
    c->h_ci.resize(c->nnzb > 0 ? c->nnzb : 1);
    if ((rc = read_host(c->h_ci.data(), col_idx, sizeof(int32_t) * c->nnzb, mem_space))) {
        free_ctx(c);
        return rc;
    }
    c->h_ci.resize(c->nnzb);
    for (int i = 0; i < T && rc == IRK_OK; ++i) {
        bool diag = false;
        for (int p = c->h_rp[i]; p < c->h_rp[i + 1]; ++p) {
            int j = c->h_ci[p];
            if (j < 0 || j >= T || (p > c->h_rp[i] && c->h_ci[p - 1] >= j)) rc = IRK_ERR_INVALID;
            if (j == i) diag = true;
        }
        if (!diag) rc = IRK_ERR_INVALID;
    }
    for (int i = 0; i < T && rc == IRK_OK; ++i)
        for (int p = c->h_rp[i]; p < c->h_rp[i + 1]; ++p) {
            int j = c->h_ci[p];
            bool found = false;
            for (int q = c->h_rp[j]; q < c->h_rp[j + 1]; ++q) found |= (c->h_ci[q] == i);
            if (!found) rc = IRK_ERR_INVALID;
        }
    if (rc) {
        free_ctx(c);
        return rc;
    }
    if (opt && opt->partition) c->h_part.assign(opt->partition, opt->partition + T);
    // tableau, inverse, shifts (Sec. 4.3.2 column rule unless given)
    if (A) {
        memcpy(c->A, A, sizeof(double) * s * s);
    } else if (!radau_iia(s, c->A)) {
        free_ctx(c);
        return IRK_ERR_INVALID;
    }
    if (!invert_small(s, c->A, c->Ainv)) {
        free_ctx(c);
        return IRK_ERR_INVALID;
    }
    for (int k = 0; k < s; ++k) {
        if (opt && opt->shift) {
            c->shift[k] = opt->shift[k];
        } else {
            double acc = 0.0;
            for (int j = 0; j < s; ++j)
                if (j != k) acc += std::fabs(c->Ainv[j * s + k]);
            c->shift[k] = acc;
        }
    }
    c->n = (long long)T * m;
    c->N = c->n * s;
    const long long mm = (long long)m * m;
    const int R = c->opt.restart;
    c->red_blocks = 152 * 4;
    bool ok = cudaMalloc(&c->d_rp, sizeof(int) * (T + 1)) == cudaSuccess &&
              cudaMalloc(&c->d_ci, sizeof(int) * (c->nnzb > 0 ? c->nnzb : 1)) == cudaSuccess &&
              cudaMalloc(&c->d_J, sizeof(vec8) * (size_t)c->nJ * c->nnzb * mm) == cudaSuccess &&
              cudaMalloc(&c->d_M, sizeof(vec8) * (size_t)T * mm) == cudaSuccess &&
              cudaMalloc(&c->d_V, sizeof(vec8) * (size_t)c->N * (R + 1)) == cudaSuccess &&
              cudaMalloc(&c->d_Z, sizeof(vec8) * (size_t)c->N * R) == cudaSuccess &&
              cudaMalloc(&c->d_x, sizeof(vec8) * (size_t)c->N) == cudaSuccess &&
              cudaMalloc(&c->d_rowctr, sizeof(int)) == cudaSuccess &&
              (c->df || !c->dfop || (cudaMalloc(&c->d_xdf, sizeof(vec8) * (size_t)c->N) == cudaSuccess &&
                                     cudaMalloc(&c->d_ydf, sizeof(vec8) * (size_t)c->N) == cudaSuccess)) &&
              cudaMalloc(&c->d_b, sizeof(vec8) * (size_t)c->N) == cudaSuccess &&
              cudaMalloc(&c->d_io, sizeof(double) * (size_t)c->N) == cudaSuccess &&
              cudaMalloc(&c->d_H, sizeof(double) * (R + 1) * R) == cudaSuccess &&
              cudaMalloc(&c->d_cs, sizeof(double) * R) == cudaSuccess &&
              cudaMalloc(&c->d_sn, sizeof(double) * R) == cudaSuccess &&
              cudaMalloc(&c->d_g, sizeof(double) * (R + 1)) == cudaSuccess &&
              cudaMalloc(&c->d_yls, sizeof(double) * R) == cudaSuccess &&
              cudaMalloc(&c->d_scal, IRK_SCAL_SLOTS * IRK_SCAL_BYTES) == cudaSuccess &&
              cudaMalloc(&c->d_part, sizeof(vec8) * IRK_PART_SLOTS) == cudaSuccess &&
              cudaMalloc(&c->d_ticket, 4 * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&c->d_err, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&c->d_vscale, 2 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->d_amax, 4 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMallocHost(&c->h_scal, 4 * IRK_SCAL_BYTES) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        return IRK_ERR_NOMEM;
    }
    c->d_gbar = c->d_ticket + 2;
    cudaMemsetAsync(c->d_ticket, 0, 4 * sizeof(unsigned int), c->stream);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    cudaMemsetAsync(c->d_scal, 0, IRK_SCAL_SLOTS * IRK_SCAL_BYTES, c->stream);
    cudaMemsetAsync(c->d_H, 0, sizeof(double) * (R + 1) * R, c->stream);
    cudaMemcpyAsync(c->d_rp, c->h_rp.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, c->stream);
    if (c->nnzb > 0)
        cudaMemcpyAsync(c->d_ci, c->h_ci.data(), sizeof(int) * c->nnzb, cudaMemcpyHostToDevice, c->stream);
    if ((rc = load_values(c, J, M, mem_space)) || (rc = pc_build_pattern(c))) {
        free_ctx(c);
        return rc;
    }
    if ((rc = cuda_status(cudaStreamSynchronize(c->stream)))) {
        free_ctx(c);
        return rc;
    }
    c->stats.levels_lower = c->pc.lo_ptr.empty() ? 0 : (int)c->pc.lo_ptr.size() - 1;
    c->stats.levels_upper = c->pc.up_ptr.empty() ? 0 : (int)c->pc.up_ptr.size() - 1;
    *out = c;
    return IRK_OK;
}

int irk_update_values(irk_ctx *c, const double *J, const double *M, int mem_space) {
    if (!c || !J || !M || (mem_space != IRK_HOST && mem_space != IRK_DEVICE)) return IRK_ERR_INVALID;
    c->factored = false;
    return load_values(c, J, M, mem_space);
}

// The factorisation's launches between two events; the caller synchronises
// (the error word must be clear before) and then calls factor_finish.
static int factor_enqueue(irk_ctx *c, double dt, cudaEvent_t e0, cudaEvent_t e1) {
    if (c->opt.timing != 2) c->tused = 0;
    cudaEventRecord(e0, c->stream);
    const int rc = pc_factor(c, dt);
    cudaEventRecord(e1, c->stream);
    return rc;
}

// After a synchronisation covering the factorisation; rc is its outcome.
static void factor_finish(irk_ctx *c, double dt, int rc, cudaEvent_t e0, cudaEvent_t e1, long long l0) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c->opt.timing != 2) tcollect_factor(c);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->stats.factor_ms = ms;
    c->stats.kernel_launches = c->launches - l0;
    c->factored = (rc == IRK_OK);
    c->factored_dt = dt;
}

int irk_factor(irk_ctx *c, double dt) {
    if (!c || !dt_ok(c, dt)) return IRK_ERR_INVALID;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const long long l0 = c->launches;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    int rc = factor_enqueue(c, dt, e0, e1);
    if (rc == IRK_OK) rc = sync_err(c);
    factor_finish(c, dt, rc, e0, e1, l0);
    return rc;
}

int irk_apply_operator(irk_ctx *c, const double *X, double *Y, double dt, int mem_space) {
    if (!c || !X || !Y || !dt_ok(c, dt)) return IRK_ERR_INVALID;
    vec8 *xi = c->d_V, *yi = c->d_V + c->N;
    int rc = IRK_OK;
    const double *sc = nullptr;
    if ((rc = copy_in(c->d_io, X, sizeof(double) * c->N, mem_space, c->stream)) ||
        ((sc = rhs_scale(c, &rc)), rc) ||
        (rc = launch_to_internal(c, c->d_io, xi, sc)) || (rc = launch_matvec(c, xi, yi, nullptr, dt, 0)) ||
        (rc = launch_to_external(c, yi, c->d_io, sc)) ||
        (rc = copy_out(Y, c->d_io, sizeof(double) * c->N, mem_space, c->stream)))
        return rc;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

int irk_apply_precond(irk_ctx *c, const double *V, double *Z, int mem_space) {
    if (!c || !V || !Z) return IRK_ERR_INVALID;
    if (!c->factored && c->opt.precond != IRK_PC_NONE) return IRK_ERR_STATE;
    vec8 *vi = c->d_V, *zi = c->d_Z;
    int rc = IRK_OK;
    const double *sc = nullptr;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if ((rc = copy_in(c->d_io, V, sizeof(double) * c->N, mem_space, c->stream)) ||
        ((sc = rhs_scale(c, &rc)), rc) ||
        (rc = launch_to_internal(c, c->d_io, vi, sc)) || (rc = pc_apply(c, vi, zi)) ||
        (rc = launch_to_external(c, zi, c->d_io, sc)) ||
        (rc = copy_out(Z, c->d_io, sizeof(double) * c->N, mem_space, c->stream)))
        return rc;
    return sync_err(c);
}

int irk_solve(irk_ctx *c, const double *Rhs, double dt, double rtol, double *W, int mem_space, int *iters,
              double *relres) {
    if (!c || !Rhs || !W || !(rtol >= 0.0) || !dt_ok(c, dt)) return IRK_ERR_INVALID;
    int rc;
    const long long l0 = c->launches;  // counts the refactorisation too, if any
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    cudaMemsetAsync(c->d_gbar, 0, 2 * sizeof(unsigned int), c->stream);
    // a refactorisation is enqueued ahead of the solve; the synchronisation
    // that reads ||R|| below also reports its errors (no round trip of its own)
    const bool refactor = c->opt.precond != IRK_PC_NONE && (!c->factored || c->factored_dt != dt);
    // a host R is copied on a second stream during the refactorisation
    bool r_in = false;
    if (refactor && mem_space == IRK_HOST) {
        if (!c->in_stream && cudaStreamCreateWithFlags(&c->in_stream, cudaStreamNonBlocking) != cudaSuccess)
            c->in_stream = nullptr;
        if (c->in_stream && !c->in_ev && cudaEventCreateWithFlags(&c->in_ev, cudaEventDisableTiming) != cudaSuccess)
            c->in_ev = nullptr;
        if (c->in_stream && c->in_ev) {
            if ((rc = copy_in(c->d_io, Rhs, sizeof(double) * c->N, mem_space, c->in_stream))) return rc;
            cudaEventRecord(c->in_ev, c->in_stream);
            r_in = true;
        }
    }
    cudaEvent_t fe0 = nullptr, fe1 = nullptr;
    if (refactor) {
        cudaEventCreate(&fe0);
        cudaEventCreate(&fe1);
        if ((rc = factor_enqueue(c, dt, fe0, fe1))) {
            cudaStreamSynchronize(c->stream);
            if (r_in) cudaStreamSynchronize(c->in_stream);
            factor_finish(c, dt, rc, fe0, fe1, l0);
            return rc;
        }
    }
    if (r_in) cudaStreamWaitEvent(c->stream, c->in_ev, 0);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    if (c->opt.timing != 2 && !refactor) c->tused = 0;
    const long long N = c->N;
    const int Rs = c->opt.restart;
    double *est_h = c->h_scal, *beta_h = c->h_scal + 1, *hn_h = c->h_scal + 2;
    int total = 0, cycles = 0;
    double bnorm = 0.0, beta = 0.0;
    rc = r_in ? IRK_OK : copy_in(c->d_io, Rhs, sizeof(double) * N, mem_space, c->stream);
    const double *sc = nullptr;
    if (!rc) sc = rhs_scale(c, &rc);
    if (!rc) rc = launch_to_internal(c, c->d_io, c->d_b, sc);
    if (!rc) rc = launch_axpy_dot_slot(c, c->d_b, nullptr, 0, nullptr, 1, 1, 0, nullptr);
    if (!rc) rc = cuda_status(cudaMemcpyAsync(beta_h, irk_beta_ptr(c), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (!rc) rc = sync_err(c);
    if (refactor) {
        factor_finish(c, dt, rc, fe0, fe1, l0);
        if (rc) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
        }
    }
    if (!rc) rc = launch_fill_zero(c, c->d_x, N);
    bnorm = *beta_h;
    if (!rc && !std::isfinite(bnorm)) rc = IRK_ERR_NONFINITE;
    bool x_zero = true;
    // binary32 factors write binary32-valued z_j = P^{-1} v_j (double-float
    // with zero low words): their operator products skip those words
    const int z_f32 = c->dfop && c->pc.kind != IRK_PC_NONE && c->fprec != IRK_FACTOR_FP64;
    while (rc == IRK_OK && bnorm > 0.0) {
        vec8 *V0 = c->d_V;
        if (x_zero) {
            // x = 0: the residual is R itself and its norm, in slot 0, is ||R||
            // (the same kernel on the same data as the true-residual path)
            if ((rc = cuda_status(
                     cudaMemcpyAsync(V0, c->d_b, sizeof(vec8) * N, cudaMemcpyDeviceToDevice, c->stream))))
                break;
            beta = bnorm;
            x_zero = false;
        } else {
            if ((rc = launch_matvec(c, c->d_x, V0, c->d_b, dt, 1))) break;
            if ((rc = launch_axpy_dot_slot(c, V0, nullptr, 0, nullptr, 1, 1, 0, nullptr))) break;
            cudaMemcpyAsync(beta_h, irk_beta_ptr(c), sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            if ((rc = sync_err(c))) break;
            beta = *beta_h;
        }
        if (!std::isfinite(beta)) {
            rc = IRK_ERR_NONFINITE;
            break;
        }
        if (beta <= rtol * bnorm) break;
        if (total >= c->opt.max_iter) {
            rc = IRK_NOT_CONVERGED;
            break;
        }
        ++cycles;
        if ((rc = launch_cycle_start(c, Rs)) || (rc = launch_scale_slot(c, V0, 0))) break;
        int jl = -1;
        for (int j = 0; j < Rs; ++j) {
            vec8 *Vj = c->d_V + (long long)j * N, *Zj = c->d_Z + (long long)j * N, *w = Vj + N;
            int tm = tmark_begin(c);
            if ((rc = pc_apply(c, Vj, Zj))) break;
            tmark_end(c, tm, 1);
            tm = tmark_begin(c);
            if ((rc = launch_matvec(c, Zj, w, nullptr, dt, 0, z_f32))) break;
            tmark_end(c, tm, 0);
            tm = tmark_begin(c);
            rc = launch_arnoldi(c, j, Rs, w);
            const bool one_launch = rc != IRK_ERR_INVALID;
            if (rc == IRK_ERR_INVALID) {
                // no cooperative launch: one launch per Gram-Schmidt step
                rc = IRK_OK;
                for (int i = 0; i <= j && !rc; ++i)
                    rc = launch_axpy_dot_slot(c, w, i > 0 ? c->d_V + (long long)(i - 1) * N : nullptr, 2 + i - 1,
                                              c->d_V + (long long)i * N, 0, 0, 2 + i, c->d_H + i * Rs + j);
                if (rc) break;
                if ((rc = launch_axpy_dot_slot(c, w, Vj, 2 + j, nullptr, 1, 1, 2 + j + 1,
                                               c->d_H + (j + 1) * Rs + j)))
                    break;
                if ((rc = launch_scale_slot(c, w, 2 + j + 1)) || (rc = launch_givens(c, j, Rs))) break;
            }
            if (rc) break;
            tmark_end(c, tm, 2);
            ++total;
            jl = j;
            // residual estimate and h_{j+1,j} (kept in its scalar slot: the
            // rotation zeroes H[j+1][j]) for the stopping and breakdown tests;
            // the one-launch step leaves them with the error word in one block
            if (one_launch) {
                double *st = c->h_scal + 8;
                if ((rc = cuda_status(cudaMemcpyAsync(st, irk_status_ptr(c), 3 * sizeof(double),
                                                      cudaMemcpyDeviceToHost, c->stream))) ||
                    (rc = cuda_status(cudaStreamSynchronize(c->stream))) || (rc = err_code((int)st[2])))
                    break;
                *est_h = st[0];
                *hn_h = st[1];
            } else {
                cudaMemcpyAsync(est_h, irk_est_ptr(c), sizeof(double), cudaMemcpyDeviceToHost, c->stream);
                cudaMemcpyAsync(hn_h, reinterpret_cast<char *>(c->d_scal) + (size_t)(2 + j + 1) * IRK_SCAL_BYTES,
                                sizeof(double), cudaMemcpyDeviceToHost, c->stream);
                if ((rc = sync_err(c))) break;
            }
            if (*est_h <= rtol * bnorm || total >= c->opt.max_iter || *hn_h == 0.0) break;
        }
        if (rc) break;
        if (jl >= 0 && (rc = launch_lsq_update(c, jl, Rs))) break;
    }
    if (rc == IRK_OK || rc == IRK_NOT_CONVERGED) {
        int rc2;
        if ((rc2 = launch_to_external(c, c->d_x, c->d_io, sc)) ||
            (rc2 = copy_out(W, c->d_io, sizeof(double) * N, mem_space, c->stream)) ||
            (rc2 = cuda_status(cudaStreamSynchronize(c->stream))))
            rc = rc2;
    }
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (c->opt.timing != 2) tcollect(c);
    c->stats.iters = total;
    c->stats.cycles = cycles;
    c->stats.relres = bnorm > 0.0 ? beta / bnorm : 0.0;
    c->stats.solve_ms = ms;
    c->stats.kernel_launches = c->launches - l0;
    if (iters) *iters = total;
    if (relres) *relres = c->stats.relres;
    return rc;
}

// Step outputs (Sec. 4.1) on the stage-major boundary layout, binary64:
// K[k] = sum_l Ainv[k][l] W[l], u1 = u0 + dt sum_l wt[l] W[l] (l increasing).
struct StepCoef {
    double Ainv[IRK_MAX_S * IRK_MAX_S];
    double wt[IRK_MAX_S];
};

__global__ void k_step_outputs(long long n, int s, const double *__restrict__ W, StepCoef cf,
                               const double *__restrict__ u0, double dt, double *K, double *u1) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double w[IRK_MAX_S];
        for (int l = 0; l < s; ++l) w[l] = W[l * n + e];
        if (K)
            for (int k = 0; k < s; ++k) {
                double acc = 0.0;
                for (int l = 0; l < s; ++l) acc = fma(cf.Ainv[k * s + l], w[l], acc);
                K[k * n + e] = acc;
            }
        if (u1) {
            double acc = 0.0;
            for (int l = 0; l < s; ++l) acc = fma(cf.wt[l], w[l], acc);
            u1[e] = fma(dt, acc, u0[e]);
        }
    }
}

static int launch_step_outputs(irk_ctx *c, const double *W, const double *wt, const double *u0, double dt,
                               double *K, double *u1) {
    StepCoef cf;
    memset(&cf, 0, sizeof(cf));
    for (int q = 0; q < c->s * c->s; ++q) cf.Ainv[q] = c->Ainv[q];
    for (int l = 0; l < c->s; ++l) cf.wt[l] = wt[l];
    const long long n = (long long)c->T * c->m;
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    k_step_outputs<<<(int)std::max(1LL, g), 256, 0, c->stream>>>(n, c->s, W, cf, u0, dt, K, u1);
    c->launches++;
    return cuda_status(cudaGetLastError());
}

int irk_step_outputs(irk_ctx *c, const double *W, const double *b, const double *u0, double dt, double *K,
                     double *u1, int mem_space) {
    if (!c || !W || (u1 && !u0) || !std::isfinite(dt) || (mem_space != IRK_HOST && mem_space != IRK_DEVICE))
        return IRK_ERR_INVALID;
    const int s = c->s;
    // weights b^T A^{-1}; a stiffly accurate tableau (b = last row of A) has e_s^T exactly
    double wt[IRK_MAX_S];
    for (int l = 0; l < s; ++l) wt[l] = 0.0;
    if (!b) {
        wt[s - 1] = 1.0;
    } else {
        for (int l = 0; l < s; ++l)
            for (int j = 0; j < s; ++j) wt[l] += b[j] * c->Ainv[j * s + l];
    }
    const long long N = c->N, n = (long long)c->T * c->m;
    if (mem_space == IRK_DEVICE) {
        int rc = launch_step_outputs(c, W, wt, u0, dt, K, u1);
        if (rc == IRK_OK) rc = cuda_status(cudaStreamSynchronize(c->stream));
        return rc;
    }
    // host buffers: W, u0 in and K, u1 out through one device temporary
    double *tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(double) * (size_t)(2 * N + 2 * n)) != cudaSuccess) return IRK_ERR_NOMEM;
    double *dW = tmp, *dK = tmp + N, *du0 = tmp + 2 * N, *du1 = tmp + 2 * N + n;
    int rc = cuda_status(cudaMemcpyAsync(dW, W, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream));
    if (rc == IRK_OK && u1)
        rc = cuda_status(cudaMemcpyAsync(du0, u0, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    if (rc == IRK_OK) rc = launch_step_outputs(c, dW, wt, u1 ? du0 : nullptr, dt, K ? dK : nullptr, u1 ? du1 : nullptr);
    if (rc == IRK_OK && K) rc = cuda_status(cudaMemcpyAsync(K, dK, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    if (rc == IRK_OK && u1)
        rc = cuda_status(cudaMemcpyAsync(u1, du1, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    const int rs = cuda_status(cudaStreamSynchronize(c->stream));
    cudaFree(tmp);
    return rc != IRK_OK ? rc : rs;
}

void irk_default_kernel_options(irk_kernel_options *ko) {
    if (!ko) return;
    ko->matvec_variant = -1;
    ko->sweep_two_colour = 1;
    ko->sweep_compiled_levels = 1;
    ko->sweep_shared_upper = 1;
    ko->factor_fused = 2;
    ko->factor_gj_rows = 1;
    ko->factor_gj_threads = 0;
    ko->factor_gj_split_min = 0;
    ko->arnoldi_form = 0;
}

int irk_set_kernel_options(irk_ctx *c, const irk_kernel_options *ko) {
    if (!c || !ko) return IRK_ERR_INVALID;
    if (ko->matvec_variant < -1 || ko->matvec_variant >= irk_matvec_variants() || ko->sweep_two_colour < 0 ||
        ko->sweep_two_colour > 1 || ko->sweep_shared_upper < 0 || ko->sweep_shared_upper > 1 ||
        ko->sweep_compiled_levels < 0 || ko->sweep_compiled_levels > 1 ||
        ko->factor_fused < 0 || ko->factor_fused > 2 || ko->factor_gj_rows < 0 || ko->factor_gj_rows > 1 ||
        (ko->factor_gj_threads != 0 && (ko->factor_gj_threads < 32 || ko->factor_gj_threads > 256)) ||
        ko->factor_gj_split_min < 0 || ko->arnoldi_form < 0 || ko->arnoldi_form > 2)
        return IRK_ERR_INVALID;
    c->ko = *ko;
    c->mv_variant = -1;  // re-chosen (or pinned) at the next product
    return IRK_OK;
}

int irk_set_spin_limit(irk_ctx *c, int spin_limit) {
    if (!c || spin_limit < 0) return IRK_ERR_INVALID;
    c->opt.spin_limit = spin_limit;
    c->spin = spin_limit > 0 ? spin_limit : IRK_DEFAULT_SPIN_LIMIT;
    return IRK_OK;
}

int irk_set_timing(irk_ctx *c, int timing) {
    if (!c || timing < 0 || timing > 2) return IRK_ERR_INVALID;
    if (c->opt.timing == 2 && timing != 2) {
        // keep what was recorded in the running totals (read at the next
        // irk_get_stats under timing = 2)
        cudaStreamSynchronize(c->stream);
        tflush(c);
    }
    if (c->opt.timing == 1 && timing != 1) c->tused = 0;
    c->opt.timing = timing;
    return IRK_OK;
}

int irk_get_stats(const irk_ctx *cc, irk_stats *out) {
    if (!cc || !out) return IRK_ERR_INVALID;
    if (cc->opt.timing == 2) {
        // deferred marks: read every pending event pair now (the context's
        // own timing state; the object itself is never const)
        irk_ctx *c = const_cast<irk_ctx *>(cc);
        cudaStreamSynchronize(c->stream);
        treport(c);
        c->stats.kernel_launches = c->launches - c->launches_at_stats;
        c->launches_at_stats = c->launches;
    }
    const irk_ctx *c = cc;
    *out = c->stats;
    out->matvec_variant = c->mv_variant;
    return IRK_OK;
}

void irk_destroy(irk_ctx *c) {
    if (c) {
        cudaStreamSynchronize(c->stream);
        if (c->in_stream) {
            cudaStreamSynchronize(c->in_stream);
            cudaStreamDestroy(c->in_stream);
        }
        if (c->in_ev) cudaEventDestroy(c->in_ev);
    }
    free_ctx(c);
}

}  // extern "C"
