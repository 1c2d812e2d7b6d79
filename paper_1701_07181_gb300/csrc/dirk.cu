// dirk.cu -- diagonally implicit Runge-Kutta steps on the stage-system
// machinery (Sec. 3: the DIRK comparison schemes, App. A tableaux).
//
// Stage k of a lower-triangular tableau solves one n x n system
//     (M - dt a_kk J) k_k = J (u0 + dt sum_{j<k} a_kj k_j)
// with a single-stage context (s = 1, A = [[a_kk]], untransformed form, so
// its operator is M - dt a_kk J and its coupled preconditioner the block
// ILU(0) of that matrix).  Stages sharing a_kk share the context and so one
// factorisation per dt.  An explicit stage (a_kk = 0) solves M k_k = J u0
// with a context whose operator is M (A = [[1]], dt = 0: its ILU(0) is the
// exact block factorisation of M, factored once).  The right-hand sides are
// formed on the device: an FP64 linear combination of u0 and the previous
// stages, then the Jacobian product in the contexts' arithmetic.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "irk_internal.h"

struct irk_dirk {
    int s = 0, T = 0, m = 0;
    long long n = 0;
    double A[IRK_MAX_S * IRK_MAX_S];
    double b[IRK_MAX_S];
    std::vector<irk_ctx *> ctx;  // one per distinct nonzero a_kk
    irk_ctx *mass = nullptr;     // explicit stages (operator M)
    int stage_ctx[IRK_MAX_S];    // index into ctx, -1 = explicit stage
    cudaStream_t stream = nullptr;
    double *d_u0 = nullptr, *d_K = nullptr, *d_v = nullptr, *d_rhs = nullptr, *d_u1 = nullptr;
};

namespace {

struct Comb {
    double c[IRK_MAX_S];
};

// out = base + sum_{j < nk} c_j K_j (binary64)
__global__ void k_dirk_combine(long long n, int nk, const double *__restrict__ base, const double *__restrict__ K,
                               Comb c, double *__restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double v = base[e];
        for (int j = 0; j < nk; ++j) v = fma(c.c[j], K[(long long)j * n + e], v);
        out[e] = v;
    }
}

int grid_for_n(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1LL, std::min(g, 152LL * 8));
}

void free_dirk(irk_dirk *d) {
    if (!d) return;
    for (irk_ctx *c : d->ctx) irk_destroy(c);
    if (d->mass) irk_destroy(d->mass);
    cudaFree(d->d_u0);
    cudaFree(d->d_K);
    cudaFree(d->d_v);
    cudaFree(d->d_rhs);
    cudaFree(d->d_u1);
    delete d;
}

}  // namespace

extern "C" {

int irk_dirk_setup(irk_dirk **out, int s, const double *A, const double *b, int T, int m, const int32_t *row_ptr,
                   const int32_t *col_idx, const double *J, const double *M, int mem_space, const irk_options *opt) {
    if (!out || !A || !b || s < 1 || s > IRK_MAX_S || T < 1 || m < 1) return IRK_ERR_INVALID;
    *out = nullptr;
    for (int k = 0; k < s; ++k) {
        if (!(A[k * s + k] >= 0.0) || !std::isfinite(A[k * s + k]) || !std::isfinite(b[k])) return IRK_ERR_INVALID;
        for (int j = 0; j < s; ++j) {
            if (j > k && A[k * s + j] != 0.0) return IRK_ERR_INVALID;
            if (!std::isfinite(A[k * s + j])) return IRK_ERR_INVALID;
        }
    }
    irk_dirk *d = new irk_dirk();
    d->s = s;
    d->T = T;
    d->m = m;
    d->n = (long long)T * m;
    memcpy(d->A, A, sizeof(double) * s * s);
    memcpy(d->b, b, sizeof(double) * s);
    irk_options o;
    irk_default_options(&o);
    if (opt) o = *opt;
    o.formulation = IRK_UNTRANSFORMED;
    o.precond = (opt && opt->precond == IRK_PC_NONE) ? IRK_PC_NONE : IRK_PC_COUPLED;
    o.shift = nullptr;
    o.stage_jacobians = 0;
    d->stream = (cudaStream_t)o.stream;
    std::vector<double> gam;
    int rc = IRK_OK;
    for (int k = 0; k < s && rc == IRK_OK; ++k) {
        const double g = A[k * s + k];
        if (g == 0.0) {
            d->stage_ctx[k] = -1;
            if (!d->mass) {
                const double one = 1.0;
                rc = irk_setup(&d->mass, 1, &one, T, m, row_ptr, col_idx, J, M, mem_space, &o);
            }
            continue;
        }
        int idx = -1;
        for (size_t q = 0; q < gam.size(); ++q)
            if (gam[q] == g) idx = (int)q;
        if (idx < 0) {
            irk_ctx *c = nullptr;
            rc = irk_setup(&c, 1, &g, T, m, row_ptr, col_idx, J, M, mem_space, &o);
            if (rc) break;
            gam.push_back(g);
            d->ctx.push_back(c);
            idx = (int)gam.size() - 1;
        }
        d->stage_ctx[k] = idx;
    }
    if (rc == IRK_OK) {
        const size_t nb = sizeof(double) * (size_t)d->n;
        if (cudaMalloc(&d->d_u0, nb) != cudaSuccess || cudaMalloc(&d->d_K, nb * s) != cudaSuccess ||
            cudaMalloc(&d->d_v, nb) != cudaSuccess || cudaMalloc(&d->d_rhs, nb) != cudaSuccess ||
            cudaMalloc(&d->d_u1, nb) != cudaSuccess)
            rc = IRK_ERR_NOMEM;
    }
    if (rc != IRK_OK) {
        free_dirk(d);
        return rc;
    }
    *out = d;
    return IRK_OK;
}

int irk_dirk_step(irk_dirk *d, const double *u0, double dt, double rtol, double *u1, double *K, int mem_space,
                  int *iters, double *relres) {
    if (!d || !u0 || !u1 || !(dt > 0.0) || !(rtol > 0.0) || (mem_space != IRK_HOST && mem_space != IRK_DEVICE))
        return IRK_ERR_INVALID;
    const long long n = d->n;
    const size_t nb = sizeof(double) * (size_t)n;
    cudaStream_t st = d->stream;
    const cudaMemcpyKind hin = mem_space == IRK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind hout = mem_space == IRK_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int rc = cuda_status(cudaMemcpyAsync(d->d_u0, u0, nb, hin, st));
    double worst = 0.0;
    bool not_conv = false;
    // the Jacobian product runs in the first available context's arithmetic
    irk_ctx *jc = d->ctx.empty() ? d->mass : d->ctx[0];
    for (int k = 0; k < d->s && rc == IRK_OK; ++k) {
        Comb cb;
        for (int j = 0; j < k; ++j) cb.c[j] = dt * d->A[k * d->s + j];
        k_dirk_combine<<<grid_for_n(n), 256, 0, st>>>(n, k, d->d_u0, d->d_K, cb, d->d_v);
        if ((rc = cuda_status(cudaGetLastError()))) break;
        // rhs = J v through the context's internal layout (s = 1: same order)
        if ((rc = launch_to_internal(jc, d->d_v, jc->d_x)) || (rc = launch_jacobian(jc, jc->d_x, jc->d_V)) ||
            (rc = launch_to_external(jc, jc->d_V, d->d_rhs)))
            break;
        irk_ctx *c = d->stage_ctx[k] < 0 ? d->mass : d->ctx[d->stage_ctx[k]];
        const double sdt = d->stage_ctx[k] < 0 ? 0.0 : dt;
        int it = 0;
        double rr = 0.0;
        const int r = irk_solve(c, d->d_rhs, sdt, rtol, d->d_K + (long long)k * n, IRK_DEVICE, &it, &rr);
        if (r == IRK_NOT_CONVERGED) {
            not_conv = true;
        } else if (r != IRK_OK) {
            rc = r;
            break;
        }
        if (iters) iters[k] = d->stage_ctx[k] < 0 ? 0 : it;
        worst = std::max(worst, rr);
    }
    if (rc == IRK_OK) {
        Comb cb;
        for (int k = 0; k < d->s; ++k) cb.c[k] = dt * d->b[k];
        k_dirk_combine<<<grid_for_n(n), 256, 0, st>>>(n, d->s, d->d_u0, d->d_K, cb, d->d_u1);
        rc = cuda_status(cudaGetLastError());
    }
    if (rc == IRK_OK) rc = cuda_status(cudaMemcpyAsync(u1, d->d_u1, nb, hout, st));
    if (rc == IRK_OK && K) rc = cuda_status(cudaMemcpyAsync(K, d->d_K, nb * d->s, hout, st));
    if (rc == IRK_OK) rc = cuda_status(cudaStreamSynchronize(st));
    if (relres) *relres = worst;
    if (rc == IRK_OK && not_conv) rc = IRK_NOT_CONVERGED;
    return rc;
}

void irk_dirk_destroy(irk_dirk *d) {
    if (d && d->stream) cudaStreamSynchronize(d->stream);
    free_dirk(d);
}

}  // extern "C"
