/*
 * irk_oracle.c -- plain, serial, FP64 reference of the per-time-step linear
 * solve of the coupled s-stage implicit Runge-Kutta system of Pazner & Persson,
 * "Stage-parallel fully implicit Runge-Kutta solvers for discontinuous Galerkin
 * fluid simulations" (arXiv 1701.07181).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg call it; the library's CUDA path never links, loads or
 * calls this file, and the two share no code, header or table.
 *
 * Everything here is the plain definition or the algorithm's steps in the
 * paper's order: no blocking, fusion or reordering.  Each function cites the
 * section / equation / algorithm it follows.
 *
 * Conventions (all matrices row-major, all values double):
 *   T elements, m dofs per element, n = T*m, s stages (Sec. 2.1, Sec. 3).
 *   Jacobian J: block-CSR with T block rows: row_ptr[T+1], col_idx[nnzb]
 *     (column indices sorted, diagonal present), vals[nnzb*m*m].
 *     Stage k uses J + k*jstride (jstride = 0: one Jacobian shared by all
 *     stages; jstride = nnzb*m*m: one Jacobian J_k per stage, Sec. 4.1).
 *   Mass matrix M: T diagonal blocks, M[T*m*m] (Sec. 2.1).
 *   Stage vectors are stacked stage-major, X[(k*T + i)*m + a], the stacking
 *   (x_1, ..., x_s) of Sec. 4.1.
 *
 * Return codes: 0 ok, 1 not converged, -1 bad argument, -2 out of memory,
 * -3 singular diagonal block, -4 non-finite value.
 *
 * Multi-core build.  Compiled with -fopenmp (libirk_oracle_omp.so) the same
 * source spreads independent work over threads: the operator's block rows
 * (every (stage, element) row of Sec. 4.1 is computed on its own), the
 * stages of the uncoupled preconditioner (the s independent factorisations
 * and sweeps of Sec. 4.3.2, the paper's stage parallelism of Sec. 4.5), the
 * element blocks of its assembly, and the vector operations and inner
 * products of FGMRES.  Every row, block and factor is computed by the same
 * operations in the same order as in the serial build; only the inner
 * products' partial sums are added in a different order.  Without
 * -fopenmp (libirk_oracle.so, the build the tests check) the pragmas are
 * ignored and everything runs serially.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REF_OK 0
#define REF_NOT_CONVERGED 1
#define REF_EINVAL (-1)
#define REF_ENOMEM (-2)
#define REF_SINGULAR (-3)
#define REF_NONFINITE (-4)

/* ------------------------------------------------------------------------ */
/* Dense helpers (n x n, row-major).                                        */
/* ------------------------------------------------------------------------ */

/* LU factorisation with partial pivoting, P a = L U, in place (unit L below
 * the diagonal, U on and above it); piv[k] is the row swapped with row k at
 * step k.  Returns 0, or REF_SINGULAR on an exactly zero pivot. */
static int lu_factor(int n, double *a, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            if (fabs(a[i * n + k]) > best) {
                best = fabs(a[i * n + k]);
                p = i;
            }
        }
        piv[k] = p;
        if (best == 0.0) return REF_SINGULAR;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = a[k * n + j];
                a[k * n + j] = a[p * n + j];
                a[p * n + j] = t;
            }
        }
        for (int i = k + 1; i < n; ++i) {
            double l = a[i * n + k] / a[k * n + k];
            a[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
        }
    }
    return REF_OK;
}

/* Solve a x = b in place (x holds b on entry) from the factors of lu_factor. */
static void lu_solve(int n, const double *lu, const int *piv, double *x)
{
    for (int k = 0; k < n; ++k) {
        if (piv[k] != k) {
            double t = x[k];
            x[k] = x[piv[k]];
            x[piv[k]] = t;
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) x[i] -= lu[i * n + j] * x[j];
    for (int i = n - 1; i >= 0; --i) {
        for (int j = i + 1; j < n; ++j) x[i] -= lu[i * n + j] * x[j];
        x[i] /= lu[i * n + i];
    }
}

/* inv = a^{-1}, column by column from the pivoted LU of a. */
static int invert(int n, const double *a, double *inv)
{
    double *lu = (double *)malloc(sizeof(double) * n * n);
    int *piv = (int *)malloc(sizeof(int) * n);
    double *col = (double *)malloc(sizeof(double) * n);
    if (!lu || !piv || !col) {
        free(lu); free(piv); free(col);
        return REF_ENOMEM;
    }
    memcpy(lu, a, sizeof(double) * n * n);
    int rc = lu_factor(n, lu, piv);
    if (rc == REF_OK) {
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i) col[i] = (i == j) ? 1.0 : 0.0;
            lu_solve(n, lu, piv, col);
            for (int i = 0; i < n; ++i) inv[i * n + j] = col[i];
        }
    }
    free(lu); free(piv); free(col);
    return rc;
}

/* c = a * b */
static void mat_mul(int n, const double *a, const double *b, double *c)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += a[i * n + k] * b[k * n + j];
            c[i * n + j] = acc;
        }
}

/* c -= a * b */
static void mat_mul_sub(int n, const double *a, const double *b, double *c)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += a[i * n + k] * b[k * n + j];
            c[i * n + j] -= acc;
        }
}

/* y += alpha * a * x */
static void mat_vec_add(int n, double alpha, const double *a, const double *x, double *y)
{
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += a[i * n + j] * x[j];
        y[i] += alpha * acc;
    }
}

/* Position of block (i, j) in a block-CSR pattern, or -1. */
static long find_block(const int *row_ptr, const int *col_idx, int i, int j)
{
    for (long p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
        if (col_idx[p] == j) return p;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Stage-system operators.                                                  */
/* ------------------------------------------------------------------------ */

/* Transformed operator of Sec. 4.1 (eq. modified-IRK and its Newton system,
 * eq. big-irk):  Y = (A^{-1} (x) M - dt diag(J_1..J_s)) X, i.e. for stage k,
 * element i:
 *     Y_{k,i} = sum_l (A^{-1})_{kl} M_i X_{l,i} - dt sum_j (J_k)_{ij} X_{k,j}. */
int irk_ref_apply_transformed(int s, const double *Ainv, int T, int m,
                              const int *row_ptr, const int *col_idx,
                              const double *J, long jstride, const double *M,
                              double dt, const double *X, double *Y)
{
    if (s < 1 || T < 0 || m < 1) return REF_EINVAL;
    long n = (long)T * m;
    long mm = (long)m * m;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < s; ++k) {
        for (int i = 0; i < T; ++i) {
            const double *Jk = J + k * jstride;
            double *y = Y + k * n + (long)i * m;
            for (int a = 0; a < m; ++a) y[a] = 0.0;
            for (int l = 0; l < s; ++l)
                mat_vec_add(m, Ainv[k * s + l], M + i * mm, X + l * n + (long)i * m, y);
            for (long p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                mat_vec_add(m, -dt, Jk + p * mm, X + k * n + (long)col_idx[p] * m, y);
        }
    }
    return REF_OK;
}

/* Untransformed operator of Sec. 4.1 (eq. newton-system-2):
 *     Y = (I_s (x) M - dt [a_{kl} J_k]) K, i.e.
 *     Y_{k,i} = M_i K_{k,i} - dt sum_l a_{kl} sum_j (J_k)_{ij} K_{l,j}. */
int irk_ref_apply_untransformed(int s, const double *A, int T, int m,
                                const int *row_ptr, const int *col_idx,
                                const double *J, long jstride, const double *M,
                                double dt, const double *K, double *Y)
{
    if (s < 1 || T < 0 || m < 1) return REF_EINVAL;
    long n = (long)T * m;
    long mm = (long)m * m;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < s; ++k) {
        for (int i = 0; i < T; ++i) {
            const double *Jk = J + k * jstride;
            double *y = Y + k * n + (long)i * m;
            for (int a = 0; a < m; ++a) y[a] = 0.0;
            mat_vec_add(m, 1.0, M + i * mm, K + k * n + (long)i * m, y);
            for (int l = 0; l < s; ++l)
                for (long p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                    mat_vec_add(m, -dt * A[k * s + l], Jk + p * mm,
                                K + l * n + (long)col_idx[p] * m, y);
        }
    }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Block ILU(0), Sec. 4.2.1.                                                */
/* ------------------------------------------------------------------------ */

/* Generic block ILU(0) of a block-CSR matrix (nb block rows, b x b blocks),
 * in place, in the textbook row-by-row (IKJ) form: the standard block LU
 * factorisation with every block outside the pattern discarded (Sec. 4.2.1).
 * For each block row j, for each pattern column i < j in increasing order:
 *     B_ji <- B_ji B_ii^{-1};   B_jk <- B_jk - B_ji B_ik  for pattern k > i
 *                               with (i, k) also in the pattern.
 * On return the strict lower blocks hold L~ (unit diagonal implied), the
 * diagonal and upper blocks hold U~, and dlu / dpiv hold the pivoted LU
 * factors of each diagonal block U~_jj (used by irk_ref_bilu0_apply).
 * Under the condition of Alg. 2 (no two neighbours of an element are
 * neighbours) this equals Alg. 1 and Alg. 2; where it fails it also performs
 * the updates i < k < j that Alg. 1 as printed omits (textbook form). */
int irk_ref_bilu0(int nb, int b, const int *row_ptr, const int *col_idx,
                  double *vals, double *dlu, int *dpiv)
{
    long bb = (long)b * b;
    /* inv + i*bb holds B_ii^{-1} once row i is complete (B_ii is then final). */
    double *inv = (double *)malloc(sizeof(double) * bb * (nb > 0 ? nb : 1));
    double *tmp = (double *)malloc(sizeof(double) * bb);
    if (!inv || !tmp) { free(inv); free(tmp); return REF_ENOMEM; }
    int rc = REF_OK;
    for (int j = 0; j < nb && rc == REF_OK; ++j) {
        for (long p = row_ptr[j]; p < row_ptr[j + 1]; ++p) {
            int i = col_idx[p];
            if (i >= j) break;
            mat_mul(b, vals + p * bb, inv + i * bb, tmp);
            memcpy(vals + p * bb, tmp, sizeof(double) * bb);
            for (long q = p + 1; q < row_ptr[j + 1]; ++q) {
                int k = col_idx[q];
                long pik = find_block(row_ptr, col_idx, i, k);
                if (pik >= 0) mat_mul_sub(b, vals + p * bb, vals + pik * bb, vals + q * bb);
            }
        }
        if (rc != REF_OK) break;
        long pjj = find_block(row_ptr, col_idx, j, j);
        if (pjj < 0) { rc = REF_EINVAL; break; }
        rc = invert(b, vals + pjj * bb, inv + j * bb);
        if (rc != REF_OK) break;
        memcpy(dlu + j * bb, vals + pjj * bb, sizeof(double) * bb);
        rc = lu_factor(b, dlu + j * bb, dpiv + (long)j * b);
    }
    free(inv);
    free(tmp);
    return rc;
}

/* Apply the factors of irk_ref_bilu0: z = (L~ U~)^{-1} v.  Forward sweep with
 * the unit lower factor, then backward sweep with the block upper factor,
 * the diagonal blocks solved by their pivoted LU (Sec. 4.2.1). */
void irk_ref_bilu0_apply(int nb, int b, const int *row_ptr, const int *col_idx,
                         const double *vals, const double *dlu, const int *dpiv,
                         const double *v, double *z)
{
    long bb = (long)b * b;
    /* forward: y_j = v_j - sum_{i<j} L_ji y_i   (y stored in z) */
    for (int j = 0; j < nb; ++j) {
        double *y = z + (long)j * b;
        memcpy(y, v + (long)j * b, sizeof(double) * b);
        for (long p = row_ptr[j]; p < row_ptr[j + 1]; ++p) {
            int i = col_idx[p];
            if (i >= j) break;
            mat_vec_add(b, -1.0, vals + p * bb, z + (long)i * b, y);
        }
    }
    /* backward: z_j = U_jj^{-1} (y_j - sum_{k>j} U_jk z_k) */
    for (int j = nb - 1; j >= 0; --j) {
        double *y = z + (long)j * b;
        for (long p = row_ptr[j]; p < row_ptr[j + 1]; ++p) {
            int k = col_idx[p];
            if (k <= j) continue;
            mat_vec_add(b, -1.0, vals + p * bb, z + (long)k * b, y);
        }
        lu_solve(b, dlu + j * bb, dpiv + (long)j * b, y);
    }
}

/* Alg. 2 (simplified block ILU(0)), literally: for i = 1..T, for neighbours
 * j > i of i:  B_ji <- B_ji B_ii^{-1};  B_jj <- B_jj - B_ji B_ij.
 * Valid when no two neighbours of an element are neighbours of each other.
 * Same storage convention as irk_ref_bilu0 (dlu/dpiv filled at the end). */
int irk_ref_ilu_alg2(int T, int m, const int *row_ptr, const int *col_idx,
                     double *vals, double *dlu, int *dpiv)
{
    long mm = (long)m * m;
    double *inv = (double *)malloc(sizeof(double) * mm);
    double *tmp = (double *)malloc(sizeof(double) * mm);
    if (!inv || !tmp) { free(inv); free(tmp); return REF_ENOMEM; }
    int rc = REF_OK;
    for (int i = 0; i < T && rc == REF_OK; ++i) {
        long pii = find_block(row_ptr, col_idx, i, i);
        rc = invert(m, vals + pii * mm, inv);
        if (rc != REF_OK) break;
        for (long q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            int j = col_idx[q];
            if (j <= i) continue;
            long pji = find_block(row_ptr, col_idx, j, i);
            long pjj = find_block(row_ptr, col_idx, j, j);
            if (pji < 0 || pjj < 0) { rc = REF_EINVAL; break; }
            mat_mul(m, vals + pji * mm, inv, tmp);
            memcpy(vals + pji * mm, tmp, sizeof(double) * mm);
            mat_mul_sub(m, vals + pji * mm, vals + q * mm, vals + pjj * mm);
        }
    }
    for (int j = 0; j < T && rc == REF_OK; ++j) {
        long pjj = find_block(row_ptr, col_idx, j, j);
        memcpy(dlu + j * mm, vals + pjj * mm, sizeof(double) * mm);
        rc = lu_factor(m, dlu + j * mm, dpiv + (long)j * m);
    }
    free(inv);
    free(tmp);
    return rc;
}

/* Alg. 3 (stage-coupled block ILU(0) of the transformed system, eq. big-irk),
 * in the corrected reading: the unknowns are ordered stage-major (stage k,
 * then element i) and, when the pivot block (k, i) is eliminated,
 *   - within stage k, for neighbours j > i of i:
 *         B_kk,ji <- B_kk,ji B_kk,ii^{-1};  B_kk,jj <- B_kk,jj - B_kk,ji B_kk,ij
 *   - for every later stage l > k:
 *         B_lk,ii <- B_lk,ii B_kk,ii^{-1}
 *         B_lq,ii <- B_lq,ii - B_lk,ii B_kq,ii   for every q > k (q = l is the
 *                                                 diagonal block B_ll,ii)
 * Fill into blocks outside the pattern (e.g. (l, neighbour of i)) is dropped.
 * As printed, the update line reads B_ll,ii - B_lk,ii B_kk,ii, which after the
 * multiplier step is the old B_lk,ii itself (not an LU step) and, for s >= 3,
 * misses the updates of the off-diagonal stage blocks; the reading above is
 * the block ILU(0) of the stage-major matrix.
 * Storage: Bd[k] (nnzb*m*m, the pattern of J) holds B_kk; Bo[(k*s + l)*T*m*m
 * + i*m*m] holds the block-diagonal B_kl,ii for k != l.  On return both hold
 * the factors; dlu/dpiv ((k*T + i) ordered) hold the LU of each pivot block. */
int irk_ref_ilu_alg3(int s, int T, int m, const int *row_ptr, const int *col_idx,
                     double *Bd, double *Bo, double *dlu, int *dpiv)
{
    long mm = (long)m * m;
    long nnzb = row_ptr[T];
    long Tmm = (long)T * mm;
    double *inv = (double *)malloc(sizeof(double) * mm);
    double *tmp = (double *)malloc(sizeof(double) * mm);
    if (!inv || !tmp) { free(inv); free(tmp); return REF_ENOMEM; }
    int rc = REF_OK;
    for (int k = 0; k < s && rc == REF_OK; ++k) {
        double *Bkk = Bd + k * nnzb * mm;
        for (int i = 0; i < T && rc == REF_OK; ++i) {
            long pii = find_block(row_ptr, col_idx, i, i);
            rc = invert(m, Bkk + pii * mm, inv);
            if (rc != REF_OK) break;
            for (long q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
                int j = col_idx[q];
                if (j <= i) continue;
                long pji = find_block(row_ptr, col_idx, j, i);
                long pjj = find_block(row_ptr, col_idx, j, j);
                if (pji < 0 || pjj < 0) { rc = REF_EINVAL; break; }
                mat_mul(m, Bkk + pji * mm, inv, tmp);
                memcpy(Bkk + pji * mm, tmp, sizeof(double) * mm);
                mat_mul_sub(m, Bkk + pji * mm, Bkk + q * mm, Bkk + pjj * mm);
            }
            for (int l = k + 1; l < s && rc == REF_OK; ++l) {
                double *Blk = Bo + ((long)l * s + k) * Tmm + i * mm;
                mat_mul(m, Blk, inv, tmp);
                memcpy(Blk, tmp, sizeof(double) * mm);
                for (int q = k + 1; q < s; ++q) {
                    double *target = (q == l)
                        ? Bd + q * nnzb * mm + find_block(row_ptr, col_idx, i, i) * mm
                        : Bo + ((long)l * s + q) * Tmm + i * mm;
                    const double *Bkq = Bo + ((long)k * s + q) * Tmm + i * mm;
                    mat_mul_sub(m, Blk, Bkq, target);
                }
            }
        }
    }
    for (int k = 0; k < s && rc == REF_OK; ++k)
        for (int i = 0; i < T && rc == REF_OK; ++i) {
            long pii = find_block(row_ptr, col_idx, i, i);
            long d = (long)k * T + i;
            memcpy(dlu + d * mm, Bd + k * nnzb * mm + pii * mm, sizeof(double) * mm);
            rc = lu_factor(m, dlu + d * mm, dpiv + d * m);
        }
    free(inv);
    free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Assembled forms of the system matrix (for the generic block ILU(0)).     */
/* ------------------------------------------------------------------------ */

/* Stage-major block-CSR of the whole system (s*T block rows of m x m blocks;
 * block row k*T + i is stage k, element i).  form 0: transformed B of
 * eq. big-irk, C = A^{-1}:  block ((k,i),(l,j)) = C_kl M_i [i==j] - dt [k==l] (J_k)_ij.
 * form 1: untransformed matrix of eq. newton-system-2, C = A:
 *   block ((k,i),(l,j)) = [k==l][i==j] M_i - dt C_kl (J_k)_ij.
 * Blocks are stored where the structure can be non-zero: form 0 has the
 * pattern of J inside each stage plus the diagonal coupling blocks (l, i);
 * form 1 has (l, j) for every l and every j in the pattern of row i.
 * With out_rp == NULL only the number of blocks is returned. */
long irk_ref_assemble_stage_major(int form, int s, const double *C, int T, int m,
                                  const int *row_ptr, const int *col_idx,
                                  const double *J, long jstride, const double *M,
                                  double dt, int *out_rp, int *out_ci, double *out_vals)
{
    long mm = (long)m * m;
    long nnzb = row_ptr[T];
    long total = (form == 0) ? s * nnzb + (long)s * (s - 1) * T : (long)s * s * nnzb;
    if (!out_rp) return total;
    long pos = 0;
    for (int k = 0; k < s; ++k) {
        const double *Jk = J + k * jstride;
        for (int i = 0; i < T; ++i) {
            out_rp[k * T + i] = (int)pos;
            for (int l = 0; l < s; ++l) {
                if (form == 0 && l != k) {
                    out_ci[pos] = l * T + i;
                    double *blk = out_vals + pos * mm;
                    for (long e = 0; e < mm; ++e) blk[e] = C[k * s + l] * M[i * mm + e];
                    ++pos;
                    continue;
                }
                for (long p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                    int j = col_idx[p];
                    out_ci[pos] = l * T + j;
                    double *blk = out_vals + pos * mm;
                    if (form == 0) {
                        for (long e = 0; e < mm; ++e)
                            blk[e] = (j == i ? C[k * s + k] * M[i * mm + e] : 0.0) - dt * Jk[p * mm + e];
                    } else {
                        for (long e = 0; e < mm; ++e)
                            blk[e] = (j == i && l == k ? M[i * mm + e] : 0.0) - dt * C[k * s + l] * Jk[p * mm + e];
                    }
                    ++pos;
                }
            }
        }
    }
    out_rp[s * T] = (int)pos;
    return pos;
}

/* Element-major block-CSR of the whole system: T block rows of (s*m) x (s*m)
 * blocks, the pattern of J; inside a block, row (k, a) and column (l, b) are
 * at k*m + a and l*m + b.  form 0 (transformed, C = A^{-1}):
 *   C_kl M_i[a][b] [i==j] - dt [k==l] (J_k)_ij[a][b];
 * form 1 (untransformed, C = A):  [k==l][i==j] M_i[a][b] - dt C_kl (J_k)_ij[a][b].
 * The vector ordering is element-major: index (i*s + k)*m + a. */
void irk_ref_assemble_element_major(int form, int s, const double *C, int T, int m,
                                    const int *row_ptr, const int *col_idx,
                                    const double *J, long jstride, const double *M,
                                    double dt, double *out_vals)
{
    long mm = (long)m * m;
    long sm = (long)s * m;
    for (int i = 0; i < T; ++i)
        for (long p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int j = col_idx[p];
            double *blk = out_vals + p * sm * sm;
            for (int k = 0; k < s; ++k)
                for (int l = 0; l < s; ++l)
                    for (int a = 0; a < m; ++a)
                        for (int b = 0; b < m; ++b) {
                            double mass = (j == i) ? M[i * mm + a * m + b] : 0.0;
                            double jac = J[k * jstride + p * mm + a * m + b];
                            double v;
                            if (form == 0)
                                v = C[k * s + l] * mass - (k == l ? dt * jac : 0.0);
                            else
                                v = (k == l ? mass : 0.0) - dt * C[k * s + l] * jac;
                            blk[((long)k * m + a) * sm + (long)l * m + b] = v;
                        }
        }
}

/* One stage's matrix for the stage-uncoupled preconditioner of Sec. 4.3.2:
 * d M - dt J_k (the pattern of J), with d = (A^{-1})_kk + alpha_k. */
void irk_ref_assemble_shifted(int T, int m, const int *row_ptr, const int *col_idx,
                              const double *Jk, const double *M, double d, double dt,
                              double *out_vals)
{
    long mm = (long)m * m;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < T; ++i)
        for (long p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            for (long e = 0; e < mm; ++e)
                out_vals[p * mm + e] = (col_idx[p] == i ? d * M[i * mm + e] : 0.0) - dt * Jk[p * mm + e];
}

/* ------------------------------------------------------------------------ */
/* Flexible GMRES(restart), right preconditioned (Sec. 4 and Sec. 5.1.1:     */
/* one operator product and one preconditioner application per iteration). */
/* ------------------------------------------------------------------------ */

typedef void (*ref_op_fn)(void *ctx, const double *x, double *y);

static double dot(long N, const double *a, const double *b)
{
    double acc = 0.0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
    for (long q = 0; q < N; ++q) acc += a[q] * b[q];
    return acc;
}

/* Threads the multi-core build uses (n > 0 sets them); 1 in the serial build. */
int irk_ref_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Restarted flexible GMRES with modified Gram-Schmidt and Givens rotations,
 * right preconditioned: x = x0 + Z y, Z = [P v_0 .. P v_{k-1}].  x holds the
 * initial guess on entry.  Stops when the Givens residual estimate reaches
 * rtol * ||b||; the true residual is recomputed at the end of every cycle and
 * a new cycle starts while it exceeds rtol * ||b|| and fewer than max_iter
 * inner iterations were taken.  est_hist (optional, max_iter + 1 entries)
 * receives the relative estimate before the first and after every iteration. */
int irk_ref_fgmres(long N, ref_op_fn apply_A, void *actx, ref_op_fn apply_P, void *pctx,
                   const double *b, double *x, double rtol, int restart, int max_iter,
                   int *iters_out, double *relres_out, double *est_hist, int *cycles_out)
{
    if (N < 0 || restart < 1 || max_iter < 0) return REF_EINVAL;
    int R = restart;
    double *V = (double *)malloc(sizeof(double) * N * (R + 1));
    double *Z = (double *)malloc(sizeof(double) * N * R);
    double *r = (double *)malloc(sizeof(double) * N);
    double *H = (double *)calloc((size_t)(R + 1) * R, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * R);
    double *sn = (double *)malloc(sizeof(double) * R);
    double *g = (double *)malloc(sizeof(double) * (R + 1));
    double *y = (double *)malloc(sizeof(double) * R);
    if (!V || !Z || !r || !H || !cs || !sn || !g || !y) {
        free(V); free(Z); free(r); free(H); free(cs); free(sn); free(g); free(y);
        return REF_ENOMEM;
    }
    int rc = REF_OK, total = 0, cycles = 0;
    double bnorm = sqrt(dot(N, b, b));
    double beta = 0.0;
    if (bnorm == 0.0) {
        for (long q = 0; q < N; ++q) x[q] = 0.0;
        if (est_hist) est_hist[0] = 0.0;
        goto done;
    }
    apply_A(actx, x, r);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < N; ++q) r[q] = b[q] - r[q];
    beta = sqrt(dot(N, r, r));
    if (est_hist) est_hist[0] = beta / bnorm;
    while (1) {
        if (!isfinite(beta)) { rc = REF_NONFINITE; break; }
        if (beta <= rtol * bnorm) break;
        if (total >= max_iter) { rc = REF_NOT_CONVERGED; break; }
        ++cycles;
#pragma omp parallel for schedule(static)
        for (long q = 0; q < N; ++q) V[q] = r[q] / beta;
        for (int q = 0; q <= R; ++q) g[q] = 0.0;
        g[0] = beta;
        int jlast = -1;
        for (int j = 0; j < R; ++j) {
            double *vj = V + (long)j * N, *zj = Z + (long)j * N, *w = V + (long)(j + 1) * N;
            apply_P(pctx, vj, zj);
            apply_A(actx, zj, w);
            for (int i = 0; i <= j; ++i) {
                double h = dot(N, w, V + (long)i * N);
                H[i * R + j] = h;
#pragma omp parallel for schedule(static)
                for (long q = 0; q < N; ++q) w[q] -= h * V[(long)i * N + q];
            }
            double hnext = sqrt(dot(N, w, w));
            H[(j + 1) * R + j] = hnext;
            if (hnext != 0.0) {
#pragma omp parallel for schedule(static)
                for (long q = 0; q < N; ++q) w[q] /= hnext;
            }
            /* previous rotations on the new column */
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * H[i * R + j] + sn[i] * H[(i + 1) * R + j];
                H[(i + 1) * R + j] = -sn[i] * H[i * R + j] + cs[i] * H[(i + 1) * R + j];
                H[i * R + j] = t;
            }
            /* new rotation annihilating H[j+1][j] */
            double rho = hypot(H[j * R + j], H[(j + 1) * R + j]);
            if (rho == 0.0 || !isfinite(rho)) { rc = isfinite(rho) ? REF_SINGULAR : REF_NONFINITE; break; }
            cs[j] = H[j * R + j] / rho;
            sn[j] = H[(j + 1) * R + j] / rho;
            H[j * R + j] = rho;
            H[(j + 1) * R + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            jlast = j;
            double est = fabs(g[j + 1]);
            if (est_hist) est_hist[total] = est / bnorm;
            if (est <= rtol * bnorm || total >= max_iter || hnext == 0.0) break;
        }
        if (rc != REF_OK) break;
        /* least squares: upper triangular H y = g, then x += Z y */
        for (int i = jlast; i >= 0; --i) {
            double acc = g[i];
            for (int k = i + 1; k <= jlast; ++k) acc -= H[i * R + k] * y[k];
            y[i] = acc / H[i * R + i];
        }
        for (int i = 0; i <= jlast; ++i) {
#pragma omp parallel for schedule(static)
            for (long q = 0; q < N; ++q) x[q] += y[i] * Z[(long)i * N + q];
        }
        apply_A(actx, x, r);
#pragma omp parallel for schedule(static)
        for (long q = 0; q < N; ++q) r[q] = b[q] - r[q];
        beta = sqrt(dot(N, r, r));
    }
done:
    if (iters_out) *iters_out = total;
    if (relres_out) *relres_out = bnorm > 0.0 ? beta / bnorm : 0.0;
    if (cycles_out) *cycles_out = cycles;
    free(V); free(Z); free(r); free(H); free(cs); free(sn); free(g); free(y);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The stage-system solve: operator + preconditioner + FGMRES.              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int form, s, T, m;
    const double *C; /* A^{-1} (transformed) or A (untransformed) */
    const int *row_ptr, *col_idx;
    const double *J, *M;
    long jstride;
    double dt;
} ref_operator;

static void ref_operator_apply(void *ctx, const double *x, double *y)
{
    ref_operator *o = (ref_operator *)ctx;
    if (o->form == 0)
        irk_ref_apply_transformed(o->s, o->C, o->T, o->m, o->row_ptr, o->col_idx, o->J,
                                  o->jstride, o->M, o->dt, x, y);
    else
        irk_ref_apply_untransformed(o->s, o->C, o->T, o->m, o->row_ptr, o->col_idx, o->J,
                                    o->jstride, o->M, o->dt, x, y);
}

/* Preconditioner kinds */
#define REF_PC_NONE 0
#define REF_PC_UNCOUPLED 1 /* Sec. 4.3.2: per-stage ILU(0) of d_k M - dt J_k  */
#define REF_PC_STAGE_MAJOR 2 /* block ILU(0) of the whole stage-major system (Alg. 3 for form 0) */
#define REF_PC_ELEMENT_MAJOR 3 /* block ILU(0) of the whole element-major system (s*m blocks) */

typedef struct {
    int kind, s, T, m, nb, b;
    const int *rp, *ci; /* pattern of the factored matrix */
    int *own_rp, *own_ci;
    double *vals, *dlu;
    int *dpiv;
    long nnzb; /* blocks per factored matrix */
    double *work, *work2;
} ref_precond;

static void ref_precond_apply(void *ctx, const double *v, double *z)
{
    ref_precond *p = (ref_precond *)ctx;
    long n = (long)p->T * p->m;
    long N = n * p->s;
    long mm = (long)p->m * p->m;
    if (p->kind == REF_PC_NONE) {
        memcpy(z, v, sizeof(double) * N);
    } else if (p->kind == REF_PC_UNCOUPLED) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < p->s; ++k)
            irk_ref_bilu0_apply(p->T, p->m, p->rp, p->ci, p->vals + k * p->nnzb * mm,
                                p->dlu + (long)k * p->T * mm, p->dpiv + (long)k * p->T * p->m,
                                v + k * n, z + k * n);
    } else if (p->kind == REF_PC_STAGE_MAJOR) {
        irk_ref_bilu0_apply(p->nb, p->b, p->rp, p->ci, p->vals, p->dlu, p->dpiv, v, z);
    } else {
        /* stage-major -> element-major, solve, and back */
        for (int k = 0; k < p->s; ++k)
            for (int i = 0; i < p->T; ++i)
                memcpy(p->work + ((long)i * p->s + k) * p->m, v + k * n + (long)i * p->m,
                       sizeof(double) * p->m);
        irk_ref_bilu0_apply(p->nb, p->b, p->rp, p->ci, p->vals, p->dlu, p->dpiv, p->work, p->work2);
        for (int k = 0; k < p->s; ++k)
            for (int i = 0; i < p->T; ++i)
                memcpy(z + k * n + (long)i * p->m, p->work2 + ((long)i * p->s + k) * p->m,
                       sizeof(double) * p->m);
    }
}

static void ref_precond_free(ref_precond *p)
{
    free(p->own_rp); free(p->own_ci); free(p->vals); free(p->dlu); free(p->dpiv);
    free(p->work); free(p->work2);
}

/* Column shift rule of Sec. 4.3.2: alpha_k = sum_{j != k} |(A^{-1})_{jk}|. */
void irk_ref_shift_column_rule(int s, const double *Ainv, double *alpha)
{
    for (int k = 0; k < s; ++k) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j)
            if (j != k) acc += fabs(Ainv[j * s + k]);
        alpha[k] = acc;
    }
}

/* Build (factor) the preconditioner.  C is A^{-1} for form 0, A for form 1;
 * Ainv is always A^{-1} (the uncoupled preconditioner uses its diagonal). */
static int ref_precond_build(ref_precond *p, int kind, int form, int s, const double *C,
                             const double *Ainv, int T, int m, const int *row_ptr,
                             const int *col_idx, const double *J, long jstride,
                             const double *M, double dt, const double *shift)
{
    memset(p, 0, sizeof(*p));
    p->kind = kind; p->s = s; p->T = T; p->m = m;
    long mm = (long)m * m;
    long nnzb = row_ptr[T];
    if (kind == REF_PC_NONE) return REF_OK;
    if (kind == REF_PC_UNCOUPLED) {
        if (form != 0) return REF_EINVAL;
        double alpha[64];
        if (s > 64) return REF_EINVAL;
        if (shift) memcpy(alpha, shift, sizeof(double) * s);
        else irk_ref_shift_column_rule(s, Ainv, alpha);
        p->rp = row_ptr; p->ci = col_idx; p->nnzb = nnzb; p->nb = T; p->b = m;
        p->vals = (double *)malloc(sizeof(double) * s * nnzb * mm);
        p->dlu = (double *)malloc(sizeof(double) * s * T * mm);
        p->dpiv = (int *)malloc(sizeof(int) * s * T * m);
        if (!p->vals || !p->dlu || !p->dpiv) return REF_ENOMEM;
        int rcs[64];
#pragma omp parallel for schedule(static)
        for (int k = 0; k < s; ++k) {
            double *vk = p->vals + k * nnzb * mm;
            irk_ref_assemble_shifted(T, m, row_ptr, col_idx, J + k * jstride, M,
                                     Ainv[k * s + k] + alpha[k], dt, vk);
            rcs[k] = irk_ref_bilu0(T, m, row_ptr, col_idx, vk, p->dlu + (long)k * T * mm,
                                   p->dpiv + (long)k * T * m);
        }
        for (int k = 0; k < s; ++k)
            if (rcs[k] != REF_OK) return rcs[k];
        return REF_OK;
    }
    if (kind == REF_PC_STAGE_MAJOR) {
        long nb2 = irk_ref_assemble_stage_major(form, s, C, T, m, row_ptr, col_idx, J, jstride,
                                                M, dt, NULL, NULL, NULL);
        p->nb = s * T; p->b = m; p->nnzb = nb2;
        p->own_rp = (int *)malloc(sizeof(int) * (s * T + 1));
        p->own_ci = (int *)malloc(sizeof(int) * nb2);
        p->vals = (double *)malloc(sizeof(double) * nb2 * mm);
        p->dlu = (double *)malloc(sizeof(double) * s * T * mm);
        p->dpiv = (int *)malloc(sizeof(int) * s * T * m);
        if (!p->own_rp || !p->own_ci || !p->vals || !p->dlu || !p->dpiv) return REF_ENOMEM;
        irk_ref_assemble_stage_major(form, s, C, T, m, row_ptr, col_idx, J, jstride, M, dt,
                                     p->own_rp, p->own_ci, p->vals);
        p->rp = p->own_rp; p->ci = p->own_ci;
        return irk_ref_bilu0(p->nb, p->b, p->rp, p->ci, p->vals, p->dlu, p->dpiv);
    }
    if (kind == REF_PC_ELEMENT_MAJOR) {
        long sm = (long)s * m;
        p->nb = T; p->b = (int)sm; p->nnzb = nnzb;
        p->rp = row_ptr; p->ci = col_idx;
        p->vals = (double *)malloc(sizeof(double) * nnzb * sm * sm);
        p->dlu = (double *)malloc(sizeof(double) * T * sm * sm);
        p->dpiv = (int *)malloc(sizeof(int) * T * sm);
        p->work = (double *)malloc(sizeof(double) * T * sm);
        p->work2 = (double *)malloc(sizeof(double) * T * sm);
        if (!p->vals || !p->dlu || !p->dpiv || !p->work || !p->work2) return REF_ENOMEM;
        irk_ref_assemble_element_major(form, s, C, T, m, row_ptr, col_idx, J, jstride, M, dt, p->vals);
        return irk_ref_bilu0(T, (int)sm, row_ptr, col_idx, p->vals, p->dlu, p->dpiv);
    }
    return REF_EINVAL;
}

/* Solve the stage system for one right-hand side R (stage-major, s*T*m).
 * form 0: B W = R with B = A^{-1} (x) M - dt diag(J_k)  (eq. big-irk), X = W.
 * form 1: (I (x) M - dt [a_kl J_k]) K = R  (eq. newton-system-2), X = K.
 * X holds the initial guess on entry (zero for a plain solve). */
int irk_ref_solve(int form, int s, const double *A, const double *Ainv, int T, int m,
                  const int *row_ptr, const int *col_idx, const double *J, long jstride,
                  const double *M, double dt, int precond, const double *shift,
                  int restart, int max_iter, double rtol, const double *R, double *X,
                  int *iters, double *relres, double *est_hist, int *cycles)
{
    if (form != 0 && form != 1) return REF_EINVAL;
    const double *C = form == 0 ? Ainv : A;
    ref_operator op = {form, s, T, m, C, row_ptr, col_idx, J, M, jstride, dt};
    ref_precond pc;
    int rc = ref_precond_build(&pc, precond, form, s, C, Ainv, T, m, row_ptr, col_idx, J,
                               jstride, M, dt, shift);
    if (rc == REF_OK)
        rc = irk_ref_fgmres((long)s * T * m, ref_operator_apply, &op, ref_precond_apply, &pc,
                            R, X, rtol, restart, max_iter, iters, relres, est_hist, cycles);
    ref_precond_free(&pc);
    return rc;
}

/* Apply the preconditioner alone (z = P^{-1} v), for tests of the factors. */
int irk_ref_precond_apply(int form, int s, const double *A, const double *Ainv, int T, int m,
                          const int *row_ptr, const int *col_idx, const double *J, long jstride,
                          const double *M, double dt, int precond, const double *shift,
                          const double *v, double *z)
{
    const double *C = form == 0 ? Ainv : A;
    ref_precond pc;
    int rc = ref_precond_build(&pc, precond, form, s, C, Ainv, T, m, row_ptr, col_idx, J,
                               jstride, M, dt, shift);
    if (rc == REF_OK) ref_precond_apply(&pc, v, z);
    ref_precond_free(&pc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.5: reordered and partitioned stage-uncoupled block ILU(0).         */
/* ------------------------------------------------------------------------ */

/* Build, for one stage, the shifted matrix d M - dt J_k restricted to the
 * blocks whose two elements share a partition (part[i] == part[j]; part NULL
 * = one partition), with the elements renumbered so that element perm[q] is
 * the q-th eliminated (perm NULL = natural order).  Returns the number of
 * blocks; with out_rp == NULL only counts. */
long irk_ref_assemble_ordered(int T, int m, const int *row_ptr, const int *col_idx, const double *Jk,
                              const double *M, double d, double dt, const int *perm, const int *part,
                              int *out_rp, int *out_ci, double *out_vals)
{
    long mm = (long)m * m;
    int *inv = (int *)malloc(sizeof(int) * (T > 0 ? T : 1));
    if (!inv) return -1;
    for (int q = 0; q < T; ++q) inv[perm ? perm[q] : q] = q;
    long pos = 0;
    for (int q = 0; q < T; ++q) {
        int e = perm ? perm[q] : q;
        if (out_rp) out_rp[q] = (int)pos;
        /* neighbours of e kept in the preconditioner, in increasing new index */
        int cnt = 0;
        int cols[64];
        long src[64];
        for (long p = row_ptr[e]; p < row_ptr[e + 1]; ++p) {
            int j = col_idx[p];
            if (part && part[j] != part[e]) continue;
            if (cnt >= 64) { free(inv); return -1; }
            cols[cnt] = inv[j];
            src[cnt] = p;
            ++cnt;
        }
        for (int a = 1; a < cnt; ++a) /* insertion sort by new column */
            for (int b2 = a; b2 > 0 && cols[b2 - 1] > cols[b2]; --b2) {
                int tc = cols[b2]; cols[b2] = cols[b2 - 1]; cols[b2 - 1] = tc;
                long ts = src[b2]; src[b2] = src[b2 - 1]; src[b2 - 1] = ts;
            }
        for (int a = 0; a < cnt; ++a) {
            if (out_rp) {
                out_ci[pos] = cols[a];
                double *blk = out_vals + pos * mm;
                int j = col_idx[src[a]];
                for (long x = 0; x < mm; ++x)
                    blk[x] = (j == e ? d * M[(long)e * mm + x] : 0.0) - dt * Jk[src[a] * mm + x];
            }
            ++pos;
        }
    }
    if (out_rp) out_rp[T] = (int)pos;
    free(inv);
    return pos;
}

typedef struct {
    int s, T, m;
    const int *perm;
    int *rp, *ci; /* one pattern shared by the stages */
    double *vals, *dlu;
    int *dpiv;
    long nnzb;
    double *work, *work2;
} ref_ordered_pc;

static void ref_ordered_apply(void *ctx, const double *v, double *z)
{
    ref_ordered_pc *p = (ref_ordered_pc *)ctx;
    long n = (long)p->T * p->m;
    long mm = (long)p->m * p->m;
    for (int k = 0; k < p->s; ++k) {
        for (int q = 0; q < p->T; ++q) {
            int e = p->perm ? p->perm[q] : q;
            memcpy(p->work + (long)q * p->m, v + k * n + (long)e * p->m, sizeof(double) * p->m);
        }
        irk_ref_bilu0_apply(p->T, p->m, p->rp, p->ci, p->vals + k * p->nnzb * mm,
                            p->dlu + (long)k * p->T * mm, p->dpiv + (long)k * p->T * p->m, p->work, p->work2);
        for (int q = 0; q < p->T; ++q) {
            int e = p->perm ? p->perm[q] : q;
            memcpy(z + k * n + (long)e * p->m, p->work2 + (long)q * p->m, sizeof(double) * p->m);
        }
    }
}

static void ref_ordered_free(ref_ordered_pc *p)
{
    free(p->rp); free(p->ci); free(p->vals); free(p->dlu); free(p->dpiv); free(p->work); free(p->work2);
}

static int ref_ordered_build(ref_ordered_pc *p, int s, const double *Ainv, int T, int m,
                             const int *row_ptr, const int *col_idx, const double *J, long jstride,
                             const double *M, double dt, const double *shift, const int *perm,
                             const int *part)
{
    memset(p, 0, sizeof(*p));
    p->s = s; p->T = T; p->m = m; p->perm = perm;
    long mm = (long)m * m;
    double alpha[64];
    if (s > 64) return REF_EINVAL;
    if (shift) memcpy(alpha, shift, sizeof(double) * s);
    else irk_ref_shift_column_rule(s, Ainv, alpha);
    long nb = irk_ref_assemble_ordered(T, m, row_ptr, col_idx, J, M, 0.0, dt, perm, part, NULL, NULL, NULL);
    if (nb < 0) return REF_EINVAL;
    p->nnzb = nb;
    p->rp = (int *)malloc(sizeof(int) * (T + 1));
    p->ci = (int *)malloc(sizeof(int) * (nb > 0 ? nb : 1));
    p->vals = (double *)malloc(sizeof(double) * s * nb * mm);
    p->dlu = (double *)malloc(sizeof(double) * s * T * mm);
    p->dpiv = (int *)malloc(sizeof(int) * s * T * m);
    p->work = (double *)malloc(sizeof(double) * T * m);
    p->work2 = (double *)malloc(sizeof(double) * T * m);
    if (!p->rp || !p->ci || !p->vals || !p->dlu || !p->dpiv || !p->work || !p->work2) return REF_ENOMEM;
    for (int k = 0; k < s; ++k) {
        double *vk = p->vals + k * nb * mm;
        irk_ref_assemble_ordered(T, m, row_ptr, col_idx, J + k * jstride, M, Ainv[k * s + k] + alpha[k], dt,
                                 perm, part, p->rp, p->ci, vk);
        int rc = irk_ref_bilu0(T, m, p->rp, p->ci, vk, p->dlu + (long)k * T * mm, p->dpiv + (long)k * T * m);
        if (rc != REF_OK) return rc;
    }
    return REF_OK;
}

/* Transformed solve (eq. big-irk) with the reordered / partitioned
 * stage-uncoupled preconditioner. */
int irk_ref_solve_ordered(int s, const double *Ainv, int T, int m, const int *row_ptr, const int *col_idx,
                          const double *J, long jstride, const double *M, double dt, const double *shift,
                          const int *perm, const int *part, int restart, int max_iter, double rtol,
                          const double *R, double *X, int *iters, double *relres, int *cycles)
{
    ref_operator op = {0, s, T, m, Ainv, row_ptr, col_idx, J, M, jstride, dt};
    ref_ordered_pc pc;
    int rc = ref_ordered_build(&pc, s, Ainv, T, m, row_ptr, col_idx, J, jstride, M, dt, shift, perm, part);
    if (rc == REF_OK)
        rc = irk_ref_fgmres((long)s * T * m, ref_operator_apply, &op, ref_ordered_apply, &pc, R, X, rtol,
                            restart, max_iter, iters, relres, NULL, cycles);
    ref_ordered_free(&pc);
    return rc;
}

int irk_ref_precond_apply_ordered(int s, const double *Ainv, int T, int m, const int *row_ptr,
                                  const int *col_idx, const double *J, long jstride, const double *M,
                                  double dt, const double *shift, const int *perm, const int *part,
                                  const double *v, double *z)
{
    ref_ordered_pc pc;
    int rc = ref_ordered_build(&pc, s, Ainv, T, m, row_ptr, col_idx, J, jstride, M, dt, shift, perm, part);
    if (rc == REF_OK) ref_ordered_apply(&pc, v, z);
    ref_ordered_free(&pc);
    return rc;
}
