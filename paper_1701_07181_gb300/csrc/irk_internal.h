// irk_internal.h -- internal declarations shared by the library's translation
// units (context layout, kernel launchers).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/irk_gb300.h"

#define IRK_MAX_S 8
#define IRK_MAX_M 128

// Device-side error word values (set by kernels, read by the host).
#define IRK_DEV_ERR_SINGULAR 1
#define IRK_DEV_ERR_NONFINITE 2
#define IRK_DEV_ERR_TIMEOUT 4

// Polls a wait on another thread block makes before giving up (the default
// of irk_options.spin_limit).
#define IRK_DEFAULT_SPIN_LIMIT (1 << 20)

// Element type of every Krylov vector: 8 bytes, either a binary64 or a
// double-float pair (hi, lo).  Vectors are stored element-interleaved:
// index (i*s + k)*m + a for element i, stage k, component a.
typedef unsigned long long vec8;

// Coefficients of one system-block of the assembled preconditioner matrix:
// value = cm * M[mi] + cj * J[jp] (m x m blocks); ids index tables of
// coefficients rebuilt for every dt.
struct AsmEntry {
    int jp;        // position of the J block, or -1
    int mi;        // element whose mass block enters, or -1
    int cm_id;     // index into the mass-coefficient table
    int cj_id;     // index into the Jacobian-coefficient table
};

// Assembled block system whose block ILU(0) is the preconditioner.
struct PcSystem {
    int kind = IRK_PC_NONE;
    int nb = 0, b = 0;  // block rows, block size
    long long nnz = 0;  // stored blocks
    int element_major = 0;  // 1: one (s m)-block per J block (assembled by its own kernel)
    // pattern (device): row pointers, columns, diagonal position, vector offset
    int *d_rp = nullptr, *d_ci = nullptr, *d_diag = nullptr, *d_voff = nullptr;
    AsmEntry *d_asm = nullptr;
    int *d_rowof = nullptr;  // element-major kind: block row of each stored block
    // factor-update lists: for lower entry p, pairs (q, pos): B_q -= L_p B_pos
    int *d_upd_ptr = nullptr, *d_upd = nullptr;
    // level schedules (rows grouped by level; host copies of the level bounds)
    std::vector<int> lo_ptr, up_ptr;
    int *d_lo_rows = nullptr, *d_up_rows = nullptr;
    // uncoupled kind with every stage's upper blocks equal to -dt J (no
    // factor update reaches them): backward levels as stage-0 rows only
    int shared_upper = 0;
    std::vector<int> up0_ptr;
    int *d_up0_rows = nullptr;
    // every factor update of a lower entry lands on its row's diagonal block:
    // most lower entries of a row (the fused factorisation kernel), else 0
    int fused_r = 0;
    // two lower levels, the second without upper entries, the first level of
    // the upper DAG without lower entries, together every row: the
    // preconditioner applies in two launches (k_sweep_fd, k_sweep_bu)
    int two_colour = 0;
    // values, column-major blocks: working precision (double or float)
    void *d_vals = nullptr, *d_dinv = nullptr;
    // bf16 copies used by the sweeps when factor_prec == IRK_FACTOR_BF16
    void *d_vals16 = nullptr, *d_dinv16 = nullptr;
    // intermediate vector of the sweeps (compute precision, element-interleaved)
    void *d_y = nullptr;
    int n_cm = 0, n_cj = 0;  // coefficient-table sizes
    // persistent sweeps: forward / backward results as self-validating words
    // {32 value bits, epoch}; the epoch increases with every application
    int persistent = 0;
    unsigned long long *d_yll = nullptr, *d_zll = nullptr;
    int epoch = 0;
    int coop_blocks = 0;
    size_t coop_smem = 0;
    int max_item_blocks = 1;  // most blocks one sweep item reads (incl. D^{-1})
};

struct irk_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    // host right-hand sides: copied on their own non-blocking stream while a
    // refactorisation runs (created at the first such solve)
    cudaStream_t in_stream = nullptr;
    cudaEvent_t in_ev = nullptr;
    int s = 0, T = 0, m = 0, nnzb = 0;
    int nJ = 1;  // Jacobians stored: 1 (shared by the stages) or s (one per stage)
    long long n = 0, N = 0;  // n = T m, N = s n
    double A[IRK_MAX_S * IRK_MAX_S], Ainv[IRK_MAX_S * IRK_MAX_S], shift[IRK_MAX_S];
    irk_options opt;
    int df = 0;    // 1: Krylov vectors and arithmetic are double-float
    int dfop = 0;  // 1: J, M and the operator product are double-float (DF64, FP64_DFOP)
    int fprec = IRK_FACTOR_FP64;
    std::vector<int> h_rp, h_ci;
    std::vector<int> h_part;  // optional partition id per element (Sec. 4.5)
    int *d_rp = nullptr, *d_ci = nullptr;
    vec8 *d_J = nullptr;  // nnzb blocks, column-major, binary64 or double-float
    vec8 *d_M = nullptr;  // T blocks, column-major
    PcSystem pc;
    bool factored = false;
    double factored_dt = 0.0;
    // Krylov workspace
    vec8 *d_V = nullptr, *d_Z = nullptr, *d_x = nullptr, *d_b = nullptr, *d_r = nullptr;
    vec8 *d_xdf = nullptr, *d_ydf = nullptr;  // FP64_DFOP: the operator's input and output as pairs
    int *d_rowctr = nullptr;  // row counter of the dynamically scheduled operator kernel
    double *d_io = nullptr;  // stage-major binary64 staging for inputs / outputs (2 N)
    double *d_H = nullptr;   // (restart+1) x restart Hessenberg, binary64
    double *d_cs = nullptr, *d_sn = nullptr, *d_g = nullptr, *d_yls = nullptr;
    double *d_scal = nullptr;  // scalars: [0] h / norm results ...
    double *h_scal = nullptr;  // pinned host mirror of a few scalars
    void *d_part = nullptr;    // per-CTA partial sums of the reductions
    unsigned int *d_ticket = nullptr;
    unsigned int *d_gbar = nullptr;  // grid-barrier words of k_arnoldi (in d_ticket's allocation)
    int *d_err = nullptr;
    // power-of-two scaling of double-float right-hand sides: [0] the factor
    // applied on the way in, [1] its inverse on the way out
    double *d_vscale = nullptr;
    unsigned long long *d_amax = nullptr;  // |x| bits of the largest magnitude seen
    double jmax = 0.0, mmax = 0.0;         // largest magnitudes of J and M
    int spin = IRK_DEFAULT_SPIN_LIMIT;     // effective irk_options.spin_limit
    irk_kernel_options ko;                 // kernel choices (irk_set_kernel_options)
    int red_blocks = 0;
    irk_stats stats;
    long long launches = 0;
    long long launches_at_stats = 0;  // timing = 2: launch count at the last irk_get_stats
    // timing = 2: phase totals of the marks already read since the last
    // irk_get_stats (marks are read when the stats are asked for, or when
    // IRK_TMARK_FLUSH pairs are pending)
    double tacc_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int tacc_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int mv_variant = -1;  // operator-product launch variant (autotuned on first use)
    // phase timing (irk_options.timing): event pool and (kind, start, end) marks
    std::vector<cudaEvent_t> tev;
    std::vector<int> tkind;
    int tused = 0;
};

// ---- launchers (k_matvec.cu) ----
// number of operator-product launch variants (irk_kernel_options.matvec_variant)
int irk_matvec_variants();
// y = B x (mode 0) or y = rhs - B x (mode 1); form: IRK_TRANSFORMED / UNTRANSFORMED;
// x_f32: every value of x is binary32 (a preconditioned vector from binary32
// factors), which lets the double-float kernel skip the low-word products
int launch_matvec(irk_ctx *c, const vec8 *x, vec8 *y, const vec8 *rhs, double dt, int mode, int x_f32 = 0);
// y = (I (x) J) x in the context's arithmetic (internal layout)
int launch_jacobian(irk_ctx *c, const vec8 *x, vec8 *y);
// operator-product form value for the Jacobian alone (internal; beside the
// public IRK_TRANSFORMED / IRK_UNTRANSFORMED)
#define IRK_FORM_JACOBIAN 2
// raise a kernel's dynamic shared-memory limit to the device maximum (once)
int irk_allow_max_smem(const void *func);
// phase timing marks (api.cu): no-ops unless irk_options.timing
int tmark_begin(irk_ctx *c);
void tmark_end(irk_ctx *c, int slot, int kind);
// stage-major binary64 <-> element-interleaved vec8; scale (device pair or
// null): the way in multiplies by scale[0], the way out by scale[1]
int launch_to_internal(irk_ctx *c, const double *src, vec8 *dst, const double *scale = nullptr);
int launch_to_external(irk_ctx *c, const vec8 *src, double *dst, const double *scale = nullptr);
int launch_to_internal_on(cudaStream_t st, const irk_ctx *c, const double *src, vec8 *dst, const double *scale);
int launch_to_external_on(cudaStream_t st, const irk_ctx *c, const vec8 *src, double *dst, const double *scale);
// scale[0..1] = (2^-e, 2^e) with 2^e <= max_q |src[q]| < 2^(e+1) (1, 1 for a
// zero or non-finite maximum); amax is a device word used as scratch
int launch_pow2_scale(cudaStream_t st, long long n, const double *src, unsigned long long *amax, double *scale);
// J/M (row-major binary64, device) -> internal column-major vec8 blocks;
// records the largest |value| (as binary64 bits) in *amax and raises
// IRK_DEV_ERR_NONFINITE in *err for a NaN or infinity
int launch_convert_blocks(irk_ctx *c, const double *src, vec8 *dst, long long nblocks, unsigned long long *amax,
                          int *err);

// ---- launchers (k_krylov.cu) ----
// Scalars live in 32-byte slots of c->d_scal (128 slots): 0 = norm results,
// 1 = residual estimate, 2 + i = h_{i,j} of the current column, 64 + i = y_i.
#define IRK_SCAL_SLOTS 128
#define IRK_SCAL_BYTES 32
// entries of the per-CTA partial-sum buffer d_part (>= red_blocks)
#define IRK_PART_SLOTS 16384
#define IRK_MAX_RESTART 60
// w <- w - h[hprev_slot] vprev (if vprev), then slot out = <w, v> (self: v = w;
// take_sqrt: store the square root); H_out (if non-null) receives the value.
int launch_axpy_dot_slot(irk_ctx *c, vec8 *w, const vec8 *vprev, int hprev_slot, const vec8 *v,
                         int self, int take_sqrt, int out_slot, double *H_out);
// w <- w / value(slot)  (0 when the value is 0)
int launch_scale_slot(irk_ctx *c, vec8 *w, int slot);
// Givens step for column j; writes the residual estimate to slot 1
int launch_givens(irk_ctx *c, int j, int restart);
// back-substitution for y (size jl+1) and x += Z y
// returns IRK_ERR_INVALID when no cooperative launch is possible (the caller
// runs the step as separate launches); on success the kernel has written
// the iteration's status block (irk_status_ptr: estimate, h_{j+1,j}, error word)
int launch_arnoldi(irk_ctx *c, int j, int restart, vec8 *w);
double *irk_status_ptr(irk_ctx *c);
int launch_lsq_update(irk_ctx *c, int jl, int restart);
// g = (beta, 0, ..., 0) with beta from slot 0
int launch_cycle_start(irk_ctx *c, int restart);
int launch_fill_zero(irk_ctx *c, vec8 *v, long long n);
double *irk_est_ptr(irk_ctx *c);
double *irk_beta_ptr(irk_ctx *c);

// ---- (k_ilu.cu) ----
int pc_build_pattern(irk_ctx *c);  // host: pattern, levels, update lists, uploads
int pc_factor(irk_ctx *c, double dt);
int pc_apply(irk_ctx *c, const vec8 *v, vec8 *z);
void pc_free(PcSystem &p);

// ---- used by the multi-request engine (group.cu), defined in k_ilu.cu ----
int ilu_assemble(cudaStream_t st, int fprec, long long nnz, int m, const AsmEntry *ent, const vec8 *J,
                 const vec8 *M, int df, const double *cm, int ncm, const double *cj, int ncj, void *vals);
int ilu_factor_level(cudaStream_t st, int fprec, const int *rows, int nrows, int b, const int *rp, const int *ci,
                     const int *diag, const int *upd_ptr, const int *upd, void *vals, void *dinv, int *err);
int ilu_sweep_group(cudaStream_t st, int dev, int fprec, int df, int nitems, int b, int max_item_blocks,
                    const int *lo, const int *up, const int *rp, const int *ci, const int *voff, const void *vals,
                    const void *dinv, vec8 *vpool, unsigned long long *llpool, int ep, int *err,
                    const int *lane_of_row, const long long *vin, const long long *zout, const long long *yll,
                    const long long *zll, int spin);

// ---- helpers (api.cu) ----
int cuda_status(cudaError_t e);
