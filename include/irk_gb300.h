/*
 * irk_gb300.h -- C ABI of the GB300 (sm_103a) stage-system solver.
 *
 * One call of irk_factor + irk_solve performs the per-time-step linear solve
 * of a fully implicit s-stage Runge-Kutta method applied to a discontinuous
 * Galerkin semi-discretisation M du/dt = f(u) (Pazner & Persson,
 * arXiv 1701.07181):
 *
 *     B W = R,   B = A^{-1} (x) M - dt (I_s (x) J)          (Sec. 4.3, eq. big-irk)
 *
 * (the "transformed" system of Sec. 4.1, eq. modified-IRK), or optionally the
 * untransformed system (I_s (x) M - dt (A (x) J)) K = R (Sec. 4.1,
 * eq. newton-system-2), by restarted flexible GMRES (Sec. 4) preconditioned
 * with block ILU(0) (Sec. 4.2-4.3).  The new step is u1 = u0 + dt w_s
 * (Sec. 4.1: b^T A^{-1} = e_s^T for Radau IIA).
 *
 * Notation (Sec. 2.1): T elements, m unknowns per element, n = T m; J is a
 * T x T block matrix of dense m x m blocks (diagonal + one block per face
 * neighbour), M is block diagonal.
 *
 * Data layout at this boundary (all row-major, all double):
 *   row_ptr[T+1], col_idx[nnzb]  block-CSR pattern of J, int32, columns sorted
 *                                ascending within a row, diagonal present.
 *   J[nnzb*m*m]                  blocks of J in pattern order, each m x m
 *                                row-major.
 *   M[T*m*m]                     diagonal blocks of M, each m x m row-major.
 *   R, W[s*T*m]                  stage vectors stacked stage-major:
 *                                X[(k*T + i)*m + a] = component a of element
 *                                i of stage k (the stacking of Sec. 4.1).
 *
 * Memory spaces: every pointer argument that carries data is in the memory
 * space given by the call's mem_space argument (IRK_HOST: host memory, the
 * library copies through its own staging; IRK_DEVICE: device memory of the
 * context's GPU).  The caller keeps ownership of every buffer it passes; the
 * library copies inputs into buffers it owns and writes outputs into the
 * caller's buffers.  No pointer is retained after a call returns.
 *
 * Errors: every int-returning call returns IRK_OK (0), IRK_NOT_CONVERGED (1,
 * a result is still written), or a negative IRK_ERR_* code; irk_strerror
 * gives a message.  A context is not thread safe; distinct contexts are
 * independent.  All work of a context is ordered on the stream in its options
 * (NULL = the legacy default stream); calls return after that work completed.
 */
#ifndef IRK_GB300_H
#define IRK_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define IRK_API __attribute__((visibility("default")))
#else
#define IRK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct irk_ctx irk_ctx;

enum irk_status {
    IRK_OK = 0,
    IRK_NOT_CONVERGED = 1, /* max_iter reached; best iterate written */
    IRK_ERR_INVALID = -1,  /* bad argument or pattern */
    IRK_ERR_NOMEM = -2,    /* device or host allocation failed */
    IRK_ERR_SINGULAR = -3, /* zero pivot in a diagonal block of the ILU(0) */
    IRK_ERR_NONFINITE = -4,/* NaN/Inf in an input (J, M, R) or a Krylov quantity */
    IRK_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    IRK_ERR_CUDA = -6,     /* a CUDA runtime call failed */
    IRK_ERR_STATE = -7,    /* call out of order (e.g. apply before factor) */
    IRK_ERR_SCRATCH_LIMIT = -8 /* problem too large for the fixed scratch of
                                  irk_apply_precond_noalloc */
};

enum irk_mem_space { IRK_HOST = 0, IRK_DEVICE = 1 };

/* Preconditioners (Sec. 4.3). */
enum irk_precond_kind {
    IRK_PC_NONE = 0,
    /* Sec. 4.3.2: s independent block ILU(0) factors of
     * (A^{-1}_kk + alpha_k) M - dt J, applied to all stages at once. */
    IRK_PC_UNCOUPLED = 1,
    /* Sec. 4.3.1, Alg. 3: block ILU(0) of the whole system with the
     * unknowns ordered stage-major (stage, element). */
    IRK_PC_COUPLED = 2,
    /* block ILU(0) of the whole system ordered element-major, with one
     * (s m) x (s m) block per element pair (any formulation). */
    IRK_PC_ELEMENT = 3
};

/* Storage / arithmetic precision of the ILU(0) factors and sweeps. */
enum irk_factor_precision { IRK_FACTOR_FP64 = 0, IRK_FACTOR_FP32 = 1, IRK_FACTOR_BF16 = 2 };

/* Arithmetic of the outer Krylov method (operator product, Gram-Schmidt,
 * residuals).  FP64: IEEE binary64 on the FP64 pipe.  DF64: double-float
 * (pairs of binary32 with error-free transformations, about 48 significant
 * bits) on the FP32 pipe, which GB300 executes about 60x faster.
 * FP64_DFOP: binary64 Krylov vectors, Gram-Schmidt, Givens rotations and
 * true residual, with the operator product alone in double-float: J and M
 * are held as double-float pairs, each product's input is split into pairs
 * before it and its result rounded back to binary64 after it (the residual
 * form subtracts in binary64); the operator's accuracy is double-float's
 * (about 1e-14 relative), the rest of the iteration binary64's.  J, M, dt and
 * right-hand sides are treated as for DF64 (range checks and power-of-two
 * scaling below).  Not accepted by irk_group_create. */
enum irk_krylov_arith { IRK_KRYLOV_FP64 = 0, IRK_KRYLOV_DF64 = 1, IRK_KRYLOV_FP64_DFOP = 2 };

enum irk_formulation { IRK_TRANSFORMED = 0, IRK_UNTRANSFORMED = 1 };

/* Orthogonalisation of the Arnoldi process (Sec. 4 does not fix it).  MGS:
 * modified Gram-Schmidt, j + 2 dependent inner products in step j.  CGS2:
 * classical Gram-Schmidt applied twice: all inner products of a pass at
 * once, two passes, so two grid-wide reductions per step whatever j; it
 * reads the basis three times against MGS's twice.  Both keep the basis
 * orthonormal to working precision; the iterates differ by rounding. */
enum irk_orthogonalization { IRK_ORTHO_MGS = 0, IRK_ORTHO_CGS2 = 1 };

/* Scheduling of the preconditioner's block triangular sweeps.  AUTO: one
 * persistent launch per application, rows synchronised through published
 * values (block size <= 128), unless the levels are wide (on average >= 4096
 * block rows per level, e.g. a multicolour order), where one launch per
 * level is faster.  LEVELS: one launch per level of the block-triangular
 * dependency graph. */
enum irk_sweep_mode { IRK_SWEEP_AUTO = 0, IRK_SWEEP_LEVELS = 1 };

/* Elimination order of the element blocks in the ILU(0) factorisation (the
 * paper leaves the ordering open).  NATURAL: the input element order.
 * MULTICOLOR: first-fit greedy colouring of the face-neighbour graph in
 * input order, then elements sorted by (colour, index); on a two-colourable
 * mesh every sweep has two levels.  A different order is a different
 * preconditioner (same operator, same solution, other iteration count).
 * Orderings and partitions apply to the stage-major kinds (UNCOUPLED,
 * COUPLED); IRK_PC_ELEMENT accepts only the natural, unpartitioned form. */
enum irk_ordering { IRK_ORDER_NATURAL = 0, IRK_ORDER_MULTICOLOR = 1 };

typedef struct {
    int restart;       /* GMRES restart length (default 30) */
    int max_iter;      /* total inner iterations (default 3000) */
    int precond;       /* enum irk_precond_kind (default IRK_PC_UNCOUPLED) */
    int factor_prec;   /* enum irk_factor_precision (default IRK_FACTOR_FP64) */
    int krylov_arith;  /* enum irk_krylov_arith (default IRK_KRYLOV_FP64) */
    int formulation;   /* enum irk_formulation (default IRK_TRANSFORMED) */
    const double *shift; /* host array of s shifts alpha_k for IRK_PC_UNCOUPLED;
                            NULL = alpha_k = sum_{j != k} |A^{-1}_jk| (Sec. 4.3.2);
                            copied at irk_setup */
    void *stream;      /* cudaStream_t for all work of the context; NULL = default */
    int timing;        /* 1: time each phase of irk_factor / irk_solve with CUDA
                          events on the context's stream (see irk_stats); the
                          events are read back at the end of each call.
                          2: the same events, left unread until irk_get_stats,
                          which then reports the phase times, phase counts
                          and kernel launches summed over every irk_factor /
                          irk_solve since the previous irk_get_stats call (no
                          event query on the solve's path).  Default 0 */
    int sweep;         /* enum irk_sweep_mode: how the preconditioner sweeps run */
    int ordering;      /* enum irk_ordering: elimination order of the ILU(0) */
    int partitions;    /* > 1: partitioned ILU(0) (Sec. 4.5) with this many
                          contiguous ranges of element indices; 0/1: none */
    const int32_t *partition; /* optional host array of T partition ids (overrides
                          partitions); blocks coupling two different ids are
                          dropped from the preconditioner; copied at irk_setup */
    int stage_jacobians; /* 0 (default): one J shared by all stages, J holds
                          nnzb*m*m values.  1: one Jacobian per stage (Sec. 4.1,
                          J_k at the state of stage k), J holds s*nnzb*m*m
                          values, stage after stage; stage k's rows use J_k
                          (transformed: A^{-1} (x) M - dt diag(J_1..J_s);
                          untransformed: I (x) M - dt [a_kl J_k]).  Not
                          accepted by irk_group_create. */
    int spin_limit;    /* polls a device-side wait on another thread block
                          makes before it gives up: the persistent sweep's
                          waits for published rows and the grid barrier of the
                          Arnoldi launch.  A wait that gives up records
                          IRK_ERR_TIMEOUT, lets its own bulk copies land and
                          leaves the kernel; the call returns IRK_ERR_TIMEOUT
                          and the context stays usable.  0 (default) = 2^20
                          polls (about a second); must be >= 0. */
    int orthogonalization; /* enum irk_orthogonalization (default IRK_ORTHO_MGS);
                          irk_group_create accepts MGS only */
} irk_options;

/* Fill *opt with the defaults listed above. */
IRK_API void irk_default_options(irk_options *opt);

/* Magnitude range of the double-float Krylov arithmetic (IRK_KRYLOV_DF64, and
 * IRK_KRYLOV_FP64_DFOP, whose operator product is double-float).
 * A double-float value is a pair of binary32 numbers, so its exponent range
 * is binary32's: a magnitude above about 3.4e38 overflows, and below about
 * 1e-31 the low word turns subnormal and the value keeps fewer than 48
 * significant bits.  The library therefore
 *   - refuses (IRK_ERR_INVALID, at irk_setup / irk_update_values) a J or M
 *     whose largest magnitude is neither 0 nor within
 *     [IRK_DF64_MIN_MAGNITUDE, IRK_DF64_MAX_MAGNITUDE] (2^-100 .. 2^100,
 *     about 7.9e-31 .. 1.3e30), and (at irk_factor / irk_solve) a dt with
 *     dt * max|J| above IRK_DF64_MAX_MAGNITUDE;
 *   - scales every right-hand side (irk_solve, irk_apply_operator,
 *     irk_apply_precond) by the power of two that brings its largest
 *     magnitude into [1, 2) before the conversion to double-float, and the
 *     result back by the inverse power: exact in binary64, so R of any
 *     finite magnitude is accepted and, away from the binary32 limits, the
 *     result is bit for bit the unscaled one.
 * IRK_KRYLOV_FP64 has binary64's range and none of these limits. */
#define IRK_DF64_MIN_MAGNITUDE 7.888609052210118e-31 /* 2^-100 */
#define IRK_DF64_MAX_MAGNITUDE 1.2676506002282294e30 /* 2^100 */

/* Create a context for one stage system (Sec. 4.1, eq. big-irk).
 *   s         number of stages, 1 <= s <= 8.
 *   A         host s*s row-major Butcher matrix, invertible; NULL = Radau IIA
 *             with s stages (App. A; computed by collocation).
 *   T, m      elements and block size, T >= 1, 1 <= m <= 128; with binary64
 *             factors m <= 120 (the factorisation keeps two b x b blocks
 *             and a column in one CTA's 227 KB of shared memory; b = m, or
 *             s m for IRK_PC_ELEMENT), else IRK_ERR_INVALID.
 *   row_ptr, col_idx, J, M   as in the layout notes above, in mem_space.
 *   opt       NULL = defaults.  The pattern must be structurally symmetric.
 * Copies everything; allocates the Krylov workspace for the given restart.
 * Returns IRK_ERR_INVALID for a malformed pattern (unsorted, missing
 * diagonal, out-of-range column, not symmetric) or, with IRK_KRYLOV_DF64,
 * values outside the double-float range above; IRK_ERR_NONFINITE when J or
 * M holds a NaN or an infinity (checked while the values are copied in). */
IRK_API int irk_setup(irk_ctx **out, int s, const double *A, int T, int m, const int32_t *row_ptr,
              const int32_t *col_idx, const double *J, const double *M, int mem_space,
              const irk_options *opt);

/* Replace the values of J and M (same pattern; J holds s Jacobians when
 * the context was set up with stage_jacobians = 1), e.g. at a new Newton
 * iterate (Sec. 4.1).  Invalidates the factors.  IRK_ERR_NONFINITE for a NaN
 * or infinity in J or M, IRK_ERR_INVALID for values outside the
 * double-float range (IRK_KRYLOV_DF64); the context then holds no usable
 * values until a later irk_update_values succeeds. */
IRK_API int irk_update_values(irk_ctx *ctx, const double *J, const double *M, int mem_space);

/* Build the preconditioner for time step dt (once per linear solve,
 * Sec. 4.4): assemble the system blocks and compute their block ILU(0)
 * (Alg. 2 / Alg. 3 / textbook form), level by level.  IRK_ERR_SINGULAR if a
 * diagonal block has a zero pivot. */
IRK_API int irk_factor(irk_ctx *ctx, double dt);

/* Solve B W = R (or the untransformed system for K) to
 * ||R - B W||_2 <= rtol ||R||_2 by restarted right-preconditioned FGMRES
 * from W = 0.  Refactors if dt differs from the factored dt.
 *   R, W      s*T*m stage-major, in mem_space; W may not alias R.
 *   iters     total inner iterations (may be NULL).
 *   relres    final true relative residual ||R - B W|| / ||R|| (may be NULL).
 * Returns IRK_OK, IRK_NOT_CONVERGED (W holds the last iterate) or an error. */
IRK_API int irk_solve(irk_ctx *ctx, const double *R, double dt, double rtol, double *W, int mem_space,
              int *iters, double *relres);

/* Step outputs from a stage solution W of the transformed system (Sec. 4.1:
 * W stacks w_i = sum_j a_ij k_j): the stage derivatives
 *     K = (A^{-1} (x) I_n) W,   k_i = sum_j (A^{-1})_ij w_j,
 * and the new state
 *     u1 = u0 + dt (b^T A^{-1} (x) I_n) W
 * (Radau IIA: b^T A^{-1} = e_s^T, so u1 = u0 + dt w_s).  One binary64 pass
 * over W on the context's stream; the sums run over j in increasing order.
 *   W    s*T*m stage-major (as irk_solve writes it), in mem_space.
 *   b    host array of the s weights, or NULL: b = the last row of A (a
 *        stiffly accurate tableau, as the built-in Radau IIA), and then
 *        b^T A^{-1} = e_s^T is used exactly.
 *   u0   T*m in mem_space, or NULL when u1 is NULL.
 *   K    s*T*m stage-major output in mem_space, or NULL.
 *   u1   T*m output in mem_space, or NULL.
 * Host buffers go through a device temporary allocated for the call.
 * IRK_ERR_INVALID for a NULL context or W, u1 without u0, or a bad mem_space;
 * IRK_ERR_NOMEM if the temporary cannot be allocated. */
IRK_API int irk_step_outputs(irk_ctx *ctx, const double *W, const double *b, const double *u0, double dt,
                             double *K, double *u1, int mem_space);

/* Y = B X for the context's formulation and dt (the operator product of
 * Sec. 4.1 alone; Table 2's transformed / untransformed matrix-vector
 * product).  X, Y stage-major s*T*m in mem_space. */
IRK_API int irk_apply_operator(irk_ctx *ctx, const double *X, double *Y, double dt, int mem_space);

/* Z = P^{-1} V with the current factors (Sec. 4.2-4.3); IRK_ERR_STATE if
 * irk_factor has not run.  V, Z stage-major s*T*m in mem_space. */
IRK_API int irk_apply_precond(irk_ctx *ctx, const double *V, double *Z, int mem_space);

/* Preconditioner application that allocates nothing.
 * The paper has no counterpart; this is a convenience of this library.
 *
 * Who needs it: callers that cannot allocate device memory at the moment
 * they apply the preconditioner -- for instance a time-stepping driver whose
 * GPU memory is entirely held by another allocator's pool (a framework's
 * caching allocator that has already reserved the device), or a loop with a
 * rule against allocation after start-up because cudaMalloc synchronises the
 * device and stalls latency-critical work.  irk_apply_precond uses buffers the
 * context allocated at irk_setup; this variant instead keeps its working
 * vectors in one fixed array of IRK_NOALLOC_SCRATCH_BYTES bytes that the
 * library declares in device memory, so the call itself never calls
 * cudaMalloc, cudaFree or any allocating routine.
 *
 * Computes Z = P^{-1} V exactly like irk_apply_precond (same kernels, same
 * factors) for a context that irk_factor has prepared.
 *   V, Z    DEVICE pointers, s*T*m values, stage-major (as irk_solve); Z must
 *           not alias V.  The caller owns both.
 *   stream  cudaStream_t to run on (NULL = legacy default stream); the call
 *           waits for its own work before returning.
 * Limits and errors:
 *   - the working set is 16 + 16*w bytes per unknown (w = 1 with FP32/BF16
 *     factors, 2 with FP64 factors) plus 256 bytes; a larger system returns
 *     IRK_ERR_SCRATCH_LIMIT (up to 2,097,120 unknowns with FP32/BF16
 *     factors, 1,398,080 with FP64 factors);
 *   - IRK_ERR_STATE if the context is not factored; IRK_ERR_INVALID if it has
 *     no preconditioner, uses per-level sweeps (block size > 128,
 *     IRK_SWEEP_LEVELS, or AUTO choosing per-level launches for wide levels),
 *     or belongs to another device than the current one;
 *   - the device error word of the sweep is reported in full: IRK_ERR_SINGULAR,
 *     IRK_ERR_NONFINITE or IRK_ERR_TIMEOUT (a wait on another thread block
 *     that gave up, see irk_options.spin_limit), in that order of precedence.
 * Set-up: the first call on a device (with that device current) looks up
 * the array's device address once; make that first call before any stream
 * capture.  The array is shared by every call on a device and keeps the last
 * call's contents (each call clears what it needs cleared), so calls that
 * overlap on the GPU -- from several threads or streams at once -- race and
 * must be serialised by the caller.  Every GPU that loads the library holds
 * the array until the process exits. */
#define IRK_NOALLOC_SCRATCH_BYTES (64u << 20)
IRK_API int irk_apply_precond_noalloc(irk_ctx *ctx, const double *V, double *Z, void *stream);

/* ------------------------------------------------------------------------
 * Multi-request engine (continuous batching).
 *
 * An irk_group holds many independent stage systems (one per request: its
 * own mesh pattern, J, M, right-hand side, dt and rtol) of one class --
 * same s, Butcher matrix, block size m and options -- in device pools sized
 * at creation.  irk_group_step advances every active request by one FGMRES
 * iteration with one launch per phase for all of them (the operator product
 * of all requests, one persistent sweep over the level-merged rows of all
 * requests, Gram-Schmidt with per-request deterministic reductions, Givens
 * rotations per request).  Requests are submitted and collected between
 * steps: a request that arrives while others are being solved joins at the
 * next step, and a finished request frees its pools for the next.
 * Each request follows exactly the algorithm of irk_solve (same
 * preconditioner, same stopping test); only its floating-point reductions
 * are partitioned differently, so its result matches irk_solve within the
 * solve tolerance.  Preconditioners: IRK_PC_UNCOUPLED or IRK_PC_NONE;
 * factors FP32 or FP64; any ordering; formulation transformed.
 * ------------------------------------------------------------------------ */
typedef struct irk_group irk_group;

/* max_elements / max_blocks: capacity in elements and J blocks summed over the
 * requests held at once; max_requests: most requests held at once. */
IRK_API int irk_group_create(irk_group **out, int s, const double *A, int m, int max_elements,
                             int max_blocks, int max_requests, const irk_options *opt);

/* Admit one request (copies everything; factors it for dt on the device).
 * Layouts as for irk_setup / irk_solve (R stage-major), in mem_space.
 * Returns IRK_ERR_NOMEM when the pools cannot hold it now (retry after a
 * request has been collected); *slot receives the request's handle. */
IRK_API int irk_group_submit(irk_group *g, int T, const int32_t *row_ptr, const int32_t *col_idx,
                             const double *J, const double *M, const double *R, double dt,
                             double rtol, int mem_space, int *slot);

/* One FGMRES iteration for every active request (plus the residual and
 * restart bookkeeping of requests at a cycle boundary).  *n_active receives
 * the number of requests not yet finished. */
IRK_API int irk_group_step(irk_group *g, int *n_active);

/* State of a request: returns 1 while it runs, 0 when finished (its result
 * may be collected), or an error code.  iters / relres / status may be NULL;
 * status receives IRK_OK, IRK_NOT_CONVERGED or an error of the request. */
IRK_API int irk_group_query(const irk_group *g, int slot, int *iters, double *relres, int *status);

/* Copy a finished request's W (s*T*m, stage-major) to mem_space and free its
 * slot and pools. */
IRK_API int irk_group_collect(irk_group *g, int slot, double *W, int mem_space);

/* Device bytes the group holds (pools and work arrays). */
IRK_API long long irk_group_device_bytes(const irk_group *g);

IRK_API void irk_group_destroy(irk_group *g);

/* ---------------------------------------------------------------------------
 * Diagonally implicit Runge-Kutta steps (Sec. 3, Table 1, App. A: the DIRK
 * comparison schemes DIRK33 and ESDIRK65, or any lower-triangular tableau).
 *
 * One step of M u' = J u (the linear(ised) system whose stage equations are
 * M k_k = J (u0 + dt sum_j a_kj k_j)) with a lower-triangular A: stage k
 * solves the single n x n system
 *     (M - dt a_kk J) k_k = J (u0 + dt sum_{j<k} a_kj k_j),   n = T m,
 * by restarted FGMRES preconditioned with the block ILU(0) of that matrix
 * (the baseline DIRK solver of Sec. 5), or, when a_kk = 0 (the explicit
 * first stage of an ESDIRK scheme), M k_k = J u0 (block-diagonal M: one
 * iteration with its exact block factorisation); then
 *     u1 = u0 + dt sum_k b_k k_k.
 * Stages with the same a_kk share one factorisation per dt (one for all
 * implicit stages of DIRK33 or ESDIRK65).  Sec. 5 counts the cost of a step
 * as equivalent multiplications: the sum of the stages' iterations.
 * -------------------------------------------------------------------------*/
typedef struct irk_dirk irk_dirk;

/* Create a DIRK stepper.
 *   s         stages, 1 <= s <= 8; A host s*s row-major, lower triangular
 *             (entries above the diagonal exactly 0), a_kk >= 0; b host s
 *             weights.
 *   T, m, row_ptr, col_idx, J, M, mem_space   as for irk_setup.
 *   opt       NULL = defaults; restart, max_iter, factor_prec, krylov_arith,
 *             stream, sweep, ordering and partitions are used; the
 *             preconditioner is the block ILU(0) of each stage matrix
 *             (IRK_PC_NONE in opt->precond switches it off).
 * Copies everything (one single-stage context per distinct nonzero a_kk,
 * plus one for explicit stages).  IRK_ERR_INVALID for a bad tableau. */
IRK_API int irk_dirk_setup(irk_dirk **out, int s, const double *A, const double *b, int T, int m,
                           const int32_t *row_ptr, const int32_t *col_idx, const double *J, const double *M,
                           int mem_space, const irk_options *opt);

/* One step from u0 (T*m values in mem_space) with step dt; every stage solve
 * to relative residual rtol.
 *   u1        T*m result in mem_space.
 *   K         s*T*m stage derivatives k_1..k_s (stage-major) or NULL.
 *   iters     s per-stage iteration counts (0 for explicit stages) or NULL.
 *   relres    largest final relative residual over the stages or NULL.
 * Returns IRK_OK, IRK_NOT_CONVERGED (a stage hit max_iter; u1 still formed
 * from the last iterates) or an error. */
IRK_API int irk_dirk_step(irk_dirk *d, const double *u0, double dt, double rtol, double *u1, double *K,
                          int mem_space, int *iters, double *relres);

IRK_API void irk_dirk_destroy(irk_dirk *d);

/* Counters of the last irk_factor / irk_solve (host values). */
typedef struct {
    int iters, cycles, levels_lower, levels_upper;
    double relres, factor_ms, solve_ms;
    long long kernel_launches;  /* kernels launched by the last factor + solve
                                   (timing = 2: since the previous irk_get_stats) */
    /* with irk_options.timing = 1 (else 0): device time of each phase of the
     * last irk_solve, summed over its calls, from CUDA events on the stream
     * (timing = 2: over every call since the previous irk_get_stats) */
    double matvec_ms, precond_ms, ortho_ms;
    int n_matvec, n_precond, n_ortho;
    /* launch variant of the operator product chosen by the autotuner for this
     * context's (m, s, arithmetic): 0-3 register-streaming kernel (chunk
     * width 8/4/2 columns, 256/128 threads), 4-6 bulk-copy pipelined kernel
     * (2 or 3 shared-memory stages, one or two CTAs per SM; where a stage does
     * not fit or m is odd it runs variant 0's launch), 7 register-streaming
     * kernel with the block size fixed at compile time (double-float Krylov,
     * s = 2..4, m = 12, 20, 24, 40 or 50; else variant 0's launch), 8 the
     * same register-blocked (four rows per thread, two for m = 50), 9 as 7
     * with eight columns of loads in flight per thread, 10 as 7 with the
     * block loads issued one chunk ahead, 11 the TMA-fed kernel (a producer
     * warp streams 8-column chunks of the blocks and the matching stage
     * values into shared memory, the other warps compute from there), 12
     * and 13 the TMA-fed kernel with 16-column chunks and two units in
     * flight, and with 8-column chunks and three, 14-16 the TMA-fed kernel
     * with two rows per consumer thread in packed two-lane binary32
     * arithmetic and about 128 consumer threads per CTA ((8, 3) and (8, 2)
     * chunk columns and units, and (8, 2) with registers capped for five
     * CTAs per SM), 17 and 18 the (8, 2) two-row kernel taking element rows
     * from a run-time counter (five and four CTAs per SM); -1 before the
     * first product.  irk_kernel_options.matvec_variant pins the variant.  Every variant
     * gives the same result bit for bit. */
    int matvec_variant;
    /* with irk_options.timing = 1: device time of the kernels of the last
     * factorisation (assembly of the blocks, block products, inversion of
     * the diagonal blocks) and of the forward and backward sweeps of the
     * last irk_solve's preconditioner applications (per-level sweeps only;
     * 0 for the persistent form) */
    double factor_assemble_ms, factor_products_ms, factor_inverse_ms;
    double sweep_fwd_ms, sweep_bwd_ms;
    /* levels of the last factorisation whose block products ran as whole
     * staged rows (binary32 factors, every update of a lower block landing on
     * its row's diagonal block: Alg. 2 with the row's products independent);
     * irk_kernel_options.factor_fused = 0 turns that kernel off */
    int factor_fused_levels;
    /* 1 when the last preconditioner application ran in the two-colour form:
     * two launches, the forward sweep of the second colour fused with its
     * diagonal-block products, then the backward sweep of the first colour
     * (two lower levels, the second without upper entries, as the
     * two-colour order gives on a two-colourable mesh); 0 otherwise.
     * irk_kernel_options.sweep_two_colour = 0 turns that form off. */
    int sweep_two_colour;
} irk_stats;
IRK_API int irk_get_stats(const irk_ctx *ctx, irk_stats *out);

/* Kernel choices of a context.  The defaults are the library's own choices;
 * the other values select alternative launch forms of the same computation,
 * for measurement and for the tests that compare the forms.  Every choice
 * gives the same result bit for bit except where noted. */
typedef struct {
    int matvec_variant;     /* -1 (default): operator-product launch variant
                               autotuned per (m, s, arithmetic); 0..18 pin one
                               (see irk_stats.matvec_variant) */
    int sweep_two_colour;   /* 1 (default): the two-launch preconditioner
                               application where the element order allows it
                               (see irk_stats.sweep_two_colour); 0: the level
                               sweeps */
    int sweep_compiled_levels; /* 1 (default): level sweeps of binary32 factors
                               with double-float Krylov vectors by kernels
                               compiled for block sizes 12/20/24/40/50; 0: the
                               generic level kernels */
    int sweep_shared_upper; /* 1 (default): backward sweeps read each upper
                               block once for all stages where no factor update
                               reaches the upper blocks; 0: once per stage */
    int factor_fused;       /* 2 (default): staged-row block products, the
                               compile-time form for block sizes 12/20/24/40/50;
                               1: the generic staged-row kernel; 0: one lower
                               entry at a time (the factors of the staged-row
                               forms differ from it by binary32 rounding: they
                               sum a row's Schur updates in one accumulator) */
    int factor_gj_rows;     /* 1 (default): Gauss-Jordan inverses with one block
                               row per thread in registers for block sizes
                               12/20/24/40/50; 0: the shared-memory kernel */
    int factor_gj_threads;  /* threads per CTA of the shared-memory inversion
                               kernel, 32..256; 0 (default) = 128 */
    int factor_gj_split_min;/* rows in a level from which its inversions run in
                               their own launch after its products; 0
                               (default) = 2048, 1 = always */
    int arnoldi_form;       /* 0 (default): one launch per Arnoldi step, the
                               vector kept in shared memory when a slice fits;
                               1: the streaming form, 1024-thread CTAs; 2: the
                               streaming form, 256-thread CTAs */
} irk_kernel_options;

/* Fill *ko with the defaults listed above. */
IRK_API void irk_default_kernel_options(irk_kernel_options *ko);

/* Set the kernel choices of a live context for the calls that follow (a
 * pinned operator-product variant takes effect at the next product).
 * IRK_ERR_INVALID for a NULL argument or a value out of range. */
IRK_API int irk_set_kernel_options(irk_ctx *ctx, const irk_kernel_options *ko);

/* Change irk_options.spin_limit of a live context for the calls that follow
 * (0 = the default of 2^20 polls).  IRK_ERR_INVALID for a negative value or
 * a NULL context. */
IRK_API int irk_set_spin_limit(irk_ctx *ctx, int spin_limit);

/* Change irk_options.timing of a live context (0, 1 or 2) for the calls that
 * follow, e.g. to time a sample of a long run.  Leaving timing = 2 keeps the
 * marks already recorded: the next irk_get_stats made with timing = 2 still
 * reports them.  IRK_ERR_INVALID for another value or a NULL context. */
IRK_API int irk_set_timing(irk_ctx *ctx, int timing);

/* Release every resource of the context (NULL is allowed). */
IRK_API void irk_destroy(irk_ctx *ctx);

/* Static message for a status code. */
IRK_API const char *irk_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* IRK_GB300_H */
