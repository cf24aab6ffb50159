/*
 * sislice.h -- C ABI of the GB300 slice-solve library (shift-invert spectrum slicing
 * of a sparse symmetric-definite pencil, A x = lambda B x, A symmetric, B SPD;
 * problem statement Eq. 1 of arXiv 1908.06043).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an ss_status.  SS_OK is 0; on failure ss_last_error(ctx)
 *   returns a one-line message (owned by the context, valid until the next call).
 * - "device" pointers are CUDA global-memory pointers on the context's device;
 *   "host" pointers are ordinary CPU memory.  The caller owns every buffer it passes
 *   and the CUDA stream; the library owns the opaque handles and frees their memory
 *   in the matching *_destroy call.  No call allocates memory that the caller sees.
 * - All device work is ordered on the context's stream.  Calls that return host
 *   values (ss_inertia, ss_slice_solve, ss_dos_estimate) synchronise that stream.
 * - Dense blocks of vectors (V, X, right-hand sides) are N x k ROW-MAJOR: element
 *   (i, j) -- component i of vector j -- sits at offset i*k + j.
 * - The sparse pattern is the FULL symmetric CSR pattern of A union B (both triangles
 *   stored, diagonal included, column indices sorted within each row); value arrays
 *   a_vals / b_vals are aligned with it (an entry absent from one matrix is an
 *   explicit 0).  Indices are 0-based.
 */
#ifndef SISLICE_H
#define SISLICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ss_status;
enum {
    SS_OK = 0,
    SS_ERR_ARG = 1,       /* bad argument (null pointer, size, index out of range)   */
    SS_ERR_CUDA = 2,      /* a CUDA runtime call failed                               */
    SS_ERR_OOM = 3,       /* device or host allocation failed                        */
    SS_ERR_SINGULAR = 4,  /* a pivot fell below the threshold: sigma is (near) an
                             eigenvalue; move sigma and refactor                      */
    SS_ERR_NOT_SPD = 5,   /* B is not positive definite (DOS needs its Cholesky)      */
    SS_ERR_NOCONV = 6,    /* the in-slice iteration hit its iteration cap             */
    SS_ERR_TIMEOUT = 7,   /* a bounded device wait expired                            */
    SS_ERR_INTERNAL = 8
};

enum { SS_FP64 = 0, SS_MIXED = 1 };      /* factor precision                     */
enum { SS_MIXED_TC = 3 };                  /* FP64 fronts, FP32 solves from the rounded factor */
enum { SS_INERTIA_ONLY = 4 };              /* or-ed into the precision of ss_factor: FP64
                                              fronts, only the inertia is kept          */
enum { SS_FP64_SOLVE32 = 2 };              /* reported only: FP64 factor, FP32 solves */
enum { SS_SUBSPACE = 0, SS_BLOCK_LANCZOS = 1 };  /* in-slice driver             */

typedef struct ss_ctx ss_ctx;
typedef struct ss_symbolic ss_symbolic;
typedef struct ss_numeric ss_numeric;

/* Options of the symbolic analysis.  Zero fields take the defaults in brackets. */
typedef struct ss_options {
    int32_t nd_leaf;        /* nested dissection stops at this many vertices [64]    */
    int32_t panel;          /* panel width of the blocked front factorisation [64]   */
    int32_t reserved[6];
} ss_options;

/* Summary of a symbolic analysis (all counts are exact, from the analysis). */
typedef struct ss_symbolic_info {
    int64_t n, nnz;
    int64_t n_supernodes, n_levels, n_panels, n_panel_levels;
    int64_t max_front;          /* largest front dimension m                        */
    int64_t factor_entries;     /* sum over supernodes of m * ncol (stored L panels) */
    int64_t front_entries;      /* sum over supernodes of m * m (front arena)        */
    double factor_flops;        /* algorithmic sparse LDL^T flops: sum over
                                   supernodes of s^3/3 + s^2 b + s b^2, s = ncol,
                                   b = off-diagonal rows                             */
    double schur_flops;         /* Schur-update flops per factorisation: sum over panel
                                   steps of 2 w r(r+1)/2 (lower triangle, r trailing
                                   rows, w panel width)                              */
    double panel_flops;         /* panel-transform flops: sum of 2 r w^2             */
    int64_t l_offdiag_entries;  /* sum over panels of r w: L entries below the panel
                                   diagonal blocks (read once per triangular sweep)  */
    int64_t l_diag_entries;     /* sum over panels of w^2                            */
    double analyze_seconds;
    /* memory plan of one shift's factorisation (entries of the factor's type):         */
    int64_t l_storage_entries;  /* L kept for the solves: sum of m * ncol, 256-byte
                                   aligned blocks                                   */
    int64_t workspace_entries;  /* the fronts of the widest level (reused per level) */
    int64_t cb_pool_entries;    /* peak of the contribution blocks awaiting their
                                   parent's extend-add                              */
} ss_symbolic_info;

/* Per-probe statistics of one slice solve. */
typedef struct ss_probe_stats {
    int32_t iterations;         /* operator applications of the in-slice driver      */
    int32_t refine_steps;       /* total FP64 refinement corrections applied         */
    int32_t converged;          /* 1 when every Ritz value in (lo, hi] met tol       */
    int32_t reserved;
    double max_resid_in_slice;  /* max normalised residual over Ritz values in slice */
    double seconds;
} ss_probe_stats;

/* Options of one slice solve.  Zero fields take the defaults in brackets. */
typedef struct ss_solve_opts {
    int32_t driver;             /* SS_SUBSPACE | SS_BLOCK_LANCZOS [SS_SUBSPACE]      */
    int32_t max_iter;           /* SS_SUBSPACE: iteration cap [200];
                                   SS_BLOCK_LANCZOS: Krylov blocks in the basis [6]  */
    int32_t check_every;        /* Rayleigh-Ritz + residual check period [1]; c < 0:
                                   first check after |c| iterations, later ones where
                                   the residual's reduction per iteration between the
                                   last two checks predicts convergence (1 .. 8 apart) */
    int32_t refine;             /* FP64 refinement corrections per solve, mixed
                                   factor only [2]                                   */
    double tol;                 /* normalised residual target [1e-10]                */
    int32_t n_expect;           /* keep iterating until at least this many Ritz values
                                   lie in (lo, hi] (e.g. an inertia count) [0]        */
    int32_t k_out;              /* Ritz pairs returned (SS_BLOCK_LANCZOS: the k_out
                                   nearest sigma, <= k * max_iter) [k]               */
    int32_t refine_from_start;  /* SS_SUBSPACE: 1 refines every solve from the first
                                   iteration (a restart from converging vectors); 0
                                   starts refining once the window is within 1e-6 or
                                   its residuals stop improving [0]                  */
    int32_t reserved;
    double refine_ratio;        /* FP32 solves refine until their residual is this
                                   fraction of the window's current residual (clamped
                                   to 1e-14 .. 1e-8) [1e-1]                          */
} ss_solve_opts;

/* ---- context ---------------------------------------------------------------------
 * ss_create: bind a context to CUDA device `device` and stream `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The stream is borrowed.
 * device = -1 makes a host-only context: ss_analyze, ss_symbolic_info_get,
 * ss_symbolic_perm and ss_symbolic_validate work without a GPU; every device call
 * returns SS_ERR_ARG.  Errors: SS_ERR_ARG (null ctx), SS_ERR_CUDA (bad device). */
ss_status ss_create(ss_ctx **ctx, int32_t device, void *cuda_stream);
ss_status ss_destroy(ss_ctx *ctx);
const char *ss_last_error(const ss_ctx *ctx);

/* How the level-scheduled triangular sweeps of every solve (ss_solve, the probes of
 * ss_slice_solve, the DOS Lanczos) are launched -- an implementation choice with no
 * paper counterpart.  SS_SOLVE_SWEEP_KERNEL (default): one cooperative launch per solve
 * that walks all levels with a bounded grid barrier between steps (a barrier that waits
 * about 1 s makes the solve return SS_ERR_TIMEOUT); SS_SOLVE_PER_STEP: one launch per
 * level and step.  Both compute the same sums; the atomics make the rounding order
 * differ.  ss_solve_noalloc always launches per step.  Errors: SS_ERR_ARG. */
enum { SS_SOLVE_SWEEP_KERNEL = 0, SS_SOLVE_PER_STEP = 1 };
ss_status ss_set_solve_mode(ss_ctx *ctx, int32_t mode);

/* FP32 sweep solves (implementation choice, no paper counterpart): a level whose fused
 * items -- (rows-below tiles + panels) x ceil(k / 32) -- number at most max_items runs them
 * with one grid barrier instead of two: every update item solves its panel's diagonal
 * block for its own 32 columns, and the last gather item of a panel runs its backward
 * diagonal step.  0 (default): never; -1: levels whose fused items fit in one pass of the
 * resident blocks.  Measured on GB300 (N = 16,384, k = 304): 6.5 ms per FP32 solve unfused,
 * 7.7 ms with -1 and 13.1 ms with every level fused -- the extra work of the fused items
 * costs more than the barriers they save, so the default leaves it off.
 * Errors: SS_ERR_ARG (max_items < -1). */
ss_status ss_set_sweep_fusion(ss_ctx *ctx, int32_t max_items);

/* Where the FP64 Schur-complement updates of ss_factor run (Alg. 2 step 2; an
 * implementation choice with no paper counterpart).  SS_SCHUR_TENSOR (default): a factor
 * step whose Schur update has at least min_flops algorithmic flops [2e7] runs on the FP16
 * tensor cores (tcgen05.mma, operands staged by bulk copies into shared memory, FP32
 * accumulators in tensor memory) with the operands cut into 7 exactly representable
 * 8-bit slices per row, so that the update is as accurate as an FP64 product (the
 * error-free splitting of Ozaki, Ogita, Oishi and Rump); smaller steps, and every FP32
 * factor, run on the CUDA cores.  SS_SCHUR_SIMT: every update on the CUDA cores.
 * Errors: SS_ERR_ARG. */
enum { SS_SCHUR_TENSOR = 0, SS_SCHUR_SIMT = 1 };
ss_status ss_set_schur_mode(ss_ctx *ctx, int32_t mode, double min_flops);

/* Where the probes' FP64 products run (the sparse products A X, B X and (A - sigma B) X of
 * Alg. 2 steps 3-5, and the Gram matrices and tall products of Cholesky-QR and
 * Rayleigh-Ritz, steps 4-5; an implementation choice with no paper counterpart).
 * SS_GEMM_TENSOR (default): products with at least 2,048 rows and small dimensions >= 48 run on the
 * FP16 tensor cores: every operand row (a row of A or B, a column of X) is split exactly
 * into 7 digit slices of 8 bits under one power-of-two scale, the 28 leading digit
 * products are summed exactly (FP32 accumulators in tensor memory, read out as integers
 * every 128 terms of the reduction) and the sum rounded once to FP64; the error is a few
 * units of 2^-53 of K max|a_row| max|b_row| (K the reduction length).  A factor keeps the
 * slices of its A and B (7 x 16 KB per 128-row tile and 64-column piece holding entries)
 * from its first product until ss_factor_destroy; where they do not fit the factor falls
 * back to the CUDA cores.  SS_GEMM_SIMT: CUDA-core FP64.  Errors: SS_ERR_ARG. */
enum { SS_GEMM_TENSOR = 0, SS_GEMM_SIMT = 1 };
ss_status ss_set_gemm_mode(ss_ctx *ctx, int32_t mode);

/* The probes' two dense FP64 products, on the stream of ctx and in the mode that
 * ss_set_gemm_mode chose (Alg. 2 steps 4-5: the Gram matrices of Cholesky-QR and
 * Rayleigh-Ritz, and the tall products that apply R^-T and the Ritz rotations).
 * Device pointers, row-major.
 *   ss_dense_gram:  G (k1 x k2, contiguous) = X^T Y, X n x k1 with row stride ldx >= k1,
 *                   Y n x k2 with row stride ldy >= k2.
 *   ss_dense_gemm:  Y (n x k2, row stride ldy >= k2) = beta Y + alpha X Q, X n x k1 (row
 *                   stride ldx >= k1), Q k1 x k2 contiguous, or with transq = 1, Y = beta
 *                   Y + alpha X Q^T with Q k2 x k1 contiguous.  beta = 0 does not read Y.
 * n >= 0, k1, k2 >= 1.  Returns after the launches are queued (the tensor-core path also
 * synchronises the stream to read its status word).  Errors: SS_ERR_ARG, SS_ERR_CUDA,
 * SS_ERR_OOM (scratch of the tensor-core path), SS_ERR_TIMEOUT (a bounded wait of the
 * tensor-core kernel ran out; the context stays usable). */
ss_status ss_dense_gram(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int32_t k1, const double *Y,
                        int64_t ldy, int32_t k2, double *G);
ss_status ss_dense_gemm(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int32_t k1, const double *Q,
                        int32_t k2, int32_t transq, double alpha, double beta, double *Y, int64_t ldy);

/* Replay of captured factorisations (batching of Alg. 2 step 2; no paper counterpart).
 * on = 1: ss_factor records the launches of one wave of shifts of an analysis -- every
 * level's memsets, assembly, extend-add, panel, Schur and store kernels -- into a CUDA
 * graph the first time it meets that (number of shifts, precision, Schur settings), keeps
 * the graph and its scratch with the analysis (freed by ss_symbolic_destroy), and on later
 * calls only uploads the table of per-shift pointers and shifts and launches the graph.
 * Waves whose scratch exceeds 8 GB, and factorisations timed per launch (ss_profile), run
 * launch by launch.  The first call for a wave shape must not itself be inside a stream
 * capture.  on = 0 (default): launch by launch.  Errors: SS_ERR_ARG. */
ss_status ss_set_factor_graph(ss_ctx *ctx, int32_t on);

/* Self-test of the tensor-core path (no paper counterpart): one 128 x 64 x 64 FP16 MMA tile
 * with seeded integer operands in [-128, 128], staged and read back exactly as the Schur
 * update does; *max_abs_err (HOST) is the largest deviation from the exact product (0 when
 * the operand layout and descriptors are right).  Errors: SS_ERR_ARG, SS_ERR_CUDA,
 * SS_ERR_TIMEOUT (a bounded wait ran out; the context stays usable). */
ss_status ss_selftest_tc(ss_ctx *ctx, uint64_t seed, double *max_abs_err);

/* Self-test of the bounded grid barrier used by the cooperative kernels (no paper
 * counterpart): one block per SM waits at a barrier that expects extra_arrivals (0 or 1)
 * more blocks than are launched, polling at most `limit` times (1 .. 1e8; a poll takes
 * about 64-100 ns).  extra_arrivals = 0 returns SS_OK; 1 makes every wait run out and
 * returns SS_ERR_TIMEOUT with the context still usable.  Errors: SS_ERR_ARG, SS_ERR_CUDA,
 * SS_ERR_TIMEOUT. */
ss_status ss_selftest_barrier(ss_ctx *ctx, int32_t extra_arrivals, int64_t limit);

/* ---- ss_analyze (Section 2.1: the sparse LDL^T of A - sigma B is the major cost;
 * Section 5: the paper's solver orders with nested dissection) --------------------
 * Host CSR pattern in, symbolic analysis out: nested-dissection ordering, supernodes
 * (the dissection blocks), the assembly tree and its level schedule, front index
 * maps, panel solve schedule and flop counts.  Done once per pattern and reused for
 * every shift and every pencil on that pattern.  rowptr[n+1] (int64) and colind[nnz]
 * (int32) are HOST arrays; they are copied.
 * Errors: SS_ERR_ARG (n <= 0, unsorted / out-of-range / asymmetric pattern),
 * SS_ERR_OOM. */
ss_status ss_analyze(ss_ctx *ctx, int64_t n, const int64_t *rowptr, const int32_t *colind,
                     const ss_options *opt, ss_symbolic **out);
ss_status ss_symbolic_info_get(const ss_symbolic *sym, ss_symbolic_info *info);
/* Fill-reducing permutation, host int32[n]: perm[new] = old. */
ss_status ss_symbolic_perm(const ss_symbolic *sym, int32_t *perm);
ss_status ss_symbolic_destroy(ss_symbolic *sym);
/* Consistency check of a symbolic analysis (no paper counterpart; a diagnostic): every
 * index the device kernels derive from it -- arena offsets, assembly destinations,
 * extend-add maps, panel / step / solve-level descriptors and scratch extents -- is
 * checked against the buffer it addresses, the ordering is checked to be a permutation
 * and every stored entry to lie inside its supernode's front.  Host only.
 * Errors: SS_ERR_INTERNAL with the first violation in ss_last_error. */
ss_status ss_symbolic_validate(const ss_symbolic *sym);

/* ---- ss_factor (Alg. 2 step 2: (L, D) <- LDL^T of A - sigma B) ------------------
 * Numeric supernodal multifrontal LDL^T of A - sigma_j B for each of the n_shift
 * shifts sigma[] (HOST array), one factor per shift, all sharing `sym`.  a_vals /
 * b_vals are DEVICE float64[nnz] aligned with the analysed pattern; they must stay
 * alive and unchanged while the factor is used (solves read them for residuals).
 * Pivoting is Bunch-Kaufman (1x1 / 2x2) restricted to each panel's diagonal block,
 * computed in FP64.  precision = SS_FP64 keeps fronts in FP64; SS_MIXED keeps fronts
 * and Schur updates in FP32 with FP64 diagonal blocks, and solves with FP64 iterative
 * refinement.  SS_MIXED checks every shift's FP32 factor: one FP32 solve of a fixed
 * probe vector must reduce the residual to rho <= 1e-2 of the right-hand side, else that
 * shift is refactored in FP64.  The FP64 factor of such a shift is then rounded once to
 * FP32; if one FP32 solve from the rounded copy contracts by rho <= 0.25, the shift's
 * solves run in FP32 inside FP64 refinement, else in FP64 (ss_factor_quality reports
 * which).  precision = SS_MIXED_TC factors every shift with FP64 fronts (the Schur updates
 * on the tensor cores, see ss_set_schur_mode) and rounds the factor once to FP32; where one
 * FP32 solve from that copy contracts by rho <= 0.25 the shift's solves run in FP32 inside
 * FP64 refinement, else in FP64 (no FP32 factorisation is attempted).
 * precision | SS_INERTIA_ONLY factors in FP64 and keeps no L (inertia,
 * ss_factor_stats only; solves on such a factor return SS_ERR_ARG): the counts at many
 * shifts at a fraction of the memory.
 * Memory: each shift keeps its L storage (info.l_storage_entries); while it is factored
 * it also holds a level workspace and a contribution-block pool (workspace_entries +
 * cb_pool_entries), so shifts are factored in waves of as many as the free device memory
 * holds.
 * Errors: SS_ERR_ARG, SS_ERR_OOM, SS_ERR_CUDA, SS_ERR_SINGULAR (a pivot fell below
 * 64 u ||A - sigma B||_1 for some shift; the factor is still returned and
 * ss_inertia reports which shift). */
ss_status ss_factor(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                    const double *sigma, int32_t n_shift, int32_t precision,
                    ss_numeric **out);
ss_status ss_factor_destroy(ss_numeric *f);

/* Autotuner of the Schur-update path per factor step (no paper counterpart): factors
 * A - sigma B (DEVICE a_vals, b_vals; inertia only, FP64) once with every eligible step's
 * Schur update on the tensor cores and once with every step on the CUDA cores, times each
 * step's update with CUDA events, and records for every step the faster path in the
 * analysis; later ss_factor calls on it follow these choices in place of the min_flops
 * rule of ss_set_schur_mode (while the Schur mode is SS_SCHUR_TENSOR).  The steps are the
 * analysis's front-size buckets, so the choice holds for every shift and every pencil on
 * the pattern.  *n_tc_steps (HOST, may be NULL): steps that chose the tensor cores.
 * Errors: SS_ERR_ARG, SS_ERR_OOM, SS_ERR_CUDA, SS_ERR_TIMEOUT. */
ss_status ss_autotune_schur(ss_symbolic *sym, const double *a_vals, const double *b_vals, double sigma,
                            int32_t *n_tc_steps);

/* ---- ss_factor_segments (Alg. 2 step 2 for many pencils; Section 2.2) -------------
 * Batched factorisation of many independent pencils of uneven size in the same launches:
 * the caller stacks the pencils into one block-diagonal pattern (each pencil's rows and
 * columns contiguous or not; no stored entry may couple rows of two pencils) and analyses
 * it once; ss_analyze's dissection keeps every pencil in its own subtrees, so each level
 * of the factorisation is one launch over the fronts of all pencils.  Shift j of the call
 * factors A_p - sigma[j * n_seg + p] B_p for every pencil p at once (HOST sigma, n_shift x
 * n_seg row-major; HOST row_segment, N entries, the pencil in [0, n_seg) of each
 * original row; DEVICE a_vals, b_vals as for ss_factor).  The factor is FP64 and
 * inertia-only (no L kept: solves return SS_ERR_ARG); ss_inertia gives the counts of the
 * whole stack, ss_inertia_segments those of each pencil.  It is what the validation of
 * every pencil's windows needs (exact counts at the window bounds, Section 2.2).
 * Errors: SS_ERR_ARG (bad pencil index, an entry coupling two pencils, non-finite shift),
 * SS_ERR_OOM, SS_ERR_CUDA, SS_ERR_SINGULAR (a pivot of some pencil fell below
 * 64 u (||A||_1 + max_p |sigma_jp| ||B||_1); the factor is still returned and
 * ss_inertia_segments reports which pencils). */
ss_status ss_factor_segments(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                             const int32_t *row_segment, int32_t n_seg, const double *sigma,
                             int32_t n_shift, ss_numeric **out);

/* Inertia of A_p - sigma_jp B_p for every pencil p of an ss_factor_segments factor: the
 * 1x1 and 2x2 pivots of D classified as by ss_inertia and counted per pencil.  HOST int64
 * outputs of n_seg entries each; n_tiny (may be NULL): pivots of the pencil below the
 * singularity threshold.  Errors: SS_ERR_ARG (also for a factor made by ss_factor),
 * SS_ERR_OOM, SS_ERR_CUDA. */
ss_status ss_inertia_segments(const ss_numeric *f, int32_t shift_idx, int64_t *n_neg, int64_t *n_zero,
                              int64_t *n_pos, int64_t *n_tiny);

/* ---- ss_inertia (Section 2.2: Sylvester's law of inertia) ------------------------
 * Inertia of A - sigma_j B from the block-diagonal D: n_neg = #negative 1x1 pivots
 * + one per 2x2 block with det < 0 (+ two per 2x2 block with det > 0 and negative
 * trace).  n_neg equals the number of eigenvalues of (A, B) below sigma_j.  Host
 * int64 outputs.  *tiny_pivot (may be NULL) is set to 1 if any pivot of this shift
 * fell below the singularity threshold.  Errors: SS_ERR_ARG. */
ss_status ss_inertia(const ss_numeric *f, int32_t shift_idx, int64_t *n_neg, int64_t *n_zero,
                     int64_t *n_pos, int32_t *tiny_pivot);

/* Precision shift j was finally factored and solved in: SS_MIXED (FP32 factor),
 * SS_FP64 (FP64 factor and solves) or SS_FP64_SOLVE32 (FP64 factor, FP32 solves from its
 * rounded copy), and the measured contraction factor rho of one FP32 solve (of the FP32
 * factor, or of the rounded copy when one is kept; 0 for precision = SS_FP64).
 * Host outputs, each may be NULL.  Errors: SS_ERR_ARG. */
ss_status ss_factor_quality(const ss_numeric *f, int32_t shift_idx, int32_t *precision_used,
                            double *rho);

/* Numerical diagnostics of shift j's factor (no paper counterpart): the smallest pivot
 * magnitude relative to ||A||_1 + |sigma| ||B||_1 (for a 2x2 block, its smaller
 * eigenvalue magnitude), the largest |L| entry (element growth), and the number of 2x2
 * pivot blocks.  Host outputs, each may be NULL.  Errors: SS_ERR_ARG. */
ss_status ss_factor_stats(const ss_numeric *f, int32_t shift_idx, double *min_pivot_ratio,
                          double *max_abs_l, int64_t *n_2x2);

/* ---- ss_solve (Alg. 2 step 3 without B: X = (A - sigma_j B)^-1 R) ------------------
 * R and X are DEVICE float64 N x k row-major (may alias).  `refine` FP64 iterative
 * refinement corrections are applied (X += M^-1 (R - (A - sigma_j B) X)); for a shift
 * solved in FP32 at least as many as its contraction factor needs to reach 1e-13 (at
 * most 8).  The residual uses the values of A - sigma_j B, formed on the shift's first
 * refined solve and kept with the factor (nnz doubles per shift).
 * Errors: SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_OOM, SS_ERR_TIMEOUT (sweep kernel barrier). */
ss_status ss_solve(ss_numeric *f, int32_t shift_idx, const double *R, int32_t k, double *X,
                   int32_t refine);

/* ---- ss_solve_noalloc (no paper counterpart) ---------------------------------------
 * The FP64 solve of ss_solve (refine = 0) for callers that cannot allocate device
 * memory -- code running under another framework's fixed memory budget or where the
 * allocator must not be called -- so this entry point allocates nothing, not even
 * temporarily.  Its working space is a file-scope device array of 4,194,304 doubles
 * (32 MiB, held by every GPU that loads the library until exit): the permuted N x k
 * right-hand sides followed by (widest solve level) x 64 x k doubles of gather buffer.
 * The caller passes R and X (DEVICE float64 N x k row-major, may alias) as for
 * ss_solve.  The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  The address is kept
 * for the life of the process: a cudaDeviceReset (which destroys the array with the
 * device's context) leaves it stale, so do not call this entry point on a device after
 * resetting it.  Every call shares
 * the array and it keeps the last call's contents (the call clears the parts it needs
 * cleared), so calls that overlap on the GPU -- on two streams, or two contexts of the
 * same device -- race: serialise them.
 * Errors: SS_ERR_ARG (bad argument; the shift was factored in FP32 -- use ss_solve; or
 * N k + 64 k (widest solve level) beyond 4,194,304, with the numbers in
 * ss_last_error), SS_ERR_CUDA. */
ss_status ss_solve_noalloc(ss_numeric *f, int32_t shift_idx, const double *R, int32_t k, double *X);

/* ---- ss_slice_solve (Alg. 2: shift-invert subspace iteration with Cholesky-QR in
 * the B inner product, Rayleigh-Ritz, residual norms; Section 2.1; or the shift-invert
 * block Lanczos the paper names as its alternative, Section 1) ----------------------
 * Builds the spectral probe of shift sigma_j.  V0 is the DEVICE N x k start block
 * (seeded N(0,1) or a previous probe's X; required; k <= min(N, 4096)).  Solves of a
 * shift solved in FP32 are refined once the window is near convergence, until their
 * residual is 1e-1 of the window's current residual (1e-13 .. 1e-8).  SS_SUBSPACE iterates on k
 * vectors and returns k Ritz pairs.  SS_BLOCK_LANCZOS builds max_iter blocks of width k
 * (O = (A - sigma B)^-1 B, full B-re-orthogonalisation), does one Rayleigh-Ritz on the
 * whole basis and returns the k_out Ritz pairs nearest sigma.
 * A Ritz pair is converged when its normalised residual
 * ||A x - theta B x||_2 / (||A||_1 ||x||_2) <= opts->tol.  Iterates until at least
 * opts->n_expect Ritz values in (lo, hi] are converged (n_expect > 0, e.g. an exact
 * count from inertia), or every Ritz value in (lo, hi] is (n_expect = 0), or max_iter.
 * Unconverged Ritz values inside the window can be spurious mixtures of eigenvectors
 * at equal distance on both sides of sigma; validation (Section 2.2) discards them.
 * Outputs (k_out entries; k_out = k for SS_SUBSPACE): lambda (HOST float64: the Rayleigh
 * quotients x^T A x / x^T B x of the returned vectors, summed and divided in double-double,
 * in the ascending order of the Ritz values), X (DEVICE N x k_out, B-orthonormal Ritz
 * vectors in the same order),
 * resid (HOST float64), n_found (HOST: #converged Ritz values in (lo, hi]), stats
 * (HOST, may be NULL).
 * Errors: SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_OOM, SS_ERR_NOCONV (outputs still valid). */
ss_status ss_slice_solve(ss_numeric *f, int32_t shift_idx, double lo, double hi,
                         const ss_solve_opts *opts, const double *V0, int32_t k,
                         double *lambda, double *X, double *resid, int32_t *n_found,
                         ss_probe_stats *stats);

/* ---- ss_dos_estimate (Section 3.1, Eqs. 4-5: Lanczos DOS of G^-1 A G^-T) --------
 * Factors B = G G^T (the LDL^T at sigma = 0 of the pencil (B, 0), G = P L D^1/2), then
 * runs `steps` Lanczos steps on G^-1 A G^-T with full re-orthogonalisation for each of
 * the n_vec DEVICE start vectors y0 in start (N x n_vec row-major, seeded N(0,1)).  It
 * is computed as B-orthonormal Lanczos on B^-1 A from x0 = G^-T y0; because the start
 * vectors are i.i.d. N(0,1) the estimate's distribution does not depend on which
 * square root G of B is used.
 * Outputs (HOST): theta[n_vec*steps], zeta2[n_vec*steps] (squared first components
 * of the tridiagonal's eigenvectors, per run, ascending theta), m_run[n_vec] (steps
 * actually taken per run; entries past m_run are 0).
 * Errors: SS_ERR_ARG, SS_ERR_NOT_SPD, SS_ERR_CUDA, SS_ERR_OOM. */
ss_status ss_dos_estimate(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                          int32_t steps, int32_t n_vec, const double *start,
                          double *theta, double *zeta2, int32_t *m_run);
/* ss_dos_lanczos: the same Lanczos run from explicit start vectors x0 of the
 * B-orthonormal form (Section 3.1's second form): x_1 = x0 / ||x0||_B, operator B^-1 A.
 * Same outputs and errors as ss_dos_estimate. */
ss_status ss_dos_lanczos(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                         int32_t steps, int32_t n_vec, const double *x0,
                         double *theta, double *zeta2, int32_t *m_run);

/* ---- ss_band_energy_grad (Hellmann-Feynman; not in the paper) ----------------------
 * For E = sum_{i < n_e} lambda_i with B-orthonormal eigenvectors X (DEVICE N x n_e
 * row-major) and lambda (DEVICE float64[n_e]):
 *   grad_a[e] = sum_i X[r,i] X[c,i],  grad_b[e] = -sum_i lambda_i X[r,i] X[c,i]
 * for every stored entry e = (r, c) of the pattern (DEVICE float64[nnz] each; either
 * may be NULL).  This is the per-stored-entry derivative; a symmetric parameter tying
 * (r, c) and (c, r) gets the sum of both entries.  Errors: SS_ERR_ARG, SS_ERR_CUDA. */
ss_status ss_band_energy_grad(ss_symbolic *sym, const double *X, const double *lambda,
                              int32_t n_e, double *grad_a, double *grad_b);

/* ---- SpMM helper (the CSR sweep of Section 3.1 and the residual of Alg. 2) -------
 * Y[i, j] = sum_e (alpha[j] a_vals[e] + beta[j] b_vals[e]) X[col(e), j] over row i,
 * X, Y DEVICE float64 N x k row-major; alpha, beta DEVICE float64[k] (NULL alpha = 1,
 * NULL beta = no B term).  With ss_set_gemm_mode(SS_GEMM_TENSOR), N >= 2,048 and k >= 48
 * the products run on the tensor cores (digit slices of the values made for this call:
 * 7 x 16 KB per 128-row tile and 64-column piece holding entries), A X and B X each
 * rounded once to FP64.  Errors: SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_OOM, SS_ERR_TIMEOUT. */
ss_status ss_spmm(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                  const double *alpha, const double *beta, const double *X, int32_t k,
                  double *Y);

/* Measured arithmetic peak of the context's GPU (no paper counterpart; the roofline
 * denominator of the CUDA-core kernels): one launch of kIlp = 8 independent fused
 * multiply-add chains per thread, 4 blocks of 256 threads per SM, its length grown until
 * the launch takes about `seconds` (0 < seconds <= 10).  *tflops (HOST) = 2 flops per FMA
 * over the launch's CUDA-event time.  kind: SS_PEAK_FP64_FMA or SS_PEAK_FP32_FMA.
 * Errors: SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_OOM. */
enum { SS_PEAK_FP64_FMA = 0, SS_PEAK_FP32_FMA = 1 };
ss_status ss_measure_peak(ss_ctx *ctx, int32_t kind, double seconds, double *tflops);

/* Device synchronisation of the context's stream (convenience for bindings). */
ss_status ss_sync(ss_ctx *ctx);

/* ---- measurement hooks (no paper counterpart) -------------------------------------
 * Kernel classes, for per-class timing (bit c of a mask = class c; at most 32).
 * ss_launch_count returns the number of
 * kernels this library has launched since it was loaded (all contexts).
 * ss_profile(ctx, mask) starts timing every launch of the classes whose bit is set
 * in mask (bit c = class c) with CUDA events recorded on the launching stream, and
 * clears the previous totals; mask = 0 stops.  ss_profile_query synchronises the
 * stream and returns the launch count and summed device time of class cls since the
 * last ss_profile call.  Errors: SS_ERR_ARG, SS_ERR_CUDA. */
enum {
    SS_K_ASSEMBLE = 0, SS_K_EXTEND_ADD, SS_K_DIAG_BK, SS_K_PANEL, SS_K_SCHUR, SS_K_FWD_DIAG,
    SS_K_FWD_UPDATE, SS_K_BWD_GATHER, SS_K_BWD_DIAG, SS_K_PERMUTE, SS_K_SPMM, SS_K_GRAM,
    SS_K_GEMM, SS_K_SMALL_DENSE, SS_K_JACOBI, SS_K_LANCZOS, SS_K_SDDMM, SS_K_MISC,
    SS_K_PANEL_F32, SS_K_SCHUR_F32, SS_K_FWD_UPDATE_F32, SS_K_BWD_GATHER_F32,
    SS_K_SOLVE, SS_K_SOLVE_F32,   /* whole-solve sweep kernel (SS_SOLVE_SWEEP_KERNEL) */
    SS_K_SCHUR_TC,                /* tensor-core Schur update (slicing + MMA tiles)    */
    SS_K_GEMM_TC,                 /* tensor-core Gram / tall products                  */
    SS_K_SPMM_TC,                 /* tensor-core sparse products A X, B X              */
    SS_K_COUNT
};
int64_t ss_launch_count(void);
ss_status ss_profile(ss_ctx *ctx, uint32_t mask);
/* *flops (may be NULL): algorithmic flops of the timed launches of the classes that
 * count them (panel, Schur (both paths), solve sweeps, SpMM, Gram, GEMM; 2 per multiply-add,
 * lower triangle only for the Schur update); 0 for the others.  Classes ending in _F32 are the
 * FP32 instantiations of the mixed-precision factor and solves. */
ss_status ss_profile_query(ss_ctx *ctx, int32_t cls, int64_t *launches, double *seconds, double *flops);
/* For the tensor-core classes (SS_K_SCHUR_TC, SS_K_GEMM_TC, SS_K_SPMM_TC): the FP16 MMA
 * work (2 M N K per MMA, zero padding of sparse tiles included) their launches issued since
 * the last ss_profile call; 0 for the other classes.  Call after ss_profile_query (which
 * synchronises).  Errors: SS_ERR_ARG. */
ss_status ss_profile_query_tensor(ss_ctx *ctx, int32_t cls, double *tensor_flops);

#ifdef __cplusplus
}
#endif
#endif /* SISLICE_H */
