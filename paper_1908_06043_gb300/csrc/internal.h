// Internal structures of the slice-solve library (host side).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sislice.h"

struct GridBar;   // grid_sync.cuh

struct ss_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;       // private stream that graph captures record on
    int sm_count = 0;
    std::string err;
    int solve_mode = SS_SOLVE_SWEEP_KERNEL;   // how the triangular sweeps are launched
    int schur_mode = SS_SCHUR_TENSOR;         // FP64 Schur update: tensor cores or CUDA cores
    int factor_graph = 0;                     // replay captured CUDA graphs of the factorisation
    int gemm_mode = SS_GEMM_TENSOR;           // probes' FP64 products: tensor cores or CUDA cores
    bool capturing = false;                   // a factorisation is being captured (launches not counted)
    std::vector<double> *step_times = nullptr;   // per factor step Schur time (autotuner), or null
    int64_t plan_gen = 0;                     // bumped when a setting baked into captured graphs changes
    double tc_min_flops = 2.0e7;              // a factor step's Schur flops below which it stays on CUDA cores
    GridBar *d_bar = nullptr;                 // grid barrier state of the sweep kernel
    int sweep_blocks_per_sm[2] = {0, 0};      // resident sweep-kernel blocks per SM (FP64, FP32)
    int sweep_fuse_max = 0;                   // FP32 sweep: fuse levels with at most this many items
                                              // (-1: the resident blocks; 0: never)
    // per-class launch timing (ss_profile): event pairs recorded around launches
    uint32_t prof_mask = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_used;     // (class, index of the start event)
    int64_t prof_launches[SS_K_COUNT] = {};
    double prof_seconds[SS_K_COUNT] = {};
    double prof_flops[SS_K_COUNT] = {};
    double prof_tensor_flops[SS_K_COUNT] = {};   // FP16 MMA work the tensor-core classes issued
    void add_tensor_flops(int cls, double f) {
        if (prof_mask & (1u << cls)) prof_tensor_flops[cls] += f;
    }
    void add_flops(int cls, double f) {
        if (prof_mask & (1u << cls)) prof_flops[cls] += f;
    }
    int set_error(int code, const std::string &msg) {
        err = msg;
        return code;
    }
    ~ss_ctx() {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (d_bar) cudaFree(d_bar);
    }
};

extern std::atomic<int64_t> g_ss_launches;
size_t ss_prof_begin(ss_ctx *ctx, int cls);
void ss_prof_end(ss_ctx *ctx, int cls, size_t slot);

#ifdef __CUDACC__
// Every kernel of the library is launched through here: it counts the launch and, when
// the class is being profiled, brackets it with events on the launching stream.
template <typename... KArgs, typename... Args>
inline void ss_launch(ss_ctx *ctx, int cls, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t st, Args &&...args) {
    if (!ctx->capturing) g_ss_launches.fetch_add(1, std::memory_order_relaxed);
    if (ctx->prof_mask & (1u << cls)) {
        size_t slot = ss_prof_begin(ctx, cls);
        kern<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
        ss_prof_end(ctx, cls, slot);
    } else {
        kern<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
    }
}
#endif

// Operand slices of the tensor-core Schur update (tc_kernels.cuh): kTcSlices FP16 blocks
// of 128 rows x 64 columns per 128-row tile of L21 and of W.
constexpr int kTcSlices = 7;
constexpr int64_t kTcSliceBytes = 128 * 64 * 2;

// One panel of the blocked front factorisation: columns [k0, k0+w) of front `sn`.
// The panel's L rows below its diagonal block are front rows [k0+w, m), whose global
// (permuted) indices are idx[idx_off + k0 + w ...].
struct PanelDesc {
    int64_t front_off;   // L storage offset (entries) of the supernode's m x ncol panel columns
                         // (column-major, leading dimension m)
    int64_t idx_off;     // offset of the front's global index list in idx
    int32_t m;           // front dimension
    int32_t k0;          // first front column of the panel
    int32_t w;           // panel width (<= nb)
    int32_t g0;          // global (permuted) index of the panel's first column
    int32_t sn;          // owning supernode
    int32_t pad;
};

// One front taking part in factor step (level, t): panel `panel` is eliminated and
// the trailing front [k0+w, m) x [k0+w, m) is updated.
struct StepTask {
    int64_t front_off;   // workspace offset of the m x m front (column-major)
    int64_t wbuf_off;    // offset of this task's W = L21 D block (r x w, col-major) in W scratch
    int32_t m, k0, w, r; // r = m - k0 - w
    int32_t panel;
    int32_t mt_slot;     // slot of the w x w transform in the Mt scratch
    int32_t tiles4_pre;  // exclusive prefix of panel-transform row tiles
    int32_t tiles3_pre;  // exclusive prefix of Schur-update tiles
    int32_t sl_pre;      // exclusive prefix of 128-row slice tiles (2 per 128 rows: L21, W)
    int32_t tc_pre;      // exclusive prefix of 128 x 64 tensor-core Schur tiles
    int64_t sl_off;      // byte offset of this task's operand slices in the slice scratch
    int64_t ex_off;      // offset of its row exponents (r for L21, then r for W)
};

struct StepDesc {
    int64_t task_off;    // into tasks
    int32_t count;       // fronts in this step
    int32_t tiles4, tiles3;
    int32_t level;
    double flops4, flops3;   // algorithmic flops of the panel transform / Schur update
    int32_t sl_tiles, tc_tiles;   // slice tiles and tensor-core Schur tiles of the step
    int64_t sl_bytes, ex_count;   // slice scratch bytes and row exponents of the step
};

// Child -> parent extend-add unit: the child's contribution block (pool, packed lower
// triangle of order child_m = its nr; child_ncol = 0) added into the parent front
// (workspace) through relmap.
struct ExtendTask {
    int64_t child_off, parent_off;
    int64_t rel_off;     // into relmap (length nr)
    int32_t child_m, child_ncol, parent_m, col_pre;  // col_pre: exclusive prefix of columns
};

// After a level is factored: copy front columns of one supernode out of the workspace.
// Column c < ncol goes to L storage (the whole column, m entries); column ncol + j (the
// contribution block) goes to the pool, rows j .. nr-1 (nr = m - ncol), packed lower
// triangle: column j starts at j (2 nr - j + 1) / 2.
struct StoreTask {
    int64_t ws_off, l_off, cb_off;   // cb_off < 0: no contribution block (a root)
    int32_t m, ncol, col_pre, pad;   // col_pre: exclusive prefix of columns in the level
};

struct ExtendPass {     // one non-conflicting pass (the q-th child of each parent)
    int64_t task_off;
    int32_t count, cols;
};

struct SolveLevel {      // panels whose forward step can run together
    int64_t panel_off;   // into solve_panels
    int32_t count;
    int32_t row_tiles;   // total row tiles (64 rows) of the panels' below-diagonal rows
    double offdiag;      // sum over its panels of (rows below the diagonal block) x w
};

// A captured factorisation of `ns` shifts (one wave) in one precision: persistent scratch
// and the instantiated CUDA graph of the whole level loop.  A replay only refreshes the
// device table of per-shift pointers and values (dp) the kernels read.
struct FactorPlan {
    int ns = 0;
    int fp32 = 0;          // fronts in FP32
    int tc = 0;            // tensor-core Schur steps enabled
    void *mt = nullptr, *wb = nullptr, *ws = nullptr, *cb = nullptr, *sl = nullptr, *ex = nullptr, *dp = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernel_nodes = 0;
    int64_t gen = 0;       // ss_ctx::plan_gen at capture
};

struct OzPlan;   // tensor-core products: (tile, piece) pairs of the pattern (oz.cu)
struct OzVals;   // tensor-core products: digit slices of one value array (oz.cu)

struct ss_symbolic {
    ss_ctx *ctx = nullptr;
    OzPlan *oz_plan = nullptr;
    std::vector<FactorPlan *> plans;         // captured factorisations (freed with the analysis)
    std::vector<int8_t> step_mode;           // per factor step: -1 rule of ss_set_schur_mode,
                                             // 0 CUDA cores, 1 tensor cores (autotuner)
    int64_t n = 0, nnz = 0;
    int nb = 64;
    std::vector<int32_t> perm, iperm;        // perm[new] = old, iperm[old] = new
    std::vector<int64_t> rowptr;             // host copy of the pattern
    std::vector<int32_t> colind;

    int32_t nsn = 0;
    std::vector<int32_t> sn_first;           // nsn + 1
    std::vector<int32_t> sn_parent, sn_nrow, sn_level;
    std::vector<int64_t> sn_idx_off;         // nsn + 1
    std::vector<int32_t> idx;                // per supernode: [its columns, its rows]
    // memory plan of the numeric factorisation (entries, per shift)
    std::vector<int64_t> front_off;          // front offset in its level's workspace
    std::vector<int64_t> l_off;              // L storage offset (m x ncol, leading dim m)
    std::vector<int64_t> cb_off;             // contribution-block pool offset (-1: none)
    std::vector<int64_t> lev_ws;             // workspace entries used by each level
    int64_t ws_total = 0, l_total = 0, cb_total = 0;
    std::vector<StoreTask> store_tasks;
    std::vector<int32_t> lev_store_off;      // nlev + 1, into store_tasks
    std::vector<int32_t> lev_store_cols;     // columns stored per level
    int32_t nlev = 0;

    // assembly of the original entries, grouped by level
    std::vector<int64_t> asm_lev_off;        // nlev + 1
    std::vector<int32_t> asm_e;              // CSR entry index
    std::vector<int64_t> asm_dest;           // workspace offset

    std::vector<int32_t> relmap;             // child rows -> parent front positions
    std::vector<ExtendTask> ext_tasks;
    std::vector<ExtendPass> ext_pass;
    std::vector<int32_t> lev_ext_pass_off;   // nlev + 1, into ext_pass

    std::vector<PanelDesc> panels;
    std::vector<StepTask> tasks;
    std::vector<StepDesc> steps;
    std::vector<int32_t> lev_step_off;       // nlev + 1, into steps
    int64_t wbuf_max = 0;                    // max W scratch entries over steps
    int64_t sl_max = 0, ex_max = 0;          // max slice bytes / row exponents over steps
    int32_t mt_max = 0;                      // max fronts in one step

    std::vector<int32_t> solve_panels;       // panel ids grouped by solve level
    std::vector<SolveLevel> solve_levels;
    std::vector<int32_t> solve_tile_pre;     // per solve_panels entry: exclusive row-tile prefix

    ss_symbolic_info info{};

    // device mirrors
    int64_t *d_rowptr = nullptr;
    int32_t *d_colind = nullptr;
    int32_t *d_iperm = nullptr;              // old -> new
    int32_t *d_perm = nullptr;               // new -> old
    int32_t *d_idx = nullptr;
    int32_t *d_asm_e = nullptr;
    int64_t *d_asm_dest = nullptr;
    int32_t *d_relmap = nullptr;
    ExtendTask *d_ext_tasks = nullptr;
    PanelDesc *d_panels = nullptr;
    StoreTask *d_store_tasks = nullptr;
    StepTask *d_tasks = nullptr;
    int32_t *d_solve_panels = nullptr;
    int32_t *d_solve_tile_pre = nullptr;
    int32_t *d_col_panel = nullptr;          // permuted column -> panel
    void *d_sweep_lev = nullptr;             // solve levels for the sweep kernel (SweepLevel)
};

struct ss_numeric {
    ss_symbolic *sym = nullptr;
    int precision = SS_FP64;              // requested precision
    int32_t n_shift = 0;
    std::vector<int> shift_prec;          // precision each shift was factored in
    std::vector<double> rho;              // mixed: contraction factor of one FP32 solve
    std::vector<double> sigma;
    const double *a_vals = nullptr, *b_vals = nullptr;   // caller-owned device arrays
    double norm_a1 = 0, norm_b1 = 0;
    bool inertia_only = false;            // no L storage kept: inertia counts only
    // per shift
    std::vector<void *> arena;            // L storage (double or float), l_total entries
    std::vector<float *> arena_lo;        // FP32 rounding of an FP64 L storage that solves read, or null
    std::vector<double *> linv;           // npanels * nb * nb, L11^-1 of each panel
    std::vector<double *> dblk;           // npanels * nb * 2: D diagonal, D sub-diagonal
    std::vector<int32_t *> piv;           // npanels * nb: local pivot order
    std::vector<double *> mvals;          // values of A - sigma_j B on the pattern (made by the
                                          // first refined solve of shift j), or null
    unsigned long long *d_counts = nullptr;   // per shift: neg, zero, pos, tiny
    std::vector<unsigned long long> h_counts;
    bool counts_valid = false;
    OzVals *oz[2] = {nullptr, nullptr};  // digit slices of A and B for tensor-core products, or null
    bool oz_failed = false;               // those slices did not fit: products on the CUDA cores
    // several pencils in one block-diagonal pattern (ss_factor_segments): a shift per pencil
    int32_t n_seg = 0;
    int32_t *d_eseg = nullptr;            // pencil of each stored entry (nnz)
    int32_t *d_rowseg = nullptr;          // pencil of each original row (n)
    double *d_seg_sigma = nullptr;        // n_shift x n_seg shifts
};

// solves of shift j run in FP32 (an FP32 factor, or an FP64 factor with a rounded copy)
inline bool ss_solves_f32(const ss_numeric *f, int j) {
    return f->shift_prec[j] == SS_MIXED || f->arena_lo[j] != nullptr;
}

// helpers implemented in the .cu files
int ss_symbolic_upload(ss_symbolic *s);
void ss_symbolic_free_device(ss_symbolic *s);
void ss_free_plans(ss_symbolic *s);
int ss_factor_fetch_counts(ss_numeric *f);
// seg (optional): several pencils of one block-diagonal pattern, each with its own shifts
struct SegShifts {
    int32_t n_seg;
    const int32_t *row_seg;   // host, n: pencil of each row
    const double *sigma;      // host, n_shift x n_seg
};
int ss_factor_create(ss_symbolic *sym, const double *a_vals, const double *b_vals, const double *sigma,
                     int32_t n_shift, int32_t precision, ss_numeric **out, const SegShifts *seg = nullptr);
constexpr int SS_NCOUNT = 8;   // per-shift device counters: neg, zero, pos, tiny, min pivot, 2x2, max |L|,
                               // device waits that ran out
int ss_norm1(ss_symbolic *s, const double *vals, double *out);
int solve_contraction(ss_numeric *f, int j, double *rho);
// in-place solve (A - sigma_j B) x = b of a permuted-order N x k block
template <typename T> int solve_permuted(ss_numeric *f, int j, T *b, int k);
// X = (A - sigma_j B)^-1 R in the original order (FP64 in/out, refinement for mixed)
// target > 0 (FP32 solves only): refine until max|R - M X| <= target max|R|, at most
// max(refine, 12) steps
int solve_apply(ss_numeric *f, int j, const double *R, int k, double *X, int refine, int *steps_done,
                double target = 0.0);
int spmm_launch(ss_symbolic *s, const double *a, const double *b, const double *alpha, const double *beta,
                const double *X, int k, double *Y);
int spmm_launch_ld(ss_symbolic *s, const double *a, const double *b, const double *alpha, const double *beta,
                   const double *X, int64_t ldx, int k, double *Y, int64_t ldy);
// FP64-accurate products on the tensor cores (oz.cu; ss_set_gemm_mode)
bool oz_dense_ok(const ss_ctx *ctx, int64_t n, int k1, int k2);
bool oz_spmm_ok(const ss_numeric *f, int k);
int oz_gram(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int k1, const double *Y, int64_t ldy, int k2,
            double *G);
int oz_gemm(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int k1, const double *Q, int k2, int transq,
            double alpha, double beta, double *Y, int64_t ldy);
// npass passes over X: pass p adds alpha[p] diag(colscale[p]) M_p X with M_p = A (which 0)
// or B (which 1) of f; the first pass overwrites Y
int oz_spmm(ss_numeric *f, int npass, const int *which, const double *const *colscale, const double *alpha,
            const double *X, int64_t ldx, int k, double *Y, int64_t ldy);
// the same for any value arrays, sliced for this call only
int oz_spmm_vals(ss_symbolic *s, const double *a, const double *b, const double *alpha, const double *beta,
                 const double *X, int64_t ldx, int k, double *Y, int64_t ldy);
// Y = diag(alpha) A X + diag(beta) B X for value arrays a, b (tensor cores where possible)
int spmm_f(ss_numeric *f, const double *a, const double *b, const double *alpha, const double *beta, const double *X,
           int64_t ldx, int k, double *Y, int64_t ldy);
void oz_free_numeric(ss_numeric *f);
void oz_free_symbolic(ss_symbolic *s);
// x = P L^-T D^-1/2 y (y permuted order, x original order), SPD factors only
int solve_half_backward(ss_numeric *f, int j, const double *y, int k, double *x);

#define SS_CUDA_TRY(ctx, call)                                                           \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError(); /* clear a non-sticky error so later calls start clean */ \
            return (ctx)->set_error(e_ == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA, \
                                    std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                \
    } while (0)
