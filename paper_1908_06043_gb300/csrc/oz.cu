// Host side of the FP64-accurate tensor-core products (tc_gemm.cuh): operand slicing, the
// (tile, piece) plan of the sparse pattern, the digit slices of a factor's A and B kept for
// the factor's lifetime, and the launches.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"
#include "tc_gemm.cuh"

struct OzPlan {
    int32_t nrt = 0;
    int64_t npairs = 0;
    int32_t *d_tile_ptr = nullptr, *d_pair_tile = nullptr, *d_pair_piece = nullptr;
    int64_t *d_seg = nullptr;
};

struct OzVals {
    const double *vals = nullptr;
    unsigned char *sl = nullptr;   // npairs x 7 slice blocks
    int *em = nullptr;             // per row: largest biased exponent
};

namespace {

using sstc::OzOperand;

inline unsigned cdivu(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// FP16 MMA work of one (output tile, piece): 36 digit products x 2 K steps of 128 x 64 x 16
constexpr double kPieceTensorFlops = 36.0 * 2.0 * 2.0 * 128 * 64 * 16;

// per-call device scratch from the stream-ordered pool
struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        cudaError_t e = cudaMallocAsync((void **)p, sizeof(T) * std::max<size_t>(count, 1), st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

#define OZ_ALLOC(ctx, expr)                                                                               \
    do {                                                                                                  \
        cudaError_t e_ = (expr);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            cudaGetLastError();                                                                           \
            return (ctx)->set_error(SS_ERR_OOM, std::string("device allocation failed: ") +             \
                                                    cudaGetErrorString(e_));                              \
        }                                                                                                 \
    } while (0)

void oz_attrs(int device) {
    static std::mutex mu;
    static std::vector<char> seen;
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0) return;
    if ((size_t)device >= seen.size()) seen.resize(device + 1, 0);
    if (seen[device]) return;
    seen[device] = 1;
    cudaFuncSetAttribute(sstc::k_oz_mm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sstc::kOzGemmSmem);
    cudaFuncSetAttribute(sstc::k_oz_slice_csr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sstc::kOzCsrSmem);
}

// exponents and digit slices of a dense operand (blocks kc * nrt + rt)
int slice_dense(ss_ctx *ctx, const OzOperand &op, Scratch &buf, unsigned char **sl, int **em) {
    const unsigned nrt = cdivu(op.rows, 128), nkc = cdivu(op.kdim, sstc::kOzK);
    OZ_ALLOC(ctx, buf.get(sl, (size_t)nrt * nkc * sstc::kOzStageA));
    OZ_ALLOC(ctx, buf.get(em, (size_t)op.rows));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(*em, 0, sizeof(int) * op.rows, ctx->stream));
    const int64_t per_k = std::max<int64_t>(64, (int64_t)cdivu(op.kdim, std::max<unsigned>(1, 4 * ctx->sm_count / nrt)));
    ss_launch(ctx, SS_K_GEMM_TC, sstc::k_oz_expmax, dim3(nrt, cdivu(op.kdim, per_k)), 128, 0, ctx->stream, op, per_k,
              *em);
    ss_launch(ctx, SS_K_GEMM_TC, sstc::k_oz_slice, dim3(nrt, nkc), 128, 0, ctx->stream, op, (const int *)*em, *sl);
    return SS_OK;
}

int run_mm(ss_ctx *ctx, sstc::OzMM g, dim3 grid, int cls) {
    Scratch buf(ctx->stream);
    OZ_ALLOC(ctx, buf.get(&g.status, 1));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(g.status, 0, sizeof(int), ctx->stream));
    ss_launch(ctx, cls, sstc::k_oz_mm, grid, sstc::kOzThreads, sstc::kOzGemmSmem, ctx->stream, g);
    int h = 0;
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(&h, g.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return ctx->set_error(SS_ERR_TIMEOUT, "tensor-core product: a bounded wait ran out");
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// dense product: mode 0 (G += alpha A B^T, split over the reduction) or mode 1
int dense_mm(ss_ctx *ctx, const OzOperand &A, const OzOperand &B, int mode, double alpha, double beta, double *out,
             int64_t ldo, double flops) {
    oz_attrs(ctx->device);
    Scratch buf(ctx->stream);
    unsigned char *sa, *sb;
    int *ea, *eb;
    int rc;
    if ((rc = slice_dense(ctx, A, buf, &sa, &ea)) != SS_OK) return rc;
    if ((rc = slice_dense(ctx, B, buf, &sb, &eb)) != SS_OK) return rc;
    const int nrtA = (int)cdivu(A.rows, 128), nrtB = (int)cdivu(B.rows, 128), nkc = (int)cdivu(A.kdim, sstc::kOzK);
    const int nct = (int)cdivu(B.rows, 64);
    const int64_t tiles = (int64_t)nrtA * nct;
    int per = nkc;
    if (mode == 0) {
        // split the reduction until about two CTAs per SM
        const int64_t want = std::max<int64_t>(1, std::min<int64_t>(nkc, cdivu(2ll * ctx->sm_count, tiles)));
        per = (int)cdivu(nkc, want);
    }
    const int nsplit = (int)cdivu(nkc, per);
    sstc::OzMM g{};
    g.slA = sa; g.emA = ea; g.nrtA = nrtA; g.rowsA = A.rows;
    g.slB = sb; g.emB = eb; g.nrtB = nrtB; g.rowsB = B.rows;
    g.nkc = nkc; g.per = per; g.mode = mode; g.alpha = alpha; g.beta = beta;
    g.out = out; g.ldo = ldo;
    ctx->add_flops(SS_K_GEMM_TC, flops);
    ctx->add_tensor_flops(SS_K_GEMM_TC, kPieceTensorFlops * nrtA * nct * nkc);
    return run_mm(ctx, g, dim3(nct, nrtA, nsplit), SS_K_GEMM_TC);
}

// (tile, piece) pairs of the pattern: for each 128-row tile the 32-column pieces that hold
// entries, and per pair and row the CSR position of the row's first entry in the piece
int plan_build(ss_symbolic *s) {
    ss_ctx *ctx = s->ctx;
    const int64_t n = s->n;
    const int32_t nrt = (int32_t)cdivu(n, 128);
    const int64_t npieces = (n + sstc::kOzK - 1) / sstc::kOzK;
    std::vector<int32_t> tile_ptr(nrt + 1, 0), pair_tile, pair_piece, mark(npieces, -1), list;
    std::vector<int64_t> seg;
    for (int32_t rt = 0; rt < nrt; ++rt) {
        list.clear();
        const int64_t r0 = (int64_t)rt * 128, r1 = std::min<int64_t>(n, r0 + 128);
        for (int64_t p = s->rowptr[r0]; p < s->rowptr[r1]; ++p) {
            const int32_t pc = s->colind[p] / sstc::kOzK;
            if (mark[pc] != rt) {
                mark[pc] = rt;
                list.push_back(pc);
            }
        }
        std::sort(list.begin(), list.end());
        const size_t base = pair_tile.size();
        for (int32_t pc : list) {
            pair_tile.push_back(rt);
            pair_piece.push_back(pc);
        }
        seg.resize(pair_tile.size() * 128, 0);
        for (int r = 0; r < 128; ++r) {
            const int64_t row = r0 + r;
            int64_t ptr = row < n ? s->rowptr[row] : 0;
            const int64_t end = row < n ? s->rowptr[row + 1] : 0;
            for (size_t u = 0; u < list.size(); ++u) {
                while (ptr < end && s->colind[ptr] < (int64_t)list[u] * sstc::kOzK) ++ptr;
                seg[(base + u) * 128 + r] = ptr;
            }
        }
        tile_ptr[rt + 1] = (int32_t)pair_tile.size();
    }
    OzPlan *pl = new OzPlan();
    pl->nrt = nrt;
    pl->npairs = (int64_t)pair_tile.size();
    cudaError_t e = cudaMalloc(&pl->d_tile_ptr, sizeof(int32_t) * tile_ptr.size());
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_pair_tile, sizeof(int32_t) * std::max<size_t>(1, pair_tile.size()));
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_pair_piece, sizeof(int32_t) * std::max<size_t>(1, pair_piece.size()));
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_seg, sizeof(int64_t) * std::max<size_t>(1, seg.size()));
    s->oz_plan = pl;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx->set_error(SS_ERR_OOM, "tensor-core product plan: device allocation failed");
    }
    SS_CUDA_TRY(ctx, cudaMemcpy(pl->d_tile_ptr, tile_ptr.data(), sizeof(int32_t) * tile_ptr.size(),
                                cudaMemcpyHostToDevice));
    if (!pair_tile.empty()) {
        SS_CUDA_TRY(ctx, cudaMemcpy(pl->d_pair_tile, pair_tile.data(), sizeof(int32_t) * pair_tile.size(),
                                    cudaMemcpyHostToDevice));
        SS_CUDA_TRY(ctx, cudaMemcpy(pl->d_pair_piece, pair_piece.data(), sizeof(int32_t) * pair_piece.size(),
                                    cudaMemcpyHostToDevice));
        SS_CUDA_TRY(ctx, cudaMemcpy(pl->d_seg, seg.data(), sizeof(int64_t) * seg.size(), cudaMemcpyHostToDevice));
    }
    return SS_OK;
}

// exponents and digit slices of one value array on the pattern, into v (device memory from
// buf, or owned by v when buf is null)
int vals_make(ss_symbolic *s, const double *vals, OzVals *v, Scratch *buf) {
    ss_ctx *ctx = s->ctx;
    int rc;
    if (!s->oz_plan && (rc = plan_build(s)) != SS_OK) return rc;
    const OzPlan *pl = s->oz_plan;
    const size_t bytes = (size_t)std::max<int64_t>(1, pl->npairs) * sstc::kOzStageA;
    v->vals = vals;
    if (buf) {
        OZ_ALLOC(ctx, buf->get(&v->sl, bytes));
        OZ_ALLOC(ctx, buf->get(&v->em, (size_t)s->n));
    } else {
        cudaError_t e = cudaMalloc(&v->sl, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&v->em, sizeof(int) * s->n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctx->set_error(SS_ERR_OOM, "tensor-core product: slices of the pencil do not fit");
        }
    }
    oz_attrs(ctx->device);
    ss_launch(ctx, SS_K_SPMM_TC, sstc::k_oz_csr_expmax, cdivu(s->n, 256), 256, 0, ctx->stream, s->n,
              (const int64_t *)s->d_rowptr, vals, v->em);
    if (pl->npairs > 0)
        ss_launch(ctx, SS_K_SPMM_TC, sstc::k_oz_slice_csr, (unsigned)pl->npairs, 128, sstc::kOzCsrSmem, ctx->stream,
                  s->n, (const int64_t *)s->d_rowptr, (const int32_t *)s->d_colind, vals, (const int64_t *)pl->d_seg,
                  (const int32_t *)pl->d_pair_tile, (const int32_t *)pl->d_pair_piece, (const int *)v->em, v->sl);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// digit slices of value array `which` (0: A, 1: B) of f, made on first use
int vals_get(ss_numeric *f, int which, OzVals **out) {
    *out = f->oz[which];
    if (*out) return SS_OK;
    OzVals *v = new OzVals();
    f->oz[which] = v;        // freed with the factor, also after a failure here
    const int rc = vals_make(f->sym, which == 0 ? f->a_vals : f->b_vals, v, nullptr);
    if (rc == SS_OK) *out = v;
    return rc;
}

// pass p adds alpha[p] diag(colscale[p]) M_p X, M_p the array sliced in v[p]; the first
// pass overwrites Y
int spmm_core(ss_symbolic *s, int npass, OzVals *const *v, const double *const *colscale, const double *alpha,
              const double *X, int64_t ldx, int k, double *Y, int64_t ldy) {
    ss_ctx *ctx = s->ctx;
    int rc;
    Scratch buf(ctx->stream);
    unsigned char *sx;
    int *ex;
    // operand rows of X = its k columns, reduction over the n rows
    const OzOperand xo{X, 1, ldx, k, s->n};
    if ((rc = slice_dense(ctx, xo, buf, &sx, &ex)) != SS_OK) return rc;
    const OzPlan *pl = s->oz_plan;
    for (int p = 0; p < npass; ++p) {
        sstc::OzMM g{};
        g.slA = v[p]->sl; g.emA = v[p]->em; g.nrtA = pl->nrt; g.rowsA = s->n;
        g.tile_ptr = pl->d_tile_ptr; g.pair_piece = pl->d_pair_piece;
        g.slB = sx; g.emB = ex; g.nrtB = (int)cdivu(k, 128); g.rowsB = k;
        g.mode = 1; g.alpha = alpha[p]; g.beta = p == 0 ? 0.0 : 1.0; g.colscale = colscale[p];
        g.out = Y; g.ldo = ldy;
        ctx->add_flops(SS_K_SPMM_TC, 2.0 * (double)s->nnz * k);
        ctx->add_tensor_flops(SS_K_SPMM_TC, kPieceTensorFlops * (double)pl->npairs * cdivu(k, 64));
        if ((rc = run_mm(ctx, g, dim3(cdivu(k, 64), pl->nrt, 1), SS_K_SPMM_TC)) != SS_OK) return rc;
    }
    return SS_OK;
}

}  // namespace

bool oz_dense_ok(const ss_ctx *ctx, int64_t n, int k1, int k2) {
    return ctx->gemm_mode == SS_GEMM_TENSOR && n >= 2048 && k1 >= 48 && k2 >= 48;
}

bool oz_spmm_ok(const ss_numeric *f, int k) {
    return f->sym->ctx->gemm_mode == SS_GEMM_TENSOR && f->sym->n >= 2048 && k >= 48 && !f->oz_failed;
}

int oz_gram(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int k1, const double *Y, int64_t ldy, int k2,
            double *G) {
    // operand rows = the columns of X and of Y, reduction over the n rows; G zeroed here
    SS_CUDA_TRY(ctx, cudaMemsetAsync(G, 0, sizeof(double) * k1 * k2, ctx->stream));
    const OzOperand a{X, 1, ldx, k1, n}, b{Y, 1, ldy, k2, n};
    return dense_mm(ctx, a, b, 0, 1.0, 0.0, G, k2, 2.0 * (double)n * k1 * k2);
}

int oz_gemm(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int k1, const double *Q, int k2, int transq,
            double alpha, double beta, double *Y, int64_t ldy) {
    // operand rows = the rows of X and the columns of the effective k1 x k2 Q, reduction over k1
    const OzOperand a{X, ldx, 1, n, k1};
    const OzOperand b = transq ? OzOperand{Q, k1, 1, k2, k1} : OzOperand{Q, 1, k2, k2, k1};
    return dense_mm(ctx, a, b, 1, alpha, beta, Y, ldy, 2.0 * (double)n * k1 * k2);
}

int oz_spmm(ss_numeric *f, int npass, const int *which, const double *const *colscale, const double *alpha,
            const double *X, int64_t ldx, int k, double *Y, int64_t ldy) {
    int rc;
    OzVals *v[2] = {nullptr, nullptr};
    for (int p = 0; p < npass; ++p)
        if ((rc = vals_get(f, which[p], &v[p])) != SS_OK) return rc;
    return spmm_core(f->sym, npass, v, colscale, alpha, X, ldx, k, Y, ldy);
}

int oz_spmm_vals(ss_symbolic *s, const double *a, const double *b, const double *alpha, const double *beta,
                 const double *X, int64_t ldx, int k, double *Y, int64_t ldy) {
    Scratch buf(s->ctx->stream);
    OzVals va, vb;
    int rc;
    if ((rc = vals_make(s, a, &va, &buf)) != SS_OK) return rc;
    if (beta && (rc = vals_make(s, b, &vb, &buf)) != SS_OK) return rc;
    OzVals *v[2] = {&va, &vb};
    const double *cs[2] = {alpha, beta};
    const double al[2] = {1.0, 1.0};
    return spmm_core(s, beta ? 2 : 1, v, cs, al, X, ldx, k, Y, ldy);
}

// Y = diag(alpha) A X + diag(beta) B X on the tensor cores when the mode, the sizes and the
// value arrays (the factor's own A and B) allow, else on the CUDA cores
int spmm_f(ss_numeric *f, const double *a, const double *b, const double *alpha, const double *beta, const double *X,
           int64_t ldx, int k, double *Y, int64_t ldy) {
    ss_symbolic *s = f->sym;
    const int ia = a == f->a_vals ? 0 : (a == f->b_vals ? 1 : -1);
    const int ib = !beta ? 0 : (b == f->a_vals ? 0 : (b == f->b_vals ? 1 : -1));
    if (oz_spmm_ok(f, k) && ia >= 0 && ib >= 0) {
        const int which[2] = {ia, ib};
        const double *cs[2] = {alpha, beta};
        const double al[2] = {1.0, 1.0};
        const int rc = oz_spmm(f, beta ? 2 : 1, which, cs, al, X, ldx, k, Y, ldy);
        if (rc != SS_ERR_OOM) return rc;
        // the pencil's slices do not fit beside the factor: CUDA cores from now on
        f->oz_failed = true;
        s->ctx->err.clear();
    }
    return spmm_launch_ld(s, a, b, alpha, beta, X, ldx, k, Y, ldy);
}

void oz_free_numeric(ss_numeric *f) {
    auto drop = [](OzVals *&v) {
        if (!v) return;
        if (v->sl) cudaFree(v->sl);
        if (v->em) cudaFree(v->em);
        delete v;
        v = nullptr;
    };
    for (OzVals *&v : f->oz) drop(v);
}

void oz_free_symbolic(ss_symbolic *s) {
    OzPlan *pl = s->oz_plan;
    if (!pl) return;
    void *ptrs[] = {pl->d_tile_ptr, pl->d_pair_tile, pl->d_pair_piece, pl->d_seg};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete pl;
    s->oz_plan = nullptr;
}
