// In-slice eigensolver (Alg. 2: shift-invert subspace iteration, Cholesky-QR in the B
// inner product, Rayleigh-Ritz, residual norms) and the Lanczos density-of-states
// estimate (Section 3.1).  All arithmetic runs in the kernels of dense_kernels.cuh and
// the factor/solve kernels; this file sequences them on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dense_kernels.cuh"
#include "internal.h"
#include "rq_kernels.cuh"

namespace {

struct DevBuf {
    std::vector<void *> ptrs;
    cudaStream_t st;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        cudaError_t e = cudaMallocAsync((void **)p, sizeof(T) * std::max<size_t>(count, 1), st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~DevBuf() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

#define TRY_ALLOC(ctx, expr)                                                                     \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return (ctx)->set_error(SS_ERR_OOM, std::string("device allocation failed: ") +    \
                                                    cudaGetErrorString(e_));                     \
        }                                                                                        \
    } while (0)

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// G = X^T Y (k1 x k2, contiguous); X, Y n x k with leading dimensions ldx, ldy
int gram_ld(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int k1, const double *Y, int64_t ldy, int k2,
            double *G, int sym = 0) {
    cudaStream_t st = ctx->stream;
    SS_CUDA_TRY(ctx, cudaMemsetAsync(G, 0, sizeof(double) * k1 * k2, st));
    if (oz_dense_ok(ctx, n, k1, k2)) return oz_gram(ctx, X, ldx, n, k1, Y, ldy, k2, G);
    const int64_t t1 = cdiv(k1, 32), t2 = cdiv(k2, 32);
    const int64_t bxy = sym ? t1 * (t1 + 1) / 2 : t1 * t2;     // tiles that do work
    int64_t nz = std::max<int64_t>(1, (4 * (int64_t)ctx->sm_count + bxy - 1) / bxy);
    nz = std::min<int64_t>(nz, std::max<int64_t>(1, n / 256));
    int64_t per = ((n + nz - 1) / nz + 31) / 32 * 32;
    nz = (n + per - 1) / per;
    ss_launch(ctx, SS_K_GRAM, ssd::k_gram, dim3(cdiv(k1, 32), cdiv(k2, 32), (unsigned)std::max<int64_t>(1, nz)), 256,
              0, st, n, X, ldx, k1, Y, ldy, k2, per, sym, G);
    ctx->add_flops(SS_K_GRAM, sym ? (double)n * k1 * (k2 + 1) : 2.0 * (double)n * k1 * k2);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

int gram(ss_ctx *ctx, const double *X, int64_t n, int k1, const double *Y, int k2, double *G, int sym = 0) {
    return gram_ld(ctx, X, k1, n, k1, Y, k2, k2, G, sym);
}

// Y = beta Y + alpha X Q (Q k1 x k2) or X Q^T (Q k2 x k1)
int gemm_ld(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int k1, const double *Q, int k2, int transq,
            double alpha, double beta, double *Y, int64_t ldy, int tri = 0) {
    if (oz_dense_ok(ctx, n, k1, k2)) return oz_gemm(ctx, X, ldx, n, k1, Q, k2, transq, alpha, beta, Y, ldy);
    ss_launch(ctx, SS_K_GEMM, ssd::k_gemm_tall, dim3(cdiv(n, 64), cdiv(k2, 32)), 256, 0, ctx->stream, n, X, ldx, k1,
              Q, k2, transq, alpha, beta, Y, ldy, tri);
    ctx->add_flops(SS_K_GEMM, tri ? (double)n * k2 * (k2 + 1) : 2.0 * (double)n * k1 * k2);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

int gemm_tall(ss_ctx *ctx, const double *X, int64_t n, int k1, const double *Q, int k2, int transq, double *Y,
              int tri = 0) {
    return gemm_ld(ctx, X, k1, n, k1, Q, k2, transq, 1.0, 0.0, Y, k2, tri);
}

__global__ void k_symmetrize(double *H, int k) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)k * k) return;
    const int i = (int)(q / k), j = (int)(q % k);
    if (i < j) {
        double v = 0.5 * (H[(int64_t)i * k + j] + H[(int64_t)j * k + i]);
        H[(int64_t)i * k + j] = v;
        H[(int64_t)j * k + i] = v;
    }
}

__global__ void k_add_shift_diag(double *G, int k, double rel) {
    // G += rel * trace(G) * I  (one block)
    __shared__ double s_tr;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < k; ++i) t += G[(int64_t)i * k + i];
        s_tr = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) G[(int64_t)i * k + i] += rel * s_tr;
}

// Symmetric eigenproblem of H (k x k, destroyed): ascending evals (device) and Q.
// eigenpairs of the symmetric k x k H by parallel-ordered Jacobi, stopped once the
// off-diagonal Frobenius norm is below tol times the whole norm
int sym_eig(ss_ctx *ctx, double *H, int k, double *evals, double *Q, DevBuf &buf, double tol = 1e-14) {
    cudaStream_t st = ctx->stream;
    double *V;
    TRY_ALLOC(ctx, buf.get(&V, (size_t)k * k));
    const unsigned g = cdiv((int64_t)k * k, 256);
    ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, g, 256, 0, st, H, k);
    ss_launch(ctx, SS_K_JACOBI, ssd::k_set_identity, g, 256, 0, st, V, k);
    if (k > 1 && k <= 96) {
        const int np = (k + (k & 1)) / 2;
        const size_t smem = sizeof(int) * (2 * np + 2) + sizeof(double) * 2 * np;
        ss_launch(ctx, SS_K_JACOBI, ssd::k_jacobi_block, 1, 1024, smem, st, H, V, k, 1e-18, tol, 40,
                  (int *)nullptr);
    } else if (k > 96) {
        // cooperative grid: every block resident, rounds separated by a bounded barrier
        const int np = (k + (k & 1)) / 2, max_sweeps = 40;
        const size_t smem = (sizeof(double2) + sizeof(int2)) * (size_t)np;
        double *acc, *H2;
        ssd::GridBar *bar;
        int *status;
        TRY_ALLOC(ctx, buf.get(&H2, (size_t)k * k));
        TRY_ALLOC(ctx, buf.get(&acc, (size_t)2 * max_sweeps));
        TRY_ALLOC(ctx, buf.get(&bar, 1));
        TRY_ALLOC(ctx, buf.get(&status, 1));
        SS_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * 2 * max_sweeps, st));
        SS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, sizeof(ssd::GridBar), st));
        SS_CUDA_TRY(ctx, cudaFuncSetAttribute(ssd::k_jacobi_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)std::max<size_t>(smem, 1)));
        int per_sm = 0;
        SS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ssd::k_jacobi_grid, 256, smem));
        const int64_t want = ((int64_t)np * np + 255) / 256;
        int nb = (int)std::min<int64_t>(std::max(1, std::min(per_sm, 2)) * (int64_t)ctx->sm_count, std::max<int64_t>(1, want));
        const double thr = 1e-18;
        const long long limit = 20000000;      // units of 64 ns: ~1.3 s
        int *sw = status;
        void *args[] = {(void *)&H, (void *)&H2, (void *)&V, (void *)&k, (void *)&thr, (void *)&tol,
                        (void *)&max_sweeps, (void *)&acc, (void *)&bar, (void *)&limit, (void *)&sw};
        g_ss_launches.fetch_add(1, std::memory_order_relaxed);
        size_t slot = 0;
        const bool prof = ctx->prof_mask & (1u << SS_K_JACOBI);
        if (prof) slot = ss_prof_begin(ctx, SS_K_JACOBI);
        SS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void *)ssd::k_jacobi_grid, dim3(nb), dim3(256), args, smem, st));
        if (prof) ss_prof_end(ctx, SS_K_JACOBI, slot);
        int herr = 0;
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, &bar->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        if (herr) return ctx->set_error(SS_ERR_TIMEOUT, "Jacobi eigensolver: grid barrier timed out");
    }
    ss_launch(ctx, SS_K_JACOBI, ssd::k_eig_sort, cdiv(k, 256), 256, 0, st, (const double *)H, (const double *)V, k,
              evals, Q);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// G = R R^T in place (lower R, upper part zeroed) by the multi-block blocked Cholesky;
// *info (device) is 0 or the first failing pivot index + 1.
int chol_small(ss_ctx *ctx, double *G, int k, int *info) {
    cudaStream_t st = ctx->stream;
    SS_CUDA_TRY(ctx, cudaMemsetAsync(info, 0, sizeof(int), st));
    for (int j0 = 0; j0 < k; j0 += ssd::CH_NB) {
        const int w = std::min(ssd::CH_NB, k - j0), rem = k - j0 - w;
        ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_chol_diag, 1, 32, 0, st, G, k, j0, info);
        if (rem > 0) {
            ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_chol_trsm, cdiv(rem, 8), 256, 0, st, G, k, j0, (const int *)info);
            const int nt = (int)cdiv(rem, 32);
            ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_chol_syrk, (unsigned)(nt * (nt + 1) / 2), 256, 0, st, G, k, j0,
                      (const int *)info);
        }
    }
    ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_zero_upper, cdiv((int64_t)k * k, 256), 256, 0, st, G, k);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// V <- V R^-T with R R^T = V^T B V (Cholesky-QR in the B inner product, run twice; the
// first pass adds a small diagonal shift when the plain Gram matrix is not numerically
// positive definite -- shifted Cholesky-QR).  BV scratch n x k, G/Rinv k x k.
int cholqr_b(ss_numeric *f, double *&V, double *&Wk, int k, double *G, double *Rinv, int *info, DevBuf &buf) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    int rc;
    for (int pass = 0; pass < 2; ++pass) {
        if ((rc = spmm_f(f, f->b_vals, f->b_vals, nullptr, nullptr, V, k, k, Wk, k)) != SS_OK) return rc;
        if ((rc = gram(ctx, V, s->n, k, Wk, k, G, 1)) != SS_OK) return rc;
        ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, cdiv((int64_t)k * k, 256), 256, 0, st, G, k);
        int hinfo = 0;
        for (int attempt = 0; attempt < 3; ++attempt) {
            if (attempt > 0) {
                // restore G from Wk (still B V) and shift it
                if ((rc = gram(ctx, V, s->n, k, Wk, k, G, 1)) != SS_OK) return rc;
                ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, cdiv((int64_t)k * k, 256), 256, 0, st, G, k);
                const double rel = 11.0 * ((double)s->n * k + (double)k * (k + 1)) * 1.1102230246251565e-16 *
                                   (attempt == 1 ? 1.0 : 1e4);
                ss_launch(ctx, SS_K_SMALL_DENSE, k_add_shift_diag, 1, 256, 0, st, G, k, rel);
            }
            if ((rc = chol_small(ctx, G, k, info)) != SS_OK) return rc;
            SS_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
            SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            if (hinfo == 0) break;
        }
        if (hinfo != 0)
            return ctx->set_error(SS_ERR_NOCONV, "Cholesky-QR: basis is numerically rank deficient");
        ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_trinv_lower, cdiv(k, 32), 256, 0, st, (const double *)G, k, Rinv);
        if ((rc = gemm_tall(ctx, V, s->n, k, Rinv, k, 1, Wk, 1)) != SS_OK) return rc;
        std::swap(V, Wk);
    }
    (void)buf;
    return SS_OK;
}

// B-orthonormalise W in place, carrying BW = B W along: G = W^T BW = R R^T,
// W <- W R^-T, BW <- BW R^-T, twice (Cholesky-QR2); a failed Cholesky is retried with
// a diagonal shift of G (shifted Cholesky-QR).  Wt, BWt: n x k scratch (swapped in).
int cholqr_track(ss_numeric *f, double *&W, double *&BW, double *&Wt, double *&BWt, int k, double *G, double *Rinv,
                 int *info, int passes = 2) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    int rc;
    for (int pass = 0; pass < passes; ++pass) {
        int hinfo = 0;
        for (int attempt = 0; attempt < 3; ++attempt) {
            if ((rc = gram(ctx, W, s->n, k, BW, k, G, 1)) != SS_OK) return rc;
            ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, cdiv((int64_t)k * k, 256), 256, 0, st, G, k);
            if (attempt > 0) {
                const double rel = 11.0 * ((double)s->n * k + (double)k * (k + 1)) * 1.1102230246251565e-16 *
                                   (attempt == 1 ? 1.0 : 1e4);
                ss_launch(ctx, SS_K_SMALL_DENSE, k_add_shift_diag, 1, 256, 0, st, G, k, rel);
            }
            if ((rc = chol_small(ctx, G, k, info)) != SS_OK) return rc;
            SS_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
            SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            if (hinfo == 0) break;
        }
        if (hinfo != 0) return ctx->set_error(SS_ERR_NOCONV, "Cholesky-QR: basis is numerically rank deficient");
        ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_trinv_lower, cdiv(k, 32), 256, 0, st, (const double *)G, k, Rinv);
        if ((rc = gemm_tall(ctx, W, s->n, k, Rinv, k, 1, Wt, 1)) != SS_OK) return rc;
        if ((rc = gemm_tall(ctx, BW, s->n, k, Rinv, k, 1, BWt, 1)) != SS_OK) return rc;
        std::swap(W, Wt);
        std::swap(BW, BWt);
    }
    return SS_OK;
}

// Rayleigh quotients x^T A x / x^T B x of the k columns of X (N x k), summed and divided
// in double-double: the eigenvalue estimates a probe returns.  A Rayleigh-Ritz value
// carries the rounding of forming W^T A W, about u ||A|| ||x||_2^2 -- up to 2e-9 on the
// low tail of the Gaussian pencils, whose B-normalised eigenvectors have ||x||_2 of
// hundreds -- while the quotient of the Ritz vector is second-order in the vector's error.
int rq_polish(ss_numeric *f, const double *X, int k, double *theta_d, DevBuf &buf) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    const int64_t n = s->n;
    const int nby = (int)cdiv(k, 128);
    const int64_t nbx = std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 16), cdiv(32ll * ctx->sm_count, nby)));
    const int64_t rows_per = (n + nbx - 1) / nbx;
    const int64_t nparts = (n + rows_per - 1) / rows_per;
    double *part;
    TRY_ALLOC(ctx, buf.get(&part, (size_t)nparts * k * 4));
    ss_launch(ctx, SS_K_MISC, sss::k_rq_dd_partial, dim3((unsigned)nparts, nby), 128, 0, ctx->stream, n, s->d_rowptr,
              s->d_colind, f->a_vals, f->b_vals, X, k, rows_per, part);
    ss_launch(ctx, SS_K_MISC, sss::k_rq_dd_finish, cdiv(k, 256), 256, 0, ctx->stream, k, (int)nparts,
              (const double *)part, theta_d);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// Alg. 2 with a Rayleigh-Ritz step every check_every iterations.  Per iteration: one
// solve (A - sigma B) W = B V, one SpMM for B W, Cholesky-QR2 in the B inner product
// carrying B W, and at a check one SpMM for A W, H = W^T A W = Q Theta Q^T, X = W Q with
// A X and B X formed as (A W) Q and (B W) Q, the residual norms, and V = X, B V = B X.
int slice_solve_impl(ss_numeric *f, int j, double lo, double hi, const ss_solve_opts &o, const double *V0, int k,
                     double *lambda, double *X, double *resid, int32_t *n_found, ss_probe_stats *stats) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = s->n;
    DevBuf buf(st);
    double *V, *BV, *W, *BW, *T1, *T2, *G, *Rinv, *Q, *theta_d, *resid_d, *rr;
    int *info;
    TRY_ALLOC(ctx, buf.get(&V, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&BV, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&W, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&BW, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&T1, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&T2, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&G, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&Rinv, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&Q, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&theta_d, (size_t)k));
    TRY_ALLOC(ctx, buf.get(&resid_d, (size_t)k));
    TRY_ALLOC(ctx, buf.get(&rr, (size_t)2 * k));
    TRY_ALLOC(ctx, buf.get(&info, 1));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(V, V0, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, st));
    int rc;
    if ((rc = spmm_f(f, f->b_vals, f->b_vals, nullptr, nullptr, V, k, k, BV, k)) != SS_OK) return rc;
    if ((rc = cholqr_track(f, V, BV, T1, T2, k, G, Rinv, info)) != SS_OK) return rc;
    std::vector<double> th(k), rs(k);
    int it = 0, refine_total = 0;
    bool conv = false, have_rr = false, near_conv = o.refine_from_start != 0;
    std::vector<double> hist;
    double maxr = 0.0, maxr_all = INFINITY;
    int nf = 0;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 200;
    // check_every < 0: the first Rayleigh-Ritz after |check_every| iterations, later ones
    // where the residual's observed reduction per iteration predicts convergence
    const bool adaptive = o.check_every < 0;
    const int every = o.check_every > 0 ? o.check_every : (adaptive ? -o.check_every : 1);
    int next_rr = every, it_prev_rr = 0;
    const int refine = o.refine > 0 ? o.refine : 2;
    const double tol = o.tol > 0 ? o.tol : 1e-10;
    const double ratio = o.refine_ratio > 0 ? std::min(o.refine_ratio, 1.0) : 1e-1;
    const int64_t per = 2048;
    while (it < max_iter) {
        ++it;
        // W = (A - sigma B)^-1 B V (Alg. 2 step 3); a mixed factor runs plain FP32 solves
        // while the window's residuals are above 1e-6 and FP64 refinement afterwards
        int done_ref = 0;
        const int ref_now = near_conv ? (ss_solves_f32(f, j) ? refine : 1) : 0;
        // FP32 solves refine until their residual is 1e-1 of the window's current residual
        // (1e-13 before the first Rayleigh-Ritz of this call, at most 1e-8): inexact inverse
        // iteration keeps converging while the solve error falls in step with the residual
        double ref_target = 0.0;
        if (near_conv && ss_solves_f32(f, j))
            ref_target = hist.empty() ? 1e-13 : std::max(1e-14, std::min(1e-8, ratio * hist.back()));
        if ((rc = solve_apply(f, j, BV, k, W, ref_now, &done_ref, ref_target)) != SS_OK) return rc;
        refine_total += done_ref;
        if ((rc = spmm_f(f, f->b_vals, f->b_vals, nullptr, nullptr, W, k, k, BW, k)) != SS_OK) return rc;
        // Alg. 2 step 4; one Cholesky-QR pass when no Rayleigh-Ritz follows (the next
        // solve only needs a well-conditioned basis), two before a Rayleigh-Ritz
        const bool rr_now = adaptive ? (it >= next_rr || it == max_iter) : ((it % every == 0) || it == max_iter);
        if ((rc = cholqr_track(f, W, BW, T1, T2, k, G, Rinv, info, rr_now ? 2 : 1)) != SS_OK) return rc;
        if (!rr_now) {
            std::swap(V, W);
            std::swap(BV, BW);
            continue;
        }
        // Rayleigh-Ritz: H = W^T A W; the dead V / BV buffers take A W and A X
        double *AW = V, *AX = BV;
        if ((rc = spmm_f(f, f->a_vals, f->a_vals, nullptr, nullptr, W, k, k, AW, k)) != SS_OK) return rc;
        if ((rc = gram(ctx, W, n, k, AW, k, G, 1)) != SS_OK) return rc;
        // the eigenvectors of H need only be a little more accurate than the window's
        // current residual: the residuals below are computed from the rotated basis itself,
        // so a looser rotation only shows as a larger residual, never a false convergence
        const double jtol = hist.empty() ? 1e-10 : std::min(1e-8, std::max(1e-14, 1e-3 * hist.back()));
        if ((rc = sym_eig(ctx, G, k, theta_d, Q, buf, jtol)) != SS_OK) return rc;
        if ((rc = gemm_tall(ctx, W, n, k, Q, k, 0, T1)) != SS_OK) return rc;      // X
        if ((rc = gemm_tall(ctx, BW, n, k, Q, k, 0, T2)) != SS_OK) return rc;     // B X
        if ((rc = gemm_tall(ctx, AW, n, k, Q, k, 0, AX)) != SS_OK) return rc;     // A X
        SS_CUDA_TRY(ctx, cudaMemsetAsync(rr, 0, sizeof(double) * 2 * k, st));
        ss_launch(ctx, SS_K_MISC, ssd::k_resid_sumsq, dim3(cdiv(k, 128), cdiv(n, per)), 128, 0, st, n, k,
                  (const double *)AX, (const double *)T2, (const double *)theta_d, per, rr);
        ss_launch(ctx, SS_K_MISC, ssd::k_col_sumsq, dim3(cdiv(k, 128), cdiv(n, per)), 128, 0, st, n, k,
                  (const double *)T1, per, rr + k);
        ss_launch(ctx, SS_K_MISC, ssd::k_resid_finish, cdiv(k, 256), 256, 0, st, k, (const double *)rr,
                  (const double *)(rr + k), f->norm_a1, resid_d);
        // V = X, B V = B X
        std::swap(V, T1);
        std::swap(BV, T2);
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(th.data(), theta_d, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(rs.data(), resid_d, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        have_rr = true;
        // a Ritz value in the window counts once its residual meets tol; unconverged
        // ones in the window may be spurious mixtures from the edge of the basis
        // (eigenvalues at equal distance on both sides of sigma), which validation by
        // inertia counts removes (Section 2.2), so with n_expect given the probe stops
        // as soon as n_expect of them have converged
        nf = 0;
        maxr = 0.0;
        maxr_all = 0.0;
        int nin = 0;
        for (int i = 0; i < k; ++i) {
            if (th[i] > lo && th[i] <= hi) {
                ++nin;
                maxr_all = std::max(maxr_all, rs[i]);
                if (rs[i] <= tol) {
                    ++nf;
                    maxr = std::max(maxr, rs[i]);
                }
            }
        }
        const bool done = o.n_expect > 0 ? (nf >= o.n_expect) : (nf == nin);
        if (done && it >= 2) { conv = true; break; }
        // refinement of the solves (FP64 residuals) starts once the window's target count
        // is within 1e-6, or when the target-th best window residual stops improving
        // (the solve's own error then limits the eigenvectors far from sigma)
        {
            std::vector<double> wr;
            for (int i = 0; i < k; ++i)
                if (th[i] > lo && th[i] <= hi) wr.push_back(rs[i]);
            std::sort(wr.begin(), wr.end());
            const int target = o.n_expect > 0 ? o.n_expect : std::max(1, nin - 2);
            const double rt = (int)wr.size() >= target ? wr[target - 1] : INFINITY;
            hist.push_back(rt);
            if (adaptive) {
                // iterations until the target-th window residual reaches tol at the rate seen
                // between the last two checks (at most 8, at least 1)
                int gap = every;
                const size_t h2 = hist.size();
                if (h2 >= 2 && std::isfinite(hist[h2 - 1]) && std::isfinite(hist[h2 - 2]) && hist[h2 - 1] > 0.0 &&
                    hist[h2 - 1] < hist[h2 - 2] && it > it_prev_rr) {
                    const double rate = std::pow(hist[h2 - 1] / hist[h2 - 2], 1.0 / (double)(it - it_prev_rr));
                    const double need = rt <= tol ? 1.0 : std::log(tol / rt) / std::log(rate);
                    gap = (int)std::max(1.0, std::min(8.0, std::ceil(need)));
                }
                it_prev_rr = it;
                next_rr = it + gap;
            }
            const size_t h = hist.size();
            const bool stalled = h >= 5 && !(hist[h - 1] < 0.5 * hist[h - 4]);
            near_conv = near_conv || rt <= 1e-6 || stalled;
        }
    }
    (void)maxr_all;
    // the returned eigenvalues: double-double Rayleigh quotients of the Ritz vectors
    if (have_rr) {
        if ((rc = rq_polish(f, V, k, theta_d, buf)) != SS_OK) return rc;
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(th.data(), theta_d, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    }
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(X, V, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    std::memcpy(lambda, th.data(), sizeof(double) * k);
    std::memcpy(resid, rs.data(), sizeof(double) * k);
    if (n_found) *n_found = nf;
    if (stats) {
        stats->iterations = it;
        stats->refine_steps = refine_total;
        stats->converged = conv ? 1 : 0;
        stats->max_resid_in_slice = maxr;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!conv) return ctx->set_error(SS_ERR_NOCONV, "ss_slice_solve: iteration cap reached");
    return SS_OK;
}

// Shift-invert block Lanczos (the SI-Lanczos the paper names as the alternative to
// Alg. 2, Section 1) in the B inner product with full re-orthogonalisation: V_1 =
// CholQR_B(V0), V_{i+1} = CholQR_B((I - P) O V_i) with O = (A - sigma B)^-1 B and P the
// B-orthogonal projector on every earlier block (applied twice), then one Rayleigh-Ritz
// on the whole basis (H = V^T A V) and the k_out Ritz pairs nearest sigma.
int block_lanczos_impl(ss_numeric *f, int j, double lo, double hi, const ss_solve_opts &o, const double *V0,
                       int p, int kout, double *lambda, double *X, double *resid, int32_t *n_found,
                       ss_probe_stats *stats) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = s->n;
    const int m = o.max_iter > 0 ? o.max_iter : 6;
    const int64_t dmax = (int64_t)m * p;
    if (kout > dmax) return ctx->set_error(SS_ERR_ARG, "ss_slice_solve: k_out exceeds the Krylov basis");
    const int refine = o.refine > 0 ? o.refine : 2;
    const double tol = o.tol > 0 ? o.tol : 1e-10;
    const double sigma = f->sigma[j];
    DevBuf buf(st);
    double *Vb, *AV, *W, *Wk, *T, *Gp, *Rinv, *Hc, *H, *Q, *theta_d, *Qsel, *resid_d, *rr, *be;
    int *info;
    TRY_ALLOC(ctx, buf.get(&Vb, (size_t)n * dmax));
    TRY_ALLOC(ctx, buf.get(&AV, (size_t)n * dmax));
    TRY_ALLOC(ctx, buf.get(&W, (size_t)n * p));
    TRY_ALLOC(ctx, buf.get(&Wk, (size_t)n * std::max<int64_t>(p, kout)));
    TRY_ALLOC(ctx, buf.get(&T, (size_t)n * std::max<int64_t>(p, kout)));
    TRY_ALLOC(ctx, buf.get(&Gp, (size_t)p * p));
    TRY_ALLOC(ctx, buf.get(&Rinv, (size_t)p * p));
    TRY_ALLOC(ctx, buf.get(&Hc, (size_t)dmax * p));
    TRY_ALLOC(ctx, buf.get(&H, (size_t)dmax * dmax));
    TRY_ALLOC(ctx, buf.get(&Q, (size_t)dmax * dmax));
    TRY_ALLOC(ctx, buf.get(&theta_d, (size_t)dmax));
    TRY_ALLOC(ctx, buf.get(&Qsel, (size_t)dmax * kout));
    TRY_ALLOC(ctx, buf.get(&resid_d, (size_t)kout));
    TRY_ALLOC(ctx, buf.get(&rr, (size_t)2 * kout));
    TRY_ALLOC(ctx, buf.get(&be, (size_t)kout));
    TRY_ALLOC(ctx, buf.get(&info, 1));
    int rc;
    const unsigned gcopy = cdiv(n * p, 256);
    // V_1 = CholQR_B(V0)
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(W, V0, sizeof(double) * n * p, cudaMemcpyDeviceToDevice, st));
    if ((rc = cholqr_b(f, W, Wk, p, Gp, Rinv, info, buf)) != SS_OK) return rc;
    ss_launch(ctx, SS_K_MISC, ssd::k_copy_cols, gcopy, 256, 0, st, n, p, (const double *)W, (int64_t)p, Vb, dmax);
    int64_t cur = p;
    int refine_total = 0, blocks = 1;
    for (int blk = 1; blk < m; ++blk) {
        // W = O V_blk = (A - sigma B)^-1 B V_blk
        if ((rc = spmm_f(f, f->b_vals, f->b_vals, nullptr, nullptr, Vb + (cur - p), dmax, p, T, p)) != SS_OK)
            return rc;
        int done_ref = 0;
        if ((rc = solve_apply(f, j, T, p, W, refine, &done_ref)) != SS_OK) return rc;
        refine_total += done_ref;
        for (int pass = 0; pass < 2; ++pass) {    // W -= V (V^T B W), twice
            if ((rc = spmm_f(f, f->b_vals, f->b_vals, nullptr, nullptr, W, p, p, T, p)) != SS_OK) return rc;
            if ((rc = gram_ld(ctx, Vb, dmax, n, (int)cur, T, p, p, Hc)) != SS_OK) return rc;
            if ((rc = gemm_ld(ctx, Vb, dmax, n, (int)cur, Hc, p, 0, -1.0, 1.0, W, p)) != SS_OK) return rc;
        }
        if ((rc = cholqr_b(f, W, Wk, p, Gp, Rinv, info, buf)) != SS_OK) return rc;
        ss_launch(ctx, SS_K_MISC, ssd::k_copy_cols, gcopy, 256, 0, st, n, p, (const double *)W, (int64_t)p,
                  Vb + cur, dmax);
        cur += p;
        ++blocks;
    }
    // Rayleigh-Ritz on the basis: H = V^T A V
    const int d = (int)cur;
    if ((rc = spmm_f(f, f->a_vals, f->a_vals, nullptr, nullptr, Vb, dmax, d, AV, dmax)) != SS_OK) return rc;
    if ((rc = gram_ld(ctx, Vb, dmax, n, d, AV, dmax, d, H, 1)) != SS_OK) return rc;
    if ((rc = sym_eig(ctx, H, d, theta_d, Q, buf)) != SS_OK) return rc;
    std::vector<double> th(d), hq((size_t)d * d);
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(th.data(), theta_d, sizeof(double) * d, cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(hq.data(), Q, sizeof(double) * d * d, cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    // the kout Ritz values nearest sigma, returned in ascending order
    std::vector<int> idx(d);
    for (int i = 0; i < d; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return std::fabs(th[x] - sigma) < std::fabs(th[y] - sigma);
    });
    idx.resize(kout);
    std::sort(idx.begin(), idx.end());
    std::vector<double> qs((size_t)d * kout);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < kout; ++c) qs[(size_t)r * kout + c] = hq[(size_t)r * d + idx[c]];
    std::vector<double> ths(kout);
    for (int c = 0; c < kout; ++c) ths[c] = th[idx[c]];
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(Qsel, qs.data(), sizeof(double) * d * kout, cudaMemcpyHostToDevice, st));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(theta_d, ths.data(), sizeof(double) * kout, cudaMemcpyHostToDevice, st));
    if ((rc = gemm_ld(ctx, Vb, dmax, n, d, Qsel, kout, 0, 1.0, 0.0, X, kout)) != SS_OK) return rc;
    // residuals ||A x - theta B x|| / (||A||_1 ||x||)
    ss_launch(ctx, SS_K_MISC, ssd::k_neg_scale, cdiv(kout, 256), 256, 0, st, kout, (const double *)theta_d, be);
    if ((rc = spmm_f(f, f->a_vals, f->b_vals, nullptr, be, X, kout, kout, T, kout)) != SS_OK) return rc;
    SS_CUDA_TRY(ctx, cudaMemsetAsync(rr, 0, sizeof(double) * 2 * kout, st));
    const int64_t per = 2048;
    ss_launch(ctx, SS_K_MISC, ssd::k_col_sumsq, dim3(cdiv(kout, 128), cdiv(n, per)), 128, 0, st, n, kout,
              (const double *)T, per, rr);
    ss_launch(ctx, SS_K_MISC, ssd::k_col_sumsq, dim3(cdiv(kout, 128), cdiv(n, per)), 128, 0, st, n, kout,
              (const double *)X, per, rr + kout);
    ss_launch(ctx, SS_K_MISC, ssd::k_resid_finish, cdiv(kout, 256), 256, 0, st, kout, (const double *)rr,
              (const double *)(rr + kout), f->norm_a1, resid_d);
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(resid, resid_d, sizeof(double) * kout, cudaMemcpyDeviceToHost, st));
    // the returned eigenvalues: double-double Rayleigh quotients of the Ritz vectors
    if ((rc = rq_polish(f, X, kout, theta_d, buf)) != SS_OK) return rc;
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(ths.data(), theta_d, sizeof(double) * kout, cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    std::memcpy(lambda, ths.data(), sizeof(double) * kout);
    int nf = 0;
    double maxr = 0.0;
    for (int i = 0; i < kout; ++i)
        if (ths[i] > lo && ths[i] <= hi && resid[i] <= tol) { ++nf; maxr = std::max(maxr, resid[i]); }
    if (n_found) *n_found = nf;
    const bool conv = o.n_expect > 0 ? nf >= o.n_expect : true;
    if (stats) {
        stats->iterations = blocks;
        stats->refine_steps = refine_total;
        stats->converged = conv ? 1 : 0;
        stats->max_resid_in_slice = maxr;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!conv) return ctx->set_error(SS_ERR_NOCONV, "ss_slice_solve: fewer than n_expect converged Ritz pairs");
    return SS_OK;
}

// B = P L D L^T P^T: the multifrontal LDL^T at sigma = 0 of the pencil (B, 0), FP64.
// Fails with SS_ERR_NOT_SPD unless every eigenvalue of D is positive.
int factor_spd_b(ss_symbolic *s, const double *b_vals, ss_numeric **out) {
    ss_ctx *ctx = s->ctx;
    const double zero = 0.0;
    ss_numeric *fb = nullptr;
    int rc = ss_factor_create(s, b_vals, b_vals, &zero, 1, SS_FP64, &fb);
    if (rc != SS_OK && rc != SS_ERR_SINGULAR) return rc;
    int64_t neg = 0, zr = 0, pos = 0;
    ss_inertia(fb, 0, &neg, &zr, &pos, nullptr);
    if (neg != 0 || zr != 0 || rc == SS_ERR_SINGULAR) {
        ss_factor_destroy(fb);
        return ctx->set_error(SS_ERR_NOT_SPD, "B is not positive definite (inertia " + std::to_string(neg) + "/" +
                                                  std::to_string(zr) + "/" + std::to_string(pos) + ")");
    }
    *out = fb;
    return SS_OK;
}

int lanczos_impl(ss_symbolic *s, ss_numeric *fb, const double *a_vals, const double *b_vals, int steps, int nv,
                 const double *start, double *theta, double *zeta2, int32_t *m_run) {
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t n = s->n;
    int rc;
    DevBuf buf(st);
    const int64_t blk = n * nv;
    double *X, *BX, *u, *w, *bw, *h, *alpha, *beta, *nrm;
    TRY_ALLOC(ctx, buf.get(&X, (size_t)(steps + 1) * blk));
    TRY_ALLOC(ctx, buf.get(&BX, (size_t)(steps + 1) * blk));
    TRY_ALLOC(ctx, buf.get(&u, (size_t)blk));
    TRY_ALLOC(ctx, buf.get(&w, (size_t)blk));
    TRY_ALLOC(ctx, buf.get(&bw, (size_t)blk));
    TRY_ALLOC(ctx, buf.get(&h, (size_t)(steps + 1) * nv));
    TRY_ALLOC(ctx, buf.get(&alpha, (size_t)steps * nv));
    TRY_ALLOC(ctx, buf.get(&beta, (size_t)steps * nv));
    TRY_ALLOC(ctx, buf.get(&nrm, (size_t)nv));
    const unsigned g = cdiv(blk, 256);
    auto coldot = [&](const double *x, const double *y, double *out) -> int {
        SS_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(double) * nv, st));
        unsigned gb = std::min<unsigned>(cdiv(blk, 256), 4 * ctx->sm_count);
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_col_dot, gb, 256, 0, st, n, nv, x, y, out);
        return SS_OK;
    };
    auto reorth = [&](int j) -> int {   // w, bw -= X h, BX h with h = X^T bw  (j+1 vectors)
        SS_CUDA_TRY(ctx, cudaMemsetAsync(h, 0, sizeof(double) * (j + 1) * nv, st));
        const int64_t per = 32768;
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_dots, dim3(j + 1, cdiv(blk, per)), 256, 0, st, X, n, nv, j + 1, bw, per, h);
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_sub, g, 256, 0, st, X, n, nv, j + 1, h, w);
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_sub, g, 256, 0, st, BX, n, nv, j + 1, h, bw);
        return SS_OK;
    };
    // x_1 = start / ||start||_B
    if ((rc = spmm_launch(s, b_vals, b_vals, nullptr, nullptr, start, nv, bw)) != SS_OK) return rc;
    coldot(start, bw, nrm);
    ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_normalize, g, 256, 0, st, n, nv, start, nrm, beta /*scratch*/, X);
    ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_normalize, g, 256, 0, st, n, nv, bw, nrm, beta, BX);
    for (int j = 0; j < steps; ++j) {
        double *xj = X + (int64_t)j * blk;
        if ((rc = spmm_launch(s, a_vals, a_vals, nullptr, nullptr, xj, nv, u)) != SS_OK) return rc;
        coldot(xj, u, alpha + (int64_t)j * nv);
        if ((rc = solve_apply(fb, 0, u, nv, w, 0, nullptr)) != SS_OK) return rc;
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_three_term, g, 256, 0, st, n, nv, xj, j > 0 ? xj - blk : nullptr, alpha + (int64_t)j * nv,
                                                 j > 0 ? beta + (int64_t)(j - 1) * nv : nullptr, w);
        if ((rc = spmm_launch(s, b_vals, b_vals, nullptr, nullptr, w, nv, bw)) != SS_OK) return rc;
        reorth(j);
        reorth(j);
        coldot(w, bw, nrm);
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_normalize, g, 256, 0, st, n, nv, w, nrm, beta + (int64_t)j * nv, X + (int64_t)(j + 1) * blk);
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_normalize, g, 256, 0, st, n, nv, bw, nrm, beta + (int64_t)j * nv, BX + (int64_t)(j + 1) * blk);
    }
    SS_CUDA_TRY(ctx, cudaGetLastError());
    std::vector<double> ha((size_t)steps * nv), hb((size_t)steps * nv);
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * steps * nv, cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(hb.data(), beta, sizeof(double) * steps * nv, cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    std::memset(theta, 0, sizeof(double) * steps * nv);
    std::memset(zeta2, 0, sizeof(double) * steps * nv);
    double *T, *Q, *ev;
    TRY_ALLOC(ctx, buf.get(&T, (size_t)steps * steps));
    TRY_ALLOC(ctx, buf.get(&Q, (size_t)steps * steps));
    TRY_ALLOC(ctx, buf.get(&ev, (size_t)steps));
    std::vector<double> hq(steps);
    for (int c = 0; c < nv; ++c) {
        int m = steps;
        for (int j = 0; j + 1 < steps; ++j)
            if (hb[(size_t)j * nv + c] <= 1e-13 * std::max(1.0, std::fabs(ha[(size_t)j * nv + c]))) { m = j + 1; break; }
        m_run[c] = m;
        ss_launch(ctx, SS_K_LANCZOS, ssd::k_lz_tridiag, cdiv((int64_t)m * m, 256), 256, 0, st, alpha, beta, nv, c, m, T);
        if ((rc = sym_eig(ctx, T, m, ev, Q, buf)) != SS_OK) return rc;
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(theta + (size_t)c * steps, ev, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(hq.data(), Q, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        for (int i = 0; i < m; ++i) zeta2[(size_t)c * steps + i] = hq[i] * hq[i];
    }
    return SS_OK;
}

}  // namespace

extern "C" ss_status ss_slice_solve(ss_numeric *f, int32_t j, double lo, double hi, const ss_solve_opts *opts,
                                    const double *V0, int32_t k, double *lambda, double *X, double *resid,
                                    int32_t *n_found, ss_probe_stats *stats) {
    if (!f) return SS_ERR_ARG;
    ss_ctx *ctx = f->sym->ctx;
    if (j < 0 || j >= f->n_shift || !V0 || !X || !lambda || !resid || k <= 0 || k > f->sym->n || k > 4096 ||
        !(lo < hi) || f->inertia_only)
        return ctx->set_error(SS_ERR_ARG, "ss_slice_solve: bad argument (or an inertia-only factor)");
    ss_solve_opts o{};
    if (opts) o = *opts;
    if (o.driver != SS_SUBSPACE && o.driver != SS_BLOCK_LANCZOS)
        return ctx->set_error(SS_ERR_ARG, "ss_slice_solve: unknown driver");
    const int kout = o.k_out > 0 ? o.k_out : k;
    if (o.driver == SS_SUBSPACE && kout != k)
        return ctx->set_error(SS_ERR_ARG, "ss_slice_solve: the subspace driver returns k pairs (k_out = k)");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    try {
        if (o.driver == SS_BLOCK_LANCZOS)
            return block_lanczos_impl(f, j, lo, hi, o, V0, k, kout, lambda, X, resid, n_found, stats);
        return slice_solve_impl(f, j, lo, hi, o, V0, k, lambda, X, resid, n_found, stats);
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_slice_solve: host allocation failed");
    }
}

extern "C" ss_status ss_dense_gram(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int32_t k1, const double *Y,
                                   int64_t ldy, int32_t k2, double *G) {
    if (!ctx) return SS_ERR_ARG;
    if (n < 0 || k1 < 1 || k2 < 1 || ldx < k1 || ldy < k2 || !G || (n > 0 && (!X || !Y)))
        return ctx->set_error(SS_ERR_ARG, "ss_dense_gram: bad argument");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (n == 0) {
        SS_CUDA_TRY(ctx, cudaMemsetAsync(G, 0, sizeof(double) * k1 * k2, ctx->stream));
        return SS_OK;
    }
    return gram_ld(ctx, X, ldx, n, k1, Y, ldy, k2, G);
}

extern "C" ss_status ss_dense_gemm(ss_ctx *ctx, const double *X, int64_t ldx, int64_t n, int32_t k1, const double *Q,
                                   int32_t k2, int32_t transq, double alpha, double beta, double *Y, int64_t ldy) {
    if (!ctx) return SS_ERR_ARG;
    if (n < 0 || k1 < 1 || k2 < 1 || ldx < k1 || ldy < k2 || !Q || (transq != 0 && transq != 1) ||
        (n > 0 && (!X || !Y)))
        return ctx->set_error(SS_ERR_ARG, "ss_dense_gemm: bad argument");
    if (n == 0) return SS_OK;
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return gemm_ld(ctx, X, ldx, n, k1, Q, k2, transq, alpha, beta, Y, ldy);
}

extern "C" ss_status ss_dos_estimate(ss_symbolic *s, const double *a_vals, const double *b_vals, int32_t steps,
                                     int32_t n_vec, const double *start, double *theta, double *zeta2,
                                     int32_t *m_run) {
    if (!s) return SS_ERR_ARG;
    ss_ctx *ctx = s->ctx;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "ss_dos_estimate: host-only context");
    if (!a_vals || !b_vals || !start || !theta || !zeta2 || !m_run || steps <= 0 || steps > 2048 || n_vec <= 0 ||
        256 % n_vec != 0)
        return ctx->set_error(SS_ERR_ARG, "ss_dos_estimate: bad argument (n_vec must divide 256)");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    try {
        ss_numeric *fb = nullptr;
        int rc = factor_spd_b(s, b_vals, &fb);
        if (rc != SS_OK) return rc;
        double *x0 = nullptr;
        rc = cudaMallocAsync((void **)&x0, sizeof(double) * s->n * n_vec, ctx->stream) == cudaSuccess ? SS_OK
             : ctx->set_error(SS_ERR_OOM, "ss_dos_estimate: device allocation failed");
        // start vectors of Lanczos on G^-1 A G^-T (B = G G^T) become x0 = G^-T y0 for the
        // equivalent B-orthonormal Lanczos on B^-1 A
        if (rc == SS_OK) rc = solve_half_backward(fb, 0, start, n_vec, x0);
        if (rc == SS_OK) rc = lanczos_impl(s, fb, a_vals, b_vals, steps, n_vec, x0, theta, zeta2, m_run);
        if (x0) cudaFreeAsync(x0, ctx->stream);
        ss_factor_destroy(fb);
        return rc;
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_dos_estimate: host allocation failed");
    }
}

extern "C" ss_status ss_dos_lanczos(ss_symbolic *s, const double *a_vals, const double *b_vals, int32_t steps,
                                    int32_t n_vec, const double *x0, double *theta, double *zeta2, int32_t *m_run) {
    if (!s) return SS_ERR_ARG;
    ss_ctx *ctx = s->ctx;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "ss_dos_lanczos: host-only context");
    if (!a_vals || !b_vals || !x0 || !theta || !zeta2 || !m_run || steps <= 0 || steps > 2048 || n_vec <= 0 ||
        256 % n_vec != 0)
        return ctx->set_error(SS_ERR_ARG, "ss_dos_lanczos: bad argument (n_vec must divide 256)");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    try {
        ss_numeric *fb = nullptr;
        int rc = factor_spd_b(s, b_vals, &fb);
        if (rc != SS_OK) return rc;
        rc = lanczos_impl(s, fb, a_vals, b_vals, steps, n_vec, x0, theta, zeta2, m_run);
        ss_factor_destroy(fb);
        return rc;
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_dos_lanczos: host allocation failed");
    }
}
