// In-slice eigensolver (Alg. 2: shift-invert subspace iteration, Cholesky-QR in the B
// inner product, Rayleigh-Ritz, residual norms) and the Lanczos density-of-states
// estimate (Section 3.1).  All arithmetic runs in the kernels of dense_kernels.cuh and
// the factor/solve kernels; this file sequences them on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dense_kernels.cuh"
#include "internal.h"

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

// G = X^T Y (k1 x k2)
int gram(ss_ctx *ctx, const double *X, int64_t n, int k1, const double *Y, int k2, double *G) {
    cudaStream_t st = ctx->stream;
    SS_CUDA_TRY(ctx, cudaMemsetAsync(G, 0, sizeof(double) * k1 * k2, st));
    const int64_t bxy = (int64_t)cdiv(k1, 32) * cdiv(k2, 32);
    int64_t nz = std::max<int64_t>(1, (4 * (int64_t)ctx->sm_count + bxy - 1) / bxy);
    nz = std::min<int64_t>(nz, std::max<int64_t>(1, n / 256));
    int64_t per = ((n + nz - 1) / nz + 31) / 32 * 32;
    nz = (n + per - 1) / per;
    ss_launch(ctx, SS_K_GRAM, ssd::k_gram, dim3(cdiv(k1, 32), cdiv(k2, 32), (unsigned)std::max<int64_t>(1, nz)), 256, 0, st, 
        n, X, k1, Y, k2, per, G);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

int gemm_tall(ss_ctx *ctx, const double *X, int64_t n, int k1, const double *Q, int k2, int transq, double *Y) {
    ss_launch(ctx, SS_K_GEMM, ssd::k_gemm_tall, dim3(cdiv(n, 64), cdiv(k2, 32)), 256, 0, ctx->stream, n, X, k1, Q, k2, transq, Y);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
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
int sym_eig(ss_ctx *ctx, double *H, int k, double *evals, double *Q, DevBuf &buf) {
    cudaStream_t st = ctx->stream;
    double *H2, *V, *V2;
    int *done;
    TRY_ALLOC(ctx, buf.get(&H2, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&V, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&V2, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&done, 1));
    const unsigned g = cdiv((int64_t)k * k, 256);
    ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, g, 256, 0, st, H, k);
    ss_launch(ctx, SS_K_JACOBI, ssd::k_set_identity, g, 256, 0, st, V, k);
    SS_CUDA_TRY(ctx, cudaMemsetAsync(done, 0, sizeof(int), st));
    const int kp = k + (k & 1);
    int hdone = 0;
    for (int sweep = 0; sweep < 30 && !hdone && k > 1; ++sweep) {
        for (int r = 0; r < kp - 1; ++r) {
            ss_launch(ctx, SS_K_JACOBI, ssd::k_jacobi_round, g, 256, 0, st, H, H2, V, V2, k, kp, r, 1e-18, done);
            std::swap(H, H2);
            std::swap(V, V2);
        }
        ss_launch(ctx, SS_K_JACOBI, ssd::k_jacobi_check, 1, 1024, 0, st, H, k, 1e-15, done);
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(&hdone, done, sizeof(int), cudaMemcpyDeviceToHost, st));
        SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    }
    ss_launch(ctx, SS_K_JACOBI, ssd::k_eig_sort, cdiv(k, 256), 256, 0, st, H, V, k, evals, Q);
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
        if ((rc = spmm_launch(s, f->b_vals, f->b_vals, nullptr, nullptr, V, k, Wk)) != SS_OK) return rc;
        if ((rc = gram(ctx, V, s->n, k, Wk, k, G)) != SS_OK) return rc;
        ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, cdiv((int64_t)k * k, 256), 256, 0, st, G, k);
        int hinfo = 0;
        for (int attempt = 0; attempt < 3; ++attempt) {
            if (attempt > 0) {
                // restore G from Wk (still B V) and shift it
                if ((rc = gram(ctx, V, s->n, k, Wk, k, G)) != SS_OK) return rc;
                ss_launch(ctx, SS_K_SMALL_DENSE, k_symmetrize, cdiv((int64_t)k * k, 256), 256, 0, st, G, k);
                const double rel = 11.0 * ((double)s->n * k + (double)k * (k + 1)) * 1.1102230246251565e-16 *
                                   (attempt == 1 ? 1.0 : 1e4);
                ss_launch(ctx, SS_K_SMALL_DENSE, k_add_shift_diag, 1, 256, 0, st, G, k, rel);
            }
            ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_chol_small, 1, 1024, 0, st, G, k, info);
            SS_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
            SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            if (hinfo == 0) break;
        }
        if (hinfo != 0)
            return ctx->set_error(SS_ERR_NOCONV, "Cholesky-QR: basis is numerically rank deficient");
        ss_launch(ctx, SS_K_SMALL_DENSE, ssd::k_trinv_lower, cdiv(k, 128), 128, 0, st, G, k, Rinv);
        if ((rc = gemm_tall(ctx, V, s->n, k, Rinv, k, 1, Wk)) != SS_OK) return rc;
        std::swap(V, Wk);
    }
    (void)buf;
    return SS_OK;
}

// Rayleigh-Ritz on B-orthonormal V: H = V^T A V = Q Theta Q^T, X = V Q, and the
// normalised residuals ||A x - theta B x|| / (||A||_1 ||x||).  V <- X.
int rayleigh_ritz(ss_numeric *f, double *&V, double *&Wk, double *T, int k, double *H, double *Q,
                  double *theta_d, double *resid_d, double *rr, double *xx, double *be, DevBuf &buf) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    int rc;
    if ((rc = spmm_launch(s, f->a_vals, f->a_vals, nullptr, nullptr, V, k, Wk)) != SS_OK) return rc;
    if ((rc = gram(ctx, V, s->n, k, Wk, k, H)) != SS_OK) return rc;
    if ((rc = sym_eig(ctx, H, k, theta_d, Q, buf)) != SS_OK) return rc;
    if ((rc = gemm_tall(ctx, V, s->n, k, Q, k, 0, Wk)) != SS_OK) return rc;
    std::swap(V, Wk);
    ss_launch(ctx, SS_K_MISC, ssd::k_neg_scale, cdiv(k, 256), 256, 0, st, k, theta_d, be);
    if ((rc = spmm_launch(s, f->a_vals, f->b_vals, nullptr, be, V, k, T)) != SS_OK) return rc;
    SS_CUDA_TRY(ctx, cudaMemsetAsync(rr, 0, sizeof(double) * 2 * k, st));
    const int64_t per = 2048;
    ss_launch(ctx, SS_K_MISC, ssd::k_col_sumsq, dim3(cdiv(k, 128), cdiv(s->n, per)), 128, 0, st, s->n, k, T, per, rr);
    ss_launch(ctx, SS_K_MISC, ssd::k_col_sumsq, dim3(cdiv(k, 128), cdiv(s->n, per)), 128, 0, st, s->n, k, V, per, xx);
    ss_launch(ctx, SS_K_MISC, ssd::k_resid_finish, cdiv(k, 256), 256, 0, st, k, rr, xx, f->norm_a1, resid_d);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

int slice_solve_impl(ss_numeric *f, int j, double lo, double hi, const ss_solve_opts &o, const double *V0, int k,
                     double *lambda, double *X, double *resid, int32_t *n_found, ss_probe_stats *stats) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = s->n;
    DevBuf buf(st);
    double *V, *Wk, *T, *G, *Rinv, *Q, *theta_d, *resid_d, *rr, *be;
    int *info;
    TRY_ALLOC(ctx, buf.get(&V, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&Wk, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&T, (size_t)n * k));
    TRY_ALLOC(ctx, buf.get(&G, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&Rinv, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&Q, (size_t)k * k));
    TRY_ALLOC(ctx, buf.get(&theta_d, (size_t)k));
    TRY_ALLOC(ctx, buf.get(&resid_d, (size_t)k));
    TRY_ALLOC(ctx, buf.get(&rr, (size_t)2 * k));
    TRY_ALLOC(ctx, buf.get(&be, (size_t)k));
    TRY_ALLOC(ctx, buf.get(&info, 1));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(V, V0, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, st));
    int rc;
    if ((rc = cholqr_b(f, V, Wk, k, G, Rinv, info, buf)) != SS_OK) return rc;
    std::vector<double> th(k), rs(k);
    int it = 0, refine_total = 0;
    bool conv = false;
    double maxr = 0.0;
    int nf = 0;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 200;
    const int every = o.check_every > 0 ? o.check_every : 1;
    const int refine = o.refine > 0 ? o.refine : 2;
    const double tol = o.tol > 0 ? o.tol : 1e-10;
    while (it < max_iter) {
        ++it;
        // V <- (A - sigma B)^-1 B V  (Alg. 2 step 3), then B-orthonormalise (step 4)
        if ((rc = spmm_launch(s, f->b_vals, f->b_vals, nullptr, nullptr, V, k, T)) != SS_OK) return rc;
        int done_ref = 0;
        if ((rc = solve_apply(f, j, T, k, V, refine, &done_ref)) != SS_OK) return rc;
        refine_total += done_ref;
        if ((rc = cholqr_b(f, V, Wk, k, G, Rinv, info, buf)) != SS_OK) return rc;
        if (it % every == 0 || it == max_iter) {
            if ((rc = rayleigh_ritz(f, V, Wk, T, k, G, Q, theta_d, resid_d, rr, rr + k, be, buf)) != SS_OK)
                return rc;
            SS_CUDA_TRY(ctx, cudaMemcpyAsync(th.data(), theta_d, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            SS_CUDA_TRY(ctx, cudaMemcpyAsync(rs.data(), resid_d, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
            SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            // a Ritz value in the window counts once its residual meets tol; unconverged
            // ones in the window may be spurious mixtures from the edge of the basis
            // (eigenvalues at equal distance on both sides of sigma), which validation by
            // inertia counts removes (Section 2.3), so with n_expect given the probe stops
            // as soon as n_expect of them have converged
            nf = 0;
            maxr = 0.0;
            int nin = 0;
            for (int i = 0; i < k; ++i) {
                if (th[i] > lo && th[i] <= hi) {
                    ++nin;
                    if (rs[i] <= tol) {
                        ++nf;
                        maxr = std::max(maxr, rs[i]);
                    }
                }
            }
            const bool done = o.n_expect > 0 ? (nf >= o.n_expect) : (nf == nin);
            if (done && it >= 2) { conv = true; break; }
        }
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

// B-orthonormal Lanczos on B^-1 A (Section 3.1) for n_vec start vectors at once.
int dos_impl(ss_symbolic *s, const double *a_vals, const double *b_vals, int steps, int nv, const double *start,
             double *theta, double *zeta2, int32_t *m_run) {
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t n = s->n;
    const double zero = 0.0;
    ss_numeric *fb = nullptr;
    // B = P L D L^T P^T: the same multifrontal LDL^T at sigma = 0 of the pencil (B, 0)
    int rc = ss_factor_create(s, b_vals, b_vals, &zero, 1, SS_FP64, &fb);
    if (rc != SS_OK && rc != SS_ERR_SINGULAR) return rc;
    struct Guard { ss_numeric *f; ~Guard() { ss_factor_destroy(f); } } guard{fb};
    int64_t neg = 0, zr = 0, pos = 0;
    ss_inertia(fb, 0, &neg, &zr, &pos, nullptr);
    if (neg != 0 || zr != 0 || rc == SS_ERR_SINGULAR)
        return ctx->set_error(SS_ERR_NOT_SPD, "ss_dos_estimate: B is not positive definite (inertia " +
                                                  std::to_string(neg) + "/" + std::to_string(zr) + "/" +
                                                  std::to_string(pos) + ")");
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
        !(lo < hi))
        return ctx->set_error(SS_ERR_ARG, "ss_slice_solve: bad argument");
    ss_solve_opts o{};
    if (opts) o = *opts;
    if (o.driver != SS_SUBSPACE) return ctx->set_error(SS_ERR_ARG, "ss_slice_solve: unsupported driver");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    try {
        return slice_solve_impl(f, j, lo, hi, o, V0, k, lambda, X, resid, n_found, stats);
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_slice_solve: host allocation failed");
    }
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
        return dos_impl(s, a_vals, b_vals, steps, n_vec, start, theta, zeta2, m_run);
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_dos_estimate: host allocation failed");
    }
}
