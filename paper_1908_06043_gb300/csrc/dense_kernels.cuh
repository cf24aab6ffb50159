// Dense helper kernels of the in-slice solver and the DOS sweeps (FP64).
//   Gram        G = X^T Y (Cholesky-QR Gram matrix V^T B V, projected V^T A V)
//   GEMM        Y = X Q (tall-skinny times small square: V R^-T, V Q)
//   Cholesky    G = R R^T of a small SPD matrix; R^-1
//   Jacobi      eigenpairs of a small symmetric matrix by parallel-ordered cyclic
//               Jacobi (one launch per round of k/2 disjoint rotations)
//   Lanczos     batched dot products / updates for full re-orthogonalisation
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ssd {

// ---------------------------------------------------------------- Gram G += X^T Y
// block = 32 x 32 tile of G over one chunk of rows; 256 threads, 2 x 2 outputs each
__global__ void __launch_bounds__(256) k_gram(int64_t n, const double *__restrict__ X, int k1,
                                              const double *__restrict__ Y, int k2, int64_t rows_per,
                                              double *G) {
    __shared__ double Xs[32][33], Ys[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int64_t r_begin = blockIdx.z * rows_per;
    const int64_t r_end = min(n, r_begin + rows_per);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int64_t r0 = r_begin; r0 < r_end; r0 += 32) {
        for (int q = tid; q < 32 * 32; q += 256) {
            int rr = q >> 5, c = q & 31;
            int64_t r = r0 + rr;
            Xs[rr][c] = (r < r_end && i0 + c < k1) ? X[r * k1 + i0 + c] : 0.0;
            Ys[rr][c] = (r < r_end && j0 + c < k2) ? Y[r * k2 + j0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
            double x0 = Xs[rr][tx], x1 = Xs[rr][tx + 16];
            double y0 = Ys[rr][ty], y1 = Ys[rr][ty + 16];
            acc[0][0] += x0 * y0; acc[0][1] += x0 * y1;
            acc[1][0] += x1 * y0; acc[1][1] += x1 * y1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
            if (i < k1 && j < k2) atomicAdd(&G[(int64_t)i * k2 + j], acc[a][b]);
        }
}

// ---------------------------------------------------------------- Y = X Q  (or X Q^T)
// block = 64 rows x 32 columns of Y; k1 chunks of 32 through shared memory
__global__ void __launch_bounds__(256) k_gemm_tall(int64_t n, const double *__restrict__ X, int k1,
                                                   const double *__restrict__ Q, int k2, int transq,
                                                   double *__restrict__ Y) {
    __shared__ double Xs[64][33], Qs[32][33];
    const int64_t r0 = blockIdx.x * 64ll;
    const int j0 = blockIdx.y * 32;
    const int tid = threadIdx.x, tc = tid & 31, tr = tid >> 5;   // column tc, rows tr + 8 a
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t0 = 0; t0 < k1; t0 += 32) {
        for (int q = tid; q < 64 * 32; q += 256) {
            int rr = q >> 5, c = q & 31;
            int64_t r = r0 + rr;
            Xs[rr][c] = (r < n && t0 + c < k1) ? X[r * k1 + t0 + c] : 0.0;
        }
        for (int q = tid; q < 32 * 32; q += 256) {
            int t = q >> 5, c = q & 31;
            double v = 0.0;
            if (t0 + t < k1 && j0 + c < k2)
                v = transq ? Q[(int64_t)(j0 + c) * k1 + t0 + t] : Q[(int64_t)(t0 + t) * k2 + j0 + c];
            Qs[t][c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 32; ++t) {
            double qv = Qs[t][tc];
#pragma unroll
            for (int a = 0; a < 8; ++a) acc[a] += Xs[tr + 8 * a][t] * qv;
        }
        __syncthreads();
    }
    if (j0 + tc < k2)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            int64_t r = r0 + tr + 8 * a;
            if (r < n) Y[r * k2 + j0 + tc] = acc[a];
        }
}

// ---------------------------------------------------------------- small Cholesky
// G (k x k, row-major, symmetric) -> lower R with G = R R^T, upper part zeroed.
// info[0] = 0 ok, j+1 if the j-th pivot was not positive.  One block.
__global__ void __launch_bounds__(1024) k_chol_small(double *G, int k, int *info) {
    __shared__ double s_d;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            double d = G[(int64_t)j * k + j];
            if (!(d > 0.0)) { s_bad = j + 1; d = 1.0; }
            s_d = sqrt(d);
            G[(int64_t)j * k + j] = s_d;
        }
        __syncthreads();
        if (s_bad) break;
        const double inv = 1.0 / s_d;
        for (int i = j + 1 + tid; i < k; i += nt) G[(int64_t)i * k + j] *= inv;
        __syncthreads();
        const int rem = k - j - 1;
        const int64_t tot = (int64_t)rem * (rem + 1) / 2;
        for (int64_t q = tid; q < tot; q += nt) {
            // (i, l) with j < l <= i, enumerated row by row
            int ii = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
            while ((int64_t)(ii + 1) * (ii + 2) / 2 <= q) ++ii;
            while ((int64_t)ii * (ii + 1) / 2 > q) --ii;
            int ll = (int)(q - (int64_t)ii * (ii + 1) / 2);
            int i = j + 1 + ii, l = j + 1 + ll;
            G[(int64_t)i * k + l] -= G[(int64_t)i * k + j] * G[(int64_t)l * k + j];
        }
        __syncthreads();
    }
    if (tid == 0) info[0] = s_bad;
    __syncthreads();
    for (int64_t q = tid; q < (int64_t)k * k; q += nt) {
        int i = (int)(q / k), l = (int)(q % k);
        if (l > i) G[q] = 0.0;
    }
}

// Rinv = R^-1 for lower-triangular R (k x k row-major); one thread per column.
__global__ void k_trinv_lower(const double *__restrict__ R, int k, double *__restrict__ Rinv) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
        for (int i = 0; i < j; ++i) Rinv[(int64_t)i * k + j] = 0.0;
        Rinv[(int64_t)j * k + j] = 1.0 / R[(int64_t)j * k + j];
        for (int i = j + 1; i < k; ++i) {
            double acc = 0.0;
            for (int t = j; t < i; ++t) acc -= R[(int64_t)i * k + t] * Rinv[(int64_t)t * k + j];
            Rinv[(int64_t)i * k + j] = acc / R[(int64_t)i * k + i];
        }
    }
}

// ---------------------------------------------------------------- Jacobi eigensolver
// Round r of a sweep pairs index i with partner(i) (circle method over kp = k rounded up
// to even; index kp-1 is a dummy when k is odd).  Every pair (p, q), p < q, is rotated
// by the classical Jacobi angle that annihilates H[p][q]:
//   theta = (H_qq - H_pp) / (2 H_pq), t = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
//   c = 1 / sqrt(t^2 + 1), s = t c;  H' = J^T H J, V' = V J.
__device__ __forceinline__ int jac_partner(int i, int r, int kp) {
    const int m = kp - 1;
    if (i == m) return r;
    if (i == r) return m;
    int p = (2 * r - i) % m;
    if (p < 0) p += m;
    return p;
}

__device__ __forceinline__ void jac_coeffs(const double *H, int k, int kp, int r, int i, double thr,
                                           double &al, double &be, int &y) {
    y = jac_partner(i, r, kp);
    al = 1.0;
    be = 0.0;
    if (y >= k || i >= k) { y = i; return; }
    const int p = min(i, y), q = max(i, y);
    const double hpq = H[(int64_t)p * k + q];
    const double hpp = H[(int64_t)p * k + p], hqq = H[(int64_t)q * k + q];
    if (fabs(hpq) <= thr * sqrt(fabs(hpp * hqq)) || hpq == 0.0) { y = i; return; }
    const double th = (hqq - hpp) / (2.0 * hpq);
    const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
    const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
    al = c;
    be = (i == p) ? -s : s;
}

__global__ void k_jacobi_round(const double *__restrict__ H, double *__restrict__ H2,
                               const double *__restrict__ V, double *__restrict__ V2, int k, int kp,
                               int r, double thr, const int *__restrict__ done) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)k * k) return;
    if (*done) {                       // converged: copy through so the ping-pong stays valid
        H2[q] = H[q];
        V2[q] = V[q];
        return;
    }
    const int i = (int)(q / k), j = (int)(q % k);
    double ai, bi, aj, bj;
    int yi, yj;
    jac_coeffs(H, k, kp, r, i, thr, ai, bi, yi);
    jac_coeffs(H, k, kp, r, j, thr, aj, bj, yj);
    double h = ai * aj * H[(int64_t)i * k + j];
    if (bj != 0.0) h += ai * bj * H[(int64_t)i * k + yj];
    if (bi != 0.0) h += bi * aj * H[(int64_t)yi * k + j];
    if (bi != 0.0 && bj != 0.0) h += bi * bj * H[(int64_t)yi * k + yj];
    if (i != j && ((i == yj) || (j == yi)) && bi != 0.0) h = 0.0;     // annihilated pair
    H2[q] = h;
    // V' = V J: column j mixes with its partner
    double v = aj * V[(int64_t)i * k + j];
    if (bj != 0.0) v += bj * V[(int64_t)i * k + yj];
    V2[q] = v;
}

// sets *done when off(H)^2 <= tol^2 * ||H||_F^2 (one block)
__global__ void k_jacobi_check(const double *__restrict__ H, int k, double tol, int *done) {
    __shared__ double s_off[32], s_all[32];
    double off = 0.0, all = 0.0;
    for (int64_t q = threadIdx.x; q < (int64_t)k * k; q += blockDim.x) {
        double v = H[q] * H[q];
        all += v;
        if (q / k != q % k) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_down_sync(0xffffffffu, off, o);
        all += __shfl_down_sync(0xffffffffu, all, o);
    }
    if ((threadIdx.x & 31) == 0) { s_off[threadIdx.x >> 5] = off; s_all[threadIdx.x >> 5] = all; }
    __syncthreads();
    if (threadIdx.x == 0) {
        off = 0; all = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { off += s_off[w]; all += s_all[w]; }
        if (off <= tol * tol * all) *done = 1;
    }
}

// ascending eigenvalues with their eigenvector columns: rank by (value, index)
__global__ void k_eig_sort(const double *__restrict__ H, const double *__restrict__ V, int k,
                           double *__restrict__ evals, double *__restrict__ Q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const double li = H[(int64_t)i * k + i];
    int rank = 0;
    for (int j = 0; j < k; ++j) {
        double lj = H[(int64_t)j * k + j];
        if (lj < li || (lj == li && j < i)) ++rank;
    }
    evals[rank] = li;
    for (int r = 0; r < k; ++r) Q[(int64_t)r * k + rank] = V[(int64_t)r * k + i];
}

__global__ void k_set_identity(double *V, int k) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < (int64_t)k * k) V[q] = (q / k == q % k) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------- column reductions
// out[c] += sum_r X[r][c] * Y[r][c]
__global__ void k_col_dot(int64_t n, int k, const double *__restrict__ X, const double *__restrict__ Y,
                          double *out) {
    // requires 256 % k == 0 so that each thread keeps one column
    __shared__ double s[256];
    const int tid = threadIdx.x;
    double acc = 0.0;
    const int64_t tot = n * k;
    for (int64_t q = blockIdx.x * 256ll + tid; q < tot; q += (int64_t)gridDim.x * 256)
        acc += X[q] * Y[q];
    s[tid] = acc;
    __syncthreads();
    if (tid < k) {
        double v = 0.0;
        for (int t = tid; t < 256; t += k) v += s[t];
        atomicAdd(&out[tid], v);
    }
}

// out[c] += sum_r X[r][c]^2 for any k (block per row chunk)
__global__ void k_col_sumsq(int64_t n, int k, const double *__restrict__ X, int64_t rows_per,
                            double *out) {
    const int64_t r0 = blockIdx.y * rows_per, r1 = min(n, r0 + rows_per);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r) {
            double v = X[r * k + c];
            acc += v * v;
        }
        atomicAdd(&out[c], acc);
    }
}

// resid[c] = sqrt(rr[c]) / (normA * sqrt(xx[c]))
__global__ void k_resid_finish(int k, const double *__restrict__ rr, const double *__restrict__ xx,
                               double normA, double *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < k) out[c] = sqrt(rr[c]) / (normA * sqrt(xx[c]));
}

__global__ void k_neg_scale(int k, const double *__restrict__ x, double *__restrict__ y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < k) y[c] = -x[c];
}

// ---------------------------------------------------------------- Lanczos helpers
// h[i][c] = sum_r Q_i[r][c] w[r][c], i < j; grid (j, chunks); 256 % nv == 0
__global__ void k_lz_dots(const double *__restrict__ Qb, int64_t n, int nv, int j,
                          const double *__restrict__ w, int64_t per, double *h) {
    __shared__ double s[256];
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t tot = n * nv;
    const int64_t e0 = blockIdx.y * per, e1 = min(tot, e0 + per);
    const double *q = Qb + (int64_t)i * tot;
    double acc = 0.0;
    for (int64_t e = e0 + tid; e < e1; e += 256) acc += q[e] * w[e];
    s[tid] = acc;
    __syncthreads();
    if (tid < nv) {
        double v = 0.0;
        for (int t = tid; t < 256; t += nv) v += s[t];
        atomicAdd(&h[(int64_t)i * nv + tid], v);
    }
}

// w[r][c] -= sum_{i<j} Q_i[r][c] h[i][c]
__global__ void k_lz_sub(const double *__restrict__ Qb, int64_t n, int nv, int j,
                         const double *__restrict__ h, double *w) {
    const int64_t tot = n * nv;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const int c = (int)(e % nv);
    double acc = w[e];
    for (int i = 0; i < j; ++i) acc -= Qb[(int64_t)i * tot + e] * h[(int64_t)i * nv + c];
    w[e] = acc;
}

// w -= alpha_c q + beta_c q_prev (beta from the previous step, may be null)
__global__ void k_lz_three_term(int64_t n, int nv, const double *__restrict__ q,
                                const double *__restrict__ qp, const double *__restrict__ alpha,
                                const double *__restrict__ beta_prev, double *w) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * nv) return;
    const int c = (int)(e % nv);
    double v = w[e] - alpha[c] * q[e];
    if (beta_prev) v -= beta_prev[c] * qp[e];
    w[e] = v;
}

// q_next = w / beta (0 where beta is tiny)
__global__ void k_lz_normalize(int64_t n, int nv, const double *__restrict__ w,
                               const double *__restrict__ nrm2, double *__restrict__ beta,
                               double *__restrict__ qn) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nv) beta[e] = sqrt(nrm2[e]);
    if (e >= n * nv) return;
    const int c = (int)(e % nv);
    const double b = sqrt(nrm2[c]);
    qn[e] = b > 0.0 ? w[e] / b : 0.0;
}

// dense tridiagonal matrix of run c from alpha[j*nv+c], beta[j*nv+c]
__global__ void k_lz_tridiag(const double *__restrict__ alpha, const double *__restrict__ beta,
                             int nv, int c, int m, double *T) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)m * m) return;
    const int i = (int)(q / m), j = (int)(q % m);
    double v = 0.0;
    if (i == j) v = alpha[(int64_t)i * nv + c];
    else if (j == i + 1) v = beta[(int64_t)i * nv + c];
    else if (i == j + 1) v = beta[(int64_t)j * nv + c];
    T[q] = v;
}

}  // namespace ssd
