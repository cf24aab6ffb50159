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

#include "grid_sync.cuh"

namespace ssd {

// ---------------------------------------------------------------- Gram G += X^T Y
// block = 32 x 32 tile of G over one chunk of rows; 256 threads, 2 x 2 outputs each
__global__ void __launch_bounds__(256) k_gram(int64_t n, const double *__restrict__ X, int64_t ldx, int k1,
                                              const double *__restrict__ Y, int64_t ldy, int k2,
                                              int64_t rows_per, int sym, double *G) {
    __shared__ double Xs[32][33], Ys[32][33];
    // sym: G is symmetric (X^T M X-type products): tiles above the diagonal only, each
    // written to both triangles
    if (sym && blockIdx.x > blockIdx.y) return;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int64_t r_begin = blockIdx.z * rows_per;
    const int64_t r_end = min(n, r_begin + rows_per);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int64_t r0 = r_begin; r0 < r_end; r0 += 32) {
        for (int q = tid; q < 32 * 32; q += 256) {
            int rr = q >> 5, c = q & 31;
            int64_t r = r0 + rr;
            Xs[rr][c] = (r < r_end && i0 + c < k1) ? X[r * ldx + i0 + c] : 0.0;
            Ys[rr][c] = (r < r_end && j0 + c < k2) ? Y[r * ldy + j0 + c] : 0.0;
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
            if (i < k1 && j < k2) {
                atomicAdd(&G[(int64_t)i * k2 + j], acc[a][b]);
                if (sym && blockIdx.x != blockIdx.y) atomicAdd(&G[(int64_t)j * k2 + i], acc[a][b]);
            }
        }
}

// ---------------------------------------------------------------- Y = beta Y + alpha X Q  (or X Q^T)
// block = 64 rows x 32 columns of Y; k1 chunks of 32 through shared memory.  Q is k1 x k2
// (ldq = k2) or, transposed, k2 x k1 (ldq = k1).  beta = 0 does not read Y.  tri: the
// effective Q (k1 x k2) is upper triangular (a lower-triangular Q used transposed), so
// chunks below column block j0's diagonal are skipped.
__global__ void __launch_bounds__(256) k_gemm_tall(int64_t n, const double *__restrict__ X, int64_t ldx, int k1,
                                                   const double *__restrict__ Q, int k2, int transq,
                                                   double alpha, double beta, double *__restrict__ Y,
                                                   int64_t ldy, int tri) {
    __shared__ double Xs[64][33], Qs[32][33];
    const int64_t r0 = blockIdx.x * 64ll;
    const int j0 = blockIdx.y * 32;
    const int tid = threadIdx.x, tc = tid & 31, tr = tid >> 5;   // column tc, rows tr + 8 a
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int t_end = tri ? min(k1, j0 + 32) : k1;
    for (int t0 = 0; t0 < t_end; t0 += 32) {
        for (int q = tid; q < 64 * 32; q += 256) {
            int rr = q >> 5, c = q & 31;
            int64_t r = r0 + rr;
            Xs[rr][c] = (r < n && t0 + c < k1) ? X[r * ldx + t0 + c] : 0.0;
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
            if (r < n) {
                double *y = Y + r * ldy + j0 + tc;
                *y = (beta != 0.0 ? beta * *y : 0.0) + alpha * acc[a];
            }
        }
}

// ---------------------------------------------------------------- small Cholesky
constexpr int CH_NB = 32;

// Multi-block blocked Cholesky, one 32-column panel per three launches:
//   k_chol_diag  factors the panel's diagonal block (one warp, shared memory);
//   k_chol_trsm  solves the rows below against it (one warp per row);
//   k_chol_syrk  updates the trailing lower triangle, one 32 x 32 tile per block.
// info[0] != 0 (a non-positive pivot) makes every later launch return at once.
__global__ void __launch_bounds__(32) k_chol_diag(double *G, int k, int j0, int *info) {
    __shared__ double Dg[CH_NB][CH_NB + 1];
    if (info[0]) return;
    const int lane = threadIdx.x, w = min(CH_NB, k - j0);
    for (int q = lane; q < w * w; q += 32) {
        int i = q / w, c = q % w;
        Dg[i][c] = (c <= i) ? G[(int64_t)(j0 + i) * k + j0 + c] : 0.0;
    }
    __syncwarp();
    int bad = 0;
    for (int c = 0; c < w; ++c) {
        double d = Dg[c][c];
        if (!(d > 0.0)) { if (!bad) bad = j0 + c + 1; d = 1.0; }
        const double sd = sqrt(d);
        __syncwarp();
        if (lane == 0) Dg[c][c] = sd;
        __syncwarp();
        const double inv = 1.0 / sd;
        for (int i = c + 1 + lane; i < w; i += 32) Dg[i][c] *= inv;
        __syncwarp();
        for (int i = c + 1 + lane; i < w; i += 32)
            for (int l = c + 1; l <= i; ++l) Dg[i][l] -= Dg[i][c] * Dg[l][c];
        __syncwarp();
    }
    for (int q = lane; q < w * w; q += 32) {
        int i = q / w, c = q % w;
        if (c <= i) G[(int64_t)(j0 + i) * k + j0 + c] = Dg[i][c];
    }
    if (lane == 0 && bad) info[0] = bad;
}

__global__ void __launch_bounds__(256) k_chol_trsm(double *G, int k, int j0, const int *info) {
    __shared__ double Dg[CH_NB][CH_NB + 1];
    if (info[0]) return;
    const int w = min(CH_NB, k - j0), lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < w * w; q += 256) {
        int i = q / w, c = q % w;
        Dg[i][c] = (c <= i) ? G[(int64_t)(j0 + i) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    const int i = j0 + w + blockIdx.x * 8 + wid;
    if (i >= k) return;
    double x = (lane < w) ? G[(int64_t)i * k + j0 + lane] : 0.0;
    for (int c = 0; c < w; ++c) {
        double xc = __shfl_sync(0xffffffffu, x, c) / Dg[c][c];
        if (lane == c) x = xc;
        if (lane > c && lane < w) x -= xc * Dg[lane][c];
    }
    if (lane < w) G[(int64_t)i * k + j0 + lane] = x;
}

__global__ void __launch_bounds__(256) k_chol_syrk(double *G, int k, int j0, const int *info) {
    __shared__ double Pi[CH_NB][CH_NB + 1], Pl[CH_NB][CH_NB + 1];
    if (info[0]) return;
    const int w = min(CH_NB, k - j0), base = j0 + w;
    int q = blockIdx.x, bi = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
    while (bi * (bi + 1) / 2 > q) --bi;
    const int bj = q - bi * (bi + 1) / 2;
    const int i0 = base + 32 * bi, l0 = base + 32 * bj;
    for (int e = threadIdx.x; e < 32 * CH_NB; e += 256) {
        int r = e / CH_NB, c = e % CH_NB;
        Pi[r][c] = (i0 + r < k && c < w) ? G[(int64_t)(i0 + r) * k + j0 + c] : 0.0;
        Pl[r][c] = (l0 + r < k && c < w) ? G[(int64_t)(l0 + r) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int r = e >> 5, c = e & 31;
        const int i = i0 + r, l = l0 + c;
        if (i >= k || l > i) continue;
        double acc = 0.0;
#pragma unroll 8
        for (int t = 0; t < CH_NB; ++t) acc += Pi[r][t] * Pl[c][t];
        G[(int64_t)i * k + l] -= acc;
    }
}

__global__ void k_zero_upper(double *G, int k) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < (int64_t)k * k && q % k > q / k) G[q] = 0.0;
}

// Rinv = R^-1 for lower-triangular R (k x k row-major).  Column blocks of R^-1 are
// independent: block b solves R X = E for columns [32 b, 32 b + 32) by forward
// substitution over the rows; per row the dot product is split across the 8 warps.
__global__ void __launch_bounds__(256) k_trinv_lower(const double *__restrict__ R, int k, double *__restrict__ Rinv) {
    __shared__ double part[8][33];
    const int c0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int c = c0 + lane;
    for (int i = 0; i < k; ++i) {
        const double *ri = R + (int64_t)i * k;
        double acc = 0.0;
        if (c < k)      // Rinv[t][c] = 0 for t < c, so every lane can walk the same t
            for (int t = c0 + wid; t < i; t += 8) acc += ri[t] * Rinv[(int64_t)t * k + c];
        part[wid][lane] = acc;
        __syncthreads();
        if (wid == 0 && c < k) {
            double sum = 0.0;
            for (int w = 0; w < 8; ++w) sum += part[w][lane];
            double v = 0.0;
            if (c <= i) v = ((c == i ? 1.0 : 0.0) - sum) / ri[i];
            Rinv[(int64_t)i * k + c] = v;
        }
        __syncthreads();
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

// The whole eigensolve in one block: every round computes the k/2 rotations from the
// current H, then each thread rotates whole 2 x 2 blocks {p, q} x {p', q'} of H in place
// (H' = J^T H J touches only the rows/columns of the pairs) and row pairs of V (V' = V J).
// Sweeps stop once off(H)^2 <= tol^2 ||H||_F^2 or after max_sweeps.  H and V are k x k
// row-major in global memory (V must hold the identity or a previous rotation on entry).
// Shared memory: 3 * (kp / 2) values (pair, c, s).
__global__ void __launch_bounds__(1024) k_jacobi_block(double *H, double *V, int k, double thr, double tol,
                                                       int max_sweeps, int *sweeps_done) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kp = k + (k & 1);
    const int np = kp / 2;
    int *pp = reinterpret_cast<int *>(smem_raw);             // p of pair t (p < q)
    int *pq = pp + np;                                        // q of pair t
    double *pc = reinterpret_cast<double *>(pq + np + (np & 1));
    double *ps = pc + np;
    __shared__ double red_off[32], red_all[32];
    __shared__ int s_stop;
    const int tid = threadIdx.x, nt = blockDim.x;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence test
        double off = 0.0, all = 0.0;
        for (int64_t q = tid; q < (int64_t)k * k; q += nt) {
            double v = H[q] * H[q];
            all += v;
            if (q / k != q % k) off += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_down_sync(0xffffffffu, off, o);
            all += __shfl_down_sync(0xffffffffu, all, o);
        }
        if ((tid & 31) == 0) { red_off[tid >> 5] = off; red_all[tid >> 5] = all; }
        __syncthreads();
        if (tid == 0) {
            double o2 = 0.0, a2 = 0.0;
            for (int w = 0; w < (nt >> 5); ++w) { o2 += red_off[w]; a2 += red_all[w]; }
            s_stop = (o2 <= tol * tol * a2) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        for (int r = 0; r < kp - 1; ++r) {
            // rotations of this round
            for (int t = tid; t < np; t += nt) {
                int i = (t == 0) ? kp - 1 : (r + t) % (kp - 1);
                int y = jac_partner(i, r, kp);
                int p = min(i, y), q = max(i, y);
                double c = 1.0, sn = 0.0;
                if (q < k) {
                    const double hpq = H[(int64_t)p * k + q];
                    const double hpp = H[(int64_t)p * k + p], hqq = H[(int64_t)q * k + q];
                    if (hpq != 0.0 && fabs(hpq) > thr * sqrt(fabs(hpp * hqq))) {
                        const double th = (hqq - hpp) / (2.0 * hpq);
                        const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                pp[t] = p; pq[t] = q; pc[t] = c; ps[t] = sn;
            }
            __syncthreads();
            // H <- J^T H J on 2 x 2 blocks (pair a rows) x (pair b columns)
            for (int64_t e = tid; e < (int64_t)np * np; e += nt) {
                const int ta = (int)(e / np), tb = (int)(e % np);
                const int p1 = pp[ta], q1 = pq[ta], p2 = pp[tb], q2 = pq[tb];
                const double c1 = pc[ta], s1 = ps[ta], c2 = pc[tb], s2 = ps[tb];
                if (s1 == 0.0 && s2 == 0.0) continue;
                const bool rq = q1 < k, cq = q2 < k;
                double h11 = H[(int64_t)p1 * k + p2];
                double h12 = cq ? H[(int64_t)p1 * k + q2] : 0.0;
                double h21 = rq ? H[(int64_t)q1 * k + p2] : 0.0;
                double h22 = (rq && cq) ? H[(int64_t)q1 * k + q2] : 0.0;
                // columns: new_p = c h_p - s h_q, new_q = s h_p + c h_q
                double a11 = c2 * h11 - s2 * h12, a12 = s2 * h11 + c2 * h12;
                double a21 = c2 * h21 - s2 * h22, a22 = s2 * h21 + c2 * h22;
                // rows
                double b11 = c1 * a11 - s1 * a21, b21 = s1 * a11 + c1 * a21;
                double b12 = c1 * a12 - s1 * a22, b22 = s1 * a12 + c1 * a22;
                if (ta == tb && s1 != 0.0) { b12 = 0.0; b21 = 0.0; }   // the annihilated pair
                H[(int64_t)p1 * k + p2] = b11;
                if (cq) H[(int64_t)p1 * k + q2] = b12;
                if (rq) H[(int64_t)q1 * k + p2] = b21;
                if (rq && cq) H[(int64_t)q1 * k + q2] = b22;
            }
            // V <- V J on row pairs (column pair tb)
            for (int64_t e = tid; e < (int64_t)k * np; e += nt) {
                const int row = (int)(e / np), tb = (int)(e % np);
                const double s2 = ps[tb];
                if (s2 == 0.0) continue;
                const int p2 = pp[tb], q2 = pq[tb];
                const double c2 = pc[tb];
                double *vr = V + (int64_t)row * k;
                const double vp = vr[p2], vq = vr[q2];
                vr[p2] = c2 * vp - s2 * vq;
                vr[q2] = s2 * vp + c2 * vq;
            }
            __syncthreads();
        }
    }
    if (tid == 0 && sweeps_done) *sweeps_done = sweep;
}

// ---------------------------------------------------------------- grid-wide Jacobi
using ::GridBar;
using ::grid_barrier;

// The same parallel-ordered Jacobi as k_jacobi_block, spread over a cooperative grid with
// one grid barrier per round: H is double-buffered (round r reads Ha and writes every
// entry of Hb, then the two swap), so each block can compute all of the round's rotations
// itself from Ha into shared memory (np x 24 bytes of dynamic shared memory) while other
// blocks already write Hb.  acc: 2 * max_sweeps doubles (zeroed) for the per-sweep
// off-diagonal / total norms.  On return the matrix is in H (copied back from the scratch
// buffer H2 when the last round left it there).
__global__ void __launch_bounds__(256) k_jacobi_grid(double *H, double *H2, double *V, int k, double thr, double tol,
                                                     int max_sweeps, double *acc, GridBar *bar, long long limit,
                                                     int *sweeps_done) {
    extern __shared__ __align__(16) unsigned char jac_smem[];
    const int kp = k + (k & 1);
    const int np = kp / 2;
    double2 *s_cs = reinterpret_cast<double2 *>(jac_smem);
    int2 *s_pq = reinterpret_cast<int2 *>(jac_smem + sizeof(double2) * np);
    const unsigned int nb = gridDim.x;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)nb * blockDim.x;
    __shared__ double red_off[8], red_all[8];
    double *Ha = H, *Hb = H2;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, all = 0.0;
        for (int64_t q = gtid; q < (int64_t)k * k; q += gthreads) {
            double v = Ha[q] * Ha[q];
            all += v;
            if (q / k != q % k) off += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_down_sync(0xffffffffu, off, o);
            all += __shfl_down_sync(0xffffffffu, all, o);
        }
        if ((threadIdx.x & 31) == 0) { red_off[threadIdx.x >> 5] = off; red_all[threadIdx.x >> 5] = all; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double o2 = 0.0, a2 = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { o2 += red_off[w]; a2 += red_all[w]; }
            atomicAdd(&acc[2 * sweep], o2);
            atomicAdd(&acc[2 * sweep + 1], a2);
        }
        if (!grid_barrier(bar, nb, limit)) return;
        const double o2 = *(volatile double *)&acc[2 * sweep], a2 = *(volatile double *)&acc[2 * sweep + 1];
        if (o2 <= tol * tol * a2) break;
        for (int r = 0; r < kp - 1; ++r) {
            // the round's rotations, from Ha, by every block
            for (int t = threadIdx.x; t < np; t += blockDim.x) {
                int i = (t == 0) ? kp - 1 : (int)((r + t) % (kp - 1));
                int y = jac_partner(i, r, kp);
                int p = min(i, y), q = max(i, y);
                double c = 1.0, sn = 0.0;
                if (q < k) {
                    const double hpq = Ha[(int64_t)p * k + q];
                    const double hpp = Ha[(int64_t)p * k + p], hqq = Ha[(int64_t)q * k + q];
                    if (hpq != 0.0 && fabs(hpq) > thr * sqrt(fabs(hpp * hqq))) {
                        const double th = (hqq - hpp) / (2.0 * hpq);
                        const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                s_pq[t] = make_int2(p, q);
                s_cs[t] = make_double2(c, sn);
            }
            __syncthreads();
            // Hb = J^T Ha J, every 2 x 2 block written (copied where both rotations are trivial)
            for (int64_t e = gtid; e < (int64_t)np * np; e += gthreads) {
                const int ta = (int)(e / np), tb = (int)(e % np);
                const double2 r1 = s_cs[ta], r2 = s_cs[tb];
                const double c1 = r1.x, s1 = r1.y, c2 = r2.x, s2 = r2.y;
                const int2 a1 = s_pq[ta], a2p = s_pq[tb];
                const int p1 = a1.x, q1 = a1.y, p2 = a2p.x, q2 = a2p.y;
                const bool rq = q1 < k, cq = q2 < k;
                const double h11 = Ha[(int64_t)p1 * k + p2];
                const double h12 = cq ? Ha[(int64_t)p1 * k + q2] : 0.0;
                const double h21 = rq ? Ha[(int64_t)q1 * k + p2] : 0.0;
                const double h22 = (rq && cq) ? Ha[(int64_t)q1 * k + q2] : 0.0;
                double b11 = h11, b12 = h12, b21 = h21, b22 = h22;
                if (s1 != 0.0 || s2 != 0.0) {
                    const double x11 = c2 * h11 - s2 * h12, x12 = s2 * h11 + c2 * h12;
                    const double x21 = c2 * h21 - s2 * h22, x22 = s2 * h21 + c2 * h22;
                    b11 = c1 * x11 - s1 * x21;
                    b21 = s1 * x11 + c1 * x21;
                    b12 = c1 * x12 - s1 * x22;
                    b22 = s1 * x12 + c1 * x22;
                    if (ta == tb && s1 != 0.0) { b12 = 0.0; b21 = 0.0; }
                }
                Hb[(int64_t)p1 * k + p2] = b11;
                if (cq) Hb[(int64_t)p1 * k + q2] = b12;
                if (rq) Hb[(int64_t)q1 * k + p2] = b21;
                if (rq && cq) Hb[(int64_t)q1 * k + q2] = b22;
            }
            // V = V J (each entry updated by exactly one thread per round)
            for (int64_t e = gtid; e < (int64_t)k * np; e += gthreads) {
                const int row = (int)(e / np), tb = (int)(e % np);
                const double2 r2 = s_cs[tb];
                if (r2.y == 0.0) continue;
                const int2 a2p = s_pq[tb];
                double *vr = V + (int64_t)row * k;
                const double vp = vr[a2p.x], vq = vr[a2p.y];
                vr[a2p.x] = r2.x * vp - r2.y * vq;
                vr[a2p.y] = r2.y * vp + r2.x * vq;
            }
            if (!grid_barrier(bar, nb, limit)) return;
            double *t = Ha;
            Ha = Hb;
            Hb = t;
        }
    }
    if (Ha != H)
        for (int64_t q = gtid; q < (int64_t)k * k; q += gthreads) H[q] = Ha[q];
    if (gtid == 0 && sweeps_done) *sweeps_done = sweep;
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

// copy an n x k block between leading dimensions
__global__ void k_copy_cols(int64_t n, int k, const double *__restrict__ X, int64_t ldx, double *__restrict__ Y,
                            int64_t ldy) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * k) return;
    const int64_t r = q / k;
    const int c = (int)(q - r * k);
    Y[r * ldy + c] = X[r * ldx + c];
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

// out[c] += sum_r (AX[r][c] - theta[c] BX[r][c])^2  (residual column norms, squared)
__global__ void k_resid_sumsq(int64_t n, int k, const double *__restrict__ AX, const double *__restrict__ BX,
                              const double *__restrict__ theta, int64_t rows_per, double *out) {
    const int64_t r0 = blockIdx.y * rows_per, r1 = min(n, r0 + rows_per);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        const double th = theta[c];
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r) {
            double v = AX[r * k + c] - th * BX[r * k + c];
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
