// Sparse kernels over the CSR pattern of A union B (FP64).
//   SpMM   Y = (alpha_j A + beta_j B) X with row-major blocks: the SpMV sweeps of the DOS
//          estimate (Section 3.1), B V of Alg. 2 step 3, and the residual A X - B X Lambda
//          that follows Alg. 2.
//   SDDMM  band-energy gradient sampled on the stored pattern.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sss {

// ---------------------------------------------------------------- SpMM
// one warp per row, lanes over right-hand-side columns (k >= 16)
__global__ void k_spmm_cols(int64_t n, const int64_t *__restrict__ rowptr,
                            const int32_t *__restrict__ colind, const double *__restrict__ a,
                            const double *__restrict__ b, const double *__restrict__ alpha,
                            const double *__restrict__ beta, const double *__restrict__ X, int64_t ldx, int k,
                            double *__restrict__ Y, int64_t ldy) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    for (int c0 = 0; c0 < k; c0 += 32) {
        const int c = c0 + lane;
        if (c >= k) break;
        const double al = alpha ? alpha[c] : 1.0, be = beta ? beta[c] : 0.0;
        double acc = 0.0;
        for (int64_t p = p0; p < p1; ++p) {
            double v = al * a[p] + (be != 0.0 ? be * b[p] : 0.0);
            acc += v * X[(int64_t)colind[p] * ldx + c];
        }
        Y[row * ldy + c] = acc;
    }
}

// one warp per row, every column in one pass over the row: lane l owns columns
// l, l+32, ..., NC accumulators (k <= 32 NC)
template <int NC>
__global__ void __launch_bounds__(256) k_spmm_rows(int64_t n, const int64_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colind, const double *__restrict__ a,
                                                   const double *__restrict__ b, const double *__restrict__ alpha,
                                                   const double *__restrict__ beta, const double *__restrict__ X,
                                                   int64_t ldx, int k, double *__restrict__ Y, int64_t ldy) {
    // FP64 is the scarce unit: one FMA per (nonzero, column) for A alone, two when B
    // takes part (sums of A x and B x kept apart, combined once per row)
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const bool use_b = beta != nullptr;
    double acc_a[NC], acc_b[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) { acc_a[t] = 0.0; acc_b[t] = 0.0; }
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    // the row's column indices and values are loaded 32 at a time (one per lane) and
    // broadcast, so consecutive X-row loads do not wait on each other
    for (int64_t q0 = p0; q0 < p1; q0 += 32) {
        const int cnt = (int)min((int64_t)32, p1 - q0);
        const int64_t q = q0 + lane;
        const int my_col = lane < cnt ? colind[q] : 0;
        const double my_a = lane < cnt ? a[q] : 0.0;
        const double my_b = (use_b && lane < cnt) ? b[q] : 0.0;
#pragma unroll 4
        for (int e = 0; e < cnt; ++e) {
            const int col = __shfl_sync(0xffffffffu, my_col, e);
            const double av = __shfl_sync(0xffffffffu, my_a, e);
            const double bv = __shfl_sync(0xffffffffu, my_b, e);
            const double *x = X + (int64_t)col * ldx;
#pragma unroll
            for (int t = 0; t < NC; ++t) {
                const int c = lane + 32 * t;
                if (c < k) {
                    const double xv = x[c];
                    acc_a[t] += av * xv;
                    if (use_b) acc_b[t] += bv * xv;
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < NC; ++t) {
        const int c = lane + 32 * t;
        if (c < k) {
            const double al = alpha ? alpha[c] : 1.0;
            Y[row * ldy + c] = use_b ? al * acc_a[t] + beta[c] * acc_b[t] : al * acc_a[t];
        }
    }
}

// one warp per row, lanes over nonzeros (k < 16), KMAX accumulators per lane
template <int KMAX>
__global__ void k_spmm_nnz(int64_t n, const int64_t *__restrict__ rowptr,
                           const int32_t *__restrict__ colind, const double *__restrict__ a,
                           const double *__restrict__ b, const double *__restrict__ alpha,
                           const double *__restrict__ beta, const double *__restrict__ X, int64_t ldx, int k,
                           double *__restrict__ Y, int64_t ldy) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double al[KMAX], be[KMAX], acc[KMAX];
#pragma unroll
    for (int c = 0; c < KMAX; ++c) {
        al[c] = (c < k) ? (alpha ? alpha[c] : 1.0) : 0.0;
        be[c] = (c < k) ? (beta ? beta[c] : 0.0) : 0.0;
        acc[c] = 0.0;
    }
    const int64_t p0 = rowptr[row], p1 = rowptr[row + 1];
    for (int64_t p = p0 + lane; p < p1; p += 32) {
        const double av = a[p], bv = b ? b[p] : 0.0;
        const double *x = X + (int64_t)colind[p] * ldx;
#pragma unroll
        for (int c = 0; c < KMAX; ++c)
            if (c < k) acc[c] += (al[c] * av + be[c] * bv) * x[c];
    }
#pragma unroll
    for (int c = 0; c < KMAX; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && c < k) Y[row * ldy + c] = v;
    }
}

// ---------------------------------------------------------------- SDDMM gradient
// block per row r; X[r][:] (and lambda-weighted) in shared memory; warp per nonzero
__global__ void __launch_bounds__(256) k_sddmm(int64_t n, const int64_t *__restrict__ rowptr,
                                               const int32_t *__restrict__ colind,
                                               const double *__restrict__ X,
                                               const double *__restrict__ lam, int ne,
                                               double *__restrict__ ga, double *__restrict__ gb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *xr = reinterpret_cast<double *>(smem_raw);
    double *xl = xr + ne;
    const int64_t r = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < ne; i += 256) {
        double v = X[r * ne + i];
        xr[i] = v;
        xl[i] = v * lam[i];
    }
    __syncthreads();
    for (int64_t p = rowptr[r] + wid; p < rowptr[r + 1]; p += 8) {
        const double *xc = X + (int64_t)colind[p] * ne;
        double sa = 0.0, sb = 0.0;
        for (int i = lane; i < ne; i += 32) {
            double v = xc[i];
            sa += xr[i] * v;
            sb += xl[i] * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_down_sync(0xffffffffu, sa, o);
            sb += __shfl_down_sync(0xffffffffu, sb, o);
        }
        if (lane == 0) {
            if (ga) ga[p] = sa;
            if (gb) gb[p] = -sb;
        }
    }
}

}  // namespace sss
