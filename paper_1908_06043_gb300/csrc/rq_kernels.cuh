// Rayleigh quotients x^T A x / x^T B x of a block of vectors over the CSR pattern of
// A union B, in double-double arithmetic: the eigenvalues a probe returns (after Alg. 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sss {

// ---------------------------------------------------------------- Rayleigh quotients
// Error-free transformations (Knuth's TwoSum, the FMA form of Dekker's TwoProduct) and the
// compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM
// J. Sci. Comput. 2005): the sum is accumulated as hi + lo, every rounding error of a
// product or an addition carried into lo.
struct DD {
    double hi, lo;
};
__device__ __forceinline__ void dd_add_prod(DD &s, double a, double b) {
    const double p = a * b, pe = fma(a, b, -p);
    const double t = s.hi + p, z = t - s.hi;
    const double se = (s.hi - (t - z)) + (p - z);
    s.hi = t;
    s.lo += se + pe;
}
__device__ __forceinline__ void dd_add(DD &s, double hi, double lo) {
    const double t = s.hi + hi, z = t - s.hi;
    const double se = (s.hi - (t - z)) + (hi - z);
    s.hi = t;
    s.lo += se + lo;
}

// Block (bx, by): rows [bx*rows_per, ...) x columns [128 by, 128 by + 128), one thread per
// column.  For each row i, y = (A x)_i and z = (B x)_i in double-double, then x_i y and
// x_i z are added to the thread's double-double numerator and denominator.  Partial
// sums: part[(bx k + c) * 4 + {num hi, num lo, den hi, den lo}].
__global__ void __launch_bounds__(128) k_rq_dd_partial(int64_t n, const int64_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colind,
                                                       const double *__restrict__ a, const double *__restrict__ b,
                                                       const double *__restrict__ X, int k, int64_t rows_per,
                                                       double *__restrict__ part) {
    const int c = blockIdx.y * 128 + threadIdx.x;
    if (c >= k) return;
    const int64_t r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    DD num{0.0, 0.0}, den{0.0, 0.0};
    for (int64_t i = r0; i < r1; ++i) {
        DD y{0.0, 0.0}, z{0.0, 0.0};
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double xv = X[(int64_t)colind[p] * k + c];
            dd_add_prod(y, a[p], xv);
            dd_add_prod(z, b[p], xv);
        }
        const double xi = X[i * k + c];
        dd_add_prod(num, xi, y.hi);
        dd_add_prod(num, xi, y.lo);
        dd_add_prod(den, xi, z.hi);
        dd_add_prod(den, xi, z.lo);
    }
    double *o = part + ((int64_t)blockIdx.x * k + c) * 4;
    o[0] = num.hi;
    o[1] = num.lo;
    o[2] = den.hi;
    o[3] = den.lo;
}

// theta[c] = (sum of numerators) / (sum of denominators), summed and divided in
// double-double, rounded once
__global__ void k_rq_dd_finish(int k, int nparts, const double *__restrict__ part, double *__restrict__ theta) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    DD num{0.0, 0.0}, den{0.0, 0.0};
    for (int q = 0; q < nparts; ++q) {
        const double *o = part + ((int64_t)q * k + c) * 4;
        dd_add(num, o[0], o[1]);
        dd_add(den, o[2], o[3]);
    }
    const double nh = num.hi + num.lo, nl = num.lo - (nh - num.hi);
    const double dh = den.hi + den.lo, dl = den.lo - (dh - den.hi);
    const double qv = nh / dh;
    const double rem = (fma(-qv, dh, nh) + nl - qv * dl) / dh;
    theta[c] = qv + rem;
}

}  // namespace sss
