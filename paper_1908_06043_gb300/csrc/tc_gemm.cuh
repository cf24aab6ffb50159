// FP64-accurate products on the FP16 tensor cores: the probes' Gram matrices and tall
// products (Cholesky-QR of Alg. 2 step 4, Rayleigh-Ritz) and the sparse products A X and
// B X of the subspace iteration (Alg. 2 steps 3-5), by error-free splitting (Ozaki, Ogita,
// Oishi and Rump) -- the same splitting as the tensor-core Schur update (tc_kernels.cuh),
// here with one scale per operand row and an exact integer sum over the whole reduction.
//
// Operand.  Element (row, t) of a dense operand sits at M[row * ld_row + t * ld_k]: for the
// Gram matrix G = X^T Y the operand rows are the columns of X (ld_row = 1, ld_k = ldx); for
// the product X Q the rows of X (ld_row = ldx, ld_k = 1) and the columns of Q; for the
// sparse product A X the rows of A (CSR) and the columns of X.
// Splitting.  Every operand row is scaled by a power of two fixed by its largest entry over
// the whole reduction (|x| < 2^E, em = E + 1022 is the largest biased exponent of the row);
// Y = round(x 2^(55 - E)) is a 56-bit integer whose balanced base-256 digits q_0 .. q_6
// (|q_p| <= 128, exact in FP16) are the slices: x = 2^(E - 7) sum_p q_p 2^(-8p) up to
// 2^(E - 56).  The digits are cut from the FP64 bit pattern with integer arithmetic.
// Slice layout.  For 128-row tile rt and reduction piece kc (64 wide), seven 16 KB blocks of
// digits in the MMA's core-matrix layout (tc_ptx.cuh) at block index kc * nrt + rt (dense)
// or at the index of the (tile, piece) pair (sparse A: only pieces that hold entries).
// Products.  An output tile of 128 x 64 entries takes, per piece, the 28 digit products
// with p + q <= 6 on the tensor cores into 7 FP32 accumulators D_d = sum_{p+q=d} (exact for
// two pieces: |D_d| <= 7 * 128 * 2^14 < 2^24).  Every two pieces the accumulators are read
// out and summed as integers,
//     hi += D_0 2^16 + D_1 2^8 + D_2,   lo += D_3 2^24 + D_4 2^16 + D_5 2^8 + D_6,
// so the result, (hi 2^32 + lo) 2^(E_a + E_b - 62), is the exact sum of the truncated
// digit expansion rounded once to FP64: its error is a few units of 2^-53 of
// K max|a_row| max|b_row| (K the reduction length).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"

namespace sstc {

constexpr int kOzSlices = 7;
constexpr uint32_t kOzBlock = 128 * 64 * 2;          // one slice block: 128 rows x 64 K, FP16
constexpr uint32_t kOzHalf = 64 * 64 * 2;            // its 64-row half
constexpr int kOzThreads = 256;
constexpr size_t kOzGemmSmem = 1024 + (size_t)kOzSlices * kOzBlock + (size_t)kOzSlices * kOzHalf;
constexpr size_t kOzCsrSmem = (size_t)kOzSlices * kOzBlock;
constexpr long long kOzWaitLimit = 1ll << 24;
constexpr uint32_t kTmemColsOz = 512;                // 7 accumulators x 64 columns, rounded up

struct OzOperand {
    const double *M;
    int64_t ld_row, ld_k;
    int64_t rows, kdim;
};

// the 7 balanced base-256 digits (top first) of round(x 2^(55 - E)), |x| < 2^E
__device__ __forceinline__ void oz_digits(double x, int E, int (&q)[kOzSlices]) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    long long y = 0;
    if (ex != 0) {
        const long long m = (bits & ((1ll << 52) - 1)) | (1ll << 52);
        const int sh = ex - 1020 - E;                 // y = m 2^sh, sh <= 2
        if (sh >= 0) y = m << sh;
        else if (sh > -60) y = (m + (1ll << (-sh - 1))) >> (-sh);
        if (bits < 0) y = -y;
    }
#pragma unroll
    for (int p = kOzSlices - 1; p > 0; --p) {
        int d = (int)(y & 255);
        if (d >= 128) d -= 256;
        q[p] = d;
        y = (y - d) >> 8;
    }
    q[0] = (int)y;
}

__device__ __forceinline__ int biased_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7ff); }

// em[row] = max(em[row], largest biased exponent of the row over reduction range
// [blockIdx.y per_k, (blockIdx.y + 1) per_k)); em zeroed by the caller.  Thread = row.
__global__ void __launch_bounds__(128) k_oz_expmax(OzOperand op, int64_t per_k, int *__restrict__ em) {
    const int64_t row = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (row >= op.rows) return;
    const int64_t t0 = (int64_t)blockIdx.y * per_k, t1 = min(op.kdim, t0 + per_k);
    int m = 0;
    for (int64_t t = t0; t < t1; ++t) m = max(m, biased_exp(op.M[row * op.ld_row + t * op.ld_k]));
    if (m > 0) atomicMax(&em[row], m);
}

// em[row] = largest biased exponent of CSR row `row` (0 for an empty or zero row)
__global__ void k_oz_csr_expmax(int64_t n, const int64_t *__restrict__ rowptr, const double *__restrict__ vals,
                                int *__restrict__ em) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    int m = 0;
    for (int64_t p = rowptr[row]; p < rowptr[row + 1]; ++p) m = max(m, biased_exp(vals[p]));
    em[row] = m;
}

// Block (rt, kc), thread = row of the tile.  Zero rows / columns pad the operand.
__global__ void __launch_bounds__(128) k_oz_slice(OzOperand op, const int *__restrict__ em,
                                                  unsigned char *__restrict__ sl) {
    const int rt = blockIdx.x, kc = blockIdx.y;
    const int nrt = gridDim.x;
    const int rho = threadIdx.x;
    const int64_t row = (int64_t)rt * 128 + rho;
    const int64_t t0 = (int64_t)kc * 64;
    const bool live = row < op.rows;
    const int E = (live ? em[row] : 0) - 1022;
    unsigned char *blk = sl + ((uint64_t)kc * nrt + rt) * kOzSlices * kOzBlock;
    for (int c = 0; c < 8; ++c) {
        __align__(16) __half h[kOzSlices][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t t = t0 + 8 * c + u;
            const double v = (live && t < op.kdim) ? op.M[row * op.ld_row + t * op.ld_k] : 0.0;
            int q[kOzSlices];
            oz_digits(v, E, q);
#pragma unroll
            for (int p = 0; p < kOzSlices; ++p) h[p][u] = __int2half_rn(q[p]);   // |q| <= 128: exact
        }
#pragma unroll
        for (int p = 0; p < kOzSlices; ++p)
            *reinterpret_cast<uint4 *>(blk + (uint64_t)p * kOzBlock + core_offset(rho, 8 * c)) =
                *reinterpret_cast<const uint4 *>(h[p]);
    }
}

// Sparse operand: block = (tile, piece) pair q, thread = row of the tile.  seg[q * 128 + r]
// is the CSR position of row r's first entry in the piece (columns 64 piece ..).  The
// digits are placed in shared memory (zero elsewhere) and the 7 blocks copied out whole.
__global__ void __launch_bounds__(128) k_oz_slice_csr(int64_t n, const int64_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ colind,
                                                      const double *__restrict__ vals,
                                                      const int64_t *__restrict__ seg,
                                                      const int32_t *__restrict__ pair_tile,
                                                      const int32_t *__restrict__ pair_piece,
                                                      const int *__restrict__ em, unsigned char *__restrict__ sl) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int q = blockIdx.x;
    const int rho = threadIdx.x;
    for (uint32_t o = rho * 16; o < kOzCsrSmem; o += 128 * 16)
        *reinterpret_cast<uint4 *>(sm + o) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int64_t row = (int64_t)pair_tile[q] * 128 + rho;
    if (row < n) {
        const int E = em[row] - 1022;
        const int64_t c0 = (int64_t)pair_piece[q] * 64;
        const int64_t end = rowptr[row + 1];
        for (int64_t p = seg[(int64_t)q * 128 + rho]; p < end && colind[p] < c0 + 64; ++p) {
            int d[kOzSlices];
            oz_digits(vals[p], E, d);
            const uint32_t off = core_offset(rho, (int)(colind[p] - c0));
#pragma unroll
            for (int s = 0; s < kOzSlices; ++s)
                *reinterpret_cast<__half *>(sm + (uint32_t)s * kOzBlock + off) = __int2half_rn(d[s]);
        }
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(sl + (uint64_t)q * kOzSlices * kOzBlock);
    for (uint32_t o = rho; o < kOzCsrSmem / 16; o += 128) dst[o] = reinterpret_cast<const uint4 *>(sm)[o];
}

// 32 lanes x 32 bits, 32 consecutive columns per thread, load and wait in one statement
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

struct OzMM {
    const unsigned char *slA;
    const int *emA;
    int nrtA;
    int64_t rowsA;
    const int32_t *tile_ptr;     // sparse A: pairs of row tile rt are [tile_ptr[rt], tile_ptr[rt + 1])
    const int32_t *pair_piece;   // sparse A: reduction piece of pair q (slice block q)
    const unsigned char *slB;
    const int *emB;
    int nrtB;
    int64_t rowsB;
    int nkc, per;                // dense A: pieces [z per, min(nkc, (z + 1) per)), block kc * nrtA + rt
    int mode;                    // 0: out += alpha r (atomic); 1: out = alpha s_col r + beta out
    double alpha, beta;
    const double *colscale;      // mode 1: per-column factor s_col (null: 1)
    double *out;
    int64_t ldo;
    int *status;                 // raised when a bounded wait runs out
};

// Output tile (rt, bj) = rows 128 rt .., columns 64 bj ..  (beta = 0 does not read out).
// blockIdx.x = bj varies fastest, so the CTAs that share one A tile run together and read
// its slices from L2 after the first.
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_mm(const OzMM g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sa = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    unsigned char *sb = sa + kOzSlices * kOzBlock;
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const int bj = blockIdx.x, rt = blockIdx.y;
    const bool sparse = g.tile_ptr != nullptr;
    int q0, q1;
    if (sparse) {
        q0 = g.tile_ptr[rt];
        q1 = g.tile_ptr[rt + 1];
    } else {
        q0 = blockIdx.z * g.per;
        q1 = min(g.nkc, q0 + g.per);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t row = (int64_t)rt * 128 + 32 * quarter + lane;
    const int64_t col0 = (int64_t)bj * 64 + 32 * half;
    if (q0 >= q1) {                  // no entries in this tile's rows: the product is zero
        if (g.mode == 1 && row < g.rowsA)
            for (int c = 0; c < 32; ++c) {
                const int64_t col = col0 + c;
                if (col >= g.rowsB) break;
                double *o = g.out + row * g.ldo + col;
                *o = g.beta != 0.0 ? g.beta * *o : 0.0;
            }
        return;
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, kTmemColsOz);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        s_ok = 1;
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_f16_f32(128, 64);
    const uint64_t da = smem_desc(smem_u32(sa)), db = smem_desc(smem_u32(sb));
    auto issue_loads = [&](int q) {
        const int kc = sparse ? g.pair_piece[q] : q;
        const unsigned char *ga = g.slA + (uint64_t)(sparse ? q : kc * g.nrtA + rt) * kOzSlices * kOzBlock;
        const unsigned char *gb = g.slB + ((uint64_t)kc * g.nrtB + (bj >> 1)) * kOzSlices * kOzBlock +
                                  (uint64_t)(bj & 1) * kOzHalf;
        mbar_arrive_expect_tx(&bar[0], kOzSlices * (kOzBlock + kOzHalf));
        bulk_g2s(sa, ga, kOzSlices * kOzBlock, &bar[0]);
        for (int p = 0; p < kOzSlices; ++p) bulk_g2s(sb + p * kOzHalf, gb + (uint64_t)p * kOzBlock, kOzHalf, &bar[0]);
    };
    long long hi[32], lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        hi[c] = 0;
        lo[c] = 0;
    }
    if (threadIdx.x == 0) issue_loads(q0);
    for (int q = q0; q < q1; ++q) {
        const int i = q - q0;
        const uint32_t parity = (uint32_t)(i & 1);
        if (threadIdx.x == 0 && s_ok) {
            if (!mbar_wait_bounded(&bar[0], parity, kOzWaitLimit)) {
                s_ok = 0;
                mbar_wait_bounded(&bar[0], parity, kOzWaitLimit);    // let copies in flight land
            } else {
                // accumulators restart every two pieces
                issue_digit_mmas<kOzBlock, kOzHalf, 64>(tmem, da, db, idesc, (i & 1) == 0);
                mma_commit(&bar[1]);
                if (!mbar_wait_bounded(&bar[1], parity, kOzWaitLimit)) {
                    s_ok = 0;
                    mbar_wait_bounded(&bar[1], parity, kOzWaitLimit);
                } else if (q + 1 < q1) {
                    issue_loads(q + 1);             // the next piece loads during the read-out
                }
            }
        }
        if ((i & 1) == 0 && q + 1 < q1) continue;  // the next piece adds into the same accumulators
        __syncthreads();
        if (!s_ok) break;
        tc_fence_after();
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * half);
#pragma unroll
        for (int d = 0; d < kOzSlices; ++d) {
            uint32_t r[32];
            tmem_ld32(lane_base + (uint32_t)(d * 64), r);
            const int sh = d < 3 ? 8 * (2 - d) : 8 * (6 - d);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const long long v = (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
                if (d < 3) hi[c] += v;
                else lo[c] += v;
            }
        }
        tc_fence_before();
        __syncthreads();                            // accumulators read: the next MMAs may overwrite
    }
    if (s_ok && row < g.rowsA) {
        const int Ea = g.emA[row] - 1022;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int64_t col = col0 + c;
            if (col >= g.rowsB) continue;
            const int E = Ea + g.emB[col] - 1022 - 62;
            const double sc = (E >= -1022 && E <= 1023) ? __longlong_as_double((long long)(E + 1023) << 52)
                                                        : ldexp(1.0, E);
            const double r = fma(__ll2double_rn(hi[c]), 4294967296.0, __ll2double_rn(lo[c])) * sc;
            double *o = g.out + row * g.ldo + col;
            if (g.mode == 0) {
                atomicAdd(o, g.alpha * r);
            } else {
                const double s = g.colscale ? g.colscale[col] : 1.0;
                *o = g.alpha * s * r + (g.beta != 0.0 ? g.beta * *o : 0.0);
            }
        }
    }
    if (!s_ok && threadIdx.x == 0) atomicExch(g.status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemColsOz);
}

}  // namespace sstc
