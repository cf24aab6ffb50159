// FP64-accurate products on the FP16 tensor cores: the probes' Gram matrices and tall
// products (Cholesky-QR of Alg. 2 step 4, Rayleigh-Ritz) and the sparse products A X and
// B X of the subspace iteration (Alg. 2 steps 3-5), by error-free splitting (Ozaki, Ogita,
// Oishi and Rump), with one scale per operand row and an exact integer sum over the whole
// reduction.
//
// Operand.  Element (row, t) of a dense operand sits at M[row * ld_row + t * ld_k]: for the
// Gram matrix G = X^T Y the operand rows are the columns of X (ld_row = 1, ld_k = ldx); for
// the product X Q the rows of X (ld_row = ldx, ld_k = 1) and the columns of Q; for the
// sparse product A X the rows of A (CSR) and the columns of X.
// Splitting.  Every operand row is scaled by a power of two fixed by its largest entry over
// the whole reduction (|x| < 2^E, em = E + 1022 is the largest biased exponent of the row);
// Y = round(x 2^(55 - E)) is a 56-bit integer whose 8 balanced base-128 digits q_0 .. q_7
// (|q_p| <= 64, exact in FP16) are the slices: x = 2^(E - 6) sum_p q_p 2^(-7p) up to
// 2^(E - 56).  The digits are cut from the FP64 bit pattern with integer arithmetic.
// Slice layout.  The reduction is cut into pieces of 32.  For 128-row tile rt and piece kc,
// eight 8 KB blocks of digits in the MMA's core-matrix layout (oz_offset below) at block
// index kc * nrt + rt (dense) or at the index of the (tile, piece) pair (sparse A: only
// pieces that hold entries).
// Products.  An output tile of 128 x 64 entries takes, per piece, the 36 digit products with
// p + q <= 7 on the tensor cores into 8 FP32 accumulators D_d = sum_{p+q=d} (8 x 64 = 512
// tensor-memory columns), exact over 16 pieces: |D_d| <= 8 * 512 * 64^2 = 2^24.  Every 16
// pieces the accumulators are read out and summed as integers,
//     hi += D_0 2^21 + D_1 2^14 + D_2 2^7 + D_3,   lo += D_4 2^21 + D_5 2^14 + D_6 2^7 + D_7,
// so the result, (hi 2^28 + lo) 2^(E_a + E_b - 61), is the exact sum of the truncated digit
// expansion rounded once to FP64: its error is a few units of 2^-53 of
// K max|a_row| max|b_row| (K the reduction length).
// Pipeline.  Two shared-memory stages of one piece each (64 KB of A, 32 KB of B): the loads
// of piece i + 1 run while the tensor cores work on piece i.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"

namespace sstc {

constexpr int kOzSlices = 8;
constexpr int kOzK = 32;                              // piece width along the reduction
constexpr uint32_t kOzBlock = 128 * kOzK * 2;         // one slice block: 128 rows x 32 K, FP16
constexpr uint32_t kOzHalf = 64 * kOzK * 2;           // its 64-row half
constexpr uint32_t kOzStageA = kOzSlices * kOzBlock;  // 64 KB
constexpr uint32_t kOzStageB = kOzSlices * kOzHalf;   // 32 KB
constexpr int kOzThreads = 256;
constexpr int kOzReadEvery = 16;                      // pieces per exact FP32 accumulation
constexpr size_t kOzGemmSmem = 1024 + 2 * (size_t)(kOzStageA + kOzStageB);
constexpr size_t kOzCsrSmem = (size_t)kOzStageA;
constexpr long long kOzWaitLimit = 1ll << 24;
constexpr uint32_t kTmemColsOz = 512;                 // 8 accumulators x 64 columns

// Byte offset of element (row, k) of an R x 32 FP16 tile: 8 x 8 core matrices of 16-byte
// rows, no swizzle; 4 K-adjacent core matrices 128 bytes apart, 8-row groups 512 bytes apart.
__host__ __device__ __forceinline__ uint32_t oz_offset(int row, int k) {
    return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// descriptor of an R x 32 tile in that layout (leading byte offset 128, stride 512)
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;     // descriptor version of the sm_100 family; layout type 0 = no swizzle
    return d;
}

struct OzOperand {
    const double *M;
    int64_t ld_row, ld_k;
    int64_t rows, kdim;
};

// the 8 balanced base-128 digits (top first) of round(x 2^(55 - E)), |x| < 2^E
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
        int d = (int)(y & 127);
        if (d >= 64) d -= 128;
        q[p] = d;
        y = (y - d) >> 7;
    }
    q[0] = (int)y;                                    // |y| < 2^55: |q_0| <= 64
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
    const int64_t t0 = (int64_t)kc * kOzK;
    const bool live = row < op.rows;
    const int E = (live ? em[row] : 0) - 1022;
    unsigned char *blk = sl + ((uint64_t)kc * nrt + rt) * kOzStageA;
    for (int c = 0; c < kOzK / 8; ++c) {
        __align__(16) __half h[kOzSlices][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t t = t0 + 8 * c + u;
            const double v = (live && t < op.kdim) ? op.M[row * op.ld_row + t * op.ld_k] : 0.0;
            int q[kOzSlices];
            oz_digits(v, E, q);
#pragma unroll
            for (int p = 0; p < kOzSlices; ++p) h[p][u] = __int2half_rn(q[p]);   // |q| <= 64: exact
        }
#pragma unroll
        for (int p = 0; p < kOzSlices; ++p)
            *reinterpret_cast<uint4 *>(blk + (uint64_t)p * kOzBlock + oz_offset(rho, 8 * c)) =
                *reinterpret_cast<const uint4 *>(h[p]);
    }
}

// Sparse operand: block = (tile, piece) pair q, thread = row of the tile.  seg[q * 128 + r]
// is the CSR position of row r's first entry in the piece (columns 32 piece ..).  The
// digits are placed in shared memory (zero elsewhere) and the 8 blocks copied out whole.
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
        const int64_t c0 = (int64_t)pair_piece[q] * kOzK;
        const int64_t end = rowptr[row + 1];
        for (int64_t p = seg[(int64_t)q * 128 + rho]; p < end && colind[p] < c0 + kOzK; ++p) {
            int d[kOzSlices];
            oz_digits(vals[p], E, d);
            const uint32_t off = oz_offset(rho, (int)(colind[p] - c0));
#pragma unroll
            for (int s = 0; s < kOzSlices; ++s)
                *reinterpret_cast<__half *>(sm + (uint32_t)s * kOzBlock + off) = __int2half_rn(d[s]);
        }
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(sl + (uint64_t)q * kOzStageA);
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

// The 144 MMAs of one 32-wide piece: accumulator d (tensor-memory columns 64 d ..) gets
// sum_{p + q = d} A_p B_q^T, p, q < 8, d <= 7.  da, db: descriptors of slice 0 of the
// stage's A and B.  fresh: the first MMA into each accumulator overwrites it.
__device__ __forceinline__ void oz_issue_piece(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, bool fresh) {
    const uint32_t keep_first = fresh ? 0u : 1u;
#pragma unroll
    for (int d = 0; d < kOzSlices; ++d) {
#pragma unroll
        for (int p = 0; p <= d; ++p) {
            const uint64_t a = da + (uint64_t)(p * (kOzBlock >> 4));
            const uint64_t b = db + (uint64_t)((d - p) * (kOzHalf >> 4));
            mma_f16(tmem + (uint32_t)d * 64, a, b, idesc, p == 0 ? keep_first : 1u);
            mma_f16(tmem + (uint32_t)d * 64, a + (256 >> 4), b + (256 >> 4), idesc, 1u);   // second K step
        }
    }
}

// Output tile (rt, bj) = rows 128 rt .., columns 64 bj ..  (beta = 0 does not read out).
// blockIdx.x = bj varies fastest, so the CTAs that share one A tile run together and read
// its slices from L2 after the first.  Thread 0 stages the pieces (two stages) and issues the
// MMAs; all 8 warps read the accumulators out every 16 pieces (warp w: tensor-memory lanes
// 32 (w mod 4) .., columns 32 (w / 4) ..).
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_mm(const OzMM g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *stage_a[2], *stage_b[2];
    stage_a[0] = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    stage_b[0] = stage_a[0] + kOzStageA;
    stage_a[1] = stage_b[0] + kOzStageB;
    stage_b[1] = stage_a[1] + kOzStageA;
    __shared__ __align__(8) uint64_t full[2], empty[2], accfull, drain;
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
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(&accfull, 1);
        mbar_init(&drain, 1);
        fence_mbar_init();
        s_ok = 1;
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_f16_f32(128, 64);
    auto issue_loads = [&](int q, int b) {
        const int kc = sparse ? g.pair_piece[q] : q;
        const unsigned char *ga = g.slA + (uint64_t)(sparse ? q : kc * g.nrtA + rt) * kOzStageA;
        const unsigned char *gb = g.slB + ((uint64_t)kc * g.nrtB + (bj >> 1)) * kOzStageA + (uint64_t)(bj & 1) * kOzHalf;
        mbar_arrive_expect_tx(&full[b], kOzStageA + kOzStageB);
        bulk_g2s(stage_a[b], ga, kOzStageA, &full[b]);
        for (int p = 0; p < kOzSlices; ++p)
            bulk_g2s(stage_b[b] + p * kOzHalf, gb + (uint64_t)p * kOzBlock, kOzHalf, &full[b]);
    };
    long long hi[32], lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        hi[c] = 0;
        lo[c] = 0;
    }
    int n_loaded = 0, n_landed = 0;                  // pieces whose loads were issued / waited for
    if (threadIdx.x == 0) {
        issue_loads(q0, 0);
        n_loaded = 1;
    }
    int n_read = 0;                                  // read-outs done (phase of accfull)
    for (int q = q0; q < q1; ++q) {
        const int i = q - q0, b = i & 1;
        const bool readout = (i % kOzReadEvery) == kOzReadEvery - 1 || q + 1 == q1;
        if (threadIdx.x == 0 && s_ok) {
            // piece i: wait for its stage, issue its MMAs, release the stage on completion
            if (!mbar_wait_bounded(&full[b], (uint32_t)((i >> 1) & 1), kOzWaitLimit)) {
                s_ok = 0;
                mbar_wait_bounded(&full[b], (uint32_t)((i >> 1) & 1), kOzWaitLimit);   // copies in flight land
            } else {
                n_landed = i + 1;
                uint32_t sa_addr = smem_u32(stage_a[b]), sb_addr = smem_u32(stage_b[b]);
                asm volatile("" : "+r"(sa_addr), "+r"(sb_addr));   // keep the descriptors per piece
                oz_issue_piece(tmem, oz_desc(sa_addr), oz_desc(sb_addr), idesc, (i % kOzReadEvery) == 0);
                mma_commit(&empty[b]);
                if (readout) mma_commit(&accfull);
                // piece i + 1 goes to the other stage once piece i - 1's MMAs have read it
                if (q + 1 < q1) {
                    if (i >= 1 && !mbar_wait_bounded(&empty[b ^ 1], (uint32_t)(((i - 1) >> 1) & 1), kOzWaitLimit)) {
                        s_ok = 0;
                    } else {
                        issue_loads(q + 1, b ^ 1);
                        n_loaded = i + 2;
                    }
                }
            }
        }
        if (!readout) continue;
        if (threadIdx.x == 0 && s_ok && !mbar_wait_bounded(&accfull, (uint32_t)(n_read & 1), kOzWaitLimit)) s_ok = 0;
        ++n_read;
        __syncthreads();                               // accumulators complete (or a wait ran out)
        if (!s_ok) break;
        tc_fence_after();
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * half);
#pragma unroll
        for (int d = 0; d < kOzSlices; ++d) {
            const int sh = 7 * (3 - (d & 3));
#pragma unroll
            for (int h16 = 0; h16 < 2; ++h16) {
                float r[16];
                tmem_ld16(lane_base + (uint32_t)(d * 64 + 16 * h16), r);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const long long v = (long long)__float2int_rn(r[c]) << sh;
                    if (d < 4) hi[16 * h16 + c] += v;
                    else lo[16 * h16 + c] += v;
                }
            }
        }
        tc_fence_before();
        __syncthreads();                               // accumulators read: the next MMAs may overwrite
    }
    if (threadIdx.x == 0 && !s_ok) {
        // let MMAs and copies in flight finish before the CTA frees its memory (bounded)
        mma_commit(&drain);
        mbar_wait_bounded(&drain, 0, kOzWaitLimit);
        for (int j = n_landed; j < n_loaded; ++j) mbar_wait_bounded(&full[j & 1], (uint32_t)((j >> 1) & 1), kOzWaitLimit);
        atomicExch(g.status, 1);
    }
    if (s_ok && row < g.rowsA) {
        const int Ea = g.emA[row] - 1022;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int64_t col = col0 + c;
            if (col >= g.rowsB) continue;
            const int E = Ea + g.emB[col] - 1022 - 61;
            const double sc = (E >= -1022 && E <= 1023) ? __longlong_as_double((long long)(E + 1023) << 52)
                                                        : ldexp(1.0, E);
            const double r = fma(__ll2double_rn(hi[c]), 268435456.0, __ll2double_rn(lo[c])) * sc;
            double *o = g.out + row * g.ldo + col;
            if (g.mode == 0) {
                atomicAdd(o, g.alpha * r);
            } else {
                const double s = g.colscale ? g.colscale[col] : 1.0;
                *o = g.alpha * s * r + (g.beta != 0.0 ? g.beta * *o : 0.0);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemColsOz);
}

}  // namespace sstc
