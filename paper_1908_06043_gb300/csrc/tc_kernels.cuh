// Tensor-core Schur-complement update of the FP64 multifrontal factorisation (K3 of
// Alg. 2 step 2: F22 -= L21 W^T, W = L21 D) on the FP16 tensor cores, FP64-accurate by an
// error-free splitting of the operands (the slicing scheme of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication", Numer. Algorithms 2012).
//
// Splitting.  Each row x of L21 (or of W) is scaled by 2^-e, e the exponent with
// max |x_t| < 2^e, and cut into kSlices balanced 8-bit digits:
//   y_1 = x 2^(7-e),  q_p = rint(y_p),  y_(p+1) = (y_p - q_p) 2^8,
// so x = 2^(e-7) sum_p q_p 2^(-8(p-1)) up to 2^(e-56), every |q_p| <= 128 (exact in FP16).
// Product.  sum_t x_it z_jt = 2^(e_i + f_j - 14) sum_{p,q} 2^(-8(p+q-2)) D_pq with the
// integer matrices D_pq = Q_p^A (Q_q^B)^T.  The pairs with p + q <= kSlices + 1 are kept
// (the rest lie below 2^-56 of the row scales); pairs of equal p + q share one FP32
// accumulator in tensor memory.  Over K = 64 every partial sum is an integer of magnitude
// below 7 * 64 * 128^2 < 2^23, so the FP32 accumulation is exact.
// Combination.  With a_d the accumulator of p + q = d + 2 (d = 0..6), the update is
//   2^(e_i + f_j - 62) (hi 2^32 + lo),  hi = a_0 2^16 + a_1 2^8 + a_2,
//   lo = a_3 2^24 + a_4 2^16 + a_5 2^8 + a_6.
// The accumulators are converted to 32-bit integers (the 64-bit conversions run at the FP64
// rate on this GPU), hi and lo are formed in 64-bit integers (exact, below 2^40 and 2^49),
// converted to FP64 (exact) and combined by one FMA, hi 2^32 + lo, rounded once; a second
// FMA applies it to the front.  Every bit of lo is kept: dropping its low bits costs about
// 2^-45 of a typical product per update, which the many updates of a front and the
// conditioning of A - sigma B amplify past an FP64 factorisation's accuracy.
//
// Data flow per factor step: k_panel writes L21 (in place) and W (scratch) in FP64;
// k_tc_slice writes their slices, already in the MMA's shared-memory layout (see
// tc_ptx.cuh), as one 16 KB block per (operand, 128-row tile, slice), and the row
// exponents; k_schur_tc computes one 128 x 64 output tile per CTA: one bulk copy brings
// the 7 A-slices of its row tile, seven bring the B-slices of its column half-tile, one
// thread issues the 28 x 4 MMAs, and four warps read the 7 accumulators back and update
// the FP64 front.  Every wait is bounded; a wait that runs out records a timeout in the
// shift's counters, and the CTA still releases its tensor memory.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "factor_kernels.cuh"
#include "tc_ptx.cuh"

namespace sstc {

constexpr int kSlices = kTcSlices;
constexpr int kTileM = 128;                   // output rows per CTA (TMEM lanes)
constexpr int kTileN = 64;                    // output columns per CTA
constexpr uint32_t kSliceBytes = (uint32_t)kTcSliceBytes;   // one 128 x 64 FP16 block
constexpr uint32_t kHalfSliceBytes = 64 * 64 * 2;           // its 64-row half
constexpr int kAccum = kSlices;               // accumulators, one per p + q
constexpr uint32_t kTmemCols = 512;           // 7 x 64 columns, rounded to a power of two
constexpr size_t kSchurTcSmem = 1024 + (size_t)kSlices * kSliceBytes + (size_t)kSlices * kHalfSliceBytes;
constexpr size_t kSelftestSmem = 1024 + (size_t)kSliceBytes + kHalfSliceBytes;
constexpr int kSchurTcThreads = 256;          // 8 warps: lane quarter w % 4, column half w / 4
constexpr long long kWaitLimit = 1ll << 24;   // mbarrier polls (about a second)

// ---------------------------------------------------------------- self-test
// One 128 x 64 x 64 MMA tile of FP16 operands given in the core-matrix layout (A: 128
// rows, B: 64 rows), FP32 result written row-major to D.  status[0] = 0 ok, 1 a wait ran
// out.
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const unsigned char *__restrict__ A,
                                                         const unsigned char *__restrict__ B, float *D,
                                                         int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sa = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);   // swizzle atoms: 1024-aligned
    unsigned char *sb = sa + kSliceBytes;
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        tmem_alloc(&s_tmem, 64);
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
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar[0], kSliceBytes + kHalfSliceBytes);
        bulk_g2s(sa, A, kSliceBytes, &bar[0]);
        bulk_g2s(sb, B, kHalfSliceBytes, &bar[0]);
        if (!mbar_wait_bounded(&bar[0], 0, kWaitLimit)) {
            s_ok = 0;
        } else {
            const uint32_t idesc = idesc_f16_f32(kTileM, kTileN);
            for (int kk = 0; kk < 4; ++kk)
                mma_f16(tmem, smem_desc(smem_u32(sa) + kk * kKStepBytes), smem_desc(smem_u32(sb) + kk * kKStepBytes), idesc,
                        kk > 0);
            mma_commit(&bar[1]);
            if (!mbar_wait_bounded(&bar[1], 0, kWaitLimit)) s_ok = 0;
        }
    }
    __syncthreads();
    tc_fence_after();
    if (s_ok) {
        for (int c0 = 0; c0 < kTileN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
            for (int i = 0; i < 16; ++i) D[(32 * warp + lane) * kTileN + c0 + i] = v[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 64);
    if (threadIdx.x == 0) status[0] = s_ok ? 0 : 1;
}

// ---------------------------------------------------------------- slice producer
// Block = one 128-row tile of L21 (the first nrt tiles of a task) or of W (the next nrt);
// thread = one row.  Writes kSlices blocks of 16 KB and the row exponents.
__global__ void __launch_bounds__(128) k_tc_slice(const StepTask *__restrict__ tasks, int32_t ntask,
                                                  const ssk::ShiftPtrs<double> *sp) {
    const ssk::ShiftPtrs<double> s = sp[blockIdx.y];
    const int32_t tile = blockIdx.x;
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].sl_pre <= tile) lo = mid; else hi = mid - 1;
    }
    const StepTask tk = tasks[lo];
    const int nrt = (tk.r + kTileM - 1) / kTileM;
    const int tt = tile - tk.sl_pre;               // 0 .. 2 nrt - 1
    const bool side_b = tt >= nrt;
    const int ti = side_b ? tt - nrt : tt;
    const int rho = threadIdx.x;
    const int i = ti * kTileM + rho;
    const bool live = i < tk.r;
    const int w = tk.w, m = tk.m;
    const double *F = s.ws + tk.front_off;
    const double *W = s.wbuf + tk.wbuf_off;
    const int64_t base = tk.k0 + w;
    // the element (row i, column t) of this operand; 0 outside the task
    auto elem = [&](int t) -> double {
        if (!live || t >= w) return 0.0;
        return side_b ? W[(int64_t)t * tk.r + i] : F[(int64_t)(tk.k0 + t) * m + base + i];
    };
    double mx = 0.0;
    for (int t = 0; t < w; ++t) mx = fmax(mx, fabs(elem(t)));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);                   // mx = f 2^e, f in [0.5, 1): |x| < 2^e
    if (live) s.ex[tk.ex_off + (side_b ? tk.r : 0) + i] = e;
    const double sc = ldexp(1.0, 7 - e);           // a power of two: scaling is exact
    unsigned char *blk = s.sl + tk.sl_off + (uint64_t)((side_b ? nrt : 0) + ti) * kSlices * kSliceBytes;
    for (int c = 0; c < 8; ++c) {
        double y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) y[u] = elem(8 * c + u) * sc;
#pragma unroll
        for (int p = 0; p < kSlices; ++p) {
            __align__(16) __half h[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const double qv = rint(y[u]);
                y[u] = (y[u] - qv) * 256.0;
                h[u] = __float2half_rn((float)qv);  // |qv| <= 128: exact
            }
            *reinterpret_cast<uint4 *>(blk + (uint64_t)p * kSliceBytes + core_offset(rho, 8 * c)) =
                *reinterpret_cast<const uint4 *>(h);
        }
    }
}

// ---------------------------------------------------------------- Schur update
// Block = one 128 x 64 tile (bi, bj) of the lower triangle of a task's trailing r x r
// block; tiles of a task are numbered q = bi (bi + 1) + bj, bj <= 2 bi + 1.  256 threads:
// warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its rows) and columns 32 (w / 4)
// .. + 31 of every accumulator.
__global__ void __launch_bounds__(kSchurTcThreads, 1) k_schur_tc(const StepTask *__restrict__ tasks, int32_t ntask,
                                                                  const ssk::ShiftPtrs<double> *sp) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sa = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    unsigned char *sb = sa + kSlices * kSliceBytes;
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;
    const ssk::ShiftPtrs<double> s = sp[blockIdx.y];
    const int32_t tile = blockIdx.x;
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tc_pre <= tile) lo = mid; else hi = mid - 1;
    }
    const StepTask tk = tasks[lo];
    const int q = tile - tk.tc_pre;
    int bi = (int)((sqrt(4.0 * q + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) <= q) ++bi;
    while (bi * (bi + 1) > q) --bi;
    const int bj = q - bi * (bi + 1);
    const int nrt = (tk.r + kTileM - 1) / kTileM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        tmem_alloc(&s_tmem, kTmemCols);
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
    if (threadIdx.x == 0) {
        const unsigned char *ga = s.sl + tk.sl_off + (uint64_t)bi * kSlices * kSliceBytes;
        const unsigned char *gb = s.sl + tk.sl_off + (uint64_t)(nrt + (bj >> 1)) * kSlices * kSliceBytes +
                                  (uint64_t)(bj & 1) * kHalfSliceBytes;
        mbar_arrive_expect_tx(&bar[0], kSlices * (kSliceBytes + kHalfSliceBytes));
        bulk_g2s(sa, ga, kSlices * kSliceBytes, &bar[0]);
        for (int p = 0; p < kSlices; ++p)
            bulk_g2s(sb + p * kHalfSliceBytes, gb + (uint64_t)p * kSliceBytes, kHalfSliceBytes, &bar[0]);
        if (!mbar_wait_bounded(&bar[0], 0, kWaitLimit)) {
            s_ok = 0;
        } else {
            const uint32_t idesc = idesc_f16_f32(kTileM, kTileN);
            static_assert(kSlices == 7 && kAccum == 7, "the issue loop covers 7 slices and 7 accumulators");
            issue_digit_mmas<kSliceBytes, kHalfSliceBytes, kTileN>(tmem, smem_desc(smem_u32(sa)),
                                                                    smem_desc(smem_u32(sb)), idesc, true);
            mma_commit(&bar[1]);
            if (!mbar_wait_bounded(&bar[1], 0, kWaitLimit)) {
                s_ok = 0;
                mbar_wait_bounded(&bar[1], 0, kWaitLimit);     // let MMAs in flight finish
            }
        }
        if (!s_ok) atomicAdd(&s.counts[7], 1ull);
    }
    __syncthreads();
    tc_fence_after();
    if (s_ok) {
        const int r = tk.r, m = tk.m;
        const int64_t base = tk.k0 + tk.w;
        const int quarter = warp & 3, half = warp >> 2;
        const int i = bi * kTileM + 32 * quarter + lane;          // trailing row of this thread
        const int ei = i < r ? s.ex[tk.ex_off + i] : 0;
        double *F = s.ws + tk.front_off;
        const int32_t *fex = s.ex + tk.ex_off + r;
        for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 16) {
            float a[kAccum][16];
#pragma unroll
            for (int d = 0; d < kAccum; ++d)
                tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(d * kTileN + c0), a[d]);
            const int j0 = bj * kTileN + c0;
            // this thread's 16 front entries, loaded before any is used
            double cv[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int j = j0 + c;
                cv[c] = (i < r && j <= i) ? F[(base + j) * (int64_t)m + base + i] : 0.0;
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int j = j0 + c;
                if (i >= r || j > i) continue;
                const long long h2 = ((long long)__float2int_rn(a[0][c]) << 16) +
                                     ((long long)__float2int_rn(a[1][c]) << 8) + (long long)__float2int_rn(a[2][c]);
                const long long l2 = ((long long)__float2int_rn(a[3][c]) << 24) +
                                     ((long long)__float2int_rn(a[4][c]) << 16) +
                                     ((long long)__float2int_rn(a[5][c]) << 8) + (long long)__float2int_rn(a[6][c]);
                const double v = fma(__ll2double_rn(h2), 4294967296.0, __ll2double_rn(l2));
                const int E = ei + fex[j] - 62;
                const double sc = (E >= -1022 && E <= 1023) ? __longlong_as_double((long long)(E + 1023) << 52)
                                                            : ldexp(1.0, E);
                F[(base + j) * (int64_t)m + base + i] = fma(-v, sc, cv[c]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace sstc
