// Level-scheduled panel triangular solves with the multifrontal factor (Alg. 2 step 3:
// V <- L^-T D^-1 L^-1 (B V)).  Right-hand sides are N x k row-major in the permuted
// (analysis) order.  For a panel with pivot order P, unit lower L11 (its inverse stored),
// block-diagonal D and below-diagonal rows L21 (front rows [k0+w, m)):
//   forward:  y = L11^-1 P b1 (stored in place of b1),  b2 -= L21 y       (push, atomics)
//   backward: z = L21^T x2 (gathered, atomics into a per-panel buffer),
//             x1 = P^T L11^-T (D^-1 y - z)                                 (scatter)
// Panels in one solve level are independent; levels run in order (forward) or reverse
// order (backward).  T is the factor / right-hand-side type.
//
// Each step is a device function over one work item (a panel or a row tile, times a
// chunk of right-hand-side columns).  Two drivers run them: one kernel launch per level
// and step (k_fwd_diag, k_fwd_update, ...), or k_solve_sweeps, a single cooperative
// launch that walks every level of both sweeps with a bounded grid barrier between
// steps.  The right-hand sides and the gather buffer are written by other blocks of the
// same launch there, so they are read through plain (coherent) loads, never through the
// read-only path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "grid_sync.cuh"
#include "internal.h"

namespace ssk {

constexpr int KC = 32;     // right-hand-side columns per block of the update / gather kernels
constexpr int KD = 8;      // right-hand-side columns per block of the diagonal kernels: they
                           // run alone on the long chain of root panels, so narrow chunks
                           // spread each level over more SMs
constexpr int LT_LD = NB + 4;   // row stride of the FP32 gather's transposed panel tile

// dynamic shared memory of the solve steps
template <typename T> constexpr size_t diag_solve_smem() { return sizeof(T) * NB * ((KD + 1) + (NB + 1)); }
template <typename T> constexpr size_t tile_solve_smem() { return sizeof(T) * (NB * (TR + 1) + TR * (KC + 1)); }
constexpr size_t tile_solve_smem_f32() { return sizeof(float) * (TR * LT_LD + TR * KC); }
// shared memory of the per-step update / gather kernels for T
template <typename T> constexpr size_t tile_kernel_smem() {
    return std::is_same<T, float>::value ? tile_solve_smem_f32() : tile_solve_smem<T>();
}
template <typename T> constexpr size_t sweep_smem() {
    return diag_solve_smem<T>() > tile_kernel_smem<T>() ? diag_solve_smem<T>() : tile_kernel_smem<T>();
}

__device__ __forceinline__ void atomic_add_t(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_t(float *p, float v) { atomicAdd(p, v); }

__device__ __forceinline__ void atomic_add_pair(float *p, float v0, float v1, bool both, bool paired) {
    if (paired) {
        atomicAdd(reinterpret_cast<float2 *>(p), make_float2(v0, v1));
    } else {
        atomicAdd(p, v0);
        if (both) atomicAdd(p + 1, v1);
    }
}

// panel slot of a row tile: the last slot whose tile prefix is <= tile
__device__ __forceinline__ int tile_slot(const int32_t *__restrict__ tile_pre, int32_t count, int tile) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_pre[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- step bodies
// Each body starts with a block barrier, so a block may run several items in a row on
// the same shared memory.

// forward diagonal step of panel slot `slot`, right-hand-side chunk `chunk` (KD columns)
template <typename T>
__device__ __forceinline__ void fwd_diag_item(unsigned char *smem_raw, int slot, int chunk,
                                              const int32_t *__restrict__ lvl_panels,
                                              const PanelDesc *__restrict__ panels,
                                              const double *__restrict__ linv,
                                              const int32_t *__restrict__ piv, T *b, int k) {
    T (*Y)[KD + 1] = reinterpret_cast<T (*)[KD + 1]>(smem_raw);
    T (*Lm)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smem_raw + sizeof(T) * NB * (KD + 1));
    const int p = lvl_panels[slot];
    const PanelDesc pd = panels[p];
    const int w = pd.w, c0 = chunk * KD, kc = min(KD, k - c0);
    const int tid = threadIdx.x;
    // all loads before the first store to shared memory (one memory latency per item)
    constexpr int MU = NB * NB / 256, YU = NB * KD / 256;
    double mv[MU];
    T yv[YU];
    int sv[YU];
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int i = (tid + 256 * u) / KD;
        sv[u] = i < w ? piv[(int64_t)p * NB + i] : 0;
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) mv[u] = linv[(int64_t)p * NB * NB + tid + 256 * u];
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u, i = q / KD, c = q % KD;
        yv[u] = (i < w && c < kc) ? b[(int64_t)(pd.g0 + sv[u]) * k + c0 + c] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u;
        Y[q / KD][q % KD] = yv[u];
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) {
        const int q = tid + 256 * u;
        Lm[q / NB][q % NB] = (T)mv[u];
    }
    __syncthreads();
    // rows i and i + 32 of column c accumulate side by side
    {
        constexpr int RU = NB * KD / 256;
        const int c = tid % KD, i0 = tid / KD;
        T acc[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) acc[u] = 0;
        for (int t = 0; t < w; ++t) {
            const T yt = Y[t][c];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int i = i0 + (256 / KD) * u;
                acc[u] += (t <= i) ? Lm[i][t] * yt : (T)0;
            }
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int i = i0 + (256 / KD) * u;
            if (i < w && c < kc) b[(int64_t)(pd.g0 + i) * k + c0 + c] = acc[u];
        }
    }
}

// forward update of row tile `tile`, chunk `chunk` (KC columns): b2 -= L21 y
template <typename T>
__device__ __forceinline__ void fwd_update_item(unsigned char *smem_raw, int tile, int chunk,
                                                const int32_t *__restrict__ lvl_panels,
                                                const int32_t *__restrict__ tile_pre, int32_t count,
                                                const PanelDesc *__restrict__ panels,
                                                const int32_t *__restrict__ idx,
                                                const T *__restrict__ arena, T *b, int k) {
    T (*Ls)[TR + 1] = reinterpret_cast<T (*)[TR + 1]>(smem_raw);                 // Ls[t][row]
    T (*Y)[KC + 1] = reinterpret_cast<T (*)[KC + 1]>(smem_raw + sizeof(T) * NB * (TR + 1));
    const int lo = tile_slot(tile_pre, count, tile);
    const PanelDesc pd = panels[lvl_panels[lo]];
    const int w = pd.w, m = pd.m;
    const int r0 = (tile - tile_pre[lo]) * TR;
    const int nr = min(TR, m - pd.k0 - w - r0);
    const int c0 = chunk * KC, kc = min(KC, k - c0);
    const T *F = arena + pd.front_off;
    const int64_t rowbase = pd.k0 + w + r0;
    const int tid = threadIdx.x;
    // all loads before the first store to shared memory (one memory latency per item)
    constexpr int LU = NB * TR / 256, YU = NB * KC / 256;
    T lv[LU], yv[YU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u, t = q / TR, i = q % TR;
        lv[u] = (t < w && i < nr) ? F[(int64_t)(pd.k0 + t) * m + rowbase + i] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u, t = q / KC, c = q % KC;
        yv[u] = (t < w && c < kc) ? b[(int64_t)(pd.g0 + t) * k + c0 + c] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u;
        Ls[q / TR][q % TR] = lv[u];
    }
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u;
        Y[q / KC][q % KC] = yv[u];
    }
    __syncthreads();
    const int *gi = idx + pd.idx_off + rowbase;
    // thread: column c = tid % 32, rows (tid / 32) + 8 a
    const int c = tid & 31, rr = tid >> 5;
    if (c < kc) {
        for (int a = 0; a < TR / 8; ++a) {
            int i = rr + 8 * a;
            if (i >= nr) break;
            T acc = 0;
            for (int t = 0; t < w; ++t) acc += Ls[t][i] * Y[t][c];
            atomic_add_t(&b[(int64_t)gi[i] * k + c0 + c], -acc);
        }
    }
}

// FP32 forward update.  With FP32 arithmetic the one-FMA-per-two-shared-loads loop above
// is bound by shared-memory bandwidth, so each thread keeps a 4 x 2 register tile (one
// 16-byte and one 8-byte shared load per 8 FMAs) and adds with paired atomics where the
// row stride allows.
__device__ __forceinline__ void fwd_update_f32_item(unsigned char *smem_raw, int tile, int chunk,
                                                    const int32_t *__restrict__ lvl_panels,
                                                    const int32_t *__restrict__ tile_pre, int32_t count,
                                                    const PanelDesc *__restrict__ panels,
                                                    const int32_t *__restrict__ idx,
                                                    const float *__restrict__ arena, float *b, int k) {
    float (*Ls)[TR] = reinterpret_cast<float (*)[TR]>(smem_raw);                 // Ls[t][row]
    float (*Y)[KC] = reinterpret_cast<float (*)[KC]>(smem_raw + sizeof(float) * NB * TR);
    const int lo = tile_slot(tile_pre, count, tile);
    const PanelDesc pd = panels[lvl_panels[lo]];
    const int w = pd.w, m = pd.m;
    const int r0 = (tile - tile_pre[lo]) * TR;
    const int nr = min(TR, m - pd.k0 - w - r0);
    const int c0 = chunk * KC, kc = min(KC, k - c0);
    const float *F = arena + pd.front_off;
    const int64_t rowbase = pd.k0 + w + r0;
    const int tid = threadIdx.x;
    // every load of the tile is issued before the first store to shared memory, so the
    // item waits for one memory latency instead of one per loop trip
    constexpr int LU = NB * TR / 256, YU = NB * KC / 256;
    float lv[LU], yv[YU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u, t = q / TR, i = q % TR;
        lv[u] = (t < w && i < nr) ? F[(int64_t)(pd.k0 + t) * m + rowbase + i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u, t = q / KC, c = q % KC;
        yv[u] = (t < w && c < kc) ? b[(int64_t)(pd.g0 + t) * k + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u;
        Ls[q / TR][q % TR] = lv[u];
    }
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u;
        Y[q / KC][q % KC] = yv[u];
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;          // columns 2tx, 2tx+1; rows 4ty .. 4ty+3
    float acc[4][2] = {};
    for (int t = 0; t < w; ++t) {
        const float4 l = *reinterpret_cast<const float4 *>(&Ls[t][4 * ty]);
        const float2 y = *reinterpret_cast<const float2 *>(&Y[t][2 * tx]);
        acc[0][0] += l.x * y.x; acc[0][1] += l.x * y.y;
        acc[1][0] += l.y * y.x; acc[1][1] += l.y * y.y;
        acc[2][0] += l.z * y.x; acc[2][1] += l.z * y.y;
        acc[3][0] += l.w * y.x; acc[3][1] += l.w * y.y;
    }
    const int c = 2 * tx;
    if (c >= kc) return;
    const bool both = c + 1 < kc, paired = both && (k % 2 == 0);
    const int *gi = idx + pd.idx_off + rowbase;
    for (int r = 0; r < 4; ++r) {
        const int i = 4 * ty + r;
        if (i < nr) atomic_add_pair(&b[(int64_t)gi[i] * k + c0 + c], -acc[r][0], -acc[r][1], both, paired);
    }
}

// backward gather of row tile `tile`: z[slot][t][c] += sum_rows L21[row][t] x[idx[row]][c]
template <typename T>
__device__ __forceinline__ void bwd_gather_item(unsigned char *smem_raw, int tile, int chunk,
                                                const int32_t *__restrict__ lvl_panels,
                                                const int32_t *__restrict__ tile_pre, int32_t count,
                                                const PanelDesc *__restrict__ panels,
                                                const int32_t *__restrict__ idx,
                                                const T *__restrict__ arena, const T *x, int k, T *zbuf) {
    T (*Ls)[TR + 1] = reinterpret_cast<T (*)[TR + 1]>(smem_raw);
    T (*Xs)[KC + 1] = reinterpret_cast<T (*)[KC + 1]>(smem_raw + sizeof(T) * NB * (TR + 1));
    const int lo = tile_slot(tile_pre, count, tile);
    const PanelDesc pd = panels[lvl_panels[lo]];
    const int w = pd.w, m = pd.m;
    const int r0 = (tile - tile_pre[lo]) * TR;
    const int nr = min(TR, m - pd.k0 - w - r0);
    const int c0 = chunk * KC, kc = min(KC, k - c0);
    const T *F = arena + pd.front_off;
    const int64_t rowbase = pd.k0 + w + r0;
    const int *gi = idx + pd.idx_off + rowbase;
    const int tid = threadIdx.x;
    // all loads before the first store to shared memory (one memory latency per item, plus
    // one for the row indices)
    constexpr int LU = NB * TR / 256, XU = TR * KC / 256;
    T lv[LU], xv[XU];
    int gv[XU];
#pragma unroll
    for (int u = 0; u < XU; ++u) {
        const int i = (tid + 256 * u) / KC;
        gv[u] = i < nr ? gi[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u, t = q / TR, i = q % TR;
        lv[u] = (t < w && i < nr) ? F[(int64_t)(pd.k0 + t) * m + rowbase + i] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < XU; ++u) {
        const int q = tid + 256 * u, i = q / KC, c = q % KC;
        xv[u] = (i < nr && c < kc) ? x[(int64_t)gv[u] * k + c0 + c] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u;
        Ls[q / TR][q % TR] = lv[u];
    }
#pragma unroll
    for (int u = 0; u < XU; ++u) {
        const int q = tid + 256 * u;
        Xs[q / KC][q % KC] = xv[u];
    }
    __syncthreads();
    T *z = zbuf + (int64_t)lo * NB * k;
    for (int q = tid; q < w * KC; q += 256) {
        int t = q / KC, c = q % KC;
        if (c >= kc) continue;
        T acc = 0;
        for (int i = 0; i < nr; ++i) acc += Ls[t][i] * Xs[i][c];
        atomic_add_t(&z[(int64_t)t * k + c0 + c], acc);
    }
}

// FP32 backward gather with a 4 x 2 register tile per thread (see the FP32 update)
__device__ __forceinline__ void bwd_gather_f32_item(unsigned char *smem_raw, int tile, int chunk,
                                                    const int32_t *__restrict__ lvl_panels,
                                                    const int32_t *__restrict__ tile_pre, int32_t count,
                                                    const PanelDesc *__restrict__ panels,
                                                    const int32_t *__restrict__ idx,
                                                    const float *__restrict__ arena, const float *x, int k,
                                                    float *zbuf) {
    float (*Lt)[LT_LD] = reinterpret_cast<float (*)[LT_LD]>(smem_raw);          // Lt[row][t]
    float (*Xs)[KC] = reinterpret_cast<float (*)[KC]>(smem_raw + sizeof(float) * TR * LT_LD);
    const int lo = tile_slot(tile_pre, count, tile);
    const PanelDesc pd = panels[lvl_panels[lo]];
    const int w = pd.w, m = pd.m;
    const int r0 = (tile - tile_pre[lo]) * TR;
    const int nr = min(TR, m - pd.k0 - w - r0);
    const int c0 = chunk * KC, kc = min(KC, k - c0);
    const float *F = arena + pd.front_off;
    const int64_t rowbase = pd.k0 + w + r0;
    const int *gi = idx + pd.idx_off + rowbase;
    const int tid = threadIdx.x;
    // all loads first (see the FP32 update); the row indices of this thread's right-hand
    // side entries are loaded one step ahead of the entries themselves
    constexpr int LU = NB * TR / 256, XU = TR * KC / 256;
    float lv[LU], xv[XU];
    int gv[XU];
#pragma unroll
    for (int u = 0; u < XU; ++u) {
        const int i = (tid + 256 * u) / KC;
        gv[u] = i < nr ? gi[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u, t = q / TR, i = q % TR;
        lv[u] = (i < nr && t < w) ? F[(int64_t)(pd.k0 + t) * m + rowbase + i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < XU; ++u) {
        const int q = tid + 256 * u, i = q / KC, c = q % KC;
        xv[u] = (i < nr && c < kc) ? x[(int64_t)gv[u] * k + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u;
        Lt[q % TR][q / TR] = lv[u];
    }
#pragma unroll
    for (int u = 0; u < XU; ++u) {
        const int q = tid + 256 * u;
        Xs[q / KC][q % KC] = xv[u];
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;          // columns 2tx, 2tx+1; panel columns 4ty .. 4ty+3
    float acc[4][2] = {};
    for (int i = 0; i < nr; ++i) {
        const float4 l = *reinterpret_cast<const float4 *>(&Lt[i][4 * ty]);
        const float2 v = *reinterpret_cast<const float2 *>(&Xs[i][2 * tx]);
        acc[0][0] += l.x * v.x; acc[0][1] += l.x * v.y;
        acc[1][0] += l.y * v.x; acc[1][1] += l.y * v.y;
        acc[2][0] += l.z * v.x; acc[2][1] += l.z * v.y;
        acc[3][0] += l.w * v.x; acc[3][1] += l.w * v.y;
    }
    const int c = 2 * tx;
    if (c >= kc) return;
    const bool both = c + 1 < kc, paired = both && (k % 2 == 0);
    float *z = zbuf + (int64_t)lo * NB * k;
    for (int r = 0; r < 4; ++r) {
        const int t = 4 * ty + r;
        if (t < w) atomic_add_pair(&z[(int64_t)t * k + c0 + c], acc[r][0], acc[r][1], both, paired);
    }
}

// backward diagonal step of panel slot `slot`: x1 = P^T L11^-T (D^-1 y - z)
template <typename T>
__device__ __forceinline__ void bwd_diag_item(unsigned char *smem_raw, int slot, int chunk,
                                              const int32_t *__restrict__ lvl_panels,
                                              const PanelDesc *__restrict__ panels,
                                              const double *__restrict__ linv,
                                              const double *__restrict__ dblk,
                                              const int32_t *__restrict__ piv,
                                              const T *zbuf, int use_z, T *x, int k, int dinv) {
    T (*U)[KD + 1] = reinterpret_cast<T (*)[KD + 1]>(smem_raw);
    T (*Lm)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smem_raw + sizeof(T) * NB * (KD + 1));
    __shared__ double sd[NB], se[NB];
    const int p = lvl_panels[slot];
    const PanelDesc pd = panels[p];
    const int w = pd.w, c0 = chunk * KD, kc = min(KD, k - c0);
    const int tid = threadIdx.x;
    // all loads before the first store to shared memory (one memory latency per item)
    constexpr int MU = NB * NB / 256, UU = NB * KD / 256;
    double mv[MU], dv = 0.0, ev = 0.0;
    T uv[UU];
    if (tid < NB) {
        dv = dblk[(int64_t)p * 2 * NB + tid];
        ev = dblk[(int64_t)p * 2 * NB + NB + tid];
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) mv[u] = linv[(int64_t)p * NB * NB + tid + 256 * u];
#pragma unroll
    for (int u = 0; u < UU; ++u) {
        const int q = tid + 256 * u, i = q / KD, c = q % KD;
        uv[u] = (i < w && c < kc) ? x[(int64_t)(pd.g0 + i) * k + c0 + c] : (T)0;
    }
    __syncthreads();
    if (tid < NB) {
        sd[tid] = dv;
        se[tid] = ev;
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) {
        const int q = tid + 256 * u;
        Lm[q / NB][q % NB] = (T)mv[u];
    }
#pragma unroll
    for (int u = 0; u < UU; ++u) {
        const int q = tid + 256 * u;
        U[q / KD][q % KD] = uv[u];
    }
    __syncthreads();
    T val[NB * KD / 256];
    // u = Dinv y - z, each thread handles entries (i, c) with i = tid/KD + (256/KD) a
    const int c = tid % KD, rr = tid / KD;
    constexpr int RS = 256 / KD;
    for (int a = 0; a < NB * KD / 256; ++a) {
        int i = rr + RS * a;
        double u = 0.0;
        if (i < w && c < kc) {
            if (!dinv) {                            // half solve: D^-1/2 applied beforehand
                u = (double)U[i][c];
            } else if (se[i] != 0.0) {              // first row of a 2x2 block
                double A = sd[i], B = se[i], C = sd[i + 1], det = A * C - B * B;
                u = (C * (double)U[i][c] - B * (double)U[i + 1][c]) / det;
            } else if (i > 0 && se[i - 1] != 0.0) { // second row of a 2x2 block
                double A = sd[i - 1], B = se[i - 1], C = sd[i], det = A * C - B * B;
                u = (-B * (double)U[i - 1][c] + A * (double)U[i][c]) / det;
            } else {
                u = sd[i] != 0.0 ? (double)U[i][c] / sd[i] : 0.0;
            }
            if (use_z) u -= (double)zbuf[(int64_t)slot * NB * k + (int64_t)i * k + c0 + c];
        }
        val[a] = (T)u;
    }
    __syncthreads();
    for (int a = 0; a < NB * KD / 256; ++a) {
        int i = rr + RS * a;
        if (i < w) U[i][c] = val[a];
    }
    __syncthreads();
    // x'[i] = sum_{t >= i} Linv[t][i] u[t];  x[g0 + piv[i]] = x'[i]  (rows i and i + 32
    // of column cc accumulate side by side)
    {
        constexpr int RU = NB * KD / 256;
        const int cc = tid % KD, i0 = tid / KD;
        T acc[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) acc[u] = 0;
        for (int t = 0; t < w; ++t) {
            const T ut = U[t][cc];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int i = i0 + (256 / KD) * u;
                acc[u] += (t >= i) ? Lm[t][i] * ut : (T)0;
            }
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int i = i0 + (256 / KD) * u;
            if (i < w && cc < kc) x[(int64_t)(pd.g0 + piv[(int64_t)p * NB + i]) * k + c0 + cc] = acc[u];
        }
    }
}

// ---------------------------------------------------------------- one launch per step
template <typename T>
__global__ void __launch_bounds__(256) k_fwd_diag(const int32_t *__restrict__ lvl_panels,
                                                   const PanelDesc *__restrict__ panels,
                                                   const double *__restrict__ linv,
                                                   const int32_t *__restrict__ piv, T *b, int k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fwd_diag_item<T>(smem_raw, blockIdx.x, blockIdx.y, lvl_panels, panels, linv, piv, b, k);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fwd_update(const int32_t *__restrict__ lvl_panels,
                                                     const int32_t *__restrict__ tile_pre,
                                                     int32_t count, const PanelDesc *__restrict__ panels,
                                                     const int32_t *__restrict__ idx,
                                                     const T *__restrict__ arena, T *b, int k) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (std::is_same<T, float>::value)
        fwd_update_f32_item(smem_raw, blockIdx.x, blockIdx.y, lvl_panels, tile_pre, count, panels, idx, arena, b, k);
    else
        fwd_update_item<T>(smem_raw, blockIdx.x, blockIdx.y, lvl_panels, tile_pre, count, panels, idx, arena, b, k);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bwd_gather(const int32_t *__restrict__ lvl_panels,
                                                     const int32_t *__restrict__ tile_pre,
                                                     int32_t count, const PanelDesc *__restrict__ panels,
                                                     const int32_t *__restrict__ idx,
                                                     const T *__restrict__ arena, const T *x,
                                                     int k, T *zbuf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (std::is_same<T, float>::value)
        bwd_gather_f32_item(smem_raw, blockIdx.x, blockIdx.y, lvl_panels, tile_pre, count, panels, idx, arena, x, k,
                            zbuf);
    else
        bwd_gather_item<T>(smem_raw, blockIdx.x, blockIdx.y, lvl_panels, tile_pre, count, panels, idx, arena, x, k,
                           zbuf);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bwd_diag(const int32_t *__restrict__ lvl_panels,
                                                   const PanelDesc *__restrict__ panels,
                                                   const double *__restrict__ linv,
                                                   const double *__restrict__ dblk,
                                                   const int32_t *__restrict__ piv,
                                                   const T *zbuf, int use_z, T *x, int k, int dinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bwd_diag_item<T>(smem_raw, blockIdx.x, blockIdx.y, lvl_panels, panels, linv, dblk, piv, zbuf, use_z, x, k,
                     dinv);
}

// ---------------------------------------------------------------- one launch per solve
struct SweepLevel {        // device copy of a solve level
    int32_t panel_off;     // into the level-ordered panel list
    int32_t count;         // panels
    int32_t row_tiles;     // row tiles of their below-diagonal rows
    int32_t pad;
};

struct SweepArgs {
    const SweepLevel *lev;
    int32_t nlev;
    int32_t k;
    const int32_t *solve_panels;
    const int32_t *tile_pre;
    const PanelDesc *panels;
    const int32_t *idx;
    const double *linv;
    const double *dblk;
    const int32_t *piv;
    int32_t forward, backward, dinv, nsm_slots;
    GridBar *bar;
    long long limit;
    int32_t *sm_slots;     // nsm_slots zeroed counters (blocks seen per SM id), or null
    int32_t *arrive;       // fused FP32 sweep: (number of panels) x (k / KC chunks) zeroed
                           // counters of finished gather items, or null
    int32_t fuse_max;      // FP32 levels with at most this many fused items take them
};

// Position of this block in the order (rank on its SM, SM id), so that the first items
// of a step land on distinct SMs: a cooperative launch may place consecutive blocks on
// the same SM, where small steps would then share one SM's FP64 units.  Falls back to
// blockIdx.x when the SM ids exceed the counter array (the same for every block).
__device__ __forceinline__ int spread_block_id(const SweepArgs &a, bool *ok) {
    __shared__ int s_r, s_vb;
    unsigned smid, nsmid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
    const bool use = a.sm_slots != nullptr && (int)nsmid <= a.nsm_slots;
    if (use && threadIdx.x == 0) s_r = atomicAdd(&a.sm_slots[smid], 1);
    *ok = grid_barrier(a.bar, gridDim.x, a.limit);
    if (!use || !*ok) return blockIdx.x;
    if (threadIdx.x == 0) {
        const int r = s_r;
        int v = 0;
        for (int q = 0; q < (int)nsmid; ++q) {
            const int c = ((volatile int *)a.sm_slots)[q];
            v += min(c, r) + ((q < (int)smid && c > r) ? 1 : 0);
        }
        s_vb = v;
    }
    __syncthreads();
    return s_vb;
}

// ---------------------------------------------------------------- fused FP32 sweep items
// With FP32 arithmetic a solve is bound by the chain of levels, not by its flops, so the
// FP32 sweep takes one grid barrier per level and sweep instead of two:
//  * forward: every update item (row tile, KC columns) of a panel computes the panel's
//    y = L11^-1 P b1 for its own columns itself (the diagonal block's 64 x 64 x KC
//    multiply-adds, half of the update's) and pushes L21 y; the panel's first item (or its
//    only item, when no rows lie below the panel) writes y to the separate array yout, so
//    no item overwrites a b1 that another item of the level still reads;
//  * backward: the gather items of a panel count their arrivals on the panel's counter
//    (after a memory fence); the last one to arrive runs the panel's diagonal step for its
//    KC columns, reading the gathered z from L2 -- no block waits for another.
constexpr size_t fused_fwd_smem() { return sizeof(float) * (NB * (NB + 1) + 2 * NB * KC + NB * TR); }
constexpr size_t fused_bwd_smem() { return sizeof(float) * (NB * (NB + 1) + NB * KC); }
constexpr size_t fused_smem() {
    return fused_fwd_smem() > tile_solve_smem_f32() ? fused_fwd_smem() : tile_solve_smem_f32();
}

// dynamic shared memory of a k_solve_sweeps<T> launch (the FP32 kernel also runs the fused sweep)
template <typename T> constexpr size_t sweep_launch_smem() {
    return std::is_same<T, float>::value ? (sweep_smem<T>() > fused_smem() ? sweep_smem<T>() : fused_smem())
                                         : sweep_smem<T>();
}

// rows below panel slot `slot` of a level, in row tiles
__device__ __forceinline__ int slot_tiles(const int32_t *__restrict__ tile_pre, int32_t count, int32_t row_tiles,
                                          int slot) {
    return (slot + 1 < count ? tile_pre[slot + 1] : row_tiles) - tile_pre[slot];
}

// forward item: panel slot `slot`, its row tile `rt` (rt < 0: the panel has no rows below),
// right-hand-side chunk `chunk` (KC columns)
__device__ __forceinline__ void fwd_fused_f32_item(unsigned char *smem_raw, int slot, int rt, int chunk,
                                                   const int32_t *__restrict__ lvl_panels,
                                                   const PanelDesc *__restrict__ panels,
                                                   const int32_t *__restrict__ idx,
                                                   const double *__restrict__ linv,
                                                   const int32_t *__restrict__ piv,
                                                   const float *__restrict__ arena, float *b, float *yout, int k) {
    float (*Lm)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(smem_raw);
    float (*Y0)[KC] = reinterpret_cast<float (*)[KC]>(smem_raw + sizeof(float) * NB * (NB + 1));
    float (*Y)[KC] = reinterpret_cast<float (*)[KC]>(smem_raw + sizeof(float) * (NB * (NB + 1) + NB * KC));
    float (*Ls)[TR] = reinterpret_cast<float (*)[TR]>(smem_raw + sizeof(float) * (NB * (NB + 1) + 2 * NB * KC));
    const int p = lvl_panels[slot];
    const PanelDesc pd = panels[p];
    const int w = pd.w, m = pd.m;
    const int c0 = chunk * KC, kc = min(KC, k - c0);
    const int tid = threadIdx.x;
    const int r0 = rt < 0 ? 0 : rt * TR;
    const int nr = rt < 0 ? 0 : min(TR, m - pd.k0 - w - r0);
    const int64_t rowbase = pd.k0 + w + r0;
    const float *F = arena + pd.front_off;
    // every load first: L11^-1, the pivoted b1 chunk, the L21 tile
    constexpr int MU = NB * NB / 256, YU = NB * KC / 256, LU = NB * TR / 256;
    double mv[MU];
    float yv[YU], lv[LU];
    int sv[YU];
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int i = (tid + 256 * u) / KC;
        sv[u] = i < w ? piv[(int64_t)p * NB + i] : 0;
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) mv[u] = linv[(int64_t)p * NB * NB + tid + 256 * u];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u, t = q / TR, i = q % TR;
        lv[u] = (t < w && i < nr) ? F[(int64_t)(pd.k0 + t) * m + rowbase + i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u, i = q / KC, c = q % KC;
        yv[u] = (i < w && c < kc) ? b[(int64_t)(pd.g0 + sv[u]) * k + c0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < MU; ++u) {
        const int q = tid + 256 * u;
        Lm[q / NB][q % NB] = (float)mv[u];
    }
#pragma unroll
    for (int u = 0; u < YU; ++u) {
        const int q = tid + 256 * u;
        Y0[q / KC][q % KC] = yv[u];
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
        const int q = tid + 256 * u;
        Ls[q / TR][q % TR] = lv[u];
    }
    __syncthreads();
    // y = L11^-1 (P b1): thread column c, rows rr + 8 a (a warp shares its rows); the
    // eight rows accumulate side by side so their multiply-adds do not wait on each other
    {
        const int c = tid & 31, rr = tid >> 5;
        const bool write = rt <= 0 && c < kc;
        float acc[NB / 8];
#pragma unroll
        for (int a = 0; a < NB / 8; ++a) acc[a] = 0.f;
        for (int t = 0; t < w; ++t) {
            const float yt = Y0[t][c];
#pragma unroll
            for (int a = 0; a < NB / 8; ++a) {
                const int i = rr + 8 * a;
                acc[a] += (t <= i) ? Lm[i][t] * yt : 0.f;
            }
        }
#pragma unroll
        for (int a = 0; a < NB / 8; ++a) {
            const int i = rr + 8 * a;
            const float v = i < w ? acc[a] : 0.f;
            Y[i][c] = v;
            if (write && i < w) yout[(int64_t)(pd.g0 + i) * k + c0 + c] = v;
        }
    }
    if (rt < 0) return;
    __syncthreads();
    // b2 -= L21 y (the FP32 update's 4 x 2 register tile)
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][2] = {};
    for (int t = 0; t < w; ++t) {
        const float4 l = *reinterpret_cast<const float4 *>(&Ls[t][4 * ty]);
        const float2 y = *reinterpret_cast<const float2 *>(&Y[t][2 * tx]);
        acc[0][0] += l.x * y.x; acc[0][1] += l.x * y.y;
        acc[1][0] += l.y * y.x; acc[1][1] += l.y * y.y;
        acc[2][0] += l.z * y.x; acc[2][1] += l.z * y.y;
        acc[3][0] += l.w * y.x; acc[3][1] += l.w * y.y;
    }
    const int c = 2 * tx;
    if (c >= kc) return;
    const bool both = c + 1 < kc, paired = both && (k % 2 == 0);
    const int *gi = idx + pd.idx_off + rowbase;
    for (int r = 0; r < 4; ++r) {
        const int i = 4 * ty + r;
        if (i < nr) atomic_add_pair(&b[(int64_t)gi[i] * k + c0 + c], -acc[r][0], -acc[r][1], both, paired);
    }
}

// backward diagonal step of panel slot `slot` for KC columns: x1 = P^T L11^-T (D^-1 y - z),
// y read from yin (the forward sweep's output), z (when use_z) from L2
__device__ __forceinline__ void bwd_diag_kc_f32_item(unsigned char *smem_raw, int slot, int chunk,
                                                     const int32_t *__restrict__ lvl_panels,
                                                     const PanelDesc *__restrict__ panels,
                                                     const double *__restrict__ linv,
                                                     const double *__restrict__ dblk,
                                                     const int32_t *__restrict__ piv, const float *zslot,
                                                     int use_z, const float *__restrict__ yin, float *x, int k) {
    float (*Lm)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(smem_raw);
    float (*U)[KC] = reinterpret_cast<float (*)[KC]>(smem_raw + sizeof(float) * NB * (NB + 1));
    __shared__ double sd[NB], se[NB];
    const int p = lvl_panels[slot];
    const PanelDesc pd = panels[p];
    const int w = pd.w, c0 = chunk * KC, kc = min(KC, k - c0);
    const int tid = threadIdx.x;
    constexpr int MU = NB * NB / 256, UU = NB * KC / 256;
    double mv[MU], dv = 0.0, ev = 0.0;
    float uv[UU], zv[UU];
    if (tid < NB) {
        dv = dblk[(int64_t)p * 2 * NB + tid];
        ev = dblk[(int64_t)p * 2 * NB + NB + tid];
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) mv[u] = linv[(int64_t)p * NB * NB + tid + 256 * u];
#pragma unroll
    for (int u = 0; u < UU; ++u) {
        const int q = tid + 256 * u, i = q / KC, c = q % KC;
        const bool in = i < w && c < kc;
        uv[u] = in ? yin[(int64_t)(pd.g0 + i) * k + c0 + c] : 0.f;
        zv[u] = (in && use_z) ? __ldcg(zslot + (int64_t)i * k + c0 + c) : 0.f;
    }
    __syncthreads();
    if (tid < NB) {
        sd[tid] = dv;
        se[tid] = ev;
    }
#pragma unroll
    for (int u = 0; u < MU; ++u) {
        const int q = tid + 256 * u;
        Lm[q / NB][q % NB] = (float)mv[u];
    }
#pragma unroll
    for (int u = 0; u < UU; ++u) {
        const int q = tid + 256 * u;
        U[q / KC][q % KC] = uv[u];
    }
    __syncthreads();
    // u = D^-1 y - z (1x1 and 2x2 blocks of D, in FP64)
    float val[UU];
#pragma unroll
    for (int u = 0; u < UU; ++u) {
        const int q = tid + 256 * u, i = q / KC, c = q % KC;
        double v = 0.0;
        if (i < w && c < kc) {
            if (se[i] != 0.0) {                     // first row of a 2x2 block
                const double A = sd[i], B = se[i], C = sd[i + 1], det = A * C - B * B;
                v = (C * (double)U[i][c] - B * (double)U[i + 1][c]) / det;
            } else if (i > 0 && se[i - 1] != 0.0) { // second row of a 2x2 block
                const double A = sd[i - 1], B = se[i - 1], C = sd[i], det = A * C - B * B;
                v = (-B * (double)U[i - 1][c] + A * (double)U[i][c]) / det;
            } else {
                v = sd[i] != 0.0 ? (double)U[i][c] / sd[i] : 0.0;
            }
            v -= (double)zv[u];
        }
        val[u] = (float)v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < UU; ++u) {
        const int q = tid + 256 * u;
        U[q / KC][q % KC] = val[u];
    }
    __syncthreads();
    // x'[i] = sum_{t >= i} Linv[t][i] u[t];  x[g0 + piv[i]] = x'[i]
    // (the eight rows of a thread accumulate side by side, as in the forward item)
    const int c = tid & 31, rr = tid >> 5;
    float acc[NB / 8];
#pragma unroll
    for (int a = 0; a < NB / 8; ++a) acc[a] = 0.f;
    for (int t = 0; t < w; ++t) {
        const float ut = U[t][c];
#pragma unroll
        for (int a = 0; a < NB / 8; ++a) {
            const int i = rr + 8 * a;
            acc[a] += (t >= i) ? Lm[t][i] * ut : 0.f;
        }
    }
    if (c >= kc) return;
#pragma unroll
    for (int a = 0; a < NB / 8; ++a) {
        const int i = rr + 8 * a;
        if (i < w) x[(int64_t)(pd.g0 + piv[(int64_t)p * NB + i]) * k + c0 + c] = acc[a];
    }
}

// One level of the FP32 forward sweep with the fused items (see above); no barrier.
__device__ __forceinline__ void fwd_level_fused_f32(const SweepArgs &a, unsigned char *smem_raw, int vb,
                                                    const SweepLevel &lv, const float *__restrict__ arena, float *b,
                                                    float *ybuf) {
    const int k = a.k, nchunk = (k + KC - 1) / KC;
    const unsigned nb = gridDim.x;
    const int32_t *lp = a.solve_panels + lv.panel_off;
    const int32_t *tp = a.tile_pre + lv.panel_off;
    const int nup = lv.row_tiles * nchunk;
    for (int q = vb; q < nup + lv.count * nchunk; q += nb) {
        if (q < nup) {
            const int tile = q % lv.row_tiles, chunk = q / lv.row_tiles;
            const int slot = tile_slot(tp, lv.count, tile);
            __syncthreads();
            fwd_fused_f32_item(smem_raw, slot, tile - tp[slot], chunk, lp, a.panels, a.idx, a.linv, a.piv, arena, b,
                               ybuf, k);
        } else {
            const int slot = (q - nup) % lv.count, chunk = (q - nup) / lv.count;
            if (slot_tiles(tp, lv.count, lv.row_tiles, slot) > 0) continue;   // done by its tile items
            __syncthreads();
            fwd_fused_f32_item(smem_raw, slot, -1, chunk, lp, a.panels, a.idx, a.linv, a.piv, arena, b, ybuf, k);
        }
    }
}

// One level of the FP32 backward sweep with the fused items: gathers, and the diagonal
// step of each (panel, chunk) run by its last gather item; no barrier.
__device__ __forceinline__ void bwd_level_fused_f32(const SweepArgs &a, unsigned char *smem_raw, int vb,
                                                    const SweepLevel &lv, const float *__restrict__ arena, float *b,
                                                    float *zall, const float *ybuf) {
    const int k = a.k, nchunk = (k + KC - 1) / KC;
    const unsigned nb = gridDim.x;
    __shared__ int s_last;
    const int32_t *lp = a.solve_panels + lv.panel_off;
    const int32_t *tp = a.tile_pre + lv.panel_off;
    float *z = zall + (int64_t)lv.panel_off * NB * k;
    const int ngt = lv.row_tiles * nchunk;
    for (int q = vb; q < ngt + lv.count * nchunk; q += nb) {
        if (q < ngt) {
            const int tile = q % lv.row_tiles, chunk = q / lv.row_tiles;
            bwd_gather_f32_item(smem_raw, tile, chunk, lp, tp, lv.count, a.panels, a.idx, arena, b, k, z);
            // the panel's last gather item for this chunk runs its diagonal step
            const int slot = tile_slot(tp, lv.count, tile);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const int need = slot_tiles(tp, lv.count, lv.row_tiles, slot);
                const int old = atomicAdd(&a.arrive[(int64_t)(lv.panel_off + slot) * nchunk + chunk], 1);
                s_last = old == need - 1;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                bwd_diag_kc_f32_item(smem_raw, slot, chunk, lp, a.panels, a.linv, a.dblk, a.piv,
                                     z + (int64_t)slot * NB * k, 1, ybuf, b, k);
            }
        } else {
            const int slot = (q - ngt) % lv.count, chunk = (q - ngt) / lv.count;
            if (slot_tiles(tp, lv.count, lv.row_tiles, slot) > 0) continue;   // done by its last gather
            __syncthreads();
            bwd_diag_kc_f32_item(smem_raw, slot, chunk, lp, a.panels, a.linv, a.dblk, a.piv, nullptr, 0, ybuf, b, k);
        }
    }
}

// whether level lv of an FP32 solve takes the fused items: only levels whose items all
// fit in one pass of the resident blocks (a level with more items is bound by the items'
// throughput, where the fused items' extra work costs more than the barrier it saves)
__device__ __forceinline__ bool level_fused(const SweepArgs &a, const SweepLevel &lv, int nchunk) {
    return a.arrive != nullptr && (int64_t)(lv.row_tiles + lv.count) * nchunk <= a.fuse_max;
}

// Forward and/or backward sweep over every level in one cooperative launch.  The work
// items of a step are spread over the resident blocks; a grid barrier separates
// consecutive steps.  zall: (number of panels) x NB x k, zero on entry (each level
// gathers into its own slots).  On a barrier timeout bar->err is set and every block
// returns.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_solve_sweeps(SweepArgs a, const T *__restrict__ arena, T *b, T *zall,
                                                         T *ybuf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = a.k;
    const int nchunk = (k + KC - 1) / KC, ndchunk = (k + KD - 1) / KD;
    const unsigned nb = gridDim.x;
    bool ok = true;
    const int vb = spread_block_id(a, &ok);
    if (!ok) return;
    if (a.forward) {
        for (int L = 0; L < a.nlev; ++L) {
            const SweepLevel lv = a.lev[L];
            const int32_t *lp = a.solve_panels + lv.panel_off;
            if constexpr (std::is_same<T, float>::value) {
                if (level_fused(a, lv, nchunk)) {       // y of this level goes to ybuf
                    fwd_level_fused_f32(a, smem_raw, vb, lv, arena, b, ybuf);
                    if (!grid_barrier(a.bar, nb, a.limit)) return;
                    continue;
                }
            }
            for (int q = vb; q < lv.count * ndchunk; q += nb)
                fwd_diag_item<T>(smem_raw, q % lv.count, q / lv.count, lp, a.panels, a.linv, a.piv, b, k);
            if (!grid_barrier(a.bar, nb, a.limit)) return;
            if (lv.row_tiles == 0) continue;
            const int32_t *tp = a.tile_pre + lv.panel_off;
            for (int q = vb; q < lv.row_tiles * nchunk; q += nb) {
                if constexpr (std::is_same<T, float>::value)
                    fwd_update_f32_item(smem_raw, q % lv.row_tiles, q / lv.row_tiles, lp, tp, lv.count, a.panels,
                                        a.idx, arena, b, k);
                else
                    fwd_update_item<T>(smem_raw, q % lv.row_tiles, q / lv.row_tiles, lp, tp, lv.count, a.panels,
                                       a.idx, arena, b, k);
            }
            if (!grid_barrier(a.bar, nb, a.limit)) return;
        }
    }
    if (!a.backward) return;
    for (int L = a.nlev - 1; L >= 0; --L) {
        const SweepLevel lv = a.lev[L];
        const int32_t *lp = a.solve_panels + lv.panel_off;
        T *z = zall + (int64_t)lv.panel_off * NB * k;
        if constexpr (std::is_same<T, float>::value) {
            if (level_fused(a, lv, nchunk)) {
                bwd_level_fused_f32(a, smem_raw, vb, lv, arena, b, zall, ybuf);
                if (L > 0 && !grid_barrier(a.bar, nb, a.limit)) return;
                continue;
            }
        }
        if (lv.row_tiles > 0) {
            const int32_t *tp = a.tile_pre + lv.panel_off;
            for (int q = vb; q < lv.row_tiles * nchunk; q += nb) {
                if constexpr (std::is_same<T, float>::value)
                    bwd_gather_f32_item(smem_raw, q % lv.row_tiles, q / lv.row_tiles, lp, tp, lv.count, a.panels,
                                        a.idx, arena, b, k, z);
                else
                    bwd_gather_item<T>(smem_raw, q % lv.row_tiles, q / lv.row_tiles, lp, tp, lv.count, a.panels,
                                       a.idx, arena, b, k, z);
            }
            if (!grid_barrier(a.bar, nb, a.limit)) return;
        }
        for (int q = vb; q < lv.count * ndchunk; q += nb)
            bwd_diag_item<T>(smem_raw, q % lv.count, q / lv.count, lp, a.panels, a.linv, a.dblk, a.piv, z,
                             lv.row_tiles > 0 ? 1 : 0, b, k, a.dinv);
        if (L > 0 && !grid_barrier(a.bar, nb, a.limit)) return;
    }
}

// y <- D^-1/2 y for every panel (SPD factor: 1x1 blocks d > 0, 2x2 blocks E with the
// symmetric inverse square root E^-1/2 = [c+s, -b; -b, a+s] / (s t), s = sqrt(det E),
// t = sqrt(a + c + 2 s)); y in the permuted order, N x k, written to yo.
template <typename T>
__global__ void k_dhalf(int64_t n, const int32_t *__restrict__ col_panel, const PanelDesc *__restrict__ panels,
                        const double *__restrict__ dblk, const T *__restrict__ y, T *__restrict__ yo, int k) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * k) return;
    const int64_t i = q / k;
    const int c = (int)(q - i * k);
    const int p = col_panel[i];
    const int li = (int)(i - panels[p].g0);
    const double *dd = dblk + (int64_t)p * 2 * NB, *de = dd + NB;
    double out;
    if (de[li] != 0.0 || (li > 0 && de[li - 1] != 0.0)) {
        const int f = de[li] != 0.0 ? li : li - 1;            // first row of the 2x2 block
        const double a = dd[f], b = de[f], cc = dd[f + 1];
        const double sd = sqrt(a * cc - b * b), t = sqrt(a + cc + 2.0 * sd);
        const double y0 = (double)y[(i - (li - f)) * k + c], y1 = (double)y[(i - (li - f) + 1) * k + c];
        out = (li == f) ? ((cc + sd) * y0 - b * y1) / (sd * t) : (-b * y0 + (a + sd) * y1) / (sd * t);
    } else {
        out = (double)y[q] / sqrt(dd[li]);
    }
    yo[q] = (T)out;
}

// row permutation: mode 0 gather dst[i] = src[perm[i]]; 1 scatter dst[perm[i]] = src[i];
// 2 scatter-add dst[perm[i]] += src[i]
template <typename TD, typename TS>
__global__ void k_permute_rows(int64_t n, int k, const int32_t *__restrict__ perm,
                               const TS *__restrict__ src, TD *dst, int mode) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * k) return;
    int64_t i = q / k;
    int c = (int)(q - i * k);
    int64_t j = perm[i];
    if (mode == 1) dst[j * k + c] = (TD)src[q];
    else if (mode == 2) dst[j * k + c] += (TD)src[q];
    else dst[q] = (TD)src[j * k + c];
}

}  // namespace ssk
