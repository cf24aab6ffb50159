// Numeric multifrontal LDL^T kernels (Alg. 2 step 2: (L, D) <- LDL^T of A - sigma B).
//
// A front is a dense column-major m x m block in the level workspace; only its lower
// triangle is meaningful.  Its first ncol columns are eliminated in panels of width
// w <= 64; each panel step is
//   K2 diag:  FP64 Bunch-Kaufman on the w x w diagonal block, pivots restricted to the
//             block: P F11 P^T = L D L^T.  Writes L^-1, D, the local pivot order and
//             the transform Mt = P^T L^-T D^-1, and counts the inertia of D.
//   K4 panel: L21 = F21 Mt (in place) and W = L21 D (scratch), 64-row tiles.
//   K3 Schur: F22 -= L21 W^T on the lower-triangular 64 x 64 tiles of the trailing front.
// Before a level's steps its fronts are zeroed, the stored entries of A - sigma B are
// scattered in (assembly) and the children's contribution blocks are added from the pool
// (extend-add, one pass per child slot so that no two blocks of a pass write the same
// parent entry).  After them the fronts' panel columns go to L storage and their trailing
// blocks to the pool (store), so the workspace holds one level at a time.
// Every kernel is batched over shifts with blockIdx.y.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace ssk {

constexpr int NB = 64;     // panel width
constexpr int TR = 64;     // row tile of the panel transform / Schur update
constexpr size_t kDiagSmem = 2 * NB * (NB + 1) * sizeof(double);
template <typename T> constexpr size_t panel_smem() { return 3 * NB * (TR + 1) * sizeof(T); }
template <typename T> constexpr size_t schur_smem() { return 2 * NB * (TR + 1) * sizeof(T); }

template <typename T>
struct ShiftPtrs {
    const double *a, *b;            // pencil values on the pattern (caller-owned)
    T *ws;                          // level workspace (fronts of the level being factored)
    T *cb;                          // contribution-block pool
    T *lst;                         // L storage (null: inertia only, nothing kept)
    double *linv;                   // npanels * NB * NB, row-major L^-1 of each panel
    double *dblk;                   // npanels * 2 * NB: D diagonal then sub-diagonal
    int32_t *piv;                   // npanels * NB
    T *mt;                          // mt_max * NB * NB
    T *wbuf;                        // wbuf_max
    unsigned char *sl;              // operand slices of the tensor-core Schur update
    int32_t *ex;                    // their row exponents
    unsigned long long *counts;     // [neg, zero, pos, tiny, min_pivot_bits, n2x2, max_abs_l_bits, timeouts]
    const double *seg_sigma;        // several pencils in one block-diagonal pattern: the shift
    const int32_t *eseg;            // of each pencil (seg_sigma) and the pencil of each stored
                                    // entry (eseg); null for one pencil (sigma)
    double sigma;
    double tiny_thr;                // pivots below this are flagged
    double norm;                    // ||A - sigma B||_1 bound (for min-pivot ratio)
};

// ---------------------------------------------------------------- assembly
template <typename T>
__global__ void k_assemble(int64_t count, const int32_t *__restrict__ asm_e,
                           const int64_t *__restrict__ asm_dest, const ShiftPtrs<T> *sp) {
    const ShiftPtrs<T> s = sp[blockIdx.y];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = asm_e[q];
        const double sg = s.eseg ? s.seg_sigma[s.eseg[e]] : s.sigma;
        s.ws[asm_dest[q]] = (T)(s.a[e] - sg * s.b[e]);
    }
}

// Inertia of D per pencil of a block-diagonal pattern: every panel's 1x1 and 2x2 pivots
// (the classification of k_diag_bk) counted for the pencil its rows belong to.  seg:
// pencil of each original row; perm: permuted -> original row; out: n_seg x 4
// (neg, zero, pos, tiny).
__global__ void k_segment_inertia(int32_t npan, const PanelDesc *__restrict__ panels,
                                  const double *__restrict__ dblk, const int32_t *__restrict__ perm,
                                  const int32_t *__restrict__ seg, double tiny_thr,
                                  unsigned long long *__restrict__ out) {
    const int p = blockIdx.x;
    if (p >= npan) return;
    const PanelDesc pd = panels[p];
    const int i = threadIdx.x;
    if (i >= pd.w) return;
    const double *dd = dblk + (int64_t)p * 2 * NB, *de = dd + NB;
    unsigned long long *o = out + 4ll * seg[perm[pd.g0]];
    if (i > 0 && de[i - 1] != 0.0) return;                 // second row of a 2x2 block
    if (de[i] != 0.0) {                                     // 2x2 block (i, i+1)
        const double a = dd[i], b = de[i], c = dd[i + 1], det = a * c - b * b, tr = a + c;
        if (det < 0) { atomicAdd(&o[0], 1ull); atomicAdd(&o[2], 1ull); }
        else if (det > 0) atomicAdd(&o[tr > 0 ? 2 : 0], 2ull);
        else { atomicAdd(&o[1], 1ull); atomicAdd(&o[tr > 0 ? 2 : (tr < 0 ? 0 : 1)], 1ull); }
        const double emax = fabs(0.5 * tr) + sqrt(0.25 * (a - c) * (a - c) + b * b);
        const double emin = emax > 0 ? fabs(det) / emax : 0.0;
        if (emin < tiny_thr) atomicAdd(&o[3], 1ull);
    } else {
        const double d = dd[i];
        atomicAdd(&o[d < 0 ? 0 : (d > 0 ? 2 : 1)], 1ull);
        if (fabs(d) < tiny_thr) atomicAdd(&o[3], 1ull);
    }
}

// ---------------------------------------------------------------- extend-add
// One block per contribution column: parent[rel[i], rel[j]] += cb[i, j], i >= j.  A block
// in the pool is its lower triangle packed by columns: column j (rows j .. nr-1) starts
// at j (2 nr - j + 1) / 2.
template <typename T>
__global__ void k_extend_add(const ExtendTask *__restrict__ tasks, int32_t ntask,
                             const int32_t *__restrict__ relmap, const ShiftPtrs<T> *sp) {
    const ShiftPtrs<T> s = sp[blockIdx.y];
    const int32_t col = blockIdx.x;
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].col_pre <= col) lo = mid; else hi = mid - 1;
    }
    const ExtendTask t = tasks[lo];
    const int32_t j = col - t.col_pre;
    const int32_t nr = t.child_m - t.child_ncol;
    const int32_t *rel = relmap + t.rel_off;
    const T *cc = s.cb + t.child_off + (int64_t)j * (2 * (int64_t)nr - j - 1) / 2;   // cc[i]: row i >= j
    T *pc = s.ws + t.parent_off + (int64_t)rel[j] * t.parent_m;
    for (int32_t i = j + threadIdx.x; i < nr; i += blockDim.x) pc[rel[i]] += cc[i];
}

// ---------------------------------------------------------------- store
// One block per front column of a level: column c < ncol to L storage (all m rows),
// column ncol + j to the contribution-block pool (rows j .. nr-1, packed lower triangle).
template <typename T>
__global__ void k_level_store(const StoreTask *__restrict__ tasks, int32_t ntask, const ShiftPtrs<T> *sp) {
    const ShiftPtrs<T> s = sp[blockIdx.y];
    const int32_t col = blockIdx.x;
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].col_pre <= col) lo = mid; else hi = mid - 1;
    }
    const StoreTask t = tasks[lo];
    const int32_t c = col - t.col_pre;
    const T *src = s.ws + t.ws_off + (int64_t)c * t.m;
    if (c < t.ncol) {
        if (!s.lst) return;
        T *dst = s.lst + t.l_off + (int64_t)c * t.m;
        for (int32_t i = threadIdx.x; i < t.m; i += blockDim.x) dst[i] = src[i];
    } else {
        const int32_t j = c - t.ncol, nr = t.m - t.ncol;
        T *dst = s.cb + t.cb_off + (int64_t)j * (2 * (int64_t)nr - j - 1) / 2;    // dst[i]: row i >= j
        src += t.ncol;
        for (int32_t i = j + threadIdx.x; i < nr; i += blockDim.x) dst[i] = src[i];
    }
}

// ---------------------------------------------------------------- K2: diagonal block
// Dynamic shared memory: 2 * NB * (NB + 1) doubles.
template <typename T>
__global__ void __launch_bounds__(256) k_diag_bk(const StepTask *__restrict__ tasks,
                                                  const ShiftPtrs<T> *sp, int nopivot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *smem = reinterpret_cast<double *>(smem_raw);
    const ShiftPtrs<T> s = sp[blockIdx.y];
    const StepTask tk = tasks[blockIdx.x];
    const int w = tk.w, m = tk.m, k0 = tk.k0;
    constexpr int LD = NB + 1;
    double *A = smem;                  // w x w full symmetric, row i at A[i*LD]
    double *Li = smem + NB * LD;       // L^-1
    __shared__ int perm[NB];
    __shared__ double dd[NB], de[NB];
    __shared__ int s_kind, s_r;        // pivot decision
    __shared__ double s_lam;
    __shared__ unsigned long long c_neg, c_zero, c_pos, c_tiny, c_2x2;
    __shared__ double s_minpiv;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T *F = s.ws + tk.front_off;

    for (int q = tid; q < w * w; q += nt) {
        int j = q / w, i = q % w;            // column j, row i (coalesced on i)
        if (i >= j) {
            double v = (double)F[(int64_t)(k0 + j) * m + (k0 + i)];
            A[i * LD + j] = v;
            A[j * LD + i] = v;
        }
    }
    if (tid < NB) { perm[tid] = tid; dd[tid] = 0.0; de[tid] = 0.0; }
    if (tid == 0) { c_neg = c_zero = c_pos = c_tiny = c_2x2 = 0; s_minpiv = 1e300; }
    __syncthreads();

    const double alpha = 0.6403882032022076;   // (1 + sqrt(17)) / 8
    int k = 0;
    while (k < w) {
        if (tid < 32) {
            // lambda = max_{i>k} |A[i][k]|, r = its row (first on ties)
            double lam = -1.0;
            int r = k;
            for (int i = k + 1 + tid; i < w; i += 32) {
                double v = fabs(A[i * LD + k]);
                if (v > lam) { lam = v; r = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                double ol = __shfl_down_sync(0xffffffffu, lam, o);
                int orr = __shfl_down_sync(0xffffffffu, r, o);
                if (ol > lam || (ol == lam && orr < r)) { lam = ol; r = orr; }
            }
            lam = __shfl_sync(0xffffffffu, lam, 0);
            r = __shfl_sync(0xffffffffu, r, 0);
            if (lam < 0.0) lam = 0.0;
            double akk = fabs(A[k * LD + k]);
            int kind = 1;                        // 1: 1x1 at k; 2: 1x1 with swap k<->r; 3: 2x2 (k+1<->r)
            if (!nopivot && akk < alpha * lam) {
                double sig = 0.0;
                for (int j = k + tid; j < w; j += 32)
                    if (j != r) sig = fmax(sig, fabs(A[r * LD + j]));
                for (int o = 16; o > 0; o >>= 1) sig = fmax(sig, __shfl_down_sync(0xffffffffu, sig, o));
                sig = __shfl_sync(0xffffffffu, sig, 0);
                if (akk * sig >= alpha * lam * lam) kind = 1;
                else if (fabs(A[r * LD + r]) >= alpha * sig) kind = 2;
                else kind = 3;
            }
            if (tid == 0) { s_kind = kind; s_r = r; s_lam = lam; }
        }
        __syncthreads();
        const int kind = s_kind, r = s_r;
        if (kind >= 2) {
            const int a = (kind == 2) ? k : k + 1;
            if (a != r) {
                for (int j = tid; j < w; j += nt) {
                    double t = A[a * LD + j]; A[a * LD + j] = A[r * LD + j]; A[r * LD + j] = t;
                }
                __syncthreads();
                for (int i = tid; i < w; i += nt) {
                    double t = A[i * LD + a]; A[i * LD + a] = A[i * LD + r]; A[i * LD + r] = t;
                }
                if (tid == 0) { int t = perm[a]; perm[a] = perm[r]; perm[r] = t; }
                __syncthreads();
            }
        }
        if (kind <= 2) {
            const double d = A[k * LD + k];
            if (tid == 0) {
                dd[k] = d;
                double ad = fabs(d);
                if (d < 0) c_neg++; else if (d > 0) c_pos++; else c_zero++;
                if (ad < s.tiny_thr) c_tiny++;
                if (ad < s_minpiv) s_minpiv = ad;
            }
            const int rem = w - k - 1;
            if (d != 0.0) {
                const double inv = 1.0 / d;
                for (int q = tid; q < rem * rem; q += nt) {
                    int i = k + 1 + q / rem, j = k + 1 + q % rem;
                    A[i * LD + j] -= A[i * LD + k] * inv * A[j * LD + k];
                }
                __syncthreads();
                for (int i = k + 1 + tid; i < w; i += nt) A[i * LD + k] *= inv;
            } else {
                for (int i = k + 1 + tid; i < w; i += nt) A[i * LD + k] = 0.0;
            }
            __syncthreads();
            k += 1;
        } else {
            const double a = A[k * LD + k], b = A[(k + 1) * LD + k], c = A[(k + 1) * LD + k + 1];
            const double det = a * c - b * b;
            if (tid == 0) {
                dd[k] = a; dd[k + 1] = c; de[k] = b; de[k + 1] = 0.0;
                c_2x2++;
                double tr = a + c;
                if (det < 0) { c_neg++; c_pos++; }
                else if (det > 0) { if (tr > 0) c_pos += 2; else c_neg += 2; }
                else { c_zero++; if (tr > 0) c_pos++; else if (tr < 0) c_neg++; else c_zero++; }
                double emax = fabs(0.5 * tr) + sqrt(0.25 * (a - c) * (a - c) + b * b);
                double emin = emax > 0 ? fabs(det) / emax : 0.0;
                if (emin < s.tiny_thr) c_tiny++;
                if (emin < s_minpiv) s_minpiv = emin;
            }
            const int rem = w - k - 2;
            const double id = 1.0 / det;
            for (int q = tid; q < rem * rem; q += nt) {
                int i = k + 2 + q / rem, j = k + 2 + q % rem;
                double ci0 = A[i * LD + k], ci1 = A[i * LD + k + 1];
                double li0 = (c * ci0 - b * ci1) * id, li1 = (-b * ci0 + a * ci1) * id;
                A[i * LD + j] -= li0 * A[j * LD + k] + li1 * A[j * LD + k + 1];
            }
            __syncthreads();
            for (int i = k + 2 + tid; i < w; i += nt) {
                double ci0 = A[i * LD + k], ci1 = A[i * LD + k + 1];
                A[i * LD + k] = (c * ci0 - b * ci1) * id;
                A[i * LD + k + 1] = (-b * ci0 + a * ci1) * id;
            }
            if (tid == 0) A[(k + 1) * LD + k] = 0.0;   // the 2x2 coupling lives in D, not L
            __syncthreads();
            k += 2;
        }
    }
    // L^-1 of the unit lower triangle, one column per thread
    if (tid < w) {
        const int j = tid;
        for (int i = 0; i < j; ++i) Li[i * LD + j] = 0.0;
        Li[j * LD + j] = 1.0;
        for (int i = j + 1; i < w; ++i) {
            double acc = 0.0;
            for (int t = j; t < i; ++t) acc -= A[i * LD + t] * Li[t * LD + j];
            Li[i * LD + j] = acc;
        }
    }
    __syncthreads();
    const int p = tk.panel;
    double *linv = s.linv + (int64_t)p * NB * NB;
    for (int q = tid; q < NB * NB; q += nt) {
        int i = q / NB, j = q % NB;
        linv[q] = (i < w && j < w) ? Li[i * LD + j] : 0.0;
    }
    if (tid < NB) {
        s.dblk[(int64_t)p * 2 * NB + tid] = tid < w ? dd[tid] : 0.0;
        s.dblk[(int64_t)p * 2 * NB + NB + tid] = tid < w ? de[tid] : 0.0;
        s.piv[(int64_t)p * NB + tid] = tid < w ? perm[tid] : tid;
    }
    // Mt[perm[i]][j] = sum_{t in block(j)} Li[t][i] Dinv[t][j]
    T *mt = s.mt + (int64_t)tk.mt_slot * NB * NB;
    for (int q = tid; q < w * w; q += nt) {
        int i = q / w, j = q % w;
        double v;
        bool first2 = (de[j] != 0.0);                    // j is the first row of a 2x2 block
        bool second2 = (j > 0 && de[j - 1] != 0.0);      // j is the second row
        if (first2) {
            double a = dd[j], b = de[j], c = dd[j + 1], det = a * c - b * b;
            v = (Li[j * LD + i] * c - Li[(j + 1) * LD + i] * b) / det;
        } else if (second2) {
            double a = dd[j - 1], b = de[j - 1], c = dd[j], det = a * c - b * b;
            v = (-Li[(j - 1) * LD + i] * b + Li[j * LD + i] * a) / det;
        } else {
            v = dd[j] != 0.0 ? Li[j * LD + i] / dd[j] : 0.0;
        }
        mt[perm[i] * NB + j] = (T)v;
    }
    if (tid == 0) {
        atomicAdd(&s.counts[0], c_neg);
        atomicAdd(&s.counts[1], c_zero);
        atomicAdd(&s.counts[2], c_pos);
        if (c_tiny) atomicAdd(&s.counts[3], c_tiny);
        double ratio = s_minpiv / (s.norm > 0 ? s.norm : 1.0);
        atomicMin(&s.counts[4], (unsigned long long)__double_as_longlong(ratio));
        if (c_2x2) atomicAdd(&s.counts[5], c_2x2);
    }
    // largest |L| entry of the diagonal block (element growth diagnostic)
    double lmax = 0.0;
    for (int q = tid; q < w * w; q += nt) {
        int i = q / w, j = q % w;
        if (i > j) lmax = fmax(lmax, fabs(A[i * LD + j]));
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_down_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0 && lmax > 0.0) atomicMax(&s.counts[6], (unsigned long long)__double_as_longlong(lmax));
}

// ---------------------------------------------------------------- K4: panel transform
// Block = (task, 64-row tile).  L21 = F21 Mt written in place; W = L21 D to scratch.
// Dynamic shared memory: 3 * NB * (TR + 1) * sizeof(T).
template <typename T>
__global__ void __launch_bounds__(256) k_panel(const StepTask *__restrict__ tasks, int32_t ntask,
                                                const ShiftPtrs<T> *sp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*Fs)[TR + 1] = reinterpret_cast<T (*)[TR + 1]>(smem_raw);                // Fs[t][row]
    T (*Ms)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smem_raw + sizeof(T) * NB * (TR + 1));
    T (*Ls)[TR + 1] = reinterpret_cast<T (*)[TR + 1]>(smem_raw + 2 * sizeof(T) * NB * (TR + 1));
    __shared__ double sd[NB], se[NB];
    const ShiftPtrs<T> s = sp[blockIdx.y];
    const int32_t tile = blockIdx.x;
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tiles4_pre <= tile) lo = mid; else hi = mid - 1;
    }
    const StepTask tk = tasks[lo];
    const int w = tk.w, m = tk.m;
    const int r0 = (tile - tk.tiles4_pre) * TR;           // first row within the r rows
    const int nr = min(TR, tk.r - r0);
    T *F = s.ws + tk.front_off;
    const int64_t rowbase = tk.k0 + w + r0;
    const T *mt = s.mt + (int64_t)tk.mt_slot * NB * NB;
    const int tid = threadIdx.x;
    for (int q = tid; q < w * TR; q += 256) {
        int t = q / TR, i = q % TR;
        Fs[t][i] = i < nr ? F[(int64_t)(tk.k0 + t) * m + rowbase + i] : (T)0;
    }
    for (int q = tid; q < w * w; q += 256) Ms[q / w][q % w] = mt[(q / w) * NB + (q % w)];
    if (tid < NB) {
        sd[tid] = tid < w ? s.dblk[(int64_t)tk.panel * 2 * NB + tid] : 0.0;
        se[tid] = tid < w ? s.dblk[(int64_t)tk.panel * 2 * NB + NB + tid] : 0.0;
    }
    __syncthreads();
    // each thread: rows i = tx + 16*a, cols j = ty + 16*b, a,b in 0..3
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int t = 0; t < w; ++t) {
        T fa[4], mb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) fa[a] = Fs[t][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) mb[b] = Ms[t][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += fa[a] * mb[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) Ls[ty + 16 * b][tx + 16 * a] = acc[a][b];
    __syncthreads();
    T *W = s.wbuf + tk.wbuf_off;
    double lmax = 0.0;
    for (int q = tid; q < w * TR; q += 256) {
        int j = q / TR, i = q % TR;
        if (i >= nr) continue;
        T l = Ls[j][i];
        lmax = fmax(lmax, fabs((double)l));
        F[(int64_t)(tk.k0 + j) * m + rowbase + i] = l;
        double wv = (double)l * sd[j];
        if (se[j] != 0.0) wv += (double)Ls[j + 1][i] * se[j];
        if (j > 0 && se[j - 1] != 0.0) wv += (double)Ls[j - 1][i] * se[j - 1];
        W[(int64_t)j * tk.r + r0 + i] = (T)wv;
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_down_sync(0xffffffffu, lmax, o));
    if ((tid & 31) == 0 && lmax > 0.0) atomicMax(&s.counts[6], (unsigned long long)__double_as_longlong(lmax));
}

// ---------------------------------------------------------------- K3: Schur update
// Block = (task, lower-triangular tile pair).  C[i][j] -= sum_t L21[i][t] W[j][t].
// Dynamic shared memory: 2 * NB * (TR + 1) * sizeof(T).
template <typename T>
__global__ void __launch_bounds__(256) k_schur(const StepTask *__restrict__ tasks, int32_t ntask,
                                                const ShiftPtrs<T> *sp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*As)[TR + 1] = reinterpret_cast<T (*)[TR + 1]>(smem_raw);                // As[t][i] = L21[i][t]
    T (*Bs)[TR + 1] = reinterpret_cast<T (*)[TR + 1]>(smem_raw + sizeof(T) * NB * (TR + 1));
    const ShiftPtrs<T> s = sp[blockIdx.y];
    const int32_t tile = blockIdx.x;
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tiles3_pre <= tile) lo = mid; else hi = mid - 1;
    }
    const StepTask tk = tasks[lo];
    const int q = tile - tk.tiles3_pre;
    int bi = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
    while (bi * (bi + 1) / 2 > q) --bi;
    const int bj = q - bi * (bi + 1) / 2;
    const int w = tk.w, m = tk.m, r = tk.r;
    const int i0 = bi * TR, j0 = bj * TR;
    const int ni = min(TR, r - i0), nj = min(TR, r - j0);
    T *F = s.ws + tk.front_off;
    const T *W = s.wbuf + tk.wbuf_off;
    const int64_t base = tk.k0 + w;               // first trailing row/col in the front
    const int tid = threadIdx.x;
    for (int e = tid; e < w * TR; e += 256) {
        int t = e / TR, i = e % TR;
        As[t][i] = i < ni ? F[(int64_t)(tk.k0 + t) * m + base + i0 + i] : (T)0;
        Bs[t][i] = i < nj ? W[(int64_t)t * r + j0 + i] : (T)0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int t = 0; t < w; ++t) {
        T fa[4], fb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) fa[a] = As[t][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) fb[b] = Bs[t][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += fa[a] * fb[b];
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int j = ty + 16 * b;
        if (j >= nj) continue;
        T *col = F + (base + j0 + j) * (int64_t)m + base + i0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int i = tx + 16 * a;
            if (i < ni && i0 + i >= j0 + j) col[i] -= acc[a][b];
        }
    }
}

}  // namespace ssk
