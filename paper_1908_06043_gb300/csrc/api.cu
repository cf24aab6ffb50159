// C ABI: context, symbolic upload, numeric factorisation, inertia, solves, SpMM, gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "factor_kernels.cuh"
#include "internal.h"
#include "solve_kernels.cuh"
#include "sparse_kernels.cuh"
#include "tc_kernels.cuh"

using namespace ssk;

// ------------------------------------------------------------------ launch accounting
std::atomic<int64_t> g_ss_launches{0};

size_t ss_prof_begin(ss_ctx *ctx, int cls) {
    size_t slot = 2 * ctx->ev_used.size();
    while (ctx->ev_pool.size() < slot + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ctx->ev_pool.push_back(e);
    }
    ctx->ev_used.push_back({cls, slot});
    cudaEventRecord(ctx->ev_pool[slot], ctx->stream);
    return slot;
}

void ss_prof_end(ss_ctx *ctx, int cls, size_t slot) {
    (void)cls;
    cudaEventRecord(ctx->ev_pool[slot + 1], ctx->stream);
}

extern "C" int64_t ss_launch_count(void) { return g_ss_launches.load(); }

static void prof_collect(ss_ctx *ctx) {
    for (auto &u : ctx->ev_used) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[u.second], ctx->ev_pool[u.second + 1]) == cudaSuccess) {
            ctx->prof_launches[u.first] += 1;
            ctx->prof_seconds[u.first] += ms * 1e-3;
        }
    }
    ctx->ev_used.clear();
}

extern "C" ss_status ss_profile(ss_ctx *ctx, uint32_t mask) {
    if (!ctx) return SS_ERR_ARG;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "host-only context");
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->ev_used.clear();
    for (int c = 0; c < SS_K_COUNT; ++c) {
        ctx->prof_launches[c] = 0;
        ctx->prof_seconds[c] = 0.0;
        ctx->prof_flops[c] = 0.0;
        ctx->prof_tensor_flops[c] = 0.0;
    }
    ctx->prof_mask = mask;
    return SS_OK;
}

extern "C" ss_status ss_profile_query(ss_ctx *ctx, int32_t cls, int64_t *launches, double *seconds, double *flops) {
    if (!ctx || cls < 0 || cls >= SS_K_COUNT) return SS_ERR_ARG;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "host-only context");
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    if (launches) *launches = ctx->prof_launches[cls];
    if (seconds) *seconds = ctx->prof_seconds[cls];
    if (flops) *flops = ctx->prof_flops[cls];
    return SS_OK;
}

extern "C" ss_status ss_profile_query_tensor(ss_ctx *ctx, int32_t cls, double *tensor_flops) {
    if (!ctx || cls < 0 || cls >= SS_K_COUNT || !tensor_flops) return SS_ERR_ARG;
    *tensor_flops = ctx->prof_tensor_flops[cls];
    return SS_OK;
}

// ------------------------------------------------------------------ context
extern "C" ss_status ss_create(ss_ctx **ctx, int32_t device, void *cuda_stream) {
    if (!ctx) return SS_ERR_ARG;
    *ctx = nullptr;
    ss_ctx *c = new (std::nothrow) ss_ctx();
    if (!c) return SS_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (device == -1) {            // host-only context: symbolic analysis without a GPU
        *ctx = c;
        return SS_OK;
    }
    if (device < 0 || cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return SS_ERR_CUDA;
    }
    *ctx = c;
    return SS_OK;
}

extern "C" ss_status ss_destroy(ss_ctx *ctx) {
    delete ctx;
    return SS_OK;
}

extern "C" const char *ss_last_error(const ss_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// every block waits at one grid barrier that expects `expected` arrivals
__global__ void k_barrier_selftest(GridBar *bar, unsigned int expected, long long limit) {
    grid_barrier(bar, expected, limit);
}

extern "C" ss_status ss_selftest_barrier(ss_ctx *ctx, int32_t extra_arrivals, int64_t limit) {
    if (!ctx) return SS_ERR_ARG;
    if (ctx->device < 0 || extra_arrivals < 0 || extra_arrivals > 1 || limit <= 0 || limit > 100000000)
        return ctx->set_error(SS_ERR_ARG, "ss_selftest_barrier: bad argument or host-only context");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    GridBar *bar = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&bar, sizeof(GridBar), st));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, sizeof(GridBar), st));
    const unsigned int nb = (unsigned int)ctx->sm_count;          // one block per SM: resident
    unsigned int expected = nb + (unsigned int)extra_arrivals;
    long long lim = limit;
    void *args[] = {(void *)&bar, (void *)&expected, (void *)&lim};
    g_ss_launches.fetch_add(1, std::memory_order_relaxed);
    SS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void *)k_barrier_selftest, dim3(nb), dim3(256), args, 0, st));
    int herr = 0;
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, &bar->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaFreeAsync(bar, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (herr) return ctx->set_error(SS_ERR_TIMEOUT, "ss_selftest_barrier: grid barrier timed out");
    return SS_OK;
}

extern "C" ss_status ss_set_solve_mode(ss_ctx *ctx, int32_t mode) {
    if (!ctx) return SS_ERR_ARG;
    if (mode != SS_SOLVE_SWEEP_KERNEL && mode != SS_SOLVE_PER_STEP)
        return ctx->set_error(SS_ERR_ARG, "ss_set_solve_mode: unknown mode");
    ctx->solve_mode = mode;
    return SS_OK;
}

template <typename T>
static void set_smem_attrs(int device);

extern "C" ss_status ss_set_sweep_fusion(ss_ctx *ctx, int32_t max_items) {
    if (!ctx) return SS_ERR_ARG;
    if (max_items < -1) return ctx->set_error(SS_ERR_ARG, "ss_set_sweep_fusion: max_items must be >= -1");
    ctx->sweep_fuse_max = max_items;
    return SS_OK;
}

extern "C" ss_status ss_set_schur_mode(ss_ctx *ctx, int32_t mode, double min_flops) {
    if (!ctx) return SS_ERR_ARG;
    if ((mode != SS_SCHUR_TENSOR && mode != SS_SCHUR_SIMT) || !(min_flops >= 0.0))
        return ctx->set_error(SS_ERR_ARG, "ss_set_schur_mode: bad argument");
    ctx->schur_mode = mode;
    ctx->tc_min_flops = min_flops;
    ctx->plan_gen++;
    return SS_OK;
}

extern "C" ss_status ss_set_gemm_mode(ss_ctx *ctx, int32_t mode) {
    if (!ctx) return SS_ERR_ARG;
    if (mode != SS_GEMM_TENSOR && mode != SS_GEMM_SIMT) return ctx->set_error(SS_ERR_ARG, "ss_set_gemm_mode: bad mode");
    ctx->gemm_mode = mode;
    return SS_OK;
}

extern "C" ss_status ss_set_factor_graph(ss_ctx *ctx, int32_t on) {
    if (!ctx) return SS_ERR_ARG;
    if (on != 0 && on != 1) return ctx->set_error(SS_ERR_ARG, "ss_set_factor_graph: on must be 0 or 1");
    ctx->factor_graph = on;
    return SS_OK;
}

// One 128 x 64 x 64 FP16 MMA tile on the tensor cores against the exact product: the
// operands are small integers, so every product and sum is exact in FP32.
extern "C" ss_status ss_selftest_tc(ss_ctx *ctx, uint64_t seed, double *max_abs_err) {
    if (!ctx || !max_abs_err) return SS_ERR_ARG;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "ss_selftest_tc: host-only context");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    set_smem_attrs<double>(ctx->device);
    const int M = sstc::kTileM, N = sstc::kTileN, K = sstc::kTileK;
    std::vector<float> a((size_t)M * K), b((size_t)N * K);
    uint64_t x = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto next = [&]() {                       // integers in [-128, 128]
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        return (float)((int)((x >> 33) % 257) - 128);
    };
    for (float &v : a) v = next();
    for (float &v : b) v = next();
    std::vector<__half> ha(sstc::kSliceBytes / 2), hb(sstc::kHalfSliceBytes / 2);
    for (int r = 0; r < M; ++r)
        for (int k = 0; k < K; ++k) ha[sstc::core_offset(r, k) / 2] = __float2half(a[(size_t)r * K + k]);
    for (int r = 0; r < N; ++r)
        for (int k = 0; k < K; ++k) hb[sstc::core_offset(r, k) / 2] = __float2half(b[(size_t)r * K + k]);
    unsigned char *dA = nullptr, *dB = nullptr;
    float *dD = nullptr;
    int *dst = nullptr;
    cudaStream_t st = ctx->stream;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dA, sstc::kSliceBytes, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dB, sstc::kHalfSliceBytes, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dD, sizeof(float) * M * N, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dst, sizeof(int), st));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(dA, ha.data(), sstc::kSliceBytes, cudaMemcpyHostToDevice, st));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(dB, hb.data(), sstc::kHalfSliceBytes, cudaMemcpyHostToDevice, st));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(dD, 0, sizeof(float) * M * N, st));
    ss_launch(ctx, SS_K_SCHUR_TC, sstc::k_tc_selftest, 1, 128, sstc::kSelftestSmem, st,
              (const unsigned char *)dA, (const unsigned char *)dB, dD, dst);
    std::vector<float> D((size_t)M * N);
    int status = -1;
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(D.data(), dD, sizeof(float) * M * N, cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(&status, dst, sizeof(int), cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    cudaFreeAsync(dA, st);
    cudaFreeAsync(dB, st);
    cudaFreeAsync(dD, st);
    cudaFreeAsync(dst, st);
    if (status != 0) return ctx->set_error(SS_ERR_TIMEOUT, "ss_selftest_tc: a bounded wait ran out");
    double err = 0.0;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) {
            double ref = 0.0;
            for (int k = 0; k < K; ++k) ref += (double)a[(size_t)i * K + k] * b[(size_t)j * K + k];
            err = std::max(err, std::fabs(ref - (double)D[(size_t)i * N + j]));
        }
    *max_abs_err = err;
    return SS_OK;
}

extern "C" ss_status ss_sync(ss_ctx *ctx) {
    if (!ctx) return SS_ERR_ARG;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "host-only context");
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

// ------------------------------------------------------------------ symbolic upload
template <typename V>
static int upload_vec(ss_ctx *ctx, const std::vector<V> &h, V **d) {
    *d = nullptr;
    if (h.empty()) return SS_OK;
    SS_CUDA_TRY(ctx, cudaMalloc((void **)d, sizeof(V) * h.size()));
    SS_CUDA_TRY(ctx, cudaMemcpy(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
    return SS_OK;
}

int ss_symbolic_upload(ss_symbolic *s) {
    ss_ctx *ctx = s->ctx;
    if (ctx->device < 0) return SS_OK;     // host-only context
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc;
#define UP(h, d) if ((rc = upload_vec(ctx, h, &d)) != SS_OK) return rc
    UP(s->rowptr, s->d_rowptr);
    UP(s->colind, s->d_colind);
    UP(s->iperm, s->d_iperm);
    UP(s->perm, s->d_perm);
    UP(s->idx, s->d_idx);
    UP(s->asm_e, s->d_asm_e);
    UP(s->asm_dest, s->d_asm_dest);
    UP(s->relmap, s->d_relmap);
    UP(s->ext_tasks, s->d_ext_tasks);
    UP(s->panels, s->d_panels);
    UP(s->store_tasks, s->d_store_tasks);
    UP(s->tasks, s->d_tasks);
    UP(s->solve_panels, s->d_solve_panels);
    UP(s->solve_tile_pre, s->d_solve_tile_pre);
    std::vector<int32_t> col_panel(s->n);
    for (size_t p = 0; p < s->panels.size(); ++p)
        for (int i = 0; i < s->panels[p].w; ++i) col_panel[s->panels[p].g0 + i] = (int32_t)p;
    UP(col_panel, s->d_col_panel);
    std::vector<SweepLevel> lev(s->solve_levels.size());
    for (size_t L = 0; L < lev.size(); ++L)
        lev[L] = SweepLevel{(int32_t)s->solve_levels[L].panel_off, s->solve_levels[L].count,
                            s->solve_levels[L].row_tiles, 0};
    SweepLevel *dl = nullptr;
    UP(lev, dl);
    s->d_sweep_lev = dl;
#undef UP
    return SS_OK;
}

void ss_symbolic_free_device(ss_symbolic *s) {
    void *ptrs[] = {s->d_rowptr, s->d_colind, s->d_iperm, s->d_perm, s->d_idx, s->d_asm_e,
                    s->d_asm_dest, s->d_relmap, s->d_ext_tasks, s->d_panels, s->d_store_tasks, s->d_tasks,
                    s->d_solve_panels, s->d_solve_tile_pre, s->d_col_panel, s->d_sweep_lev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    s->d_rowptr = nullptr; s->d_colind = nullptr; s->d_iperm = nullptr; s->d_perm = nullptr;
    s->d_idx = nullptr; s->d_asm_e = nullptr; s->d_asm_dest = nullptr; s->d_relmap = nullptr;
    s->d_ext_tasks = nullptr; s->d_panels = nullptr; s->d_store_tasks = nullptr; s->d_tasks = nullptr;
    s->d_solve_panels = nullptr; s->d_solve_tile_pre = nullptr; s->d_col_panel = nullptr;
    s->d_sweep_lev = nullptr;
}

// ------------------------------------------------------------------ norms
__global__ void k_row_abs_max(int64_t n, const int64_t *__restrict__ rowptr, const double *__restrict__ v,
                              unsigned long long *out) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (r < n)
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) s += fabs(v[p]);
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

int ss_norm1(ss_symbolic *s, const double *vals, double *out) {
    ss_ctx *ctx = s->ctx;
    unsigned long long *d = nullptr, h = 0;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&d, sizeof(unsigned long long), ctx->stream));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, sizeof(unsigned long long), ctx->stream));
    ss_launch(ctx, SS_K_MISC, k_row_abs_max, (unsigned)((s->n + 255) / 256), 256, 0, ctx->stream, s->n, s->d_rowptr, vals, d);
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA_TRY(ctx, cudaFreeAsync(d, ctx->stream));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double v;
    std::memcpy(&v, &h, sizeof(v));
    *out = v;
    return SS_OK;
}

// ------------------------------------------------------------------ numeric factorisation
// Large dynamic shared memory is a per-device function attribute: set once per device
// (the caller has made that device current).
static bool first_use_on_device(int device, std::mutex &mu, std::vector<char> &seen) {
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0) return false;
    if ((size_t)device >= seen.size()) seen.resize(device + 1, 0);
    if (seen[device]) return false;
    seen[device] = 1;
    return true;
}

template <typename T>
static void set_smem_attrs(int device) {
    static std::mutex mu;
    static std::vector<char> seen;
    if (!first_use_on_device(device, mu, seen)) return;
    cudaFuncSetAttribute(k_diag_bk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiagSmem);
    cudaFuncSetAttribute(k_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem<T>());
    cudaFuncSetAttribute(k_schur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)schur_smem<T>());
    cudaFuncSetAttribute(k_fwd_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diag_solve_smem<T>());
    cudaFuncSetAttribute(k_bwd_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diag_solve_smem<T>());
    cudaFuncSetAttribute(k_fwd_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_kernel_smem<T>());
    cudaFuncSetAttribute(k_bwd_gather<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_kernel_smem<T>());
    cudaFuncSetAttribute(k_solve_sweeps<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_launch_smem<T>());
    if (std::is_same<T, double>::value) {
        cudaFuncSetAttribute(sstc::k_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sstc::kSchurTcSmem);
        cudaFuncSetAttribute(sstc::k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sstc::kSelftestSmem);
    }
}

// Scratch of one wave of ns shifts: W = L21 D, the Mt transforms, level workspace,
// contribution-block pool, tensor-core operand slices and their row exponents.
struct WaveScratch {
    int64_t ws_n, cb_n, mt_n, wb_n, sl_n, ex_n;
};

template <typename T>
static WaveScratch wave_sizes(const ss_symbolic *s, bool tc) {
    WaveScratch z;
    z.ws_n = std::max<int64_t>(1, s->ws_total);
    z.cb_n = std::max<int64_t>(1, s->cb_total);
    z.mt_n = std::max<int64_t>(1, (int64_t)s->mt_max * NB * NB);
    z.wb_n = std::max<int64_t>(1, s->wbuf_max);
    z.sl_n = tc ? std::max<int64_t>(16, s->sl_max) : 16;
    z.ex_n = tc ? std::max<int64_t>(1, s->ex_max) : 1;
    return z;
}

template <typename T>
static double wave_bytes(const WaveScratch &z) {
    return (double)sizeof(T) * (double)(z.ws_n + z.cb_n + z.mt_n + z.wb_n) + (double)z.sl_n + 4.0 * (double)z.ex_n;
}

// whether factor step q runs its Schur update on the tensor cores
static bool step_uses_tc(const ss_symbolic *s, const ss_ctx *ctx, int q, bool tc) {
    const StepDesc &sd = s->steps[q];
    if (!tc || sd.tiles3 <= 0 || sd.tc_tiles <= 0) return false;
    const int mode = q < (int)s->step_mode.size() ? s->step_mode[q] : -1;
    if (mode >= 0) return mode == 1;
    return sd.flops3 >= ctx->tc_min_flops;
}

// The launches of one factorisation of ns shifts over every level (no host
// synchronisation: this sequence is also what a CUDA graph captures).  hp: the host copy of
// the shift table dp (its scratch pointers give the workspace memsets).
template <typename T>
static int factor_levels(ss_numeric *f, int ns, ShiftPtrs<T> *dp, const std::vector<ShiftPtrs<T>> &hp, bool tc,
                         std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *step_ev) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    for (int32_t l = 0; l < s->nlev; ++l) {
        for (int q = 0; q < ns; ++q)
            SS_CUDA_TRY(ctx, cudaMemsetAsync(hp[q].ws, 0, sizeof(T) * s->lev_ws[l], st));
        const int64_t a0 = s->asm_lev_off[l], acount = s->asm_lev_off[l + 1] - a0;
        if (acount > 0) {
            unsigned gx = (unsigned)std::min<int64_t>((acount + 255) / 256, 8192);
            ss_launch(ctx, SS_K_ASSEMBLE, k_assemble<T>, dim3(gx, ns), 256, 0, st, acount, s->d_asm_e + a0,
                      s->d_asm_dest + a0, (const ShiftPtrs<T> *)dp);
        }
        for (int32_t q = s->lev_ext_pass_off[l]; q < s->lev_ext_pass_off[l + 1]; ++q) {
            const ExtendPass &ps = s->ext_pass[q];
            ss_launch(ctx, SS_K_EXTEND_ADD, k_extend_add<T>, dim3(ps.cols, ns), 128, 0, st,
                      s->d_ext_tasks + ps.task_off, ps.count, s->d_relmap, (const ShiftPtrs<T> *)dp);
        }
        for (int32_t q = s->lev_step_off[l]; q < s->lev_step_off[l + 1]; ++q) {
            const StepDesc &sd = s->steps[q];
            const StepTask *tk = s->d_tasks + sd.task_off;
            ss_launch(ctx, SS_K_DIAG_BK, k_diag_bk<T>, dim3(sd.count, ns), 256, kDiagSmem, st, tk,
                      (const ShiftPtrs<T> *)dp, 0);
            if (sd.tiles4 > 0) {
                const int cls = std::is_same<T, float>::value ? SS_K_PANEL_F32 : SS_K_PANEL;
                ss_launch(ctx, cls, k_panel<T>, dim3(sd.tiles4, ns), 256, panel_smem<T>(), st, tk, sd.count,
                          (const ShiftPtrs<T> *)dp);
                ctx->add_flops(cls, sd.flops4 * ns);
            }
            if (step_ev && sd.tiles3 > 0) {
                cudaEvent_t e0, e1;
                SS_CUDA_TRY(ctx, cudaEventCreate(&e0));
                SS_CUDA_TRY(ctx, cudaEventCreate(&e1));
                SS_CUDA_TRY(ctx, cudaEventRecord(e0, st));
                (*step_ev)[q] = {e0, e1};
            }
            if (step_uses_tc(s, ctx, q, tc)) {
                ss_launch(ctx, SS_K_SCHUR_TC, sstc::k_tc_slice, dim3(sd.sl_tiles, ns), 128, 0, st, tk, sd.count,
                          (const ShiftPtrs<double> *)(void *)dp);
                ss_launch(ctx, SS_K_SCHUR_TC, sstc::k_schur_tc, dim3(sd.tc_tiles, ns), sstc::kSchurTcThreads,
                          sstc::kSchurTcSmem, st, tk, sd.count, (const ShiftPtrs<double> *)(void *)dp);
                ctx->add_flops(SS_K_SCHUR_TC, sd.flops3 * ns);
                // 112 MMAs of 128 x 64 x 16 per tile
                ctx->add_tensor_flops(SS_K_SCHUR_TC, 112.0 * 2.0 * 128 * 64 * 16 * sd.tc_tiles * ns);
            } else if (sd.tiles3 > 0) {
                const int cls = std::is_same<T, float>::value ? SS_K_SCHUR_F32 : SS_K_SCHUR;
                ss_launch(ctx, cls, k_schur<T>, dim3(sd.tiles3, ns), 256, schur_smem<T>(), st, tk, sd.count,
                          (const ShiftPtrs<T> *)dp);
                ctx->add_flops(cls, sd.flops3 * ns);
            }
            if (step_ev && sd.tiles3 > 0) SS_CUDA_TRY(ctx, cudaEventRecord((*step_ev)[q].second, st));
        }
        const int32_t t0 = s->lev_store_off[l], nt = s->lev_store_off[l + 1] - t0;
        if (nt > 0 && s->lev_store_cols[l] > 0)
            ss_launch(ctx, SS_K_MISC, k_level_store<T>, dim3(s->lev_store_cols[l], ns), 128, 0, st,
                      (const StoreTask *)(s->d_store_tasks + t0), nt, (const ShiftPtrs<T> *)dp);
    }
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

template <typename T>
static void fill_shift(ss_numeric *f, int j, ShiftPtrs<T> &p) {
    p.a = f->a_vals;
    p.b = f->b_vals;
    p.lst = (T *)f->arena[j];
    p.linv = f->linv[j];
    p.dblk = f->dblk[j];
    p.piv = f->piv[j];
    p.counts = f->d_counts + SS_NCOUNT * j;
    p.seg_sigma = f->d_seg_sigma ? f->d_seg_sigma + (int64_t)f->n_seg * j : nullptr;
    p.eseg = f->d_seg_sigma ? f->d_eseg : nullptr;
    p.sigma = f->sigma[j];
    p.norm = f->norm_a1 + std::fabs(f->sigma[j]) * f->norm_b1;
    p.tiny_thr = 64.0 * 1.1102230246251565e-16 * p.norm;
}

template <typename T>
static void point_scratch(ShiftPtrs<T> &p, const WaveScratch &z, int q, T *mt, T *wb, T *ws, T *cb, unsigned char *sl,
                          int32_t *ex) {
    p.ws = ws + (int64_t)q * z.ws_n;
    p.cb = cb + (int64_t)q * z.cb_n;
    p.mt = mt + (int64_t)q * z.mt_n;
    p.wbuf = wb + (int64_t)q * z.wb_n;
    p.sl = sl + (int64_t)q * z.sl_n;
    p.ex = ex + (int64_t)q * z.ex_n;
}

void ss_free_plans(ss_symbolic *s) {
    for (FactorPlan *pl : s->plans) {
        if (pl->exec) cudaGraphExecDestroy(pl->exec);
        void *ptrs[] = {pl->mt, pl->wb, pl->ws, pl->cb, pl->sl, pl->ex, pl->dp};
        for (void *q : ptrs)
            if (q) cudaFree(q);
        delete pl;
    }
    s->plans.clear();
}

// Captured factorisations are kept while their scratch stays within this many bytes.
constexpr double kPlanScratchMax = 8.0e9;

// One wave through a captured CUDA graph: the plan for (ns, precision, tensor cores) is
// captured on first use (scratch allocated once and kept with the analysis), then every
// call only uploads the shift table and launches the graph.
template <typename T>
static int factor_wave_graph(ss_numeric *f, const std::vector<int> &js, bool tc, const WaveScratch &z) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int ns = (int)js.size();
    const int fp32 = std::is_same<T, float>::value ? 1 : 0;
    // a plan captured under other Schur settings is stale
    for (size_t q = 0; q < s->plans.size();) {
        FactorPlan *c = s->plans[q];
        if (c->gen != ctx->plan_gen) {
            SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            if (c->exec) cudaGraphExecDestroy(c->exec);
            void *ptrs[] = {c->mt, c->wb, c->ws, c->cb, c->sl, c->ex, c->dp};
            for (void *v : ptrs)
                if (v) cudaFree(v);
            delete c;
            s->plans.erase(s->plans.begin() + q);
        } else {
            ++q;
        }
    }
    FactorPlan *pl = nullptr;
    for (FactorPlan *c : s->plans)
        if (c->ns == ns && c->fp32 == fp32 && c->tc == (tc ? 1 : 0)) pl = c;
    std::vector<ShiftPtrs<T>> hp(ns);
    const bool fresh = pl == nullptr;
    if (fresh) {
        pl = new FactorPlan();
        pl->gen = ctx->plan_gen;
        pl->ns = ns;
        pl->fp32 = fp32;
        pl->tc = tc ? 1 : 0;
        cudaError_t e = cudaMalloc(&pl->mt, sizeof(T) * z.mt_n * ns);
        if (e == cudaSuccess) e = cudaMalloc(&pl->wb, sizeof(T) * z.wb_n * ns);
        if (e == cudaSuccess) e = cudaMalloc(&pl->ws, sizeof(T) * z.ws_n * ns);
        if (e == cudaSuccess) e = cudaMalloc(&pl->cb, sizeof(T) * z.cb_n * ns);
        if (e == cudaSuccess) e = cudaMalloc(&pl->sl, (size_t)z.sl_n * ns);
        if (e == cudaSuccess) e = cudaMalloc(&pl->ex, sizeof(int32_t) * z.ex_n * ns);
        if (e == cudaSuccess) e = cudaMalloc(&pl->dp, sizeof(ShiftPtrs<T>) * ns);
        s->plans.push_back(pl);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctx->set_error(SS_ERR_OOM, "ss_factor: allocation of a captured factorisation's scratch failed");
        }
    }
    for (int q = 0; q < ns; ++q) {
        fill_shift<T>(f, js[q], hp[q]);
        point_scratch<T>(hp[q], z, q, (T *)pl->mt, (T *)pl->wb, (T *)pl->ws, (T *)pl->cb, (unsigned char *)pl->sl,
                         (int32_t *)pl->ex);
    }
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(pl->dp, hp.data(), sizeof(ShiftPtrs<T>) * ns, cudaMemcpyHostToDevice, st));
    if (fresh) {
        // capture on a private stream (the context's may be the legacy default stream,
        // which cannot capture); the graph is launched on the context's stream below
        cudaGraph_t graph = nullptr;
        if (!ctx->cap_stream) SS_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        SS_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        ctx->stream = ctx->cap_stream;
        int rc = factor_levels<T>(f, ns, (ShiftPtrs<T> *)pl->dp, hp, tc, nullptr);
        ctx->stream = st;
        ctx->capturing = false;
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc != SS_OK) return rc;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctx->set_error(SS_ERR_CUDA, std::string("ss_factor: graph capture failed: ") + cudaGetErrorString(e));
        }
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
        int64_t kn = 0;
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
        }
        pl->kernel_nodes = kn;
        e = cudaGraphInstantiate(&pl->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            pl->exec = nullptr;
            return ctx->set_error(SS_ERR_CUDA, std::string("ss_factor: graph instantiation failed: ") +
                                                   cudaGetErrorString(e));
        }
    }
    SS_CUDA_TRY(ctx, cudaGraphLaunch(pl->exec, st));
    g_ss_launches.fetch_add(pl->kernel_nodes, std::memory_order_relaxed);
    return SS_OK;
}

// Factorisation of the shifts in `which`, in waves of as many shifts as the free device
// memory holds: each shift of a wave has its own level workspace, contribution-block pool
// and panel scratch for the duration of the wave; the L storage (f->arena) persists.
// With ss_set_factor_graph on (and no per-launch profiling), a wave whose scratch fits
// kPlanScratchMax replays a captured CUDA graph instead of launching kernel by kernel.
template <typename T>
static int factor_run(ss_numeric *f, const std::vector<int> &which) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    set_smem_attrs<T>(ctx->device);
    const int ns_all = (int)which.size();
    if (ns_all == 0) return SS_OK;
    // FP64 steps with enough Schur work run the tensor-core update (tc_kernels.cuh)
    const bool tc = std::is_same<T, double>::value && ctx->schur_mode == SS_SCHUR_TENSOR && s->sl_max > 0;
    const WaveScratch z = wave_sizes<T>(s, tc);
    const double per_shift = wave_bytes<T>(z);
    size_t mem_free = 0, mem_tot = 0;
    SS_CUDA_TRY(ctx, cudaMemGetInfo(&mem_free, &mem_tot));
    int wave = (int)std::max(1.0, std::min((double)std::min(ns_all, 65535), std::floor(0.8 * (double)mem_free / per_shift)));
    static const unsigned long long init[SS_NCOUNT] = {0, 0, 0, 0, 0x7ff0000000000000ull /* +inf */, 0, 0, 0};
    for (int q = 0; q < ns_all; ++q)
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(f->d_counts + SS_NCOUNT * which[q], init, sizeof(init),
                                         cudaMemcpyHostToDevice, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));    // init is a host array
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> step_ev;
    if (ctx->step_times) step_ev.assign(s->steps.size(), {nullptr, nullptr});
    for (int w0 = 0; w0 < ns_all; w0 += wave) {
        const int ns = std::min(wave, ns_all - w0);
        std::vector<int> js(which.begin() + w0, which.begin() + w0 + ns);
        if (ctx->factor_graph && !ctx->prof_mask && !ctx->step_times && per_shift * ns <= kPlanScratchMax) {
            int rc = factor_wave_graph<T>(f, js, tc, z);
            if (rc != SS_OK) return rc;
            continue;
        }
        T *mt = nullptr, *wb = nullptr, *ws = nullptr, *cb = nullptr;
        unsigned char *sl = nullptr;
        int32_t *ex = nullptr;
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&sl, (size_t)z.sl_n * ns, st));
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&ex, sizeof(int32_t) * z.ex_n * ns, st));
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&mt, sizeof(T) * z.mt_n * ns, st));
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&wb, sizeof(T) * z.wb_n * ns, st));
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&ws, sizeof(T) * z.ws_n * ns, st));
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&cb, sizeof(T) * z.cb_n * ns, st));
        std::vector<ShiftPtrs<T>> hp(ns);
        for (int q = 0; q < ns; ++q) {
            fill_shift<T>(f, js[q], hp[q]);
            point_scratch<T>(hp[q], z, q, mt, wb, ws, cb, sl, ex);
        }
        ShiftPtrs<T> *dp = nullptr;
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&dp, sizeof(ShiftPtrs<T>) * ns, st));
        SS_CUDA_TRY(ctx, cudaMemcpyAsync(dp, hp.data(), sizeof(ShiftPtrs<T>) * ns, cudaMemcpyHostToDevice, st));
        int rc = factor_levels<T>(f, ns, dp, hp, tc, ctx->step_times ? &step_ev : nullptr);
        if (rc != SS_OK) return rc;
        SS_CUDA_TRY(ctx, cudaFreeAsync(dp, st));
        SS_CUDA_TRY(ctx, cudaFreeAsync(mt, st));
        SS_CUDA_TRY(ctx, cudaFreeAsync(wb, st));
        SS_CUDA_TRY(ctx, cudaFreeAsync(ws, st));
        SS_CUDA_TRY(ctx, cudaFreeAsync(cb, st));
        SS_CUDA_TRY(ctx, cudaFreeAsync(sl, st));
        SS_CUDA_TRY(ctx, cudaFreeAsync(ex, st));
    }
    if (ctx->step_times) {
        SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        ctx->step_times->assign(s->steps.size(), 0.0);
        for (size_t q = 0; q < step_ev.size(); ++q) {
            if (!step_ev[q].first) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, step_ev[q].first, step_ev[q].second);
            (*ctx->step_times)[q] += 1e-3 * ms;
            cudaEventDestroy(step_ev[q].first);
            cudaEventDestroy(step_ev[q].second);
        }
    }
    return SS_OK;
}

// largest contraction factor of one FP32 solve for which an FP64 factor's rounded copy
// serves the solves
constexpr double kRoundedRhoMax = 0.25;

__global__ void k_round_f32(int64_t n, const double *__restrict__ x, float *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

static void factor_free(ss_numeric *f) {
    for (void *p : f->arena) if (p) cudaFree(p);
    for (float *p : f->arena_lo) if (p) cudaFree(p);
    for (double *p : f->linv) if (p) cudaFree(p);
    for (double *p : f->dblk) if (p) cudaFree(p);
    for (int32_t *p : f->piv) if (p) cudaFree(p);
    for (double *p : f->mvals) if (p) cudaFree(p);
    f->mvals.clear();
    if (f->d_counts) cudaFree(f->d_counts);
    if (f->d_eseg) cudaFree(f->d_eseg);
    if (f->d_rowseg) cudaFree(f->d_rowseg);
    if (f->d_seg_sigma) cudaFree(f->d_seg_sigma);
    f->d_eseg = f->d_rowseg = nullptr;
    f->d_seg_sigma = nullptr;
    f->arena.clear(); f->arena_lo.clear(); f->linv.clear(); f->dblk.clear(); f->piv.clear();
    f->d_counts = nullptr;
    oz_free_numeric(f);
}

int ss_factor_create(ss_symbolic *sym, const double *a_vals, const double *b_vals, const double *sigma,
                     int32_t n_shift, int32_t precision, ss_numeric **out, const SegShifts *seg) {
    ss_ctx *ctx = sym->ctx;
    *out = nullptr;
    ss_numeric *f = new (std::nothrow) ss_numeric();
    if (!f) return ctx->set_error(SS_ERR_OOM, "ss_factor: host allocation failed");
    f->sym = sym;
    f->inertia_only = (precision & SS_INERTIA_ONLY) != 0;
    precision = f->inertia_only ? SS_FP64 : precision;      // exact counts come from FP64 fronts
    f->precision = precision;
    f->n_shift = n_shift;
    f->sigma.assign(sigma, sigma + n_shift);
    f->a_vals = a_vals;
    f->b_vals = b_vals;
    int rc = SS_OK;
    const size_t esz = precision == SS_MIXED ? sizeof(float) : sizeof(double);
    const int64_t npan = (int64_t)sym->panels.size();
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if ((rc = ss_norm1(sym, a_vals, &f->norm_a1)) != SS_OK) { delete f; return rc; }
    if ((rc = ss_norm1(sym, b_vals, &f->norm_b1)) != SS_OK) { delete f; return rc; }
    f->arena.assign(n_shift, nullptr);
    f->arena_lo.assign(n_shift, nullptr);
    f->mvals.assign(n_shift, nullptr);
    f->linv.assign(n_shift, nullptr);
    f->dblk.assign(n_shift, nullptr);
    f->piv.assign(n_shift, nullptr);
    cudaError_t e = cudaMalloc((void **)&f->d_counts, sizeof(unsigned long long) * SS_NCOUNT * n_shift);
    if (seg && e == cudaSuccess) {
        // the pencil of every stored entry (from its row) and the shift table, on the device
        f->n_seg = seg->n_seg;
        std::vector<int32_t> eseg(std::max<int64_t>(1, sym->nnz));
        for (int64_t r = 0; r < sym->n; ++r)
            for (int64_t q = sym->rowptr[r]; q < sym->rowptr[r + 1]; ++q) eseg[q] = seg->row_seg[r];
        e = cudaMalloc((void **)&f->d_eseg, sizeof(int32_t) * eseg.size());
        if (e == cudaSuccess) e = cudaMalloc((void **)&f->d_rowseg, sizeof(int32_t) * std::max<int64_t>(1, sym->n));
        if (e == cudaSuccess) e = cudaMalloc((void **)&f->d_seg_sigma, sizeof(double) * n_shift * seg->n_seg);
        if (e == cudaSuccess)
            e = cudaMemcpy(f->d_eseg, eseg.data(), sizeof(int32_t) * eseg.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(f->d_rowseg, seg->row_seg, sizeof(int32_t) * sym->n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(f->d_seg_sigma, seg->sigma, sizeof(double) * n_shift * seg->n_seg,
                           cudaMemcpyHostToDevice);
    }
    for (int j = 0; j < n_shift && e == cudaSuccess; ++j) {
        if (!f->inertia_only) e = cudaMalloc(&f->arena[j], esz * std::max<int64_t>(1, sym->l_total));
        if (e == cudaSuccess) e = cudaMalloc((void **)&f->linv[j], sizeof(double) * NB * NB * npan);
        if (e == cudaSuccess) e = cudaMalloc((void **)&f->dblk[j], sizeof(double) * 2 * NB * npan);
        if (e == cudaSuccess) e = cudaMalloc((void **)&f->piv[j], sizeof(int32_t) * NB * npan);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        factor_free(f);
        delete f;
        return ctx->set_error(e == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA,
                              std::string("ss_factor: device allocation failed: ") + cudaGetErrorString(e));
    }
    std::vector<int> all(n_shift);
    for (int j = 0; j < n_shift; ++j) all[j] = j;
    f->shift_prec.assign(n_shift, precision);
    f->rho.assign(n_shift, 0.0);
    if (precision == SS_MIXED) {
        rc = factor_run<float>(f, all);
        // quality gate: the FP32 factor is kept only where one FP32 solve contracts the
        // error of an FP64 refinement step by at least 1e-2; elsewhere (sigma close to an
        // eigenvalue, large element growth) the shift is refactored in FP64
        std::vector<int> redo;
        for (int j = 0; j < n_shift && rc == SS_OK; ++j) {
            rc = solve_contraction(f, j, &f->rho[j]);
            if (rc == SS_OK && !(f->rho[j] <= 1e-2)) redo.push_back(j);
        }
        // the FP32 arena of a refactored shift is kept for the FP32 rounding below
        for (int j : redo) {
            if (rc != SS_OK) break;
            f->arena_lo[j] = (float *)f->arena[j];
            f->arena[j] = nullptr;
            cudaError_t e2 = cudaMalloc(&f->arena[j], sizeof(double) * std::max<int64_t>(1, sym->l_total));
            if (e2 != cudaSuccess) {
                cudaGetLastError();
                rc = ctx->set_error(SS_ERR_OOM, "ss_factor: device allocation for an FP64 refactor failed");
            }
            f->shift_prec[j] = SS_FP64;
        }
        if (rc == SS_OK) rc = factor_run<double>(f, redo);
        // FP64 factor, FP32 solves: the FP64 fronts rounded once to FP32 avoid the error
        // that FP32 Schur updates accumulate; the rounded copy is kept where one FP32
        // solve from it contracts by rho <= kRoundedRhoMax, else solves stay FP64
        for (int j : redo) {
            if (rc != SS_OK) break;
            const int64_t na = std::max<int64_t>(1, sym->l_total);
            const unsigned g = (unsigned)std::min<int64_t>((na + 255) / 256, (int64_t)ctx->sm_count * 16);
            ss_launch(ctx, SS_K_MISC, k_round_f32, g, 256, 0, ctx->stream, na, (const double *)f->arena[j],
                      f->arena_lo[j]);
            double rho_lo = INFINITY;
            rc = solve_contraction(f, j, &rho_lo);
            if (rc != SS_OK) break;
            if (rho_lo <= kRoundedRhoMax) {
                f->rho[j] = rho_lo;
            } else {
                SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
                cudaFree(f->arena_lo[j]);
                f->arena_lo[j] = nullptr;
            }
        }
    } else if (precision == SS_MIXED_TC) {
        // FP64 fronts (tensor-core Schur updates), every shift's factor rounded once to
        // FP32 for its solves where one FP32 solve contracts by rho <= kRoundedRhoMax
        rc = factor_run<double>(f, all);
        for (int j = 0; j < n_shift && rc == SS_OK; ++j) {
            f->shift_prec[j] = SS_FP64;
            const int64_t na = std::max<int64_t>(1, sym->l_total);
            cudaError_t e2 = cudaMalloc((void **)&f->arena_lo[j], sizeof(float) * na);
            if (e2 != cudaSuccess) {
                cudaGetLastError();
                f->arena_lo[j] = nullptr;
                continue;                               // no room for the copy: FP64 solves
            }
            const unsigned g = (unsigned)std::min<int64_t>((na + 255) / 256, (int64_t)ctx->sm_count * 16);
            ss_launch(ctx, SS_K_MISC, k_round_f32, g, 256, 0, ctx->stream, na, (const double *)f->arena[j],
                      f->arena_lo[j]);
            double rho_lo = INFINITY;
            rc = solve_contraction(f, j, &rho_lo);
            if (rc != SS_OK) break;
            if (rho_lo <= kRoundedRhoMax) {
                f->rho[j] = rho_lo;
            } else {
                SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
                cudaFree(f->arena_lo[j]);
                f->arena_lo[j] = nullptr;
            }
        }
    } else {
        rc = factor_run<double>(f, all);
    }
    if (rc == SS_OK) rc = ss_factor_fetch_counts(f);
    if (rc != SS_OK && rc != SS_ERR_SINGULAR) {
        factor_free(f);
        delete f;
        return rc;
    }
    *out = f;
    return rc;
}

int ss_factor_fetch_counts(ss_numeric *f) {
    ss_ctx *ctx = f->sym->ctx;
    f->h_counts.assign(SS_NCOUNT * f->n_shift, 0);
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(f->h_counts.data(), f->d_counts,
                                     sizeof(unsigned long long) * SS_NCOUNT * f->n_shift, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    f->counts_valid = true;
    for (int j = 0; j < f->n_shift; ++j)
        if (f->h_counts[SS_NCOUNT * j + 7])
            return ctx->set_error(SS_ERR_TIMEOUT, "ss_factor: a bounded device wait of the tensor-core Schur "
                                                  "update ran out for shift " + std::to_string(j));
    for (int j = 0; j < f->n_shift; ++j)
        if (f->h_counts[SS_NCOUNT * j + 3]) {
            return ctx->set_error(SS_ERR_SINGULAR, "ss_factor: a pivot fell below the singularity "
                                                   "threshold for shift " + std::to_string(j));
        }
    return SS_OK;
}

extern "C" ss_status ss_factor(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                               const double *sigma, int32_t n_shift, int32_t precision, ss_numeric **out) {
    if (!sym) return SS_ERR_ARG;
    ss_ctx *ctx = sym->ctx;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "ss_factor: host-only context");
    const int32_t base_prec = precision & ~SS_INERTIA_ONLY;
    if (!out || !a_vals || !b_vals || !sigma || n_shift <= 0 || n_shift > 65535 ||
        (base_prec != SS_FP64 && base_prec != SS_MIXED && base_prec != SS_MIXED_TC))
        return ctx->set_error(SS_ERR_ARG, "ss_factor: bad argument");
    for (int j = 0; j < n_shift; ++j)
        if (!std::isfinite(sigma[j])) return ctx->set_error(SS_ERR_ARG, "ss_factor: non-finite shift");
    try {
        return ss_factor_create(sym, a_vals, b_vals, sigma, n_shift, precision, out);
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_factor: host allocation failed");
    }
}

extern "C" ss_status ss_factor_segments(ss_symbolic *sym, const double *a_vals, const double *b_vals,
                                        const int32_t *row_segment, int32_t n_seg, const double *sigma,
                                        int32_t n_shift, ss_numeric **out) {
    if (!sym) return SS_ERR_ARG;
    ss_ctx *ctx = sym->ctx;
    if (ctx->device < 0) return ctx->set_error(SS_ERR_ARG, "ss_factor_segments: host-only context");
    if (!out || !a_vals || !b_vals || !row_segment || !sigma || n_seg <= 0 || n_shift <= 0 || n_shift > 65535)
        return ctx->set_error(SS_ERR_ARG, "ss_factor_segments: bad argument");
    for (int64_t r = 0; r < sym->n; ++r)
        if (row_segment[r] < 0 || row_segment[r] >= n_seg)
            return ctx->set_error(SS_ERR_ARG, "ss_factor_segments: row " + std::to_string(r) +
                                                  " has a pencil index outside [0, n_seg)");
    // the pattern must not couple rows of different pencils
    for (int64_t r = 0; r < sym->n; ++r)
        for (int64_t q = sym->rowptr[r]; q < sym->rowptr[r + 1]; ++q)
            if (row_segment[sym->colind[q]] != row_segment[r])
                return ctx->set_error(SS_ERR_ARG, "ss_factor_segments: entry (" + std::to_string(r) + ", " +
                                                      std::to_string(sym->colind[q]) +
                                                      ") couples two pencils");
    std::vector<double> smax(n_shift, 0.0);
    for (int j = 0; j < n_shift; ++j)
        for (int g = 0; g < n_seg; ++g) {
            const double v = sigma[(int64_t)j * n_seg + g];
            if (!std::isfinite(v)) return ctx->set_error(SS_ERR_ARG, "ss_factor_segments: non-finite shift");
            smax[j] = std::max(smax[j], std::fabs(v));
        }
    try {
        const SegShifts seg{n_seg, row_segment, sigma};
        return ss_factor_create(sym, a_vals, b_vals, smax.data(), n_shift, SS_FP64 | SS_INERTIA_ONLY, out, &seg);
    } catch (const std::bad_alloc &) {
        return ctx->set_error(SS_ERR_OOM, "ss_factor_segments: host allocation failed");
    }
}

extern "C" ss_status ss_inertia_segments(const ss_numeric *f, int32_t j, int64_t *n_neg, int64_t *n_zero,
                                         int64_t *n_pos, int64_t *n_tiny) {
    if (!f) return SS_ERR_ARG;
    ss_ctx *ctx = f->sym->ctx;
    if (f->n_seg <= 0 || j < 0 || j >= f->n_shift || !n_neg || !n_zero || !n_pos)
        return ctx->set_error(SS_ERR_ARG, "ss_inertia_segments: bad argument (or not an ss_factor_segments factor)");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const ss_symbolic *s = f->sym;
    const int32_t npan = (int32_t)s->panels.size();
    cudaStream_t st = ctx->stream;
    unsigned long long *d = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&d, sizeof(unsigned long long) * 4 * f->n_seg, st));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, sizeof(unsigned long long) * 4 * f->n_seg, st));
    const double tiny = 64.0 * 1.1102230246251565e-16 * (f->norm_a1 + std::fabs(f->sigma[j]) * f->norm_b1);
    if (npan > 0)
        ss_launch(ctx, SS_K_MISC, k_segment_inertia, (unsigned)npan, NB, 0, st, npan, (const PanelDesc *)s->d_panels,
                  (const double *)f->dblk[j], (const int32_t *)s->d_perm, (const int32_t *)f->d_rowseg, tiny, d);
    std::vector<unsigned long long> h(4 * (size_t)f->n_seg);
    cudaError_t e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    SS_CUDA_TRY(ctx, e);
    for (int g = 0; g < f->n_seg; ++g) {
        n_neg[g] = (int64_t)h[4 * g];
        n_zero[g] = (int64_t)h[4 * g + 1];
        n_pos[g] = (int64_t)h[4 * g + 2];
        if (n_tiny) n_tiny[g] = (int64_t)h[4 * g + 3];
    }
    return SS_OK;
}

extern "C" ss_status ss_autotune_schur(ss_symbolic *sym, const double *a_vals, const double *b_vals, double sigma,
                                       int32_t *n_tc_steps) {
    if (!sym) return SS_ERR_ARG;
    ss_ctx *ctx = sym->ctx;
    if (ctx->device < 0 || !a_vals || !b_vals || !std::isfinite(sigma))
        return ctx->set_error(SS_ERR_ARG, "ss_autotune_schur: bad argument or host-only context");
    const int saved_mode = ctx->schur_mode;
    std::vector<double> t_tc, t_simt;
    int rc = SS_OK;
    // the same inertia-only FP64 factorisation, once with every eligible step on the tensor
    // cores and once with every step on the CUDA cores, each step's Schur update timed
    ctx->schur_mode = SS_SCHUR_TENSOR;
    for (int pass = 0; pass < 2 && rc == SS_OK; ++pass) {
        std::fill(sym->step_mode.begin(), sym->step_mode.end(), (int8_t)(pass == 0 ? 1 : 0));
        std::vector<double> &dst = pass == 0 ? t_tc : t_simt;
        ctx->step_times = &dst;
        ss_numeric *f = nullptr;
        rc = ss_factor_create(sym, a_vals, b_vals, &sigma, 1, SS_FP64 | SS_INERTIA_ONLY, &f);
        ctx->step_times = nullptr;
        if (f) ss_factor_destroy(f);
        if (rc == SS_ERR_SINGULAR) rc = SS_OK;      // the timing stands; the shift is irrelevant
    }
    ctx->schur_mode = saved_mode;
    int32_t n = 0;
    for (size_t q = 0; q < sym->steps.size(); ++q) {
        const bool eligible = sym->steps[q].tiles3 > 0 && sym->steps[q].tc_tiles > 0;
        const bool use = rc == SS_OK && eligible && q < t_tc.size() && q < t_simt.size() && t_tc[q] < t_simt[q];
        sym->step_mode[q] = (int8_t)(rc == SS_OK ? (use ? 1 : 0) : -1);
        n += use ? 1 : 0;
    }
    ctx->plan_gen++;
    if (n_tc_steps) *n_tc_steps = n;
    return rc;
}

extern "C" ss_status ss_factor_destroy(ss_numeric *f) {
    if (!f) return SS_OK;
    factor_free(f);
    delete f;
    return SS_OK;
}

extern "C" ss_status ss_inertia(const ss_numeric *f, int32_t j, int64_t *n_neg, int64_t *n_zero,
                                int64_t *n_pos, int32_t *tiny) {
    if (!f || j < 0 || j >= f->n_shift || !f->counts_valid) return SS_ERR_ARG;
    if (n_neg) *n_neg = (int64_t)f->h_counts[SS_NCOUNT * j + 0];
    if (n_zero) *n_zero = (int64_t)f->h_counts[SS_NCOUNT * j + 1];
    if (n_pos) *n_pos = (int64_t)f->h_counts[SS_NCOUNT * j + 2];
    if (tiny) *tiny = f->h_counts[SS_NCOUNT * j + 3] ? 1 : 0;
    return SS_OK;
}

extern "C" ss_status ss_factor_quality(const ss_numeric *f, int32_t j, int32_t *precision_used, double *rho) {
    if (!f || j < 0 || j >= f->n_shift) return SS_ERR_ARG;
    if (precision_used) *precision_used = f->arena_lo[j] ? SS_FP64_SOLVE32 : f->shift_prec[j];
    if (rho) *rho = f->rho[j];
    return SS_OK;
}

extern "C" ss_status ss_factor_stats(const ss_numeric *f, int32_t j, double *min_pivot_ratio, double *max_abs_l,
                                     int64_t *n_2x2) {
    if (!f || j < 0 || j >= f->n_shift || !f->counts_valid) return SS_ERR_ARG;
    double v;
    if (min_pivot_ratio) { std::memcpy(&v, &f->h_counts[SS_NCOUNT * j + 4], sizeof(v)); *min_pivot_ratio = v; }
    if (max_abs_l) { std::memcpy(&v, &f->h_counts[SS_NCOUNT * j + 6], sizeof(v)); *max_abs_l = v; }
    if (n_2x2) *n_2x2 = (int64_t)f->h_counts[SS_NCOUNT * j + 5];
    return SS_OK;
}

// ------------------------------------------------------------------ solves
template <typename T>
static int solve_levels(ss_numeric *f, int j, T *b, int k, bool forward, bool backward, int dinv);

template <typename T>
int solve_permuted(ss_numeric *f, int j, T *b, int k) {
    return solve_levels<T>(f, j, b, k, true, true, 1);
}

// x = P L^-T D^-1/2 y for an SPD factor (the Cholesky frame of B = G G^T, G = P L D^1/2):
// y is read in the permuted order, x is written in the original order.
int solve_half_backward(ss_numeric *f, int j, const double *y, int k, double *x) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t tot = s->n * k;
    const unsigned g = (unsigned)((tot + 255) / 256);
    double *w = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&w, sizeof(double) * tot, st));
    ss_launch(ctx, SS_K_MISC, k_dhalf<double>, g, 256, 0, st, s->n, s->d_col_panel, s->d_panels, f->dblk[j], y, w, k);
    int rc = solve_levels<double>(f, j, w, k, false, true, 0);
    if (rc != SS_OK) return rc;
    ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, k, s->d_perm,
              (const double *)w, x, 1);
    SS_CUDA_TRY(ctx, cudaFreeAsync(w, st));
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// Both sweeps in one cooperative launch of k_solve_sweeps (every block resident, a
// bounded grid barrier between steps).  Returns SS_ERR_TIMEOUT if a barrier gave up.
template <typename T>
static int solve_sweeps(ss_numeric *f, int j, T *b, int k, bool forward, bool backward, int dinv, const T *arena) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int cls = std::is_same<T, float>::value ? SS_K_SOLVE_F32 : SS_K_SOLVE;
    constexpr int kSmSlots = 1024;
    if (!ctx->d_bar) SS_CUDA_TRY(ctx, cudaMalloc((void **)&ctx->d_bar, sizeof(GridBar) + sizeof(int32_t) * kSmSlots));
    int32_t *sm_slots = reinterpret_cast<int32_t *>(ctx->d_bar + 1);
    int &per_sm = ctx->sweep_blocks_per_sm[std::is_same<T, float>::value ? 1 : 0];
    if (per_sm == 0) {
        SS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_sweeps<T>, 256,
                                                                       sweep_launch_smem<T>()));
        if (per_sm <= 0) return ctx->set_error(SS_ERR_CUDA, "solve: sweep kernel cannot be resident");
    }
    const int nchunk = (k + KC - 1) / KC, ndchunk = (k + KD - 1) / KD;
    // FP32 solves with both sweeps may take the fused items on their small levels (one grid
    // barrier per level and sweep there)
    const bool fused = std::is_same<T, float>::value && forward && backward && dinv && ctx->sweep_fuse_max != 0;
    int64_t items = 1;
    double flops = 0.0;
    for (const SolveLevel &sl : s->solve_levels) {
        items = std::max<int64_t>(items, std::max<int64_t>((int64_t)sl.count * ndchunk, (int64_t)sl.row_tiles * nchunk));
        if (fused) items = std::max<int64_t>(items, (int64_t)(sl.row_tiles + sl.count) * nchunk);
        flops += ((forward ? 2.0 : 0.0) + (backward ? 2.0 : 0.0)) * sl.offdiag * k;
    }
    const int nb = (int)std::min<int64_t>((int64_t)per_sm * ctx->sm_count, items);
    const int64_t npan = std::max<int64_t>(1, (int64_t)s->panels.size());
    const int64_t zn = npan * NB * k;
    // fused: the arrival counters (npan x nchunk int32) and the forward output y (N x k)
    // follow z in the same allocation
    const int64_t an = fused ? (npan * nchunk * (int64_t)sizeof(int32_t) + sizeof(T) - 1) / sizeof(T) : 0;
    const int64_t yn = fused ? s->n * (int64_t)k : 0;
    T *zall = nullptr, *ybuf = nullptr;
    int32_t *arrive = nullptr;
    if (backward) {
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&zall, sizeof(T) * (zn + an + yn), st));
        SS_CUDA_TRY(ctx, cudaMemsetAsync(zall, 0, sizeof(T) * (zn + an), st));
        if (fused) {
            arrive = reinterpret_cast<int32_t *>(zall + zn);
            ybuf = zall + zn + an;
        }
    }
    SS_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_bar, 0, sizeof(GridBar) + sizeof(int32_t) * kSmSlots, st));
    SweepArgs a{};
    a.lev = (const SweepLevel *)s->d_sweep_lev;
    a.nlev = (int32_t)s->solve_levels.size();
    a.k = k;
    a.solve_panels = s->d_solve_panels;
    a.tile_pre = s->d_solve_tile_pre;
    a.panels = s->d_panels;
    a.idx = s->d_idx;
    a.linv = f->linv[j];
    a.dblk = f->dblk[j];
    a.piv = f->piv[j];
    a.forward = forward ? 1 : 0;
    a.backward = backward ? 1 : 0;
    a.dinv = dinv;
    a.bar = ctx->d_bar;
    a.limit = 20000000;        // polls of about 64 ns: ~1 s per barrier
    a.sm_slots = sm_slots;
    a.nsm_slots = kSmSlots;
    a.arrive = arrive;
    a.fuse_max = ctx->sweep_fuse_max < 0 ? nb : ctx->sweep_fuse_max;
    void *args[] = {(void *)&a, (void *)&arena, (void *)&b, (void *)&zall, (void *)&ybuf};
    g_ss_launches.fetch_add(1, std::memory_order_relaxed);
    size_t slot = 0;
    const bool prof = ctx->prof_mask & (1u << cls);
    if (prof) slot = ss_prof_begin(ctx, cls);
    SS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void *)k_solve_sweeps<T>, dim3(nb), dim3(256), args,
                                                 sweep_launch_smem<T>(), st));
    if (prof) ss_prof_end(ctx, cls, slot);
    ctx->add_flops(cls, flops);
    int herr = 0;
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, &ctx->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (zall) SS_CUDA_TRY(ctx, cudaFreeAsync(zall, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (herr) return ctx->set_error(SS_ERR_TIMEOUT, "solve: grid barrier of the sweep kernel timed out");
    return SS_OK;
}

template <typename T>
static int solve_levels(ss_numeric *f, int j, T *b, int k, bool forward, bool backward, int dinv) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    set_smem_attrs<T>(ctx->device);
    const T *arena = (const T *)f->arena[j];
    if (std::is_same<T, float>::value && f->arena_lo[j]) arena = (const T *)f->arena_lo[j];
    if (ctx->solve_mode == SS_SOLVE_SWEEP_KERNEL) return solve_sweeps<T>(f, j, b, k, forward, backward, dinv, arena);
    const int nchunk = (k + KC - 1) / KC;
    const int ndchunk = (k + KD - 1) / KD;
    const int nlev = (int)s->solve_levels.size();
    for (int L = 0; forward && L < nlev; ++L) {
        const SolveLevel &sl = s->solve_levels[L];
        const int32_t *lp = s->d_solve_panels + sl.panel_off;
        ss_launch(ctx, SS_K_FWD_DIAG, k_fwd_diag<T>, dim3(sl.count, ndchunk), 256, diag_solve_smem<T>(), st, lp, s->d_panels, f->linv[j],
                                                                               f->piv[j], b, k);
        if (sl.row_tiles > 0)
            ss_launch(ctx, std::is_same<T, float>::value ? SS_K_FWD_UPDATE_F32 : SS_K_FWD_UPDATE, k_fwd_update<T>, dim3(sl.row_tiles, nchunk), 256, tile_kernel_smem<T>(), st,
                lp, s->d_solve_tile_pre + sl.panel_off, sl.count, s->d_panels, s->d_idx, arena, b, k);
        if (sl.row_tiles > 0)
            ctx->add_flops(std::is_same<T, float>::value ? SS_K_FWD_UPDATE_F32 : SS_K_FWD_UPDATE, 2.0 * sl.offdiag * k);
    }
    if (!backward) return SS_OK;
    int32_t maxc = 0;
    for (const SolveLevel &sl : s->solve_levels) maxc = std::max(maxc, sl.count);
    T *z = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&z, sizeof(T) * (int64_t)maxc * NB * k, st));
    for (int L = nlev - 1; L >= 0; --L) {
        const SolveLevel &sl = s->solve_levels[L];
        const int32_t *lp = s->d_solve_panels + sl.panel_off;
        if (sl.row_tiles > 0) {
            SS_CUDA_TRY(ctx, cudaMemsetAsync(z, 0, sizeof(T) * (int64_t)sl.count * NB * k, st));
            ss_launch(ctx, std::is_same<T, float>::value ? SS_K_BWD_GATHER_F32 : SS_K_BWD_GATHER, k_bwd_gather<T>, dim3(sl.row_tiles, nchunk), 256, tile_kernel_smem<T>(), st,
                lp, s->d_solve_tile_pre + sl.panel_off, sl.count, s->d_panels, s->d_idx, arena, b, k, z);
            ctx->add_flops(std::is_same<T, float>::value ? SS_K_BWD_GATHER_F32 : SS_K_BWD_GATHER, 2.0 * sl.offdiag * k);
        }
        ss_launch(ctx, SS_K_BWD_DIAG, k_bwd_diag<T>, dim3(sl.count, ndchunk), 256, diag_solve_smem<T>(), st, 
            lp, s->d_panels, f->linv[j], f->dblk[j], f->piv[j], z, sl.row_tiles > 0 ? 1 : 0, b, k, dinv);
    }
    SS_CUDA_TRY(ctx, cudaFreeAsync(z, st));
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}
template int solve_permuted<double>(ss_numeric *, int, double *, int);
template int solve_permuted<float>(ss_numeric *, int, float *, int);

__global__ void k_axpy_sub(int64_t tot, const double *__restrict__ R, const double *__restrict__ Y,
                           double *__restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < tot) out[q] = R[q] - Y[q];
}

__global__ void k_fill_const(int k, double v, double *x) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < k) x[c] = v;
}

int spmm_launch_ld(ss_symbolic *s, const double *a, const double *b, const double *alpha, const double *beta,
                   const double *X, int64_t ldx, int k, double *Y, int64_t ldy) {
    ss_ctx *ctx = s->ctx;
    const int64_t threads = s->n * 32;
    const unsigned grid = (unsigned)((threads + 255) / 256);
#define SS_SPMM_ROWS(NC)                                                                                     \
    ss_launch(ctx, SS_K_SPMM, sss::k_spmm_rows<NC>, grid, 256, 0, ctx->stream, s->n, s->d_rowptr, s->d_colind, a, b, \
              alpha, beta, X, ldx, k, Y, ldy)
    if (k <= 4)
        ss_launch(ctx, SS_K_SPMM, sss::k_spmm_nnz<4>, grid, 256, 0, ctx->stream, s->n, s->d_rowptr, s->d_colind, a, b,
                  alpha, beta, X, ldx, k, Y, ldy);
    else if (k < 16)
        ss_launch(ctx, SS_K_SPMM, sss::k_spmm_nnz<16>, grid, 256, 0, ctx->stream, s->n, s->d_rowptr, s->d_colind, a,
                  b, alpha, beta, X, ldx, k, Y, ldy);
    else if (k <= 512) {
        switch ((k + 31) / 32) {     // exactly as many accumulators as the columns need
            case 1: SS_SPMM_ROWS(1); break;
            case 2: SS_SPMM_ROWS(2); break;
            case 3: SS_SPMM_ROWS(3); break;
            case 4: SS_SPMM_ROWS(4); break;
            case 5: SS_SPMM_ROWS(5); break;
            case 6: SS_SPMM_ROWS(6); break;
            case 7: SS_SPMM_ROWS(7); break;
            case 8: SS_SPMM_ROWS(8); break;
            case 9: SS_SPMM_ROWS(9); break;
            case 10: SS_SPMM_ROWS(10); break;
            case 11: SS_SPMM_ROWS(11); break;
            case 12: SS_SPMM_ROWS(12); break;
            case 13: SS_SPMM_ROWS(13); break;
            case 14: SS_SPMM_ROWS(14); break;
            case 15: SS_SPMM_ROWS(15); break;
            default: SS_SPMM_ROWS(16); break;
        }
    }
    else
        ss_launch(ctx, SS_K_SPMM, sss::k_spmm_cols, grid, 256, 0, ctx->stream, s->n, s->d_rowptr, s->d_colind, a, b,
                  alpha, beta, X, ldx, k, Y, ldy);
#undef SS_SPMM_ROWS
    ctx->add_flops(SS_K_SPMM, (beta ? 4.0 : 2.0) * (double)s->nnz * k);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

int spmm_launch(ss_symbolic *s, const double *a, const double *b, const double *alpha, const double *beta,
                const double *X, int k, double *Y) {
    return spmm_launch_ld(s, a, b, alpha, beta, X, k, k, Y, k);
}

__global__ void k_probe_vector(int64_t n, double *r) {
    // deterministic, sign-varying right-hand side: r_i = sin(0.7 i + 0.3) + 0.5 cos(1.9 i)
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) r[i] = sin(0.7 * (double)i + 0.3) + 0.5 * cos(1.9 * (double)i);
}

__global__ void k_absmax_diff(int64_t n, const double *__restrict__ r, const double *__restrict__ y,
                              unsigned long long *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double d = 0.0, m = 0.0;
    if (i < n) { d = fabs(r[i] - y[i]); m = fabs(r[i]); }
    for (int o = 16; o > 0; o >>= 1) {
        d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(isfinite(d) ? d : 1e300));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(m));
    }
}

// rho = ||r - (A - sigma B) x||_inf / ||r||_inf for one FP32 solve x of a probe vector r
int solve_contraction(ss_numeric *f, int j, double *rho) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t n = s->n;
    const unsigned g = (unsigned)((n + 255) / 256);
    double *r = nullptr, *x = nullptr, *y = nullptr, *co = nullptr;
    float *w = nullptr;
    unsigned long long *mx = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&r, sizeof(double) * (3 * n + 2), st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&w, sizeof(float) * n, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&mx, sizeof(unsigned long long) * 2, st));
    x = r + n;
    y = x + n;
    co = y + n;
    ss_launch(ctx, SS_K_MISC, k_probe_vector, g, 256, 0, st, n, r);
    ss_launch(ctx, SS_K_MISC, k_fill_const, 1, 32, 0, st, 1, 1.0, co);
    ss_launch(ctx, SS_K_MISC, k_fill_const, 1, 32, 0, st, 1, -f->sigma[j], co + 1);
    ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<float, double>, g, 256, 0, st, n, 1, s->d_perm, (const double *)r, w, 0);
    int rc = solve_permuted<float>(f, j, w, 1);
    if (rc != SS_OK) return rc;
    ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, float>, g, 256, 0, st, n, 1, s->d_perm, (const float *)w, x, 1);
    if ((rc = spmm_launch(s, f->a_vals, f->b_vals, co, co + 1, x, 1, y)) != SS_OK) return rc;
    SS_CUDA_TRY(ctx, cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 2, st));
    ss_launch(ctx, SS_K_MISC, k_absmax_diff, g, 256, 0, st, n, (const double *)r, (const double *)y, mx);
    unsigned long long h[2];
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, st));
    SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    cudaFreeAsync(r, st);
    cudaFreeAsync(w, st);
    cudaFreeAsync(mx, st);
    double d, m;
    std::memcpy(&d, &h[0], sizeof(d));
    std::memcpy(&m, &h[1], sizeof(m));
    *rho = m > 0 ? d / m : INFINITY;
    return SS_OK;
}

__global__ void k_shifted_vals(int64_t nnz, const double *__restrict__ a, const double *__restrict__ b, double sigma,
                               double *__restrict__ m) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        m[q] = a[q] - sigma * b[q];
}

// values of A - sigma_j B, made once per shift: a refinement residual then costs one
// multiply-add per nonzero and column instead of two
static int shifted_values(ss_numeric *f, int j, const double **out) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    if (!f->mvals[j]) {
        double *m = nullptr;
        SS_CUDA_TRY(ctx, cudaMalloc((void **)&m, sizeof(double) * std::max<int64_t>(1, s->nnz)));
        const unsigned g = (unsigned)std::min<int64_t>((s->nnz + 255) / 256, (int64_t)ctx->sm_count * 16);
        ss_launch(ctx, SS_K_MISC, k_shifted_vals, std::max(1u, g), 256, 0, ctx->stream, s->nnz, f->a_vals, f->b_vals,
                  f->sigma[j], m);
        f->mvals[j] = m;
    }
    *out = f->mvals[j];
    return SS_OK;
}

// Y = (A - sigma_j B) X: A X - sigma_j B X on the tensor cores (ss_set_gemm_mode), else one
// product with the values of A - sigma_j B.  (One pass over slices of A - sigma_j B was
// measured: its residuals carry the rounding of each shifted entry, and the FP32 solves
// then needed about 1.6x as many refinement steps, costing more than the pass it saves.)
static int spmm_shifted(ss_numeric *f, int j, const double *X, int k, double *Y) {
    if (oz_spmm_ok(f, k)) {
        const int which[2] = {0, 1};
        const double *cs[2] = {nullptr, nullptr};
        const double al[2] = {1.0, -f->sigma[j]};
        const int rc = oz_spmm(f, 2, which, cs, al, X, k, k, Y, k);
        if (rc != SS_ERR_OOM) return rc;
        f->oz_failed = true;
        f->sym->ctx->err.clear();
    }
    const double *mv = nullptr;
    int rc;
    if ((rc = shifted_values(f, j, &mv)) != SS_OK) return rc;
    return spmm_launch(f->sym, mv, mv, nullptr, nullptr, X, k, Y);
}

// X = (A - sigma B)^-1 R in the original order; FP64 R, X (may alias).
int solve_apply(ss_numeric *f, int j, const double *R, int k, double *X, int refine, int *steps_done, double target) {
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t tot = s->n * k;
    const unsigned g = (unsigned)((tot + 255) / 256);
    int rc;
    if (steps_done) *steps_done = 0;
    if (!ss_solves_f32(f, j)) {
        // FP64 factor: X_0 = M^-1 R, then `refine` steps X += M^-1 (R - M X) (iterative
        // refinement in the factor's own precision removes the effect of element growth
        // on the solve's backward error)
        double *w = nullptr, *x = nullptr, *y = nullptr;
        SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&w, sizeof(double) * tot, st));
        if (refine > 0) {
            SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&x, sizeof(double) * tot, st));
            SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&y, sizeof(double) * tot, st));
        }
        double *out = refine > 0 ? x : X;
        ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, k, s->d_perm, R, w, 0);
        if ((rc = solve_permuted<double>(f, j, w, k)) != SS_OK) return rc;
        ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, k, s->d_perm,
                  (const double *)w, out, 1);
        for (int it = 0; it < refine; ++it) {
            if ((rc = spmm_shifted(f, j, x, k, y)) != SS_OK) return rc;
            ss_launch(ctx, SS_K_MISC, k_axpy_sub, g, 256, 0, st, tot, R, (const double *)y, y);
            ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, k, s->d_perm,
                      (const double *)y, w, 0);
            if ((rc = solve_permuted<double>(f, j, w, k)) != SS_OK) return rc;
            ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, k, s->d_perm,
                      (const double *)w, x, 2);
            if (steps_done) (*steps_done)++;
        }
        if (refine > 0) {
            SS_CUDA_TRY(ctx, cudaMemcpyAsync(X, x, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
            cudaFreeAsync(x, st);
            cudaFreeAsync(y, st);
        }
        SS_CUDA_TRY(ctx, cudaFreeAsync(w, st));
        SS_CUDA_TRY(ctx, cudaGetLastError());
        return SS_OK;
    }
    // mixed: FP32 solves inside FP64 iterative refinement, X_0 = 0.  With a target the
    // residual decides when to stop; otherwise a requested refinement gets at least the
    // number of steps the shift's contraction factor needs to reach 1e-13
    if (target > 0.0) {
        refine = std::max(refine, 12);
    } else if (refine > 0 && f->rho[j] > 0.0 && f->rho[j] < 1.0) {
        refine = std::max(refine, std::min(8, (int)std::ceil(std::log(1e-13) / std::log(f->rho[j])) - 1));
    }
    unsigned long long *mx = nullptr;
    if (target > 0.0) SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&mx, sizeof(unsigned long long) * 2, st));
    float *wf = nullptr;
    double *r = nullptr, *y = nullptr, *x = nullptr;
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&wf, sizeof(float) * tot, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&r, sizeof(double) * tot, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&y, sizeof(double) * tot, st));
    SS_CUDA_TRY(ctx, cudaMallocAsync((void **)&x, sizeof(double) * tot, st));
    SS_CUDA_TRY(ctx, cudaMemsetAsync(x, 0, sizeof(double) * tot, st));
    for (int it = 0; it <= refine; ++it) {
        const double *rhs = R;
        if (it > 0) {
            if ((rc = spmm_shifted(f, j, x, k, y)) != SS_OK) return rc;
            if (mx) {
                SS_CUDA_TRY(ctx, cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 2, st));
                ss_launch(ctx, SS_K_MISC, k_absmax_diff, g, 256, 0, st, tot, R, (const double *)y, mx);
                unsigned long long h[2];
                SS_CUDA_TRY(ctx, cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, st));
                SS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
                double d, m;
                std::memcpy(&d, &h[0], sizeof(d));
                std::memcpy(&m, &h[1], sizeof(m));
                if (d <= target * m) break;
            }
            ss_launch(ctx, SS_K_MISC, k_axpy_sub, g, 256, 0, st, tot, R, y, r);
            rhs = r;
        }
        ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<float, double>, g, 256, 0, st, s->n, k, s->d_perm, rhs, wf, 0);
        if ((rc = solve_permuted<float>(f, j, wf, k)) != SS_OK) return rc;
        ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, float>, g, 256, 0, st, s->n, k, s->d_perm, wf, x, 2);
        if (steps_done && it > 0) (*steps_done)++;
    }
    SS_CUDA_TRY(ctx, cudaMemcpyAsync(X, x, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
    cudaFreeAsync(wf, st);
    cudaFreeAsync(r, st);
    cudaFreeAsync(y, st);
    cudaFreeAsync(x, st);
    if (mx) cudaFreeAsync(mx, st);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status ss_solve(ss_numeric *f, int32_t j, const double *R, int32_t k, double *X, int32_t refine) {
    if (!f) return SS_ERR_ARG;
    ss_ctx *ctx = f->sym->ctx;
    if (j < 0 || j >= f->n_shift || !R || !X || k <= 0 || refine < 0 || f->inertia_only)
        return ctx->set_error(SS_ERR_ARG, "ss_solve: bad argument (or an inertia-only factor)");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return solve_apply(f, j, R, k, X, refine, nullptr);
}

extern "C" ss_status ss_spmm(ss_symbolic *s, const double *a, const double *b, const double *alpha,
                             const double *beta, const double *X, int32_t k, double *Y) {
    if (!s) return SS_ERR_ARG;
    ss_ctx *ctx = s->ctx;
    if (ctx->device < 0 || !a || !X || !Y || k <= 0 || (beta && !b))
        return ctx->set_error(SS_ERR_ARG, "ss_spmm: bad argument or host-only context");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (ctx->gemm_mode == SS_GEMM_TENSOR && s->n >= 2048 && k >= 48)
        return oz_spmm_vals(s, a, b ? b : a, alpha, beta, X, k, k, Y, k);
    return spmm_launch(s, a, b ? b : a, alpha, beta, X, k, Y);
}

extern "C" ss_status ss_band_energy_grad(ss_symbolic *s, const double *X, const double *lambda, int32_t n_e,
                                         double *grad_a, double *grad_b) {
    if (!s) return SS_ERR_ARG;
    ss_ctx *ctx = s->ctx;
    if (ctx->device < 0 || !X || !lambda || n_e <= 0 || (!grad_a && !grad_b))
        return ctx->set_error(SS_ERR_ARG, "ss_band_energy_grad: bad argument or host-only context");
    const size_t smem = sizeof(double) * 2 * (size_t)n_e;
    if (smem > 220 * 1024) return ctx->set_error(SS_ERR_ARG, "ss_band_energy_grad: n_e too large (max 14080)");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    static std::mutex attr_mu;
    static std::vector<char> attr_seen;
    if (first_use_on_device(ctx->device, attr_mu, attr_seen))
        cudaFuncSetAttribute(sss::k_sddmm, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    ss_launch(ctx, SS_K_SDDMM, sss::k_sddmm, (unsigned)s->n, 256, smem, ctx->stream, s->n, s->d_rowptr, s->d_colind, X, lambda, n_e,
                                                             grad_a, grad_b);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}

// ------------------------------------------------------------------ allocation-free solve
// ss_solve_noalloc: the FP64 solve of ss_solve without any allocation, for callers that
// must not allocate device memory themselves or through a library -- code running
// under another framework's memory budget, inside a region where a new allocation would
// break an upstream memory plan, or where the allocator itself is unavailable.  Its
// working space is the file-scope array below: a permuted copy of the right-hand sides
// (N x k) followed by the per-level gather buffer of the backward sweep.
namespace {

constexpr int64_t kNoAllocScratchDoubles = 4ll * 1024 * 1024;   // 32 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// device address of g_noalloc_scratch per device, found once with that device current
std::mutex g_noalloc_mu;
double *g_noalloc_addr[64] = {};

int noalloc_scratch(ss_ctx *ctx, double **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 64) return ctx->set_error(SS_ERR_ARG, "ss_solve_noalloc: device index");
    if (!g_noalloc_addr[ctx->device]) {
        double *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return ctx->set_error(SS_ERR_CUDA, std::string("ss_solve_noalloc: cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
        }
        g_noalloc_addr[ctx->device] = p;
    }
    *out = g_noalloc_addr[ctx->device];
    return SS_OK;
}

}  // namespace

extern "C" ss_status ss_solve_noalloc(ss_numeric *f, int32_t j, const double *R, int32_t k, double *X) {
    if (!f) return SS_ERR_ARG;
    ss_symbolic *s = f->sym;
    ss_ctx *ctx = s->ctx;
    if (ctx->device < 0 || j < 0 || j >= f->n_shift || !R || !X || k <= 0 || f->inertia_only)
        return ctx->set_error(SS_ERR_ARG, "ss_solve_noalloc: bad argument, inertia-only factor or host-only context");
    if (f->shift_prec[j] != SS_FP64)
        return ctx->set_error(SS_ERR_ARG, "ss_solve_noalloc: shift was factored in FP32; use ss_solve");
    int32_t maxc = 0;
    for (const SolveLevel &sl : s->solve_levels) maxc = std::max(maxc, sl.count);
    const int64_t nk = s->n * (int64_t)k;
    const int64_t zoff = (nk + 31) / 32 * 32;                     // keep the gather buffer 256-byte aligned
    const int64_t need = zoff + (int64_t)maxc * NB * k;
    if (need > kNoAllocScratchDoubles)
        return ctx->set_error(SS_ERR_ARG, "ss_solve_noalloc: N*k + (widest solve level)*64*k = " +
                                              std::to_string(need) + " doubles exceeds the 4,194,304-double (32 MiB) "
                                              "scratch; use fewer right-hand sides or ss_solve");
    SS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    double *w = nullptr;
    int rc = noalloc_scratch(ctx, &w);
    if (rc != SS_OK) return rc;
    double *z = w + zoff;
    cudaStream_t st = ctx->stream;
    set_smem_attrs<double>(ctx->device);
    const unsigned g = (unsigned)((nk + 255) / 256);
    ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, (int)k, s->d_perm, R, w, 0);
    const double *arena = (const double *)f->arena[j];
    const int nchunk = (k + KC - 1) / KC, ndchunk = (k + KD - 1) / KD;
    const int nlev = (int)s->solve_levels.size();
    for (int L = 0; L < nlev; ++L) {
        const SolveLevel &sl = s->solve_levels[L];
        const int32_t *lp = s->d_solve_panels + sl.panel_off;
        ss_launch(ctx, SS_K_FWD_DIAG, k_fwd_diag<double>, dim3(sl.count, ndchunk), 256, diag_solve_smem<double>(), st,
                  lp, s->d_panels, (const double *)f->linv[j], (const int32_t *)f->piv[j], w, (int)k);
        if (sl.row_tiles > 0)
            ss_launch(ctx, SS_K_FWD_UPDATE, k_fwd_update<double>, dim3(sl.row_tiles, nchunk), 256,
                      tile_solve_smem<double>(), st, lp, s->d_solve_tile_pre + sl.panel_off, sl.count, s->d_panels,
                      s->d_idx, arena, w, (int)k);
    }
    for (int L = nlev - 1; L >= 0; --L) {
        const SolveLevel &sl = s->solve_levels[L];
        const int32_t *lp = s->d_solve_panels + sl.panel_off;
        if (sl.row_tiles > 0) {
            // the gather buffer keeps the previous call's contents: clear this level's part
            SS_CUDA_TRY(ctx, cudaMemsetAsync(z, 0, sizeof(double) * (int64_t)sl.count * NB * k, st));
            ss_launch(ctx, SS_K_BWD_GATHER, k_bwd_gather<double>, dim3(sl.row_tiles, nchunk), 256,
                      tile_solve_smem<double>(), st, lp, s->d_solve_tile_pre + sl.panel_off, sl.count, s->d_panels,
                      s->d_idx, arena, (const double *)w, (int)k, z);
        }
        ss_launch(ctx, SS_K_BWD_DIAG, k_bwd_diag<double>, dim3(sl.count, ndchunk), 256, diag_solve_smem<double>(), st,
                  lp, s->d_panels, (const double *)f->linv[j], (const double *)f->dblk[j],
                  (const int32_t *)f->piv[j], (const double *)z, sl.row_tiles > 0 ? 1 : 0, w, (int)k, 1);
    }
    ss_launch(ctx, SS_K_PERMUTE, k_permute_rows<double, double>, g, 256, 0, st, s->n, (int)k, s->d_perm,
              (const double *)w, X, 1);
    SS_CUDA_TRY(ctx, cudaGetLastError());
    return SS_OK;
}
