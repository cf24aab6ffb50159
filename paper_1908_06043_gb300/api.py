"""Python binding of the slice-solve library: argument marshalling over the C ABI.

PyTorch provides device memory and the stream; every step of the path runs in the
library's CUDA kernels.  Names follow the C ABI: ``analyze``, ``factor``, ``inertia``,
``solve``, ``slice_solve``, ``dos_estimate``, ``band_energy_grad``, ``spmm``.

Blocks of vectors are torch float64 CUDA tensors of shape (N, k), row-major.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


class SisliceError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _dev(t: torch.Tensor, name: str, dtype=torch.float64) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Context:
    """Binds the library to one CUDA device and a torch stream (default: current)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        """device = -1 gives a host-only context (symbolic analysis without a GPU)."""
        self.lib = L.load()
        self.device = device
        if device >= 0:
            self.stream = stream if stream is not None else torch.cuda.current_stream(device)
            handle = self.stream.cuda_stream
        else:
            self.stream, handle = None, 0
        h = C.c_void_p()
        rc = self.lib.ss_create(C.byref(h), device, C.c_void_p(handle))
        if rc != L.SS_OK:
            raise SisliceError(rc, "ss_create failed")
        self.h = h

    def check(self, rc: int, what: str, allow=()):
        if rc != L.SS_OK and rc not in allow:
            msg = self.lib.ss_last_error(self.h).decode(errors="replace")
            raise SisliceError(rc, f"{what}: {msg}")
        return rc

    def sync(self):
        self.check(self.lib.ss_sync(self.h), "ss_sync")

    def analyze(self, rowptr: np.ndarray, colind: np.ndarray, nd_leaf: int = 0, dense: bool = False) -> "Symbolic":
        return analyze(self, rowptr, colind, nd_leaf, dense)

    def set_sweep_fusion(self, max_items: int = 0):
        """FP32 sweep solves: levels with at most max_items fused items take one grid barrier
        instead of two (0, the default: never; -1: those that fit in one pass of the
        resident blocks)."""
        self.check(self.lib.ss_set_sweep_fusion(self.h, int(max_items)), "ss_set_sweep_fusion")

    def set_solve_mode(self, mode: str):
        """"sweep": one cooperative launch per solve (default); "per_step": one launch per
        solve level and step."""
        m = {"sweep": L.SS_SOLVE_SWEEP_KERNEL, "per_step": L.SS_SOLVE_PER_STEP}[mode]
        self.check(self.lib.ss_set_solve_mode(self.h, m), "ss_set_solve_mode")

    def selftest_barrier(self, extra_arrivals: int = 0, limit: int = 200000):
        """Run the bounded grid-barrier self-test (raises SisliceError on a timeout)."""
        self.check(self.lib.ss_selftest_barrier(self.h, extra_arrivals, limit), "ss_selftest_barrier")

    def set_schur_mode(self, mode: str, min_flops: float = 2e7):
        """"tensor": FP64 Schur updates of factor steps with >= min_flops flops on the
        tensor cores (sliced FP16 operands, FP64-accurate); "simt": all on CUDA cores."""
        m = {"tensor": L.SS_SCHUR_TENSOR, "simt": L.SS_SCHUR_SIMT}[mode]
        self.check(self.lib.ss_set_schur_mode(self.h, m, float(min_flops)), "ss_set_schur_mode")

    def set_gemm_mode(self, mode: str):
        """"tensor": the probes' Gram and tall FP64 products on the tensor cores (exact
        digit slices, FP64 accumulation); "simt": on the CUDA cores."""
        m = {"tensor": L.SS_GEMM_TENSOR, "simt": L.SS_GEMM_SIMT}[mode]
        self.check(self.lib.ss_set_gemm_mode(self.h, m), "ss_set_gemm_mode")

    def set_factor_graph(self, on: bool = True):
        """Replay captured CUDA graphs of the factorisation (per analysis and wave shape)."""
        self.check(self.lib.ss_set_factor_graph(self.h, 1 if on else 0), "ss_set_factor_graph")

    def selftest_tc(self, seed: int = 1) -> float:
        """Largest error of one FP16 tensor-core MMA tile against the exact product."""
        out = C.c_double()
        self.check(self.lib.ss_selftest_tc(self.h, seed, C.byref(out)), "ss_selftest_tc")
        return out.value

    def dense_gram(self, X, Y, G=None):
        """G = X^T Y for CUDA FP64 tensors X (n x k1), Y (n x k2) with unit column stride;
        the tensor-core or CUDA-core product per set_gemm_mode."""
        n, k1 = X.shape
        k2 = Y.shape[1]
        if Y.shape[0] != n or X.stride(1) != 1 or Y.stride(1) != 1 or X.dtype != torch.float64 or Y.dtype != torch.float64:
            raise ValueError("dense_gram: FP64 operands with matching rows and unit column stride")
        if G is None:
            G = torch.empty(k1, k2, dtype=torch.float64, device=X.device)
        self.check(self.lib.ss_dense_gram(self.h, X.data_ptr(), X.stride(0), n, k1, Y.data_ptr(), Y.stride(0), k2,
                                          G.data_ptr()), "ss_dense_gram")
        return G

    def dense_gemm(self, X, Q, Y, alpha=1.0, beta=0.0, transq=False):
        """Y = beta Y + alpha X Q (or X Q^T) in place; CUDA FP64, unit column strides, Q
        contiguous."""
        n, k1 = X.shape
        k2 = Q.shape[0] if transq else Q.shape[1]
        if (Q.shape[1] if transq else Q.shape[0]) != k1 or tuple(Y.shape) != (n, k2) or not Q.is_contiguous() \
                or X.stride(1) != 1 or Y.stride(1) != 1:
            raise ValueError("dense_gemm: shapes or strides")
        self.check(self.lib.ss_dense_gemm(self.h, X.data_ptr(), X.stride(0), n, k1, Q.data_ptr(), k2, int(transq),
                                          float(alpha), float(beta), Y.data_ptr(), Y.stride(0)), "ss_dense_gemm")
        return Y

    def measure_peak(self, kind: str = "fp64", seconds: float = 0.5) -> float:
        """Measured FMA throughput of this GPU in TFLOP/s ("fp64" or "fp32")."""
        k = {"fp64": L.SS_PEAK_FP64_FMA, "fp32": L.SS_PEAK_FP32_FMA}[kind]
        out = C.c_double()
        self.check(self.lib.ss_measure_peak(self.h, k, seconds, C.byref(out)), "ss_measure_peak")
        return out.value

    def launch_count(self) -> int:
        """Kernels launched by the library since it was loaded."""
        return int(self.lib.ss_launch_count())

    def profile(self, classes=()):
        """Start per-class event timing of the named kernel classes (empty: stop)."""
        mask = 0
        for c in classes:
            mask |= 1 << L.KERNEL_CLASSES.index(c)
        self.check(self.lib.ss_profile(self.h, mask), "ss_profile")

    def profile_query_tensor(self, cls: str) -> float:
        """FP16 MMA flops a tensor-core kernel class issued since profile()."""
        out = C.c_double()
        self.check(self.lib.ss_profile_query_tensor(self.h, L.KERNEL_CLASSES.index(cls), C.byref(out)),
                   "ss_profile_query_tensor")
        return out.value

    def profile_query(self, cls: str):
        """(launches, seconds, algorithmic flops) of a kernel class since profile()
        (synchronises)."""
        n, t, fl = C.c_int64(), C.c_double(), C.c_double()
        self.check(self.lib.ss_profile_query(self.h, L.KERNEL_CLASSES.index(cls), C.byref(n), C.byref(t), C.byref(fl)),
                   "ss_profile_query")
        return n.value, t.value, fl.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.ss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def analyze(ctx: Context, rowptr: np.ndarray, colind: np.ndarray, nd_leaf: int = 0,
            dense: bool = False) -> "Symbolic":
    """Symbolic analysis of the full symmetric CSR pattern (host arrays).  dense=True is
    the dense-pencil path: no dissection, one front holding the whole (connected) matrix,
    factored by the same blocked LDL^T kernels (for pencils too dense to gain from
    sparsity)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    n = rowptr.size - 1
    opt = L.ss_options()
    opt.nd_leaf = max(1, n) if dense else nd_leaf
    h = C.c_void_p()
    ctx.check(ctx.lib.ss_analyze(ctx.h, n, _ptr(rowptr), _ptr(colind), C.byref(opt), C.byref(h)), "ss_analyze")
    return Symbolic(ctx, h, n, int(rowptr[-1]))


class Symbolic:
    def __init__(self, ctx: Context, h, n: int, nnz: int):
        self.ctx, self.h, self.n, self.nnz = ctx, h, n, nnz
        inf = L.ss_symbolic_info()
        ctx.check(ctx.lib.ss_symbolic_info_get(h, C.byref(inf)), "ss_symbolic_info_get")
        self.info = {f: getattr(inf, f) for f, _ in L.ss_symbolic_info._fields_}

    def validate(self):
        """Check every device-side index of the analysis against its buffer (host only)."""
        self.ctx.check(self.ctx.lib.ss_symbolic_validate(self.h), "ss_symbolic_validate")

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int32)
        self.ctx.check(self.ctx.lib.ss_symbolic_perm(self.h, _ptr(p)), "ss_symbolic_perm")
        return p

    def factor(self, a_vals, b_vals, sigma, precision: str = "fp64", allow_singular: bool = False) -> "Factor":
        return factor(self, a_vals, b_vals, sigma, precision, allow_singular)

    def spmm(self, a_vals, b_vals, X, alpha=None, beta=None) -> torch.Tensor:
        return spmm(self, a_vals, b_vals, X, alpha, beta)

    def factor_segments(self, a_vals, b_vals, row_segment, sigma) -> "Factor":
        return factor_segments(self, a_vals, b_vals, row_segment, sigma)

    def autotune_schur(self, a_vals, b_vals, sigma: float) -> int:
        """Time every factor step's Schur update on the tensor cores and on the CUDA cores
        (one inertia-only factorisation at sigma each) and keep the faster path per step.
        Returns the number of steps that chose the tensor cores."""
        _dev(a_vals, "a_vals")
        _dev(b_vals, "b_vals")
        n = C.c_int32()
        self.ctx.check(self.ctx.lib.ss_autotune_schur(self.h, _ptr(a_vals), _ptr(b_vals), float(sigma), C.byref(n)),
                       "ss_autotune_schur")
        return n.value

    def dos_estimate(self, a_vals, b_vals, steps: int, start: torch.Tensor):
        return dos_estimate(self, a_vals, b_vals, steps, start)

    def dos_lanczos(self, a_vals, b_vals, steps: int, x0: torch.Tensor):
        return dos_lanczos(self, a_vals, b_vals, steps, x0)

    def band_energy_grad(self, X, lam):
        return band_energy_grad(self, X, lam)

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.ss_symbolic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def factor(sym: Symbolic, a_vals, b_vals, sigma, precision: str = "fp64",
           allow_singular: bool = False) -> "Factor":
    """LDL^T of A - sigma_j B for every shift (one factor per shift).  precision "fp64",
    "mixed" (FP32 fronts, refactored in FP64 where one FP32 solve does not contract),
    "mixed_tc" (FP64 fronts on the tensor cores, FP32 solves from the factor rounded once
    where they contract), or "inertia" (FP64 fronts, only the inertia kept: no solves)."""
    ctx = sym.ctx
    _dev(a_vals, "a_vals")
    _dev(b_vals, "b_vals")
    if a_vals.numel() != sym.nnz or b_vals.numel() != sym.nnz:
        raise ValueError("value arrays must match the analysed pattern")
    sig = np.ascontiguousarray(np.atleast_1d(np.asarray(sigma, dtype=np.float64)))
    prec = {"fp64": L.SS_FP64, "mixed": L.SS_MIXED, "mixed_tc": L.SS_MIXED_TC,
            "inertia": L.SS_FP64 | L.SS_INERTIA_ONLY}[precision]
    h = C.c_void_p()
    rc = ctx.lib.ss_factor(sym.h, _ptr(a_vals), _ptr(b_vals), _ptr(sig), sig.size, prec, C.byref(h))
    ctx.check(rc, "ss_factor", allow=(L.SS_ERR_SINGULAR,) if allow_singular else ())
    return Factor(sym, h, a_vals, b_vals, sig, precision, rc == L.SS_ERR_SINGULAR)


def factor_segments(sym: Symbolic, a_vals, b_vals, row_segment, sigma) -> "Factor":
    """Inertia-only FP64 factorisation of many pencils stacked into one block-diagonal
    pattern, every pencil with its own shifts, all pencils in the same launches.
    row_segment: the pencil of each row (N ints); sigma: n_shift x n_seg shifts (row j: the
    shifts of call slot j, one per pencil).  Per-pencil counts: Factor.inertia_segments.
    A pivot below the singularity threshold in some pencil does not raise: the factor's
    `singular` is set and inertia_segments reports the pencil's tiny pivots."""
    ctx = sym.ctx
    _dev(a_vals, "a_vals")
    _dev(b_vals, "b_vals")
    if a_vals.numel() != sym.nnz or b_vals.numel() != sym.nnz:
        raise ValueError("value arrays must match the analysed pattern")
    seg = np.ascontiguousarray(np.asarray(row_segment, dtype=np.int32))
    sig = np.ascontiguousarray(np.atleast_2d(np.asarray(sigma, dtype=np.float64)))
    if seg.size != sym.n:
        raise ValueError("row_segment needs one entry per row")
    h = C.c_void_p()
    rc = ctx.lib.ss_factor_segments(sym.h, _ptr(a_vals), _ptr(b_vals), seg.ctypes.data, sig.shape[1],
                                    sig.ctypes.data, sig.shape[0], C.byref(h))
    ctx.check(rc, "ss_factor_segments", allow=(L.SS_ERR_SINGULAR,))
    f = Factor(sym, h, a_vals, b_vals, sig.max(axis=1), "inertia", rc == L.SS_ERR_SINGULAR)
    f.n_seg = sig.shape[1]
    return f


@dataclass
class ProbeResult:
    """One spectral probe SP(sigma) = (sigma, Lambda, X, R) plus solver statistics."""
    sigma: float
    theta: np.ndarray           # k Ritz values, ascending
    X: torch.Tensor             # N x k B-orthonormal Ritz vectors
    resid: np.ndarray           # normalised residual norms
    n_found: int                # Ritz values in (lo, hi]
    iterations: int
    refine_steps: int
    converged: bool
    max_resid_in_slice: float
    seconds: float


class Factor:
    def __init__(self, sym, h, a_vals, b_vals, sigma, precision, singular):
        self.sym, self.ctx, self.h = sym, sym.ctx, h
        self.a_vals, self.b_vals = a_vals, b_vals        # kept alive: the library reads them
        self.sigma, self.precision, self.singular = sigma, precision, singular

    def inertia(self, j: int = 0):
        """(n_neg, n_zero, n_pos, tiny_pivot) of A - sigma_j B."""
        return inertia(self, j)

    def stats(self, j: int = 0):
        """(min pivot / ||A - sigma B||_1 bound, max |L|, number of 2x2 pivots) of shift j."""
        mp, ml, n2 = C.c_double(), C.c_double(), C.c_int64()
        self.ctx.check(self.ctx.lib.ss_factor_stats(self.h, j, C.byref(mp), C.byref(ml), C.byref(n2)),
                       "ss_factor_stats")
        return mp.value, ml.value, n2.value

    def quality(self, j: int = 0):
        """(how shift j was factored and solved: "fp64", "mixed" (FP32 factor) or
        "fp64+f32solve" (FP64 factor, FP32 solves from its rounded copy), contraction factor
        rho of one FP32 solve)."""
        pr, rho = C.c_int32(), C.c_double()
        self.ctx.check(self.ctx.lib.ss_factor_quality(self.h, j, C.byref(pr), C.byref(rho)), "ss_factor_quality")
        name = {L.SS_FP64: "fp64", L.SS_MIXED: "mixed", L.SS_FP64_SOLVE32: "fp64+f32solve"}[pr.value]
        return name, rho.value

    def solve(self, j: int, R: torch.Tensor, refine: int = 2) -> torch.Tensor:
        return solve(self, j, R, refine)

    def inertia_segments(self, j: int = 0):
        """Per-pencil (n_neg, n_zero, n_pos, n_tiny) arrays of slot j of a factor_segments factor."""
        n = getattr(self, "n_seg", 0)
        if n <= 0:
            raise ValueError("not a factor_segments factor")
        out = [np.zeros(n, dtype=np.int64) for _ in range(4)]
        self.ctx.check(self.ctx.lib.ss_inertia_segments(self.h, j, *[o.ctypes.data for o in out]),
                       "ss_inertia_segments")
        return tuple(out)

    def slice_solve(self, j: int, lo: float, hi: float, V0: torch.Tensor, **kw) -> ProbeResult:
        return slice_solve(self, j, lo, hi, V0, **kw)

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.ss_factor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def inertia(f: Factor, j: int = 0):
    neg, zero, pos, tiny = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()
    f.ctx.check(f.ctx.lib.ss_inertia(f.h, j, C.byref(neg), C.byref(zero), C.byref(pos), C.byref(tiny)),
                "ss_inertia")
    return neg.value, zero.value, pos.value, bool(tiny.value)


def solve(f: Factor, j: int, R: torch.Tensor, refine: int = 2) -> torch.Tensor:
    _dev(R, "R")
    R2 = R if R.dim() == 2 else R[:, None]
    X = torch.empty_like(R2)
    f.ctx.check(f.ctx.lib.ss_solve(f.h, j, _ptr(R2), R2.shape[1], _ptr(X), refine), "ss_solve")
    return X.view_as(R)


def slice_solve(f: Factor, j: int, lo: float, hi: float, V0: torch.Tensor, tol: float = 1e-10,
                max_iter: int = 0, check_every: int = 1, refine: int = 2, n_expect: int = 0,
                allow_noconv: bool = False, driver: str = "subspace", k_out: int = 0,
                refine_from_start: bool = False, refine_ratio: float = 0.0) -> ProbeResult:
    """Spectral probe of shift j: shift-invert subspace iteration (Alg. 2; max_iter
    iterations) or shift-invert block Lanczos (max_iter blocks of width V0.shape[1],
    returning the k_out Ritz pairs nearest sigma_j)."""
    _dev(V0, "V0")
    n, k = V0.shape
    kout = k_out if (driver == "lanczos" and k_out > 0) else k
    opts = L.ss_solve_opts()
    opts.driver = {"subspace": L.SS_SUBSPACE, "lanczos": L.SS_BLOCK_LANCZOS}[driver]
    opts.max_iter, opts.check_every, opts.refine, opts.tol, opts.n_expect = max_iter, check_every, refine, tol, n_expect
    opts.k_out = kout
    opts.refine_from_start = 1 if refine_from_start else 0
    opts.refine_ratio = refine_ratio
    lam = np.empty(kout)
    res = np.empty(kout)
    X = torch.empty((n, kout), dtype=torch.float64, device=V0.device)
    nf = C.c_int32()
    st = L.ss_probe_stats()
    rc = f.ctx.lib.ss_slice_solve(f.h, j, lo, hi, C.byref(opts), _ptr(V0), k, _ptr(lam), _ptr(X), _ptr(res),
                                  C.byref(nf), C.byref(st))
    f.ctx.check(rc, "ss_slice_solve", allow=(L.SS_ERR_NOCONV,) if allow_noconv else ())
    return ProbeResult(float(f.sigma[j]), lam, X, res, nf.value, st.iterations, st.refine_steps,
                       bool(st.converged), st.max_resid_in_slice, st.seconds)


def _lanczos_call(fn, name, sym, a_vals, b_vals, steps, start):
    _dev(start, "start")
    nv = start.shape[1]
    th = np.zeros(steps * nv)
    z2 = np.zeros(steps * nv)
    m = np.zeros(nv, dtype=np.int32)
    sym.ctx.check(fn(sym.h, _ptr(a_vals), _ptr(b_vals), steps, nv, _ptr(start), _ptr(th), _ptr(z2), _ptr(m)), name)
    return [(th[c * steps:c * steps + m[c]].copy(), z2[c * steps:c * steps + m[c]].copy()) for c in range(nv)]


def dos_estimate(sym: Symbolic, a_vals, b_vals, steps: int, start: torch.Tensor):
    """Lanczos DOS runs on G^-1 A G^-T (B = G G^T) from i.i.d. N(0,1) start vectors y0
    (columns of start): list of (theta, zeta2) per run."""
    return _lanczos_call(sym.ctx.lib.ss_dos_estimate, "ss_dos_estimate", sym, a_vals, b_vals, steps, start)


def dos_lanczos(sym: Symbolic, a_vals, b_vals, steps: int, x0: torch.Tensor):
    """The same Lanczos runs in the B-orthonormal form from explicit start vectors x0."""
    return _lanczos_call(sym.ctx.lib.ss_dos_lanczos, "ss_dos_lanczos", sym, a_vals, b_vals, steps, x0)


def spmm(sym: Symbolic, a_vals, b_vals, X, alpha=None, beta=None) -> torch.Tensor:
    """Y = (alpha_j A + beta_j B) X (alpha defaults to 1, beta to 0)."""
    _dev(X, "X")
    k = X.shape[1]
    dev = X.device
    al = None if alpha is None else torch.tensor(np.broadcast_to(alpha, (k,)).copy(), dtype=torch.float64, device=dev)
    be = None if beta is None else torch.tensor(np.broadcast_to(beta, (k,)).copy(), dtype=torch.float64, device=dev)
    Y = torch.empty_like(X)
    sym.ctx.check(sym.ctx.lib.ss_spmm(sym.h, _ptr(a_vals), _ptr(b_vals), _ptr(al), _ptr(be), _ptr(X), k, _ptr(Y)),
                  "ss_spmm")
    return Y


def band_energy_grad(sym: Symbolic, X: torch.Tensor, lam: torch.Tensor):
    """Per-stored-entry dE/dA and dE/dB for E = sum(lam), X B-orthonormal (N x n_e)."""
    _dev(X, "X")
    lam = _dev(lam.contiguous(), "lambda")
    ga = torch.empty(sym.nnz, dtype=torch.float64, device=X.device)
    gb = torch.empty_like(ga)
    sym.ctx.check(sym.ctx.lib.ss_band_energy_grad(sym.h, _ptr(X), _ptr(lam), X.shape[1], _ptr(ga), _ptr(gb)),
                  "ss_band_energy_grad")
    return ga, gb


class BandEnergy(torch.autograd.Function):
    """E = sum of the n_e eigenvalues returned by ``solver(a_vals, b_vals)``.

    ``solver`` returns (lam [n_e] CUDA float64, X [N, n_e] B-orthonormal) or (lam, X,
    differentiable).  The backward pass is the SDDMM kernel of ``band_energy_grad``
    (Hellmann-Feynman): dE/dA sampled on the pattern is X X^T, dE/dB is -X Lambda X^T.
    When the solver reports E as not differentiable (lambda_(n_e+1) too close to
    lambda_(n_e)), both gradients are NaN."""

    @staticmethod
    def forward(ctx, a_vals, b_vals, sym, solver):
        out = solver(a_vals.detach(), b_vals.detach())
        lam, X = out[0], out[1]
        ctx.differentiable = bool(out[2]) if len(out) > 2 else True
        ctx.sym = sym
        ctx.save_for_backward(X, lam)
        return lam.sum()

    @staticmethod
    def backward(ctx, g):
        X, lam = ctx.saved_tensors
        ga, gb = band_energy_grad(ctx.sym, X.contiguous(), lam)
        if not ctx.differentiable:
            ga, gb = torch.full_like(ga, float("nan")), torch.full_like(gb, float("nan"))
        return g * ga, g * gb, None, None
