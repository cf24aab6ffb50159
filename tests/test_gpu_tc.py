"""Tensor-core Schur update (tcgen05.mma on sliced FP16 operands, FP64-accurate) against
the CUDA-core FP64 path and the oracle: the MMA tile self-test (exact integer products),
the inertia of factors whose every Schur step runs on the tensor cores (bit-exact against
the dense oracle's eigenvalue counts), and solves with those factors against the dense
solution and against the CUDA-core factor."""
import numpy as np
import pytest
import torch

from oracle import dense, spectral
from tests.gpu_util import mid_gap_shifts, setup
from workloads.pencils import config_pencil, normal_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mma_tile_selftest_exact(gpu_lib, seed):
    ctx = gpu_lib.Context(0)
    assert ctx.selftest_tc(seed) == 0.0


def _factor_pair(gpu_lib, p, shifts):
    ctx, sym, a, b = setup(gpu_lib, p)
    ctx.set_schur_mode("tensor", 0.0)            # every Schur step on the tensor cores
    n0 = ctx.launch_count()
    ctx.profile(["schur_tc", "schur"])
    ft = sym.factor(a, b, shifts, "fp64")
    tc_launches = ctx.profile_query("schur_tc")[0]
    simt_launches = ctx.profile_query("schur")[0]
    ctx.profile(())
    ctx.set_schur_mode("simt")
    fs = sym.factor(a, b, shifts, "fp64")
    ctx.set_schur_mode("tensor")
    return ctx, sym, a, b, ft, fs, tc_launches, simt_launches


def test_config1_tensor_core_factor_inertia_and_solves(gpu_lib):
    p = config_pencil(1)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    shifts = mid_gap_shifts(lam, [0, 10, 40, 85, 300, 600])
    ctx, sym, a, b, ft, fs, n_tc, n_simt = _factor_pair(gpu_lib, p, shifts)
    assert n_tc > 0 and n_simt == 0
    for j, s in enumerate(shifts):
        assert ft.inertia(j)[0] == spectral.count_below(lam, s)
        assert ft.inertia(j)[:3] == fs.inertia(j)[:3]
    A, B = p.dense("a"), p.dense("b")
    R = torch.tensor(normal_block(p.n, 6, 11), device="cuda")
    for j in (0, 3, 5):
        Xt = ft.solve(j, R, refine=0).cpu().numpy()
        Xs = fs.solve(j, R, refine=0).cpu().numpy()
        ref = np.linalg.solve(A - shifts[j] * B, R.cpu().numpy())
        assert np.abs(Xt - ref).max() <= 1e-9 * np.abs(ref).max()
        # the two factors agree as closely as two FP64 factorisations in another order
        assert np.abs(Xt - Xs).max() <= 1e-9 * np.abs(Xs).max()


def test_gauss16_tensor_core_inertia_matches_golden(gpu_lib):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gauss16_inertia.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    sig = [float(r[0]) for r in rows]
    neg = [int(r[1]) for r in rows]
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    ctx.set_schur_mode("tensor")
    ctx.profile(["schur_tc"])
    f = sym.factor(a, b, sig, "fp64")
    assert ctx.profile_query("schur_tc")[0] > 0
    ctx.profile(())
    for j in range(len(sig)):
        assert f.inertia(j)[0] == neg[j]
    # solve to 1e-10 with one refinement step against the pencil's own residual
    R = torch.tensor(normal_block(p.n, 4, 3), device="cuda")
    for j in (0, 3):
        X = f.solve(j, R, refine=1)
        res = sym.spmm(a, b, X, 1.0, -sig[j]) - R
        assert (res.norm() / R.norm()).item() <= 1e-10


def test_gauss16_mixed_tc_factor(gpu_lib):
    """SS_MIXED_TC: FP64 fronts on the tensor cores, FP32 solves from the rounded factor
    inside FP64 refinement: inertia bit-exact against the goldens, solves to 1e-10."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gauss16_inertia.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    sig = [float(r[0]) for r in rows]
    neg = [int(r[1]) for r in rows]
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    f = sym.factor(a, b, sig, "mixed_tc")
    R = torch.tensor(normal_block(p.n, 4, 3), device="cuda")
    used = []
    for j in range(len(sig)):
        assert f.inertia(j)[0] == neg[j]
        used.append(f.quality(j)[0])
        X = f.solve(j, R, refine=2)
        res = sym.spmm(a, b, X, 1.0, -sig[j]) - R
        assert (res.norm() / R.norm()).item() <= 1e-10
    assert set(used) <= {"fp64", "fp64+f32solve"} and "fp64+f32solve" in used


def _golden_inertia():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gauss16_inertia.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    return [float(r[0]) for r in rows], [int(r[1]) for r in rows]


@pytest.mark.parametrize("precision", ["fp64", "mixed_tc"])
def test_factor_graph_replay_matches_launches(gpu_lib, precision):
    """A captured factorisation replayed for new shifts gives the factor the kernel-by-kernel
    launches give: the same inertia, and solves that agree to rounding.  The solve kernels
    sum with atomics, so two solves with one factor already differ in the last bits; the
    FP32 solves of the mixed factor are compared after FP64 refinement."""
    sig, neg = _golden_inertia()
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    R = torch.tensor(normal_block(p.n, 3, 4), device="cuda")
    rf, tol = (0, 1e-10) if precision == "fp64" else (3, 1e-9)
    ref = []
    for s_ in sig[:3]:
        f = sym.factor(a, b, [s_], precision)
        ref.append((f.inertia(0)[0], f.solve(0, R, refine=rf)))
        f.close()
    ctx.set_factor_graph(True)
    n0 = ctx.launch_count()
    for t, s_ in enumerate(sig[:3]):              # capture on the first, replay on the others
        f = sym.factor(a, b, [s_], precision)
        assert f.inertia(0)[0] == ref[t][0] == neg[t]
        x = f.solve(0, R, refine=rf)
        assert ((x - ref[t][1]).abs().max() / ref[t][1].abs().max()).item() <= tol
        f.close()
    assert ctx.launch_count() - n0 > 3 * 100      # the replayed kernels are counted
    ctx.set_factor_graph(False)


def test_schur_autotuner(gpu_lib):
    """The autotuner times every factor step's Schur update on both paths and keeps the
    faster one per step; factors afterwards keep the exact inertia."""
    sig, neg = _golden_inertia()
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    n_tc = sym.autotune_schur(a, b, -1.0)
    assert 0 <= n_tc <= sym.info["n_panels"]
    f = sym.factor(a, b, sig, "fp64")
    assert [f.inertia(j)[0] for j in range(len(sig))] == neg
