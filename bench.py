#!/usr/bin/env python
"""Benchmark: slice solves per second on synthetic Gaussian-orbital pencils.

A step is one pass of the whole hot path over one pencil: Lanczos DOS estimate
(Section 3.1), shift placement by CDOS roots, one batched LDL^T of A - sigma_j B for
every shift plus the two region bounds, inertia counts, shift-invert subspace
iterations on every probe until every slice validates (Section 2.2), and validation.
value = shifts (slice solves) completed per second; every validated eigenpair must
meet the normalised residual 1e-10.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun, one rank per GPU): every rank solves its own replica of the
workload (replicas only -- probes are independent and nothing is exchanged).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "gauss16": dict(config=2, n_e=1640, n_s=16,
                    name="gaussian-s 16x16x16 lattice, 4 fn/atom, N=16384, n_e=1640, 16 shifts"),
    "gauss6": dict(config=1, n_e=86, n_s=4,
                   name="gaussian-s 6x6x6 lattice, 4 fn/atom, N=864, n_e=86, 4 shifts"),
}
METRIC = "slice solves/s at N=110,592 (mixed vs FP64, resid<=1e-10); factor TFLOP/s"
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
FP64_ALU_PEAK_TFLOPS = 1.25                               # GB300 FP64 nominal: 152 SMs x 2 FMA/clk x 2 x 2.07 GHz
FLOP_CLASSES = {"schur", "panel", "fwd_update", "bwd_gather", "spmm", "gram", "gemm", "solve",
                "schur_f32", "panel_f32", "fwd_update_f32", "bwd_gather_f32", "solve_f32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gauss16", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-side", action="store_true", help="skip the FP64 side-by-side step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--sequence", type=int, default=0,
                    help="instead of the benchmark: solve this many pencils A_i = A_0 + 0.1 2^-i R of the "
                         "workload with probe migration and print one JSON line per pencil")
    ap.add_argument("--only-probe", action="store_true",
                    help="profiling case: factor one shift of the workload and run its probe for 6 iterations")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = sorted(float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit())
        mx = max((float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        if args.impl == "ours":
            torch.cuda.set_device(local)
    return ws, rank, local


def barrier_max(ws, value):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_rate(ws, units_per_rank, seconds_local):
    """Whole-job throughput of ws independent replicas: all ranks' units over the slowest
    rank's time (max over ranks)."""
    return ws * units_per_rank / barrier_max(ws, seconds_local)


# ----------------------------------------------------------------- oracle (CPU) leg
def oracle_sample(wl, seconds_budget=20.0):
    """Time the CPU oracle on a bounded sample and scale it to slice solves/s of the
    workload: the oracle's route to every slice's eigenpairs is one dense generalised
    eigensolve (O(N^3)); it is timed on the 6^3 pencil (N=864) and scaled by (N/864)^3."""
    from oracle import dense
    from workloads.pencils import config_pencil
    from oracle.build_oracle import build
    build()
    p1 = config_pencil(1)
    A, B = p1.dense("a"), p1.dense("b")
    reps, t0 = 0, time.perf_counter()
    while True:
        dense.gen_eig(A, B, vectors=True)
        reps += 1
        if time.perf_counter() - t0 > min(seconds_budget, 3.0) and reps >= 1:
            break
    t864 = (time.perf_counter() - t0) / reps
    n = 16384 if wl["config"] == 2 else 864
    t_full = t864 * (n / 864) ** 3
    return dict(value=wl["n_s"] / t_full, unit="slice solves/s", cores=dense.num_threads(), kind="oracle",
                sample=f"dense generalised eigensolve (Cholesky + Householder + QL, all eigenpairs) of the "
                       f"N=864 pencil, {reps} run(s) x {t864:.3f} s, scaled by (N/864)^3 to N={n} "
                       f"and divided among {wl['n_s']} slices"), t864


def run_reference(args, wl):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(wl, 1.0)
    vals = []
    for _ in range(args.steps):
        base, _ = oracle_sample(wl, 2.0)
        vals.append(base["value"])
    v = sum(vals) / len(vals)
    base["value"] = v
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "slice solves/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * wl["n_s"] / v, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": wl["name"], "l2": "inputs larger than L2"},
                      "cpu_baseline": base,
                      "e2e": {"value": v, "unit": "slice solves/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


# ----------------------------------------------------------------- GPU leg
def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    import numpy as np
    import torch

    from paper_1908_06043_gb300 import api, build
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver, default_basis_width
    from workloads.pencils import config_pencil, normal_block

    build()
    ws, rank, local = dist_setup(args)
    dev = torch.cuda.current_device()
    p = config_pencil(wl["config"])
    ctx = api.Context(dev)
    sym = ctx.analyze(p.rowptr, p.colind)
    info = sym.info
    a = torch.tensor(p.a, device="cuda")
    b = torch.tensor(p.b, device="cuda")
    n_e, n_s = wl["n_e"], wl["n_s"]
    k = 0                                     # probe basis: 2 c + 16 per window of c eigenvalues
    steps_dos, n_vec = 100, 4
    ha = torch.tensor(p.a).pin_memory()
    hb = torch.tensor(p.b).pin_memory()

    def step(precision, a_dev, b_dev, seed):
        t0 = time.perf_counter()
        start = torch.tensor(normal_block(p.n, n_vec, 1000 + seed), device="cuda")
        runs = sym.dos_estimate(a_dev, b_dev, steps_dos, start)
        model = DosModel(p.n, runs)
        solver = SliceSolver(sym, a_dev, b_dev, precision=precision)
        lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, n_e, n_s)
        t1 = time.perf_counter()
        res = solver.run(shifts, lam_min, lam_max, model, seed=seed, splits=splits, ks=ks)
        # band-energy gradient of the delivered eigenpairs (SDDMM on the stored pattern)
        tg = time.perf_counter()
        lam_d = torch.tensor(res.eigenvalues, device="cuda")
        ga, gb = sym.band_energy_grad(res.eigenvectors, lam_d)
        res.timings["grad"] = (ga, gb)
        res.timings["grad_s"] = time.perf_counter() - tg
        if args.verbose:
            print(f"[step {precision} seed={seed}] dos+place {t1 - t0:.3f}s factor {res.timings['factor_s']:.3f}s "
                  f"probes {res.timings['solve_s']:.3f}s total {time.perf_counter() - t0:.3f}s rounds {res.rounds} "
                  f"found {len(res.eigenvalues)} (nu(max)={res.timings['n_below_max']}) "
                  f"maxres {res.residuals.max() if len(res.residuals) else -1:.2e} "
                  f"slices {[i[:3] for i in res.slices]} "
                  f"quality {[(q[0], float(f'{q[1]:.2e}')) for q in res.timings['quality']]}", file=sys.stderr, flush=True)
        return res

    def check(res):
        ok = bool(res.timings["converged"]) and len(res.residuals) > 0 and float(res.residuals.max()) <= 1e-10
        ok = ok and all(n_conv >= n_exact for n_exact, _, n_conv, _ in res.slices)
        return ok

    if args.sequence:
        # SCF-like pencil sequence: DOS placement for the first pencil, k-means probe
        # migration with warm starts afterwards; per-pencil wall time and iterations
        from paper_1908_06043_gb300.driver import solve_sequence
        from workloads.pencils import scf_pencil, scf_sequence_perturbation
        r = scf_sequence_perturbation(p, seed=33)
        a_list = [torch.tensor(scf_pencil(p, r, i).a, device="cuda") for i in range(args.sequence)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = solve_sequence(sym, a_list, b, n_e, n_s, precision=args.precision,
                             start=torch.tensor(normal_block(p.n, n_vec, 1000), device="cuda"),
                             uniforms=np.random.default_rng(7).random(n_s))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for i, rs in enumerate(res):
            mig = rs.timings["migration"]
            print(json.dumps({"sequence_step": i, "workload": wl["name"], "precision": args.precision,
                              "seconds": rs.timings["total_s"], "factor_s": rs.timings["factor_s"],
                              "rounds": rs.rounds, "probe_iterations": rs.timings["iterations"],
                              "validated": check(rs), "eigenpairs": int(len(rs.eigenvalues)),
                              "max_resid": float(rs.residuals.max()),
                              "shifts": [float(x) for x in rs.shifts], "n_probes": len(rs.shifts),
                              "migration_init": mig["init"] if mig else "DOS placement",
                              "cluster_sizes": mig["sizes"] if mig else None}), flush=True)
        print(json.dumps({"sequence_total_s": t1 - t0, "pencils": len(res)}), flush=True)
        return

    if args.only_probe:
        # one representative probe of the workload (shift 8 of the placement), for ncu; a
        # short DOS run (20 steps, one vector) keeps the launch count small
        start = torch.tensor(normal_block(p.n, 1, 1000), device="cuda")
        model = DosModel(p.n, sym.dos_estimate(a, b, 20, start))
        solver = SliceSolver(sym, a, b, precision="fp64")
        lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, n_e, n_s)
        j = n_s // 2
        f = sym.factor(a, b, [shifts[j]], "fp64")
        V0 = torch.tensor(normal_block(p.n, ks[j], 7), device="cuda")
        t0 = time.perf_counter()
        pr = f.slice_solve(0, splits[j], splits[j + 1], V0, max_iter=6, check_every=2, allow_noconv=True)
        torch.cuda.synchronize()
        print(json.dumps({"only_probe": True, "sigma": shifts[j], "k": ks[j], "iterations": pr.iterations,
                          "seconds": time.perf_counter() - t0}), flush=True)
        return

    # warm-up; the last warm-up step is profiled per kernel class (CUDA events on the
    # launching stream) to pick the dominant kernel whose roofline the timed steps report
    for w in range(args.warmup):
        if w == args.warmup - 1:
            ctx.profile(api.L.KERNEL_CLASSES)
        res = step(args.precision, a, b, w)
    prof = {c: ctx.profile_query(c) for c in api.L.KERNEL_CLASSES}
    ctx.profile(())
    if args.warmup == 0:                       # nothing profiled: report the solve sweep
        prof["fwd_update"] = (1, 1e-9, 0.0)
    dom = max(prof, key=lambda c: prof[c][1])
    tot_prof = sum(v[1] for v in prof.values())

    # timed region (device-resident inputs)
    clocks = Clocks(dev)
    torch.cuda.synchronize()
    barrier(ws)
    clocks.start()
    ctx.profile([dom])
    n0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    results = []
    for s in range(args.steps):
        results.append(step(args.precision, a, b, 200 + s))
    e1.record()
    torch.cuda.synchronize()
    launches = ctx.launch_count() - n0
    dom_n, dom_t, dom_flops = ctx.profile_query(dom)
    ctx.profile(())
    clk = clocks.stop()
    barrier(ws)
    t_local = e0.elapsed_time(e1) / 1e3 / args.steps
    value = replica_rate(ws, n_s, t_local)
    t_step = ws * n_s / value
    all_ok = all(check(r) for r in results)
    factor_s = sum(r.timings["factor_s"] for r in results) / len(results)
    factor_tflops = (n_s + 2) * info["factor_flops"] / factor_s / 1e12

    # end to end through the public API with host buffers: H2D of the pencil values,
    # the step, D2H of the eigenvalues and residuals
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        d2h = 0
        for s in range(args.steps):
            a2 = ha.to("cuda", non_blocking=True)
            b2 = hb.to("cuda", non_blocking=True)
            r = step(args.precision, a2, b2, 300 + s)
            lam_h = torch.tensor(r.eigenvalues).cpu().numpy()
            d2h += lam_h.nbytes + r.residuals.nbytes
        torch.cuda.synchronize()
        e2e = {"value": replica_rate(ws, n_s, (time.perf_counter() - t0) / args.steps), "unit": "slice solves/s",
               "h2d_bytes_per_step": int(2 * p.nnz * 8),
               "d2h_bytes_per_step": int(d2h // args.steps)}

    # FP64 side by side (one step, same workload)
    fp64 = None
    if not args.no_fp64_side and args.precision == "mixed" and rank == 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = step("fp64", a, b, 400)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        fp64 = {"value": n_s / t64, "unit": "slice solves/s", "validated": check(r64),
                "factor_tflops": (n_s + 2) * info["factor_flops"] / r64.timings["factor_s"] / 1e12,
                "max_resid": float(r64.residuals.max()) if len(r64.residuals) else None}

    # roofline of the dominant kernel class: algorithmic flops of its launches in the
    # timed region (counted by the library from the schedule) over their event time
    per_launch = dom_t / max(dom_n, 1)
    if dom in FLOP_CLASSES and dom_t > 0:
        achieved = dom_flops / dom_t / 1e12
        f32 = dom.endswith("_f32")
        peak = FP32_ALU_PEAK_TFLOPS if f32 else FP64_ALU_PEAK_TFLOPS
        bound, unit = "alu", "TFLOP/s"
        peak_src = ("derived: 152 SMs x 128 FP32 lanes x 2 flops/FMA x 2.07 GHz" if f32 else
                    "nominal GB300 FP64 rate 1.25 TFLOP/s = 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz "
                    "(CUDA-core FP64; MEASURED_PEAKS.json has no FP64 figure)")
    else:
        achieved, bound, unit, peak, peak_src = None, "unknown", None, None, None
    traffic, traffic_src = None, None
    if dom == "solve" and dom_n > 0 and info["l_offdiag_entries"] > 0:
        # DRAM bytes per launch of the FP64 sweep solve, scaled from one ncu capture
        # (k = 304 probe solve on this pencil: 832.3 MB read + 91.1 MB written) by the
        # launch's width: L is read once per sweep, the N x k right-hand sides four times
        k_avg = dom_flops / dom_n / (4.0 * info["l_offdiag_entries"])
        def model(k):
            return 2 * 8.0 * info["l_offdiag_entries"] + 4 * 8.0 * p.n * k
        traffic = (832.3e6 + 91.1e6) * model(k_avg) / model(304)
        traffic_src = (f"ncu dram__bytes_read+write of one k=304 launch on the N=16384 pencil, scaled to the "
                       f"mean launch width k={k_avg:.0f} by the L + 4 N k model")
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": (achieved / peak) if achieved and peak else None, "traffic": traffic,
                "traffic_source": traffic_src,
                "launches": dom_n, "avg_launch_ms": 1e3 * per_launch,
                "share_of_profiled_time": prof[dom][1] / tot_prof if tot_prof else None,
                "peak_source": peak_src}

    cpu = None
    if rank == 0:
        cpu, _ = oracle_sample(wl)
    r0 = results[-1]
    out = {"metric": METRIC, "value": value, "unit": "slice solves/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": wl["name"], "precision": args.precision,
                      "probe_driver": "shift-invert subspace iteration (Alg. 2), Rayleigh-Ritz every 3rd iteration in the first round, once per later round",
                      "shift_placement": "DOS ball partition (radius 2h ball <= basis)",
                      "lanczos_steps": steps_dos, "lanczos_vectors": n_vec, "parallelism": f"replicas x{ws}",
                      "l2": "inputs larger than L2 (factor arena > 129 MB)",
                      "eigenpairs_validated": int(len(r0.eigenvalues)), "all_validated": all_ok,
                      "max_resid": float(r0.residuals.max()) if len(r0.residuals) else None,
                      "factor_tflops": factor_tflops, "factor_s_per_step": factor_s,
                      "rounds": r0.rounds, "probe_iterations": r0.timings["iterations"],
                      "shift_solve_precision": [q[0] for q in r0.timings["quality"]]},
           "fp64_side": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(launches), "clocks": clk,
           "profile_ms": {c: round(1e3 * v[1], 3) for c, v in prof.items() if v[0]},
           "profile_tflops": {c: round(v[2] / v[1] / 1e12, 3) for c, v in prof.items() if v[0] and v[2] > 0}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
