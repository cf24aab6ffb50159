"""Host-side SISLICE logic over the CUDA library (Alg. 1, Sections 2-3).

The device work -- factorisations, inertia, in-slice iterations, DOS sweeps -- runs in
the library; this module sequences it and holds the O(n_s k) scalar logic:

* ``DosModel``: the Lanczos DOS / CDOS closed forms (Eqs. 4-5) with Gaussian widths
  nu_j = d_j / 3, d_j the larger neighbour gap of the Ritz values (floored), averaged
  over start vectors; the interval expectation shift (Eqs. 7-8).
* ``cdos_partition``: n_s intervals of equal CDOS mass (Eq. 6, read as
  Phi(omega) = Phi(a) + K j), one shift per interval at its DOS expectation.
* ``region_for_lowest``: [lambda_min, lambda_max] holding exactly the n_e lowest
  eigenvalues, from the DOS estimate and exact inertia counts.
* ``validate``: candidates split at the slice midpoints, exact counts from inertia,
  the three cases of Section 2.2.
* ``ball_partition`` and ``dos_cluster_partition``: shift placement for non-uniform and
  clustered spectra (the latter is Alg. 3, DOSCluster, with its refinement).
* ``kmeans_shifts``, ``kmeans_pp_seeds``, ``migrate_probes``: k-means++ seeding, Lloyd
  iterations and the probe migration between SCF steps (Section 3.2); the uniforms are
  passed in.
* ``SliceSolver.run``: factor every shift (one batched call), inertia, probes, rounds of
  subspace iterations until every slice validates; ``run_with_recovery`` inserts probes
  where eigenvalues are missing (Section 3.3).
* ``plan_slices`` / ``solve_slice``: the same work one slice at a time -- shifts, window
  bounds and their exact counts placed once per pencil, then per slice one factor, its
  inertia, its probe and its validation (the benchmark's unit of work).
* ``solve_sequence``: a sequence of pencils on one pattern with migration, warm starts and
  the trace monitor of Eq. 9.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch
from scipy.special import erf

from . import api


# ----------------------------------------------------------------- DOS model
class DosModel:
    """phi / Phi of Eqs. 4-5 averaged over Lanczos runs [(theta, zeta2), ...]."""

    def __init__(self, n: int, runs):
        self.n = n
        self.runs = []
        for th, z2 in runs:
            th = np.asarray(th, dtype=np.float64)
            self.runs.append((th, np.asarray(z2, dtype=np.float64), self.widths(th)))

    @staticmethod
    def widths(theta: np.ndarray) -> np.ndarray:
        m = theta.size
        if m == 1:
            return np.ones(1)
        gap = np.diff(theta)
        d = np.empty(m)
        d[0], d[-1] = gap[0], gap[-1]
        if m > 2:
            d[1:-1] = np.maximum(gap[:-1], gap[1:])
        d = np.maximum(d, 1e-3 * (theta[-1] - theta[0]) / m)
        return d / 3.0

    def _kappa(self, w, th, nu):
        return (np.atleast_1d(w)[:, None] - th[None, :]) / (nu[None, :] * math.sqrt(2.0))

    def phi(self, w):
        out = 0.0
        for th, z2, nu in self.runs:
            k = self._kappa(w, th, nu)
            out = out + self.n / math.sqrt(2 * math.pi) * (z2 / nu * np.exp(-k * k)).sum(axis=1)
        return out / len(self.runs)

    def Phi(self, w):
        out = 0.0
        for th, z2, nu in self.runs:
            k = self._kappa(w, th, nu)
            out = out + 0.5 * self.n * (z2 * (erf(k) + 1.0)).sum(axis=1)
        return out / len(self.runs)

    def expectation(self, l, u):
        num = 0.0
        for th, z2, nu in self.runs:
            k = self._kappa(np.array([l, u]), th, nu)
            ps = th / 2 * erf(k) - nu / math.sqrt(2 * math.pi) * np.exp(-k * k)
            num += self.n * float((z2 * (ps[1] - ps[0])).sum())
        num /= len(self.runs)
        den = float(self.Phi(u)[0] - self.Phi(l)[0])
        return num / den if den > 0 else 0.5 * (l + u)

    def root(self, target, lo, hi, rel=1e-12):
        """omega in [lo, hi] with Phi(omega) = target (bisection; Phi is nondecreasing)."""
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if hi - lo <= rel * max(1.0, abs(mid)):
                break
            if self.Phi(mid)[0] < target:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    def theta_range(self):
        lo = min(float((th - 3 * nu).min()) for th, _, nu in self.runs)
        hi = max(float((th + 3 * nu).max()) for th, _, nu in self.runs)
        return lo, hi


def cdos_partition(model: DosModel, a: float, b: float, n_s: int):
    """n_s intervals of equal CDOS mass on [a, b] and the expectation shift of each."""
    Pa, Pb = float(model.Phi(a)[0]), float(model.Phi(b)[0])
    K = (Pb - Pa) / n_s
    roots = [a] + [model.root(Pa + K * j, a, b) for j in range(1, n_s)] + [b]
    iv = [(roots[j], roots[j + 1]) for j in range(n_s)]
    shifts = [model.expectation(l, u) for l, u in iv]
    return iv, shifts


def dos_clusters(model: DosModel, a: float, b: float, n_omega: int):
    """Alg. 3 (DOSCluster): cut [a, b] at the DOS minima between its local maxima on an
    n_omega-point grid and keep the pieces that hold a Lanczos Ritz value."""
    grid = np.linspace(a, b, n_omega)
    grid[0], grid[-1] = a, b
    f = model.phi(grid)
    up = np.empty(n_omega, dtype=bool)
    up[0] = f[0] > f[1]
    up[1:] = f[1:] > f[:-1]
    down = np.ones(n_omega, dtype=bool)
    down[1:-1] = f[1:-1] >= f[2:]
    peaks = np.flatnonzero(up & down)
    if peaks.size <= 1:
        return [(a, b)]
    cuts = [a]
    for p0, p1 in zip(peaks[:-1], peaks[1:]):
        if p1 - p0 >= 2:
            cuts.append(float(grid[p0 + 1 + int(np.argmin(f[p0 + 1:p1]))]))
        else:
            cuts.append(0.5 * float(grid[p0] + grid[p1]))
    cuts.append(b)
    ritz = np.concatenate([th for th, _, _ in model.runs])
    keep = [(cuts[j], cuts[j + 1]) for j in range(len(cuts) - 1)
            if np.any((ritz > cuts[j]) & (ritz <= cuts[j + 1])) or (j == 0 and np.any(ritz == cuts[0]))]
    return keep or [(a, b)]


def dos_cluster_partition(model: DosModel, a: float, b: float, n_s: int, n_omega: int,
                          merge_tol: float = 2.0, refine_tol: float = 50.0, max_rounds: int = 20):
    """Shift placement for clustered spectra (Section 3.1): Alg. 3 on a coarse grid;
    intervals holding fewer than merge_tol estimated eigenvalues join their adjacent
    neighbour with fewer; intervals holding more than refine_tol are searched again at
    2 C(l,u)/C(a,b) times the resolution until nothing splits; then gaps are closed at
    their midpoints and intervals are split at their CDOS median (largest first) or
    merged (smallest first, into the adjacent neighbour with fewer) until there are
    exactly n_s.  Returns (intervals, expectation shifts of Eq. 7)."""
    def count(iv):
        return float(model.Phi(iv[1])[0] - model.Phi(iv[0])[0])

    total = count((a, b))
    ivs = dos_clusters(model, a, b, n_omega)
    searched = set()
    for _ in range(max_rounds):
        merged = True
        while merged:                       # step 2
            merged = False
            for j, iv in enumerate(ivs):
                if count(iv) >= merge_tol:
                    continue
                adj = [q for q in (j - 1, j + 1) if 0 <= q < len(ivs)
                       and (ivs[q][1] == iv[0] if q < j else ivs[q][0] == iv[1])]
                if not adj:
                    continue
                t = min(adj, key=lambda q: (count(ivs[q]), q))
                joined = (min(ivs[t][0], iv[0]), max(ivs[t][1], iv[1]))
                ivs = sorted([x for q, x in enumerate(ivs) if q not in (j, t)] + [joined])
                merged = True
                break
        out, split = [], False              # steps 3 and 4
        for iv in ivs:
            c = count(iv)
            if c > refine_tol and iv not in searched:
                searched.add(iv)
                sub = dos_clusters(model, iv[0], iv[1], max(3, int(math.ceil(2.0 * c / total * n_omega))))
                if len(sub) >= 2:
                    out += sub
                    split = True
                    continue
            out.append(iv)
        ivs = sorted(out)
        if not split:
            break
    m = len(ivs)
    ivs = [((a if j == 0 else 0.5 * (ivs[j - 1][1] + ivs[j][0])),
            (b if j == m - 1 else 0.5 * (ivs[j][1] + ivs[j + 1][0]))) for j in range(m)]
    while len(ivs) < n_s:
        j = max(range(len(ivs)), key=lambda q: (count(ivs[q]), -q))
        lo, hi = ivs[j]
        mid = model.root(0.5 * float(model.Phi(lo)[0] + model.Phi(hi)[0]), lo, hi)
        ivs[j:j + 1] = [(lo, mid), (mid, hi)]
    while len(ivs) > n_s:
        j = min(range(len(ivs)), key=lambda q: (count(ivs[q]), q))
        t = min([q for q in (j - 1, j + 1) if 0 <= q < len(ivs)], key=lambda q: (count(ivs[q]), q))
        joined = (min(ivs[t][0], ivs[j][0]), max(ivs[t][1], ivs[j][1]))
        ivs = sorted([x for q, x in enumerate(ivs) if q not in (j, t)] + [joined])
    return ivs, [model.expectation(l, u) for l, u in ivs]


# ----------------------------------------------------------------- validation
def validate(shifts, lam_min, lam_max, probes, nneg_shift, nneg_min, nneg_max, tol, taus=None):
    """Section 2.2.  probes[j] = (theta, resid); taus[s] (optional) is the point that
    splits slice s = (shifts[s-1], shifts[s]) between its two probes (default: the
    midpoint).  Returns (selected [(probe, ritz)], per-slice records (n_exact, n_cand,
    n_conv, status))."""
    ns = len(shifts)
    bounds = [nneg_min] + list(nneg_shift) + [nneg_max]
    selected, info = [], []
    for s in range(ns + 1):
        lo = lam_min if s == 0 else shifts[s - 1]
        hi = lam_max if s == ns else shifts[s]
        cand = []
        if s == 0:
            th = probes[0][0]
            cand += [(0, i) for i in np.nonzero((th >= lam_min) & (th < hi))[0]]
        elif s == ns:
            th = probes[ns - 1][0]
            cand += [(ns - 1, i) for i in np.nonzero((th > lo) & (th <= lam_max))[0]]
        else:
            tau = 0.5 * (lo + hi) if taus is None else taus[s]
            th = probes[s - 1][0]
            cand += [(s - 1, i) for i in np.nonzero((th > lo) & (th <= tau))[0]]
            th = probes[s][0]
            cand += [(s, i) for i in np.nonzero((th > tau) & (th < hi))[0]]
        n_exact = bounds[s + 1] - bounds[s]
        cand.sort(key=lambda pi: (probes[pi[0]][1][pi[1]], pi[0], pi[1]))
        n_conv = sum(1 for pj, i in cand if probes[pj][1][i] <= tol)
        if n_exact == len(cand):
            status = "ok"
        elif n_exact > len(cand):
            status = "missing"
        else:
            status = "excess"
        selected += cand[:n_exact]
        info.append((n_exact, len(cand), n_conv, status))
    return selected, info


# ----------------------------------------------------------------- k-means migration
def kmeans_shifts(values, n_s, uniforms, max_iter=1000):
    """k-means++ seeding (first centroid uniform, then D^2-weighted) and Lloyd steps."""
    x = np.sort(np.asarray(values, dtype=np.float64))
    n = x.size
    cent = [x[min(n - 1, int(uniforms[0] * n))]]
    for c in range(1, n_s):
        d2 = np.min((x[:, None] - np.asarray(cent)[None, :]) ** 2, axis=1)
        tot = d2.sum()
        if tot <= 0:
            cent.append(x[min(n - 1, int(uniforms[c] * n))])
            continue
        idx = int(np.searchsorted(np.cumsum(d2) / tot, uniforms[c], side="right"))
        cent.append(x[min(n - 1, idx)])
    cent = np.asarray(cent)
    assign = None
    for _ in range(max_iter):
        a = np.argmin(np.abs(x[:, None] - cent[None, :]), axis=1)
        if assign is not None and np.array_equal(a, assign):
            break
        assign = a
        for c in range(n_s):
            m = a == c
            if m.any():
                cent[c] = x[m].mean()
    return np.sort(cent)


def _nearest(x, cent):
    return np.argmin(np.abs(x[:, None] - cent[None, :]), axis=1)


def _lloyd_keep_order(x, cent, max_iter=1000):
    """Lloyd steps from `cent` (order kept, empty clusters keep their centroid)."""
    cent = np.array(cent, dtype=np.float64)
    lab = _nearest(x, cent)
    for _ in range(max_iter):
        sums = np.bincount(lab, weights=x, minlength=cent.size)
        cnts = np.bincount(lab, minlength=cent.size)
        cent = np.where(cnts > 0, sums / np.maximum(cnts, 1), cent)
        new = _nearest(x, cent)
        if np.array_equal(new, lab):
            break
        lab = new
    return cent, lab


def kmeans_pp_seeds(values, n_s, uniforms):
    """k-means++ starting centroids (Section 3.2): the first uniformly, each next one
    with probability proportional to the squared distance to the nearest chosen one."""
    x = np.asarray(values, dtype=np.float64)
    n = x.size
    seeds = [x[min(n - 1, int(uniforms[0] * n))]]
    for c in range(1, n_s):
        d2 = np.min((x[:, None] - np.asarray(seeds)[None, :]) ** 2, axis=1)
        tot = d2.sum()
        pick = (min(n - 1, int(uniforms[c] * n)) if tot <= 0
                else min(n - 1, int(np.searchsorted(np.cumsum(d2) / tot, uniforms[c], side="right"))))
        seeds.append(x[pick])
    return np.asarray(seeds)


def migrate_probes(values, owner, old_shifts, init, balance=None):
    """Move the probes of one SCF step to the next (Section 3.2).

    The validated eigenvalues `values` (owner[i] = probe that produced values[i]) are
    split into len(old_shifts) clusters by k-means started from `init`.  Every
    non-empty cluster goes to the probe that produced most of its values (ties: nearest
    old shift, then lower index); clusters sharing a probe merge.  A probe left without
    a cluster is dropped and replaced: the largest cluster is split in two by 2-means
    (started from its extreme values), its probe keeps the half with more of its own
    values (ties: the half nearer its old shift) and a new probe takes the other half.
    With `balance`, a probe holding more than balance x the mean count is split the same
    way (insertion for load balance), up to twice as many probes as before.
    Returns [(shift, member indices)] sorted by shift, shift = mean of the members."""
    x = np.asarray(values, dtype=np.float64)
    owner = np.asarray(owner)
    old = np.asarray(old_shifts, dtype=np.float64)
    n_s = old.size
    _, lab = _lloyd_keep_order(x, init)
    owned = [[] for _ in range(n_s)]
    for c in np.unique(lab):
        idx = np.flatnonzero(lab == c)
        votes = np.bincount(owner[idx], minlength=n_s)
        top = np.flatnonzero(votes == votes.max())
        mu = x[idx].mean()
        owned[min(top, key=lambda q: (abs(old[q] - mu), q))].extend(idx.tolist())
    groups = [(p, np.array(sorted(m))) for p, m in enumerate(owned) if m]
    missing = n_s - len(groups)
    cap = float(balance) * x.size / n_s if balance else np.inf
    while missing > 0 or (len(groups) < 2 * n_s and max(m.size for _, m in groups) > cap):
        missing -= 1
        g = max(range(len(groups)), key=lambda q: (groups[q][1].size, -q))
        p, idx = groups[g]
        v = x[idx]
        if v.min() == v.max():
            break
        _, lab2 = _lloyd_keep_order(v, [v.min(), v.max()])
        halves = [idx[lab2 == 0], idx[lab2 == 1]]

        def rank(h):
            if p < 0:
                return (0, abs(x[h].mean() - x[idx].mean()))
            return (-int(np.count_nonzero(owner[h] == p)), abs(x[h].mean() - old[p]))
        keep = 0 if rank(halves[0]) <= rank(halves[1]) else 1
        groups[g] = (p, halves[keep])
        groups.append((-1, halves[1 - keep]))
    out = [(float(x[m].mean()), m.tolist()) for _, m in groups]
    return sorted(out, key=lambda t: t[0])


# ----------------------------------------------------------------- solver
@dataclass
class SliceResult:
    shifts: list
    lam_min: float
    lam_max: float
    eigenvalues: np.ndarray
    eigenvectors: torch.Tensor
    residuals: np.ndarray
    slices: list
    probes: list
    rounds: int
    timings: dict = field(default_factory=dict)
    owners: np.ndarray = None       # probe that produced each returned eigenpair


class SliceSolver:
    """Lowest-n_e eigenpairs of (A, B) by spectrum slicing on one GPU."""

    def __init__(self, sym: api.Symbolic, a_vals, b_vals, precision="mixed", tol=1e-10, refine=2,
                 refine_ratio=0.0, check_every=3):
        self.sym, self.a, self.b = sym, a_vals, b_vals
        self.precision, self.tol, self.refine = precision, tol, refine
        self.refine_ratio = refine_ratio       # 0: the library default (1e-1)
        self.check_every = check_every         # first-round Rayleigh-Ritz period (< 0: predictive)

    def count_below(self, sigmas):
        """Exact eigenvalue counts below each sigma (inertia of one batched FP64 factor
        that keeps no L)."""
        f = self.sym.factor(self.a, self.b, sigmas, "inertia")
        out = [f.inertia(j)[0] for j in range(len(sigmas))]
        f.close()
        return out

    def region_for_lowest(self, model: DosModel, n_e: int):
        """[lambda_min, lambda_max] with nu(lambda_min) = 0 and nu(lambda_max) = n_e."""
        lo_t, hi_t = model.theta_range()
        lam_min = lo_t
        span = hi_t - lo_t
        while self.count_below([lam_min])[0] > 0:
            lam_min -= 0.1 * span
        guess = model.root(n_e + 0.5, lo_t, hi_t)
        return lam_min, self.bound_at_count(guess, n_e, lam_min, span)

    def bound_at_count(self, guess: float, n_e: int, lam_min: float, span: float) -> float:
        """A point lambda with nu(lambda) = n_e (mid-gap within 1e-3 span), bracketed from
        `guess` and refined by bisection on inertia counts."""
        hi_t = guess + span
        c = self.count_below([guess])[0]
        lo, hi = (lam_min, guess) if c > n_e else (guess, guess)
        step = 0.01 * span
        while c <= n_e and hi < hi_t + span:         # bracket from above
            lo, hi = hi, hi + step
            step *= 2
            c = self.count_below([hi])[0]
        # nu(lo) <= n_e < nu(hi): bisect until a point with nu == n_e that sits
        # mid-gap is found
        clo = self.count_below([lo])[0]
        for _ in range(80):
            if clo == n_e and c > n_e and (hi - lo) < 1e-3 * span:
                break
            mid = 0.5 * (lo + hi)
            cm = self.count_below([mid])[0]
            if cm <= n_e:
                lo, clo = mid, cm
            else:
                hi, c = mid, cm
        return lo

    def run(self, shifts, lam_min, lam_max, model: DosModel = None, k=None, V0=None, max_rounds=30,
            block=64, seed=0, driver="subspace", iters_per_round=3, first_iters=80, splits=None, ks=None,
            warm=False):
        """Factor the shifts and the two region bounds in one batched call, build every
        probe, validate every slice, and refine the probes next to any slice that does
        not validate yet (fewer converged candidates than its exact count).

        Subspace probes (Alg. 2, default): basis k = 2 c + 16 (rounded up to 16) for a
        window holding about c eigenvalues (half of each neighbouring slice's exact count);
        the first round iterates until c - 2 window Ritz pairs converge, later rounds add
        `iters_per_round` iterations.  Block Lanczos probes: a Krylov basis of about 2.5x
        the count in blocks of `block` columns, restarted from the Ritz vectors."""
        t0 = time.perf_counter()
        ns = len(shifts)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        f = self.sym.factor(self.a, self.b, list(shifts) + [lam_min, lam_max], self.precision)
        ev1.record()
        counts = [f.inertia(j)[0] for j in range(ns + 2)]
        nneg, nneg_min, nneg_max = counts[:ns], counts[ns], counts[ns + 1]
        torch.cuda.synchronize()
        t_factor = ev0.elapsed_time(ev1) / 1e3
        n = self.sym.n
        tau = [None] + [0.5 * (shifts[s_ - 1] + shifts[s_]) if splits is None or splits[s_] is None else splits[s_]
                        for s_ in range(1, ns)]
        windows = []
        for j in range(ns):
            lo = lam_min if j == 0 else tau[j]
            hi = lam_max if j == ns - 1 else tau[j + 1]
            windows.append((lo, hi))
        # exact counts of the windows themselves: inertia at the split points between
        # neighbouring probes (one inertia-only factor), so each probe's first round stops
        # once its window's eigenvalues have converged
        inner = [windows[j][1] for j in range(ns - 1)]
        below = [nneg_min] + (self.count_below(inner) if inner else []) + [nneg_max]
        wcount = [below[j + 1] - below[j] for j in range(ns)]
        # basis sizes from the exact counts at the shifts (the window holds about half of
        # each neighbouring slice) or the DOS
        kout, m1, cnt = [], [], []
        for j in range(ns):
            left = (nneg[j] - (nneg[j - 1] if j > 0 else nneg_min)) * (0.5 if j > 0 else 1.0)
            right = ((nneg[j + 1] if j < ns - 1 else nneg_max) - nneg[j]) * (0.5 if j < ns - 1 else 1.0)
            c = int(math.ceil(left + right))
            cnt.append(c)
            ko = int(min(n, max(16, math.ceil(1.3 * c) + 16)))
            kout.append(ko)
            m1.append(int(max(2, math.ceil(2.5 * ko / block))))
        g = torch.Generator(device="cuda").manual_seed(seed)
        probes = [None] * ns
        Xs = [None] * ns
        f64 = {}                  # FP64 refactors of mixed shifts whose probes stalled
        stall = [0] * ns
        restarts = [0] * ns
        grown = [0] * ns
        best = [np.inf] * ns
        active = list(range(ns))
        rounds = 0
        t_solve = 0.0
        iters = [0] * ns
        info, sel = [], []
        while active and rounds < max_rounds:
            rounds += 1
            ts = time.perf_counter()
            for j in active:
                lo, hi = windows[j]
                if driver == "lanczos":
                    if Xs[j] is None:
                        v0 = V0[j] if V0 is not None and V0[j] is not None else torch.randn(n, min(block, n), generator=g, device="cuda",
                                                                     dtype=torch.float64)
                        mb = min(m1[j], max(1, n // v0.shape[1]))
                    else:
                        v0, mb = Xs[j], 2
                    ko = min(kout[j], mb * v0.shape[1])
                    pr = f.slice_solve(j, lo, hi, v0, tol=self.tol, max_iter=mb, refine=self.refine,
                                       driver="lanczos", k_out=ko, allow_noconv=True)
                else:
                    kk = k or (ks[j] if ks is not None else min(n, -(-(2 * cnt[j] + 16) // 16) * 16))
                    kk = min(n, 4096, max(kk, -(-(cnt[j] + 16) // 16) * 16, -(-(wcount[j] + 16) // 16) * 16))
                    if Xs[j] is None:
                        v0 = V0[j] if V0 is not None and V0[j] is not None else torch.randn(n, kk, generator=g, device="cuda",
                                                                     dtype=torch.float64)
                        # the first round stops once as many window Ritz pairs as the
                        # window's exact count have converged (a window without
                        # eigenvalues gets three iterations); validation then tops up
                        # with short rounds
                        mi, ne = (first_iters, wcount[j]) if wcount[j] > 0 else (3, 1)
                    else:
                        v0, mi, ne = Xs[j], iters_per_round, v0_never(Xs[j])
                    fj, jj = (f64[j], 0) if j in f64 else (f, j)
                    # Rayleigh-Ritz (the convergence check) every 3rd iteration in a first
                    # round and once at the end of a restart round: the iterated subspace
                    # does not depend on it
                    pr = fj.slice_solve(jj, lo, hi, v0, tol=self.tol, max_iter=mi, refine=self.refine,
                                        n_expect=ne, allow_noconv=True, refine_from_start=Xs[j] is not None or (warm and V0 is not None and V0[j] is not None),
                                        check_every=3 if Xs[j] is None else mi)
                probes[j] = pr
                Xs[j] = pr.X
                iters[j] += pr.iterations
            t_solve += time.perf_counter() - ts
            sel, info = validate(shifts, lam_min, lam_max, [(p.theta, p.resid) for p in probes], nneg,
                                 nneg_min, nneg_max, self.tol, taus=tau + [None])
            bad = set()
            for s_, (n_exact, n_cand, n_conv, status) in enumerate(info):
                if n_conv < n_exact:
                    if s_ > 0:
                        bad.add(s_ - 1)
                    if s_ < ns:
                        bad.add(s_)
            active = sorted(bad)
            # a probe whose slice is still short after every 4th restart round gets a
            # wider basis (+50 %, at least 16 random columns): its window holds more
            # eigenvalues near sigma than the estimate it was sized from
            for j in active:
                restarts[j] += 1
                cap = min(n, 4096)
                if driver != "lanczos" and restarts[j] % 4 == 0 and Xs[j] is not None and Xs[j].shape[1] < cap:
                    extra = min(cap - Xs[j].shape[1], max(16, Xs[j].shape[1] // 2))
                    Xs[j] = torch.cat([Xs[j], torch.randn(n, extra, generator=g, device="cuda",
                                                          dtype=torch.float64)], dim=1).contiguous()
                    grown[j] += 1
            # a mixed-precision probe whose window residuals stop improving is moved to an
            # FP64 factor of its shift (the FP32 factor limits its accuracy)
            for j in active:
                if self.precision not in ("mixed", "mixed_tc") or j in f64 or f.quality(j)[0] == "fp64":
                    continue
                lo, hi = windows[j]
                pr = probes[j]
                inw = (pr.theta > lo) & (pr.theta <= hi)
                r = float(np.sort(pr.resid[inw])[-1]) if inw.any() else np.inf
                stall[j] = stall[j] + 1 if not (r < 0.5 * best[j]) else 0
                best[j] = min(best[j], r)
                if stall[j] >= 3:
                    f64[j] = self.sym.factor(self.a, self.b, [shifts[j]], "fp64")
        lam = np.array([probes[pj].theta[i] for pj, i in sel])
        res = np.array([probes[pj].resid[i] for pj, i in sel])
        order = np.argsort(lam, kind="stable")
        X = torch.stack([probes[sel[q][0]].X[:, sel[q][1]] for q in order], dim=1) if sel else None
        quality = [("fp64", 0.0) if j in f64 else f.quality(j) for j in range(ns)]
        f.close()
        for g64 in f64.values():
            g64.close()
        return SliceResult(list(shifts), lam_min, lam_max, lam[order], X, res[order], info, probes, rounds,
                           dict(factor_s=t_factor, solve_s=t_solve, total_s=time.perf_counter() - t0,
                                iterations=iters, n_below_max=nneg_max, n_below_min=nneg_min,
                                converged=not active, fp64_refactors=sorted(f64), quality=quality,
                                basis_growth=grown),
                           owners=np.array([sel[q][0] for q in order], dtype=np.int64))

    def run_with_recovery(self, shifts, lam_min, lam_max, model: DosModel = None, max_inserts: int = 2,
                          **kw):
        """run(), then recovery of missing eigenvalues (Section 3.3): while some slice
        holds fewer converged eigenpairs than its inertia count, new probes are inserted
        in each such slice (two placed in it by ball_partition on the DOS, else one at its
        midpoint) and the probes run again, the old ones restarted from their Ritz
        vectors.  Returns
        the last SliceResult; timings["inserted"] lists the shifts added per attempt."""
        res = self.run(shifts, lam_min, lam_max, model, **kw)
        inserted = []
        shifts = list(shifts)
        while not res.timings["converged"] and len(inserted) < max_inserts:
            ns = len(shifts)
            add = []
            for s_, (n_exact, _, n_conv, _) in enumerate(res.slices):
                if n_conv >= n_exact:
                    continue
                lo = lam_min if s_ == 0 else shifts[s_ - 1]
                hi = lam_max if s_ == ns else shifts[s_]
                if model is not None:               # two probes placed in the slice by the DOS
                    add += [x for x in ball_partition(model, lo, hi, 2)[1] if lo < x < hi]
                else:
                    add.append(0.5 * (lo + hi))
            inserted.append(add)
            old = {sh: pr.X for sh, pr in zip(shifts, res.probes)}
            shifts = sorted(shifts + add)
            V0 = [old.get(sh) for sh in shifts]
            kw2 = dict(kw)
            kw2.pop("splits", None)
            kw2.pop("ks", None)
            res = self.run(shifts, lam_min, lam_max, model, V0=V0, warm=True, **kw2)
        res.timings["inserted"] = inserted
        return res

    def place_shifts(self, model: DosModel, n_e: int, n_s: int, margin: float = 0.01, mode: str = "ball"):
        """Region and shifts from the DOS alone: lambda_min below every Ritz value,
        lambda_max at Phi = (1 + margin) n_e + 1, and n_s intervals between them, by the
        CDOS roots of Eq. 6 with expectation shifts (mode "cdos"), by DOSCluster (Alg. 3,
        mode "cluster") or by ball_partition (mode "ball").  Returns (lambda_min, lambda_max, shifts, splits, basis sizes):
        splits[s] divides slice s between probes s-1 and s (None: the midpoints)."""
        lo_t, hi_t = model.theta_range()
        lam_min = lo_t
        lam_max = model.root((1.0 + margin) * n_e + 1.0, lo_t, hi_t)
        if mode == "cdos":
            _, shifts = cdos_partition(model, lam_min, lam_max, n_s)
            return lam_min, lam_max, shifts, None, None
        if mode == "cluster":
            # DOSCluster intervals (Alg. 3 with refinement), expectation shifts; each basis
            # covers the estimated eigenvalues within its shift's distance to the far end
            n_om = 10 * max(len(th) for th, _, _ in model.runs)
            iv, shifts = dos_cluster_partition(model, lam_min, lam_max, n_s, n_om)
            ks = []
            for s_, (l, u) in zip(shifts, iv):
                r = max(s_ - l, u - s_)
                ks.append(int(-(-(1.15 * float(model.Phi(s_ + r)[0] - model.Phi(s_ - r)[0]) + 16) // 16) * 16))
            return lam_min, lam_max, shifts, [None] + [iv[j][0] for j in range(1, n_s)], ks
        iv, shifts, balls = ball_partition(model, lam_min, lam_max, n_s)
        splits = [None] + [iv[j][0] for j in range(1, n_s)]
        ks = [int(-(-(1.15 * bc + 16) // 16) * 16) for bc in balls]
        return lam_min, lam_max, shifts, splits, ks


@dataclass
class SlicePlan:
    """Shifts and windows of one pencil, placed once and reused by every slice solve:
    probe j owns the window (bounds[j], bounds[j+1]] around shifts[j]; counts[i] is the
    exact number of eigenvalues below bounds[i] (Sylvester inertia of an FP64 factor)."""
    shifts: list
    bounds: list
    counts: list
    ks: list
    lam_min: float
    lam_max: float

    def window(self, j: int):
        return self.bounds[j], self.bounds[j + 1]

    def exact(self, j: int) -> int:
        return self.counts[j + 1] - self.counts[j]


@dataclass
class SliceOutcome:
    """One validated slice solve: the eigenpairs of window j (Section 2.2 validation)."""
    j: int
    sigma: float
    theta: np.ndarray
    X: torch.Tensor
    resid: np.ndarray
    n_exact: int
    n_neg_sigma: int
    ok: bool
    factor_s: float
    iterations: int
    rounds: int
    precision_used: str


def plan_slices(solver: "SliceSolver", model: "DosModel", n_e: int, n_s: int, mode: str = "ball",
                windows=None) -> SlicePlan:
    """Place n_s shifts for the lowest n_e eigenvalues (place_shifts) and count the
    eigenvalues below the window bounds with one batched inertia-only FP64 factor: below
    every bound, or (windows = a list of window indices) only below the bounds of those
    windows (the other counts stay None and those windows cannot be solved)."""
    lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, n_e, n_s, mode=mode)
    inner = [splits[j] if splits is not None and splits[j] is not None else 0.5 * (shifts[j - 1] + shifts[j])
             for j in range(1, n_s)]
    bounds = [lam_min] + inner + [lam_max]
    need = sorted(set(range(n_s + 1)) if windows is None else {b for j in windows for b in (j, j + 1)})
    got = solver.count_below([bounds[b] for b in need]) if need else []
    counts = [None] * (n_s + 1)
    for b, c in zip(need, got):
        counts[b] = c
    if ks is None:
        ks = [None] * n_s
    n = solver.sym.n
    out = []
    for j, k in enumerate(ks):
        c = counts[j + 1] - counts[j] if counts[j] is not None and counts[j + 1] is not None else 0
        out.append(min(n, 4096, max(k or 0, _ceil16(2 * c + 16), _ceil16(c + 16))))
    return SlicePlan(list(shifts), bounds, counts, out, lam_min, lam_max)


def count_below_stacked(sym_stack, a_stack, b_stack, row_segment, sigmas):
    """Exact eigenvalue counts of many independent pencils at once: the pencils stacked
    into one block-diagonal pattern (workloads.pencils.stack_pencils), sigmas[p] the list
    of shifts of pencil p (lists of any lengths).  One inertia-only FP64 factorisation of
    the stack per call slot, every pencil at its own shift in the same launches
    (ss_factor_segments); a pencil with fewer shifts repeats its last one.  Returns one
    list of counts per pencil.  Raises if a shift is within the singularity threshold of
    an eigenvalue of its pencil."""
    n_seg = len(sigmas)
    width = max(len(x) for x in sigmas)
    tab = np.array([[float(sigmas[p][min(j, len(sigmas[p]) - 1)]) for p in range(n_seg)] for j in range(width)])
    f = sym_stack.factor_segments(a_stack, b_stack, row_segment, tab)
    out = [[] for _ in range(n_seg)]
    try:
        for j in range(width):
            neg, _, _, tiny = f.inertia_segments(j)
            for p in range(n_seg):
                if j < len(sigmas[p]):
                    if tiny[p]:
                        raise api.SisliceError(api.L.SS_ERR_SINGULAR, f"pencil {p}: shift {tab[j, p]} is within the "
                                                                  f"singularity threshold of an eigenvalue")
                    out[p].append(int(neg[p]))
    finally:
        f.close()
    return out


def plan_with_counts(plan: SlicePlan, counts, n: int) -> SlicePlan:
    """The plan of an N = n pencil with its window-bound counts (and the basis widths that
    follow from them, as plan_slices sets them) taken from `counts` (one per bound)."""
    ks = []
    for j, k in enumerate(plan.ks):
        c = counts[j + 1] - counts[j]
        ks.append(min(n, 4096, max(k or 0, _ceil16(2 * c + 16), _ceil16(c + 16))))
    return SlicePlan(list(plan.shifts), list(plan.bounds), list(counts), ks, plan.lam_min, plan.lam_max)


def solve_slice(solver: "SliceSolver", plan: SlicePlan, j: int, seed: int = 0, first_iters: int = 80,
                iters_per_round: int = 3, max_rounds: int = 30, V0: torch.Tensor = None) -> SliceOutcome:
    """One slice solve (the unit of the benchmark): factor A - sigma_j B, its inertia,
    the shift-invert probe of window j (Alg. 2) until as many Ritz pairs as the window's
    exact count meet the residual tolerance, then validation (Section 2.2): the window's
    converged count equals its inertia count, and the converged values below sigma_j
    number n_neg(sigma_j) - nu(lower bound).  A probe still short after a round restarts
    from its Ritz vectors; every 4th restart widens its basis by half (at least 16
    columns); a mixed-precision probe whose residuals stall for 3 rounds moves to an FP64
    factor of its shift.  Extra converged candidates (case 3) keep the smallest
    residuals.  V0 (N x c, optional) warm-starts the probe, e.g. with the window's
    eigenvectors of a nearby pencil; N(0,1) columns fill it up to the planned width."""
    sym, n = solver.sym, solver.sym.n
    lo, hi = plan.window(j)
    exact = plan.exact(j)
    sigma = plan.shifts[j]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    f = sym.factor(solver.a, solver.b, [sigma], solver.precision)
    ev1.record()
    neg = f.inertia(0)[0]
    g = torch.Generator(device="cuda").manual_seed(seed)
    kk = plan.ks[j]
    warm = V0 is not None
    if warm:
        extra = max(0, kk - V0.shape[1])
        V0 = torch.cat([V0, torch.randn(n, extra, generator=g, device="cuda", dtype=torch.float64)],
                       dim=1).contiguous() if extra else V0.contiguous()
    else:
        V0 = torch.randn(n, kk, generator=g, device="cuda", dtype=torch.float64)
    pr = f.slice_solve(0, lo, hi, V0, tol=solver.tol, max_iter=first_iters, refine=solver.refine,
                       n_expect=max(1, exact), allow_noconv=True, check_every=solver.check_every,
                       refine_from_start=warm,
                       refine_ratio=solver.refine_ratio)
    iters, rounds = pr.iterations, 1
    f64, best, stall = None, np.inf, 0

    def n_conv(q):
        return int(np.sum((q.theta > lo) & (q.theta <= hi) & (q.resid <= solver.tol)))

    while n_conv(pr) < exact and rounds < max_rounds:
        rounds += 1
        X = pr.X
        if rounds % 4 == 0 and X.shape[1] < min(n, 4096):
            extra = min(min(n, 4096) - X.shape[1], max(16, X.shape[1] // 2))
            X = torch.cat([X, torch.randn(n, extra, generator=g, device="cuda", dtype=torch.float64)],
                          dim=1).contiguous()
        if solver.precision in ("mixed", "mixed_tc") and f64 is None and f.quality(0)[0] != "fp64":
            inw = (pr.theta > lo) & (pr.theta <= hi)
            r = float(np.sort(pr.resid[inw])[-1]) if inw.any() else np.inf
            stall = stall + 1 if not (r < 0.5 * best) else 0
            best = min(best, r)
            if stall >= 3:
                f64 = sym.factor(solver.a, solver.b, [sigma], "fp64")
        fj = f64 if f64 is not None else f
        pr = fj.slice_solve(0, lo, hi, X, tol=solver.tol, max_iter=iters_per_round, refine=solver.refine,
                            n_expect=max(1, exact), allow_noconv=True, refine_from_start=True,
                            check_every=iters_per_round, refine_ratio=solver.refine_ratio)
        iters += pr.iterations
    torch.cuda.synchronize()
    factor_s = ev0.elapsed_time(ev1) / 1e3
    quality = "fp64" if f64 is not None else f.quality(0)[0]
    inw = (pr.theta > lo) & (pr.theta <= hi) & (pr.resid <= solver.tol)
    idx = np.nonzero(inw)[0]
    if idx.size > exact:                      # case 3: keep the smallest residuals
        idx = np.sort(idx[np.argsort(pr.resid[idx], kind="stable")[:exact]])
    theta = pr.theta[idx]
    ok = idx.size == exact and int(np.sum(theta < sigma)) == neg - plan.counts[j]
    X = pr.X[:, torch.as_tensor(idx, device=pr.X.device)] if idx.size else pr.X[:, :0]
    f.close()
    if f64 is not None:
        f64.close()
    return SliceOutcome(j, sigma, theta, X, pr.resid[idx], exact, neg, bool(ok), factor_s, iters, rounds, quality)


def solve_plan(solver: "SliceSolver", plan: SlicePlan, seed: int = 0, warm=None, first_iters: int = 80):
    """Every window of the plan (solve_slice), optionally warm-started from a list of
    per-window start blocks.  Returns (eigenvalues ascending, eigenvectors N x n_e as a
    CUDA tensor, outcomes); raises if a window does not validate."""
    outs = []
    for j in range(len(plan.shifts)):
        o = solve_slice(solver, plan, j, seed=seed + j, first_iters=first_iters,
                        V0=None if warm is None else warm[j])
        if not o.ok:
            raise RuntimeError(f"window {j} did not validate ({o.theta.size} of {o.n_exact})")
        outs.append(o)
    lam = np.concatenate([o.theta for o in outs])
    X = torch.cat([o.X for o in outs], dim=1)
    order = np.argsort(lam, kind="stable")
    return lam[order], X[:, torch.as_tensor(order, device=X.device)].contiguous(), outs


def energy_differentiable(solver: "SliceSolver", lam: np.ndarray, gap: float = 1e-8) -> bool:
    """The band energy E = sum of the n_e lowest eigenvalues is differentiable when
    lambda_(n_e+1) - lambda_(n_e) >= gap: Sylvester's inertia at lambda_(n_e) + gap must
    still count n_e eigenvalues below it."""
    n_e = int(np.asarray(lam).size)
    return solver.count_below([float(np.max(lam)) + gap])[0] == n_e


def v0_never(X) -> int:
    """An n_expect no probe can reach: run exactly max_iter iterations."""
    return X.shape[1] + 1


def ball_partition(model: DosModel, a: float, b: float, n_s: int, ratio: float = 2.0):
    """Intervals for shift-invert probes when the DOS is far from uniform.

    A probe at sigma converges the eigenvalues of its interval [l, u] (sigma the midpoint,
    half-width h) at a rate set by the first eigenvalue outside its basis; if its basis
    holds every eigenvalue within ratio * h of sigma, that rate is about 1 / ratio per
    iteration.  Greedily from a, each interval is made as wide as possible with
    Phi(sigma + ratio h) - Phi(sigma - ratio h) <= K; the budget K is bisected until the
    greedy pass uses at most n_s intervals, and the intervals with the largest counts are
    then halved until there are exactly n_s.  Returns (intervals, shifts, ball counts)."""
    def count(x, y):
        return float(model.Phi(y)[0] - model.Phi(x)[0])

    def greedy(K, limit):
        iv, l = [], a
        while l < b and len(iv) <= limit:
            if count(2 * a - b, b) <= K:           # everything left fits in one ball
                u = b
            else:
                lo, hi = l, b
                for _ in range(60):
                    u = 0.5 * (lo + hi)
                    s_, h = 0.5 * (l + u), 0.5 * (u - l)
                    if count(s_ - ratio * h, s_ + ratio * h) <= K:
                        lo = u
                    else:
                        hi = u
                u = lo if lo > l else hi
                if count(u, b) < 0.5:               # nothing left for another interval
                    u = b
            iv.append((l, u))
            l = u
        return iv

    Kl, Kh = 1.0, 2.0 * count(2 * a - b, 2 * b - a) + 16
    for _ in range(50):
        Km = 0.5 * (Kl + Kh)
        if len(greedy(Km, n_s)) <= n_s:
            Kh = Km
        else:
            Kl = Km
    iv = greedy(Kh, n_s)
    while len(iv) < n_s:
        c = [count(l, u) for l, u in iv]
        i = int(np.argmax(c))
        l, u = iv[i]
        iv[i:i + 1] = [(l, 0.5 * (l + u)), (0.5 * (l + u), u)]
    shifts = [0.5 * (l + u) for l, u in iv]
    balls = [count(s_ - ratio * 0.5 * (u - l), s_ + ratio * 0.5 * (u - l)) for s_, (l, u) in zip(shifts, iv)]
    return iv, shifts, balls


def default_basis_width(n_e: int, n_s: int) -> int:
    """k = 2 ceil(n_e / n_s) + 16 rounded up to a multiple of 16."""
    k = 2 * (-(-n_e // n_s)) + 16
    return -(-k // 16) * 16


def _ceil16(x: float) -> int:
    return int(-(-x // 16) * 16)


def _inside_region(groups, lam_min: float, lam_max: float):
    """Probes whose migrated shift left the new region [lambda_min, lambda_max] hand their
    members to the nearest probe inside it (a region bound moves with the pencil)."""
    inside = [g for g in groups if lam_min < g[0] < lam_max]
    if not inside:
        return [(0.5 * (lam_min + lam_max), sorted(i for _, m in groups for i in m))]
    out = [(s_, list(m)) for s_, m in inside]
    for s_, m in groups:
        if lam_min < s_ < lam_max:
            continue
        q = min(range(len(out)), key=lambda t: abs(out[t][0] - s_))
        out[q] = (out[q][0], sorted(out[q][1] + list(m)))
    return out


def migrated_windows(values, groups, lam_min: float, lam_max: float):
    """Slice boundaries and basis widths for migrated probes (groups from
    migrate_probes, sorted by shift), using the previous step's eigenvalues as the
    spectrum estimate.  The boundary between two probes lies midway between the last
    member of the lower probe and the first of the upper one (the midpoint of the shifts
    if the member sets interleave); each basis covers the eigenvalues within the probe's
    ball -- the largest distance from its shift to its window ends -- as in ball_partition.
    Above lambda_max the count is extrapolated from the same distance below it."""
    x = np.sort(np.asarray(values, dtype=np.float64))
    sh = [s_ for s_, _ in groups]
    ns = len(groups)
    splits = [None]
    for j in range(1, ns):
        lo_m = float(np.max(np.asarray(values)[groups[j - 1][1]]))
        hi_m = float(np.min(np.asarray(values)[groups[j][1]]))
        t = 0.5 * (lo_m + hi_m)
        splits.append(t if sh[j - 1] < t < sh[j] and lo_m < hi_m else 0.5 * (sh[j - 1] + sh[j]))
    ks = []
    for j in range(ns):
        lo = lam_min if j == 0 else splits[j]
        hi = lam_max if j == ns - 1 else splits[j + 1]
        r = max(sh[j] - lo, hi - sh[j])
        a, b = sh[j] - r, sh[j] + r
        c = int(np.count_nonzero((x >= a) & (x <= b)))
        if b > lam_max:
            c += int(np.count_nonzero((x >= 2 * lam_max - b) & (x <= lam_max)))
        # the ball can reach far into the spectrum for a centroid shift of a wide cluster;
        # the basis stays within 4x its members + 16 (validation widens it if needed)
        ks.append(min(_ceil16(1.15 * c + 16), _ceil16(4 * (len(groups[j][1]) + 16)), 4096))
    return splits, ks


class SpectrumCount:
    """The count function Phi(w) = #{previous eigenvalues < w} of a validated spectrum, in
    the interface of DosModel (Phi returns an array), for placing the probes of the next
    pencil.  Above the last value the count is continued with the mean spacing of the top
    tenth of the spectrum."""

    def __init__(self, values):
        self.x = np.sort(np.asarray(values, dtype=np.float64))
        top = self.x[-max(2, self.x.size // 10):]
        self.spacing = max(float(np.mean(np.diff(top))), 1e-12) if top.size > 1 else 1.0

    def Phi(self, w):
        w = np.atleast_1d(np.asarray(w, dtype=np.float64))
        c = np.searchsorted(self.x, w, side="left").astype(np.float64)
        above = w > self.x[-1]
        c[above] = self.x.size + (w[above] - self.x[-1]) / self.spacing
        return c


def ball_windows_from_spectrum(values, lam_min: float, lam_max: float, n_s: int):
    """Ball placement (ball_partition) on the previous pencil's validated eigenvalues:
    (shifts, splits, basis widths), the widths as in place_shifts."""
    model = SpectrumCount(values)
    iv, shifts, balls = ball_partition(model, lam_min, lam_max, n_s)
    splits = [None] + [iv[j][0] for j in range(1, n_s)]
    ks = [min(4096, _ceil16(1.15 * bc + 16)) for bc in balls]
    return shifts, splits, ks


def solve_sequence(sym: api.Symbolic, a_list, b_vals, n_e: int, n_s: int, precision: str = "mixed",
                   tol: float = 1e-10, lanczos_steps: int = 100, n_vec: int = 4, seed: int = 0,
                   start=None, uniforms=None, eta_tol: float = np.inf, balance: float = 2.0,
                   on_step=None):
    """Lowest n_e eigenpairs of a sequence of pencils (A_i, B) on one pattern, as the SCF
    loop of Alg. 1 produces them (Section 3.2).  Step 0 places the shifts from a Lanczos
    DOS estimate.  Every later step migrates the probes: k-means of the previous step's
    validated eigenvalues (k-means++ seeds after the DOS placement, the previous shifts
    afterwards), then migrate_probes; each probe starts from the Ritz vectors of its
    cluster, padded with random columns to the basis width of migrated_windows.  The region keeps
    nu(lambda_max) = n_e at every step (bisection on inertia from the previous bound).
    start: N x n_vec device block of DOS start vectors (seeded N(0,1) if None);
    uniforms: the n_s k-means++ uniforms (seeded if None).  Every step recovers missing
    eigenvalues by probe insertion (Section 3.3).  eta_tol: relative change of
    Tr(X^T A X) over the previous eigenvectors (Eq. 9) above which a step is placed from a
    new DOS estimate instead of by migration (inf: never).  balance: a migrated probe with
    more than balance x the mean number of eigenvalues gets an inserted neighbour (None:
    only deleted probes are replaced).  When the migrated windows would need more than
    twice the total basis of a ball placement on the previous step's eigenvalues (k-means
    on a tail-heavy spectrum leaves wide clusters in the dense part), the step is placed by
    that ball placement instead, each probe warm-started from the previous eigenvectors
    in its window.  Returns one SliceResult per
    pencil; timings["migration"] records the shifts and cluster sizes chosen and
    timings["eta"] the monitor's (old, new, changed).  on_step(i, result), if given, is
    called as soon as pencil i is solved."""
    n = sym.n
    rng = np.random.default_rng(seed)
    etas = []
    if uniforms is None:
        uniforms = rng.random(n_s)
    g = torch.Generator(device="cuda").manual_seed(seed)
    results = []
    for i, a_vals in enumerate(a_list):
        solver = SliceSolver(sym, a_vals, b_vals, precision=precision, tol=tol)
        redo_dos = i == 0
        if i > 0:
            # eta monitor (Eq. 9): Tr(X^T A X) over the previous eigenvectors under the old
            # and the new A; a relative change above eta_tol sends this step back to a DOS
            # placement instead of migration
            prev = results[-1]
            eta_old = float(np.sum(prev.eigenvalues))
            eta_new = trace_form(sym, a_vals, prev.eigenvectors)
            changed = abs(eta_new - eta_old) > eta_tol * max(1.0, abs(eta_old))
            etas.append((eta_old, eta_new, changed))
            redo_dos = changed
        if redo_dos:
            st = start if start is not None else torch.randn(n, n_vec, generator=g, device="cuda",
                                                             dtype=torch.float64)
            model = DosModel(n, sym.dos_estimate(a_vals, b_vals, lanczos_steps, st))
            lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, n_e, n_s)
            lam_max = solver.bound_at_count(lam_max, n_e, lam_min, lam_max - lam_min)
            res = solver.run_with_recovery(shifts, lam_min, lam_max, model, splits=splits, ks=ks, seed=seed)
            res.timings["migration"] = None
        else:
            prev = results[-1]
            after_dos = prev.timings["migration"] is None
            init = kmeans_pp_seeds(prev.eigenvalues, n_s, uniforms) if after_dos else np.asarray(prev.shifts)
            migrated = migrate_probes(prev.eigenvalues, prev.owners, prev.shifts, init, balance=balance)
            span = float(prev.lam_max - prev.lam_min)
            lam_min = prev.lam_min
            while solver.count_below([lam_min])[0] > 0:
                lam_min -= 0.1 * span
            lam_max = solver.bound_at_count(prev.lam_max, n_e, lam_min, span)
            groups = _inside_region(migrated, lam_min, lam_max)
            shifts = [s_ for s_, _ in groups]
            splits, ks = migrated_windows(prev.eigenvalues, groups, lam_min, lam_max)
            b_shifts, b_splits, b_ks = ball_windows_from_spectrum(prev.eigenvalues, lam_min, lam_max, n_s)
            fallback = sum(ks) > 2 * sum(b_ks)
            if fallback:
                shifts, splits, ks = b_shifts, b_splits, b_ks
                bounds = [lam_min] + [splits[j] for j in range(1, len(shifts))] + [lam_max]
                ev = np.asarray(prev.eigenvalues)
                groups = [(shifts[j], [int(i) for i in np.flatnonzero((ev > bounds[j]) & (ev <= bounds[j + 1]))])
                          for j in range(len(shifts))]
            V0 = []
            for (_, m), kk in zip(groups, ks):
                kk = min(n, max(kk, len(m) + 16))
                fill = torch.randn(n, kk - len(m), generator=g, device="cuda", dtype=torch.float64)
                V0.append(torch.cat([prev.eigenvectors[:, m], fill], dim=1).contiguous())
            res = solver.run_with_recovery(shifts, lam_min, lam_max, None, V0=V0, ks=ks, splits=splits,
                                           seed=seed + i, warm=True)
            res.timings["migration"] = dict(shifts=[s_ for s_, _ in migrated], sizes=[len(m) for _, m in migrated],
                                            init="kmeans++" if after_dos else "previous shifts",
                                            shifts_used=shifts, balance=balance,
                                            ball_fallback=bool(fallback))
        res.timings["eta"] = etas[-1] if i > 0 else None
        results.append(res)
        if on_step is not None:
            on_step(i, res)
    return results


def trace_form(sym: api.Symbolic, a_vals, X) -> float:
    """eta(X, A) = Tr(X^T A X) (Eq. 9), A X by the library's SpMM."""
    AX = sym.spmm(a_vals, None, X)
    return float((X * AX).sum().item())
