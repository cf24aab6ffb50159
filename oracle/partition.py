"""Slice partition, validation and shift migration (Sections 2.2, 3.1, 3.2).

Test infrastructure only.  Readings where the paper is silent or garbled:
* CDOS roots (Eq. 6) are read as Phi(omega) = Phi(a) + K j, j = 0..n_s,
  K = (Phi(b) - Phi(a)) / n_s, found by bisection to 1e-12 relative width.
* The interval midpoint is (l + u)/2.
* End slices are [lambda_min, sigma_1) and (sigma_ns, lambda_max].
* A candidate exactly at tau goes to the lower probe; residual ties are broken by
  (residual, probe index, Ritz index).
* k-means++ draws its uniforms from an input array (one per centroid) so that both
  sides see the same random numbers.
* DOSCluster (Alg. 3, Section 3.1): a grid point is a local maximiser of phi if it is
  larger than its left neighbour and not smaller than its right one; an end point must
  be larger than its single neighbour (a flat tail is no maximum); no maximiser counts
  as one.  Between two maximisers
  the minimiser is taken over the grid points strictly between them (the midpoint of
  the two if there are none).  The refinement merges an interval with
  gamma < merge_tol into the adjacent interval (sharing an end) with the fewer
  estimated eigenvalues and reruns Alg. 3 on intervals with gamma > refine_tol at
  n_omega' = ceil(2 C(l,u) / C(a,b) n_omega) points, at most `max_rounds` times.  The
  safeguards split the interval with the most estimated eigenvalues at its CDOS median
  and merge the interval with the fewest into its adjacent neighbour with fewer
  (skipping intervals with no adjacent one).  Gaps left by removed intervals are
  closed at their midpoints so that the intervals tile [a, b].
* Probe update after clustering (Section 3.2): a cluster maps to the probe that
  produced most of its values (ties: the probe whose old shift is nearest the cluster
  centroid, then the lower index).  The 2-means split of the largest cluster starts
  from its smallest and largest values; the old probe keeps the part holding more of
  its own values (ties: the part whose centroid is nearer its old shift), the inserted
  probe takes the other.  An empty k-means cluster maps to no probe.  If the largest
  cluster has a single distinct value it cannot be split and fewer probes result.
"""
from __future__ import annotations

import numpy as np

from .dos import cdos_Phi, dos_phi, expectation_shift


def bisect_root(f, lo, hi, target, rel=1e-12, maxit=200):
    """Smallest-bracket root of f(x) = target for nondecreasing f on [lo, hi]."""
    flo = f(lo) - target
    for _ in range(maxit):
        mid = 0.5 * (lo + hi)
        if hi - lo <= rel * max(1.0, abs(mid)):
            break
        if f(mid) - target < 0.0:
            lo = mid
        else:
            hi = mid
    del flo
    return 0.5 * (lo + hi)


def cdos_root_intervals(a, b, n_s, n, runs):
    """Intervals (l_j, u_j) with about equal CDOS mass (Eq. 6)."""
    Pa = float(cdos_Phi(a, n, runs)[0])
    Pb = float(cdos_Phi(b, n, runs)[0])
    K = (Pb - Pa) / n_s
    f = lambda w: float(cdos_Phi(w, n, runs)[0])
    roots = [a]
    for j in range(1, n_s):
        roots.append(bisect_root(f, a, b, Pa + K * j))
    roots.append(b)
    return [(roots[j], roots[j + 1]) for j in range(n_s)]


def candidates(shifts, lam_min, lam_max, probes):
    """Validation candidates per slice (Section 2.2).

    probes[j] = (theta[k], resid[k]) of the probe at shifts[j].  Returns a list over the
    n_s + 1 slices of lists of (probe j, ritz index i)."""
    ns = len(shifts)
    out = []
    for s in range(ns + 1):
        cand = []
        lo = lam_min if s == 0 else shifts[s - 1]
        hi = lam_max if s == ns else shifts[s]
        if s == 0:
            th = probes[0][0]
            cand += [(0, i) for i in range(len(th)) if lam_min <= th[i] < shifts[0]]
        elif s == ns:
            th = probes[ns - 1][0]
            cand += [(ns - 1, i) for i in range(len(th)) if shifts[-1] < th[i] <= lam_max]
        else:
            tau = 0.5 * (lo + hi)
            th = probes[s - 1][0]
            cand += [(s - 1, i) for i in range(len(th)) if lo < th[i] <= tau]
            th = probes[s][0]
            cand += [(s, i) for i in range(len(th)) if tau < th[i] < hi]
        out.append(cand)
    return out


def validate(shifts, lam_min, lam_max, probes, nneg_shift, nneg_min, nneg_max):
    """Apply the three validation cases per slice (Section 2.2).

    nneg_shift[j] = #negative pivots of LDL^T(A - shifts[j] B); nneg_min / nneg_max
    are the counts at the region bounds.  Returns (validated list of (probe, ritz),
    per-slice (n_exact, n_cand, status)) with status 'ok' / 'missing' / 'excess'."""
    ns = len(shifts)
    cands = candidates(shifts, lam_min, lam_max, probes)
    bounds = [nneg_min] + list(nneg_shift) + [nneg_max]
    validated, info = [], []
    for s in range(ns + 1):
        n_exact = bounds[s + 1] - bounds[s]
        c = cands[s]
        if n_exact == len(c):
            validated += c
            info.append((n_exact, len(c), "ok"))
        elif n_exact > len(c):
            validated += c
            info.append((n_exact, len(c), "missing"))
        else:
            key = sorted(c, key=lambda pi: (probes[pi[0]][1][pi[1]], pi[0], pi[1]))
            validated += key[:n_exact]
            info.append((n_exact, len(c), "excess"))
    return validated, info


def kmeans_pp_init(x, n_c, uniforms):
    """k-means++ seeding on 1-D data (Section 3.2): the first centroid uniformly, the
    rest with probability proportional to D(x)^2, D = distance to nearest centroid."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    cent = [x[min(n - 1, int(uniforms[0] * n))]]
    for c in range(1, n_c):
        d2 = np.min((x[:, None] - np.asarray(cent)[None, :]) ** 2, axis=1)
        tot = d2.sum()
        if tot <= 0.0:
            cent.append(x[min(n - 1, int(uniforms[c] * n))])
            continue
        cdf = np.cumsum(d2) / tot
        idx = int(np.searchsorted(cdf, uniforms[c], side="right"))
        cent.append(x[min(n - 1, idx)])
    return np.asarray(cent)


def lloyd(x, cent, maxit=1000):
    """Lloyd iterations until the assignment stops changing; returns sorted centroids."""
    x = np.asarray(x, dtype=np.float64)
    cent = np.asarray(cent, dtype=np.float64).copy()
    assign = None
    for _ in range(maxit):
        a = np.argmin(np.abs(x[:, None] - cent[None, :]), axis=1)
        if assign is not None and np.array_equal(a, assign):
            break
        assign = a
        for c in range(cent.size):
            m = a == c
            if m.any():
                cent[c] = x[m].mean()
    return np.sort(cent)


def kmeans_shifts(ritz_values, n_s, uniforms):
    """New shifts = k-means centroids of the validated Ritz values (Section 3.2)."""
    return lloyd(ritz_values, kmeans_pp_init(ritz_values, n_s, uniforms))


def _assign(x, cent):
    """Index of the nearest centroid of each value (the lower index on a tie)."""
    return np.argmin(np.abs(np.asarray(x)[:, None] - np.asarray(cent)[None, :]), axis=1)


def lloyd_assign(x, cent, maxit=1000):
    """Lloyd iterations from the given centroids, keeping their order; an empty
    cluster keeps its centroid.  Returns (centroids, assignment)."""
    x = np.asarray(x, dtype=np.float64)
    cent = np.asarray(cent, dtype=np.float64).copy()
    a = _assign(x, cent)
    for _ in range(maxit):
        for c in range(cent.size):
            if (a == c).any():
                cent[c] = x[a == c].mean()
        a2 = _assign(x, cent)
        if np.array_equal(a2, a):
            break
        a = a2
    return cent, a


def migrate(values, owner, old_shifts, init_centroids, balance=None):
    """Shift migration between two SCF steps (Section 3.2).

    values: validated eigenvalues of the previous step; owner[i]: the probe that
    produced values[i]; old_shifts: that step's shifts (one per probe);
    init_centroids: the k-means start (k-means++ after a DOS placement, else the old
    shifts).  Steps, in the paper's order: k-means into n_s clusters; each cluster to
    the probe with maximal overlap; clusters on one probe merged (shift = centroid of
    the merged values); probes with no cluster deleted; for each deletion the largest
    cluster split by 2-means, one part kept by its probe and the other given to an
    inserted probe.  Returns a list of (shift, member indices into values), sorted by
    shift; an inserted probe's start vectors are the Ritz vectors of its members.
    balance: if given, a probe holding more than balance * len(values) / n_s values is
    split the same way (the paper's probe insertion for load balance), up to 2 n_s
    probes."""
    x = np.asarray(values, dtype=np.float64)
    owner = np.asarray(owner)
    old = np.asarray(old_shifts, dtype=np.float64)
    n_s = old.size
    cent, a = lloyd_assign(x, init_centroids)
    members = {p: [] for p in range(n_s)}
    for c in range(cent.size):
        idx = np.nonzero(a == c)[0]
        if idx.size == 0:
            continue
        overlap = np.array([(owner[idx] == p).sum() for p in range(n_s)])
        best = np.nonzero(overlap == overlap.max())[0]
        mu = x[idx].mean()
        p = min(best, key=lambda q: (abs(old[q] - mu), q))
        members[p].extend(idx.tolist())
    probes = []          # (old probe index or -1 for an inserted one, member indices)
    for p in range(n_s):
        if members[p]:
            probes.append([p, sorted(members[p])])
    deleted = n_s - len(probes)
    limit = float(balance) * x.size / n_s if balance else np.inf
    splits_done = 0
    while splits_done < deleted or (len(probes) < 2 * n_s and max(len(m) for _, m in probes) > limit):
        splits_done += 1
        big = max(range(len(probes)), key=lambda q: (len(probes[q][1]), -q))
        p, idx = probes[big]
        idx = np.array(idx)
        v = x[idx]
        if v.min() == v.max():
            break
        _, a2 = lloyd_assign(v, [v.min(), v.max()])
        parts = [idx[a2 == 0], idx[a2 == 1]]
        home = p if p >= 0 else None
        def keep_key(part):
            own = int((owner[part] == home).sum()) if home is not None else 0
            ref = old[home] if home is not None else x[idx].mean()
            return (-own, abs(x[part].mean() - ref))
        order = sorted(range(2), key=lambda t: keep_key(parts[t]))
        probes[big] = [p, sorted(parts[order[0]].tolist())]
        probes.append([-1, sorted(parts[order[1]].tolist())])
    out = [(float(x[np.array(m)].mean()), m) for _, m in probes]
    out.sort(key=lambda t: t[0])
    return out


def dos_cluster(n, runs, a, b, n_omega):
    """Alg. 3: intervals of [a, b] around the local maxima of phi on n_omega grid points,
    split at the minima between them; intervals without a Ritz value are dropped."""
    S = a + (b - a) / (n_omega - 1) * np.arange(n_omega)
    ph = dos_phi(S, n, runs)
    maxi = []
    for i in range(n_omega):
        if i == 0:
            is_max = ph[0] > ph[1]
        else:
            is_max = ph[i] > ph[i - 1] and (i == n_omega - 1 or ph[i] >= ph[i + 1])
        if is_max:
            maxi.append(i)
    if len(maxi) <= 1:
        return [(a, b)]
    mu = [a]
    for j in range(len(maxi) - 1):
        lo_i, hi_i = maxi[j], maxi[j + 1]
        if hi_i - lo_i >= 2:
            inner = np.arange(lo_i + 1, hi_i)
            mu.append(float(S[inner[np.argmin(ph[inner])]]))
        else:
            mu.append(0.5 * float(S[lo_i] + S[hi_i]))
    mu.append(b)
    theta = np.concatenate([th for th, _, _ in runs])
    out = []
    for j in range(len(mu) - 1):
        l, u = mu[j], mu[j + 1]
        if np.any((theta > l) & (theta <= u)) or (j == 0 and np.any(theta == l)):
            out.append((l, u))
    return out if out else [(a, b)]


def _gamma(n, runs, l, u):
    return float(cdos_Phi(u, n, runs)[0] - cdos_Phi(l, n, runs)[0])


def _merge_small(n, runs, I, merge_tol):
    """Refinement step 2: merge intervals holding fewer than merge_tol eigenvalues into
    the adjacent interval with fewer eigenvalues (intervals without one stay)."""
    changed = True
    while changed:
        changed = False
        for j, (l, u) in enumerate(I):
            if _gamma(n, runs, l, u) >= merge_tol:
                continue
            nb = []
            if j > 0 and I[j - 1][1] == l:
                nb.append(j - 1)
            if j + 1 < len(I) and I[j + 1][0] == u:
                nb.append(j + 1)
            if not nb:
                continue
            t = min(nb, key=lambda q: (_gamma(n, runs, *I[q]), q))
            lo, hi = min(I[t][0], l), max(I[t][1], u)
            I = [iv for q, iv in enumerate(I) if q not in (j, t)]
            I.append((lo, hi))
            I.sort()
            changed = True
            break
    return I


def dos_cluster_partition(n, runs, a, b, n_s, n_omega, merge_tol=2.0, refine_tol=50.0, max_rounds=20):
    """Cluster intervals of Alg. 3 with the refinement strategy and the safeguards that
    give exactly n_s intervals (Section 3.1); returns (intervals, expectation shifts)."""
    C_ab = _gamma(n, runs, a, b)
    I = dos_cluster(n, runs, a, b, n_omega)
    done = set()
    for _ in range(max_rounds):
        I = _merge_small(n, runs, I, merge_tol)
        new = []
        grew = False
        for (l, u) in I:
            g = _gamma(n, runs, l, u)
            if g > refine_tol and (l, u) not in done:
                done.add((l, u))
                m = max(3, int(np.ceil(2.0 * g / C_ab * n_omega)))
                sub = dos_cluster(n, runs, l, u, m)
                if len(sub) >= 2:
                    new.extend(sub)
                    grew = True
                    continue
            new.append((l, u))
        I = sorted(new)
        if not grew:
            break
    # close the gaps left by dropped intervals at their midpoints
    tiled = []
    for j, (l, u) in enumerate(I):
        lo = a if j == 0 else 0.5 * (I[j - 1][1] + l)
        hi = b if j == len(I) - 1 else 0.5 * (u + I[j + 1][0])
        tiled.append((lo, hi))
    I = tiled
    while len(I) < n_s:
        j = max(range(len(I)), key=lambda q: (_gamma(n, runs, *I[q]), -q))
        l, u = I[j]
        target = 0.5 * (float(cdos_Phi(l, n, runs)[0]) + float(cdos_Phi(u, n, runs)[0]))
        m = bisect_root(lambda w: float(cdos_Phi(w, n, runs)[0]), l, u, target)
        I[j:j + 1] = [(l, m), (m, u)]
    while len(I) > n_s:
        order = sorted(range(len(I)), key=lambda q: (_gamma(n, runs, *I[q]), q))
        j = order[0]
        nb = [q for q in (j - 1, j + 1) if 0 <= q < len(I)]
        t = min(nb, key=lambda q: (_gamma(n, runs, *I[q]), q))
        lo, hi = min(I[t][0], I[j][0]), max(I[t][1], I[j][1])
        I = [iv for q, iv in enumerate(I) if q not in (j, t)] + [(lo, hi)]
        I.sort()
    shifts = [expectation_shift(l, u, n, runs) for l, u in I]
    return I, shifts
