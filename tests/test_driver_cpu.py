"""CPU tests of the host-side slicing logic (Sections 2.3, 3.1, 3.2) against the oracle's
independent implementation and against invariants."""
import numpy as np
import pytest

from oracle import dos as odos
from oracle import partition as opart
from paper_1908_06043_gb300.driver import DosModel, ball_partition, cdos_partition, kmeans_shifts, validate


def _runs(seed, m=120, nv=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nv):
        th = np.sort(np.concatenate([rng.uniform(-30, -5, 8), rng.uniform(-5, 4, m - 8)]))
        z = rng.random(m)
        out.append((th, z / z.sum()))
    return out


def test_dos_model_matches_oracle_formulas():
    runs = _runs(1)
    model = DosModel(5000, runs)
    oruns = [(th, z2, odos.gaussian_widths(th)) for th, z2 in runs]
    w = np.linspace(-35, 6, 57)
    assert np.allclose(model.Phi(w), odos.cdos_Phi(w, 5000, oruns), rtol=1e-13, atol=1e-9)
    assert np.allclose(model.phi(w), odos.dos_phi(w, 5000, oruns), rtol=1e-13, atol=1e-9)
    assert model.expectation(-2.0, 1.0) == pytest.approx(odos.expectation_shift(-2.0, 1.0, 5000, oruns), rel=1e-12)


def test_cdos_partition_matches_oracle():
    runs = _runs(2)
    model = DosModel(5000, runs)
    oruns = [(th, z2, odos.gaussian_widths(th)) for th, z2 in runs]
    iv, shifts = cdos_partition(model, -10.0, 3.0, 7)
    oiv = opart.cdos_root_intervals(-10.0, 3.0, 7, 5000, oruns)
    assert np.allclose(np.array(iv), np.array(oiv), atol=1e-9)


def test_ball_partition_invariants():
    runs = _runs(3)
    model = DosModel(20000, runs)
    a, b, ns = -32.0, 3.0, 12
    iv, shifts, balls = ball_partition(model, a, b, ns)
    assert len(iv) == ns and iv[0][0] == a and iv[-1][1] == b
    assert all(iv[i][1] == iv[i + 1][0] for i in range(ns - 1))
    assert all(l < s < u for (l, u), s in zip(iv, shifts))
    # every ball stays within the largest budget used
    K = max(balls)
    for (l, u), s in zip(iv, shifts):
        h = 0.5 * (u - l)
        assert model.Phi(s + 2 * h)[0] - model.Phi(s - 2 * h)[0] <= K + 1e-6
    # the sparse tail gets a wider, emptier interval than the dense body
    counts = [model.Phi(u)[0] - model.Phi(l)[0] for l, u in iv]
    assert counts[0] < np.median(counts)


def test_validate_matches_oracle_with_midpoints():
    rng = np.random.default_rng(4)
    shifts = [0.0, 1.0, 2.0]
    probes = [(np.sort(rng.uniform(-1, 3, 30)), rng.choice([1e-12, 1e-3], 30)) for _ in shifts]
    nneg = [5, 12, 20]
    sel, info = validate(shifts, -1.0, 3.0, probes, nneg, 0, 27, 1e-10)
    osel, oinfo = opart.validate(shifts, -1.0, 3.0, probes, nneg, 0, 27)
    assert sorted(map(tuple, sel)) == sorted(map(tuple, osel))
    assert [i[3] for i in info] == [i[2] for i in oinfo]


def test_validate_custom_split_point():
    shifts = [0.0, 1.0]
    probes = [(np.array([0.2, 0.7]), np.array([1e-12, 1e-12])), (np.array([0.7, 0.9]), np.array([1e-12, 1e-12]))]
    # split at 0.8 instead of the midpoint: 0.7 belongs to the lower probe
    sel, info = validate(shifts, -1.0, 2.0, probes, [0, 3], 0, 3, 1e-10, taus=[None, 0.8, None])
    assert info[1][:3] == (3, 3, 3)
    assert (0, 1) in sel and (1, 0) not in sel


def test_kmeans_matches_oracle():
    rng = np.random.default_rng(5)
    x = np.sort(np.concatenate([rng.normal(0, 0.1, 50), rng.normal(3, 0.2, 80), rng.normal(7, 0.1, 40)]))
    u = rng.random(3)
    assert np.allclose(kmeans_shifts(x, 3, u), opart.kmeans_shifts(x, 3, u), atol=1e-14)


def test_migrate_probes_matches_oracle():
    from oracle import partition
    from paper_1908_06043_gb300.driver import kmeans_pp_seeds, migrate_probes
    rng = np.random.default_rng(11)
    for trial in range(40):
        n_s = int(rng.integers(2, 9))
        v = np.sort(np.concatenate([rng.normal(c, 0.2, int(rng.integers(1, 30)))
                                    for c in rng.uniform(-5, 5, int(rng.integers(2, 8)))]))
        old = np.sort(rng.uniform(v.min() - 2, v.max() + 2, n_s))
        owner = np.searchsorted(0.5 * (old[1:] + old[:-1]), v)
        u = rng.random(n_s)
        seeds = kmeans_pp_seeds(v, n_s, u)
        assert np.array_equal(seeds, partition.kmeans_pp_init(v, n_s, u))
        for init, bal in ((old, None), (seeds, None), (old, 1.5), (seeds, 2.0)):
            got = migrate_probes(v, owner, old, init, balance=bal)
            ref = partition.migrate(v, owner, old, init, balance=bal)
            assert len(got) == len(ref)
            for (s1, m1), (s2, m2) in zip(got, ref):
                assert m1 == m2 and abs(s1 - s2) <= 1e-12 * max(1.0, abs(s2))


def test_dos_cluster_partition_matches_oracle():
    from oracle import partition
    from oracle.dos import gaussian_widths
    from paper_1908_06043_gb300.driver import DosModel, dos_cluster_partition, dos_clusters
    rng = np.random.default_rng(12)
    for trial in range(12):
        centres = np.sort(rng.uniform(-10, 10, int(rng.integers(1, 6))))
        theta = np.sort(np.concatenate([c + rng.uniform(0.02, 0.5) * rng.standard_normal(int(rng.integers(3, 25)))
                                        for c in centres]))
        z2 = rng.random(theta.size)
        z2 /= z2.sum()
        n = int(rng.integers(200, 5000))
        model = DosModel(n, [(theta, z2)])
        runs = [(theta, z2, gaussian_widths(theta))]
        a, b = theta[0] - 1.0, theta[-1] + 1.0
        n_om = 10 * theta.size
        assert dos_clusters(model, a, b, n_om) == partition.dos_cluster(n, runs, a, b, n_om)
        for n_s in (1, 3, 8):
            I1, s1 = dos_cluster_partition(model, a, b, n_s, n_om)
            I2, s2 = partition.dos_cluster_partition(n, runs, a, b, n_s, n_om)
            assert len(I1) == len(I2) == n_s
            assert np.allclose(np.array(I1), np.array(I2), rtol=1e-9, atol=1e-9)
            assert np.allclose(s1, s2, rtol=1e-9, atol=1e-9)


def test_migrated_windows_and_region_filter():
    from paper_1908_06043_gb300.driver import _inside_region, migrate_probes, migrated_windows
    rng = np.random.default_rng(21)
    v = np.sort(np.concatenate([rng.uniform(-40, -10, 12), rng.uniform(-2, 0.3, 150)]))
    old = np.array([-30.0, -1.5, -0.9, -0.3, 0.1])
    owner = np.searchsorted(0.5 * (old[1:] + old[:-1]), v)
    groups = migrate_probes(v, owner, old, old)
    lam_min, lam_max = -45.0, 0.31
    splits, ks = migrated_windows(v, groups, lam_min, lam_max)
    sh = [s_ for s_, _ in groups]
    assert splits[0] is None and len(splits) == len(sh) == len(ks)
    for j in range(1, len(sh)):
        assert sh[j - 1] < splits[j] < sh[j]
    for (_, m), k in zip(groups, ks):
        assert k % 16 == 0 and 16 <= k <= min(4096, 4 * (len(m) + 16) + 15)
    # a region bound that moved below the top shift: its members go to the nearest probe
    cut = 0.5 * (sh[-2] + sh[-1])
    kept = _inside_region(groups, lam_min, cut)
    assert len(kept) == len(groups) - 1
    assert sorted(i for _, m in kept for i in m) == list(range(v.size))
    assert all(lam_min < s_ < cut for s_, _ in kept)


def test_recovery_inserts_probes_in_deficient_slices():
    # host logic of Section 3.3 with the probes mocked: slice 1 reports a missing
    # eigenvalue, so the next run gets a probe inside (sigma_0, sigma_1) and the old probes
    # restart from their vectors
    from types import SimpleNamespace
    from paper_1908_06043_gb300.driver import SliceSolver
    calls = []

    class Fake(SliceSolver):
        def __init__(self):
            pass

        def run(self, shifts, lam_min, lam_max, model=None, **kw):
            calls.append((list(shifts), kw.get("V0")))
            ok = len(calls) > 1
            ns = len(shifts)
            slices = [(10, 10, 10 if ok or s_ != 1 else 9, "ok") for s_ in range(ns + 1)]
            probes = [SimpleNamespace(X="X%d" % j) for j in range(ns)]
            return SimpleNamespace(timings={"converged": ok}, slices=slices, probes=probes, shifts=list(shifts))

    res = Fake().run_with_recovery([0.0, 1.0, 2.0], -1.0, 3.0, None)
    assert res.timings["converged"] and res.timings["inserted"] == [[0.5]]
    assert calls[1][0] == [0.0, 0.5, 1.0, 2.0]
    assert calls[1][1] == ["X0", None, "X1", "X2"]


def test_ball_windows_from_previous_spectrum():
    """Migration fallback: the ball placement on a validated spectrum gives n_s shifts
    inside [lambda_min, lambda_max], increasing splits strictly between neighbouring
    shifts, and on a uniform spectrum equal interior windows (the end windows' balls reach
    past the spectrum, where it counts fewer eigenvalues, so those windows may differ)."""
    from paper_1908_06043_gb300.driver import SpectrumCount, ball_windows_from_spectrum
    v = np.linspace(0.0, 1.0, 401)
    sh, sp, ks = ball_windows_from_spectrum(v, -0.00125, 1.00125, 8)
    assert len(sh) == 8 and len(sp) == 8 and sp[0] is None
    w = np.diff([-0.00125] + sp[1:] + [1.00125])
    assert np.allclose(w[1:-1], w[1:-1].mean(), rtol=0.05)
    assert all(sh[j - 1] < sp[j] < sh[j] for j in range(1, 8))
    # the count function: exact below the last value, linear continuation above it
    m = SpectrumCount(v)
    assert m.Phi(0.5)[0] == 200 and m.Phi(-1.0)[0] == 0
    assert abs(m.Phi(1.0 + 10 * 0.0025)[0] - 411) < 1e-9
    # a tail-heavy spectrum: the sparse tail gets the wide windows, the body narrow ones
    t = np.concatenate([np.linspace(-45, -10, 37), np.linspace(-8, 0.3, 1600)])
    sh, sp, ks = ball_windows_from_spectrum(t, -46.0, 0.31, 16)
    b = [-46.0] + sp[1:] + [0.31]
    counts = [int(np.sum((t > b[j]) & (t <= b[j + 1]))) for j in range(16)]
    assert sum(counts) == t.size
    assert max(ks) <= 4096 and min(counts[2:]) > 0


def test_plan_with_counts_sets_exact_windows_and_widths():
    # the window-bound counts of a batched factorisation go into a plan: exact counts per
    # window, and basis widths of at least 2c + 16 (multiple of 16), capped at N
    from paper_1908_06043_gb300.driver import SlicePlan, plan_with_counts
    plan = SlicePlan([0.0, 1.0, 2.0], [-1.0, 0.5, 1.5, 2.5], [None] * 4, [None, 64, None], -1.0, 2.5)
    out = plan_with_counts(plan, [0, 10, 70, 75], n=120)
    assert out.counts == [0, 10, 70, 75]
    assert [out.exact(j) for j in range(3)] == [10, 60, 5]
    assert out.ks == [48, 120, 32]                  # 2*10+16=36 -> 48; 2*60+16=136 -> capped at N; 2*5+16 -> 32
    assert out.shifts == plan.shifts and out.bounds == plan.bounds
