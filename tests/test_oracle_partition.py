"""Pins for validation (Section 2.2) and k-means shift migration (Section 3.2)."""
import numpy as np

from oracle import partition


def test_validation_three_cases():
    shifts = [0.0, 1.0]
    lam_min, lam_max = -1.0, 2.0
    probes = [
        (np.array([-0.5, 0.2, 0.5, 0.9]), np.array([1e-12, 1e-12, 1e-12, 1e-3])),
        (np.array([0.1, 0.6, 1.2, 1.9, 2.5]), np.array([1e-3, 1e-12, 1e-12, 1e-12, 1e-12])),
    ]
    # slice 0: [-1,0): probe0 -0.5 -> 1 cand; slice 1 (0,1): tau=.5: p0 {0.2,0.5}, p1 {0.6}
    # slice 2 (1,2]: p1 {1.2, 1.9}
    cands = partition.candidates(shifts, lam_min, lam_max, probes)
    assert cands[0] == [(0, 0)]
    assert cands[1] == [(0, 1), (0, 2), (1, 1)]     # 0.5 == tau goes to the lower probe
    assert cands[2] == [(1, 2), (1, 3)]
    # exact counts: slice0 1 (ok), slice1 2 (excess -> keep two smallest residuals),
    # slice2 3 (missing)
    val, info = partition.validate(shifts, lam_min, lam_max, probes, [1, 3], 0, 6)
    assert [s for _, _, s in info] == ["ok", "excess", "missing"]
    assert (0, 0) in val and (1, 2) in val and (1, 3) in val
    kept = [v for v in val if v in cands[1]]
    assert kept == [(0, 1), (0, 2)]


def test_kmeans_pp_first_centroid_and_determinism():
    x = np.concatenate([np.linspace(0, 1, 50), np.linspace(10, 11, 50), np.linspace(20, 21, 50)])
    u = np.array([0.4, 0.7, 0.1])
    c0 = partition.kmeans_pp_init(x, 3, u)
    assert c0[0] == x[int(0.4 * x.size)]
    a = partition.kmeans_shifts(x, 3, u)
    b = partition.kmeans_shifts(x, 3, u)
    assert np.array_equal(a, b)
    assert np.allclose(a, [0.5, 10.5, 20.5])


def test_lloyd_fixed_point():
    rng = np.random.default_rng(3)
    x = np.sort(rng.uniform(0, 10, 300))
    c = partition.kmeans_shifts(x, 6, rng.random(6))
    a = np.argmin(np.abs(x[:, None] - c[None, :]), axis=1)
    for j in range(c.size):
        assert abs(x[a == j].mean() - c[j]) < 1e-12
    # near-uniform data: clusters come out of roughly equal size (Section 3.2)
    sizes = np.bincount(a, minlength=6)
    assert sizes.min() > 0.5 * sizes.mean()


def _fixture(name):
    import os
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        rows[key] = np.array([float(v) for v in vals])
    return rows


def test_migration_worked_example_of_section_3_2():
    g = _fixture("migration_fig.txt")
    v = g["values"]
    owner = (v > g["boundary"][0]).astype(int)          # slice of sigma_1 ends at the boundary
    # k-means started from the old shifts separates the blue and red clusters
    cent, a = partition.lloyd_assign(v, g["old_shifts"])
    assert np.array_equal(np.sort(v[a == 0]), g["blue"]) and np.array_equal(np.sort(v[a == 1]), g["red"])
    # both clusters map to sigma_2's probe; merged they centre on the figure's marker
    assert v.mean() == g["marker"][0]
    out = partition.migrate(v, owner, g["old_shifts"], g["old_shifts"])
    assert [s for s, _ in out] == list(g["new_shifts"])
    assert sorted(v[out[0][1]]) == list(g["blue"]) and sorted(v[out[1][1]]) == list(g["red"])


def test_migration_bijective_map_moves_each_shift_to_its_cluster_mean():
    rng = np.random.default_rng(4)
    centres = np.array([-3.0, 0.0, 4.0, 9.0])
    groups = [c + 0.3 * rng.standard_normal(25) for c in centres]
    v = np.concatenate(groups)
    owner = np.repeat(np.arange(4), 25)
    old = centres + np.array([0.5, -0.4, 0.3, -0.6])
    out = partition.migrate(v, owner, old, old)
    assert len(out) == 4
    for (s, m), g, p in zip(out, groups, range(4)):
        assert np.all(owner[m] == p) and len(m) == 25
        assert abs(s - g.mean()) < 1e-12


def test_migration_deletes_empty_probe_and_splits_largest_cluster():
    # probe 2's shift sits far above every value: its cluster is empty, it is deleted
    # and a probe is inserted into the largest cluster
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.uniform(0, 1, 10), rng.uniform(5, 6, 30), rng.uniform(7, 8, 30)])
    owner = np.concatenate([np.zeros(10, int), np.ones(60, int)])
    old = np.array([0.5, 6.5, 50.0])
    out = partition.migrate(v, owner, old, old)
    assert len(out) == 3
    allm = sorted(i for _, m in out for i in m)
    assert allm == list(range(v.size))
    for s, m in out:
        assert abs(s - v[m].mean()) < 1e-12
    shifts = [s for s, _ in out]
    assert shifts[0] < 1 and 5 < shifts[1] < 6 and 7 < shifts[2] < 8


def test_migration_invariants_random():
    rng = np.random.default_rng(6)
    for trial in range(20):
        n_s = int(rng.integers(2, 7))
        v = np.sort(rng.gamma(2.0, 1.0, int(rng.integers(3 * n_s, 60))))
        old = np.sort(rng.uniform(v.min() - 1, v.max() + 1, n_s))
        tau = 0.5 * (old[1:] + old[:-1])
        owner = np.searchsorted(tau, v)
        out = partition.migrate(v, owner, old, partition.kmeans_pp_init(v, n_s, rng.random(n_s)))
        assert len(out) == n_s
        assert sorted(i for _, m in out for i in m) == list(range(v.size))
        for s, m in out:
            assert len(m) > 0 and abs(s - v[m].mean()) < 1e-12


def _runs(theta, weights):
    from oracle.dos import gaussian_widths
    theta = np.asarray(theta, dtype=np.float64)
    z2 = np.asarray(weights, dtype=np.float64)
    return [(theta, z2 / z2.sum(), gaussian_widths(theta))]


def test_dos_cluster_finds_separated_clusters():
    # three groups of Ritz values far apart: Alg. 3 returns one interval per group,
    # split at the DOS minima between them
    centres = [-10.0, 0.0, 10.0]
    theta = np.concatenate([c + 0.1 * np.arange(5) for c in centres])
    runs = _runs(theta, np.ones(theta.size))
    I = partition.dos_cluster(1500, runs, -12.0, 12.0, 10 * theta.size)
    assert len(I) == 3
    for (l, u), c in zip(I, centres):
        assert l < c and c + 0.4 < u
    assert I[0][1] < -2.0 and 2.0 < I[1][1] < 8.0


def test_dos_cluster_single_maximum_returns_whole_interval():
    theta = np.linspace(-1.0, 1.0, 9)
    w = np.exp(-theta ** 2)                     # one smooth bump
    runs = [(theta, w / w.sum(), np.full(theta.size, 1.0))]
    assert partition.dos_cluster(100, runs, -3.0, 3.0, 50) == [(-3.0, 3.0)]


def test_dos_cluster_drops_intervals_without_ritz_values():
    # two narrow peaks inside [a, b] and a third maximum created only by a Ritz value
    # outside [a, b]: the interval holding no Ritz value is removed
    theta = np.array([-5.0, -4.9, 5.0, 5.1, 30.0])
    runs = [(theta, np.full(5, 0.2), np.array([0.05, 0.05, 0.05, 0.05, 12.0]))]
    I = partition.dos_cluster(100, runs, -8.0, 20.0, 281)
    theta_in = theta[theta <= 20.0]
    for l, u in I:
        assert np.any((theta_in > l) & (theta_in <= u))
    assert len(I) == 2


def test_dos_cluster_partition_exact_count_and_tiling():
    rng = np.random.default_rng(8)
    centres = [-8.0, -3.0, 0.0, 6.0]
    theta = np.sort(np.concatenate([c + 0.2 * rng.standard_normal(20) for c in centres]))
    runs = _runs(theta, np.ones(theta.size))
    for n_s in (2, 4, 7, 12):
        I, sh = partition.dos_cluster_partition(4000, runs, -10.0, 8.0, n_s, 10 * theta.size)
        assert len(I) == n_s and len(sh) == n_s
        assert I[0][0] == -10.0 and I[-1][1] == 8.0
        for j in range(n_s - 1):
            assert I[j][1] == I[j + 1][0]
        for (l, u), s in zip(I, sh):
            assert l < s < u


def test_dos_cluster_refinement_separates_close_clusters():
    # two dense clusters 0.3 apart hold ~1000 eigenvalues each; a 12-point grid sees one
    # bump, the refined search on the over-full interval separates them
    theta = np.concatenate([0.01 * np.arange(10), 0.3 + 0.01 * np.arange(10), [5.0]])
    w = np.concatenate([np.ones(20), [0.05]])
    runs = [(theta, w / w.sum(), np.full(theta.size, 0.02))]
    coarse = partition.dos_cluster(2000, runs, -1.0, 6.0, 12)
    assert len(coarse) <= 2 and coarse[0][0] == -1.0 and coarse[0][1] > 0.4
    I, _ = partition.dos_cluster_partition(2000, runs, -1.0, 6.0, 3, 12)
    cuts = [u for _, u in I[:-1]]
    assert any(0.09 < c < 0.3 for c in cuts)        # between the two clusters


def test_migration_load_balance_insertion():
    # k-means leaves clusters of 93 and 117 values (mean 105): with balance = 1.1 the
    # larger one is split in two, after which no probe holds more than 1.1x the mean
    rng = np.random.default_rng(9)
    v = np.sort(np.concatenate([rng.uniform(0, 1, 10), rng.uniform(2, 10, 200)]))
    owner = (v > 1.5).astype(int)
    old = np.array([0.5, 6.0])
    plain = partition.migrate(v, owner, old, old)
    assert sorted(len(m) for _, m in plain) == [93, 117]
    assert partition.migrate(v, owner, old, old, balance=1.2) == plain
    bal = partition.migrate(v, owner, old, old, balance=1.1)
    assert len(bal) == 3
    assert sorted(i for _, m in bal for i in m) == list(range(v.size))
    assert max(len(m) for _, m in bal) <= 1.1 * v.size / 2
    for s_, m in bal:
        assert abs(s_ - v[m].mean()) < 1e-12
