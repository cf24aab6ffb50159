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
