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
