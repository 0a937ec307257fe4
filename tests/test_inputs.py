"""The seeded input generators shared by the oracle and the CUDA path: the
guarantees the workloads rely on (non-overlapping particles inside their band,
at least a radius from every wall, reproducible per seed), and the presets'
sizes."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_1407_6704_gb300.inputs import (ensemble_workloads, populations, preset,
                                          sample_particles, velocities, workload_particles)


@pytest.mark.parametrize("n,npart,dia,rr,band", [
    ((64, 48), 300, (0.3, 0.8), (1.5, 3.0), (0.4, 1.0)),
    ((20, 18, 24), 400, 0.6, 2.0, (0.5, 1.0)),
    ((33, 17), 80, (0.5, 0.9), 2.5, (0.0, 0.3)),
])
def test_particles_do_not_overlap_and_stay_in_their_band(n, npart, dia, rr, band):
    X, D, R = sample_particles(n, npart, dia, rr, band=band, seed=5)
    d = len(n)
    assert X.shape == (npart, d) and D.shape == (npart,) and R.shape == (npart,)
    lo_d, hi_d = (dia, dia) if np.isscalar(dia) else dia
    lo_r, hi_r = (rr, rr) if np.isscalar(rr) else rr
    assert np.all((D >= lo_d) & (D <= hi_d)) and np.all((R >= lo_r) & (R <= hi_r))
    rmax = 0.5 * D.max()
    for k in range(d):
        assert np.all(X[:, k] >= rmax) and np.all(X[:, k] <= n[k] - rmax)
    assert np.all(X[:, -1] >= band[0] * n[-1]) and np.all(X[:, -1] <= band[1] * n[-1])
    # every pair at least the sum of the radii apart
    pairs = cKDTree(X).query_pairs(D.max(), output_type="ndarray")
    if pairs.size:
        i, j = pairs[:, 0], pairs[:, 1]
        dist = np.linalg.norm(X[i] - X[j], axis=1)
        assert np.all(dist >= 0.5 * (D[i] + D[j]))


def test_same_seed_same_draw_other_seed_other_draw():
    a = sample_particles((40, 30), 100, (0.3, 0.8), 2.0, band=(0.3, 1.0), seed=11)
    b = sample_particles((40, 30), 100, (0.3, 0.8), 2.0, band=(0.3, 1.0), seed=11)
    c = sample_particles((40, 30), 100, (0.3, 0.8), 2.0, band=(0.3, 1.0), seed=12)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert not np.array_equal(a[0], c[0])
    assert np.array_equal(populations([1.0, 2.0], (3, 4), seed=3),
                          populations([1.0, 2.0], (3, 4), seed=3))
    assert np.array_equal(velocities(7, 2, seed=4), velocities(7, 2, seed=4))


def test_populations_and_velocities_stay_in_their_ranges():
    base = np.array([4 / 9, 1 / 9, 1 / 36])
    f = populations(base, (5, 6), seed=2, eps=1e-3)
    assert f.shape == (3, 5, 6)
    rel = f / base.reshape(-1, 1, 1) - 1.0
    assert np.all(np.abs(rel) <= 1e-3)
    u = velocities(50, 3, seed=1, scale=2e-3)
    assert u.shape == (50, 3) and np.all(np.abs(u) <= 2e-3)


def test_presets_have_the_measured_sizes():
    c1, c2, c3, c5 = (preset(k) for k in ("c1", "c2", "c3", "c5"))
    assert (c1.q, c1.n, c1.n_particles, c1.delta_width) == (9, (128, 128), 200, 2)
    assert (c2.q, c2.n, c2.n_particles, c2.delta_width) == (9, (2048, 2048), 500_000, 4)
    assert (c3.q, c3.n, c3.n_particles, c3.delta_width) == (19, (256, 256, 256), 4_000_000, 4)
    assert (c5.q, c5.n, c5.n_particles, c5.delta_width) == (19, (96, 96, 96), 20_000, 4)
    c3s = preset("c3s")
    # the 64^3 slice keeps the particle density of the 256^3 workload
    assert c3s.n_particles / c3s.ncell == pytest.approx(c3.n_particles / c3.ncell, rel=0.01)
    X, D, R = workload_particles(c1)
    assert X.shape == (200, 2) and np.all(X[:, 1] >= 0.5 * 128)


def test_ensemble_members_respect_their_ranges_and_the_area_cap():
    members = ensemble_workloads(count=6, particles=(100, 2000))
    assert len(members) == 6
    for w, (X, D, R) in members:
        s = w.n[0]
        assert w.n == (s, s) and 64 <= s <= 512
        assert 0.55 <= w.tau <= 1.0 and 1.5 <= w.density_ratio <= 3.0
        assert len(X) == w.n_particles
        area = len(X) * np.pi * 0.25 ** 2
        assert area <= 0.3 * s * s / 2.0 + 1e-9
        assert np.all(X[:, 1] >= 0.5 * s)
