"""The OpenMP build of the oracle (cell loops and per-particle updates on all
cores, spreading serial in index order) against the serial build: bitwise equal
populations, particle state, forces and diagnostics after whole steps, with
contacts, walls and periodic axes, with and without DEM sub-cycling. CPU only."""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_1407_6704_gb300.inputs import populations, sample_particles, velocities


def _pair(q, n, periodic, npart, seed, steps, **extra):
    d = len(n)
    X, D, R = sample_particles(n, npart, (0.5, 0.9), (1.5, 3.0), band=(0.0, 1.0), seed=seed)
    # squeeze the cloud towards its centre so that many pairs overlap
    c = np.asarray(n, dtype=float) / 2
    X = c + 0.85 * (X - c)
    U = velocities(npart, d, seed=seed + 1, scale=2e-3)
    _, _, w, _ = lattice(q)
    f0 = populations(w, tuple(reversed(n)), seed=seed + 2, eps=1e-3)
    kw = dict(delta_width=4, gravity=(0.0,) * (d - 1) + (-1e-4,), x0=X, u0=U, diameter=D,
              density_ratio=R, f0=f0, **extra)
    out = []
    for par in (False, True):
        o = Oracle(q, n, periodic, 0.7, parallel=par, **kw)
        o.step(steps)
        out.append(o)
    return out


@pytest.mark.parametrize("q,n,periodic,extra", [
    (9, (40, 34), (1, 0), {}),
    (19, (14, 12, 16), (0, 1, 0), {}),
    (9, (36, 30), (0, 0), {"substeps": 3, "contact": "hertz", "young": 0.05}),
])
def test_openmp_build_is_bitwise_identical(q, n, periodic, extra):
    ser, par = _pair(q, n, periodic, 160 if q == 9 else 90, seed=5, steps=25, **extra)
    assert np.abs(ser.Fc).max() > 0  # contacts did happen
    for name in ("f", "X", "U", "g", "Fc", "F", "diag"):
        assert np.array_equal(getattr(ser, name), getattr(par, name)), name
