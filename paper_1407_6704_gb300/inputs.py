"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it draws particle positions,
diameters and density ratios (uniform random, non-overlapping, inside a band of
the domain) and random population fields around a base vector that the caller
supplies. Both the CUDA path and the oracle receive exactly these arrays.

Workload presets mirror the sedimentation set-ups used for measurement:
  c1  2D D2Q9 128x128, walls, tau 0.8, 200 particles d=0.5, rho_p/rho_f=2, top half,
      gravity 1e-5, 2-point delta
  c2  2D D2Q9 2048x2048, walls, tau 0.6, 500k particles d~U[0.3,0.8], ratio 2.5,
      top 60 %, 4-point delta
  c3  3D D3Q19 256^3, walls, tau 0.55, 4M particles d=0.6, ratio 2, top half, 4-point
  c3s the 64^3 slice of c3 with the same particle density (62,500 particles)
  c5  3D D3Q19 96^3, walls, tau 0.7, 20k particles d=0.5, ratio 2, top half, 4-point
  c4  (ensemble_workloads) 64 independent 2D instances, sides log-uniform in
      [64, 512], 100..20k particles (at most 30 % area of the top half), tau in
      [0.55, 1.0], ratio in [1.5, 3.0], d = 0.5, 2-point delta
Contacts: linear spring-dashpot, kn = 1e-2, restitution 0.9, everywhere.
"""
from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import numpy as np


@dataclass
class Workload:
    name: str
    q: int
    n: Tuple[int, ...]
    periodic: Tuple[int, ...]
    tau: float
    delta_width: int
    gravity: Tuple[float, ...]
    n_particles: int
    diameter: object          # float or (lo, hi)
    density_ratio: object     # float or (lo, hi)
    band: Tuple[float, float]  # fraction of the gravity axis holding particles
    seed: int
    kn: float = 1e-2
    restitution: float = 0.9
    steps: int = 1000
    extra: dict = field(default_factory=dict)

    @property
    def d(self):
        return len(self.n)

    @property
    def ncell(self):
        return int(np.prod(self.n))


def preset(name: str) -> Workload:
    g2 = (0.0, -1e-5)
    g3 = (0.0, 0.0, -1e-5)
    if name == "c1":
        return Workload("c1", 9, (128, 128), (0, 0), 0.8, 2, g2, 200, 0.5, 2.0, (0.5, 1.0), 1,
                        steps=1000)
    if name == "c2":
        return Workload("c2", 9, (2048, 2048), (0, 0), 0.6, 4, g2, 500_000, (0.3, 0.8), 2.5,
                        (0.4, 1.0), 2, steps=10_000)
    if name == "c3":
        return Workload("c3", 19, (256, 256, 256), (0, 0, 0), 0.55, 4, g3, 4_000_000, 0.6, 2.0,
                        (0.5, 1.0), 3)
    if name == "c3s":
        return Workload("c3s", 19, (64, 64, 64), (0, 0, 0), 0.55, 4, g3, 62_500, 0.6, 2.0,
                        (0.5, 1.0), 3)
    if name == "c5":
        return Workload("c5", 19, (96, 96, 96), (0, 0, 0), 0.7, 4, g3, 20_000, 0.5, 2.0,
                        (0.5, 1.0), 5, steps=500)
    raise KeyError(name)


def _draw(rng, spec, n):
    if np.isscalar(spec):
        return np.full(n, float(spec))
    lo, hi = spec
    return rng.uniform(lo, hi, n)


def sample_particles(n: Sequence[int], n_particles: int, diameter, density_ratio,
                     band=(0.5, 1.0), seed=0, max_rounds=400):
    """Uniform random, pairwise non-overlapping particles.

    Positions are drawn uniformly in a box that keeps every particle at least
    half the largest diameter away from each face of the domain; along the last
    axis (the gravity axis) the box is further restricted to ``band`` (fractions
    of the extent). Every round draws positions for the particles not yet placed;
    a candidate is kept when it overlaps no kept particle and no lower-index
    candidate of the same round. Returns X (np, d), diameter (np,), density ratio
    (np,), all float64.
    """
    from scipy.spatial import cKDTree

    rng = np.random.Generator(np.random.PCG64(seed))
    d = len(n)
    dia = _draw(rng, diameter, n_particles)
    rr = _draw(rng, density_ratio, n_particles)
    if n_particles == 0:
        return np.zeros((0, d)), dia, rr
    dmax = float(dia.max())
    lo = np.full(d, 0.5 * dmax)
    hi = np.array(n, dtype=np.float64) - 0.5 * dmax
    lo[-1] = max(lo[-1], band[0] * n[-1])
    hi[-1] = min(hi[-1], band[1] * n[-1])
    if np.any(hi <= lo):
        raise ValueError("empty placement region")
    X = np.zeros((n_particles, d))
    placed = np.zeros(n_particles, dtype=bool)
    # kept particles live in a large tree rebuilt rarely plus a small recent set
    base_ids = np.zeros(0, dtype=np.int64)
    base_tree = None
    recent = []
    for _ in range(max_rounds):
        todo = np.nonzero(~placed)[0]
        if todo.size == 0:
            break
        cand = lo + (hi - lo) * rng.random((todo.size, d))
        ok = np.ones(todo.size, dtype=bool)
        # against the particles already kept
        rec = np.concatenate(recent) if recent else np.zeros(0, dtype=np.int64)
        if rec.size > max(base_ids.size // 4, 1024):
            base_ids = np.concatenate([base_ids, rec])
            base_tree = cKDTree(X[base_ids])
            recent, rec = [], np.zeros(0, dtype=np.int64)
        ctree = None
        for ids, tree in ((base_ids, base_tree), (rec, None)):
            if ids.size == 0:
                continue
            if tree is None:
                tree = cKDTree(X[ids])
            if ctree is None:
                ctree = cKDTree(cand)
            pairs = ctree.sparse_distance_matrix(tree, dmax, output_type="ndarray")
            if pairs.size:
                ci, ki, dist = pairs["i"], pairs["j"], pairs["v"]
                clash = dist < 0.5 * (dia[todo[ci]] + dia[ids[ki]])
                ok[ci[clash]] = False
        # within the round: the lower index wins
        sel = np.nonzero(ok)[0]
        if sel.size > 1:
            pr = cKDTree(cand[sel]).query_pairs(dmax, output_type="ndarray")
            if pr.size:
                i, j = sel[pr.min(axis=1)], sel[pr.max(axis=1)]
                dist = np.linalg.norm(cand[i] - cand[j], axis=1)
                clash = dist < 0.5 * (dia[todo[i]] + dia[todo[j]])
                ok[j[clash]] = False
        sel = np.nonzero(ok)[0]
        X[todo[sel]] = cand[sel]
        placed[todo[sel]] = True
        recent.append(todo[sel])
    if not placed.all():
        raise RuntimeError(f"could not place {np.count_nonzero(~placed)} particles")
    return X, dia, rr


def ensemble_workloads(count=64, seed=4, side=(64, 512), particles=(100, 20_000), tau=(0.55, 1.0),
                       ratio=(1.5, 3.0), diameter=0.5, max_area_fraction=0.3):
    """The batched ensemble: ``count`` independent 2D sedimentation instances
    (D2Q9, walls, gravity 1e-5, 2-point delta, d = 0.5): square sides
    log-uniform in ``side``, particle counts log-uniform in ``particles`` but at
    most ``max_area_fraction`` of the top half's area, tau and density ratio
    uniform in their ranges. Returns (Workload, (X, diameter, ratio)) pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        s_ = int(round(np.exp(rng.uniform(np.log(side[0]), np.log(side[1])))))
        np_ = int(round(np.exp(rng.uniform(np.log(particles[0]), np.log(particles[1])))))
        cap = int(max_area_fraction * (s_ * s_ / 2.0) / (np.pi * diameter ** 2 / 4.0))
        np_ = min(np_, cap)
        t_ = float(rng.uniform(*tau))
        r_ = float(rng.uniform(*ratio))
        w = Workload(f"c4.{i}", 9, (s_, s_), (0, 0), t_, 2, (0.0, -1e-5), np_, diameter, r_,
                     (0.5, 1.0), 1000 + i, steps=2000)
        out.append((w, workload_particles(w)))
    return out


def workload_particles(w: Workload, n_particles: Optional[int] = None):
    npart = w.n_particles if n_particles is None else n_particles
    return sample_particles(w.n, npart, w.diameter, w.density_ratio, w.band, w.seed)


def populations(base, shape, seed=0, eps=1e-2):
    """Random positive populations base[a] * (1 + eps * r), r ~ U(-1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.asarray(base, dtype=np.float64)
    r = rng.uniform(-1.0, 1.0, (base.size,) + tuple(shape))
    return base.reshape((-1,) + (1,) * len(shape)) * (1.0 + eps * r)


def velocities(n_particles, d, seed=0, scale=1e-3):
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.uniform(-1.0, 1.0, (n_particles, d))
