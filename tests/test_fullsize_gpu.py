"""GPU parity at full workload sizes, on sampled outputs.

The GPU takes one coupled step of the full lattice and particle set (the same
kernels and launch configuration the benchmark times). The oracle evaluates
the same step for a sample of cells (every population that arrives at the cell,
with the spread force at each source cell summed over all particles) and a
sample of particles (interpolation, brute-force contacts over every particle,
update), from the same seeded inputs. FP64 bar 1e-10 relative; FP32 storage
bar 1e-4 relative (24-bit rounding of f - w per step, moments and weights in
FP32).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_1407_6704_gb300.inputs import populations, preset, velocities, workload_particles

pytestmark = pytest.mark.gpu

LAT = {9: "d2q9", 15: "d3q15", 19: "d3q19"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


def _sample_cells(w, rng, X, k_band=40, k_wall=8, k_any=12):
    """Cells where particles spread force (next to sampled particles), cells on
    the walls and cells anywhere."""
    n = np.array(w.n)
    cells = []
    for i in rng.choice(len(X), k_band, replace=False):
        c = np.clip(np.floor(X[i]).astype(int) + rng.integers(-1, 2, w.d), 0, n - 1)
        cells.append(c)
    for _ in range(k_wall):
        c = rng.integers(0, n)
        ax = rng.integers(0, w.d)
        c[ax] = 0 if rng.random() < 0.5 else n[ax] - 1
        cells.append(c)
    for _ in range(k_any):
        cells.append(rng.integers(0, n))
    flat = []
    for c in cells:
        f = int(c[0]) + int(n[0]) * (int(c[1]) + (int(n[1]) * int(c[2]) if w.d == 3 else 0))
        flat.append(f)
    return sorted(set(flat))


def _one_step(w, precision, f0_eps, u_scale, seed, n_part_samples=120, cell_samples=(40, 8, 12)):
    import torch
    from paper_1407_6704_gb300.pibm import Pibm

    X, dia, rr = workload_particles(w)
    U = velocities(len(X), w.d, seed=seed, scale=u_scale)
    _, _, wq, _ = lattice(w.q)
    f0 = populations(wq, tuple(reversed(w.n)), seed=seed + 1, eps=f0_eps) if f0_eps else None
    kw = dict(delta_width=w.delta_width, gravity=w.gravity, kn=w.kn, restitution=w.restitution,
              x0=X, u0=U, diameter=dia, density_ratio=rr, f0=f0)
    with Pibm(LAT[w.q], w.n, w.periodic, w.tau, precision=precision, **kw) as sim:
        sim.step(1)
        got = sim.read("pop", "x", "u")
        ffpi, fc = sim.forces()
        status = sim.status()
    torch.cuda.empty_cache()
    ref = Oracle(w.q, w.n, w.periodic, w.tau, **kw)
    rng = np.random.default_rng(seed + 2)
    parts = np.sort(rng.choice(len(X), n_part_samples, replace=False))
    cells = _sample_cells(w, rng, X, *cell_samples)
    return got, ffpi, fc, status, ref, parts, cells, X


def _check(got, ffpi, fc, status, ref, parts, cells, X, tol):
    assert status == 0
    q = ref.q
    pop = got["pop"].reshape(q, -1)
    f0 = ref.f.reshape(q, -1)
    w = ref.w[:, None]
    diff, scale = 0.0, 0.0
    for c in cells:
        exp = ref.cell_after_step(c)
        diff = max(diff, np.abs(pop[:, c] - exp).max())
        scale = max(scale, np.abs(f0[:, c:c + 1] - w).max(), np.abs(exp - ref.w).max())
    ex_x, ex_u, ex_g, ex_fc = [], [], [], []
    for i in parts:
        Xn, Un, g, Fc, _, _ = ref.particle_update(i)
        ex_x.append(Xn); ex_u.append(Un); ex_g.append(g); ex_fc.append(Fc)
    ex_x, ex_u, ex_g, ex_fc = map(np.array, (ex_x, ex_u, ex_g, ex_fc))
    Ap = np.pi * ref.dia[parts] ** 2 / 4
    e = {
        "pop": diff / scale,
        "x": np.abs(got["x"][parts] - ex_x).max() / np.abs(ex_x - X[parts]).max(),
        "u": np.abs(got["u"][parts] - ex_u).max() / np.abs(ex_u).max(),
        "f_fpi": np.abs(ffpi[parts] + Ap[:, None] * ex_g).max() / np.abs(Ap[:, None] * ex_g).max(),
    }
    if np.abs(ex_fc).max() > 0:
        e["f_c"] = np.abs(fc[parts] - ex_fc).max() / np.abs(ex_fc).max()
    bad = {k: v for k, v in e.items() if not v <= tol}
    assert not bad, (bad, e)
    return e


def test_c2_full_size_fp64_one_step():
    """2D D2Q9 2048^2, walls, tau 0.6, 500k particles, 4-point delta, FP64."""
    r = _one_step(preset("c2"), "fp64", f0_eps=1e-3, u_scale=1e-3, seed=101)
    print("c2 fp64", _check(*r, tol=1e-10))


def test_c2_full_size_fp32_one_step():
    r = _one_step(preset("c2"), "fp32", f0_eps=1e-3, u_scale=1e-3, seed=102)
    print("c2 fp32", _check(*r, tol=1e-4))


def test_c5_full_size_fp64_one_step():
    """3D D3Q19 96^3, walls, tau 0.7, 20k particles d=0.5, 4-point delta, FP64."""
    r = _one_step(preset("c5"), "fp64", f0_eps=1e-3, u_scale=1e-3, seed=103)
    print("c5 fp64", _check(*r, tol=1e-10))


def test_c3_full_size_fp32_one_step():
    """3D D3Q19 256^3, walls, tau 0.55, 4M particles d=0.6, 4-point delta, FP32.
    Fluid at rest, particles moving, so the first step spreads a non-zero force."""
    r = _one_step(preset("c3"), "fp32", f0_eps=0.0, u_scale=1e-3, seed=104, n_part_samples=40,
                  cell_samples=(8, 3, 3))
    print("c3 fp32", _check(*r, tol=1e-4))


def test_largest_lattice_the_cell_list_covers():
    """8192 x 8184 D2Q9 (67,043,328 bins, just under the scan's 8192^2 limit):
    particles released from rest in fluid at rest move by exactly
    m (1 - 1/rho_r) g / (m + 2 A_p) in the first step (no contacts)."""
    from paper_1407_6704_gb300.inputs import sample_particles
    from paper_1407_6704_gb300.pibm import Pibm

    n = (8192, 8184)
    X, dia, rr = sample_particles(n, 300, (0.3, 0.8), (1.5, 3.0), band=(0.0, 1.0), seed=7)
    g = (0.0, -1e-5)
    with Pibm("d2q9", n, (0, 0), 0.7, gravity=g, delta_width=4, precision="fp32", x0=X,
              diameter=dia, density_ratio=rr) as sim:
        sim.step(1)
        u = sim.read("u")["u"]
        assert sim.status() == 0
    m = rr * np.pi * dia ** 2 / 4
    Ap = np.pi * dia ** 2 / 4
    exp = m * (1 - 1 / rr) * g[1] / (m + 2 * Ap)
    assert np.abs(u[:, 0]).max() == 0.0
    assert np.abs(u[:, 1] - exp).max() <= 1e-6 * np.abs(exp).max()
