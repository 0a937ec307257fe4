"""Populations stored in FP16 (f - w scaled by 2^12) and BF16 (f - w) with FP32
collision and force, particles and contacts in FP64 (the particle update formed in
FP64 by default, optionally in FP32), against the FP64 oracle.

Bars, stated per field as a relative error against the FP64 oracle:
- velocity field, relative L2: FP32 <= 1e-5, FP16 <= 1e-3;
- particle displacement and velocity: FP16 <= 1e-3.
BF16 keeps 8 bits of mantissa, so each stored deviation f - w is resolved to
about 2^-9 of itself and the velocity field, carried by those deviations,
inherits an error of the same order (a few 1e-3 after 1000 steps). BF16 storage
therefore does not meet the 1e-3 velocity bar and is not one of the qualifying
reduced-precision forms; it is held to 1e-2 here only to catch breakage.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_1407_6704_gb300.inputs import populations, preset, sample_particles, velocities

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


def _errors(got, rho_r, j_r, X_r, U_r, X0):
    u = got["j"] / got["rho"]
    ur = j_r / rho_r
    return {
        "u_l2": float(np.sqrt(((u - ur) ** 2).sum() / (ur ** 2).sum())),
        "x": float(np.abs(got["x"] - X_r).max() / np.abs(X_r - X0).max()),
        "up": float(np.sqrt(((got["u"] - U_r) ** 2).sum() / (U_r ** 2).sum())),
    }


BARS = {"fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-2}


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_reduced_storage_against_fp64_oracle(precision):
    """D3Q19 20x18x24 with walls, 300 particles, 4-point delta, 200 steps from a
    perturbed state, against the FP64 CPU oracle."""
    from paper_1407_6704_gb300.pibm import Pibm

    n = (20, 18, 24)
    X, dia, rr = sample_particles(n, 300, 0.6, 2.0, band=(0.4, 1.0), seed=61)
    U = velocities(300, 3, seed=62, scale=1e-3)
    _, _, w, _ = lattice(19)
    f0 = populations(w, tuple(reversed(n)), seed=63, eps=2e-3)
    kw = dict(delta_width=4, gravity=(0, 0, -1e-4), x0=X, u0=U, diameter=dia, density_ratio=rr,
              f0=f0)
    ref = Oracle(19, n, (0, 0, 0), 0.6, **kw)
    ref.step(200)
    rho_r, j_r = ref.moments()
    with Pibm("d3q19", n, (0, 0, 0), 0.6, precision=precision, **kw) as sim:
        sim.step(200)
        got = sim.read("rho", "j", "x", "u")
        assert sim.status() == 0
    e = _errors(got, rho_r, j_r, ref.X, ref.U, X)
    print(precision, e)
    assert all(v <= BARS[precision] for v in e.values()), e


@pytest.fixture(scope="module")
def slice_32():
    """32^3 D3Q19 slice with the 256^3 workload's particle density (7812 particles,
    d = 0.6, ratio 2, top half), tau 0.55, walls, gravity 1e-5, 4-point kernel:
    the FP64 oracle (OpenMP build) after 1000 steps."""
    w = preset("c3")
    n = (32, 32, 32)
    npart = int(round(w.n_particles * (32 ** 3) / w.ncell))
    X, dia, rr = sample_particles(n, npart, w.diameter, w.density_ratio, w.band, 91)
    kw = dict(delta_width=w.delta_width, gravity=w.gravity, kn=w.kn, restitution=w.restitution,
              x0=X, diameter=dia, density_ratio=rr)
    ref = Oracle(19, n, w.periodic, w.tau, parallel=True, **kw)
    ref.step(1000)
    rho_r, j_r = ref.moments()
    return dict(n=n, w=w, kw=kw, X0=X, rho=rho_r, j=j_r, X=ref.X.copy(), U=ref.U.copy())


SLICE_BARS = {"fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-2}


@pytest.mark.parametrize("precision,update", [("fp32", "fp64"), ("fp16", "fp64"),
                                               ("bf16", "fp64"), ("fp32", "fp32"),
                                               ("fp16", "fp32")])
def test_storage_modes_on_the_32_cubed_slice_against_the_oracle(slice_32, precision, update):
    """1000 steps of the 3D workload's slice in each storage mode, in the benchmark's
    launch configuration (cell list kept for 10 steps), against the FP64 oracle;
    the particle update formed in FP64 (the default) or in FP32."""
    from paper_1407_6704_gb300.pibm import Pibm

    c = slice_32
    w = c["w"]
    with Pibm("d3q19", c["n"], w.periodic, w.tau, precision=precision, rebin_every=10,
              particle_update=update, **c["kw"]) as sim:
        sim.step(1000)
        got = sim.read("rho", "j", "x", "u")
        assert sim.status() == 0
    e = _errors(got, c["rho"], c["j"], c["X"], c["U"], c["X0"])
    print("32^3 slice", precision, "update", update, e)
    assert all(v <= SLICE_BARS[precision] for v in e.values()), e


def test_fp16_on_the_64_cubed_slice_of_the_3d_workload():
    """64^3 D3Q19 slice with the 3D workload's particle density (62,500 particles,
    d = 0.6, ratio 2, top half), 1000 steps: FP16 storage against the library's
    FP64 path at this size (a consistency check; the brute-force oracle is too slow
    for 62,500 particles, and the oracle comparison is the 32^3 test above)."""
    from paper_1407_6704_gb300.inputs import workload_particles
    from paper_1407_6704_gb300.pibm import Pibm

    w = preset("c3s")
    X, dia, rr = workload_particles(w)
    out = {}
    for prec in ("fp64", "fp16"):
        with Pibm.from_workload(w, precision=prec, particles=(X, dia, rr)) as sim:
            sim.step(1000)
            out[prec] = sim.read("rho", "j", "x", "u")
            assert sim.status() == 0
    r = out["fp64"]
    e = _errors(out["fp16"], r["rho"], r["j"], r["x"], r["u"], X)
    print("c3s fp16", e)
    assert e["u_l2"] <= 1e-3 and e["up"] <= 1e-3, e


@pytest.mark.parametrize("q,n,periodic", [
    (9, (66, 40), (0, 0)),       # pair kernel: walls, a warp with one active lane at the right wall
    (9, (64, 40), (1, 0)),       # pair kernel: periodic x, warp-edge and domain-edge wraps
    (19, (21, 18, 24), (0, 1, 0)),  # odd n[0]: one cell per thread
])
def test_fp16_storage_kernels_against_oracle(q, n, periodic):
    """16-bit storage runs one of two collide kernels: two cells per thread with
    shuffled neighbours (even n[0]) or one cell per thread (odd n[0]); both
    against the FP64 oracle, velocity L2 <= 1e-3."""
    from paper_1407_6704_gb300.pibm import Pibm

    d = len(n)
    X, dia, rr = sample_particles(n, 120, (0.3, 0.8), 2.0, band=(0.3, 1.0), seed=71)
    U = velocities(120, d, seed=72, scale=1e-3)
    _, _, w, _ = lattice(q)
    f0 = populations(w, tuple(reversed(n)), seed=73, eps=2e-3)
    kw = dict(delta_width=4, gravity=(0.0,) * (d - 1) + (-1e-4,), x0=X, u0=U, diameter=dia,
              density_ratio=rr, f0=f0)
    ref = Oracle(q, n, periodic, 0.7, **kw)
    ref.step(150)
    rho_r, j_r = ref.moments()
    lat = {9: "d2q9", 19: "d3q19"}[q]
    with Pibm(lat, n, periodic, 0.7, precision="fp16", **kw) as sim:
        sim.step(150)
        got = sim.read("rho", "j", "x", "u")
        assert sim.status() == 0
    e = _errors(got, rho_r, j_r, ref.X, ref.U, X)
    print("fp16", n, periodic, e)
    assert all(v <= 1e-3 for v in e.values()), e
