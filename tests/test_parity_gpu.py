"""GPU parity: the CUDA path against the FP64 CPU oracle on identical seeded inputs.

Every case runs whole coupled steps through the C ABI and compares, element by
element, the post-stream populations, rho, j, particle positions, velocities and
forces. FP64 bar: max |gpu - oracle| / max |oracle reference quantity| <= 1e-10
(the oracle reference quantity is the deviation from rest for populations and
density, the displacement for positions). The two sides sum in different orders
(and the spreading uses atomics), so agreement is to rounding, not bitwise.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_1407_6704_gb300.inputs import populations, preset, sample_particles, velocities

pytestmark = pytest.mark.gpu

LAT = {9: "d2q9", 15: "d3q15", 19: "d3q19"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


def make_case(q, n, periodic, tau, width, npart, seed, implicit=True, f0_eps=0.0, u_scale=0.0,
              gravity=None, dia=(0.3, 0.8), rr=(1.5, 3.0), band=(0.3, 1.0), kn=1e-2, e=0.9):
    d = len(n)
    X, D, R = sample_particles(n, npart, dia, rr, band=band, seed=seed)
    U = velocities(npart, d, seed=seed + 1, scale=u_scale) if u_scale else None
    _, _, w, _ = lattice(q)
    f0 = populations(w, tuple(reversed(n)), seed=seed + 2, eps=f0_eps) if f0_eps else None
    g = gravity if gravity is not None else (0.0,) * (d - 1) + (-1e-4,)
    return dict(q=q, n=n, periodic=periodic, tau=tau, width=width, implicit=implicit, X=X, U=U,
                D=D, R=R, f0=f0, gravity=g, kn=kn, e=e)


def run_both(c, steps, precision="fp64", deterministic=False, **gpu):
    """The oracle (OpenMP build, bitwise equal to the serial one) and the library
    from the same inputs; gpu: extra options of the library's run only
    (rebin_every, overlap), which do not change the result beyond rounding."""
    from paper_1407_6704_gb300.pibm import Pibm

    kw = dict(delta_width=c["width"], gravity=c["gravity"], kn=c["kn"], restitution=c["e"],
              x0=c["X"], u0=c["U"], diameter=c["D"], density_ratio=c["R"], f0=c["f0"])
    ref = Oracle(c["q"], c["n"], c["periodic"], c["tau"], implicit_drag=c["implicit"],
                 parallel=True, **kw)
    ref.step(steps)
    with Pibm(LAT[c["q"]], c["n"], c["periodic"], c["tau"], implicit=c["implicit"],
              precision=precision, deterministic=deterministic, **kw, **gpu) as sim:
        sim.step(steps)
        got = sim.read("pop", "rho", "j", "x", "u")
        got["f_fpi"], got["f_c"] = sim.forces()
        got["status"] = sim.status()
    return got, ref


def rel_errors(got, ref, X0):
    """Per field max |gpu - oracle| / max |oracle|; positions use the displacement
    X - X0. 'dpop' and 'drho' normalise by the deviation from rest instead (f - w,
    rho - 1), a much smaller quantity in these weakly driven flows."""
    rho_r, j_r = ref.moments()
    w = ref.w.reshape((-1,) + (1,) * len(ref.shape))
    e = {}
    dp = np.abs(got["pop"] - ref.f).max()
    dr = np.abs(got["rho"] - rho_r).max()
    e["pop"] = dp / np.abs(ref.f).max()
    e["rho"] = dr / np.abs(rho_r).max()
    e["dpop"] = dp / max(np.abs(ref.f - w).max(), 1e-300)
    e["drho"] = dr / max(np.abs(rho_r - 1.0).max(), 1e-300)
    e["j"] = np.abs(got["j"] - j_r).max() / max(np.abs(j_r).max(), 1e-300)
    if ref.np:
        e["x"] = np.abs(got["x"] - ref.X).max() / max(np.abs(ref.X - X0).max(), 1e-300)
        e["u"] = np.abs(got["u"] - ref.U).max() / max(np.abs(ref.U).max(), 1e-300)
        ffpi = ref.f_fpi
        e["f_fpi"] = np.abs(got["f_fpi"] - ffpi).max() / max(np.abs(ffpi).max(), 1e-300)
        if np.abs(ref.Fc).max() > 0:
            e["f_c"] = np.abs(got["f_c"] - ref.Fc).max() / np.abs(ref.Fc).max()
    return e


# FP64 bar on every field; the deviation-normalised population and density errors
# get 1e-8 (rounding of ~1e-16 per step on values near w, accumulated over up to
# 1000 steps, against deviations from rest as small as 1e-6).
TOL = {"dpop": 1e-8, "drho": 1e-8}


def assert_parity(got, ref, X0, tol=1e-10):
    assert got["status"] == 0
    e = rel_errors(got, ref, X0)
    bad = {k: v for k, v in e.items() if not v <= TOL.get(k, tol)}
    assert not bad, f"relative errors above {tol}: {bad} (all: {e})"
    return e


def test_sedimentation_2d_128_full_1000_steps():
    """128^2 D2Q9, walls, tau 0.8, 200 particles d=0.5, density ratio 2, top half,
    gravity 1e-5, 2-point delta, FP64, 1000 steps."""
    w = preset("c1")
    X, D, R = sample_particles(w.n, w.n_particles, w.diameter, w.density_ratio, w.band, w.seed)
    c = dict(q=9, n=w.n, periodic=w.periodic, tau=w.tau, width=2, implicit=True, X=X, U=None,
             D=D, R=R, f0=None, gravity=w.gravity, kn=w.kn, e=w.restitution)
    got, ref = run_both(c, w.steps)
    e = assert_parity(got, ref, X)
    print("c1 parity", e)


CASES = [
    # ragged lattice, 4-point delta, random initial populations and velocities
    ("2d_ragged_w4", dict(q=9, n=(37, 29), periodic=(0, 0), tau=0.62, width=4, npart=90,
                          seed=11, f0_eps=1e-3, u_scale=2e-3), 121),
    ("2d_ragged_w2_explicit", dict(q=9, n=(45, 23), periodic=(0, 0), tau=0.9, width=2, npart=70,
                                   seed=12, implicit=False, f0_eps=1e-3, u_scale=1e-3,
                                   rr=(2.0, 3.0)), 120),
    ("2d_periodic_x", dict(q=9, n=(33, 26), periodic=(1, 0), tau=0.7, width=4, npart=80, seed=13,
                           f0_eps=1e-3, u_scale=2e-3), 100),
    ("2d_fully_periodic", dict(q=9, n=(24, 20), periodic=(1, 1), tau=0.7, width=4, npart=50,
                               seed=14, f0_eps=1e-3, u_scale=2e-3, band=(0.0, 1.0)), 80),
    ("3d_d3q19_w4", dict(q=19, n=(13, 11, 17), periodic=(0, 0, 0), tau=0.7, width=4, npart=60,
                         seed=15, f0_eps=1e-3, u_scale=1e-3), 50),
    ("3d_d3q19_w2_periodic_xy", dict(q=19, n=(12, 10, 14), periodic=(1, 1, 0), tau=0.6, width=2,
                                     npart=70, seed=16, f0_eps=1e-3, u_scale=1e-3), 50),
    ("3d_d3q15_w4", dict(q=15, n=(10, 9, 12), periodic=(0, 0, 0), tau=0.75, width=4, npart=40,
                         seed=17, f0_eps=1e-3, u_scale=1e-3), 40),
]


@pytest.mark.parametrize("name,kw,steps", CASES, ids=[c[0] for c in CASES])
def test_parity_fp64(name, kw, steps):
    c = make_case(**kw)
    got, ref = run_both(c, steps)
    e = assert_parity(got, ref, c["X"])
    print(name, e)


def test_dense_contacts_parity():
    """Many overlapping contacts: a packed cloud squeezed so that neighbours overlap
    by up to ~20 % of a diameter, then released."""
    c = make_case(q=9, n=(24, 20), periodic=(0, 0), tau=0.7, width=2, npart=160, seed=21,
                  dia=(0.6, 0.9), rr=2.0, band=(0.25, 0.95), kn=5e-3, u_scale=2e-3)
    centre = np.array([12.0, 12.0])
    c["X"] = centre + 0.85 * (c["X"] - centre)
    got, ref = run_both(c, 60)
    assert np.count_nonzero(np.abs(ref.Fc).sum(1)) > 20
    assert_parity(got, ref, c["X"])


def test_no_particles_fluid_only():
    c = make_case(q=19, n=(9, 8, 7), periodic=(1, 0, 1), tau=0.8, width=2, npart=0, seed=22,
                  f0_eps=5e-3)
    got, ref = run_both(c, 30)
    assert_parity(got, ref, c["X"])


def test_single_particle_near_wall():
    X = np.array([[0.3, 7.9]])
    c = dict(q=9, n=(10, 8), periodic=(0, 0), tau=0.8, width=4, implicit=True, X=X,
             U=np.array([[-1e-3, 2e-3]]), D=np.array([0.8]), R=np.array([2.0]), f0=None,
             gravity=(0.0, -1e-4), kn=1e-2, e=0.9)
    got, ref = run_both(c, 41)
    assert_parity(got, ref, X)


def test_deterministic_mode_parity_and_bitwise_repeat():
    c = make_case(q=9, n=(30, 26), periodic=(0, 0), tau=0.7, width=4, npart=120, seed=23,
                  f0_eps=1e-3, u_scale=2e-3)
    got1, ref = run_both(c, 60, deterministic=True)
    assert_parity(got1, ref, c["X"])
    got2, _ = run_both(c, 60, deterministic=True)
    for k in ("pop", "x", "u"):
        assert np.array_equal(got1[k], got2[k]), k


def test_fp32_path_against_fp64_oracle():
    """Populations stored as f - w in FP32 with FP32 collision; particle state
    and contacts FP64, the per-step particle increment in FP32.
    Each step rounds the stored deviation to 24 bits (relative 6e-8 of |f - w|),
    so after 100 steps the velocity field stays within 1e-4 (relative L2)."""
    c = make_case(q=9, n=(40, 34), periodic=(0, 0), tau=0.7, width=4, npart=100, seed=24,
                  f0_eps=1e-3, u_scale=2e-3)
    got, ref = run_both(c, 100, precision="fp32")
    assert got["status"] == 0
    rho_r, j_r = ref.moments()
    ur = j_r / rho_r
    ug = got["j"] / got["rho"]
    l2 = np.sqrt(((ug - ur) ** 2).sum() / (ur ** 2).sum())
    assert l2 < 1e-4, l2
    assert np.abs(got["u"] - ref.U).max() / np.abs(ref.U).max() < 1e-4
    assert np.abs(got["x"] - ref.X).max() / np.abs(ref.X - c["X"]).max() < 1e-4


def test_invariants_match_oracle():
    from paper_1407_6704_gb300.pibm import Pibm

    c = make_case(q=9, n=(24, 20), periodic=(1, 1), tau=0.7, width=4, npart=50, seed=25,
                  f0_eps=1e-3, u_scale=2e-3, band=(0.0, 1.0))
    kw = dict(delta_width=4, gravity=c["gravity"], x0=c["X"], u0=c["U"], diameter=c["D"],
              density_ratio=c["R"], f0=c["f0"])
    ref = Oracle(9, c["n"], (1, 1), 0.7, **kw)
    with Pibm("d2q9", c["n"], (1, 1), 0.7, **kw) as sim:
        for _ in range(5):
            sim.step(3)
            ref.step(3)
            mass, J, P = sim.invariants()
            rho_r, j_r = ref.moments()
            m = (ref.rr * np.pi * ref.dia ** 2 / 4)
            assert abs(mass - rho_r.sum()) / rho_r.sum() < 1e-14
            assert np.abs(J - j_r.reshape(2, -1).sum(1)).max() < 1e-12
            assert np.abs(P - (m[:, None] * ref.U).sum(0)).max() < 1e-12 * np.abs(P).max() + 1e-18


def test_escaped_particle_is_reported():
    """A particle thrown at a wall faster than any contact can stop it is flagged
    (status PIBM_EESCAPED); the run itself stays memory-safe."""
    from paper_1407_6704_gb300 import _lib
    from paper_1407_6704_gb300.pibm import Pibm

    with Pibm("d2q9", (16, 16), (0, 0), 0.8, delta_width=4, x0=[[8.0, 1.0]], u0=[[0.0, -3.0]],
              diameter=[0.5], density_ratio=[2.0], kn=0.0) as sim:
        sim.step(2)
        assert sim.status() == _lib.PIBM_EESCAPED


def test_nonfinite_state_is_reported():
    from paper_1407_6704_gb300 import _lib
    from paper_1407_6704_gb300.pibm import Pibm

    _, _, w, _ = lattice(9)
    f0 = populations(w, (12, 12), seed=3, eps=1e-3)
    f0[3, 5, 5] = np.nan
    with Pibm("d2q9", (12, 12), (0, 0), 0.8, f0=f0) as sim:
        sim.step(2)
        assert sim.status() == _lib.PIBM_EUNSTABLE


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("q,n", [(9, (14, 12)), (19, (10, 8, 9))])
def test_mach_guard_is_reported(q, n, precision):
    """A cell whose populations carry a fluid speed of 0.35 (the equilibrium of
    Eq. 3 at that velocity, set on the host) raises PIBM_EUNSTABLE at the first
    collision; the same field at 0.25 runs clean."""
    from paper_1407_6704_gb300 import _lib
    from paper_1407_6704_gb300.pibm import Pibm

    d, e, w, _ = lattice(q)
    shape = tuple(reversed(n))
    for speed, status in ((0.25, _lib.PIBM_OK), (0.35, _lib.PIBM_EUNSTABLE)):
        u = np.zeros(3)
        u[0] = speed
        eu = e @ u
        feq = w * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u @ u))
        f0 = np.empty((q,) + shape)
        f0[:] = w.reshape((-1,) + (1,) * d)
        f0[(slice(None),) + tuple(k // 2 for k in shape)] = feq
        with Pibm(LAT[q], n, (1,) * d, 0.8, f0=f0, precision=precision) as sim:
            sim.step(1)
            assert sim.status() == status, (speed, sim.status())


def _workload_case(name, n, seed, f0_eps=1e-3, u_scale=2e-3):
    """A lattice of extent n with the particle density, diameters, density ratios,
    band, relaxation time, gravity, kernel and contact law of a preset workload;
    random initial particle velocities and perturbed populations."""
    w = preset(name)
    frac = float(np.prod(n)) / float(np.prod(w.n))
    npart = int(round(w.n_particles * frac))
    X, D, R = sample_particles(n, npart, w.diameter, w.density_ratio, w.band, seed)
    U = velocities(npart, w.d, seed=seed + 1, scale=u_scale) if u_scale else None
    _, _, wq, _ = lattice(w.q)
    f0 = populations(wq, tuple(reversed(n)), seed=seed + 2, eps=f0_eps) if f0_eps else None
    return dict(q=w.q, n=n, periodic=w.periodic, tau=w.tau, width=w.delta_width, implicit=True,
                X=X, U=U, D=D, R=R, f0=f0, gravity=w.gravity, kn=w.kn, e=w.restitution)


LONG = [
    # the 96^3 D3Q19 adjoint configuration's density (20k particles of d 0.5,
    # ratio 2, top half), tau 0.7, walls, 4-point kernel, on 24^3: 312 particles
    ("c5_shape_24cube", dict(name="c5", n=(24, 24, 24), seed=81), {}),
    # the 2048^2 benchmark workload's density (d ~ U[0.3, 0.8], ratio 2.5, top 60 %),
    # tau 0.6, walls, 4-point, on 128^2 (1953 particles), in the benchmark's launch
    # configuration: cell list kept for 10 steps, overlap on
    ("c2_shape_128sq_bench_launch", dict(name="c2", n=(128, 128), seed=82),
     dict(rebin_every=10, overlap="on")),
]


@pytest.mark.parametrize("name,case,gpu", LONG, ids=[c[0] for c in LONG])
def test_parity_fp64_1000_steps(name, case, gpu):
    """FP64 against the oracle after 1000 steps, element by element, at the 1e-10 bar."""
    c = _workload_case(**case)
    got, ref = run_both(c, 1000, **gpu)
    e = assert_parity(got, ref, c["X"])
    print(name, ref.np, e)
