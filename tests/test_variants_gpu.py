"""GPU parity of the paper-faithful variants against the FP64 oracle: the 4-point
Lagrange interpolant (Eq. 5), the Hertz normal contact (Eq. 15) and DEM
sub-cycling, alone and combined, in FP64 (bar 1e-10, as for the default path)
and FP32 storage; plus the sub-cycling skin check and deterministic repeats.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from tests.test_parity_gpu import LAT, TOL, make_case, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


def run_variant(c, steps, precision="fp64", deterministic=False, **variant):
    from paper_1407_6704_gb300.pibm import Pibm

    kw = dict(delta_width=c["width"], gravity=c["gravity"], kn=c["kn"], restitution=c["e"],
              x0=c["X"], u0=c["U"], diameter=c["D"], density_ratio=c["R"], f0=c["f0"], **variant)
    ref = Oracle(c["q"], c["n"], c["periodic"], c["tau"], implicit_drag=c["implicit"], **kw)
    ref.step(steps)
    with Pibm(LAT[c["q"]], c["n"], c["periodic"], c["tau"], implicit=c["implicit"],
              precision=precision, deterministic=deterministic, **kw) as sim:
        sim.step(steps)
        got = sim.read("pop", "rho", "j", "x", "u")
        got["f_fpi"], got["f_c"] = sim.forces()
        got["status"] = sim.status()
        got["kernels"] = sim.kernels_per_step
    return got, ref


def check(got, ref, X0, tol=1e-10, tols=None):
    assert got["status"] == 0
    e = rel_errors(got, ref, X0)
    lim = dict(TOL, **(tols or {}))
    bad = {k: v for k, v in e.items() if not v <= lim.get(k, tol)}
    assert not bad, f"relative errors above the bar: {bad} (all: {e})"
    return e


LAGRANGE = [
    ("2d_walls_spread4", dict(q=9, n=(41, 33), periodic=(0, 0), tau=0.62, width=4, npart=90,
                              seed=31, f0_eps=1e-3, u_scale=2e-3, band=(0.0, 1.0)), 100),
    ("2d_periodic_x_spread2_explicit", dict(q=9, n=(35, 26), periodic=(1, 0), tau=0.8, width=2,
                                            npart=70, seed=32, implicit=False, f0_eps=1e-3,
                                            u_scale=1e-3, rr=(2.0, 3.0)), 100),
    ("3d_d3q19_walls", dict(q=19, n=(13, 11, 17), periodic=(0, 0, 0), tau=0.7, width=4, npart=60,
                            seed=33, f0_eps=1e-3, u_scale=1e-3, band=(0.0, 1.0)), 40),
    ("3d_d3q15_periodic_xy", dict(q=15, n=(12, 10, 14), periodic=(1, 1, 0), tau=0.75, width=2,
                                  npart=50, seed=34, f0_eps=1e-3, u_scale=1e-3), 40),
]


@pytest.mark.parametrize("name,kw,steps", LAGRANGE, ids=[c[0] for c in LAGRANGE])
def test_lagrange_interpolation_parity_fp64(name, kw, steps):
    c = make_case(**kw)
    got, ref = run_variant(c, steps, interp="lagrange4")
    print(name, check(got, ref, c["X"]))


def _dense(q, n, seed, npart, dia=(0.6, 0.9)):
    c = make_case(q=q, n=n, periodic=(0,) * len(n), tau=0.7, width=2 if q == 9 else 4,
                  npart=npart, seed=seed, dia=dia, rr=2.0, band=(0.25, 0.95), u_scale=2e-3, e=0.8)
    centre = np.array(n, dtype=float) / 2
    c["X"] = centre + 0.85 * (c["X"] - centre)
    return c


@pytest.mark.parametrize("q,n", [(9, (24, 20)), (19, (10, 9, 11))])
def test_hertz_contacts_parity_fp64(q, n):
    """A squeezed cloud released with the Hertz law (E = 0.05, nu = 0.3; walls
    E = 0.2, nu = 0.25), restitution 0.8."""
    c = _dense(q, n, 41, 160 if q == 9 else 120)
    got, ref = run_variant(c, 50, contact="hertz", young=0.05, poisson=0.3, wall_young=0.2,
                           wall_poisson=0.25)
    assert np.count_nonzero(np.abs(ref.Fc).sum(1)) >= 15
    print("hertz", q, check(got, ref, c["X"]))


@pytest.mark.parametrize("q,n,S,contact", [(9, (24, 20), 4, "hertz"), (9, (24, 20), 3, "linear"),
                                           (19, (10, 9, 11), 5, "hertz")])
def test_subcycled_dem_parity_fp64(q, n, S, contact):
    """S DEM sub-steps per fluid step: contacts and particle update S times with
    rho_l, j_l fixed, the averaged force density spread once."""
    c = _dense(q, n, 42, 160 if q == 9 else 120, dia=(0.5, 0.7))
    got, ref = run_variant(c, 40, contact=contact, young=0.3, substeps=S)
    assert np.count_nonzero(np.abs(ref.Fc).sum(1)) >= 10
    assert got["kernels"] == 11 + 2 * S
    print("substeps", S, contact, check(got, ref, c["X"]))


def test_all_variants_together_explicit_periodic():
    """Lagrange interpolation, Hertz contacts and sub-cycling in one run, explicit
    drag, a periodic axis."""
    c = make_case(q=9, n=(30, 24), periodic=(1, 0), tau=0.7, width=4, npart=150, seed=43,
                  implicit=False, dia=(0.4, 0.7), rr=(2.0, 3.0), band=(0.2, 0.9), u_scale=2e-3,
                  f0_eps=1e-3, e=0.7)
    c["X"][:, 1] = 12.0 + 0.8 * (c["X"][:, 1] - 12.0)
    got, ref = run_variant(c, 40, interp="lagrange4", contact="hertz", young=0.2, substeps=3)
    assert np.count_nonzero(np.abs(ref.Fc).sum(1)) >= 8
    print("all variants", check(got, ref, c["X"]))


@pytest.mark.parametrize("variant", [dict(interp="lagrange4"),
                                     dict(contact="hertz", young=0.3, substeps=4)],
                         ids=["lagrange", "hertz_substeps"])
def test_variants_in_fp32_storage(variant):
    """FP32 storage (populations as f - w, FP32 moments, FP32 particle increments,
    FP64 particle state and contacts) against the FP64 oracle: velocity field
    relative L2 and particle fields within 1e-4 after 100 steps."""
    c = _dense(9, (40, 34), 44, 200, dia=(0.5, 0.7))
    got, ref = run_variant(c, 100, precision="fp32", **variant)
    assert got["status"] == 0
    rho_r, j_r = ref.moments()
    ur, ug = j_r / rho_r, got["j"] / got["rho"]
    l2 = np.sqrt(((ug - ur) ** 2).sum() / (ur ** 2).sum())
    ex = np.abs(got["x"] - ref.X).max() / np.abs(ref.X - c["X"]).max()
    eu = np.abs(got["u"] - ref.U).max() / np.abs(ref.U).max()
    print("fp32", variant, l2, ex, eu)
    assert l2 < 1e-4 and ex < 1e-4 and eu < 1e-4


def test_subcycled_deterministic_mode_repeats_bitwise():
    c = _dense(9, (24, 20), 45, 160, dia=(0.5, 0.7))
    runs = [run_variant(c, 30, deterministic=True, contact="hertz", young=0.3, substeps=4)
            for _ in range(2)]
    check(runs[0][0], runs[0][1], c["X"])
    for k in ("pop", "x", "u", "f_fpi", "f_c"):
        assert np.array_equal(runs[0][0][k], runs[1][0][k]), k


def test_subcycling_reports_a_particle_leaving_its_cell_neighbourhood():
    """With sub-cycling, the contacts of a step come from the cell list of the
    step start, which holds every pair that can touch only while each particle
    moves less than (1 - largest diameter) / 2 within the step; a faster particle
    is reported as PIBM_EUNSTABLE (a host-side status; the kernels stay in
    bounds)."""
    from paper_1407_6704_gb300 import _lib
    from paper_1407_6704_gb300.pibm import Pibm

    with Pibm("d2q9", (32, 32), (1, 1), 0.8, delta_width=4, x0=[[16.0, 16.0], [5.0, 5.0]],
              u0=[[0.3, 0.0], [0.0, 0.0]], diameter=[0.6, 0.6], density_ratio=[50.0, 50.0],
              substeps=2) as sim:
        sim.step(1)
        assert sim.status() == _lib.PIBM_EUNSTABLE
    with Pibm("d2q9", (32, 32), (1, 1), 0.8, delta_width=4, x0=[[16.0, 16.0], [5.0, 5.0]],
              u0=[[0.1, 0.0], [0.0, 0.0]], diameter=[0.6, 0.6], density_ratio=[50.0, 50.0],
              substeps=2) as sim:
        sim.step(1)
        assert sim.status() == 0
