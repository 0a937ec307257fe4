"""Ensembles of independent simulations and the stream-collide autotuner.

In deterministic mode every member's result is bitwise reproducible, so a member
advanced inside an ensemble (one graph launch per two steps for all members)
must equal the same simulation advanced on its own, bit for bit; so must a
simulation whose collide block shape was autotuned.
"""
import numpy as np
import pytest

from paper_1407_6704_gb300.inputs import sample_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


SPECS = [  # (lattice, extents, periodic, tau, particles, precision)
    ("d2q9", (64, 64), (0, 0), 0.8, 100, "fp32"),
    ("d2q9", (97, 53), (1, 0), 0.6, 150, "fp64"),
    ("d2q9", (40, 120), (0, 0), 0.95, 60, "fp16"),
    ("d3q19", (20, 18, 16), (0, 0, 0), 0.7, 80, "fp32"),
    ("d2q9", (150, 150), (0, 0), 0.55, 400, "fp32"),
]


def _make(spec, seed):
    from paper_1407_6704_gb300.pibm import Pibm

    lat, n, per, tau, npart, prec = spec
    d = len(n)
    X, dia, rr = sample_particles(n, npart, (0.3, 0.8), (1.5, 3.0), band=(0.4, 1.0), seed=seed)
    g = (0.0,) * (d - 1) + (-1e-4,)
    return Pibm(lat, n, per, tau, gravity=g, delta_width=4 if seed % 2 else 2, precision=prec,
                deterministic=True, x0=X, diameter=dia, density_ratio=rr)


def _state(sim):
    return sim.read("pop", "x", "u")


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("steps", [10, 7])
def test_ensemble_equals_members_stepped_alone(steps):
    from paper_1407_6704_gb300.pibm import Ensemble

    ens_members = [_make(s, 100 + i) for i, s in enumerate(SPECS)]
    alone = [_make(s, 100 + i) for i, s in enumerate(SPECS)]
    with Ensemble(ens_members) as ens:
        ens.step(steps)
        assert ens.status() == 0
    for sim in alone:
        sim.step(steps)
    for a, b in zip(ens_members, alone):
        assert _same(_state(a), _state(b))
    for s in ens_members + alone:
        s.close()


def test_member_stepped_between_ensemble_steps():
    from paper_1407_6704_gb300.pibm import Ensemble

    ens_members = [_make(s, 200 + i) for i, s in enumerate(SPECS[:3])]
    alone = [_make(s, 200 + i) for i, s in enumerate(SPECS[:3])]
    with Ensemble(ens_members) as ens:
        ens.step(4)
        ens.status()
        ens_members[1].step(1)  # parity of one member changes: the graph is rebuilt
        ens.step(4)
        assert ens.status() == 0
    for i, sim in enumerate(alone):
        sim.step(9 if i == 1 else 8)
    for a, b in zip(ens_members, alone):
        assert _same(_state(a), _state(b))
    for s in ens_members + alone:
        s.close()


@pytest.mark.parametrize("spec", [SPECS[0], SPECS[2], SPECS[3]], ids=["fp32-2d", "fp16-2d", "fp32-3d"])
def test_autotune_keeps_the_state_and_the_results(spec):
    tuned, plain = _make(spec, 300), _make(spec, 300)
    tuned.step(3)
    plain.step(3)
    before = _state(tuned)
    bx, by = tuned.autotune()
    assert bx * by <= 1024 and bx >= 32
    assert _same(before, _state(tuned))
    tuned.step(6)
    plain.step(6)
    assert _same(_state(tuned), _state(plain))
    tuned.close()
    plain.close()


ORACLE_SPECS = [  # (lattice, extents, periodic, tau, particles, precision, bar)
    ("d2q9", (48, 40), (0, 0), 0.8, 60, "fp64", 1e-10),
    ("d2q9", (40, 36), (1, 0), 0.6, 50, "fp32", 1e-4),
    ("d2q9", (64, 32), (0, 0), 0.7, 70, "fp16", 1e-3),
    ("d3q19", (14, 12, 16), (0, 0, 0), 0.7, 40, "fp32", 1e-4),
]


def test_ensemble_members_against_the_oracle():
    """Members of different lattices and storage modes advanced together (one graph
    launch per two steps), each compared element by element with the FP64 oracle
    run of the same inputs: FP64 member at the FP64 bar (1e-10 relative on every
    field, 1e-8 for populations and density against their deviation from rest);
    FP32 at 1e-4 and FP16 at 1e-3 (relative max-norm on the velocity field and
    the particles)."""
    from oracle.oracle import Oracle, lattice
    from paper_1407_6704_gb300.inputs import populations, velocities
    from paper_1407_6704_gb300.pibm import Ensemble, Pibm

    steps = 40
    sims, refs, cases = [], [], []
    for i, (lat, n, per, tau, npart, prec, bar) in enumerate(ORACLE_SPECS):
        q = {"d2q9": 9, "d3q19": 19}[lat]
        d = len(n)
        X, dia, rr = sample_particles(n, npart, (0.3, 0.8), (1.5, 3.0), band=(0.3, 1.0),
                                      seed=300 + i)
        U = velocities(npart, d, seed=310 + i, scale=1e-3)
        f0 = populations(lattice(q)[2], tuple(reversed(n)), seed=320 + i, eps=1e-3)
        kw = dict(gravity=(0.0,) * (d - 1) + (-1e-4,), delta_width=4, x0=X, u0=U, diameter=dia,
                  density_ratio=rr, f0=f0)
        sims.append(Pibm(lat, n, per, tau, precision=prec, **kw))
        ref = Oracle(q, n, per, tau, **kw)
        ref.step(steps)
        refs.append(ref)
        cases.append((prec, bar, X))
    with Ensemble(sims) as ens:
        ens.step(steps)
        assert ens.status() == 0
    for sim, ref, (prec, bar, X0) in zip(sims, refs, cases):
        got = sim.read("pop", "rho", "j", "x", "u")
        sim.close()
        rho_r, j_r = ref.moments()
        w = ref.w.reshape((-1,) + (1,) * len(ref.shape))
        e = {"u": np.abs(got["j"] / got["rho"] - j_r / rho_r).max() / np.abs(j_r / rho_r).max(),
             "x": np.abs(got["x"] - ref.X).max() / np.abs(ref.X - X0).max(),
             "up": np.abs(got["u"] - ref.U).max() / np.abs(ref.U).max()}
        bars = dict.fromkeys(e, bar)
        if prec == "fp64":
            e["dpop"] = np.abs(got["pop"] - ref.f).max() / np.abs(ref.f - w).max()
            e["drho"] = np.abs(got["rho"] - rho_r).max() / np.abs(rho_r - 1.0).max()
            bars.update(dpop=1e-8, drho=1e-8)
        print("ensemble member", prec, e)
        assert all(e[k] <= bars[k] for k in e), (prec, e)
