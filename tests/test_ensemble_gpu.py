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
