"""The persistent ensemble kernel: one cooperative launch runs every phase of the
coupled step for all members, with grid-wide barriers between the phases.

- In deterministic mode a member advanced by the persistent kernel must equal,
  bit for bit, the same simulation advanced on its own (the kernel runs the same
  device functions), for whole graph launches (10 steps), direct launches and
  both, with cell lists rebuilt every step or kept (each member its own period),
  and with members stepped on their own in between.
- With atomic spreading the members are compared with the FP64 oracle.
- The grid barrier's bounded wait: a CTA that skips its arrival makes every wait
  give up after the limit, and the host reads PIBM_ETIMEOUT; nothing hangs.
"""
import time

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


# (extents, periodic, tau, particles, rebin_every)
SPECS = [
    ((64, 64), (0, 0), 0.8, 100, 1),
    ((97, 53), (1, 0), 0.6, 150, 5),
    ((40, 120), (0, 0), 0.95, 60, 1),
    ((150, 150), (0, 0), 0.55, 400, 10),
    ((33, 200), (0, 1), 0.7, 90, 3),
    ((256, 96), (0, 0), 0.65, 700, 1),
    ((48, 48), (0, 0), 0.75, 0, 1),  # no particles
]


def _make(spec, seed, precision="fp32", deterministic=True, width=4):
    from paper_1407_6704_gb300.pibm import Pibm

    n, per, tau, npart, rebin = spec
    kw = {}
    if npart:
        X, dia, rr = sample_particles(n, npart, (0.3, 0.8), (1.5, 3.0), band=(0.4, 1.0),
                                      seed=seed)
        kw = dict(x0=X, diameter=dia, density_ratio=rr)
    return Pibm("d2q9", n, per, tau, gravity=(0.0, -1e-4), delta_width=width,
                precision=precision, deterministic=deterministic, rebin_every=rebin, **kw)


def _state(sim):
    return sim.read("pop", "x", "u")


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


def _pair(specs, seed, **kw):
    return ([_make(s, seed + i, **kw) for i, s in enumerate(specs)],
            [_make(s, seed + i, **kw) for i, s in enumerate(specs)])


def test_persistent_mode_is_chosen_for_qualifying_members():
    from paper_1407_6704_gb300.pibm import Ensemble, Pibm

    a, _ = _pair(SPECS[:3], 10)
    with Ensemble(a) as ens:
        info = ens.info()
        assert info["persistent"] == 1 and info["grid"] > 0 and info["cells_per_item"] == 1024
        assert 1 <= info["ctas_per_sm"] <= info["max_ctas_per_sm"]
    other = Pibm("d3q19", (12, 12, 12), (0, 0, 0), 0.7, gravity=(0, 0, -1e-4))
    with Ensemble([a[0], other]) as ens:  # a 3D member: branch mode
        assert ens.info()["persistent"] == 0
    for s in a + [other]:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("steps", [10, 7, 23])
def test_persistent_equals_members_stepped_alone(precision, steps):
    from paper_1407_6704_gb300.pibm import Ensemble

    ens_members, alone = _pair(SPECS, 100, precision=precision)
    with Ensemble(ens_members) as ens:
        assert ens.info()["persistent"] == 1
        ens.step(steps)
        assert ens.status() == 0
        assert ens.launch_count() == -(-steps // 10)
    for sim in alone:
        sim.step(steps)
    for i, (a, b) in enumerate(zip(ens_members, alone)):
        assert _same(_state(a), _state(b)), i
    for s in ens_members + alone:
        s.close()


def test_persistent_with_members_stepped_alone_in_between():
    """Members stepped on their own change parity and cell-list phase; the kernel's
    phase table is reloaded from the handles (kept cell lists included)."""
    from paper_1407_6704_gb300.pibm import Ensemble

    ens_members, alone = _pair(SPECS, 200)
    extra = [0, 3, 0, 7, 1, 0, 2]
    with Ensemble(ens_members) as ens:
        ens.step(4)
        assert ens.status() == 0
        for sim, k in zip(ens_members, extra):
            if k:
                sim.step(k)
        ens.step(13)
        ens.step(10)
        assert ens.status() == 0
    for sim, k in zip(alone, extra):
        sim.step(27 + k)
    for i, (a, b) in enumerate(zip(ens_members, alone)):
        assert _same(_state(a), _state(b)), i
    for s in ens_members + alone:
        s.close()


@pytest.mark.parametrize("width", [2, 4])
def test_persistent_launch_shapes_give_the_same_results(width):
    from paper_1407_6704_gb300.pibm import Ensemble

    ref_members, _ = _pair(SPECS[:4], 300, width=width)
    with Ensemble(ref_members) as ens:
        ens.step(12)
        assert ens.status() == 0
    ref = [_state(s) for s in ref_members]
    info = None
    for per_sm, cpi in [(1, 256), (2, 4096), (0, 512)]:
        members, _ = _pair(SPECS[:4], 300, width=width)
        with Ensemble(members) as ens:
            info = ens.info()
            ens.configure(min(per_sm, info["max_ctas_per_sm"]), cpi)
            ens.step(12)
            assert ens.status() == 0
        for i, s in enumerate(members):
            assert _same(_state(s), ref[i]), (per_sm, cpi, i)
            s.close()
    for s in ref_members:
        s.close()


def test_persistent_autotune_keeps_the_arithmetic():
    from paper_1407_6704_gb300.pibm import Ensemble

    ens_members, alone = _pair(SPECS[:4], 400)
    with Ensemble(ens_members) as ens:
        choice = ens.autotune(steps_per_candidate=10)
        info = ens.info()
        assert choice["candidates"] == 5 * info["max_ctas_per_sm"]
        assert info["ctas_per_sm"] == choice["ctas_per_sm"]
        assert info["cells_per_item"] == choice["cells_per_item"]
        ens.step(5)
        assert ens.status() == 0
    total = choice["candidates"] * 20 + 5
    for sim in alone:
        sim.step(total)
    for i, (a, b) in enumerate(zip(ens_members, alone)):
        assert _same(_state(a), _state(b)), i
    for s in ens_members + alone:
        s.close()


def test_mode_switch_between_persistent_and_branches():
    from paper_1407_6704_gb300.pibm import Ensemble

    specs = [s for s in SPECS if s[4] == 1]  # branch mode needs every-step cell lists
    ens_members, alone = _pair(specs, 500)
    with Ensemble(ens_members) as ens:
        ens.step(6)
        ens.set_mode(False)
        assert ens.info()["persistent"] == 0
        ens.step(6)
        ens.set_mode(True)
        ens.step(11)
        assert ens.status() == 0
    for sim in alone:
        sim.step(23)
    for i, (a, b) in enumerate(zip(ens_members, alone)):
        assert _same(_state(a), _state(b)), i
    for s in ens_members + alone:
        s.close()


ORACLE_SPECS = [  # (extents, periodic, tau, particles, rebin_every)
    ((48, 40), (0, 0), 0.8, 60, 1),
    ((40, 36), (1, 0), 0.6, 50, 4),
    ((72, 30), (0, 0), 0.7, 70, 1),
]


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_persistent_members_against_the_oracle(precision, bar):
    """Members with atomic spreading advanced by the persistent kernel, each
    compared element by element with the FP64 oracle run of the same inputs: the
    velocity field and the particles at the bar (relative max-norm), and in FP64
    also populations and density (1e-8 against their deviation from rest)."""
    from oracle.oracle import Oracle, lattice
    from paper_1407_6704_gb300.inputs import populations, velocities
    from paper_1407_6704_gb300.pibm import Ensemble, Pibm

    steps = 40
    sims, refs, cases = [], [], []
    for i, (n, per, tau, npart, rebin) in enumerate(ORACLE_SPECS):
        X, dia, rr = sample_particles(n, npart, (0.3, 0.8), (1.5, 3.0), band=(0.3, 1.0),
                                      seed=600 + i)
        U = velocities(npart, 2, seed=610 + i, scale=1e-3)
        f0 = populations(lattice(9)[2], tuple(reversed(n)), seed=620 + i, eps=1e-3)
        kw = dict(gravity=(0.0, -1e-4), delta_width=4, x0=X, u0=U, diameter=dia,
                  density_ratio=rr, f0=f0)
        sims.append(Pibm("d2q9", n, per, tau, precision=precision, rebin_every=rebin, **kw))
        ref = Oracle(9, n, per, tau, **kw)
        ref.step(steps)
        refs.append(ref)
        cases.append(X)
    with Ensemble(sims) as ens:
        assert ens.info()["persistent"] == 1
        ens.step(steps)
        assert ens.status() == 0
    for sim, ref, X0 in zip(sims, refs, cases):
        got = sim.read("pop", "rho", "j", "x", "u")
        sim.close()
        rho_r, j_r = ref.moments()
        w = ref.w.reshape((-1,) + (1,) * len(ref.shape))
        e = {"u": np.abs(got["j"] / got["rho"] - j_r / rho_r).max() / np.abs(j_r / rho_r).max(),
             "x": np.abs(got["x"] - ref.X).max() / np.abs(ref.X - X0).max(),
             "up": np.abs(got["u"] - ref.U).max() / np.abs(ref.U).max()}
        bars = dict.fromkeys(e, bar)
        if precision == "fp64":
            e["dpop"] = np.abs(got["pop"] - ref.f).max() / np.abs(ref.f - w).max()
            e["drho"] = np.abs(got["rho"] - rho_r).max() / np.abs(rho_r - 1.0).max()
            bars.update(dpop=1e-8, drho=1e-8)
        print("persistent member", precision, e)
        assert all(e[k] <= bars[k] for k in e), (precision, e)


def test_grid_barrier_passes_and_times_out():
    """The barrier of the persistent kernel, alone: all CTAs arriving pass any
    number of barriers; a CTA that does not arrive (host-set skip flag) makes
    every wait give up after the limit, and the launch returns PIBM_ETIMEOUT."""
    import torch
    from paper_1407_6704_gb300._lib import PIBM_EINVAL, PIBM_ETIMEOUT
    from paper_1407_6704_gb300.pibm import grid_barrier_test

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert grid_barrier_test(1, -1, 100, 0.5) == (0, 100)
    assert grid_barrier_test(sms, -1, 1000, 1.0) == (0, 1000)
    assert grid_barrier_test(2 * sms, -1, 200, 1.0) == (0, 200)
    t0 = time.perf_counter()
    assert grid_barrier_test(1, 0, 1, 0.2) == (PIBM_ETIMEOUT, 0)  # the one CTA skips
    assert grid_barrier_test(sms, sms // 2, 5, 0.2) == (PIBM_ETIMEOUT, 0)
    assert time.perf_counter() - t0 < 10.0
    st, _ = grid_barrier_test(10 ** 6, -1, 1, 0.2)  # cannot all be resident: refused
    assert st == PIBM_EINVAL


def test_ensemble_barrier_timeout_is_reported():
    """Fault injection on the host: one CTA of the persistent ensemble kernel does
    not arrive at its first barrier. Every wait gives up after 0.2 s, the kernel
    returns, the status is PIBM_ETIMEOUT, and later launches return at once."""
    from paper_1407_6704_gb300._lib import PIBM_ETIMEOUT
    from paper_1407_6704_gb300.pibm import Ensemble

    members, _ = _pair(SPECS[:3], 700)
    ens = Ensemble(members)
    ens.step(2)
    assert ens.status() == 0
    ens.inject_skip(0, 0.2)
    t0 = time.perf_counter()
    ens.step(1)
    assert ens.status() == PIBM_ETIMEOUT
    ens.step(20)  # returns at once: the abort word is set
    assert ens.status() == PIBM_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    ens.close()
    for s in members:
        s.close()
