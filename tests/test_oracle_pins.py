"""Pins of the FP64 oracle against closed forms, invariants and the paper's tables.

Each test checks a fact fixed by the paper or by the mathematics, chosen so that
a plausible slip in the oracle (a dropped term, a wrong sign, a transposed index)
fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, lattice, phi
from oracle import units
from paper_1407_6704_gb300.inputs import populations, sample_particles, velocities
from tests.conftest import read_golden

LATTICES = [9, 15, 19]


# --- velocity sets, Eq. (1) -------------------------------------------------------------
@pytest.mark.parametrize("q", LATTICES)
def test_lattice_isotropy(q):
    """Weights and velocities satisfy the moment identities every BGK lattice needs:
    sum w = 1, sum w e = 0, sum w e e = I/3, sum w e e e e = (dd + dd + dd)/9."""
    d, e, w, opp = lattice(q)
    e = e[:, :d].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-15
    m2 = np.einsum("a,ai,aj->ij", w, e, e)
    assert np.abs(m2 - np.eye(d) / 3.0).max() < 1e-15
    m4 = np.einsum("a,ai,aj,ak,al->ijkl", w, e, e, e, e)
    I = np.eye(d)
    ref = (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
           + np.einsum("il,jk->ijkl", I, I)) / 9.0
    assert np.abs(m4 - ref).max() < 1e-15
    for a in range(q):
        assert np.all(e[opp[a]] == -e[a])


def test_d3q15_weights_match_paper():
    """Section 2.1: w0 = 2/9, 1/9 for the six axis links, 1/72 for the eight corners."""
    d, e, w, _ = lattice(15)
    assert w[0] == 2.0 / 9.0
    assert np.all(w[1:7] == 1.0 / 9.0) and np.all(np.abs(e[1:7]).sum(1) == 1)
    assert np.all(w[7:] == 1.0 / 72.0) and np.all(np.abs(e[7:]).sum(1) == 3)


# --- delta kernel, Eqs. (10)-(11) --------------------------------------------------------
def test_cosine_kernel_values():
    """Eq. (11) at a few points: 1/2 at 0, 1/4 at +-1, 0 at and beyond +-2."""
    assert phi(4, 0.0) == pytest.approx(0.5, abs=1e-16)
    assert phi(4, 1.0) == pytest.approx(0.25, abs=1e-16)
    assert phi(4, -1.0) == pytest.approx(0.25, abs=1e-16)
    assert phi(4, 2.0) == pytest.approx(0.0, abs=1e-16)
    assert phi(4, 2.5) == 0.0
    assert phi(4, 0.5) == pytest.approx(0.25 * (1 + math.cos(math.pi / 4)), abs=1e-16)
    assert phi(2, 0.25) == 0.75 and phi(2, 1.5) == 0.0


@pytest.mark.parametrize("width", [2, 4])
def test_taps_partition_of_unity_and_centre(width):
    """Interior particles: weights sum to 1 (both kernels) and the stencil is the
    `width` nodes nearest X; the hat reproduces linear fields exactly; the cosine
    kernel puts half its weight on even and half on odd nodes."""
    o = Oracle(9, (40, 40), (0, 0), 0.8, delta_width=width)
    rng = np.random.default_rng(3)
    for X in rng.uniform(4.0, 36.0, 200):
        idx, w = o.taps(0, X)
        assert len(idx) == width
        assert abs(w.sum() - 1.0) < 1e-15
        centres = np.array(idx) + 0.5
        assert np.all(np.abs(centres - X) <= width / 2.0)
        if width == 2:
            assert abs((w * centres).sum() - X) < 1e-13
        else:
            # Eq. (11) splits evenly between even and odd nodes: phi(r) + phi(r + 2) = 1/2
            assert abs(w[0] + w[2] - 0.5) < 1e-15 and abs(w[1] + w[3] - 0.5) < 1e-15


@pytest.mark.parametrize("width", [2, 4])
def test_taps_at_walls_renormalised(width):
    o = Oracle(9, (10, 10), (0, 0), 0.8, delta_width=width)
    for X in [0.05, 0.3, 0.5, 0.9, 1.2, 9.95, 9.5, 8.8]:
        idx, w = o.taps(0, X)
        assert all(0 <= k < 10 for k in idx)
        assert abs(w.sum() - 1.0) < 1e-15


def test_taps_periodic_wrap():
    o = Oracle(9, (10, 10), (1, 1), 0.8, delta_width=4)
    idx, w = o.taps(0, 0.2)
    assert sorted(idx) == [0, 1, 8, 9]
    assert abs(w.sum() - 1.0) < 1e-15


# --- fluid: collide, stream, Guo forcing, walls -------------------------------------------
def _channel(tau, ny, gx, steps):
    o = Oracle(9, (1, ny), (1, 0), tau)
    F = np.zeros((2, ny, 1))
    F[0] = gx
    for _ in range(steps):
        o.f = o.stream(o.collide(o.f, F))
    rho, j = o.moments()
    u = (j[0, :, 0] + 0.5 * F[0, :, 0]) / rho[:, 0]
    return u


def test_poiseuille_exact_parabola():
    """Body-force-driven channel between halfway bounce-back walls: at
    tau = 1/2 + sqrt(3/16) the BGK steady state is the exact parabola
    u(y) = g/(2 nu) y (N - y), node y at k + 1/2."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    ny, gx = 12, 1e-6
    u = _channel(tau, ny, gx, 15000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    ue = gx / (2 * nu) * y * (ny - y)
    assert np.abs(u - ue).max() / ue.max() < 1e-9


def test_poiseuille_curvature_any_tau():
    """At any tau the steady profile has second differences -g/nu in the bulk."""
    tau = 0.8
    ny, gx = 12, 1e-6
    u = _channel(tau, ny, gx, 20000)
    nu = (tau - 0.5) / 3.0
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.abs(d2 + gx / nu).max() / (gx / nu) < 1e-7


@pytest.mark.parametrize("q,shape", [(9, (9, 13)), (19, (5, 6, 7)), (15, (5, 6, 7))])
def test_mass_conserved_by_collide_and_stream(q, shape):
    """Guo forcing adds no mass and halfway bounce-back loses none."""
    d, e, w, _ = lattice(q)
    n = tuple(reversed(shape))
    o = Oracle(q, n, (0,) * d, 0.7)
    f = populations(w, shape, seed=4, eps=0.05)
    F = 1e-3 * np.random.default_rng(5).uniform(-1, 1, (d,) + shape)
    f2 = o.stream(o.collide(f, F))
    assert abs(f2.sum() - f.sum()) / f.sum() < 1e-14


@pytest.mark.parametrize("q,shape", [(9, (9, 13)), (19, (5, 6, 7))])
def test_force_moment_identity(q, shape):
    """With u = (j + F/2)/rho and the Guo term, the post-collision momentum is
    j + F at every node (Eq. 8 and the modified flux of section 2.2)."""
    d, e, w, _ = lattice(q)
    n = tuple(reversed(shape))
    o = Oracle(q, n, (0,) * d, 0.63)
    f = populations(w, shape, seed=6, eps=0.05)
    F = 1e-3 * np.random.default_rng(7).uniform(-1, 1, (d,) + shape)
    fs = o.collide(f, F)
    e = e[:, :d].astype(float)
    j = np.einsum("ak,a...->k...", e, f)
    js = np.einsum("ak,a...->k...", e, fs)
    assert np.abs(js - (j + F)).max() < 1e-15
    assert np.abs(fs.sum(0) - f.sum(0)).max() < 1e-15


def test_stream_is_a_permutation():
    """Pull streaming with bounce-back moves every stored value exactly once."""
    d, e, w, _ = lattice(19)
    o = Oracle(19, (4, 3, 5), (1, 0, 0), 0.7)
    fs = np.arange(19 * 60, dtype=np.float64).reshape(19, 5, 3, 4)
    f = o.stream(fs)
    assert np.array_equal(np.sort(f.ravel()), np.sort(fs.ravel()))


# --- particle coupling, Eqs. (4)-(9), (12)-(13) -----------------------------------------
def _periodic_cloud(q=9, n=(24, 20), npart=40, seed=11, gravity=None, width=4, implicit=True):
    d = len(n)
    X, dia, rr = sample_particles(n, npart, (0.3, 0.8), (1.5, 3.0), band=(0.0, 1.0), seed=seed)
    U = velocities(npart, d, seed=seed + 1, scale=2e-3)
    _, _, w, _ = lattice(q)
    shape = tuple(reversed(n))
    f0 = populations(w, shape, seed=seed + 2, eps=1e-3)
    g = gravity if gravity is not None else (0.0,) * d
    return Oracle(q, n, (1,) * d, 0.7, delta_width=width, implicit_drag=implicit, gravity=g,
                  x0=X, u0=U, diameter=dia, density_ratio=rr, f0=f0)


def _mass(o):
    if o.d == 2:
        return o.rr * np.pi * o.dia ** 2 / 4.0
    return o.rr * np.pi * o.dia ** 3 / 6.0


@pytest.mark.parametrize("q,n", [(9, (24, 20)), (19, (10, 9, 8))])
@pytest.mark.parametrize("implicit", [True, False])
def test_momentum_exchange_balances(q, n, implicit):
    """Periodic box: the fluid gains exactly the spread force, sum F = -sum F_fpi
    (the kernel is a partition of unity), and with gravity the total
    fluid + particle momentum grows by exactly sum m (1 - 1/rho_r) g per step;
    contact pairs cancel."""
    d = len(n)
    grav = (0.0,) * (d - 1) + (-1e-4,)
    o = _periodic_cloud(q, n, npart=30, gravity=grav, implicit=implicit)
    m = _mass(o)
    buoy = (m * (1 - 1 / o.rr)).sum() * np.array(grav)
    for _ in range(5):
        _, j0 = o.moments()
        P0 = (m[:, None] * o.U).sum(0)
        J0 = j0.reshape(d, -1).sum(1)
        o.step(1)
        _, j1 = o.moments()
        J1 = j1.reshape(d, -1).sum(1)
        P1 = (m[:, None] * o.U).sum(0)
        Fsum = o.F.reshape(d, -1).sum(1)
        # absolute round-off of a sum over every population of the box
        tol = 64 * np.finfo(float).eps * o.f.sum() * (1 if d == 2 else 2)
        assert np.abs(Fsum).max() > 1e3 * tol
        assert np.abs(J1 - J0 - Fsum).max() < tol
        assert np.abs(Fsum + o.f_fpi.sum(0)).max() < 1e-12 * np.abs(o.F).sum()
        assert np.abs((J1 + P1) - (J0 + P0) - buoy).max() < tol


def test_literal_bounce_back_equals_closed_form():
    """The Q-direction sum of Eqs. (6)-(7) equals 2 (rho_l U - j_l) (the reading of
    Eq. 7); the oracle records the largest deviation."""
    o = _periodic_cloud(19, (10, 9, 8), npart=25)
    o.step(3)
    assert o.diag[0] < 1e-15


@pytest.mark.parametrize("implicit", [True, False])
def test_particle_update_satisfies_translation_law(implicit):
    """Eq. (13) discretised: m (U' - U) = m (1 - 1/rho_r) g + F_fpi + F_c, with the
    force density evaluated at U' (implicit) or U (explicit); X' = X + U'."""
    o = _periodic_cloud(9, (24, 20), npart=40, gravity=(0.0, -1e-4), implicit=implicit)
    m = _mass(o)
    for i in range(o.np):
        Xn, Un, g, Fc, dev, esc = o.particle_update(i)
        Ap = np.pi * o.dia[i] ** 2 / 4
        lhs = m[i] * (Un - o.U[i])
        rhs = m[i] * (1 - 1 / o.rr[i]) * np.array([0.0, -1e-4]) - Ap * g + Fc
        assert np.abs(lhs - rhs).max() < 1e-17 + 1e-12 * np.abs(rhs).max()
        fl = o.interp_pops(o.X[i])
        rho_l = fl.sum()
        j_l = (o.e[:, :2].T * fl).sum(1)
        Ub = Un if implicit else o.U[i]
        assert np.abs(g - 2 * (rho_l * Ub - j_l)).max() < 1e-15
        Xw = o.X[i] + Un
        Xw = np.where(Xw < 0, Xw + np.array(o.n[:2]), Xw)
        Xw = np.where(Xw >= np.array(o.n[:2]), Xw - np.array(o.n[:2]), Xw)
        assert np.abs(Xn - Xw).max() < 1e-14


def test_interpolation_of_uniform_state_is_exact():
    """Eq. (4) with any tap set reproduces a uniform population field exactly."""
    o = Oracle(19, (12, 12, 12), (0, 0, 0), 0.7, delta_width=4)
    for X in [(0.3, 5.5, 11.9), (6.0, 6.0, 6.0), (11.2, 0.1, 3.3)]:
        fl = o.interp_pops(X)
        assert np.abs(fl - o.w).max() < 1e-16


def test_sampled_evaluation_matches_full_step():
    """The per-cell and per-particle evaluators used for large lattices agree with
    a full oracle step (they are different code paths of the same definition)."""
    n = (20, 14)
    X, dia, rr = sample_particles(n, 60, (0.3, 0.8), 2.5, band=(0.3, 1.0), seed=21)
    _, _, w, _ = lattice(9)
    f0 = populations(w, (14, 20), seed=22, eps=1e-3)
    mk = lambda: Oracle(9, n, (0, 0), 0.6, delta_width=4, gravity=(0, -1e-5), x0=X,
                        u0=velocities(60, 2, 23, 1e-3), diameter=dia, density_ratio=rr, f0=f0)
    ref, smp = mk(), mk()
    ref.step(1)
    for cell in [0, 19, 77, 140, 200, 279]:
        assert np.abs(smp.force_at_cell(cell) - ref.F.reshape(2, -1)[:, cell]).max() < 1e-18
        post = smp.cell_after_step(cell)
        assert np.abs(post - ref.f.reshape(9, -1)[:, cell]).max() < 1e-16
    for i in [0, 7, 59]:
        Xn, Un, g, Fc, _, _ = smp.particle_update(i)
        assert np.array_equal(Xn, ref.X[i]) and np.array_equal(Un, ref.U[i])


# --- contacts ------------------------------------------------------------------------------
def test_pair_contact_closed_form():
    """Two overlapping particles: F = (kn delta - gamma v_n) n, with
    gamma = 2 beta sqrt(m_eff kn), beta = -ln e / sqrt(pi^2 + ln^2 e)."""
    X = np.array([[5.0, 5.0], [5.0 + 0.4 * 0.6, 5.0 + 0.4 * 0.8]])
    U = np.array([[0.0, 0.0], [-3e-3, -4e-3]])  # approaching along the normal at 5e-3
    dia = np.array([0.5, 0.6])
    rr = np.array([2.0, 3.0])
    o = Oracle(9, (10, 10), (0, 0), 0.8, kn=1e-2, restitution=0.9, x0=X, u0=U, diameter=dia,
               density_ratio=rr)
    F0 = o.contact_force(0)
    F1 = o.contact_force(1)
    delta = 0.55 - 0.4
    m0, m1 = 2.0 * np.pi * 0.25 / 4, 3.0 * np.pi * 0.36 / 4
    meff = m0 * m1 / (m0 + m1)
    beta = -math.log(0.9) / math.sqrt(math.pi ** 2 + math.log(0.9) ** 2)
    gamma = 2 * beta * math.sqrt(meff * 1e-2)
    nvec = np.array([-0.6, -0.8])  # from particle 1 to particle 0
    vn = -5e-3  # (U0 - U1) . n < 0: approaching
    expect = (1e-2 * delta - gamma * vn) * nvec
    assert np.abs(F0 - expect).max() < 1e-16
    assert np.array_equal(F1, -F0)


def test_wall_contact_closed_form():
    o = Oracle(9, (10, 10), (0, 0), 0.8, x0=[[0.2, 9.85]], u0=[[-1e-3, 2e-3]], diameter=[0.5],
               density_ratio=[2.0])
    F = o.contact_force(0)
    m = 2.0 * np.pi * 0.25 / 4
    beta = -math.log(0.9) / math.sqrt(math.pi ** 2 + math.log(0.9) ** 2)
    gw = 2 * beta * math.sqrt(m * 1e-2)
    assert F[0] == pytest.approx(1e-2 * 0.05 - gw * (-1e-3), rel=1e-14)
    assert F[1] == pytest.approx(-(1e-2 * 0.1 - gw * (-2e-3)), rel=1e-14)


def test_contact_forces_cancel_in_pairs():
    o = _periodic_cloud(9, (12, 10), npart=60, seed=31)
    # squeeze the cloud so that many pairs overlap
    o.X[:] = 6.0 + 0.35 * (o.X - 6.0)
    F = np.array([o.contact_force(i) for i in range(o.np)])
    assert np.count_nonzero(np.abs(F).sum(1)) > 10
    assert np.abs(F.sum(0)).max() < 1e-15


def test_restitution_of_head_on_collision():
    """Two equal particles collide head on in vacuum (contact force only, symplectic
    Euler, small kn): the separation speed over the approach speed is e."""
    for e_target in (0.9, 0.5):
        X = np.array([[4.0, 5.0], [5.2, 5.0]])
        U = np.array([[2e-4, 0.0], [-2e-4, 0.0]])
        o = Oracle(9, (10, 10), (1, 1), 0.8, kn=1e-5, restitution=e_target, x0=X, u0=U,
                   diameter=[1.0, 1.0], density_ratio=[2.0, 2.0])
        m = 2.0 * np.pi / 4
        for _ in range(40000):
            F0 = o.contact_force(0)
            o.U[0] += F0 / m
            o.U[1] -= F0 / m
            o.X += o.U
            if o.U[0, 0] < 0 and np.linalg.norm(o.X[0] - o.X[1]) > 1.0:
                break
        ratio = (o.U[1, 0] - o.U[0, 0]) / 4e-4
        assert ratio == pytest.approx(e_target, rel=2e-2)


# --- Stokes law and Table 2 ------------------------------------------------------------------
def test_table2_stokes_column_and_time_step():
    """Eq. (17) with Table 1 properties reproduces Table 2's Stokes column, and the
    lattice viscosity (tau - 1/2)/3 reproduces its time-step column, at the
    printed precision."""
    props = {k: float(v) for k, v in read_golden("table1_properties.txt")}
    for hd, v_stokes, v_num, tau, dt in read_golden("table2_settling.txt"):
        dp = props["h"] / float(hd)
        vs = units.stokes_velocity(props["rho_p"], props["rho_f"], dp, props["g"], props["mu"])
        assert -vs == pytest.approx(float(v_stokes), abs=0.006 * abs(float(v_stokes)))
        step = units.time_step(float(tau), props["h"], props["mu"], props["rho_f"])
        assert step == pytest.approx(float(dt), abs=0.6e-4)


def test_settling_force_balance_and_drag_closed_form():
    """Single particle of Table 2 (h/d = 4, tau = 0.65, D3Q15) in a 10x10x50 cavity:
    once steady, the reaction force balances the reduced weight (Eq. 13 with zero
    acceleration), and the slip velocity equals m (1 - 1/rho_r) g / (2 A_p rho_l)."""
    props = {k: float(v) for k, v in read_golden("table1_properties.txt")}
    tau, hd = 0.65, 4.0
    dp = props["h"] / hd
    dt = units.time_step(tau, props["h"], props["mu"], props["rho_f"])
    glu = units.accel_to_lattice(props["g"], dt, props["h"])
    rr = props["rho_p"] / props["rho_f"]
    o = Oracle(15, (10, 10, 50), (0, 0, 0), tau, delta_width=4, gravity=(0, 0, -glu),
               x0=[[5.0, 5.0, 49.0]], diameter=[dp / props["h"]], density_ratio=[rr])
    o.step(600)
    m = rr * np.pi * (dp / props["h"]) ** 3 / 6
    Ap = np.pi * (dp / props["h"]) ** 2 / 4
    weight = m * (1 - 1 / rr) * glu
    assert o.f_fpi[0, 2] == pytest.approx(weight, rel=1e-3)
    fl = o.interp_pops(o.X[0])
    slip = o.U[0, 2] - (o.e[:, 2] * fl).sum() / fl.sum()
    assert slip == pytest.approx(-weight / (2 * Ap * fl.sum()), rel=1e-3)
