"""Pins of the oracle's paper-faithful variants: the 4-point Lagrange interpolant
(Eq. 5), the Hertz normal contact (Eq. 15) and DEM sub-cycling.

Each is checked against something other than its own formula: a library
interpolation routine and polynomial exactness for Eq. (5), the analytic
solution of an elastic Hertz impact (maximum overlap and contact time) for
Eq. (15), and the closed-form geometric recurrence of the sub-stepped velocity
update for the sub-cycling, plus momentum balance.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_1407_6704_gb300.inputs import populations, sample_particles, velocities


# --- Eq. (5): 4-point Lagrange interpolation ---------------------------------------------
def _lagrange_oracle(n, periodic):
    return Oracle(9, n, periodic, 0.7, delta_width=2, interp="lagrange4")


@pytest.mark.parametrize("periodic", [0, 1])
def test_lagrange_weights_match_library_interpolant(periodic):
    """sum_t w_t v_t equals scipy's polynomial interpolant through the four nodes
    (node t at index + 1/2; barycentric form) for random node values, anywhere
    on the axis, including the one-sided blocks next to a wall."""
    interpolate = pytest.importorskip("scipy.interpolate")
    o = _lagrange_oracle((11, 9), (periodic, periodic))
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(0.0, 11.0, 40), [0.0, 0.2, 0.5, 1.49, 9.6, 10.5, 10.99]])
    for X in xs:
        idx, w = o.interp_taps(0, X)
        assert len(idx) == 4
        v = rng.normal(size=4)
        first = int(math.floor(X - 0.5)) - 1
        if not periodic:
            first = min(max(first, 0), 11 - 4)
            assert idx == list(range(first, first + 4))
        nodes = np.arange(first, first + 4) + 0.5
        ref = interpolate.BarycentricInterpolator(nodes, v)(X)
        assert abs(np.dot(w, v) - ref) < 1e-12 * (1 + abs(ref))
        if periodic:
            assert idx == [k % 11 for k in range(first, first + 4)]


def test_lagrange_weights_at_nodes_are_unit_vectors():
    o = _lagrange_oracle((12, 12), (0, 0))
    for k in range(12):
        idx, w = o.interp_taps(1, k + 0.5)
        expect = np.array([1.0 if i == k else 0.0 for i in idx])
        assert np.abs(w - expect).max() < 1e-15


@pytest.mark.parametrize("q,n", [(9, (12, 10)), (19, (7, 6, 8))])
def test_lagrange_interpolation_reproduces_cubics(q, n):
    """Populations that are cubic polynomials of the node position (a different
    one per direction) are interpolated exactly by Eq. (4) with the tensor
    Lagrange weights of Eq. (5), also next to the walls."""
    d = len(n)
    o = Oracle(q, n, (0,) * d, 0.7, interp="lagrange4")
    rng = np.random.default_rng(8)
    coef = rng.normal(size=(q, d, 4))  # per direction: product of per-axis cubics

    def field(a, pos):
        out = 1.0
        for k in range(d):
            c = coef[a, k]
            out = out * (c[0] + c[1] * pos[k] + c[2] * pos[k] ** 2 + c[3] * pos[k] ** 3)
        return out

    grids = np.meshgrid(*[np.arange(nk) + 0.5 for nk in n], indexing="ij")
    f = np.empty((q,) + tuple(reversed(n)))
    for a in range(q):
        f[a] = field(a, grids).transpose()
    o.f = f
    pts = [rng.uniform(0.0, np.array(n)) for _ in range(20)]
    pts += [np.array([0.05] * d), np.array(n) - 0.05, np.array([0.3] + list(np.array(n[1:]) - 0.4))]
    for X in pts:
        fl = o.interp_pops(X)
        exp = np.array([field(a, X) for a in range(q)])
        assert np.abs(fl - exp).max() < 1e-10 * np.abs(exp).max()


def test_lagrange_differs_from_delta_kernel_and_keeps_spreading():
    """The Lagrange option changes only the interpolation: the spreading taps are
    still the cosine kernel of Eq. (11)."""
    a = Oracle(9, (12, 12), (0, 0), 0.7, delta_width=4, interp="lagrange4")
    b = Oracle(9, (12, 12), (0, 0), 0.7, delta_width=4)
    for X in (3.3, 5.9, 0.4):
        assert a.taps(0, X)[0] == b.taps(0, X)[0]
        assert np.array_equal(a.taps(0, X)[1], b.taps(0, X)[1])
        la, lb = a.interp_taps(0, X)[1], b.interp_taps(0, X)[1]
        assert la.shape != lb.shape or not np.allclose(la, lb)


# --- Eq. (15): Hertz normal contact --------------------------------------------------------
def _hertz_pair(v0, e, young=1e-2, poisson=0.3, dia=1.0, rr=2.0):
    X = np.array([[4.0, 5.0], [4.0 + dia + 4 * v0, 5.0]])
    U = np.array([[v0 / 2, 0.0], [-v0 / 2, 0.0]])
    return Oracle(9, (12, 10), (1, 1), 0.8, contact="hertz", young=young, poisson=poisson,
                  restitution=e, x0=X, u0=U, diameter=[dia, dia], density_ratio=[rr, rr])


def _impact(o, m, dt, nmax=200000):
    """Velocity Verlet on the contact force alone (no fluid): returns (maximum
    overlap, time in contact, separation speed)."""
    d0 = 0.5 * (o.dia[0] + o.dia[1])
    F = o.contact_force(0)
    dmax, t_in, was_in = 0.0, 0.0, False
    for _ in range(nmax):
        o.U[0] += 0.5 * dt * F / m
        o.U[1] -= 0.5 * dt * F / m
        o.X += dt * o.U
        F = o.contact_force(0)
        o.U[0] += 0.5 * dt * F / m
        o.U[1] -= 0.5 * dt * F / m
        delta = d0 - np.linalg.norm(o.X[0] - o.X[1])
        if delta > 0:
            t_in += dt
            was_in = True
            dmax = max(dmax, delta)
        elif was_in:
            break
    return dmax, t_in, o.U[1, 0] - o.U[0, 0]


def test_hertz_elastic_impact_matches_analytic_solution():
    """Elastic Hertz impact (e = 1): m* delta'' = -K delta^{3/2}, K = 4/3 E* sqrt(R*).
    Energy gives delta_max = (5 m* v^2 / (4 K))^{2/5}; the contact lasts
    t_c = 2 (delta_max / v) (2/5) B(2/5, 1/2) (Johnson, Contact Mechanics)."""
    v0, E, nu = 4e-4, 1e-2, 0.3
    o = _hertz_pair(v0, 1.0, young=E, poisson=nu)
    m = 2.0 * np.pi / 4
    dmax, tc, vsep = _impact(o, m, dt=0.05)
    Es = 1.0 / (2 * (1 - nu ** 2) / E)
    Rs = 0.25
    mstar = m / 2
    K = 4.0 / 3.0 * Es * math.sqrt(Rs)
    dmax_exact = (5 * mstar * v0 ** 2 / (4 * K)) ** 0.4
    beta_int = 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
    tc_exact = 2 * dmax_exact / v0 * beta_int
    assert dmax == pytest.approx(dmax_exact, rel=2e-4)
    assert tc == pytest.approx(tc_exact, rel=2e-3)
    assert vsep == pytest.approx(v0, rel=1e-6)


def test_hertz_wall_impact_uses_wall_material_and_particle_radius():
    """A particle hitting a wall: m delta'' = -K delta^{3/2} with R* = R and
    1/E* = (1 - nu_p^2)/E_p + (1 - nu_w^2)/E_w."""
    v0, E, nu, Ew, nuw = 3e-4, 1e-2, 0.3, 5e-2, 0.2
    o = Oracle(9, (10, 10), (1, 0), 0.8, contact="hertz", young=E, poisson=nu, wall_young=Ew,
               wall_poisson=nuw, restitution=1.0, x0=[[5.0, 0.5 + 2 * v0]], u0=[[0.0, -v0]],
               diameter=[1.0], density_ratio=[2.0])
    m = 2.0 * np.pi / 4
    dt, dmax = 0.05, 0.0
    F = o.contact_force(0)
    for _ in range(100000):
        o.U[0] += 0.5 * dt * F / m
        o.X[0] += dt * o.U[0]
        F = o.contact_force(0)
        o.U[0] += 0.5 * dt * F / m
        dmax = max(dmax, 0.5 - o.X[0, 1])
        if o.U[0, 1] > 0 and o.X[0, 1] > 0.5:
            break
    Es = 1.0 / ((1 - nu ** 2) / E + (1 - nuw ** 2) / Ew)
    K = 4.0 / 3.0 * Es * math.sqrt(0.5)
    assert dmax == pytest.approx((5 * m * v0 ** 2 / (4 * K)) ** 0.4, rel=2e-4)
    assert o.U[0, 1] == pytest.approx(v0, rel=1e-6)


def test_hertz_damping_gives_a_speed_independent_restitution():
    """With the Hertz stiffness S_n = 2 E* sqrt(R* delta) in the damping, elastic
    and damping forces scale alike with the impact speed, so the restitution
    coefficient does not depend on it, and it stays close to the requested e."""
    out = []
    for v0 in (1e-4, 8e-4):
        o = _hertz_pair(v0, 0.8)
        _, _, vsep = _impact(o, 2.0 * np.pi / 4, dt=0.05)
        out.append(vsep / v0)
    assert out[0] == pytest.approx(out[1], rel=2e-3)
    assert 0.75 < out[0] < 0.85


def test_hertz_pair_forces_cancel():
    X, dia, rr = sample_particles((12, 10), 60, (0.3, 0.8), 2.0, band=(0.0, 1.0), seed=31)
    X = 6.0 + 0.35 * (X - 6.0)
    o = Oracle(9, (12, 10), (1, 1), 0.7, contact="hertz", young=1e-2, x0=X,
               u0=velocities(60, 2, 32, 1e-3), diameter=dia, density_ratio=rr)
    F = np.array([o.contact_force(i) for i in range(o.np)])
    assert np.count_nonzero(np.abs(F).sum(1)) > 10
    assert np.abs(F.sum(0)).max() < 1e-15


# --- DEM sub-cycling ------------------------------------------------------------------------
@pytest.mark.parametrize("implicit", [True, False])
@pytest.mark.parametrize("S", [1, 2, 5])
def test_substeps_follow_the_geometric_recurrence(implicit, S):
    """One particle in uniform fluid at rest (rho_l = 1, j_l = 0 exactly), no
    contacts: each sub-step maps U to r U + (1 - r) U_inf, U_inf = b / (2 A_p),
    b = m (1 - 1/rho_r) g, with r = m / (m + 2 A_p h) (implicit) or
    1 - 2 A_p h / m (explicit), h = 1/S. X moves by h times the sum of the
    velocities, and g is the sub-step average of 2 U (U after the sub-step when
    implicit, before it when explicit)."""
    grav = (0.0, -1e-3)
    o = Oracle(9, (16, 16), (1, 1), 0.7, delta_width=4, implicit_drag=implicit, gravity=grav,
               x0=[[7.3, 8.6]], u0=[[2e-3, -1e-3]], diameter=[0.8], density_ratio=[2.5],
               substeps=S)
    m = 2.5 * np.pi * 0.64 / 4
    Ap = np.pi * 0.64 / 4
    b = m * (1 - 1 / 2.5) * np.array(grav)
    h = 1.0 / S
    r = m / (m + 2 * Ap * h) if implicit else 1 - 2 * Ap * h / m
    Uinf = b / (2 * Ap)
    U0, X0 = o.U[0].copy(), o.X[0].copy()
    Us = [Uinf + (U0 - Uinf) * r ** s for s in range(S + 1)]
    o.step(1)
    assert np.abs(o.U[0] - Us[S]).max() < 1e-15
    assert np.abs(o.X[0] - (X0 + h * sum(Us[1:]))).max() < 1e-13
    seen = Us[1:] if implicit else Us[:-1]
    assert np.abs(o.g[0] - 2 * h * sum(seen)).max() < 1e-15


@pytest.mark.parametrize("S", [2, 4])
def test_substepped_coupling_balances_momentum(S):
    """Periodic box with gravity and contacts, S sub-steps: the fluid gains the
    spread force, which is minus the sum of the particles' hydrodynamic forces,
    and fluid + particle momentum grows by exactly sum m (1 - 1/rho_r) g."""
    n = (24, 20)
    X, dia, rr = sample_particles(n, 40, (0.3, 0.8), (1.5, 3.0), band=(0.0, 1.0), seed=11)
    X = 12.0 + 0.5 * (X - 12.0)  # denser, so that some pairs touch during the step
    _, _, w, _ = lattice(9)
    grav = (0.0, -1e-4)
    o = Oracle(9, n, (1, 1), 0.7, delta_width=4, gravity=grav, x0=X,
               u0=velocities(40, 2, 12, 2e-3), diameter=dia, density_ratio=rr,
               f0=populations(w, (20, 24), seed=13, eps=1e-3), substeps=S, kn=5e-2)
    m = o.rr * np.pi * o.dia ** 2 / 4.0
    buoy = (m * (1 - 1 / o.rr)).sum() * np.array(grav)
    touched = 0.0
    for _ in range(4):
        _, j0 = o.moments()
        P0 = (m[:, None] * o.U).sum(0)
        o.step(1)
        _, j1 = o.moments()
        P1 = (m[:, None] * o.U).sum(0)
        Fsum = o.F.reshape(2, -1).sum(1)
        touched += np.abs(o.Fc).sum()
        tol = 64 * np.finfo(float).eps * o.f.sum()
        assert np.abs(j1.reshape(2, -1).sum(1) - j0.reshape(2, -1).sum(1) - Fsum).max() < tol
        assert np.abs(Fsum + o.f_fpi.sum(0)).max() < 1e-12 * np.abs(o.F).sum()
        assert np.abs((j1.reshape(2, -1).sum(1) + P1) - (j0.reshape(2, -1).sum(1) + P0) - buoy).max() < tol
    assert touched > 0


def test_substepped_hertz_impact_converges_to_the_resolved_collision():
    """Two particles approaching in fluid at rest with a stiff Hertz contact:
    the post-collision velocities converge as the number of sub-steps grows
    (the sub-step error shrinks at least linearly in h)."""
    def run(S):
        X = np.array([[6.0, 6.0], [7.02, 6.0]])
        U = np.array([[2e-3, 0.0], [-2e-3, 0.0]])
        o = Oracle(9, (14, 12), (1, 1), 0.7, delta_width=4, contact="hertz", young=5.0,
                   restitution=0.9, x0=X, u0=U, diameter=[1.0, 1.0], density_ratio=[50.0, 50.0],
                   substeps=S)
        o.step(45)  # contact lasts about 25 steps
        return o.U.copy()

    u8, u16, u32, u64 = run(8), run(16), run(32), run(64)
    e1 = np.abs(u16 - u8).max()
    e2 = np.abs(u32 - u16).max()
    e3 = np.abs(u64 - u32).max()
    assert e2 < 0.75 * e1 and e3 < 0.75 * e2
    assert u64[0, 0] < 0 < u64[1, 0]  # they bounced


@pytest.mark.parametrize("S", [1, 4])
def test_substepped_contact_resolves_the_spring_collision(S):
    """Two very heavy particles (rho_r = 1e6, so the fluid barely acts) collide
    head on with a linear spring and e = 1. The sub-stepped update is then the
    symplectic Euler scheme with step h, so the largest overlap approaches
    v_rel sqrt(m*/k_n) and the pair separates at its approach speed; a contact
    force not scaled by h would make the spring look S times stiffer."""
    rr, v = 1e6, 1e-3
    m = rr * np.pi / 4
    tc = 40.0
    kn = (m / 2) * np.pi ** 2 / tc ** 2
    X = np.array([[6.0, 6.0], [7.0 + 2 * v, 6.0]])
    o = Oracle(9, (14, 12), (1, 1), 0.7, delta_width=2, kn=kn, restitution=1.0, x0=X,
               u0=[[v, 0.0], [-v, 0.0]], diameter=[1.0, 1.0], density_ratio=[rr, rr],
               substeps=S)
    dmax = 0.0
    for _ in range(80):
        o.step(1)
        dmax = max(dmax, 1.0 - np.linalg.norm(o.X[0] - o.X[1]))
    assert dmax == pytest.approx(2 * v * math.sqrt((m / 2) / kn), rel=1e-2)
    assert o.U[1, 0] - o.U[0, 0] == pytest.approx(2 * v, rel=1e-2)
