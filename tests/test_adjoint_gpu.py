"""The discrete adjoint of the coupled step (``pibm_settling_gradient``):
gradients of the mean settling velocity L = mean_p U_p[d-1] after n steps with
respect to tau, the particles' density ratios and their initial positions.

Reference: central differences of the FP64 oracle's forward run on the same
seeded inputs, L(theta + h v) - L(theta - h v) / 2h along tau and along random
directions v of the density ratios and initial positions. The 4-point kernel
is C1, so the differences converge at O(h^2); contacts and the hat kernel are
piecewise smooth and the inputs keep every particle away from a switch within h.
At the full 3D configuration (96^3, 20k particles, 500 steps, checkpoints every
50) the reference is the same central difference of the library's own forward
run, h = 1e-6.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, lattice
from paper_1407_6704_gb300.inputs import populations, sample_particles, velocities

pytestmark = pytest.mark.gpu

LAT = {9: "d2q9", 15: "d3q15", 19: "d3q19"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


def _case(q, n, periodic, tau, width, npart, seed, squeeze=None, dia=(0.5, 0.8)):
    d = len(n)
    X, D, R = sample_particles(n, npart, dia, (1.5, 3.0), band=(0.2, 0.9), seed=seed)
    if squeeze is not None:
        c = np.array(n, dtype=float) / 2
        X = c + squeeze * (X - c)
    _, _, w, _ = lattice(q)
    return dict(q=q, n=n, periodic=periodic, tau=tau, delta_width=width, x0=X,
                u0=velocities(npart, d, seed=seed + 1, scale=2e-3), diameter=D, density_ratio=R,
                f0=populations(w, tuple(reversed(n)), seed=seed + 2, eps=1e-3),
                gravity=(0.0,) * (d - 1) + (-1e-4,), kn=1e-2, restitution=0.8)


def _oracle_loss(c, steps, tau=None, rr=None, x0=None):
    kw = dict(c)
    q, n, per, t = kw.pop("q"), kw.pop("n"), kw.pop("periodic"), kw.pop("tau")
    if tau is not None:
        t = tau
    if rr is not None:
        kw["density_ratio"] = rr
    if x0 is not None:
        kw["x0"] = x0
    o = Oracle(q, n, per, t, **kw)
    o.step(steps)
    return o.U[:, o.d - 1].mean(), o


def _gpu_grad(c, steps, K):
    from paper_1407_6704_gb300.pibm import settling_gradient

    kw = dict(c)
    q = kw.pop("q")
    return settling_gradient(LAT[q], kw.pop("n"), kw.pop("periodic"), kw.pop("tau"), steps,
                             checkpoint_every=K, **kw)


def _check_against_oracle(c, steps, K, h=1e-5, tol=1e-6):
    r = _gpu_grad(c, steps, K)
    L0, o = _oracle_loss(c, steps)
    assert abs(r["loss"] - L0) <= 1e-10 * abs(L0)
    rng = np.random.default_rng(7)
    # tau
    fd_tau = (_oracle_loss(c, steps, tau=c["tau"] + h)[0] - _oracle_loss(c, steps, tau=c["tau"] - h)[0]) / (2 * h)
    # density ratios along a random direction
    v = rng.normal(size=len(c["density_ratio"]))
    rr = np.asarray(c["density_ratio"])
    fd_rho = (_oracle_loss(c, steps, rr=rr + h * v)[0] - _oracle_loss(c, steps, rr=rr - h * v)[0]) / (2 * h)
    # initial positions along a random direction
    V = rng.normal(size=np.asarray(c["x0"]).shape)
    X = np.asarray(c["x0"])
    fd_x = (_oracle_loss(c, steps, x0=X + h * V)[0] - _oracle_loss(c, steps, x0=X - h * V)[0]) / (2 * h)
    got = {"tau": r["dtau"], "rho": float(r["drho"] @ v), "x": float((r["dx0"] * V).sum())}
    ref = {"tau": fd_tau, "rho": fd_rho, "x": fd_x}
    err = {k: abs(got[k] - ref[k]) / max(abs(ref[k]), 1e-300) for k in got}
    print("adjoint vs oracle differences", got, ref, err)
    assert all(abs(ref[k]) > 0 for k in ref)
    # bar: tol relative, plus the rounding floor of a central difference in FP64,
    # about 1e-16 (the loss's intermediates are O(1)) divided by h
    bad = {k: err[k] for k in got if not abs(got[k] - ref[k]) <= tol * abs(ref[k]) + 1e-16 / h}
    assert not bad, (bad, got, ref)
    return o


@pytest.mark.parametrize("width", [2, 4])
def test_adjoint_2d_walls_against_oracle_differences(width):
    """D2Q9 24 x 20, walls, 14 particles, 40 steps, checkpoints every 15 (three
    stretches, the last one short)."""
    c = _case(9, (24, 20), (0, 0), 0.7, width, 14, seed=51)
    _check_against_oracle(c, 40, 15)


def test_adjoint_2d_with_contacts_and_periodic_axis():
    """A squeezed cloud, so that pairs and walls are in contact during the run."""
    c = _case(9, (20, 18), (1, 0), 0.75, 4, 60, seed=52, squeeze=0.85, dia=(0.6, 0.9))
    o = _check_against_oracle(c, 30, 10, tol=5e-6)
    assert np.count_nonzero(np.abs(o.Fc).sum(1)) > 5


@pytest.mark.parametrize("q", [19, 15])
def test_adjoint_3d_against_oracle_differences(q):
    c = _case(q, (10, 9, 12), (0, 1, 0), 0.8, 4, 12, seed=53)
    _check_against_oracle(c, 24, 8)


def test_adjoint_full_3d_configuration_against_its_own_differences():
    """D3Q19 96^3, walls, tau 0.7, 20,000 particles d = 0.5, density ratio 2,
    top half; 500 steps FP64; checkpoints every 50. Gradients against central
    differences of the same library's forward run (h = 1e-6)."""
    from paper_1407_6704_gb300.inputs import preset, workload_particles
    from paper_1407_6704_gb300.pibm import settling_gradient

    w = preset("c5")
    X, dia, rr = workload_particles(w)
    base = dict(gravity=w.gravity, delta_width=w.delta_width, kn=w.kn, restitution=w.restitution,
                diameter=dia)
    steps, h = 500, 1e-6

    def loss(tau=w.tau, r=rr, x=X):
        return settling_gradient("d3q19", w.n, w.periodic, tau, steps, x0=x, density_ratio=r,
                                 grads=False, **base)["loss"]

    import time
    t0 = time.perf_counter()
    g = settling_gradient("d3q19", w.n, w.periodic, w.tau, steps, checkpoint_every=50, x0=X,
                          density_ratio=rr, **base)
    t1 = time.perf_counter()
    loss()
    t2 = time.perf_counter()
    print(f"c5 500 steps: gradient run {t1 - t0:.2f} s, forward only {t2 - t1:.2f} s")
    rng = np.random.default_rng(9)
    v = rng.normal(size=len(rr))
    V = rng.normal(size=X.shape)
    got = {"tau": g["dtau"], "rho": float(g["drho"] @ v), "x": float((g["dx0"] * V).sum())}

    def floor(step):
        # rounding bound of a central difference of the computed loss: a few ulps
        # of |L| (about 2e-6 here) over 2 h; 2.8e-14 at h = 1e-6, far below the
        # 1e-4 relative bar on derivatives of 1e-9 and more
        return 64 * np.finfo(float).eps * abs(g["loss"]) / step

    # h = 1e-6 on every parameter, 1e-4 relative
    fd = {"tau": (loss(tau=w.tau + h) - loss(tau=w.tau - h)) / (2 * h),
          "rho": (loss(r=rr + h * v) - loss(r=rr - h * v)) / (2 * h),
          "x": (loss(x=X + h * V) - loss(x=X - h * V)) / (2 * h)}
    print("c5 adjoint, h = 1e-6", got, fd, {k: abs(got[k] / fd[k] - 1) for k in fd})
    for k in fd:
        assert abs(got[k] - fd[k]) <= 1e-4 * abs(fd[k]) + floor(h), (k, got, fd)
    # and the density and position directions again with h = 1e-4
    H = 1e-4
    fd2 = {"rho": (loss(r=rr + H * v) - loss(r=rr - H * v)) / (2 * H),
           "x": (loss(x=X + H * V) - loss(x=X - H * V)) / (2 * H)}
    print("c5 adjoint, h = 1e-4", got, fd2, {k: abs(got[k] / fd2[k] - 1) for k in fd2})
    for k in fd2:
        assert abs(got[k] - fd2[k]) <= 1e-4 * abs(fd2[k]) + floor(H), (k, got, fd2)


def test_autograd_function_returns_the_adjoint_gradients():
    import torch
    from paper_1407_6704_gb300.pibm import settling_gradient, settling_velocity

    c = _case(9, (16, 14), (0, 0), 0.7, 4, 6, seed=54)
    spec = dict(lattice="d2q9", n=c["n"], periodic=c["periodic"], nsteps=10, checkpoint_every=4,
                gravity=c["gravity"], delta_width=4, u0=c["u0"], diameter=c["diameter"],
                f0=c["f0"])
    tau = torch.tensor(c["tau"], dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(c["density_ratio"], dtype=torch.float64, requires_grad=True)
    x0 = torch.tensor(c["x0"], dtype=torch.float64, requires_grad=True)
    L = settling_velocity(tau, rho, x0, **spec)
    (3.0 * L).backward()
    r = settling_gradient(tau=c["tau"], density_ratio=c["density_ratio"], x0=c["x0"], **spec)
    assert float(L.detach()) == r["loss"]
    assert float(tau.grad) == 3.0 * r["dtau"]
    assert np.array_equal(rho.grad.numpy(), 3.0 * r["drho"])
    assert np.array_equal(x0.grad.numpy(), 3.0 * r["dx0"])
