"""Checkpoint and restart through the public calls: a run restarted from the
state it reports (populations, positions and velocities from pibm_read_fields,
passed to pibm_create as f0, x0 and u0) continues as the uninterrupted run. The
step keeps no other history: linear contacts have none, and g and the contact
forces are recomputed every step. FP64, the parity bar of 1e-10 relative: positions
and velocities relative to the largest displacement and speed, populations relative
to their largest deviation from the rest state w (the part of f that the run
changes; f itself is about 0.1 everywhere). The spreading's atomics may order the
sums differently run to run; on GB300 the difference measured zero."""
import numpy as np
import pytest

from oracle.oracle import lattice
from tests.test_parity_gpu import LAT, make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


# walls only along the gravity axis, with the particle band well inside them, so
# that no particle comes within its radius of a wall before the restart
@pytest.mark.parametrize("q,n,periodic,rebin", [(9, (48, 40), (1, 0), 1),
                                                 (19, (14, 12, 16), (1, 1, 0), 4)])
def test_restart_from_the_read_state_continues_the_run(q, n, periodic, rebin):
    from paper_1407_6704_gb300.pibm import Pibm

    c = make_case(q=q, n=n, periodic=periodic, tau=0.7, width=4, npart=150 if q == 9 else 80,
                  seed=61, f0_eps=1e-3, u_scale=2e-3, dia=(0.5, 0.8), rr=2.0, band=(0.3, 0.9))
    kw = dict(delta_width=c["width"], gravity=c["gravity"], kn=c["kn"], restitution=c["e"],
              diameter=c["D"], density_ratio=c["R"], rebin_every=rebin)
    args = (LAT[q], n, periodic, c["tau"])
    with Pibm(*args, x0=c["X"], u0=c["U"], f0=c["f0"], **kw) as sim:
        sim.step(30)
        whole = sim.read("pop", "x", "u")
    with Pibm(*args, x0=c["X"], u0=c["U"], f0=c["f0"], **kw) as sim:
        sim.step(18)
        mid = sim.read("pop", "x", "u")
    with Pibm(*args, x0=mid["x"], u0=mid["u"], f0=mid["pop"].reshape(q, -1), **kw) as sim:
        sim.step(12)
        got = sim.read("pop", "x", "u")
        assert sim.status() == 0
    w = lattice(q)[2].reshape((-1,) + (1,) * len(n))
    dpop = np.abs(got["pop"] - whole["pop"]).max() / np.abs(whole["pop"] - w).max()
    dx = np.abs(got["x"] - whole["x"]).max() / np.abs(whole["x"] - c["X"]).max()
    du = np.abs(got["u"] - whole["u"]).max() / np.abs(whole["u"]).max()
    print("restart", q, dpop, dx, du)
    assert dpop < 1e-10 and dx < 1e-10 and du < 1e-10
