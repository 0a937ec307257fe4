"""Steps with overlap (``overlap="on"``): the contact search, then the collision
of the free tiles (those no particle stencil reaches before the next cell-list
rebuild), run on a second stream beside the moment and coupling kernels, and the
collision of the busy tiles follows both. Every cell's arithmetic is the one of
the single-stream step, so the results meet the FP64 oracle at the same bar.

The particles sit in a band, so both kinds of tile occur; the cases cover walls
and periodic axes next to the band (a periodic wrap makes the far edge's tiles
busy), 2D and 3D, every-step and kept cell lists, graph replays and single
steps.
"""
import numpy as np
import pytest

from tests.test_parity_gpu import LAT, TOL, make_case, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_1407_6704_gb300 import build

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()


def _run(c, steps, precision="fp64", rebin=1, chunks=None, overlap="on", oracle=True,
         deterministic=False):
    from oracle.oracle import Oracle
    from paper_1407_6704_gb300.pibm import Pibm

    kw = dict(delta_width=c["width"], gravity=c["gravity"], kn=c["kn"], restitution=c["e"],
              x0=c["X"], u0=c["U"], diameter=c["D"], density_ratio=c["R"], f0=c["f0"])
    ref = None
    if oracle:
        ref = Oracle(c["q"], c["n"], c["periodic"], c["tau"], implicit_drag=c["implicit"], **kw)
        ref.step(steps)
    with Pibm(LAT[c["q"]], c["n"], c["periodic"], c["tau"], implicit=c["implicit"],
              precision=precision, rebin_every=rebin, overlap=overlap,
              deterministic=deterministic, **kw) as sim:
        for k in (chunks or [steps]):
            sim.step(k)
        got = sim.read("pop", "rho", "j", "x", "u")
        got["f_fpi"], got["f_c"] = sim.forces()
        got["status"] = sim.status()
        got["kps"] = sim.kernels_per_step
    return got, ref


def _check(got, ref, X0, tol=1e-10):
    assert got["status"] == 0
    e = rel_errors(got, ref, X0)
    bad = {k: v for k, v in e.items() if not v <= TOL.get(k, tol)}
    assert not bad, (bad, e)
    return e


CASES = [
    # name, make_case arguments, steps, rebuild period, step chunks
    ("2d_walls_band_top", dict(q=9, n=(160, 96), periodic=(0, 0), tau=0.7, width=4, npart=700,
                               seed=91, dia=(0.5, 0.8), rr=2.0, band=(0.55, 0.95),
                               u_scale=2e-3, f0_eps=1e-3, e=0.8), 60, 5, [1, 29, 30]),
    ("2d_periodic_band_at_edge", dict(q=9, n=(128, 80), periodic=(1, 1), tau=0.8, width=2,
                                      npart=500, seed=92, dia=(0.4, 0.7), rr=(1.5, 3.0),
                                      band=(0.0, 0.3), u_scale=2e-3, f0_eps=1e-3), 40, 1,
     [3, 37]),
    # 16 x 20 = 320 tiles: the tile lists span two blocks of their build kernels
    ("2d_two_list_blocks", dict(q=9, n=(512, 160), periodic=(1, 0), tau=0.7, width=4,
                                npart=1500, seed=97, dia=(0.5, 0.8), rr=2.0, band=(0.3, 0.7),
                                u_scale=2e-3, f0_eps=1e-3, e=0.8), 30, 10, [10, 20]),
    # periodic y with 33 rows: the last tile row is one cell wide, so stencils of
    # particles near y = 32 cross it and wrap into row 0, two tiles away
    ("2d_periodic_one_cell_tile", dict(q=9, n=(64, 33), periodic=(0, 1), tau=0.7, width=4,
                                       npart=40, seed=98, dia=(0.4, 0.6), rr=2.0,
                                       band=(0.86, 0.965), u_scale=1e-3, f0_eps=1e-3), 20, 5,
     [7, 13]),
    ("3d_walls_periodic_x", dict(q=19, n=(40, 24, 36), periodic=(1, 0, 0), tau=0.7, width=4,
                                 npart=400, seed=93, dia=(0.5, 0.8), rr=2.0, band=(0.5, 0.9),
                                 u_scale=2e-3, f0_eps=1e-3, e=0.8), 30, 4, [2, 28]),
    ("3d_d3q15_every_step", dict(q=15, n=(32, 24, 40), periodic=(0, 0, 0), tau=0.75, width=2,
                                 npart=300, seed=94, dia=(0.4, 0.7), rr=2.0, band=(0.6, 0.95),
                                 u_scale=1e-3, f0_eps=1e-3), 24, 1, None),
]


@pytest.mark.parametrize("name,kw,steps,rebin,chunks", CASES, ids=[c[0] for c in CASES])
def test_overlap_parity_fp64(name, kw, steps, rebin, chunks):
    c = make_case(**kw)
    got, ref = _run(c, steps, rebin=rebin, chunks=chunks)
    print(name, _check(got, ref, c["X"]))


def test_overlap_launches_one_more_kernel_and_needs_32_or_64_bit_storage():
    """The collision becomes two kernels (free tiles, busy tiles) with overlap;
    16-bit storage keeps one stream and its pair kernel, and so does ordered
    spreading (its gather writes every cell of the force field)."""
    c = make_case(q=9, n=(64, 48), periodic=(0, 0), tau=0.7, width=4, npart=60, seed=95,
                  band=(0.6, 0.9))
    on, _ = _run(c, 2, overlap="on", oracle=False)
    off, _ = _run(c, 2, overlap="off", oracle=False)
    assert on["kps"] == off["kps"] + 1
    h_on, _ = _run(c, 2, precision="fp16", overlap="on", oracle=False)
    h_off, _ = _run(c, 2, precision="fp16", overlap="off", oracle=False)
    assert h_on["kps"] == h_off["kps"] == off["kps"]
    d_on, _ = _run(c, 2, overlap="on", oracle=False, deterministic=True)
    d_off, _ = _run(c, 2, overlap="off", oracle=False, deterministic=True)
    assert d_on["kps"] == d_off["kps"]


def test_overlap_fp32_matches_single_stream():
    """FP32 storage, kept cell list: with and without overlap the runs differ only
    by the order of the spreading atomics, far below the FP32 bar to the oracle."""
    c = make_case(q=9, n=(160, 96), periodic=(0, 0), tau=0.7, width=4, npart=700, seed=96,
                  dia=(0.5, 0.8), rr=2.0, band=(0.55, 0.95), u_scale=2e-3, f0_eps=1e-3, e=0.8)
    on, ref = _run(c, 100, precision="fp32", rebin=10)
    off, _ = _run(c, 100, precision="fp32", rebin=10, overlap="off", oracle=False)
    assert on["status"] == 0 and off["status"] == 0
    rho_r, j_r = ref.moments()
    ur = j_r / rho_r
    for g in (on, off):
        ug = g["j"] / g["rho"]
        assert np.sqrt(((ug - ur) ** 2).sum() / (ur ** 2).sum()) < 1e-4
    d = np.abs(on["pop"] - off["pop"]).max() / np.abs(ref.f - ref.w.reshape((-1, 1, 1))).max()
    assert d < 1e-4, d
