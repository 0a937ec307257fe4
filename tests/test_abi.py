"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/pibm.h declares, the ctypes struct matches the C layout, and
configuration validation rejects what the header says it rejects."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1407_6704_gb300 import _lib
from paper_1407_6704_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pibm.h")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return _lib.load()


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pibm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    declared = header_functions()
    assert declared, "no declarations parsed"
    assert sorted(_lib.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pibm_[a-z_]+)\b", out))
    for name in declared:
        assert name in exported, name
        assert hasattr(lib, name)


def test_config_struct_layout_matches_c(tmp_path):
    fields = [f for f, _ in _lib.PibmConfig._fields_]
    prog = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pibm.h"', "int main(void){",
             'printf("%zu\\n", sizeof(pibm_config));']
    lines += [f'printf("%zu\\n", offsetof(pibm_config, {f}));' for f in fields]
    lines += ["return 0;}"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(_lib.PibmConfig)
    for f, off in zip(fields, vals[1:]):
        assert getattr(_lib.PibmConfig, f).offset == off, f


def test_strerror(lib):
    assert lib.pibm_strerror(0) == b"ok"
    for st in range(-8, 0):
        assert lib.pibm_strerror(st) and lib.pibm_strerror(st) != b"unknown status"


def _cfg(**over):
    X = over.pop("X", np.array([[5.0, 5.0]]))
    dia = over.pop("dia", np.array([0.5]))
    rr = over.pop("rr", np.array([2.0]))
    keep = [X, dia, rr]
    dp = ctypes.POINTER(ctypes.c_double)
    c = _lib.PibmConfig(9, (ctypes.c_int64 * 3)(16, 12, 1), (ctypes.c_int * 3)(0, 0, 1), 0.8,
                        (ctypes.c_double * 3)(0, -1e-5, 0), 2, 0, 0, 0, 1e-2, 0.9, len(X),
                        X.ctypes.data_as(dp), None, dia.ctypes.data_as(dp),
                        rr.ctypes.data_as(dp), None)
    for k, v in over.items():
        setattr(c, k, v)
    return c, keep


def _ws(lib, c):
    n = ctypes.c_size_t()
    return lib.pibm_workspace_bytes(ctypes.byref(c), ctypes.byref(n)), n.value


def test_workspace_for_valid_config(lib):
    c, keep = _cfg()
    st, n = _ws(lib, c)
    assert st == 0
    # two population buffers of 9 FP64 planes dominate
    assert n >= 2 * 9 * 16 * 12 * 8


@pytest.mark.parametrize("field,value", [
    ("tau", 0.5), ("tau", 0.3), ("lattice", 7), ("delta_width", 3), ("coupling", 5),
    ("precision", 9), ("dem_restitution", 0.0), ("dem_restitution", 1.5), ("dem_kn", -1.0),
    ("overlap", 3), ("overlap", -1),
])
def test_invalid_scalars_rejected(lib, field, value):
    c, keep = _cfg(**{field: value})
    assert _ws(lib, c)[0] == _lib.PIBM_EINVAL


def test_overlap_modes_accepted(lib):
    for mode in (_lib.PIBM_OVERLAP_AUTO, _lib.PIBM_OVERLAP_ON, _lib.PIBM_OVERLAP_OFF):
        c, keep = _cfg(overlap=mode)
        assert _ws(lib, c)[0] == 0


def test_invalid_particles_rejected(lib):
    for X, dia, rr in [
        (np.array([[-0.1, 5.0]]), np.array([0.5]), np.array([2.0])),  # outside
        (np.array([[16.0, 5.0]]), np.array([0.5]), np.array([2.0])),  # on the wall
        (np.array([[5.0, 5.0]]), np.array([1.5]), np.array([2.0])),   # wider than a cell
        (np.array([[5.0, 5.0]]), np.array([0.5]), np.array([0.0])),   # zero density
        (np.array([[np.nan, 5.0]]), np.array([0.5]), np.array([2.0])),
    ]:
        c, keep = _cfg(X=X, dia=dia, rr=rr)
        assert _ws(lib, c)[0] == _lib.PIBM_EINVAL


def test_2d_requires_unit_depth_and_limits(lib):
    c, keep = _cfg()
    c.n[2] = 3
    assert _ws(lib, c)[0] == _lib.PIBM_EINVAL
    c, keep = _cfg(n_particles=0)
    c.n[0], c.n[1] = 9000, 8000  # more cells than the cell-list scan covers
    assert _ws(lib, c)[0] == _lib.PIBM_ENOTSUP


def test_periodic_axes_need_five_cells_with_particles(lib):
    c, keep = _cfg()
    c.boundary[0] = 1
    c.n[0] = 4
    c.x0[0] = 2.0
    assert _ws(lib, c)[0] == _lib.PIBM_EINVAL
    c.n[0] = 5
    assert _ws(lib, c)[0] == 0


def test_ordered_gather_needs_its_reach_on_periodic_axes(lib):
    """The ordered spreading gathers over 2 R + 1 cells per axis (R = 2 for the
    4-point kernel, plus 1 with a kept cell list); a shorter periodic axis would
    visit a cell twice."""
    c, keep = _cfg(deterministic=1, delta_width=4, rebin_every=10)
    c.boundary[0] = 1
    c.x0[0] = 2.0
    for n, ok in ((6, False), (7, True)):
        c.n[0] = n
        assert (_ws(lib, c)[0] == 0) == ok, n
    c.rebin_every = 1
    c.n[0] = 5
    assert _ws(lib, c)[0] == 0
    c.deterministic = 0
    c.rebin_every = 10
    assert _ws(lib, c)[0] == 0


def test_empty_particle_set_is_valid(lib):
    c, keep = _cfg()
    c.n_particles = 0
    st, n = _ws(lib, c)
    assert st == 0 and n > 0


def test_noalloc_size_check_cannot_overflow(lib):
    """Extents whose product overflows 64 bits are rejected as too big. The size
    check comes before any CUDA call, so this needs no GPU and the pointers are
    never dereferenced."""
    dummy = ctypes.c_void_p(256)
    for q, n in [(9, (2**63 - 1, 1, 1)), (9, (5000, 2**62, 1)), (19, (16, 2**60, 16)),
                 (19, (4096, 4096, 2**62)), (15, (1, 1, 2**63 - 1))]:
        n3 = (ctypes.c_int64 * 3)(*n)
        assert lib.pibm_fluid_sums_noalloc(dummy, q, n3, dummy, None) == _lib.PIBM_ETOOBIG, n


def test_particle_update_modes(lib):
    """pibm_config.particle_update: PIBM_PARTICLE_FP64 (0) and PIBM_PARTICLE_FP32 (1)
    are accepted, anything else is PIBM_EINVAL."""
    for v, want in [(_lib.PIBM_PARTICLE_FP64, _lib.PIBM_OK), (_lib.PIBM_PARTICLE_FP32, _lib.PIBM_OK),
                    (2, _lib.PIBM_EINVAL), (-1, _lib.PIBM_EINVAL)]:
        c, keep = _cfg(particle_update=v)
        assert _ws(lib, c)[0] == want, v


def test_ensemble_and_barrier_entry_points_check_arguments(lib):
    """Every ensemble entry point rejects a NULL ensemble, and the barrier self-test
    rejects out-of-range arguments, before any CUDA call."""
    E = _lib.PIBM_EINVAL
    vp = ctypes.c_void_p
    out = vp()
    n = ctypes.c_int64()
    ints = (ctypes.c_int * 6)()
    assert lib.pibm_ensemble_create(None, 0, None, ctypes.byref(out)) == E
    arr = (vp * 1)(None)
    assert lib.pibm_ensemble_create(arr, 1, None, ctypes.byref(out)) == E  # NULL member
    assert lib.pibm_ensemble_step(None, 1) == E
    assert lib.pibm_ensemble_status(None) == E
    assert lib.pibm_ensemble_configure(None, 0, 0) == E
    assert lib.pibm_ensemble_autotune(None, 10, ints) == E
    assert lib.pibm_ensemble_info(None, ints) == E
    assert lib.pibm_ensemble_launch_count(None, ctypes.byref(n)) == E
    assert lib.pibm_ensemble_inject_skip(None, 0, 0.1) == E
    assert lib.pibm_ensemble_set_mode(None, 1) == E
    lib.pibm_ensemble_destroy(None)  # a no-op
    passed = ctypes.c_int(-1)
    for args in [(0, -1, 1, 0.1), (2, 2, 1, 0.1), (1, -1, 0, 0.1), (1, -1, 1, 0.0),
                 (1, -1, 1, 11.0)]:
        assert lib.pibm_grid_barrier_test(*args, ctypes.byref(passed)) == E, args
    assert lib.pibm_grid_barrier_test(1, -1, 1, 0.1, None) == E
    assert lib.pibm_strerror(_lib.PIBM_ETIMEOUT).decode().startswith("a grid barrier")
