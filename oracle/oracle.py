"""Python driver for the FP64 CPU oracle of the PIBM coupled step.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline leg use this module. It loads ``liboracle.so`` (built from
``pibm_oracle.c``) and never touches the CUDA library.

Arrays follow the C-ABI layouts: populations ``(q, nz, ny, nx)`` (``(q, ny, nx)``
in 2D), force ``(d, ...)``, particle vectors AoS ``(n_particles, d)``. The C code
keeps populations as g = f - w (see ``pibm_oracle.c``); this module converts at
its boundary, so every population array it takes or returns holds f itself.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_libs = {}


class OrParams(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("periodic", ctypes.c_int * 3),
        ("tau", ctypes.c_double),
        ("delta_width", ctypes.c_int),
        ("implicit_drag", ctypes.c_int),
        ("gravity", ctypes.c_double * 3),
        ("kn", ctypes.c_double),
        ("restitution", ctypes.c_double),
        ("interp", ctypes.c_int),
        ("contact", ctypes.c_int),
        ("young", ctypes.c_double),
        ("poisson", ctypes.c_double),
        ("wall_young", ctypes.c_double),
        ("wall_poisson", ctypes.c_double),
        ("substeps", ctypes.c_int),
    ]


def lib(parallel=False):
    """The serial oracle library, or (parallel=True) its OpenMP build."""
    if parallel not in _libs:
        path = _build.build(parallel=parallel)
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OrParams)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_lattice.argtypes = [ctypes.c_int, ip, ip, dp, ip]
        L.or_phi.argtypes = [ctypes.c_int, ctypes.c_double]
        L.or_phi.restype = ctypes.c_double
        L.or_taps.argtypes = [P, ctypes.c_int, ctypes.c_double, ip, dp]
        L.or_lagrange_taps.argtypes = [P, ctypes.c_int, ctypes.c_double, ip, dp]
        L.or_interp_taps.argtypes = [P, ctypes.c_int, ctypes.c_double, ip, dp]
        L.or_moments.argtypes = [P, dp, dp, dp]
        L.or_interp_pops.argtypes = [P, dp, dp, dp]
        L.or_contact_force.argtypes = [P, ctypes.c_long, dp, dp, dp, dp, ctypes.c_long, dp]
        L.or_particle_update.argtypes = [P, dp, ctypes.c_long, dp, dp, dp, dp, ctypes.c_long,
                                         dp, dp, dp, dp, dp]
        L.or_spread_one.argtypes = [P, dp, ctypes.c_double, dp, dp]
        L.or_collide.argtypes = [P, dp, dp, dp]
        L.or_stream.argtypes = [P, dp, dp]
        step_args = [P, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.or_step.argtypes = step_args
        L.or_run.argtypes = [P, ctypes.c_long] + step_args[1:]
        L.or_force_at_cell.argtypes = [P, dp, ctypes.c_long, dp, dp, dp, dp, ctypes.c_long, dp]
        L.or_cell_after_step.argtypes = [P, dp, ctypes.c_long, dp, dp, dp, dp, ctypes.c_long, dp]
        _libs[parallel] = L
    return _libs[parallel]


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice(q):
    """(d, e[q,3], w[q], opp[q]) of the D2Q9 / D3Q15 / D3Q19 velocity set."""
    d = ctypes.c_int()
    e = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    rc = lib().or_lattice(q, ctypes.byref(d), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          _p(w), opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc:
        raise ValueError(f"unknown lattice q={q}")
    return d.value, e, w, opp


def phi(width, a):
    return lib().or_phi(int(width), float(a))


class Oracle:
    """State of one oracle run: populations, particles and the last step's forces."""

    def __init__(self, q, n, periodic, tau, delta_width=2, implicit_drag=True,
                 gravity=(0.0, 0.0, 0.0), kn=1e-2, restitution=0.9,
                 x0=None, u0=None, diameter=None, density_ratio=None, f0=None,
                 interp="delta", contact="linear", young=1.0, poisson=0.3, wall_young=None,
                 wall_poisson=None, substeps=1, parallel=False):
        """interp: "delta" (the spreading kernel) or "lagrange4" (Eq. 5);
        contact: "linear" (k_n, e) or "hertz" (Eq. 15 with young/poisson of the
        particles and of the walls, default the particles' material, and e);
        substeps: DEM sub-steps per fluid step; parallel: whole steps run in the
        OpenMP build (bitwise identical results, all cores)."""
        self.parallel = bool(parallel)
        self.q = int(q)
        self.d, self.e, self.w, self.opp = lattice(self.q)
        n = list(n) + [1] * (3 - len(n))
        per = list(periodic) + [1] * (3 - len(periodic))
        if self.d == 2:
            n[2], per[2] = 1, 1
        self.n = n
        self.params = OrParams(self.q, (ctypes.c_int * 3)(*n), (ctypes.c_int * 3)(*per),
                               float(tau), int(delta_width), int(bool(implicit_drag)),
                               (ctypes.c_double * 3)(*(list(gravity) + [0.0] * 3)[:3]),
                               float(kn), float(restitution),
                               {"delta": 0, "lagrange4": 1}[interp],
                               {"linear": 0, "hertz": 1}[contact], float(young), float(poisson),
                               float(young if wall_young is None else wall_young),
                               float(poisson if wall_poisson is None else wall_poisson),
                               int(substeps))
        self.substeps = int(substeps)
        self.shape = (n[1], n[0]) if self.d == 2 else (n[2], n[1], n[0])
        self.ncell = n[0] * n[1] * n[2]
        self._wb = self.w.reshape((-1,) + (1,) * len(self.shape))
        if f0 is None:
            g = np.zeros((self.q,) + self.shape)  # the rest state f = w
        else:
            g = np.asarray(f0, dtype=np.float64).reshape((self.q,) + self.shape) - self._wb
        self.fdev = np.ascontiguousarray(g)  # stored populations minus w, advanced by step()
        self.fs = np.zeros_like(self.fdev)
        self.F = np.zeros((self.d,) + self.shape)
        np_ = 0 if x0 is None else len(x0)
        self.np = np_
        def own(a, shape):  # private contiguous copy: the oracle updates X, U in place
            return np.array(np.asarray(a, dtype=np.float64).reshape(shape), order="C", copy=True)
        self.X = own(x0, (np_, self.d)) if np_ else np.zeros((0, self.d))
        self.U = np.zeros_like(self.X) if u0 is None else own(u0, (np_, self.d))
        self.dia = own(diameter, (np_,)) if np_ else np.zeros(0)
        self.rr = own(density_ratio, (np_,)) if np_ else np.zeros(0)
        self.Xn = np.zeros_like(self.X)
        self.Un = np.zeros_like(self.U)
        self.g = np.zeros_like(self.X)
        self.Fc = np.zeros_like(self.X)
        self.diag = np.zeros(2)

    @property
    def f(self):
        """Post-stream populations of the current state (a new array)."""
        return self.fdev + self._wb

    @f.setter
    def f(self, value):
        self.fdev = np.ascontiguousarray(np.asarray(value, dtype=np.float64).reshape(self.fdev.shape)
                                      - self._wb)

    def _to_g(self, f):
        return np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.fdev.shape)
                                    - self._wb)

    # --- whole steps -------------------------------------------------------
    def step(self, nsteps=1):
        L = lib(self.parallel)
        L.or_run(ctypes.byref(self.params), int(nsteps), _p(self.fdev), _p(self.fs), _p(self.F),
                 self.np, _p(self.X), _p(self.U), _p(self.dia), _p(self.rr), _p(self.Xn),
                 _p(self.Un), _p(self.g), _p(self.Fc), _p(self.diag))

    @property
    def f_fpi(self):
        """Reaction force on each particle, Eq. (12): -A_p g."""
        Ap = np.pi * self.dia ** 2 / 4.0
        return -Ap[:, None] * self.g

    # --- pieces --------------------------------------------------------------
    def moments(self, f=None):
        g = self.fdev if f is None else self._to_g(f)
        rho = np.zeros(self.shape)
        j = np.zeros((self.d,) + self.shape)
        lib().or_moments(ctypes.byref(self.params), _p(g), _p(rho), _p(j))
        return rho, j

    def taps(self, axis, X):
        """Spreading taps (Eqs. 10-11) along one axis: (indices, weights)."""
        idx = (ctypes.c_int * 4)()
        w = np.zeros(4)
        cnt = lib().or_taps(ctypes.byref(self.params), int(axis), float(X), idx, _p(w))
        return [idx[i] for i in range(cnt)], w[:cnt].copy()

    def interp_taps(self, axis, X):
        """Interpolation taps of the configured interpolant along one axis."""
        idx = (ctypes.c_int * 4)()
        w = np.zeros(4)
        cnt = lib().or_interp_taps(ctypes.byref(self.params), int(axis), float(X), idx, _p(w))
        return [idx[i] for i in range(cnt)], w[:cnt].copy()

    def interp_pops(self, X):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(self.d))
        gl = np.zeros(self.q)
        lib().or_interp_pops(ctypes.byref(self.params), _p(self.fdev), _p(X), _p(gl))
        return gl + self.w

    def contact_force(self, i):
        Fc = np.zeros(self.d)
        lib().or_contact_force(ctypes.byref(self.params), self.np, _p(self.X), _p(self.U),
                               _p(self.dia), _p(self.rr), int(i), _p(Fc))
        return Fc

    def particle_update(self, i):
        """(X', U', g, Fc, |g_literal - g_closed|, escaped) for particle i from the current state."""
        assert self.substeps <= 1, "sampled evaluation covers steps without sub-cycling"
        Xn, Un, g, Fc = (np.zeros(self.d) for _ in range(4))
        dv = np.zeros(1)
        esc = lib().or_particle_update(ctypes.byref(self.params), _p(self.fdev), self.np, _p(self.X),
                                       _p(self.U), _p(self.dia), _p(self.rr), int(i), _p(Xn),
                                       _p(Un), _p(g), _p(Fc), _p(dv))
        return Xn, Un, g, Fc, float(dv[0]), bool(esc)

    def collide(self, f, F):
        g = self._to_g(f)
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.zeros_like(g)
        lib().or_collide(ctypes.byref(self.params), _p(g), _p(F), _p(out))
        return out + self._wb

    def stream(self, fs):
        gs = self._to_g(fs)
        out = np.zeros_like(gs)
        lib().or_stream(ctypes.byref(self.params), _p(gs), _p(out))
        return out + self._wb

    def spread_one(self, X, dia, g, F):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(self.d))
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(self.d))
        lib().or_spread_one(ctypes.byref(self.params), _p(X), float(dia), _p(g), _p(F))

    # --- sampled evaluation of one step (large lattices) ---------------------
    def force_at_cell(self, cell):
        assert self.substeps <= 1, "sampled evaluation covers steps without sub-cycling"
        out = np.zeros(self.d)
        lib().or_force_at_cell(ctypes.byref(self.params), _p(self.fdev), self.np, _p(self.X),
                               _p(self.U), _p(self.dia), _p(self.rr), int(cell), _p(out))
        return out

    def cell_after_step(self, cell):
        assert self.substeps <= 1, "sampled evaluation covers steps without sub-cycling"
        out = np.zeros(self.q)
        lib().or_cell_after_step(ctypes.byref(self.params), _p(self.fdev), self.np, _p(self.X),
                                 _p(self.U), _p(self.dia), _p(self.rr), int(cell), _p(out))
        return out + self.w
