"""Python binding of the PIBM C ABI: argument marshalling around ``libpibm.so``.

PyTorch provides the device workspace (one uint8 tensor) and the stream; every
computation runs in the CUDA library. Arrays handed to or returned from this
module are NumPy FP64 with the layouts of ``include/pibm.h``.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (FIELD_J, FIELD_POP, FIELD_RHO, FIELD_U, FIELD_X, PibmConfig, check)

_LATTICES = {"d2q9": 9, "d3q15": 15, "d3q19": 19, 9: 9, 15: 15, 19: 19}
_PRECISION = {"fp64": _lib.PIBM_FP64, "fp32": _lib.PIBM_FP32, "fp16": _lib.PIBM_FP16,
              "bf16": _lib.PIBM_BF16}


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


class Pibm:
    """One coupled LBM-PIBM-DEM simulation living on one GPU.

    lattice: "d2q9" | "d3q15" | "d3q19"; n: extents (2 or 3 ints);
    periodic: per-axis flags (False = walls at 0 and n); tau: BGK relaxation time;
    gravity: particle acceleration; delta_width: 2 or 4; implicit: drag coupling;
    precision: "fp64" | "fp32" | "fp16" | "bf16"; deterministic: ordered spreading;
    x0, u0 (n_particles, d), diameter, density_ratio (n_particles,);
    f0: optional (q, ...) post-stream populations of step 0.
    """

    def __init__(self, lattice, n, periodic, tau, gravity=None, delta_width=2, implicit=True,
                 precision="fp64", deterministic=False, kn=1e-2, restitution=0.9, x0=None,
                 u0=None, diameter=None, density_ratio=None, f0=None, device=None, stream=None,
                 interp="delta", contact="linear", young=1.0, poisson=0.3, wall_young=None,
                 wall_poisson=None, substeps=1, rebin_every=1, overlap="auto",
                 particle_update="fp64"):
        """interp: "delta" (the spreading kernel) or "lagrange4" (Eq. 5);
        contact: "linear" (kn) or "hertz" (Eq. 15 with young/poisson of the
        particles and of the walls, default the particles'); both use the
        restitution coefficient; substeps: DEM sub-steps per fluid step;
        rebin_every: cell-list rebuild period in steps (skin-checked);
        overlap: "auto", "on" or "off", the collision of the particle-free tiles
        and the contact search on a second stream (same results);
        particle_update: "fp64" (default) or "fp32", the arithmetic of the
        particle update in the 32- and 16-bit storage modes."""
        import torch

        self._torch = torch
        L = _lib.load()
        self.q = _LATTICES[lattice]
        self.d = 2 if self.q == 9 else 3
        n = list(n) + [1] * (3 - len(n))
        self.n = n
        self.shape = (n[1], n[0]) if self.d == 2 else (n[2], n[1], n[0])
        self.ncell = n[0] * n[1] * n[2]
        per = list(periodic) + [1] * (3 - len(periodic))
        np_ = 0 if x0 is None else int(np.asarray(x0).shape[0])
        self.np = np_
        self._x0 = _f64(x0, (np_, self.d)) if np_ else None
        self._u0 = _f64(u0, (np_, self.d)) if (np_ and u0 is not None) else None
        self._dia = _f64(diameter, (np_,)) if np_ else None
        self._rr = _f64(density_ratio, (np_,)) if np_ else None
        self._f0 = _f64(f0, (self.q, self.ncell)) if f0 is not None else None
        grav = list(gravity) if gravity is not None else [0.0] * self.d
        grav = (grav + [0.0, 0.0, 0.0])[:3]
        self.cfg = PibmConfig(
            self.q, (ctypes.c_int64 * 3)(*n),
            (ctypes.c_int * 3)(*[_lib.PIBM_PERIODIC if p else _lib.PIBM_WALL for p in per]),
            float(tau), (ctypes.c_double * 3)(*grav), int(delta_width),
            _lib.PIBM_IMPLICIT if implicit else _lib.PIBM_EXPLICIT, _PRECISION[precision],
            int(bool(deterministic)), float(kn), float(restitution), np_,
            _dptr(self._x0), _dptr(self._u0), _dptr(self._dia), _dptr(self._rr),
            _dptr(self._f0),
            {"delta": _lib.PIBM_INTERP_DELTA, "lagrange4": _lib.PIBM_INTERP_LAGRANGE4}[interp],
            {"linear": _lib.PIBM_DEM_LINEAR, "hertz": _lib.PIBM_DEM_HERTZ}[contact],
            float(young), float(poisson), float(wall_young or 0.0),
            float(poisson if wall_poisson is None else wall_poisson), int(substeps),
            int(rebin_every),
            {"auto": _lib.PIBM_OVERLAP_AUTO, "on": _lib.PIBM_OVERLAP_ON,
             "off": _lib.PIBM_OVERLAP_OFF}[overlap])
        self.cfg.particle_update = {"fp64": _lib.PIBM_PARTICLE_FP64,
                                    "fp32": _lib.PIBM_PARTICLE_FP32}[particle_update]
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        nbytes = ctypes.c_size_t()
        check(L.pibm_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(nbytes)),
              "pibm_workspace_bytes")
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
            base = self._ws.data_ptr()
            self._ws_ptr = (base + 255) // 256 * 256
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            check(L.pibm_create(ctypes.byref(self.cfg), ctypes.c_void_p(self._ws_ptr),
                                nbytes.value, ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(h)), "pibm_create")
        self._h = h
        self._L = L

    # --- stepping ----------------------------------------------------------------
    def step(self, nsteps=1):
        check(self._L.pibm_step(self._h, int(nsteps)), "pibm_step")

    def profile_steps(self, nsteps):
        """Run nsteps steps phase by phase; summed device ms per phase:
        {'bin', 'contacts', 'couple', 'collide_stream', 'total'}."""
        out = np.zeros(5)
        check(self._L.pibm_profile_steps(self._h, int(nsteps), _dptr(out)), "pibm_profile_steps")
        return dict(zip(("bin", "contacts", "couple", "collide_stream", "total"), out.tolist()))

    def status(self):
        return self._L.pibm_status(self._h)

    def autotune(self):
        """Pick the stream-collide block shape by timing; returns (bx, by)."""
        out = (ctypes.c_int * 2)()
        check(self._L.pibm_autotune(self._h, out), "pibm_autotune")
        return out[0], out[1]

    @property
    def kernels_per_step(self):
        return self._L.pibm_kernels_per_step(self._h)

    @property
    def launch_count(self):
        """Kernels launched by step() on this handle so far."""
        n = ctypes.c_int64()
        check(self._L.pibm_launch_count(self._h, ctypes.byref(n)), "pibm_launch_count")
        return n.value

    # --- read-back -----------------------------------------------------------------
    def forces(self):
        """(f_fpi, f_contact), each (n_particles, d) FP64 on the host."""
        ffpi = np.zeros((self.np, self.d))
        fc = np.zeros((self.np, self.d))
        if self.np:
            check(self._L.pibm_forces(self._h, ffpi.ctypes.data_as(ctypes.c_void_p),
                                      fc.ctypes.data_as(ctypes.c_void_p), 0), "pibm_forces")
        return ffpi, fc

    def read(self, *names, out=None):
        """Host copies of the requested fields: 'rho', 'j', 'pop', 'x', 'u'. out: an
        optional dict of preallocated C-contiguous FP64 arrays (for example in pinned
        memory) to fill instead of new ones."""
        bits = {"rho": (0, FIELD_RHO, (self.ncell,)), "j": (1, FIELD_J, (self.d, self.ncell)),
                "pop": (2, FIELD_POP, (self.q, self.ncell)), "x": (3, FIELD_X, (self.np, self.d)),
                "u": (4, FIELD_U, (self.np, self.d))}
        given = out or {}
        out = {}
        dst = (ctypes.c_void_p * _lib.NFIELDS)()
        mask = 0
        for nm in names:
            k, bit, shp = bits[nm]
            if nm in given:
                arr = given[nm]
                if (arr.dtype != np.float64 or not arr.flags.c_contiguous
                        or arr.size != int(np.prod(shp))):
                    raise ValueError(f"out[{nm!r}] must be C-contiguous FP64 of {shp}")
                arr = arr.reshape(shp)
            else:
                arr = np.zeros(shp)
            out[nm] = arr
            dst[k] = arr.ctypes.data_as(ctypes.c_void_p).value if arr.size else 1
            mask |= bit if arr.size else 0
        check(self._L.pibm_read_fields(self._h, mask, dst, 0), "pibm_read_fields")
        res = {}
        for nm, arr in out.items():
            if nm == "rho":
                res[nm] = arr.reshape(self.shape)
            elif nm in ("j", "pop"):
                res[nm] = arr.reshape((arr.shape[0],) + self.shape)
            else:
                res[nm] = arr
        return res

    def invariants(self):
        """(total mass, fluid momentum (d,), particle momentum (d,))."""
        out = np.zeros(1 + 2 * self.d)
        check(self._L.pibm_invariants(self._h, _dptr(out)), "pibm_invariants")
        return out[0], out[1:1 + self.d].copy(), out[1 + self.d:].copy()

    def close(self):
        if getattr(self, "_h", None):
            self._L.pibm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- presets ---------------------------------------------------------------------
    @classmethod
    def from_workload(cls, w, precision="fp64", n_particles=None, particles=None, f0=None,
                      **kw):
        """Build a simulation from an ``inputs.Workload`` preset (seeded particles)."""
        from .inputs import workload_particles
        X, dia, rr = particles if particles is not None else workload_particles(w, n_particles)
        lat = {9: "d2q9", 15: "d3q15", 19: "d3q19"}[w.q]
        return cls(lat, w.n, w.periodic, w.tau, gravity=w.gravity, delta_width=w.delta_width,
                   precision=precision, kn=w.kn, restitution=w.restitution, x0=X, diameter=dia,
                   density_ratio=rr, f0=f0, **kw)


class Ensemble:
    """Independent simulations advanced together. Persistent mode (members of
    one kind, see ``pibm_ensemble_create``): one cooperative kernel launch runs
    up to 10 steps of every member, replayed from a CUDA graph; otherwise one
    graph branch per member."""

    def __init__(self, members, stream=None):
        import torch

        self.members = list(members)
        self._L = _lib.load()
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        self.stream = stream if stream is not None else self.members[0].stream
        h = ctypes.c_void_p()
        check(self._L.pibm_ensemble_create(arr, len(self.members),
                                           ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(h)), "pibm_ensemble_create")
        self._h = h
        self._torch = torch

    def step(self, nsteps=1):
        check(self._L.pibm_ensemble_step(self._h, int(nsteps)), "pibm_ensemble_step")

    def status(self):
        return self._L.pibm_ensemble_status(self._h)

    def info(self):
        """{persistent, ctas_per_sm, max_ctas_per_sm, cells_per_item, grid, graph}."""
        out = (ctypes.c_int * 6)()
        check(self._L.pibm_ensemble_info(self._h, out), "pibm_ensemble_info")
        keys = ("persistent", "ctas_per_sm", "max_ctas_per_sm", "cells_per_item", "grid", "graph")
        return dict(zip(keys, list(out)))

    def configure(self, ctas_per_sm=0, cells_per_item=0):
        check(self._L.pibm_ensemble_configure(self._h, int(ctas_per_sm), int(cells_per_item)),
              "pibm_ensemble_configure")

    def autotune(self, steps_per_candidate=20):
        """Time every launch shape on real steps (the ensemble advances by
        candidates x (steps, rounded up to 10, + 10) steps); keep the fastest."""
        out = (ctypes.c_int * 3)()
        check(self._L.pibm_ensemble_autotune(self._h, int(steps_per_candidate), out),
              "pibm_ensemble_autotune")
        return {"ctas_per_sm": out[0], "cells_per_item": out[1], "candidates": out[2]}

    def set_mode(self, persistent):
        check(self._L.pibm_ensemble_set_mode(self._h, 1 if persistent else 0),
              "pibm_ensemble_set_mode")

    def launch_count(self):
        n = ctypes.c_int64()
        check(self._L.pibm_ensemble_launch_count(self._h, ctypes.byref(n)),
              "pibm_ensemble_launch_count")
        return n.value

    def inject_skip(self, block, limit_s):
        """Test hook: CTA `block` skips the first barrier of the next launch."""
        check(self._L.pibm_ensemble_inject_skip(self._h, int(block), float(limit_s)),
              "pibm_ensemble_inject_skip")

    def close(self):
        if getattr(self, "_h", None):
            self._L.pibm_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def settling_gradient(lattice, n, periodic, tau, nsteps, checkpoint_every=50, gravity=None,
                      delta_width=2, kn=1e-2, restitution=0.9, x0=None, u0=None, diameter=None,
                      density_ratio=None, f0=None, stream=None, grads=True):
    """Mean settling velocity L = mean over particles of U[d-1] after nsteps FP64
    steps, and its gradients by the discrete adjoint (``pibm_settling_gradient``):
    {"loss", "dtau", "drho" (n_particles,), "dx0" (n_particles, d)}; with
    grads=False only the forward run (the gradients come back as None)."""
    import torch

    q = _LATTICES[lattice]
    d = 2 if q == 9 else 3
    n = list(n) + [1] * (3 - len(n))
    per = list(periodic) + [1] * (3 - len(periodic))
    X = _f64(x0, (-1, d))
    npart = X.shape[0]
    U = _f64(u0, (npart, d)) if u0 is not None else None
    dia = _f64(diameter, (npart,))
    rr = _f64(density_ratio, (npart,))
    F0 = _f64(f0, (q, -1)) if f0 is not None else None
    grav = ((list(gravity) if gravity is not None else [0.0] * d) + [0.0, 0.0, 0.0])[:3]
    cfg = PibmConfig(q, (ctypes.c_int64 * 3)(*n),
                     (ctypes.c_int * 3)(*[_lib.PIBM_PERIODIC if p else _lib.PIBM_WALL for p in per]),
                     float(tau), (ctypes.c_double * 3)(*grav), int(delta_width), _lib.PIBM_IMPLICIT,
                     _lib.PIBM_FP64, 1, float(kn), float(restitution), npart, _dptr(X), _dptr(U),
                     _dptr(dia), _dptr(rr), _dptr(F0))
    st = stream if stream is not None else torch.cuda.current_stream()
    loss = np.zeros(1)
    dtau = np.zeros(1)
    drho = np.zeros(npart)
    dx0 = np.zeros((npart, d))
    g = (lambda a: _dptr(a)) if grads else (lambda a: None)
    check(_lib.load().pibm_settling_gradient(ctypes.byref(cfg), int(nsteps), int(checkpoint_every),
                                             ctypes.c_void_p(st.cuda_stream), _dptr(loss),
                                             g(dtau), g(drho), g(dx0)),
          "pibm_settling_gradient")
    if not grads:
        return {"loss": float(loss[0]), "dtau": None, "drho": None, "dx0": None}
    return {"loss": float(loss[0]), "dtau": float(dtau[0]), "drho": drho, "dx0": dx0}


def _settling_function():
    import torch

    class SettlingVelocity(torch.autograd.Function):
        """torch.autograd view of ``settling_gradient``: forward(tau, density_ratio,
        x0, spec) runs the forward steps only and returns the mean settling velocity
        as a 0-d FP64 tensor; backward runs the checkpointed forward again (the run
        is deterministic, so it repeats bit for bit) and the reverse sweep, and
        returns the adjoint gradients for tau, density_ratio and x0. ``spec`` holds
        the remaining keyword arguments of ``settling_gradient``."""

        @staticmethod
        def forward(ctx, tau, density_ratio, x0, spec):
            args = dict(tau=float(tau), density_ratio=density_ratio.detach().cpu().numpy(),
                        x0=x0.detach().cpu().numpy(), **spec)
            r = settling_gradient(grads=False, **args)
            ctx.args = args
            ctx.loss = r["loss"]
            return torch.tensor(r["loss"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            r = settling_gradient(**ctx.args)
            if r["loss"] != ctx.loss:
                raise RuntimeError("the replayed forward run differs from the first one")
            gt = torch.tensor(r["dtau"], dtype=torch.float64)
            return (grad * gt, grad * torch.from_numpy(r["drho"]),
                    grad * torch.from_numpy(r["dx0"]), None)

    return SettlingVelocity


def settling_velocity(tau, density_ratio, x0, **spec):
    """Differentiable mean settling velocity (see ``settling_gradient``) of CPU
    FP64 tensors tau (0-d), density_ratio (n,), x0 (n, d)."""
    return _settling_function().apply(tau, density_ratio, x0, spec)


def grid_barrier_test(nblocks, skip_block=-1, nbarriers=1, limit_s=0.2):
    """Run the persistent kernel's grid barrier in a cooperative launch of
    nblocks CTAs (``pibm_grid_barrier_test``); returns (status, barriers passed)."""
    L = _lib.load()
    passed = ctypes.c_int()
    st = L.pibm_grid_barrier_test(int(nblocks), int(skip_block), int(nbarriers), float(limit_s),
                                  ctypes.byref(passed))
    return st, passed.value
