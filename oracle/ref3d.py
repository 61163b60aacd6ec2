"""FP64 CPU oracle of the three-dimensional extension of the two-belt Shan-Chen step -- TEST
INFRASTRUCTURE (only ``tests/`` may import it).

Wraps ``lbm_oracle3d.c``: D3Q19, Eq. FORCE over the 3-D links of |c|^2 <= 4 (attraction) and
<= 8 (repulsion) with the weights that solve Appendix B's constraints in three dimensions, the
first-belt cross repulsion, and the shifted-velocity BGK collision of Sec. II, periodic in x and
y, and in z or between bounce-back walls (Sec. IV).  It shares no code with the CUDA path.

Parity: pinned by ``tests/test_oracle3d.py`` against the isotropy sums of the weights, the
D3Q19 equilibrium moments, mass and momentum conservation, the closed-form force on sinusoidal
fields, the dispersion relation of sound on a uniform state, equal bulk pressures across a
relaxed flat interface, and the exact Couette and Poiseuille profiles between walls.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle3d.c")
_HDR = os.path.join(_HERE, "lbm_oracle3d.h")
_LIB = os.path.join(_HERE, "liblbmref3d.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liblbmref3d.so with gcc (FP64, -ffp-contract=off: no FMA contraction; OpenMP over
    independent per-site loops only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                                                         os.path.getmtime(_HDR)):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-o", tmp,
                        _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params3(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double * 2),
        ("G1", ctypes.c_double * 2),
        ("G2", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double),
        ("rho0", ctypes.c_double * 2),
        ("weight_norm", ctypes.c_double),
        ("body_force", ctypes.c_double),
        ("psi_form", ctypes.c_int),
        ("zbc", ctypes.c_int),
        ("wall_u", ctypes.c_double * 2),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
            lib.lbmref3_tables.argtypes = [ip, dp, dp, dp, ip, dp]
            lib.lbmref3_feq.argtypes = [ctypes.c_double, dp, dp]
            lib.lbmref3_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(Params3)]
            lib.lbmref3_destroy.argtypes = [vp]
            lib.lbmref3_destroy.restype = None
            lib.lbmref3_set_params.argtypes = [vp, ctypes.POINTER(Params3)]
            lib.lbmref3_set_fields.argtypes = [vp, dp]
            lib.lbmref3_set_populations.argtypes = [vp, dp]
            lib.lbmref3_site_fields.argtypes = [vp, dp, dp]
            lib.lbmref3_step.argtypes = [vp, ctypes.c_int]
            lib.lbmref3_get.argtypes = [vp, dp, dp, dp]
            lib.lbmref3_step_count.argtypes = [vp]
            lib.lbmref3_step_count.restype = ctypes.c_longlong
            _lib = lib
        return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def tables():
    """(links [92, 3], w_att [9], w_rep [9], w_cross [9] by |c|^2, c19 [19, 3], w19 [19])."""
    lib = _load()
    links = np.zeros((92, 3), dtype=np.int32)
    c19 = np.zeros((19, 3), dtype=np.int32)
    wa, wr, wc, w19 = np.zeros(9), np.zeros(9), np.zeros(9), np.zeros(19)
    ip = ctypes.POINTER(ctypes.c_int)
    n = lib.lbmref3_tables(links.ctypes.data_as(ip), _ptr(wa), _ptr(wr), _ptr(wc), c19.ctypes.data_as(ip), _ptr(w19))
    assert n == 92
    return links, wa, wr, wc, c19, w19


def feq(rho, u):
    out = np.zeros(19)
    u = np.ascontiguousarray(u, dtype=np.float64)
    _load().lbmref3_feq(float(rho), _ptr(u), _ptr(out))
    return out


def make_params(tau=1.0, G1=0.0, G2=0.0, G_AB=0.0, rho0=1.0, weight_norm=1.0 / 3.0, body_force=0.0,
                psi_form=0, zbc=0, wall_u=(0.0, 0.0)) -> Params3:
    p = Params3()
    for name, v in (("tau", tau), ("G1", G1), ("G2", G2), ("rho0", rho0)):
        v = list(v) if hasattr(v, "__len__") else [v, v]
        getattr(p, name)[0], getattr(p, name)[1] = v[0], v[-1]
    p.G_AB, p.weight_norm, p.body_force, p.psi_form = G_AB, weight_norm, body_force, psi_form
    p.zbc = zbc
    p.wall_u[0], p.wall_u[1] = wall_u
    return p


class RefLattice3D:
    """An nx x ny x nz lattice of one or two species (arrays indexed [z][y][x]), periodic in x
    and y, and in z unless zbc = 1 (walls)."""

    def __init__(self, nx, ny, nz, n_species=1, **params):
        self.lib = _load()
        self.nx, self.ny, self.nz, self.ns = nx, ny, nz, n_species
        self.p = make_params(**params)
        h = ctypes.c_void_p()
        rc = self.lib.lbmref3_create(ctypes.byref(h), nx, ny, nz, n_species, ctypes.byref(self.p))
        if rc != 0:
            raise ValueError(f"lbmref3_create rc={rc}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbmref3_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_fields(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ns, self.nz, self.ny, self.nx)
        if self.lib.lbmref3_set_fields(self.h, _ptr(rho)) != 0:
            raise ValueError("lbmref3_set_fields: densities must be positive and finite")

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ns, 19, self.nz, self.ny, self.nx)
        assert self.lib.lbmref3_set_populations(self.h, _ptr(f)) == 0

    def step(self, n=1):
        assert self.lib.lbmref3_step(self.h, int(n)) == 0

    @property
    def nstep(self):
        return self.lib.lbmref3_step_count(self.h)

    def fields(self):
        """(rho [ns, nz, ny, nx], u [3, nz, ny, nx], f [ns, 19, nz, ny, nx])."""
        shape = (self.nz, self.ny, self.nx)
        rho, u = np.zeros((self.ns,) + shape), np.zeros((3,) + shape)
        f = np.zeros((self.ns, 19) + shape)
        assert self.lib.lbmref3_get(self.h, _ptr(rho), _ptr(u), _ptr(f)) == 0
        return rho, u, f

    def site_fields(self):
        """dict psi [ns, nz, ny, nx], F [ns, 3, nz, ny, nx] (total force of each species)."""
        shape = (self.nz, self.ny, self.nx)
        psi, F = np.zeros((self.ns,) + shape), np.zeros((self.ns, 3) + shape)
        assert self.lib.lbmref3_site_fields(self.h, _ptr(psi), _ptr(F)) == 0
        return dict(psi=psi, F=F)
