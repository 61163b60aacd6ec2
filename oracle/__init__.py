"""FP64 CPU oracle of the multirange Shan-Chen lattice Boltzmann step -- TEST INFRASTRUCTURE.

This package is test infrastructure, not the product.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It wraps
``lbm_oracle.c`` (plain C, FP64, no FMA contraction), which follows the paper's equations
(Sbragaglia, Benzi, Bernaschi, Succi, arXiv:1402.6019): Eq. LB (BGK), the moments of Sec. II,
Eq. FORCE (two-belt force), the shifted-velocity forcing of Sec. II, the A/B model of Sec. IV
and the lattice stress of Sec. III / Appendix A.  It shares no code with the CUDA path.

Parity: pinned by tests/test_oracle_*.py against the paper's isotropy sums (App. B), the
equilibrium moments (Sec. II), conservation laws, closed-form forces on sinusoidal fields,
exact Couette and Poiseuille profiles, the exact lattice momentum balance of Eq. MECHANICAL at
a flat interface, and Laplace's law.  The fluidity / cooperative-length numbers the paper prints
(Sec. IV, zeta = 18 .. 68) need its multi-million-step runs: parity unpinned for those.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbmref.so")
_lock = threading.Lock()
_lib = None

PERIODIC, BOUNCEBACK = 0, 1
PSI_EXP, PSI_RHO = 0, 1
WEIGHTS_PAPER, WEIGHTS_CHEM09 = 0, 1
WALL_MIRROR, WALL_ZERO = 0, 1


def build(force: bool = False) -> str:
    """Compile liblbmref.so with gcc (FP64, -ffp-contract=off so no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    from . import ref3d  # the three-dimensional oracle (its own library)

    ref3d.build(force)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double * 2),
        ("G1", ctypes.c_double * 2),
        ("G2", ctypes.c_double * 2),
        ("G_AB", ctypes.c_double),
        ("psi_form", ctypes.c_int),
        ("rho0", ctypes.c_double * 2),
        ("weight_preset", ctypes.c_int),
        ("weight_norm", ctypes.c_double),
        ("body_force", ctypes.c_double),
        ("wall_u", ctypes.c_double * 2),
        ("psi_wall", ctypes.c_int),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


class Obs(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double * 2),
        ("momentum", ctypes.c_double * 2),
        ("gamma", ctypes.c_double),
        ("wall_force", ctypes.c_double * 2),
        ("nonfinite", ctypes.c_int),
        ("ux_z", _DP),
        ("rho_z", _DP),
        ("sxz_z", _DP),
        ("fluid_z", _DP),
        ("ps_x", _DP),
        ("pxx_x", _DP),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.lbmref_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int]
            lib.lbmref_set_params.argtypes = [vp, ctypes.POINTER(Params)]
            lib.lbmref_set_fields.argtypes = [vp, _DP, _DP]
            lib.lbmref_set_populations.argtypes = [vp, _DP]
            lib.lbmref_get_fields.argtypes = [vp, _DP, _DP, _DP]
            lib.lbmref_step.argtypes = [vp, ctypes.c_int]
            lib.lbmref_observables.argtypes = [vp, ctypes.POINTER(Obs)]
            lib.lbmref_site_fields.argtypes = [vp, _DP, _DP, _DP, _DP, _DP]
            lib.lbmref_step_count.argtypes = [vp]
            lib.lbmref_step_count.restype = ctypes.c_longlong
            lib.lbmref_destroy.argtypes = [vp]
            lib.lbmref_destroy.restype = None
            lib.lbmref_tables.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), _DP, _DP]
            lib.lbmref_tables.restype = None
            lib.lbmref_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP]
            lib.lbmref_feq.restype = None
            lib.lbmref_adjoint_step.argtypes = [vp, _DP, _DP, _DP]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def tables(preset: int = WEIGHTS_PAPER):
    """(c25 [25,2], cq [9,2], wq [9], wsh [3,9]) as the oracle holds them."""
    lib = _load()
    c25 = (ctypes.c_int * 50)()
    cq = (ctypes.c_int * 18)()
    wq = np.zeros(9)
    wsh = np.zeros(27)
    lib.lbmref_tables(preset, c25, cq, _ptr(wq), _ptr(wsh))
    return (np.array(c25[:]).reshape(25, 2), np.array(cq[:]).reshape(9, 2), wq,
            wsh.reshape(3, 9))


def feq(rho: float, ux: float, uz: float) -> np.ndarray:
    out = np.zeros(9)
    _load().lbmref_feq(rho, ux, uz, _ptr(out))
    return out


def make_params(**kw) -> Params:
    """Params with defaults tau=1, rho0=1, weight_norm=1/3 and everything else zero."""
    p = Params()
    p.tau[0] = p.tau[1] = 1.0
    p.rho0[0] = p.rho0[1] = 1.0
    p.weight_norm = 1.0 / 3.0
    for k, v in kw.items():
        if k in ("tau", "G1", "G2", "rho0", "wall_u"):
            v = list(v) if hasattr(v, "__len__") else [v, v]
            arr = getattr(p, k)
            arr[0] = v[0]
            arr[1] = v[1] if len(v) > 1 else v[0]
        else:
            setattr(p, k, v)
    return p


class RefLattice:
    """One oracle simulation; arrays are numpy float64, layouts as in lbm_oracle.h."""

    def __init__(self, nx, nz, n_species=1, z_boundary=PERIODIC, **params):
        self.lib = _load()
        self.nx, self.nz, self.ns, self.zbc = nx, nz, n_species, z_boundary
        h = ctypes.c_void_p()
        rc = self.lib.lbmref_create(ctypes.byref(h), nx, nz, n_species, z_boundary)
        if rc != 0:
            raise ValueError(f"lbmref_create rc={rc}")
        self.h = h
        self.set_params(**params)

    def set_params(self, **params):
        self.params = make_params(**params)
        rc = self.lib.lbmref_set_params(self.h, ctypes.byref(self.params))
        if rc != 0:
            raise ValueError(f"lbmref_set_params rc={rc}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbmref_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_fields(self, rho, u=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ns, self.nz, self.nx)
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, self.nz, self.nx)
        rc = self.lib.lbmref_set_fields(self.h, _ptr(rho), _ptr(u))
        if rc != 0:
            raise ValueError(f"lbmref_set_fields rc={rc}")

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ns, 9, self.nz, self.nx)
        assert self.lib.lbmref_set_populations(self.h, _ptr(f)) == 0

    def step(self, n=1):
        assert self.lib.lbmref_step(self.h, int(n)) == 0

    @property
    def nstep(self):
        return self.lib.lbmref_step_count(self.h)

    def fields(self):
        """(rho [ns,nz,nx], u [2,nz,nx], f [ns,9,nz,nx])."""
        rho = np.zeros((self.ns, self.nz, self.nx))
        u = np.zeros((2, self.nz, self.nx))
        f = np.zeros((self.ns, 9, self.nz, self.nx))
        assert self.lib.lbmref_get_fields(self.h, _ptr(rho), _ptr(u), _ptr(f)) == 0
        return rho, u, f

    def site_fields(self):
        """dict psi [ns,nz,nx], F [ns,2,nz,nx], sint [ns,3,nz,nx], P [3,nz,nx], sxz [nz,nx]."""
        ns, nz, nx = self.ns, self.nz, self.nx
        out = dict(psi=np.zeros((ns, nz, nx)), F=np.zeros((ns, 2, nz, nx)),
                   sint=np.zeros((ns, 3, nz, nx)), P=np.zeros((3, nz, nx)),
                   sxz=np.zeros((nz, nx)))
        assert self.lib.lbmref_site_fields(self.h, _ptr(out["psi"]), _ptr(out["F"]),
                                           _ptr(out["sint"]), _ptr(out["P"]),
                                           _ptr(out["sxz"])) == 0
        return out

    def scales(self):
        """Magnitudes the observables of the current state are formed from (for stating errors):
        rho_max = max rho; u_max = max |u| (barycentric); pop_scale = max over sites of
        sum_s sum_l |f_l c_l| / sum_s rho_s (the terms a velocity is a difference of);
        stress_scale = max over sites of |P_xx| + |P_zz| + 2 |P_xz| (Sec. III's tensor: the terms
        S_xz, p_s and P_xx are sums and differences of)."""
        rho, u, f = self.fields()
        P = self.site_fields()["P"]
        c = np.array([0, 1, 1, 1, 1, 1, 1, 1, 1], float)
        return dict(rho_max=float(np.abs(rho).max()), u_max=float(np.abs(u).max()),
                    pop_scale=float(((np.abs(f) * c[None, :, None, None]).sum(axis=(0, 1)) / rho.sum(0)).max()),
                    stress_scale=float((np.abs(P[0]) + np.abs(P[1]) + 2 * np.abs(P[2])).max()))

    def adjoint_step(self, lam_next, grad=None):
        """dJ/df_n from dJ/df_{n+1} at the current state (periodic lattices); adds the
        parameter derivatives to grad (G1 A, B; G2 A, B; G_AB; tau A, B; body_force)."""
        lam_next = np.ascontiguousarray(lam_next, dtype=np.float64).reshape(self.ns, 9, self.nz, self.nx)
        lam = np.zeros_like(lam_next)
        grad = np.zeros(NPARAM) if grad is None else grad
        assert self.lib.lbmref_adjoint_step(self.h, _ptr(lam_next), _ptr(lam), _ptr(grad)) == 0
        return lam, grad

    def observables(self):
        nz, nx = self.nz, self.nx
        prof = dict(ux_z=np.zeros(nz), rho_z=np.zeros(self.ns * nz), sxz_z=np.zeros(nz),
                    fluid_z=np.zeros(nz), ps_x=np.zeros(nx), pxx_x=np.zeros(nx))
        o = Obs()
        for k, v in prof.items():
            setattr(o, k, _ptr(v))
        assert self.lib.lbmref_observables(self.h, ctypes.byref(o)) == 0
        res = dict(mass=np.array(o.mass[:]), momentum=np.array(o.momentum[:]),
                   gamma=o.gamma, wall_force=np.array(o.wall_force[:]),
                   nonfinite=bool(o.nonfinite))
        prof["rho_z"] = prof["rho_z"].reshape(self.ns, nz)
        res.update(prof)
        return res


# ---------------------------------------------------------------------------------------
# Calibration objective and its gradient through a run (the adjoint written out plainly)
# ---------------------------------------------------------------------------------------
NPARAM = 8  # G1 A, G1 B, G2 A, G2 B, G_AB, tau A, tau B, body_force


def profile_objective(f, target_u, target_rho):
    """J = sum_z (ubar(z) - target_u(z))^2 + (rhobar_A(z) - target_rho(z))^2 for the populations
    f [ns, 9, nz, nx]: ubar = x-average of u = sum_s j_x,s / sum_s rho_s, rhobar_A = x-average of
    rho_A.  Returns (J, dJ/df)."""
    cq, _ = tables()[1:3]
    cx = np.array([c[0] for c in cq], dtype=float)
    ns, _, nz, nx = f.shape
    rho = f.sum(axis=1)                                 # [ns, nz, nx]
    jx = np.einsum("l,slzx->szx", cx, f)
    rt = rho.sum(axis=0)
    u = jx.sum(axis=0) / rt                             # [nz, nx]
    du = u.mean(axis=1) - target_u                      # [nz]
    dr = rho[0].mean(axis=1) - target_rho
    J = float((du ** 2).sum() + (dr ** 2).sum())
    # dJ/du(x, z) = 2 du(z) / nx; du/df_s,l = (c_lx - u) / rho_tot; dJ/drho_A(x, z) = 2 dr(z) / nx
    gu = (2.0 * du / nx)[:, None] / rt                  # [nz, nx]
    g = np.empty_like(f)
    for s in range(ns):
        for l in range(9):
            g[s, l] = gu * (cx[l] - u) + (2.0 * dr / nx)[:, None] * (1.0 if s == 0 else 0.0)
    return J, g


def rollout_gradient(nx, nz, ns, rho_init, steps, target_u, target_rho, **params):
    """J after `steps` oracle steps from the equilibrium at rest with densities rho_init, and
    its gradient with respect to rho_init [ns, nz, nx] and the parameters (NPARAM entries),
    by the discrete adjoint: forward storing every state, then lambda backwards."""
    ref = RefLattice(nx, nz, ns, PERIODIC, **params)
    ref.set_fields(rho_init)
    states = []
    for _ in range(steps):
        states.append(ref.fields()[2])
        ref.step(1)
    J, lam = profile_objective(ref.fields()[2], target_u, target_rho)
    grad = np.zeros(NPARAM)
    for f in reversed(states):
        ref.set_populations(f)
        lam, grad = ref.adjoint_step(lam, grad)
    # the initial populations are W_l rho_init (equilibrium at rest)
    wq = tables()[2]
    g_rho = np.einsum("l,slzx->szx", wq, lam)
    return J, g_rho, grad
