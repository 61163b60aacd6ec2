"""Python binding of liblbm.so (argument marshalling only).

The functions below carry the names of the C ABI in include/lbm.h and include/lbm3d.h (the
three-dimensional extension, lbm3_*) and do nothing but convert
arguments; every step of the method runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing or cannot be loaded, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_ENOMEM, LBM_ENONFINITE, LBM_ETIMEOUT = range(6)
LBM_FP64, LBM_FP32 = 0, 1
LBM_PERIODIC, LBM_BOUNCEBACK = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_FUSED, LBM_KERNEL_TWO_PASS, LBM_KERNEL_SWEEP, LBM_KERNEL_PULL = 0, 1, 2, 3, 4
LBM_PSI_EXP, LBM_PSI_RHO = 0, 1
LBM_WEIGHTS_PAPER, LBM_WEIGHTS_CHEM09 = 0, 1
LBM_WALL_MIRROR, LBM_WALL_ZERO = 0, 1
LBM_HOST, LBM_DEVICE = 0, 1

_DP = ctypes.POINTER(ctypes.c_double)


class lbm_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("n_species", ctypes.c_int),
                ("precision", ctypes.c_int), ("z_boundary", ctypes.c_int), ("kernel", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("rows_per_warp", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("n_instances", ctypes.c_int),
                ("inst_nz", ctypes.POINTER(ctypes.c_int))]


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("G1", ctypes.c_double * 2), ("G2", ctypes.c_double * 2),
                ("G_AB", ctypes.c_double), ("psi_form", ctypes.c_int), ("rho0", ctypes.c_double * 2),
                ("weight_preset", ctypes.c_int), ("weight_norm", ctypes.c_double),
                ("body_force", ctypes.c_double), ("wall_u", ctypes.c_double * 2),
                ("psi_wall", ctypes.c_int), ("rho_ref", ctypes.c_double * 2)]


class lbm_obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2), ("momentum", ctypes.c_double * 2), ("gamma", ctypes.c_double),
                ("wall_force", ctypes.c_double * 2), ("nonfinite", ctypes.c_int),
                ("step", ctypes.c_longlong), ("samples", ctypes.c_longlong),
                ("ux_z", _DP), ("rho_z", _DP), ("sxz_z", _DP), ("fluid_z", _DP), ("ps_x", _DP),
                ("pxx_x", _DP)]


class lbm3_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("n_species", ctypes.c_int),
                ("precision", ctypes.c_int), ("z_boundary", ctypes.c_int), ("device", ctypes.c_int),
                ("pad_", ctypes.c_int), ("stream", ctypes.c_void_p)]


# Every symbol declared in include/lbm.h and include/lbm3d.h: name -> (restype, argtypes)
_VP = ctypes.c_void_p
SIGNATURES = {
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(lbm_desc)]),
    "lbm_validate_desc": (ctypes.c_int, [ctypes.POINTER(lbm_desc)]),
    "lbm_validate_params": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.c_int]),
    "lbm_default_desc": (None, [ctypes.POINTER(lbm_desc)]),
    "lbm_default_params": (None, [ctypes.POINTER(lbm_params)]),
    "lbm_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(lbm_params)]),
    "lbm_set_fields": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "lbm_get_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "lbm_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm_set_observe": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm_observables": (ctypes.c_int, [_VP, ctypes.POINTER(lbm_obs)]),
    "lbm_averages": (ctypes.c_int, [_VP, ctypes.POINTER(lbm_obs), ctypes.c_int]),
    "lbm_synchronize": (ctypes.c_int, [_VP]),
    "lbm_launch_count": (ctypes.c_longlong, [_VP]),
    "lbm_profile": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_last_error": (ctypes.c_char_p, [_VP]),
    "lbm_destroy": (None, [_VP]),
    "lbm_abi_version": (ctypes.c_int, []),
    "lbm_observables_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(lbm_params), _VP, _VP]),
    "lbm_selftest_wait": (ctypes.c_int, [_VP, ctypes.c_longlong]),
    "lbm_set_instance_drive": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lbm_instance_observables": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(lbm_obs), ctypes.c_int]),
    "lbm_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "lbm_autotune_tiles": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double)]),
    "lbm_set_tile_shape": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "lbm_set_populations": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "lbm_observables_bytes": (ctypes.c_longlong, [_VP]),
    "lbm_observables_enqueue": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_wait": (ctypes.c_int, [_VP, ctypes.c_longlong]),
    "lbm_step_read": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_observables_unpack": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(lbm_obs)]),
    "lbm_profile_read_adjoint": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_snapshot_bytes": (ctypes.c_longlong, [_VP]),
    "lbm_snapshot": (ctypes.c_int, [_VP, _VP]),
    "lbm_restore": (ctypes.c_int, [_VP, _VP]),
    "lbm_restore_own": (ctypes.c_int, [_VP, _VP]),
    "lbm_export_state": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "lbm_record_states": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int]),
    "lbm_adjoint_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "lbm_adjoint_steps": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_int]),
    "lbm_adjoint_objective": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "lbm_adjoint_initial": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "lbm3_default_desc": (None, [ctypes.POINTER(lbm3_desc)]),
    "lbm3_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(lbm3_desc)]),
    "lbm3_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(lbm_params)]),
    "lbm3_set_fields": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "lbm3_get_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "lbm3_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm3_totals": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "lbm3_synchronize": (ctypes.c_int, [_VP]),
    "lbm3_profile": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm3_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "lbm3_step_totals": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "lbm3_wait": (ctypes.c_int, [_VP, ctypes.c_longlong]),
    "lbm3_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "lbm3_set_shape": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm3_last_error": (ctypes.c_char_p, [_VP]),
    "lbm3_destroy": (None, [_VP]),
}

_lib = None


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it first when it is missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing; build it with __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != LBM_OK:
        msg = load().lbm_last_error(ctx)
        raise LbmError(rc, msg.decode() if msg else "")


def _check3(rc, ctx=None):
    if rc != LBM_OK:
        msg = load().lbm3_last_error(ctx)
        raise LbmError(rc, msg.decode() if msg else "")


def _dptr(a):
    """Host float64 C-contiguous array, or an object with data_ptr() (a CUDA torch tensor)."""
    if a is None:
        return None, LBM_HOST
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), LBM_DEVICE
    assert a.dtype == np.float64 and a.flags.c_contiguous, "host arrays must be C-contiguous float64"
    return ctypes.c_void_p(a.ctypes.data), LBM_HOST


# ---- thin wrappers with the C names -------------------------------------------------------

def lbm_default_desc() -> lbm_desc:
    d = lbm_desc()
    load().lbm_default_desc(ctypes.byref(d))
    return d


def lbm_default_params() -> lbm_params:
    p = lbm_params()
    load().lbm_default_params(ctypes.byref(p))
    return p


def lbm_validate_desc(d: lbm_desc) -> int:
    return load().lbm_validate_desc(ctypes.byref(d))


def lbm_validate_params(p: lbm_params, n_species: int) -> int:
    return load().lbm_validate_params(ctypes.byref(p), n_species)


def lbm_create(d: lbm_desc):
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(h), ctypes.byref(d)), None)
    return h


def lbm_set_params(h, p: lbm_params):
    _check(load().lbm_set_params(h, ctypes.byref(p)), h)


def lbm_set_fields(h, rho, u=None):
    pr, where = _dptr(rho)
    pu, where_u = _dptr(u)
    if u is not None and where_u != where:
        raise ValueError("rho and u must both be host arrays or both device tensors")
    _check(load().lbm_set_fields(h, pr, pu, where), h)


def lbm_get_fields(h, rho=None, u=None, f=None):
    ptrs = [_dptr(a) for a in (rho, u, f)]
    wheres = {w for (p, w), a in zip(ptrs, (rho, u, f)) if a is not None}
    if len(wheres) > 1:
        raise ValueError("outputs must all be host arrays or all device tensors")
    where = wheres.pop() if wheres else LBM_HOST
    _check(load().lbm_get_fields(h, ptrs[0][0], ptrs[1][0], ptrs[2][0], where), h)


def lbm_step(h, nsteps: int):
    _check(load().lbm_step(h, int(nsteps)), h)


def lbm_set_observe(h, every: int):
    _check(load().lbm_set_observe(h, int(every)), h)


def lbm_observables(h, o: lbm_obs):
    _check(load().lbm_observables(h, ctypes.byref(o)), h)


def lbm_averages(h, o: lbm_obs, reset: bool = False):
    _check(load().lbm_averages(h, ctypes.byref(o), 1 if reset else 0), h)


def lbm_synchronize(h):
    _check(load().lbm_synchronize(h), h)


def lbm_launch_count(h) -> int:
    return load().lbm_launch_count(h)


def lbm_profile(h, enable: bool):
    _check(load().lbm_profile(h, 1 if enable else 0), h)


def lbm_profile_read(h):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(load().lbm_profile_read(h, ctypes.byref(ms), ctypes.byref(n)), h)
    return ms.value, n.value


def lbm_profile_read_adjoint(h):
    """(ms of the three adjoint kernels: moments, local, final; adjoint steps timed)."""
    ms = (ctypes.c_double * 3)()
    n = ctypes.c_longlong()
    _check(load().lbm_profile_read_adjoint(h, ms, ctypes.byref(n)), h)
    return list(ms), n.value


def lbm_last_error(h=None) -> str:
    m = load().lbm_last_error(h)
    return m.decode() if m else ""


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_abi_version() -> int:
    return load().lbm_abi_version()


def lbm_observables_noalloc(f_dev_ptr, nx, nz, n_species, z_boundary, p: lbm_params, out_dev_ptr, stream=None):
    """Observables of FP64 populations held in caller device memory, with no allocation
    (see include/lbm.h); returns the status code."""
    return load().lbm_observables_noalloc(ctypes.c_void_p(f_dev_ptr), nx, nz, n_species, z_boundary,
                                          ctypes.byref(p), ctypes.c_void_p(out_dev_ptr), ctypes.c_void_p(stream))


def lbm_selftest_wait(h, cycles: int) -> int:
    """Runs the step kernels' bounded wait on a barrier nothing completes; returns the status
    (LBM_ETIMEOUT when the expiry was detected and reported, as intended)."""
    return load().lbm_selftest_wait(h, ctypes.c_longlong(cycles))


def lbm_set_populations(h, f):
    """f: host float64 [ns, 9, nz, nx] array or a CUDA float64 tensor of that layout."""
    pf, where = _dptr(f)
    _check(load().lbm_set_populations(h, pf, where), h)


def _dev(t):
    if t is None:
        return None
    if not hasattr(t, "data_ptr"):
        raise TypeError("the adjoint entry points take CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _prec(*tensors):
    """LBM_FP64 / LBM_FP32 from the dtype of the state / adjoint tensors (all alike)."""
    kinds = {str(t.dtype) for t in tensors if t is not None}
    if kinds == {"torch.float64"}:
        return LBM_FP64
    if kinds == {"torch.float32"}:
        return LBM_FP32
    raise TypeError(f"state and adjoint tensors must all be float64 or all float32, got {kinds}")


def lbm_snapshot_bytes(h) -> int:
    return load().lbm_snapshot_bytes(h)


def lbm_snapshot(h, dst):
    """dst: CUDA tensor of at least lbm_snapshot_bytes(h) bytes (asynchronous)."""
    if dst.numel() * dst.element_size() < lbm_snapshot_bytes(h):
        raise ValueError("snapshot buffer too small")
    _check(load().lbm_snapshot(h, _dev(dst)), h)


def lbm_restore(h, src):
    """Restores the snapshot in the CUDA tensor src (reads its tail back: synchronises)."""
    _check(load().lbm_restore(h, _dev(src)), h)


def lbm_restore_own(h, src):
    """Asynchronous restore of the snapshot this context last wrote into src; an overwritten
    src is reported by the next synchronising call."""
    _check(load().lbm_restore_own(h, _dev(src)), h)


def lbm_export_state(h, f):
    """f: CUDA tensor [ns, 9, nz, nx], float64 or float32 (asynchronous)."""
    _check(load().lbm_export_state(h, _dev(f), _prec(f)), h)


def lbm_record_states(h, nsteps, states):
    """states: CUDA tensor [nsteps, ns, 9, nz, nx] (float64 or float32), written asynchronously."""
    _check(load().lbm_record_states(h, int(nsteps), _dev(states), _prec(states)), h)


def lbm_adjoint_step(h, f, lam_next, lam, grad):
    """CUDA tensors: lam <- dJ/df_n, grad[8] (float64) += dJ/dtheta (asynchronous)."""
    _check(load().lbm_adjoint_step(h, _dev(f), _dev(lam_next), _dev(lam), _dev(grad), _prec(f, lam_next, lam)), h)


def lbm_adjoint_steps(h, nsteps, states, lam, grad):
    """lam (in place): dJ/df after the recorded steps -> dJ/df before them; grad += dJ/dtheta."""
    _check(load().lbm_adjoint_steps(h, int(nsteps), _dev(states), _dev(lam), _dev(grad), _prec(states, lam)), h)


def lbm_adjoint_objective(h, f, target_u, target_rho, J, dJdf=None):
    _check(load().lbm_adjoint_objective(h, _dev(f), _dev(target_u), _dev(target_rho), _dev(J), _dev(dJdf),
                                        _prec(f, dJdf)), h)


def lbm_adjoint_initial(h, lam0, g_rho):
    _check(load().lbm_adjoint_initial(h, _dev(lam0), _dev(g_rho), _prec(lam0)), h)


# ---- convenience ---------------------------------------------------------------------------

def make_params(**kw) -> lbm_params:
    """lbm_params from keyword values; pairs may be given as scalars."""
    p = lbm_default_params()
    for k, v in kw.items():
        if k in ("tau", "G1", "G2", "rho0", "wall_u", "rho_ref"):
            v = list(v) if hasattr(v, "__len__") else [v, v]
            arr = getattr(p, k)
            arr[0] = v[0]
            arr[1] = v[1] if len(v) > 1 else v[0]
        else:
            setattr(p, k, v)
    return p


class Lattice:
    """One simulation on the GPU: create + params + fields, with numpy I/O."""

    def __init__(self, nx, nz, n_species=1, precision=LBM_FP64, z_boundary=LBM_PERIODIC,
                 kernel=LBM_KERNEL_AUTO, device=0, stream=None, rows_per_warp=0, tile_rows=0, instances=None,
                 **params):
        """instances: heights of the lattices of a batch (nz is then their sum; walls only)."""
        d = lbm_default_desc()
        if instances is not None:
            instances = [int(h) for h in instances]
            nz = sum(instances)
            self._inst_nz = (ctypes.c_int * len(instances))(*instances)  # alive while lbm_create reads it
            d.n_instances, d.inst_nz = len(instances), self._inst_nz
        d.nx, d.nz, d.n_species, d.precision = nx, nz, n_species, precision
        d.z_boundary, d.kernel, d.device, d.rows_per_warp = z_boundary, kernel, device, rows_per_warp
        d.tile_rows = tile_rows
        d.stream = stream
        self.desc = d
        self.nx, self.nz, self.ns = nx, nz, n_species
        self.instances = instances or [nz]
        self.h = lbm_create(d)
        self.set_params(**params)

    def autotune(self, steps=20):
        """Pick the pull kernel's launch shape by timing it here; returns (depth, ms per step of
        depth 1 and 2).  The state is left as it was."""
        chosen = ctypes.c_int(0)
        ms = (ctypes.c_double * 2)()
        _check(load().lbm_autotune(self.h, steps, ctypes.byref(chosen), ms), self.h)
        return chosen.value, (ms[0], ms[1])

    def autotune_tiles(self, steps=20):
        """Pick the pull kernel's tile width and depth by timing them here; returns
        ((width, depth), ms per step of (32, 1), (32, 2), (64, 1), (64, 2)).  The state is left as
        it was."""
        width, depth = ctypes.c_int(0), ctypes.c_int(0)
        ms = (ctypes.c_double * 4)()
        _check(load().lbm_autotune_tiles(self.h, int(steps), ctypes.byref(width), ctypes.byref(depth), ms), self.h)
        return (width.value, depth.value), tuple(ms[:])

    def set_tile_shape(self, width, depth):
        _check(load().lbm_set_tile_shape(self.h, int(width), int(depth)), self.h)

    def set_instance_drive(self, i, body_force=0.0, wall_u=(0.0, 0.0)):
        _check(load().lbm_set_instance_drive(self.h, i, body_force, wall_u[0], wall_u[1]), self.h)

    def instance_observables(self, i, averages=False):
        """Observables of lattice i of the batch: scalars and its z profiles."""
        nz = self.instances[i]
        prof = dict(ux_z=np.zeros(nz), rho_z=np.zeros(self.ns * nz), sxz_z=np.zeros(nz), fluid_z=np.zeros(nz))
        o = lbm_obs()
        for k, v in prof.items():
            setattr(o, k, v.ctypes.data_as(_DP))
        _check(load().lbm_instance_observables(self.h, i, ctypes.byref(o), 1 if averages else 0), self.h)
        res = dict(mass=np.array(o.mass[:]), momentum=np.array(o.momentum[:]),
                   wall_force=np.array(o.wall_force[:]), nonfinite=bool(o.nonfinite), step=o.step,
                   samples=o.samples)
        prof["rho_z"] = prof["rho_z"].reshape(self.ns, nz)
        res.update(prof)
        return res

    def set_params(self, **params):
        self.params = make_params(**params)
        lbm_set_params(self.h, self.params)

    def set_fields(self, rho, u=None):
        if not hasattr(rho, "data_ptr"):
            rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ns, self.nz, self.nx)
            if u is not None:
                u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, self.nz, self.nx)
        lbm_set_fields(self.h, rho, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def set_populations(self, f):
        if not hasattr(f, "data_ptr"):
            f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ns, 9, self.nz, self.nx)
        lbm_set_populations(self.h, f)

    def fields(self, populations=True):
        rho = np.zeros((self.ns, self.nz, self.nx))
        u = np.zeros((2, self.nz, self.nx))
        f = np.zeros((self.ns, 9, self.nz, self.nx)) if populations else None
        lbm_get_fields(self.h, rho, u, f)
        return rho, u, f

    def _obs_struct(self):
        nz, nx = self.nz, self.nx
        prof = dict(ux_z=np.zeros(nz), rho_z=np.zeros(self.ns * nz), sxz_z=np.zeros(nz),
                    fluid_z=np.zeros(nz), ps_x=np.zeros(nx), pxx_x=np.zeros(nx))
        o = lbm_obs()
        for k, v in prof.items():
            setattr(o, k, v.ctypes.data_as(_DP))
        return o, prof

    def _obs_dict(self, o, prof):
        res = dict(mass=np.array(o.mass[:]), momentum=np.array(o.momentum[:]), gamma=o.gamma,
                   wall_force=np.array(o.wall_force[:]), nonfinite=bool(o.nonfinite), step=o.step,
                   samples=o.samples)
        prof["rho_z"] = prof["rho_z"].reshape(self.ns, self.nz)
        res.update(prof)
        return res

    def observables(self):
        o, prof = self._obs_struct()
        lbm_observables(self.h, o)
        return self._obs_dict(o, prof)

    def reader(self, depth=2):
        """An ObsReader: asynchronous, double-buffered reads of this lattice's observables."""
        return ObsReader(self, depth)

    def series(self, chunk, depth=2):
        """An ObsSeries: runs of up to `chunk` steps with every step's observables read back."""
        return ObsSeries(self, chunk, depth)

    def set_observe(self, every):
        lbm_set_observe(self.h, every)

    def averages(self, reset=False):
        o, prof = self._obs_struct()
        lbm_averages(self.h, o, reset)
        return self._obs_dict(o, prof)

    def synchronize(self):
        lbm_synchronize(self.h)

    @property
    def launches(self):
        return lbm_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ObsReader:
    """Reads of a lattice's observables that do not wait for the GPU (lbm_observables_enqueue):
    each enqueue copies a raw record into one of `depth` pinned host buffers, and result(ticket)
    waits for that record only, then unpacks it.  A buffer is reused `depth` enqueues later, so
    read each result before then."""

    def __init__(self, lat, depth=2):
        import torch

        self.lat = lat
        n = load().lbm_observables_bytes(lat.h)
        self.bufs = [torch.empty(n, dtype=torch.uint8, pin_memory=True) for _ in range(depth)]
        self.k = 0

    def enqueue(self, averages=False, reset=False):
        """averages: False (the current state), True (the time sums), or "completed" (the time
        sums without a still-pending reduction: no extra launch)."""
        t = ctypes.c_longlong()
        buf = self.bufs[self.k % len(self.bufs)]
        self.k += 1
        mode = 2 if averages == "completed" else (1 if averages else 0)
        _check(load().lbm_observables_enqueue(self.lat.h, ctypes.c_void_p(buf.data_ptr()), mode,
                                              1 if reset else 0, ctypes.byref(t)), self.lat.h)
        return (t.value, buf)

    def result(self, ticket):
        t, buf = ticket
        _check(load().lbm_wait(self.lat.h, t), self.lat.h)
        o, prof = self.lat._obs_struct()
        rc = load().lbm_observables_unpack(self.lat.h, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(o))
        if rc not in (LBM_OK, LBM_ENONFINITE):
            _check(rc, self.lat.h)
        return self.lat._obs_dict(o, prof)


class ObsSeries:
    """Time series of observables (lbm_step_read): run(n) enqueues n steps, each followed by the
    copy of its record into one of `depth` pinned host buffers of `chunk` records, in one library
    call; results(ticket) waits for that run's records and unpacks them.  A buffer is reused
    `depth` runs later, so read each run's results before then.  The unpacking targets (profile
    arrays and lbm_obs structs) are set up once per buffer."""

    def __init__(self, lat, chunk, depth=2):
        import torch

        if chunk < 1 or depth < 1:
            raise ValueError("chunk and depth must be >= 1")
        self.lat, self.chunk = lat, chunk
        self.rec = load().lbm_observables_bytes(lat.h)
        self.bufs = [torch.empty(chunk * self.rec, dtype=torch.uint8, pin_memory=True) for _ in range(depth)]
        nz, nx, ns = lat.nz, lat.nx, lat.ns
        self._out = []
        for _ in range(depth):
            prof = dict(ux_z=np.zeros((chunk, nz)), rho_z=np.zeros((chunk, ns, nz)), sxz_z=np.zeros((chunk, nz)),
                        fluid_z=np.zeros((chunk, nz)), ps_x=np.zeros((chunk, nx)), pxx_x=np.zeros((chunk, nx)))
            structs = []
            for i in range(chunk):
                o = lbm_obs()
                for k, v in prof.items():
                    setattr(o, k, v[i].ctypes.data_as(_DP))
                structs.append(o)
            self._out.append((prof, structs))
        self.k = 0

    def run(self, n, averages="completed", reset=True):
        """n (<= chunk) steps; averages as in ObsReader.enqueue, applied after every step."""
        if not 0 <= n <= self.chunk:
            raise ValueError("n must be in 0 .. chunk")
        bi = self.k % len(self.bufs)
        self.k += 1
        mode = 2 if averages == "completed" else (1 if averages else 0)
        t = ctypes.c_longlong(-1)
        _check(load().lbm_step_read(self.lat.h, n, ctypes.c_void_p(self.bufs[bi].data_ptr()), self.rec, mode,
                                    1 if reset else 0, ctypes.byref(t)), self.lat.h)
        return (t.value, bi, n)

    def results(self, ticket):
        """The run's records as observable dicts, in step order (their arrays are the run's own)."""
        t, bi, n = ticket
        if n == 0:
            return []
        lib, h = load(), self.lat.h
        _check(lib.lbm_wait(h, t), h)
        prof, structs = self._out[bi]
        base = self.bufs[bi].data_ptr()
        for i in range(n):
            rc = lib.lbm_observables_unpack(h, ctypes.c_void_p(base + i * self.rec), ctypes.byref(structs[i]))
            if rc not in (LBM_OK, LBM_ENONFINITE):
                _check(rc, h)
        run = {k: v[:n].copy() for k, v in prof.items()}  # one copy per run, not per record
        out = []
        for i in range(n):
            o = structs[i]
            res = dict(mass=np.array(o.mass[:]), momentum=np.array(o.momentum[:]), gamma=o.gamma,
                       wall_force=np.array(o.wall_force[:]), nonfinite=bool(o.nonfinite), step=o.step,
                       samples=o.samples)
            for k, v in run.items():
                res[k] = v[i]
            out.append(res)
        return out


# ---- the three-dimensional extension (include/lbm3d.h) ---------------------------------------

def lbm3_default_desc() -> lbm3_desc:
    d = lbm3_desc()
    load().lbm3_default_desc(ctypes.byref(d))
    return d


def lbm3_create(d: lbm3_desc):
    h = ctypes.c_void_p()
    _check3(load().lbm3_create(ctypes.byref(h), ctypes.byref(d)), None)
    return h


class Lattice3:
    """One three-dimensional simulation on the GPU (D3Q19, lbm3_*), with numpy I/O: fields are
    [nz][ny][nx], populations [n_species][19][nz][ny][nx]."""

    def __init__(self, nx, ny, nz, n_species=2, precision=LBM_FP32, z_boundary=LBM_PERIODIC, device=0,
                 stream=None, **params):
        d = lbm3_default_desc()
        d.nx, d.ny, d.nz, d.n_species, d.precision = nx, ny, nz, n_species, precision
        d.z_boundary, d.device, d.stream = z_boundary, device, stream
        self.desc = d
        self.nx, self.ny, self.nz, self.ns = nx, ny, nz, n_species
        self.h = lbm3_create(d)
        self.set_params(**params)

    def set_params(self, **params):
        self.params = make_params(**params)
        _check3(load().lbm3_set_params(self.h, ctypes.byref(self.params)), self.h)

    def set_fields(self, rho):
        if hasattr(rho, "data_ptr"):
            _check3(load().lbm3_set_fields(self.h, ctypes.c_void_p(rho.data_ptr()), LBM_DEVICE), self.h)
            return
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ns, self.nz, self.ny, self.nx)
        _check3(load().lbm3_set_fields(self.h, ctypes.c_void_p(rho.ctypes.data), LBM_HOST), self.h)

    def step(self, n=1):
        _check3(load().lbm3_step(self.h, int(n)), self.h)

    def fields(self, populations=True):
        """(rho [ns, nz, ny, nx], u [3, nz, ny, nx], f [ns, 19, nz, ny, nx] or None)."""
        rho = np.zeros((self.ns, self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        f = np.zeros((self.ns, 19, self.nz, self.ny, self.nx)) if populations else None
        _check3(load().lbm3_get_fields(self.h, ctypes.c_void_p(rho.ctypes.data), ctypes.c_void_p(u.ctypes.data),
                                       ctypes.c_void_p(f.ctypes.data) if f is not None else None, LBM_HOST), self.h)
        return rho, u, f

    def totals(self):
        """(mass [ns], lattice momentum [3]) of the current state, FP64 sums."""
        m = (ctypes.c_double * 2)()
        j = (ctypes.c_double * 3)()
        _check3(load().lbm3_totals(self.h, m, j), self.h)
        return np.array(m[:self.ns]), np.array(j[:])

    def synchronize(self):
        _check3(load().lbm3_synchronize(self.h), self.h)

    def step_totals(self, n, out, stride=40):
        """Advance n steps, writing each new state's totals (mass A, mass B, momentum x, y, z) as 5
        doubles every `stride` bytes from `out` (a pinned CPU or CUDA float64 tensor, or a device
        or pinned address); asynchronous, returns the ticket of the last record (wait() on it)."""
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else int(out)
        t = ctypes.c_longlong(-1)
        _check3(load().lbm3_step_totals(self.h, int(n), ctypes.c_void_p(ptr), int(stride), ctypes.byref(t)), self.h)
        return t.value

    def wait(self, ticket):
        _check3(load().lbm3_wait(self.h, int(ticket)), self.h)

    def autotune(self, steps=10):
        """Pick the collide pass's tile shape by timing each here; returns (shape, ms per step of
        each shape).  The state is left as it was."""
        chosen = ctypes.c_int(0)
        ms = (ctypes.c_double * 4)()
        _check3(load().lbm3_autotune(self.h, int(steps), ctypes.byref(chosen), ms), self.h)
        return chosen.value, tuple(ms[:])

    def set_shape(self, shape):
        _check3(load().lbm3_set_shape(self.h, int(shape)), self.h)

    def profile(self, enable):
        _check3(load().lbm3_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self):
        """(ms of the density pass, ms of the collide pass, steps) since profiling was enabled."""
        ms = (ctypes.c_double * 2)()
        n = ctypes.c_longlong(0)
        _check3(load().lbm3_profile_read(self.h, ms, ctypes.byref(n)), self.h)
        return ms[0], ms[1], n.value

    def close(self):
        if getattr(self, "h", None):
            load().lbm3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
