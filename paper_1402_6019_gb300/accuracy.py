"""Stated error bounds of the library's observables against an FP64 reference of the same state.

Host arithmetic only (no method arithmetic): it compares two sets of observables, as returned by
``Lattice.observables()`` for the library and by the FP64 oracle for the reference, and states
for each one the error its inputs allow.

The state contract is a relative L-inf error ``tol`` on rho and u (1e-12 in FP64 mode, 1e-4 in
FP32 mode after 1000 steps).  An observable formed from per-site terms inherits that error
relative to the size of the terms it is formed from, not to its own size: the shear stress S_xz
of Sec. IV and the p_s = P_xx - P_zz of Sec. III are small differences of O(1) pressure-tensor
terms, and a velocity near rest is a small difference of populations.  So each bound is ``tol``
times the magnitude of the terms (``scales``, computed from the reference state):

============  ==========================================================================
observable    bound on max |library - reference|
============  ==========================================================================
mass          tol * |mass_s|                          (sum of positive terms)
momentum      total mass * bound_u                    (sum over sites of rho * u errors)
ux_z          bound_u = tol * u_max + 100 eps * pop_scale   (x-average of per-site u)
rho_z         tol * rho_max
sxz_z         tol * stress_scale                      (x-average of per-site S_xz)
ps_x, pxx_x   tol * stress_scale                      (z-average of per-site P terms)
gamma         nx * tol * stress_scale                 (sum over x of ps_x)
wall_force    tol * rho_max * pop_scale               (x-average of populations crossing)
fluid_z       (2 bound_u + |f| tol * stress_scale) / (|S_xz| - tol * stress_scale)
              where |S_xz| exceeds its own bound (elsewhere the ratio is undetermined)
============  ==========================================================================

eps is the unit roundoff of FP64 (both sides carry it in FP64 mode; the FP32 contract dwarfs
it).  ``observable_errors`` also reports each error relative to the observable's own largest
value, which is what the measured-error tables quote.
"""
from __future__ import annotations

import numpy as np

EPS64 = 2.0 ** -52
PROFILES = ("ux_z", "rho_z", "sxz_z", "fluid_z", "ps_x", "pxx_x")
SCALARS = ("mass", "momentum", "gamma", "wall_force")


def observable_errors(lib: dict, ref: dict, scales: dict, tol: float, nx: int, total_mass: float) -> dict:
    """{name: (max abs error, bound, relative error, entries checked)} for every observable of
    ``ref``.  The relative error is the error over the observable's own largest value, except
    for the total momentum, whose own value is near zero: there it is over total mass * u_max.
    The fluidity is checked only where |S_xz| exceeds twice its own bound (elsewhere the ratio
    is undetermined at this tolerance); its count of checked entries can be 0.

    ``scales``: rho_max, u_max, pop_scale, stress_scale of the reference state (the oracle's
    ``RefLattice.scales()``); ``tol``: the state contract's relative tolerance."""
    bound_u = tol * scales["u_max"] + 100 * EPS64 * scales["pop_scale"]
    bound_s = tol * scales["stress_scale"]
    bounds = {
        "mass": tol * np.abs(np.asarray(ref["mass"], float)),
        "momentum": total_mass * bound_u,
        "ux_z": bound_u,
        "rho_z": tol * scales["rho_max"],
        "sxz_z": bound_s,
        "ps_x": bound_s,
        "pxx_x": bound_s,
        "gamma": nx * bound_s,
        "wall_force": tol * scales["rho_max"] * scales["pop_scale"],
    }
    out = {}
    for k, b in bounds.items():
        if k not in ref or k not in lib:
            continue
        r = np.asarray(ref[k], float)
        d = np.abs(np.asarray(lib[k], float).reshape(r.shape) - r)
        own = total_mass * scales["u_max"] if k == "momentum" else (float(np.abs(r).max()) if r.size else 0.0)
        if np.ndim(b):  # per-entry bounds (mass): the entry with the worst ratio
            i = int(np.argmax(d / np.maximum(b, 1e-300)))
            err, bb = float(d.reshape(-1)[i]), float(np.asarray(b).reshape(-1)[i])
        else:
            err, bb = (float(d.max()) if d.size else 0.0), float(b)
        out[k] = (err, bb, float(d.max()) / own if own > 0 else 0.0, int(d.size))
    if "fluid_z" in ref and "fluid_z" in lib and "sxz_z" in ref:
        s = np.abs(np.asarray(ref["sxz_z"], float))
        f = np.asarray(ref["fluid_z"], float)
        ok = s > 2 * bound_s
        d = np.abs(np.asarray(lib["fluid_z"], float) - f)
        if ok.any():
            bz = (2 * bound_u + np.abs(f) * bound_s) / (s - bound_s)
            i = int(np.argmax(np.where(ok, d / bz, -1.0)))
            own = float(np.abs(f[ok]).max())
            out["fluid_z"] = (float(d[i]), float(bz[i]), float(d[ok].max()) / own if own > 0 else 0.0,
                              int(ok.sum()))
        else:
            out["fluid_z"] = (0.0, float("inf"), 0.0, 0)
    return out


def check(errors: dict) -> list:
    """Names of the observables whose error exceeds its bound."""
    return [k for k, e in errors.items() if not e[0] <= e[1]]
