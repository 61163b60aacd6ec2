"""The paper's experiments as measurements on the library (Secs. III-V).

Host-side analysis of what the library computes on the GPU (observables, time averages, fields):

  bulk_pressure           Eq. BULK, the pressure of a uniform phase
  mass_packing_fraction   Phi_mass of Sec. V, from the species masses (conserved separately)
  cooperative_length      fit of a fluidity profile to the cosh law of Eq. predict
  StressCorrelator        C_sigma(z, z0) of Eq. correlator over time samples of sigma_xz(z)
  flat_tension            gamma of a flat interface (Sec. III) from a slab
  laplace                 Delta P = gamma / R for droplets (Sec. III)
  facing_bubbles          two facing bubbles and the liquid film between them (Fig. 3): film
                          width h and capillary pressure, which mechanical equilibrium makes
                          the disjoining pressure Pi(h)
  couette_channel         a sheared emulsion channel (Sec. V, Fig. 6): time-averaged fluidity
                          f(z), the stress correlator, Phi_mass

Every lattice step runs in the library; this module sets up states, reads observables and
fields, and does the (small) arithmetic of the analysis in FP64 NumPy.
"""
from __future__ import annotations

import time

import numpy as np

from . import lbm as L
from . import workloads as W

CS2 = 1.0 / 3.0


# ------------------------------------------------------------------------------------------------
# analysis (no GPU)
# ------------------------------------------------------------------------------------------------

def psi_of(rho, psi_form=0, rho0=1.0):
    """The pseudopotential of Sec. IV: 1 - exp(-rho / rho0), or rho."""
    rho = np.asarray(rho, dtype=float)
    return rho if psi_form == 1 else 1.0 - np.exp(-rho / rho0)


def bulk_pressure(rho, G1, G2, weight_norm=W.WEIGHT_NORM, psi_form=0, rho0=1.0):
    """Eq. BULK for one component: P = c_s^2 rho + (G1 + G2) psi^2 / 2 times the second moment of
    the interaction weights (sum W c_x^2 = weight_norm for the tables of Appendix B scaled by
    weight_norm)."""
    psi = psi_of(rho, psi_form, rho0)
    return CS2 * np.asarray(rho, dtype=float) + weight_norm * (G1 + G2) * 0.5 * psi ** 2


def mass_packing_fraction(mass_a, volume, rho_a_dispersed, rho_a_continuous):
    """Phi_mass of Sec. V: the volume fraction of the dispersed (A-rich) phase that the mass of
    species A implies, (M_A / V - rho_A^c) / (rho_A^d - rho_A^c), with rho_A^d, rho_A^c the A
    densities of the A-rich and B-rich phases.  Mass is conserved by each species, so it is fixed
    by the initial state, while the volume of a phase is blurred by the interfaces."""
    return (mass_a / volume - rho_a_continuous) / (rho_a_dispersed - rho_a_continuous)


def cosh_law(z, H, zeta, f_b, f_w):
    """Eq. predict: f(z) = f_b + (f_w - f_b) cosh((z - H/2) / zeta) / cosh(H / (2 zeta)).  z is the
    distance from the wall at 0; the other wall is at H.  The ratio of the cosh functions is
    formed as (e^(u - v) + e^(-u - v)) / (1 + e^(-2v)), u = (z - H/2) / zeta, v = H / (2 zeta),
    which does not overflow for small zeta."""
    z = np.asarray(z, dtype=float)
    v = 0.5 * H / zeta
    u = (z - 0.5 * H) / zeta
    ratio = (np.exp(u - v) + np.exp(-u - v)) / (1.0 + np.exp(-2.0 * v))
    return f_b + (f_w - f_b) * ratio


def cooperative_length(z, f, H, f_w=None, zeta_range=(0.05, None), tol=1e-10):
    """Fit Eq. predict to a fluidity profile f(z): returns (zeta, f_b, f_w, rms residual).

    For a fixed zeta the law is linear in f_b and f_w, f = f_b (1 - g) + f_w g with g the cosh
    ratio, so both have closed-form least-squares values (f_w is held at the given value if one is
    given: the paper measures the wall fluidity directly); zeta minimises the residual by a
    golden-section search on log(zeta) over zeta_range (upper bound default 10 H)."""
    z = np.asarray(z, dtype=float)
    f = np.asarray(f, dtype=float)
    lo, hi = zeta_range[0], zeta_range[1] if zeta_range[1] is not None else 10.0 * H

    def fit(zeta):
        g = cosh_law(z, H, zeta, 0.0, 1.0)
        a = 1.0 - g
        if f_w is not None:
            r0 = f - f_w * g
            den = float(a @ a)
            fb = float(a @ r0) / den if den > 0 else float(np.mean(f))
            fw = float(f_w)
        else:
            M = np.stack([a, g], axis=1)
            (fb, fw), *_ = np.linalg.lstsq(M, f, rcond=None)
        res = f - fb * a - fw * g
        return float(res @ res), float(fb), float(fw)

    a, b = np.log(lo), np.log(hi)
    gr = 0.5 * (np.sqrt(5.0) - 1.0)
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = fit(np.exp(c))[0], fit(np.exp(d))[0]
    while b - a > tol:
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = fit(np.exp(c))[0]
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = fit(np.exp(d))[0]
    zeta = float(np.exp(0.5 * (a + b)))
    ss, fb, fw = fit(zeta)
    return zeta, fb, fw, float(np.sqrt(ss / len(f)))


class StressCorrelator:
    """Eq. correlator: C(z, z0) = (<s(z0) s(z)> - <s(z0)><s(z)>) / (<s(z0)^2> - <s(z0)>^2) over
    time samples s(z) of the x-averaged shear stress profile, for the reference rows z0."""

    def __init__(self, nz, z0s):
        self.z0s = [int(z) for z in z0s]
        self.n = 0
        self.s1 = np.zeros(nz)
        self.s2 = np.zeros((len(self.z0s), nz))

    def add(self, s):
        s = np.asarray(s, dtype=float)
        self.n += 1
        self.s1 += s
        self.s2 += s[self.z0s][:, None] * s[None, :]

    def result(self):
        """C [len(z0s), nz]."""
        m = self.s1 / self.n
        cov = self.s2 / self.n - m[self.z0s][:, None] * m[None, :]
        var = np.array([cov[i, z0] for i, z0 in enumerate(self.z0s)])
        return cov / var[:, None]


def interface_positions(profile, level):
    """Sub-cell positions where a 1-D profile crosses `level` (linear interpolation)."""
    p = np.asarray(profile, dtype=float) - level
    idx = np.nonzero(np.sign(p[:-1]) != np.sign(p[1:]))[0]
    return idx + p[idx] / (p[idx] - p[idx + 1])


# ------------------------------------------------------------------------------------------------
# experiments (library on the GPU)
# ------------------------------------------------------------------------------------------------

def _pb(rho, p):
    return bulk_pressure(rho, p["G1"][0], p["G2"][0], p["weight_norm"], p.get("psi_form", 0), p["rho0"][0])


def _film_lattice(nx, nz, precision, **params):
    return L.Lattice(nx, nz, 1, precision, L.LBM_PERIODIC, **dict(W.FILM_PARAMS, **params))


def flat_tension(nx=128, steps=20000, precision=L.LBM_FP64, **params):
    """gamma of one flat interface of the film couplings (Sec. III): a slab (liquid between two
    flat interfaces, periodic), relaxed; the library's gamma sums P_xx - P_zz over both."""
    p = dict(W.FILM_PARAMS, **params)
    lat = _film_lattice(nx, 2, precision, **params)
    x = np.arange(nx)
    prof = 0.29 + 0.55 * (np.tanh((x - nx / 4) / 3) - np.tanh((x - 3 * nx / 4) / 3))
    lat.set_fields(np.tile(prof, (1, 2, 1)))
    lat.step(steps)
    o = lat.observables()
    rho = lat.fields(populations=False)[0][0, 0]
    return dict(gamma=o["gamma"] / 2.0, rho_liquid=float(rho[nx // 2]), rho_vapour=float(rho[0]),
                p_liquid=float(_pb(rho[nx // 2], p)), p_vapour=float(_pb(rho[0], p)))


def laplace(radii=(8, 12, 16, 24), margin=32, steps=20000, precision=L.LBM_FP64, gamma=None, **params):
    """Delta P = gamma / R in 2-D (Sec. III): a liquid droplet of each radius in a periodic box,
    relaxed; P inside and outside from Eq. BULK at the centre and the corner, R from the droplet's
    mass.  Returns per radius (R, Delta P, Delta P R / gamma)."""
    p = dict(W.FILM_PARAMS, **params)
    if gamma is None:
        gamma = flat_tension(precision=precision, **params)["gamma"]
    out = []
    for R in radii:
        n = 2 * R + margin
        X, Z = np.meshgrid(np.arange(n), np.arange(n))
        r = np.hypot(X - n / 2 + 0.5, Z - n / 2 + 0.5)
        lat = _film_lattice(n, n, precision, **params)
        lat.set_fields((0.29 + 0.55 * (1 - np.tanh((r - R) / 2)))[None])
        lat.step(steps)
        rho = lat.fields(populations=False)[0][0]
        rin, rout = rho[n // 2, n // 2], rho[0, 0]
        Re = float(np.sqrt((rho - rout).sum() / (rin - rout) / np.pi))
        dP = float(_pb(rin, p) - _pb(rout, p))
        out.append(dict(R=Re, dP=dP, ratio=dP * Re / gamma))
    return dict(gamma=gamma, drops=out)


def facing_bubbles(R, h0=4, pad=24, steps=30000, precision=L.LBM_FP64, **params):
    """Two bubbles (vapour discs of radius R) facing each other across a liquid film of initial
    width h0, fully periodic, relaxed (Fig. 3).  With couplings of positive disjoining pressure the
    film holds.  Measured: the film width h along the line of centres (between the two
    interfaces, at the mid density), the bubble and liquid pressures (Eq. BULK at a bubble centre
    and far from the bubbles) and the capillary pressure Pi = P_bubble - P_liquid, which in
    mechanical equilibrium equals the disjoining pressure of the film."""
    p = dict(W.FILM_PARAMS, **params)
    nx = 4 * R + h0 + 2 * pad
    nz = 2 * R + 2 * pad
    X, Z = np.meshgrid(np.arange(nx) + 0.5, np.arange(nz) + 0.5)
    cz = nz / 2
    c1, c2 = nx / 2 - h0 / 2 - R, nx / 2 + h0 / 2 + R
    d = np.minimum(np.hypot(X - c1, Z - cz), np.hypot(X - c2, Z - cz))
    rho = 0.29 + 0.55 * (1 + np.tanh((d - R) / 2))   # liquid (1.39) outside, vapour (0.29) inside
    lat = _film_lattice(nx, nz, precision, **params)
    lat.set_fields(rho[None])
    lat.step(steps)
    rho = lat.fields(populations=False)[0][0]
    line = rho[nz // 2]
    rv, rl = float(rho[nz // 2, int(c1)]), float(rho[0, 0])
    cross = interface_positions(line, 0.5 * (rv + rl))
    mid = nx / 2
    inner = [c for c in cross if abs(c - mid) < R]
    h = float(max(inner) - min(inner)) if len(inner) >= 2 else 0.0
    Pb, Pl = float(_pb(rv, p)), float(_pb(rl, p))
    return dict(R=R, h=h, film_density=float(line[int(mid)]), rho_bubble=rv, rho_liquid=rl,
                p_bubble=Pb, p_liquid=Pl, Pi=Pb - Pl, coalesced=len(inner) < 2)


def couette_channel(nx=512, nz=128, u_wall=0.01, fraction=0.8, steps=100000, sample_every=100,
                    warm=20000, precision=L.LBM_FP32, seed=1402, z0s=None, **params):
    """A sheared emulsion channel (Sec. V, Fig. 6): the emulsion's couplings, walls moving at
    -+u_wall, a seeded disk packing; after `warm` steps, observables every `sample_every` steps.
    Returns the time-averaged profiles (u_x, sigma_xz, fluidity f = (d u_x / dz) / sigma_xz),
    the cooperative-length fit of f, the stress correlator at z0s (default H/2 and H/5) and
    Phi_mass."""
    p = dict(W.EMULSION_PARAMS, wall_u=(-u_wall, u_wall), **params)
    rho, covered = W.disk_packing(nx, nz, fraction, seed, periodic_z=False)
    lat = L.Lattice(nx, nz, 2, precision, L.LBM_BOUNCEBACK, **p)
    lat.set_fields(rho)
    t0 = time.perf_counter()
    lat.step(warm)
    z0s = z0s if z0s is not None else [nz // 2, nz // 5]
    corr = StressCorrelator(nz, z0s)
    lat.set_observe(sample_every)
    left = steps
    while left > 0:
        k = min(sample_every, left)
        lat.step(k)
        left -= k
        corr.add(lat.observables()["sxz_z"])
    avg = lat.averages()
    lat.synchronize()
    wall = time.perf_counter() - t0
    z = np.arange(nz) + 0.5  # distance from the wall at z = -1/2
    zeta, f_b, f_w, rms = cooperative_length(z, avg["fluid_z"], float(nz))
    mass = avg["mass"]
    phi = mass_packing_fraction(mass[0], nx * nz, 1.2, 0.05)
    return dict(nx=nx, nz=nz, steps=warm + steps, samples=avg["samples"], wall_s=wall,
                mlups=nx * nz * (warm + steps) / wall / 1e6, phi_mass=float(phi), covered=covered,
                ux_z=avg["ux_z"], sxz_z=avg["sxz_z"], fluid_z=avg["fluid_z"],
                zeta=zeta, f_b=f_b, f_w=f_w, fit_rms=rms, z0s=z0s, C_sigma=corr.result())


def report(mode="default"):
    """Run the suite on the GPU and return its measurements (JSON-able).  mode: "quick" (small),
    "default", or "long" (adds sheared emulsions at the paper's size, 1040 x 1040, G_AB = 0.587,
    a million steps each)."""
    t0 = time.perf_counter()
    quick = mode == "quick"
    out = {}
    ft = flat_tension()
    out["flat_tension"] = ft
    radii = (8, 12, 16) if quick else (8, 12, 16, 24, 32, 48)
    out["laplace"] = laplace(radii=radii, gamma=ft["gamma"])
    bubbles = (12, 16) if quick else (12, 16, 24, 32, 48, 64)
    out["facing_bubbles"] = [facing_bubbles(R) for R in bubbles]
    jsonable = lambda r: {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in r.items()}
    runs = []
    for frac in ((0.55,) if quick else (0.55, 0.65, 0.75)):
        runs.append(jsonable(couette_channel(fraction=frac, steps=20000 if quick else 200000,
                                             warm=5000 if quick else 50000)))
    out["couette"] = runs
    if mode == "long":
        out["couette_1040"] = [jsonable(couette_channel(nx=1040, nz=1040, fraction=frac, G_AB=0.587, warm=200000,
                                                        steps=1000000, sample_every=1000))
                               for frac in (0.55, 0.61)]
    out["wall_s"] = time.perf_counter() - t0
    return out


if __name__ == "__main__":
    import json
    import sys

    print(json.dumps(report("quick" if "--quick" in sys.argv else "long" if "--long" in sys.argv else "default")))
