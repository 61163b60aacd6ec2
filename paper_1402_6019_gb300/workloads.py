"""Seeded synthetic inputs shared by the CUDA path and its checker.

This module holds no arithmetic of the method: it only draws density fields.  Both the library
(tests, bench) and the oracle take their initial densities from here, so no random number is
ever drawn on either side of the comparison.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: draw i of stream `seed` is the
SplitMix64 output mix(seed + (i + 1) * 0x9E3779B97F4A7C15).  It is written out here so the
streams are identical on every machine and numpy version.

The workloads stand in for the paper's emulsions (Sec. IV: A-rich droplets at rho ~ 1.2 in a
B-rich matrix and vice versa, Fig. 4) and for the single-component tests of Secs. II-III.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def noise_field(nx: int, nz: int, seed: int, mean: float = 1.0, amp: float = 0.01,
                n_species: int = 1) -> np.ndarray:
    """rho [n_species, nz, nx] = mean + U(-amp, amp), one independent draw per site."""
    u = uniform(seed, n_species * nz * nx).reshape(n_species, nz, nx)
    return mean + amp * (2.0 * u - 1.0)


def disk_packing(nx: int, nz: int, fraction: float, seed: int, r_mean: float = 12.0,
                 r_spread: float = 3.0, rho_in: float = 1.2, rho_out: float = 0.05,
                 periodic_z: bool = True, max_disks: int = 1_000_000):
    """Two-species density fields of a random polydisperse disk packing.

    Disks with uniform radius in [r_mean - r_spread, r_mean + r_spread] and uniform centres are
    added one at a time (overlap allowed) until the covered area reaches `fraction`; random
    sequential addition without overlap jams near 0.55, below the packings asked for.  Inside a
    disk (rho_A, rho_B) = (rho_in, rho_out), outside (rho_out, rho_in).  Periodic in x; in z
    periodic, or clipped by walls.  Returns (rho [2, nz, nx], achieved covered fraction).
    """
    if not (0.0 <= fraction < 1.0):
        raise ValueError("fraction must be in [0, 1)")
    covered = np.zeros((nz, nx), dtype=bool)
    target = fraction * nx * nz
    count = 0
    k = 0
    while count < target and k < max_disks:
        u = uniform(seed, 3, offset=3 * k)
        cx, cz = u[0] * nx, u[1] * nz
        r = r_mean + r_spread * (2.0 * u[2] - 1.0)
        # the disk's bounding box (periodic images in x, and in z when periodic)
        ix = np.arange(int(np.floor(cx - r)), int(np.ceil(cx + r)) + 1)
        iz = np.arange(int(np.floor(cz - r)), int(np.ceil(cz + r)) + 1)
        if not periodic_z:
            iz = iz[(iz >= 0) & (iz < nz)]
        xw, zw = ix % nx, iz % nz
        # distance to the nearest image, as on the full grid
        dx = np.minimum(np.abs(xw - cx), nx - np.abs(xw - cx))
        if periodic_z:
            dz = np.minimum(np.abs(zw - cz), nz - np.abs(zw - cz))
        else:
            dz = np.abs(zw - cz)
        inside = (dz[:, None] ** 2 + dx[None, :] ** 2) <= r * r
        xu, first = np.unique(xw, return_index=True)
        zu, zfirst = np.unique(zw, return_index=True)
        inside = inside[zfirst][:, first]
        sub = covered[np.ix_(zu, xu)]
        count += int(np.count_nonzero(inside & ~sub))
        covered[np.ix_(zu, xu)] = sub | inside
        k += 1
    rho = np.empty((2, nz, nx))
    rho[0] = np.where(covered, rho_in, rho_out)
    rho[1] = np.where(covered, rho_out, rho_in)
    return rho, float(covered.mean())


def sphere_packing(nx: int, ny: int, nz: int, fraction: float, seed: int, r_mean: float = 8.0,
                   r_spread: float = 2.0, rho_in: float = 1.2, rho_out: float = 0.05, periodic_z: bool = True,
                   max_spheres: int = 1_000_000):
    """Two-species density fields [2, nz, ny, nx] of a random polydisperse sphere packing, the
    three-dimensional counterpart of disk_packing: spheres of uniform radius in
    [r_mean - r_spread, r_mean + r_spread] with uniform centres, overlap allowed, added until the
    covered volume reaches `fraction`; (rho_A, rho_B) = (rho_in, rho_out) inside, swapped outside.
    Periodic in x and y; in z periodic or clipped by walls.  Returns (rho, covered fraction)."""
    if not (0.0 <= fraction < 1.0):
        raise ValueError("fraction must be in [0, 1)")
    covered = np.zeros((nz, ny, nx), dtype=bool)
    target = fraction * nx * ny * nz
    count = 0
    k = 0
    while count < target and k < max_spheres:
        u = uniform(seed, 4, offset=4 * k)
        cx, cy, cz = u[0] * nx, u[1] * ny, u[2] * nz
        r = r_mean + r_spread * (2.0 * u[3] - 1.0)
        ax = [np.arange(int(np.floor(c - r)), int(np.ceil(c + r)) + 1) for c in (cx, cy, cz)]
        if not periodic_z:
            ax[2] = ax[2][(ax[2] >= 0) & (ax[2] < nz)]
        ix, iy, iz = ax[0] % nx, ax[1] % ny, ax[2] % nz
        dx = np.minimum(np.abs(ix - cx), nx - np.abs(ix - cx))
        dy = np.minimum(np.abs(iy - cy), ny - np.abs(iy - cy))
        dz = np.minimum(np.abs(iz - cz), nz - np.abs(iz - cz)) if periodic_z else np.abs(iz - cz)
        inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) <= r * r
        xu, fx = np.unique(ix, return_index=True)
        yu, fy = np.unique(iy, return_index=True)
        zu, fz = np.unique(iz, return_index=True)
        inside = inside[np.ix_(fz, fy, fx)]
        sub = covered[np.ix_(zu, yu, xu)]
        count += int(np.count_nonzero(inside & ~sub))
        covered[np.ix_(zu, yu, xu)] = sub | inside
        k += 1
    rho = np.empty((2, nz, ny, nx))
    rho[0] = np.where(covered, rho_in, rho_out)
    rho[1] = np.where(covered, rho_out, rho_in)
    return rho, float(covered.mean())


# Normalisation of the interaction weights: Appendix B's tables satisfy sum W c c = 1, while
# Eq. BULK (P_b = c_s^2 rho + c_s^2 (G1 + G2) psi^2 / 2) implies sum W c c = c_s^2.  The paper's
# couplings only give stable phases near its printed densities under the latter, so every
# interaction weight is scaled by c_s^2 = 1/3.
WEIGHT_NORM = 1.0 / 3.0

# Couplings of the paper's emulsion (Sec. IV): G_AA = (-9.0, 8.1), G_BB = (-8.0, 7.1),
# psi = 1 - exp(-rho/0.83).  The 1024^2 workload uses G_AB = 0.405; the paper's flow runs 0.587.
EMULSION_PARAMS = dict(tau=(1.0, 1.0), G1=(-9.0, -8.0), G2=(8.1, 7.1), G_AB=0.405,
                       psi_form=0, rho0=(0.83, 0.83), weight_norm=WEIGHT_NORM)

# Single-component frustrated couplings of Secs. III-IV with psi = 1 - exp(-rho).
SINGLE_PARAMS = dict(tau=(1.0, 1.0), G1=(-9.0, -9.0), G2=(8.1, 8.1), psi_form=0,
                     rho0=(1.0, 1.0), weight_norm=WEIGHT_NORM)

# Phase-separating single-component couplings of the thin-film test (Sec. III, Fig. 3).
FILM_PARAMS = dict(tau=(1.0, 1.0), G1=(-20.4, -20.4), G2=(16.0, 16.0), psi_form=0,
                   rho0=(1.0, 1.0), weight_norm=WEIGHT_NORM)


def workload(name: str, seed: int = 1402):
    """Named workloads: returns dict(nx, nz, n_species, z_boundary, params, rho, note)."""
    if name == "single_128":
        rho = noise_field(128, 128, seed)
        return dict(nx=128, nz=128, n_species=1, z_boundary=0, params=dict(SINGLE_PARAMS),
                    rho=rho, note="128x128 periodic, rho = 1 + U(-0.01, 0.01)")
    if name == "emulsion_1024":
        rho, frac = disk_packing(1024, 1024, 0.8, seed)
        return dict(nx=1024, nz=1024, n_species=2, z_boundary=0, params=dict(EMULSION_PARAMS),
                    rho=rho, note=f"1024x1024 periodic disk packing, covered {frac:.3f}")
    if name.startswith("emulsion_"):  # emulsion_N: an N x N lattice of the same emulsion
        n = int(name.split("_")[1])
        rho, frac = disk_packing(n, n, 0.8, seed)
        return dict(nx=n, nz=n, n_species=2, z_boundary=0, params=dict(EMULSION_PARAMS),
                    rho=rho, note=f"{n}x{n} periodic disk packing, covered {frac:.3f}")
    if name in ("channel_couette", "channel_poiseuille"):
        rho, frac = disk_packing(2048, 256, 0.85, seed, periodic_z=False)
        p = dict(EMULSION_PARAMS)
        if name == "channel_couette":
            p["wall_u"] = (-0.01, 0.01)
        else:
            p["body_force"] = 1e-6
        return dict(nx=2048, nz=256, n_species=2, z_boundary=1, params=p, rho=rho,
                    note=f"2048x256 walled channel, packing {frac:.3f}")
    if name == "channel_sweep_48":
        # the width and drive sweep behind the cooperative-length analysis (Sec. V): channels of
        # height H = 32, 64, ..., 512 and length 1024, each under body forces 1e-6, 3e-6, 1e-5,
        # every channel with its own seeded packing at fraction 0.85
        heights, drives, rhos = [], [], []
        for k, h in enumerate(range(32, 513, 32)):
            for j, g in enumerate((1e-6, 3e-6, 1e-5)):
                r, _ = disk_packing(1024, h, 0.85, seed + 97 * k + j, periodic_z=False)
                heights.append(h)
                drives.append(dict(body_force=g, wall_u=(0.0, 0.0)))
                rhos.append(r)
        return dict(nx=1024, nz=sum(heights), n_species=2, z_boundary=1, params=dict(EMULSION_PARAMS),
                    rho=np.concatenate(rhos, axis=1), instances=heights, drives=drives,
                    note="48 walled channels, 1024 x (32, 64, ..., 512) x 3 body forces, packing 0.85")
    if name == "adjoint_256":
        # calibration run: the emulsion on a 256 x 256 periodic lattice under a body force,
        # 500 steps, scored against seeded target profiles across the lattice (a velocity of the
        # order the drive reaches, a density of species A between the two phases' values)
        rho, frac = disk_packing(256, 256, 0.8, seed)
        return dict(nx=256, nz=256, n_species=2, z_boundary=0, params=dict(EMULSION_PARAMS, body_force=1e-5),
                    rho=rho, steps=500, checkpoint=25,
                    target_u=1e-3 * uniform(seed + 1, 256), target_rho=0.3 + 0.6 * uniform(seed + 2, 256),
                    note=f"256x256 periodic disk packing, covered {frac:.3f}, body force 1e-5, 500 steps")
    if name.startswith("emulsion3d_"):  # emulsion3d_N: an N^3 periodic A/B emulsion (3-D extension)
        n = int(name.split("_")[1])
        rho, frac = sphere_packing(n, n, n, 0.5, seed)
        return dict(nx=n, ny=n, nz=n, n_species=2, z_boundary=0, params=dict(EMULSION_PARAMS), rho=rho, dim=3,
                    note=f"{n}^3 periodic sphere packing, covered {frac:.3f}, radii 8 +- 2")
    raise KeyError(name)
