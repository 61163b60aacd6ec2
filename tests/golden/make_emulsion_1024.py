"""Writes tests/golden/emulsion_1024_1000.npz: the FP64 oracle's state of the 1024 x 1024 emulsion
workload after 1000 steps, at a fixed sample of sites, and its observables at that step.

Calls only the oracle (``oracle/``) and the seeded input generator (``workloads``); nothing here
comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_emulsion_1024.py

The run is 10^9 site updates of the plain FP64 oracle (minutes on a many-core host).

Sampled sites: three whole rows (z = 0, 511, 1023), two whole columns (x = 0, 700) and 8192 sites
drawn from SplitMix64 stream 1405, every site of the lattice equally likely.  Stored per site:
rho_A, rho_B and the barycentric velocity (u_x, u_z) of Sec. II (u = sum_s (j_s + F_s/2) /
sum_s rho_s).  Stored observables (Secs. III-IV): masses, momenta, gamma, the profiles
ux_z, rho_z, sxz_z, fluid_z, ps_x, pxx_x, and the magnitudes of RefLattice.scales() (max rho,
max |u|, the population and stress scales the observables are formed from).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1402_6019_gb300 import workloads as W  # noqa: E402

STEPS = 1000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emulsion_1024_1000.npz")


def sample_sites(nx, nz):
    zs, xs = [], []
    for z in (0, nz // 2 - 1, nz - 1):
        zs.append(np.full(nx, z))
        xs.append(np.arange(nx))
    for x in (0, 700):
        zs.append(np.arange(nz))
        xs.append(np.full(nz, x))
    r = W.splitmix64(1405, 8192)
    k = (r % np.uint64(nx * nz)).astype(np.int64)
    zs.append(k // nx)
    xs.append(k % nx)
    return np.concatenate(zs).astype(np.int32), np.concatenate(xs).astype(np.int32)


def main():
    w = W.workload("emulsion_1024")
    nx, nz = w["nx"], w["nz"]
    O.build()
    ref = O.RefLattice(nx, nz, 2, w["z_boundary"], **w["params"])
    ref.set_fields(w["rho"])
    t = time.time()
    ref.step(STEPS)
    dt = time.time() - t
    rho, u, _ = ref.fields()
    obs = ref.observables()
    sc = ref.scales()
    sz, sx = sample_sites(nx, nz)
    np.savez_compressed(
        OUT, steps=STEPS, z=sz, x=sx, rho=rho[:, sz, sx], u=u[:, sz, sx],
        **sc,
        mass=obs["mass"], momentum=obs["momentum"], gamma=obs["gamma"],
        ux_z=obs["ux_z"], rho_z=obs["rho_z"], sxz_z=obs["sxz_z"], fluid_z=obs["fluid_z"],
        ps_x=obs["ps_x"], pxx_x=obs["pxx_x"])
    print(f"wrote {OUT}: {len(sz)} sites, oracle {nx * nz * STEPS / dt / 1e6:.2f} MLUPS")


if __name__ == "__main__":
    main()
