"""The paper's experiments run on the library (paper_1402_6019_gb300.experiments): the runs agree
with the oracle's on the same inputs, and the measurements satisfy the laws they test."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import experiments as E
from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_droplet_run_matches_oracle(oracle):
    """A Laplace droplet (R = 8, film couplings): the GPU's FP64 run and the oracle's agree."""
    R, n, steps = 8, 48, 2000
    X, Z = np.meshgrid(np.arange(n), np.arange(n))
    r = np.hypot(X - n / 2 + 0.5, Z - n / 2 + 0.5)
    rho0 = (0.29 + 0.55 * (1 - np.tanh((r - R) / 2)))[None]
    lat = L.Lattice(n, n, 1, L.LBM_FP64, L.LBM_PERIODIC, **W.FILM_PARAMS)
    lat.set_fields(rho0)
    lat.step(steps)
    ref = oracle.RefLattice(n, n, 1, 0, **W.FILM_PARAMS)
    ref.set_fields(rho0)
    ref.step(steps)
    a, b = lat.fields(populations=False)[0], ref.fields()[0]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_laplace_law_on_the_gpu():
    """Delta P R / gamma = 1 (2-D Laplace law, Sec. III) within the lattice's finite-width
    corrections, the same bar as the oracle's pin; the ratio does not drift with R."""
    res = E.laplace(radii=(8, 12, 16, 24))
    ratios = np.array([d["ratio"] for d in res["drops"]])
    assert res["gamma"] > 0
    assert np.all((ratios > 0.95) & (ratios < 1.15)), ratios
    assert np.ptp(ratios) / ratios.mean() < 0.06, ratios


def test_facing_bubbles_hold_a_film():
    """Fig. 3's set-up with the couplings of positive disjoining pressure: the film between the
    bubbles does not break, and the capillary (= disjoining) pressure is positive and falls as the
    bubbles grow."""
    a, b = E.facing_bubbles(16), E.facing_bubbles(32)
    for r in (a, b):
        assert not r["coalesced"] and r["h"] > 0 and r["Pi"] > 0
        assert r["rho_bubble"] < 0.5 < 1.0 < r["rho_liquid"]
    assert b["Pi"] < a["Pi"]


def test_couette_channel_measurements():
    r = E.couette_channel(nx=128, nz=48, steps=2000, sample_every=50, warm=500)
    assert r["samples"] == 40
    assert r["phi_mass"] == pytest.approx(r["covered"], abs=1e-5)  # mass is conserved (FP32 rounding)
    C = r["C_sigma"]
    for i, z0 in enumerate(r["z0s"]):
        assert C[i, z0] == pytest.approx(1.0, rel=1e-9)
    assert np.all(np.isfinite(r["fluid_z"])) and np.isfinite(r["zeta"]) and r["zeta"] > 0
