"""Pins of the host-side analysis of the paper's experiments (paper_1402_6019_gb300.experiments),
each against something other than its own formula: the differential equation the cosh law
solves, closed-form correlations, the packing the masses come from, and the oracle's pressure
tensor."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import experiments as E
from paper_1402_6019_gb300 import workloads as W


@pytest.mark.parametrize("zeta", [2.0, 17.3, 60.0, 300.0])
def test_cosh_law_solves_the_fluidity_equation(zeta):
    """Eq. fluidity: zeta^2 f'' = f - f_b, with f = f_w at both walls (z = 0, H)."""
    H, fb, fw = 128.0, 0.002, 0.05
    h = 0.01 * zeta  # truncation error ~ (h / zeta)^2 / 12
    z = np.linspace(0.5, H - 0.5, 41)
    f = lambda t: E.cosh_law(t, H, zeta, fb, fw)
    d2 = (f(z + h) - 2 * f(z) + f(z - h)) / h ** 2
    assert np.allclose(zeta ** 2 * d2, f(z) - fb, rtol=1e-5, atol=1e-9 * fw)
    assert E.cosh_law(np.array([0.0, H]), H, zeta, fb, fw) == pytest.approx([fw, fw], rel=1e-12)


@pytest.mark.parametrize("zeta", [3.0, 17.3, 68.0])
def test_cooperative_length_recovers_the_parameters(zeta):
    H = 128.0
    z = np.arange(128) + 0.5
    f = E.cosh_law(z, H, zeta, 0.002, 0.05)
    got = E.cooperative_length(z, f, H)
    assert got[0] == pytest.approx(zeta, rel=1e-7)
    assert got[1] == pytest.approx(0.002, rel=1e-6)
    assert got[2] == pytest.approx(0.05, rel=1e-7)
    assert got[3] < 1e-10
    # with the wall fluidity given, as the paper measures it
    assert E.cooperative_length(z, f, H, f_w=0.05)[0] == pytest.approx(zeta, rel=1e-7)
    # noise: the estimate stays close
    noisy = f * (1 + 1e-3 * np.random.default_rng(0).standard_normal(f.size))
    assert E.cooperative_length(z, noisy, H)[0] == pytest.approx(zeta, rel=0.05)


def test_stress_correlator_closed_forms():
    rng = np.random.default_rng(1)
    nz, n = 40, 4000
    v = 1.0 + np.sin(np.arange(nz) / 5.0)
    c = np.linspace(-1, 1, nz)
    C = E.StressCorrelator(nz, [nz // 2, nz // 5])
    X = rng.standard_normal(n)
    for t in range(n):  # one mode: s = X_t v(z) + c(z)  ->  C(z, z0) = v(z) / v(z0)
        C.add(X[t] * v + c)
    got = C.result()
    for i, z0 in enumerate(C.z0s):
        assert np.allclose(got[i], v / v[z0], rtol=1e-8)
    # independent rows: C(z0, z0) = 1 and C(z, z0) ~ 0
    D = E.StressCorrelator(nz, [nz // 2])
    for t in range(n):
        D.add(rng.standard_normal(nz))
    got = D.result()[0]
    assert got[nz // 2] == pytest.approx(1.0, rel=1e-12)
    others = np.delete(got, nz // 2)
    assert np.abs(others).max() < 5.0 / np.sqrt(n)


def test_mass_packing_fraction_is_the_packing_fraction():
    """For the synthetic packings (rho_A = 1.2 in the disks, 0.05 outside) the fraction implied
    by the mass of A is exactly the covered area."""
    for frac, seed in ((0.536, 3), (0.628, 4)):
        rho, covered = W.disk_packing(200, 120, frac, seed, periodic_z=False)
        phi = E.mass_packing_fraction(rho[0].sum(), rho[0].size, 1.2, 0.05)
        assert phi == pytest.approx(covered, abs=1e-12)


def test_interface_positions():
    x = np.arange(100, dtype=float)
    prof = np.tanh((x - 30.25) / 3.0) - np.tanh((x - 70.75) / 3.0)
    pos = E.interface_positions(prof, 1.0)
    # near each interface the other tanh is -1 or 1 to ~1e-6, so the profile crosses 1 where its
    # own tanh vanishes; linear interpolation over one cell of a tanh of width 3 is within 0.01
    assert len(pos) == 2
    assert pos == pytest.approx([30.25, 70.75], abs=0.01)


def test_bulk_pressure_matches_the_oracles_pressure_tensor(oracle):
    """Eq. BULK against the normal pressure the oracle measures on a relaxed flat slab (film
    couplings): both bulk phases sit at the slab's uniform P_xx."""
    nx, nz = 96, 2  # 24 cells between an interface and the phase centre: bulk to ~1e-11
    p = dict(W.FILM_PARAMS)
    ref = oracle.RefLattice(nx, nz, 1, 0, **p)
    x = np.arange(nx)
    ref.set_fields(np.tile(0.29 + 0.55 * (np.tanh((x - 24) / 3) - np.tanh((x - 72) / 3)), (1, nz, 1)))
    ref.step(40000)
    rho = ref.fields()[0][0, 0]
    P = ref.site_fields()["P"][0]
    for r in (rho[48], rho[0]):
        assert E.bulk_pressure(r, p["G1"][0], p["G2"][0], p["weight_norm"]) == pytest.approx(P.mean(), abs=1e-9)
