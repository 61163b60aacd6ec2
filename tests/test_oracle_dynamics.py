"""Pins of the oracle's dynamics against what the paper and the mathematics fix (no GPU).

Each test names the passage it checks.  Tolerances are stated with the reason.
"""
import numpy as np
import pytest

from paper_1402_6019_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _lat(oracle, nx, nz, ns=1, zbc=0, **p):
    return oracle.RefLattice(nx, nz, ns, zbc, **p)


# --------------------------------------------------------------------------------------------
# Conservation (Eq. LB is mass conserving; Eq. FORCE is pairwise antisymmetric)
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("zbc,wall_u", [(0, (0.0, 0.0)), (1, (0.0, 0.0)), (1, (-0.02, 0.03))])
def test_mass_conserved_two_species(oracle, zbc, wall_u):
    rho, _ = W.disk_packing(40, 32, 0.6, seed=5, r_mean=6, r_spread=2, periodic_z=(zbc == 0))
    L = _lat(oracle, 40, 32, 2, zbc, **dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=wall_u))
    L.set_fields(rho)
    m0 = L.observables()["mass"]
    L.step(1000)
    m1 = L.observables()["mass"]
    # rounding only: ~1e-16 per site and step, 1000 steps
    assert np.abs(m1 - m0).max() / m0.max() < 1e-12


def test_mass_and_momentum_single_component(oracle):
    L = _lat(oracle, 33, 27, **W.SINGLE_PARAMS)
    L.set_fields(W.noise_field(33, 27, seed=11))
    o0 = L.observables()
    L.step(500)
    o1 = L.observables()
    assert abs(o1["mass"][0] - o0["mass"][0]) / o0["mass"][0] < 1e-12
    # no body force, periodic: total momentum stays zero up to rounding
    assert np.abs(o1["momentum"]).max() < 1e-12 * o0["mass"][0]


def test_momentum_grows_by_body_force(oracle):
    g = 3e-6
    rho, _ = W.disk_packing(32, 24, 0.5, seed=3, r_mean=5, r_spread=1)
    L = _lat(oracle, 32, 24, 2, 0, **dict(W.EMULSION_PARAMS, body_force=g))
    L.set_fields(rho)
    o0 = L.observables()
    L.step(50)
    o1 = L.observables()
    mtot = o0["mass"].sum()
    assert o1["momentum"][0] - o0["momentum"][0] == pytest.approx(50 * g * mtot, rel=1e-9)
    assert abs(o1["momentum"][1]) < 1e-13 * mtot


def test_zero_net_interaction_force(oracle):
    rho, _ = W.disk_packing(36, 30, 0.6, seed=9, r_mean=6, r_spread=2)
    L = _lat(oracle, 36, 30, 2, 0, **dict(W.EMULSION_PARAMS, G_AB=0.587))
    L.set_fields(rho)
    F = L.site_fields()["F"]
    scale = np.abs(F).sum()
    assert scale > 1.0
    # total over both species: intra terms cancel per species, cross terms pairwise
    assert np.abs(F.sum(axis=(0, 2, 3))).max() < 1e-13 * scale
    # intra-species alone (G_AB = 0): zero per species
    L.set_params(**dict(W.EMULSION_PARAMS, G_AB=0.0))
    F = L.site_fields()["F"]
    assert np.abs(F.sum(axis=(2, 3))).max() < 1e-13 * np.abs(F).sum()


# --------------------------------------------------------------------------------------------
# Force: closed form on sinusoidal fields (Eq. FORCE and the cross term)
# --------------------------------------------------------------------------------------------

def _kernel(c25, W_, links, kx, kz):
    """sum_l W(|c_l|^2) c_l sin(k.c_l) for the given links (vector)."""
    s = np.zeros(2)
    for l in links:
        cx, cz = c25[l]
        s += W_[cx * cx + cz * cz] * np.array([cx, cz]) * np.sin(kx * cx + kz * cz)
    return s


@pytest.mark.parametrize("mx,mz", [(1, 0), (3, 0), (2, 2), (1, 3)])
def test_intra_force_closed_form(oracle, mx, mz):
    nx, nz = 24, 18
    G1, G2 = -9.0, 8.1
    kx, kz = 2 * np.pi * mx / nx, 2 * np.pi * mz / nz
    x = np.arange(nx)[None, :]
    z = np.arange(nz)[:, None]
    a, b = 0.7, 0.2
    psi = a + b * np.sin(kx * x + kz * z)
    L = _lat(oracle, nx, nz, psi_form=oracle.PSI_RHO, G1=G1, G2=G2, weight_norm=1.0)
    L.set_fields(psi[None])
    F = L.site_fields()["F"][0]
    c25, _, _, wsh = oracle.tables()
    K = G1 * _kernel(c25, wsh[0], range(1, 13), kx, kz) + G2 * _kernel(c25, wsh[1], range(1, 25),
                                                                      kx, kz)
    # F(x) = -psi(x) sum K c psi(x+c) = -psi(x) b cos(k.x) sum K c sin(k.c)
    want = -psi * b * np.cos(kx * x + kz * z)
    assert np.allclose(F[0], want * K[0], rtol=0, atol=1e-14)
    assert np.allclose(F[1], want * K[1], rtol=0, atol=1e-14)
    # small-k limit: sum K c_x sin(k c_x) -> k e2 - k^3 e4 / 2 + ... (Eq. tensorial, App. B)
    if mz == 0:
        e2 = G1 + G2
        e4 = G1 * 2 / 5 + G2 * 4 / 7
        assert K[0] / kx == pytest.approx(e2 - kx ** 2 * e4 / 2, abs=kx ** 4 * 2)


def test_cross_force_closed_form(oracle):
    nx, nz = 20, 16
    k = 2 * np.pi * 2 / nx
    x = np.arange(nx)[None, :].repeat(nz, 0)
    rhoA = np.full((nz, nx), 0.9)
    rhoB = 0.5 + 0.3 * np.sin(k * x)
    G_AB = 0.587
    L = _lat(oracle, nx, nz, 2, 0, G1=0.0, G2=0.0, G_AB=G_AB, weight_norm=1.0)
    L.set_fields(np.stack([rhoA, rhoB]))
    F = L.site_fields()["F"]
    c25, _, _, wsh = oracle.tables()
    K = _kernel(c25, wsh[2], range(1, 9), k, 0.0)
    assert np.allclose(F[0, 0], -G_AB * rhoA * 0.3 * np.cos(k * x) * K[0], rtol=0, atol=1e-14)
    assert np.abs(F[0, 1]).max() < 1e-14
    # the other species sees a uniform neighbour field: no cross force
    assert np.abs(F[1]).max() < 1e-14


# --------------------------------------------------------------------------------------------
# Walls and drives (Sec. IV): single-phase Couette and Poiseuille
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("tau", [0.8, 1.0, 1.7])
def test_couette_exact(oracle, tau):
    nz, Ub, Ut = 12, -0.01, 0.015
    L = _lat(oracle, 3, nz, 1, 1, tau=tau, G1=0.0, G2=0.0, wall_u=(Ub, Ut))
    L.set_fields(np.ones((1, nz, 3)))
    L.step(int(40 * nz * nz / ((tau - 0.5) / 3)))
    _, u, _ = L.fields()
    z = np.arange(nz)
    exact = Ub + (Ut - Ub) * (z + 0.5) / nz  # walls at z = -1/2 and nz - 1/2
    assert np.abs(u[0, :, 0] - exact).max() < 1e-12
    o = L.observables()
    stress = (tau - 0.5) / 3 * (Ut - Ub) / nz  # rho nu du/dz with rho = 1
    assert np.allclose(o["sxz_z"], stress, rtol=1e-9)
    # the bottom wall receives +stress per step, the top wall -stress (momentum balance)
    assert o["wall_force"] == pytest.approx([stress, -stress], rel=1e-9)
    # Eq. fluidity: f = shear rate / stress = 1 / (rho nu) for a Newtonian fluid
    assert np.allclose(o["fluid_z"], 3.0 / (tau - 0.5), rtol=1e-8)


@pytest.mark.parametrize("tau", [0.7, 1.0])
def test_poiseuille(oracle, tau):
    nz, g = 16, 1e-6
    nu = (tau - 0.5) / 3
    L = _lat(oracle, 3, nz, 1, 1, tau=tau, G1=0.0, G2=0.0, body_force=g)
    L.set_fields(np.ones((1, nz, 3)))
    L.step(int(30 * nz * nz / nu))
    _, u, _ = L.fields()
    ux = u[0, :, 0]
    # interior: nu * (discrete Laplacian) = -g exactly at steady state
    lap = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    assert np.allclose(nu * lap, -g, rtol=1e-8)
    # profile: the parabola with walls at -1/2 and nz - 1/2, plus a uniform slip
    z = np.arange(nz)
    para = g / (2 * nu) * (z + 0.5) * (nz - 0.5 - z)
    slip = ux - para
    assert np.ptp(slip) < 1e-9 * ux.max()
    assert abs(slip[0]) < 0.02 * ux.max()
    assert np.allclose(ux, ux[::-1], rtol=1e-12)


# --------------------------------------------------------------------------------------------
# Stress (Sec. III, Appendix A): exact lattice divergence and the flat interface
# --------------------------------------------------------------------------------------------

def _face_stress(c25, wsh, psi, couplings):
    """Flux of x-momentum through the face between x and x+1 for a profile psi(x) uniform
    in z: every pair (a, a + c_x) with c_x > 0 crossing the face carries G W psi psi c_x."""
    nx = psi.size
    S = np.zeros(nx)
    for G, Wt, nl in couplings:
        for l in range(1, nl + 1):
            cx, cz = c25[l]
            q = cx * cx + cz * cz
            if cx <= 0 or Wt[q] == 0:
                continue
            for a_off in range(-cx + 1, 1):
                a = np.arange(nx) + a_off
                S += G * Wt[q] * psi[a % nx] * psi[(a + cx) % nx] * cx
    return S


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_flat_interface_exact_balance(oracle, tau):
    nx, nz = 96, 2
    p = dict(W.FILM_PARAMS, tau=(tau, tau))
    L = _lat(oracle, nx, nz, **p)
    x = np.arange(nx)
    prof = 0.29 + 1.1 * 0.5 * (np.tanh((x - 24) / 3) - np.tanh((x - 72) / 3))
    L.set_fields(np.tile(prof, (1, nz, 1)))
    L.step(40000)
    rho, u, f = L.fields()
    sf = L.site_fields()
    c25, _, _, wsh = oracle.tables()
    wn = p["weight_norm"]
    S = _face_stress(c25, wsh * wn, sf["psi"][0, 0], [(-20.4, wsh[0] * wn, 12),
                                                      (16.0, wsh[1] * wn, 24)])
    scale = np.abs(sf["F"]).max()
    # Eq. MECHANICAL: the force is the exact lattice divergence of the interaction stress
    assert np.abs(sf["F"][0, 0, 0] + (S - np.roll(S, 1))).max() < 1e-13 * max(scale, 1)
    # Appendix A's node stress is the mean of the two adjacent face stresses
    assert np.abs(sf["sint"][0, 0, 0] - 0.5 * (S + np.roll(S, 1))).max() < 1e-13
    # steady state: kinetic face flux + interaction face flux is uniform
    Fp = f[0][[1, 5, 8]].sum(0)[0]
    Fm = f[0][[3, 6, 7]].sum(0)[0]
    T = np.roll(Fp, -1) + Fm + S
    assert np.ptp(T) < 1e-12
    # Sec. III: the normal pressure tensor component is constant at machine precision
    assert np.ptp(sf["P"][0]) < 1e-12
    # ... and equals Eq. BULK in both bulk phases (c_s^2 normalisation of the weights)
    Pb = lambda r: CS2 * r + CS2 * (-20.4 + 16.0) / 2 * (1 - np.exp(-r)) ** 2
    assert Pb(rho[0, 0, 48]) == pytest.approx(sf["P"][0].mean(), abs=1e-9)
    assert Pb(rho[0, 0, 0]) == pytest.approx(sf["P"][0].mean(), abs=1e-9)
    assert np.abs(u).max() < 1e-12


def test_a_form_matches_shell_stress(oracle):
    """Appendix A: for a profile uniform in z, sigma_xx - sigma_zz of the shell sums equals the
    A1..A3 form (with the re-derived sign of A0's G1 term)."""
    nx, nz = 40, 3
    G1, G2 = -9.0, 8.1
    rng = np.random.default_rng(1)
    psi = 0.3 + rng.random(nx)
    L = _lat(oracle, nx, nz, psi_form=oracle.PSI_RHO, G1=G1, G2=G2, weight_norm=1.0)
    L.set_fields(np.tile(psi, (1, nz, 1)))
    si = L.site_fields()["sint"][0]
    w = {1: 4 / 15, 4: 1 / 120}
    p = {1: 4 / 21, 4: 1 / 60, 5: 2 / 315}
    A1 = G2 * (p[1] / 2 - 3 * p[5]) + G1 * w[1] / 2
    A2 = G2 * (p[4] + 1.5 * p[5]) + G1 * w[4]
    A0 = -G1 * (w[1] + 4 * w[4]) - G2 * (p[1] + 4 * p[4])
    A3 = G2 * (2 * p[4] + 3 * p[5]) + 2 * G1 * w[4]
    r = lambda k: np.roll(psi, -k)
    aform = A1 * psi * (r(1) + r(-1)) + A2 * psi * (r(2) + r(-2)) + A0 * psi * psi + A3 * r(1) * r(-1)
    assert np.abs((si[0] - si[1])[0] - aform).max() < 1e-13
    assert np.abs(si[2]).max() < 1e-14


def test_surface_tension_summed_a_form(oracle):
    """gamma = sum_x p_s(x) (Eq. DIS1).  Summing Appendix A's A-form over a periodic profile by
    parts, with 2 A1 + 2 A2 + A0 + A3 = 0, gives the exact lattice identity
        sum_x (s_xx - s_zz) = sum_x [-A1 (d1 psi)^2 - (A2 + A3/2) (d2 psi)^2],
    d_a psi = psi(x+a) - psi(x), whose continuum limit is Sec. III's C2 (psi')^2 term
    (C2 = -A1 - 4 A2 - 2 A3).  The C2/C4 Taylor estimate itself drops higher derivatives, so it
    is only checked loosely."""
    nx = 96
    L = _lat(oracle, nx, 2, **W.FILM_PARAMS)
    x = np.arange(nx)
    prof = 0.29 + 1.1 * 0.5 * (np.tanh((x - 24) / 3) - np.tanh((x - 72) / 3))
    L.set_fields(np.tile(prof, (1, 2, 1)))
    L.step(20000)
    o = L.observables()
    sf = L.site_fields()
    psi, rho, Fx = sf["psi"][0, 0], L.fields()[0][0, 0], sf["F"][0, 0, 0]
    wn = W.WEIGHT_NORM
    G1, G2 = -20.4, 16.0
    w1, w4 = wn * 4 / 15, wn / 120
    p1, p4, p5 = wn * 4 / 21, wn / 60, wn * 2 / 315
    A1 = G2 * (p1 / 2 - 3 * p5) + G1 * w1 / 2
    A2 = G2 * (p4 + 1.5 * p5) + G1 * w4
    A3 = G2 * (2 * p4 + 3 * p5) + 2 * G1 * w4
    d1 = np.roll(psi, -1) - psi
    d2 = np.roll(psi, -2) - psi
    kin = np.sum(0.25 * Fx ** 2 / rho)  # (tau - 1/2)^2 F^2 / rho at tau = 1
    exact = np.sum(-A1 * d1 ** 2 - (A2 + A3 / 2) * d2 ** 2) + kin
    assert o["gamma"] > 0
    assert o["gamma"] == pytest.approx(exact, rel=1e-10)
    C2 = wn * (20.4 / 2 * 2 / 5 - 16.0 / 2 * 4 / 7)
    C4 = wn * (-20.4 / 4 * 2 / 15 + 16.0 / 4 * 32 / 105)
    assert C2 == pytest.approx(-A1 - 4 * A2 - 2 * A3, rel=1e-12)
    c1 = (np.roll(psi, -1) - np.roll(psi, 1)) / 2
    c2 = np.roll(psi, -1) - 2 * psi + np.roll(psi, 1)
    taylor = np.sum(C2 * c1 ** 2 + C4 * c2 ** 2) + kin
    assert o["gamma"] == pytest.approx(taylor, rel=0.3)


def test_laplace_law(oracle):
    """Laplace's law in 2-D, Delta P = gamma / R (Sec. III), bulk pressures from Eq. BULK."""
    Pb = lambda r: CS2 * r + CS2 * (-20.4 + 16.0) / 2 * (1 - np.exp(-r)) ** 2
    nx = 64
    x = np.arange(nx)
    L = _lat(oracle, nx, 2, **W.FILM_PARAMS)
    L.set_fields(np.tile(0.29 + 0.55 * (np.tanh((x - 16) / 3) - np.tanh((x - 48) / 3)), (1, 2, 1)))
    L.step(15000)
    gamma = L.observables()["gamma"] / 2
    ratios = []
    for R in (8, 12, 16):
        n = 2 * R + 32
        X, Z = np.meshgrid(np.arange(n), np.arange(n))
        r = np.hypot(X - n / 2 + 0.5, Z - n / 2 + 0.5)
        L = _lat(oracle, n, n, **W.FILM_PARAMS)
        L.set_fields((0.29 + 0.55 * (1 - np.tanh((r - R) / 2)))[None])
        L.step(4000)
        rho = L.fields()[0][0]
        rin, rout = rho[n // 2, n // 2], rho[0, 0]
        Re = np.sqrt((rho - rout).sum() / (rin - rout) / np.pi)
        ratios.append((Pb(rin) - Pb(rout)) * Re / gamma)
    ratios = np.array(ratios)
    assert np.all((ratios > 0.95) & (ratios < 1.15)), ratios
    assert np.ptp(ratios) / ratios.mean() < 0.06, ratios


# --------------------------------------------------------------------------------------------
# A/B emulsion (Sec. IV)
# --------------------------------------------------------------------------------------------

def _golden():
    import os
    vals = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def test_emulsion_phase_densities_match_paper():
    """Sec. IV prints the A-rich / B-rich phases as approximately (1.2, 0.2) / (0.2, 1.2) for
    its couplings; a flat A/B interface relaxes to phases near those values."""
    import oracle

    g = _golden()
    nx = 128
    p = dict(tau=(1.0, 1.0), G1=(g["emulsion_GAA1"], g["emulsion_GBB1"]),
             G2=(g["emulsion_GAA2"], g["emulsion_GBB2"]), G_AB=g["emulsion_GAB"],
             psi_form=0, rho0=(g["emulsion_rho0"],) * 2, weight_norm=W.WEIGHT_NORM)
    L = oracle.RefLattice(nx, 2, 2, 0, **p)
    x = np.arange(nx)
    s = 0.5 * (np.tanh((x - 32) / 2) - np.tanh((x - 96) / 2))
    L.set_fields(np.stack([0.05 + 1.15 * s, 1.2 - 1.15 * s])[:, None, :].repeat(2, 1))
    L.step(20000)
    rho = L.fields()[0]
    assert abs(rho[0, 0, 64] - g["phase_rich"]) < 0.1 and abs(rho[1, 0, 64] - g["phase_poor"]) < 0.1
    assert abs(rho[1, 0, 0] - g["phase_rich"]) < 0.1 and abs(rho[0, 0, 0] - g["phase_poor"]) < 0.1
    assert L.observables()["gamma"] > 0


def test_ab_one_step_momentum_balance(oracle):
    """Exact lattice momentum balance of the mixture, one step at a time, for a z-uniform
    profile away from steady state: the change of the total x-momentum at x equals minus the
    difference across x of the face flux T(x+1/2) = [kinetic flux of both species after
    streaming] + [intra- and cross-species face stresses at time t] (Eq. MECHANICAL applied to
    the sum of the species' forces, Sec. IV)."""
    nx = 64
    g = _golden()
    p = dict(W.EMULSION_PARAMS, G_AB=g["emulsion_GAB"])
    L = _lat(oracle, nx, 2, 2, 0, **p)
    x = np.arange(nx)
    s = 0.5 * (np.tanh((x - 16) / 2) - np.tanh((x - 48) / 2))
    L.set_fields(np.stack([0.05 + 1.15 * s, 1.2 - 1.15 * s])[:, None, :].repeat(2, 1))
    L.step(300)
    c25, cq, _, wsh = oracle.tables()
    wn = p["weight_norm"]
    rho, _, f0 = L.fields()
    psi = L.site_fields()["psi"]
    S = np.zeros(nx)
    for s_ in range(2):
        S += _face_stress(c25, None, psi[s_, 0], [(p["G1"][s_], wsh[0] * wn, 12),
                                                  (p["G2"][s_], wsh[1] * wn, 24)])
    ra, rb = rho[0, 0], rho[1, 0]
    for l in range(1, 9):
        cx, cz = c25[l]
        if cx > 0:  # cross pairs carry rho_A(a) rho_B(b) + rho_B(a) rho_A(b)
            S += p["G_AB"] * wsh[2][cx * cx + cz * cz] * wn * (
                ra * np.roll(rb, -cx) + rb * np.roll(ra, -cx)) * cx
    L.step(1)
    f1 = L.fields()[2]
    J = lambda f: np.einsum("slx,l->x", f[:, :, 0, :], cq[:, 0].astype(float))
    T = S.copy()
    for s_ in range(2):
        T += np.roll(f1[s_][[1, 5, 8]].sum(0)[0], -1) + f1[s_][[3, 6, 7]].sum(0)[0]
    lhs = J(f1) - J(f0)
    rhs = -(T - np.roll(T, 1))
    assert np.abs(lhs).max() > 1e-6  # not at rest: the identity is not trivially zero
    assert np.abs(lhs - rhs).max() < 1e-14


@pytest.mark.parametrize("G_AB,grows", [(0.587, True), (0.15, False)])
def test_ab_demixing_sign(oracle, G_AB, grows):
    """The cross term is repulsive (Sec. IV): a near-symmetric mixture demixes above the linear
    stability threshold and stays mixed well below it."""
    nx = nz = 48
    rho = 0.62 + W.noise_field(nx, nz, seed=21, mean=0.0, amp=0.01, n_species=2)
    L = _lat(oracle, nx, nz, 2, 0, **dict(W.EMULSION_PARAMS, G_AB=G_AB))
    L.set_fields(rho)
    v0 = np.var(rho[0] - rho[1])
    L.step(1500)
    r = L.fields()[0]
    v1 = np.var(r[0] - r[1])
    assert (v1 > 100 * v0) if grows else (v1 < v0)


# --------------------------------------------------------------------------------------------
# Linear stability of a uniform single-component state: the dispersion relation
# --------------------------------------------------------------------------------------------

def _dispersion(oracle, k, G1, G2, rho_b, weight_norm=1.0 / 3.0):
    """Effective squared sound speed of a small density wave exp(ikx) on a uniform state rho_b:
    linearising Eq. FORCE, F_x = psi psi' S(k) drho with S(k) = sum_l K(|c_l|^2) c_lx sin(k c_lx)
    (K = G1 w on links 1..12 plus G2 p on 1..24, the exact weights), so the density obeys
    eps'' + D k^2 eps' + k^2 c_eff^2 eps = 0 with c_eff^2 = c_s^2 + psi psi' S(k) / k (Sec. III's
    continuum form of the interaction pressure, for psi = 1 - exp(-rho))."""
    c25, _, _, wsh = oracle.tables()
    S = 0.0
    for l in range(1, 25):
        cx, cz = c25[l]
        q = int(cx * cx + cz * cz)
        K = (G1 * wsh[0][q] if l <= 12 else 0.0) + G2 * wsh[1][q]
        S += weight_norm * K * cx * np.sin(k * cx)
    psi, dpsi = 1.0 - np.exp(-rho_b), np.exp(-rho_b)
    return 1.0 / 3.0 + psi * dpsi * S / k


def _wave(oracle, G1, G2, rho_b, steps, eps, nx=128, nz=4):
    """Amplitude of the k = 2 pi / nx cosine of the density, step by step, from a uniform state
    plus eps cos(kx) at rest."""
    k = 2 * np.pi / nx
    x = np.arange(nx)
    L = _lat(oracle, nx, nz, G1=G1, G2=G2, tau=1.0, rho0=1.0, weight_norm=1.0 / 3.0)
    L.set_fields(np.broadcast_to(rho_b + eps * np.cos(k * x), (1, nz, nx)).copy())
    A = np.empty(steps)
    for t in range(steps):
        r = L.fields()[0][0].mean(axis=0)
        A[t] = 2.0 / nx * np.sum((r - r.mean()) * np.cos(k * x))
        L.step(1)
    return k, A


def test_sound_speed_follows_the_interaction_pressure(oracle):
    """Stable state (G1, G2) = (-9.0, 8.1) at rho = 1: the wave oscillates at omega = k c_eff
    with c_eff^2 = 0.263 (c_s^2 = 1/3 alone would give a frequency 12 % higher).  Measured from
    the zero crossings over four periods: within 5e-4 (observed 3e-5); the continuum relation
    neglects O(k^2) lattice terms and the damping shifts omega by O((nu k / c)^2) ~ 1e-4."""
    k, A = _wave(oracle, -9.0, 8.1, 1.0, 1000, 1e-6)
    c2 = _dispersion(oracle, k, -9.0, 8.1, 1.0)
    s = np.sign(A)
    zc = np.where(s[1:] * s[:-1] < 0)[0]
    tz = zc + A[zc] / (A[zc] - A[zc + 1])
    omega = np.pi / np.mean(np.diff(tz))
    assert len(zc) >= 7
    assert omega == pytest.approx(k * np.sqrt(c2), rel=5e-4)
    assert abs(omega / (k / np.sqrt(3.0)) - 1) > 0.1


@pytest.mark.parametrize("rho_b", [0.7, 0.8])
def test_unstable_wave_grows_at_the_dispersion_rate(oracle, rho_b):
    """The film couplings (G1, G2) = (-20.4, 16.0) of Sec. III make the uniform state unstable
    (c_eff^2 < 0): the wave grows at gamma = (-D k^2 + sqrt(D^2 k^4 - 4 k^2 c_eff^2)) / 2, with
    D = 2 nu = (2 tau - 1) / 3 the longitudinal momentum diffusivity of BGK.  Measured as the
    slope of log|amplitude| over steps 250..400, after the decaying root has died out and
    before faster, shorter waves seeded by rounding take over (these couplings are frustrated:
    shorter waves grow faster): within 3 % (observed 1 %)."""
    k, A = _wave(oracle, -20.4, 16.0, rho_b, 401, 1e-6)
    c2 = _dispersion(oracle, k, -20.4, 16.0, rho_b)
    assert c2 < 0
    D = 2.0 * (1.0 - 0.5) / 3.0
    gamma = (-D * k * k + np.sqrt(D * D * k ** 4 - 4 * k * k * c2)) / 2
    t = np.arange(250, 401)
    slope = np.polyfit(t, np.log(np.abs(A[250:401])), 1)[0]
    assert slope == pytest.approx(gamma, rel=0.03)
    assert np.abs(A).max() < 1e-4  # still linear


# --------------------------------------------------------------------------------------------
# Eq. MECHANICAL on a two-dimensional state: every stress component, intra and cross
# --------------------------------------------------------------------------------------------

def _bonds(c25, wsh, wn, p, ns):
    """The pair interactions of Eq. FORCE and of the cross term as bonds (a, a + c), each counted
    once (c_z > 0, or c_z = 0 and c_x > 0): (kind, species, coupling K, c).  kind 'intra' pairs
    psi_s(a) psi_s(a + c); kind 'cross' pairs rho_A(a) rho_B(a + c) + rho_B(a) rho_A(a + c)."""
    out = []
    for l in range(1, 25):
        cx, cz = (int(v) for v in c25[l])
        if not (cz > 0 or (cz == 0 and cx > 0)):
            continue
        q = cx * cx + cz * cz
        for s in range(ns):
            K = p["G2"][s] * wsh[1][q] * wn + (p["G1"][s] * wsh[0][q] * wn if l <= 12 else 0.0)
            if K != 0.0:
                out.append(("intra", s, K, cx, cz))
        if ns == 2 and l <= 8 and p.get("G_AB", 0.0) != 0.0:
            out.append(("cross", -1, p["G_AB"] * wsh[2][q] * wn, cx, cz))
    return out


def _line_fluxes(bonds, psi, rho, select):
    """Momentum carried by the bonds across the lattice lines (periodic lattice).
    TH[i, z] is the i-momentum (i = x, z) crossing the horizontal line between rows z and z + 1
    (a bond with c_z > 0 crosses c_z such lines, each carrying K * product * c_i); TV[i, x] the
    i-momentum crossing the vertical line between columns x and x + 1 (|c_x| lines)."""
    _, nz, nx = psi.shape
    TH = np.zeros((2, nz))
    TV = np.zeros((2, nx))
    for kind, s, K, cx, cz in bonds:
        if not select(kind, s):
            continue
        sh = lambda a: np.roll(np.roll(a, -cz, axis=0), -cx, axis=1)  # a(x + c)
        if kind == "intra":
            prod = psi[s] * sh(psi[s])
        else:
            prod = rho[0] * sh(rho[1]) + rho[1] * sh(rho[0])
        row, col = prod.sum(axis=1), prod.sum(axis=0)  # per starting row / column of a
        for i, ci in enumerate((cx, cz)):
            for k in range(cz):  # lines z_a + k + 1/2
                TH[i] += K * ci * np.roll(row, k)
            for k in range(abs(cx)):  # lines x_a + 1/2 ... (c_x > 0) or x_a - 1/2 ... (c_x < 0)
                sgn = 1 if cx > 0 else -1
                shift = k if cx > 0 else -(k + 1)
                TV[i] += sgn * K * ci * np.roll(col, shift)
    return TH, TV


@pytest.mark.parametrize("G_AB", [0.0, 0.405])
def test_mechanical_balance_two_dimensional_state(oracle, G_AB):
    """Eq. MECHANICAL on a state that varies in x and z (droplets, not a flat interface), for every
    stress component including xz.  The bonds of Eq. FORCE carry momentum across the lattice's
    lines; on a periodic lattice, exactly:
      * the force summed over a row (column) is minus the difference of the line fluxes above and
        below it (left and right of it), for both components;
      * Appendix A's node stress summed over a row is the mean of the two adjacent horizontal line
        fluxes (sigma_xz for x-momentum, sigma_zz for z-momentum), and summed over a column the
        mean of the two adjacent vertical ones (sigma_xx, sigma_xz).
    The second holds shell by shell for Appendix A's split of a bond over its end points (shells
    1, 2), its midpoint (4, 8) and its two middle nodes (the c13..c16 pair terms of shell 5), so
    a wrong sign, index or node of any term fails it; the cross stress is checked the same way.
    Rounding only: 1e-13 of the largest flux."""
    nx, nz = 40, 36
    rho, _ = W.disk_packing(nx, nz, 0.55, seed=31, r_mean=5, r_spread=2)
    x = np.arange(nx)[None, :]
    z = np.arange(nz)[:, None]
    rho = rho * (1.0 + 0.05 * np.sin(2 * np.pi * (2 * x / nx + z / nz)))[None]
    p = dict(W.EMULSION_PARAMS, G_AB=G_AB, tau=(1.0, 0.8))
    L = _lat(oracle, nx, nz, 2, 0, **p)
    L.set_fields(rho)
    L.step(40)
    r, _, _ = L.fields()
    sf = L.site_fields()
    psi, F, sint, P = sf["psi"], sf["F"], sf["sint"], sf["P"]
    c25, _, _, wsh = oracle.tables()
    bonds = _bonds(c25, wsh, p["weight_norm"], p, 2)
    # the cross stress is what P holds beyond the species' own terms (Sec. III's tensor)
    kin = np.zeros_like(P)
    for s in range(2):
        k2 = (p["tau"][s] - 0.5) ** 2
        kin[0] += CS2 * r[s] + sint[s, 0] + k2 * F[s, 0] ** 2 / r[s]
        kin[1] += CS2 * r[s] + sint[s, 1] + k2 * F[s, 1] ** 2 / r[s]
        kin[2] += sint[s, 2] + k2 * F[s, 0] * F[s, 1] / r[s]
    sab = P - kin
    groups = [("intra A", lambda k, s: k == "intra" and s == 0, F[0], sint[0]),
              ("intra B", lambda k, s: k == "intra" and s == 1, F[1], sint[1])]
    if G_AB:
        # per species the cross force is not a divergence; their sum is, with the cross stress
        groups = [("all", lambda k, s: True, F[0] + F[1], sint[0] + sint[1] + sab)]
    else:
        assert np.abs(sab).max() < 1e-13
    for name, sel, Fg, sg in groups:
        TH, TV = _line_fluxes(bonds, psi, r, sel)
        scale = max(np.abs(TH).max(), np.abs(TV).max())
        assert scale > 1e-3, name  # the state is far from uniform
        tol = 1e-13 * scale
        for i in range(2):  # force: minus the difference of line fluxes
            assert np.abs(Fg[i].sum(axis=1) + (TH[i] - np.roll(TH[i], 1))).max() < tol, (name, i)
            assert np.abs(Fg[i].sum(axis=0) + (TV[i] - np.roll(TV[i], 1))).max() < tol, (name, i)
        mean = lambda T: 0.5 * (T + np.roll(T, 1))
        assert np.abs(sg[2].sum(axis=1) - mean(TH[0])).max() < tol, (name, "xz rows")
        assert np.abs(sg[1].sum(axis=1) - mean(TH[1])).max() < tol, (name, "zz rows")
        assert np.abs(sg[0].sum(axis=0) - mean(TV[0])).max() < tol, (name, "xx columns")
        assert np.abs(sg[2].sum(axis=0) - mean(TV[1])).max() < tol, (name, "xz columns")
        assert np.abs(TH[0]).max() > 1e-3 * scale and np.abs(TV[1]).max() > 1e-3 * scale, name


def test_unequal_tau_common_velocity_conserves_momentum(oracle):
    """Sec. II's shifted-velocity forcing with the common velocity of the mixture (reading: u' =
    sum_s (j_s/tau_s) / sum_s (rho_s/tau_s)): the collision changes the total momentum at every
    site by exactly the total force, sum_s F_s, whatever the species' relaxation times.  Streaming
    only moves populations, so on a periodic lattice the post-collision populations at x are the
    streamed ones at x + c_l.  Checked site by site after a step from a state whose species move
    at different velocities, with tau_A != tau_B (a plain barycentric u' breaks the identity by
    sum_s (1/tau_s)(rho_s u' - j_s), which is nonzero there) and a body force."""
    nx, nz = 30, 26
    rho, _ = W.disk_packing(nx, nz, 0.5, seed=41, r_mean=5, r_spread=1)
    p = dict(W.EMULSION_PARAMS, tau=(0.7, 1.6), body_force=2e-5)
    L = _lat(oracle, nx, nz, 2, 0, **p)
    L.set_fields(rho)
    L.step(30)  # species velocities now differ (different forces per unit mass)
    c25, cq, _, _ = oracle.tables()
    cxz = cq.astype(float)
    r0, _, f0 = L.fields()
    F = L.site_fields()["F"]
    j0 = np.einsum("slzx,lk->kzx", f0, cxz)           # total lattice momentum per site
    ja = np.einsum("lzx,lk->kzx", f0[0], cxz)
    jb = np.einsum("lzx,lk->kzx", f0[1], cxz)
    # the species move at different velocities: a barycentric u' would differ from the reading
    assert np.abs(ja / r0[0] - jb / r0[1]).max() > 1e-4
    L.step(1)
    f1 = L.fields()[2]
    post = np.empty_like(f1)  # f*_l(x) = f_l(x + c_l) after streaming
    for l in range(9):
        cx, cz = cq[l]
        post[:, l] = np.roll(np.roll(f1[:, l], -cz, axis=1), -cx, axis=2)
    j1 = np.einsum("slzx,lk->kzx", post, cxz)
    Fs = F.sum(axis=0)
    scale = np.abs(f0).max()
    assert np.abs((j1 - j0) - Fs).max() < 1e-14 * scale * 9
    # and each species keeps its mass at every site through the collision
    assert np.abs(post.sum(axis=1) - f0.sum(axis=1)).max() < 1e-14 * scale * 9
    # the lattice total: momentum grows by g sum(rho) per step
    assert (j1.sum(axis=(1, 2)) - j0.sum(axis=(1, 2)))[0] == pytest.approx(
        p["body_force"] * r0.sum(), rel=1e-9)


def test_sheared_droplet_stress_is_uniform_and_equals_the_wall_stress(oracle):
    """Sec. IV's fluidity divides the shear rate by the stress; in a channel sheared by its walls
    the x-momentum of every row is steady, so the x-averaged shear stress must be the same in
    every row and equal to the stress each wall takes (momentum balance, Eq. MECHANICAL applied
    across rows).  A droplet of the emulsion sheared between walls at -+U_w (Sec. IV's Couette
    cells) reaches a steady deformed shape; there the interaction stress (App. A shells and the
    cross term) carries a sizeable part of the stress in the droplet's rows, so a wrong sign or
    a dropped part of S_xz (interaction, species drift, forcing) breaks the balance by tens of
    percent.  Tolerance 1e-5: what is left of the approach to the steady state after 12000 steps
    (the balance is exact at the steady state)."""
    nx, nz, R, U = 40, 32, 10.0, 0.01
    X, Z = np.meshgrid(np.arange(nx), np.arange(nz))
    s = 0.5 * (1 - np.tanh((np.hypot(X - nx / 2 + 0.5, Z - nz / 2 + 0.5) - R) / 1.5))
    g = _golden()
    p = dict(W.EMULSION_PARAMS, G_AB=g["emulsion_GAB"], wall_u=(-U, U))
    L = _lat(oracle, nx, nz, 2, 1, **p)
    L.set_fields(np.stack([0.05 + 1.15 * s, 1.2 - 1.15 * s]))
    L.step(12000)
    o = L.observables()
    rho = L.fields()[0]
    assert rho[0].max() > 1.1 and rho[0].min() < 0.2  # the droplet is still there
    wb, wt = o["wall_force"]
    assert wb > 0 and wt == pytest.approx(-wb, rel=1e-6)
    assert np.abs(o["sxz_z"] / wb - 1.0).max() < 1e-5
    # the interaction stress in the droplet's rows: a large share of the total
    sf = L.site_fields()
    F, sint, P = sf["F"], sf["sint"], sf["P"]
    k2 = [(t - 0.5) ** 2 for t in p["tau"]]
    sab = P[2] - sum(sint[q, 2] + k2[q] * F[q, 0] * F[q, 1] / rho[q] for q in range(2))
    inter = (sint[0, 2] + sint[1, 2] + sab).mean(axis=1)
    assert np.abs(inter).max() > 0.1 * wb
