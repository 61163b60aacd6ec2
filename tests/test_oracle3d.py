"""Pins of the three-dimensional oracle (oracle/ref3d.py) against what the model fixes: the
isotropy conditions of Appendix B taken to three dimensions (which determine the weights), the
D3Q19 equilibrium moments, conservation of mass and momentum, closed forms of the force on
sinusoidal fields, and the dispersion relation of sound on a uniform state."""
import itertools

import numpy as np
import pytest

from oracle import ref3d

SHELLS_ATT = [1, 2, 3, 4]
SHELLS_REP = [1, 2, 3, 4, 5, 6, 8]


@pytest.fixture(scope="module")
def tab():
    return ref3d.tables()


def _moments(links, w_by_q, shells):
    """Per shell, the sums over its links of the monomials the isotropy conditions use."""
    keys = ["x2", "x4", "x2y2", "x6", "x4y2", "x2y2z2", "x8", "x6y2", "x4y4", "x4y2z2"]
    rows = {k: np.zeros(len(shells)) for k in keys}
    for c in links:
        q = int(c @ c)
        if q not in shells:
            continue
        j = shells.index(q)
        x, y, z = (float(v) for v in c)
        mono = dict(x2=x**2, x4=x**4, x2y2=x**2 * y**2, x6=x**6, x4y2=x**4 * y**2, x2y2z2=x**2 * y**2 * z**2,
                    x8=x**8, x6y2=x**6 * y**2, x4y4=x**4 * y**4, x4y2z2=x**4 * y**2 * z**2)
        for k in keys:
            rows[k][j] += mono[k]
    return rows


def _isotropy_system(rows, order):
    """Appendix B's constraints in 3-D: e2 = 1 and the isotropy of the 4th (, 6th, 8th) order
    tensors (an isotropic tensor has x4 = 3 x2y2; x6 = 5 x4y2 = 15 x2y2z2; x8 = 7 x6y2,
    5 x4y4 = 3 x6y2, x6y2 = 5 x4y2z2)."""
    A, b = [rows["x2"]], [1.0]
    A.append(rows["x4"] - 3 * rows["x2y2"]); b.append(0.0)
    if order >= 6:
        A.append(rows["x6"] - 5 * rows["x4y2"]); b.append(0.0)
        A.append(rows["x4y2"] - 3 * rows["x2y2z2"]); b.append(0.0)
    if order >= 8:
        A.append(rows["x8"] - 7 * rows["x6y2"]); b.append(0.0)
        A.append(5 * rows["x4y4"] - 3 * rows["x6y2"]); b.append(0.0)
        A.append(rows["x6y2"] - 5 * rows["x4y2z2"]); b.append(0.0)
    return np.array(A), np.array(b)


def test_link_set(tab):
    links = tab[0]
    q = (links * links).sum(axis=1)
    counts = {s: int((q == s).sum()) for s in SHELLS_REP}
    assert counts == {1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 24, 8: 12}
    assert len({tuple(c) for c in links}) == 92
    assert {tuple(-c) for c in links} == {tuple(c) for c in links}
    # every integer vector with |c|^2 <= 8 is there (7 is not a sum of three squares)
    want = {c for c in itertools.product(range(-2, 3), repeat=3) if 0 < sum(v * v for v in c) <= 8}
    assert want == {tuple(c) for c in links}


@pytest.mark.parametrize("which,shells,order", [("att", SHELLS_ATT, 6), ("rep", SHELLS_REP, 8)])
def test_weights_are_the_unique_isotropic_solution(tab, which, shells, order):
    """The weights solve the constraints, and the constraints have no other solution on these
    shells (square, nonsingular system)."""
    links, wa, wr = tab[0], tab[1], tab[2]
    w = (wa if which == "att" else wr)[shells]
    A, b = _isotropy_system(_moments(links, None, shells), order)
    assert A.shape == (len(shells), len(shells))
    assert abs(np.linalg.det(A)) > 1e-6
    assert np.allclose(np.linalg.solve(A, b), w, rtol=1e-13, atol=0)
    # other shells carry no weight
    full = wa if which == "att" else wr
    assert all(full[q] == 0 for q in range(9) if q not in shells)


def test_attraction_is_not_8th_order_isotropic(tab):
    """The attraction set is isotropic exactly to 6th order: the 8th-order conditions fail, as
    for the 2-D first belt."""
    links, wa = tab[0], tab[1]
    rows = _moments(links, None, SHELLS_ATT)
    w = wa[SHELLS_ATT]
    assert abs(w @ (rows["x8"] - 7 * rows["x6y2"])) > 1e-3


def test_isotropy_in_every_orientation(tab):
    """The tensors are isotropic, not only in the (x, y, z) components used to solve for the
    weights: sum_l w c_a c_b c_c c_d = e4 (d_ab d_cd + d_ac d_bd + d_ad d_bc) for all index sets,
    and likewise at 2nd order."""
    links, wa, wr = tab[0], tab[1], tab[2]
    d = np.eye(3)
    for full in (wa, wr):
        w = np.array([full[int(c @ c)] for c in links])
        c = links.astype(float)
        T2 = np.einsum("l,la,lb->ab", w, c, c)
        assert np.allclose(T2, np.eye(3), atol=1e-14)
        T4 = np.einsum("l,la,lb,lc,ld->abcd", w, c, c, c, c)
        e4 = T4[0, 0, 1, 1]
        iso = e4 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
        assert np.allclose(T4, iso, atol=1e-14)


def test_cross_weights_first_belt(tab):
    links, wc = tab[0], tab[3]
    first = [c for c in links if int(c @ c) <= 2]
    assert len(first) == 18  # the D3Q19 neighbours
    w = np.array([wc[int(c @ c)] for c in first])
    c = np.array(first, dtype=float)
    assert np.allclose(np.einsum("l,la,lb->ab", w, c, c), np.eye(3), atol=1e-15)
    x4 = np.sum(w * c[:, 0] ** 4)
    x2y2 = np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2)
    assert x4 == pytest.approx(3 * x2y2, abs=1e-15)


def test_d3q19_equilibrium_moments(tab):
    c19, w19 = tab[4].astype(float), tab[5]
    assert w19.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.einsum("l,la,lb->ab", w19, c19, c19), np.eye(3) / 3, atol=1e-16)
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho, u = 0.5 + rng.random(), 0.1 * rng.standard_normal(3)
        f = ref3d.feq(rho, u)
        assert f.sum() == pytest.approx(rho, rel=1e-15)
        assert np.allclose(f @ c19, rho * u, atol=1e-15)
        P = np.einsum("l,la,lb->ab", f, c19, c19)
        assert np.allclose(P, rho * np.eye(3) / 3 + rho * np.outer(u, u), atol=1e-15)


EMULSION = dict(G1=(-9.0, -8.0), G2=(8.1, 7.1), G_AB=0.405, rho0=0.83)


def test_mass_and_momentum_conserved():
    """Eq. LB conserves each species' mass; the interaction forces are pairwise antisymmetric on a
    periodic lattice, so the populations' total momentum does not change (and grows by g sum rho
    per step under a body force)."""
    rng = np.random.default_rng(11)
    rho = 0.4 + rng.random((2, 6, 7, 9))
    L = ref3d.RefLattice3D(9, 7, 6, 2, tau=(0.8, 1.3), **EMULSION)
    L.set_fields(rho)
    c19 = ref3d.tables()[4].astype(float)
    f0 = L.fields()[2]
    m0 = f0.sum(axis=(1, 2, 3, 4))
    p0 = np.einsum("slzyx,la->a", f0, c19)
    F = L.site_fields()["F"]
    assert np.abs(F.sum(axis=(0, 2, 3, 4))).max() < 1e-13 * np.abs(F).sum()
    L.step(30)
    f1 = L.fields()[2]
    assert np.allclose(f1.sum(axis=(1, 2, 3, 4)), m0, rtol=1e-13, atol=0)
    assert np.abs(np.einsum("slzyx,la->a", f1, c19) - p0).max() < 1e-12
    g = 1e-4
    L = ref3d.RefLattice3D(9, 7, 6, 2, body_force=g, **EMULSION)
    L.set_fields(rho)
    L.step(5)
    p5 = np.einsum("slzyx,la->a", L.fields()[2], c19)
    assert p5[0] == pytest.approx(5 * g * rho.sum(), rel=1e-10)
    assert np.abs(p5[1:]).max() < 1e-12


def _kernel(links, w_by_q, k, sel):
    """sum over the selected links of w(|c|^2) c sin(k . c) (a 3-vector)."""
    s = np.zeros(3)
    for c in links:
        if sel(c):
            s += w_by_q[int(c @ c)] * c * np.sin(k @ c)
    return s


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 1), (1, 1, 1), (2, -1, 1)])
def test_intra_force_closed_form(tab, m):
    """Eq. FORCE on psi = a + b sin(k.x) (psi = rho): F(x) = -psi(x) b cos(k.x) sum_l K c sin(k.c),
    exactly, with K = wn (G1 w_att + G2 w_rep)."""
    links, wa, wr = tab[0], tab[1], tab[2]
    nx, ny, nz = 12, 10, 8
    k = 2 * np.pi * np.array(m) / np.array([nx, ny, nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    psi = 0.7 + 0.2 * np.sin(ph)
    G1, G2, wn = -9.0, 8.1, 1.0 / 3.0
    L = ref3d.RefLattice3D(nx, ny, nz, 1, G1=G1, G2=G2, psi_form=1, weight_norm=wn)
    L.set_fields(psi[None])
    F = L.site_fields()["F"][0]
    K = wn * (G1 * _kernel(links, wa, k, lambda c: int(c @ c) <= 4) + G2 * _kernel(links, wr, k, lambda c: True))
    want = -psi * 0.2 * np.cos(ph)
    for d in range(3):
        assert np.allclose(F[d], want * K[d], rtol=0, atol=1e-14)


def test_cross_force_closed_form(tab):
    links, wc = tab[0], tab[3]
    nx, ny, nz = 10, 8, 6
    k = 2 * np.pi * np.array([1, 1, 0]) / np.array([nx, ny, nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = k[0] * x + k[1] * y
    rhoA = np.full((nz, ny, nx), 0.9)
    rhoB = 0.5 + 0.3 * np.sin(ph)
    G_AB, wn = 0.587, 1.0 / 3.0
    L = ref3d.RefLattice3D(nx, ny, nz, 2, G_AB=G_AB, weight_norm=wn)
    L.set_fields(np.stack([rhoA, rhoB]))
    F = L.site_fields()["F"]
    K = wn * _kernel(links, wc, k, lambda c: int(c @ c) <= 2)
    for d in range(3):
        assert np.allclose(F[0, d], -G_AB * rhoA * 0.3 * np.cos(ph) * K[d], rtol=0, atol=1e-14)
    assert np.abs(F[1]).max() < 1e-14  # B sees a uniform A


def test_sound_speed_follows_the_interaction_pressure(tab):
    """A density wave along x on a uniform state oscillates at omega = k c_eff with
    c_eff^2 = c_s^2 + psi psi' S(k) / k, S(k) = sum_l K c_x sin(k c_x) over the 3-D links
    (the linearised Eq. FORCE, as in two dimensions): within 5e-4; c_s alone is 12 % off."""
    links, wa, wr = tab[0], tab[1], tab[2]
    nx, G1, G2, wn, rb = 128, -9.0, 8.1, 1.0 / 3.0, 1.0
    k = 2 * np.pi / nx
    L = ref3d.RefLattice3D(nx, 2, 2, 1, G1=G1, G2=G2, weight_norm=wn)
    x = np.arange(nx)
    L.set_fields(np.broadcast_to(rb + 1e-6 * np.cos(k * x), (1, 2, 2, nx)).copy())
    A = np.empty(1000)
    for t in range(1000):
        r = L.fields()[0][0].mean(axis=(0, 1))
        A[t] = 2.0 / nx * np.sum((r - r.mean()) * np.cos(k * x))
        L.step(1)
    kv = np.array([k, 0.0, 0.0])
    S = wn * (G1 * _kernel(links, wa, kv, lambda c: int(c @ c) <= 4) + G2 * _kernel(links, wr, kv, lambda c: True))[0]
    c2 = 1.0 / 3.0 + (1 - np.exp(-rb)) * np.exp(-rb) * S / k
    s = np.sign(A)
    zc = np.where(s[1:] * s[:-1] < 0)[0]
    tz = zc + A[zc] / (A[zc] - A[zc + 1])
    omega = np.pi / np.mean(np.diff(tz))
    assert len(zc) >= 7
    assert omega == pytest.approx(k * np.sqrt(c2), rel=5e-4)
    assert abs(omega / (k / np.sqrt(3.0)) - 1) > 0.1


def test_flat_interface_bulk_pressures_equal():
    """A slab of the film couplings (G1, G2) = (-20.4, 16.0) relaxed to rest: mechanical
    equilibrium across a flat interface makes the two bulk pressures equal, and for a uniform
    density the lattice pressure is exactly P_b = c_s^2 rho + wn (G1 + G2) psi^2 / 2 (e2 = 1, as
    in two dimensions).  The field varies along x only, so one site across y and z carries it
    (the links wrap onto it).  Within 1e-9 (observed 2e-11) after 40000 steps."""
    G1, G2, wn = -20.4, 16.0, 1.0 / 3.0
    nx = 96
    x = np.arange(nx)
    L = ref3d.RefLattice3D(nx, 1, 1, 1, G1=G1, G2=G2, weight_norm=wn)
    L.set_fields((0.29 + 0.55 * (np.tanh((x - 24) / 3) - np.tanh((x - 72) / 3)))[None, None, None, :])
    L.step(40000)
    r, u, _ = L.fields()
    rl, rg = r[0, 0, 0, 48], r[0, 0, 0, 0]
    assert rl - rg > 1.0  # two phases
    assert np.abs(u).max() < 1e-12  # at rest
    P = lambda d: d / 3 + wn * (G1 + G2) * (1 - np.exp(-d)) ** 2 / 2
    assert abs(P(rl) - P(rg)) < 1e-9


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.7])
def test_couette_between_walls_exact(tau):
    """Walls at z = -1/2 and nz - 1/2 moving at U_b and U_t along x (halfway bounce-back with
    Ladd's term): the steady profile is exactly linear, u_x = U_b + (U_t - U_b)(z + 1/2)/nz, as in
    two dimensions; mass is conserved by the moving walls."""
    nz, Ub, Ut = 10, -0.01, 0.015
    L = ref3d.RefLattice3D(3, 2, nz, 1, tau=tau, zbc=1, wall_u=(Ub, Ut))
    L.set_fields(np.ones((1, nz, 2, 3)))
    m0 = L.fields()[0].sum()
    steps = int(40 * nz * nz / ((tau - 0.5) / 3))
    L.step(steps)
    r, u, _ = L.fields()
    z = np.arange(nz)
    exact = Ub + (Ut - Ub) * (z + 0.5) / nz
    assert np.abs(u[0, :, 0, 0] - exact).max() < 1e-12
    assert np.abs(u[1:]).max() < 1e-14
    # Ladd's term cancels between the populations a wall site reflects, up to rounding: at most
    # about one unit of 2^-52 per step (observed 2e-13 after 40000 steps)
    assert r.sum() == pytest.approx(m0, rel=steps * 2.0 ** -52)


def test_poiseuille_between_walls():
    """Body force g between resting walls: at steady state the interior obeys the discrete
    momentum balance nu (u_{z+1} - 2 u_z + u_{z-1}) = -g exactly (rho = 1), and the profile is the
    parabola g (z + 1/2)(nz - 1/2 - z) / (2 nu) up to the bounce-back slip of halfway walls."""
    nz, g, tau = 16, 1e-6, 1.0
    nu = (tau - 0.5) / 3
    L = ref3d.RefLattice3D(3, 2, nz, 1, tau=tau, zbc=1, body_force=g)
    L.set_fields(np.ones((1, nz, 2, 3)))
    L.step(int(40 * nz * nz / nu))
    u = L.fields()[1][0, :, 0, 0]
    lap = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.allclose(nu * lap, -g, rtol=1e-8, atol=0)
    z = np.arange(nz)
    parabola = g * (z + 0.5) * (nz - 0.5 - z) / (2 * nu)
    assert np.abs(u - parabola).max() < 0.02 * parabola.max()
