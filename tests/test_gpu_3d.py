"""The three-dimensional extension (include/lbm3d.h: D3Q19, Eq. FORCE over the 92 links of
|c|^2 <= 8, the first-belt cross term, the shifted-velocity BGK of Sec. II, walls of Sec. IV)
through the C ABI, against the FP64 three-dimensional oracle, element by element.

Tolerances as for the 2-D step: FP64 relative L-inf <= 1e-12 on rho and the populations, and on
u <= 1e-12 max|u| plus a rounding floor of 100 eps times the population scale the velocity is a
difference of; FP32 (deviations from W_l rho_ref) <= 1e-4 on rho and u."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4
EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def ref3d():
    from oracle import ref3d as R

    R.build()
    return R


def _ref_params(prm, zbc):
    keys = ("tau", "G1", "G2", "G_AB", "rho0", "weight_norm", "body_force", "psi_form", "wall_u")
    return dict({k: prm[k] for k in keys if k in prm}, zbc=zbc)


def pair3(ref3d, nx, ny, nz, ns, zbc, precision, rho, steps, **prm):
    ref = ref3d.RefLattice3D(nx, ny, nz, ns, **_ref_params(prm, zbc))
    ref.set_fields(rho)
    ref.step(steps)
    lat = L.Lattice3(nx, ny, nz, ns, precision, zbc, **prm)
    lat.set_fields(rho)
    lat.step(steps)
    return ref, lat


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def pop_scale(f, rho):
    c = np.array([0] + [1] * 18, float)
    return float(((np.abs(f) * c[None, :, None, None, None]).sum(axis=(0, 1)) / rho.sum(0)).max())


def check3(ref, lat, tol, pops=True):
    r_rho, r_u, r_f = ref.fields()
    g_rho, g_u, g_f = lat.fields(populations=pops)
    e_rho = rel(g_rho, r_rho)
    err_u = float(np.abs(g_u - r_u).max())
    bound_u = tol * float(np.abs(r_u).max()) + 100 * EPS * pop_scale(r_f, r_rho)
    assert e_rho <= tol, f"rho rel err {e_rho}"
    assert err_u <= bound_u, f"u err {err_u} > {bound_u}"
    if pops:
        assert rel(g_f, r_f) <= tol, f"populations rel err {rel(g_f, r_f)}"
    return e_rho, err_u


@pytest.mark.parametrize("G_AB", [0.405, 0.587])
def test_fp64_periodic_emulsion_ragged(ref3d, G_AB):
    nx, ny, nz = 37, 13, 9  # ragged in every direction (tiles of 32 x 4 x 2)
    rho, _ = W.sphere_packing(nx, ny, nz, 0.45, seed=31, r_mean=3, r_spread=1)
    ref, lat = pair3(ref3d, nx, ny, nz, 2, 0, L.LBM_FP64, rho, 60, **dict(W.EMULSION_PARAMS, G_AB=G_AB))
    check3(ref, lat, TOL64)


@pytest.mark.parametrize("ns", [1, 2])
def test_fp64_walls_and_drives(ref3d, ns):
    nx, ny, nz = 24, 10, 11
    rho, _ = W.sphere_packing(nx, ny, nz, 0.4, seed=33, r_mean=3, r_spread=1, periodic_z=False)
    if ns == 1:
        rho = (0.8 + 0.3 * (rho[0] - rho[0].mean()))[None]
        prm = dict(W.SINGLE_PARAMS, wall_u=(-0.01, 0.02), body_force=1e-5)
    else:
        prm = dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=(-0.01, 0.02), body_force=1e-5)
    ref, lat = pair3(ref3d, nx, ny, nz, ns, 1, L.LBM_FP64, rho, 60, **prm)
    check3(ref, lat, TOL64)


@pytest.mark.parametrize("precision,tol", [(L.LBM_FP64, TOL64), (L.LBM_FP32, TOL32)])
def test_unequal_tau_rho_pseudopotential(ref3d, precision, tol):
    """Unequal relaxation times and psi = rho, in FP64 and in the FP32 packed form (the two
    species then differ in every term of the pair collision)."""
    nx, ny, nz = 20, 9, 12
    rho, _ = W.sphere_packing(nx, ny, nz, 0.4, seed=35, r_mean=3, r_spread=1)
    prm = dict(W.EMULSION_PARAMS, tau=(0.8, 1.3), psi_form=1, G_AB=0.3, G1=(-1.0, -0.8), G2=(0.6, 0.5))
    ref, lat = pair3(ref3d, nx, ny, nz, 2, 0, precision, rho, 50, **prm)
    check3(ref, lat, tol, pops=precision == L.LBM_FP64)


@pytest.mark.parametrize("precision,tol", [(L.LBM_FP64, TOL64), (L.LBM_FP32, TOL32)])
@pytest.mark.parametrize("nx,ny,nz,ns,zbc", [(1, 1, 1, 1, 0), (3, 2, 5, 2, 1), (5, 7, 3, 2, 0), (2, 9, 4, 1, 1),
                                              (33, 1, 1, 2, 0), (4, 3, 1, 2, 1)])
def test_tiny_and_degenerate(ref3d, nx, ny, nz, ns, zbc, precision, tol):
    """Lattices narrower than the halo in some direction (every neighbour an image, several
    times over), with walls or periodic, in FP64 and in the FP32 packed form."""
    rho = 0.8 + 0.2 * (2.0 * W.uniform(nx * 100 + ny * 10 + nz, ns * nx * ny * nz) - 1.0)
    rho = rho.reshape(ns, nz, ny, nx)
    prm = dict(W.EMULSION_PARAMS if ns == 2 else W.SINGLE_PARAMS, wall_u=(0.01, -0.02), body_force=2e-5)
    ref, lat = pair3(ref3d, nx, ny, nz, ns, zbc, precision, rho, 20, **prm)
    check3(ref, lat, tol, pops=precision == L.LBM_FP64)


def test_fp32_emulsion_against_oracle(ref3d):
    nx, ny, nz = 48, 40, 32
    rho, _ = W.sphere_packing(nx, ny, nz, 0.5, seed=37, r_mean=5, r_spread=1)
    ref, lat = pair3(ref3d, nx, ny, nz, 2, 0, L.LBM_FP32, rho, 300, **W.EMULSION_PARAMS)
    check3(ref, lat, TOL32, pops=False)


@pytest.mark.parametrize("ns", [1, 2])
def test_fp32_walls_and_drives_against_oracle(ref3d, ns):
    """FP32 deviations between moving walls with a body force (halfway bounce-back with Ladd's
    term, the mirror images of the densities beyond the walls), 200 steps, against the FP64
    oracle at the FP32 bound; two species with unequal relaxation times."""
    nx, ny, nz = 40, 12, 18
    rho, _ = W.sphere_packing(nx, ny, nz, 0.4, seed=57, r_mean=3, r_spread=1, periodic_z=False)
    if ns == 1:
        rho = (0.8 + 0.3 * (rho[0] - rho[0].mean()))[None]
        prm = dict(W.SINGLE_PARAMS, wall_u=(-0.02, 0.02), body_force=1e-5)
    else:
        prm = dict(W.EMULSION_PARAMS, tau=(1.0, 1.2), G_AB=0.587, wall_u=(-0.02, 0.02), body_force=1e-5)
    ref, lat = pair3(ref3d, nx, ny, nz, ns, 1, L.LBM_FP32, rho, 200, **prm)
    check3(ref, lat, TOL32, pops=False)


def test_fp64_conservation_and_body_force():
    """Eq. LB conserves each species' mass; the interaction forces are pairwise antisymmetric,
    so on a periodic lattice the lattice momentum grows by exactly g sum(rho) per step."""
    nx, ny, nz, g = 30, 20, 16, 3e-6
    rho, _ = W.sphere_packing(nx, ny, nz, 0.45, seed=39, r_mean=4, r_spread=1)
    lat = L.Lattice3(nx, ny, nz, 2, L.LBM_FP64, 0, **dict(W.EMULSION_PARAMS, G_AB=0.587, body_force=g))
    lat.set_fields(rho)
    m0, j0 = lat.totals()
    lat.step(40)
    m1, j1 = lat.totals()
    assert np.abs(m1 - m0).max() < 1e-13 * m0.max()
    assert j1[0] - j0[0] == pytest.approx(40 * g * m0.sum(), rel=1e-9)
    assert np.abs(j1[1:]).max() < 1e-12 * m0.sum()


def test_fp32_full_size_bench_workload_against_oracle(ref3d):
    """The benchmarked 3-D workload (128^3 periodic A/B emulsion, FP32, two species): every site
    against the FP64 oracle after 2 steps, in the launch configuration bench.py times."""
    w = W.workload("emulsion3d_128")
    n = w["nx"]
    ref = ref3d.RefLattice3D(n, n, n, 2, **_ref_params(w["params"], 0))
    ref.set_fields(w["rho"])
    ref.step(2)
    lat = L.Lattice3(n, n, n, 2, L.LBM_FP32, 0, **w["params"])
    lat.set_fields(w["rho"])
    lat.step(2)
    check3(ref, lat, TOL32, pops=False)


def test_invalid_input_rejected():
    import torch

    lat = L.Lattice3(8, 8, 8, 2, L.LBM_FP32, 0, **W.EMULSION_PARAMS)
    rho = np.ones((2, 8, 8, 8))
    rho[1, 2, 3, 4] = -1.0
    rho[1, 5, 0, 0] = np.nan
    with pytest.raises(L.LbmError) as e:
        lat.set_fields(rho)
    assert e.value.code == L.LBM_EINVAL
    assert "rho[1][156] = -1" in str(e.value)  # the first of the two: (2 * 8 + 3) * 8 + 4
    rho[1, 2, 3, 4] = np.inf
    with pytest.raises(L.LbmError):
        lat.set_fields(torch.from_numpy(rho).cuda())
    with pytest.raises(L.LbmError):
        lat.step(1)  # no fields yet
    with pytest.raises(L.LbmError):
        lat.set_params(**dict(W.EMULSION_PARAMS, weight_preset=1))
    with pytest.raises(L.LbmError) as e:
        lat.set_params(**dict(W.EMULSION_PARAMS, psi_wall=L.LBM_WALL_ZERO))
    assert e.value.code == L.LBM_EINVAL and "mirror" in str(e.value)


@pytest.mark.parametrize("precision", [L.LBM_FP64, L.LBM_FP32])
def test_tile_shapes_are_bit_identical_and_autotune_restores_the_state(precision):
    """The collide pass's tile shapes change which CTA does which sites, not the arithmetic:
    every shape gives the same populations bit for bit (a ragged lattice with walls, so every
    shape has partial tiles); lbm3_autotune leaves the state and step counter as they were."""
    nx, ny, nz = 45, 18, 13
    rho, _ = W.sphere_packing(nx, ny, nz, 0.4, seed=43, r_mean=3, r_spread=1, periodic_z=False)
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=(-0.01, 0.01), body_force=1e-5)
    got = []
    for shape in range(4):
        lat = L.Lattice3(nx, ny, nz, 2, precision, 1, **prm)
        lat.set_shape(shape)
        lat.set_fields(rho)
        lat.step(15)
        got.append(lat.fields()[2])
    for g in got[1:]:
        assert np.array_equal(g, got[0])
    lat = L.Lattice3(nx, ny, nz, 2, precision, 1, **prm)
    lat.set_fields(rho)
    lat.step(5)
    before = lat.fields()[2]
    shape, ms = lat.autotune(3)
    assert 0 <= shape < 4 and min(ms) > 0 and ms[shape] == min(ms)
    assert np.array_equal(lat.fields()[2], before)
    lat.step(10)
    assert np.array_equal(lat.fields()[2], got[0])
    with pytest.raises(L.LbmError):
        lat.set_shape(4)


@pytest.mark.parametrize("precision", [L.LBM_FP32, L.LBM_FP64])
@pytest.mark.parametrize("nx,ny,nz,ns,zbc", [(1, 1, 1, 1, 0), (3, 2, 5, 2, 1), (5, 7, 3, 2, 0), (2, 9, 4, 1, 1),
                                              (33, 1, 1, 2, 0), (4, 3, 1, 2, 1), (37, 13, 9, 1, 0), (70, 21, 6, 1, 1)])
def test_tile_shapes_bit_identical_on_small_lattices(nx, ny, nz, ns, zbc, precision):
    """Every tile shape is a different instance of the collide kernel; the site update fixes the
    rounding of each of its operations, so one species (the scalar collision) and two agree bit
    for bit across shapes on tiny, degenerate and ragged lattices, periodic or walled."""
    rho = 0.8 + 0.2 * (2.0 * W.uniform(nx * 100 + ny * 10 + nz, ns * nx * ny * nz) - 1.0)
    rho = rho.reshape(ns, nz, ny, nx)
    prm = dict(W.EMULSION_PARAMS if ns == 2 else W.SINGLE_PARAMS, wall_u=(0.01, -0.02), body_force=2e-5)
    out = []
    for shape in range(4):
        lat = L.Lattice3(nx, ny, nz, ns, precision, zbc, **prm)
        lat.set_shape(shape)
        lat.set_fields(rho)
        lat.step(12)
        out.append(lat.fields()[2])
    for g in out[1:]:
        assert np.array_equal(g, out[0])


@pytest.mark.parametrize("precision,ns", [(L.LBM_FP32, 2), (L.LBM_FP64, 2), (L.LBM_FP32, 1)])
def test_step_totals_records_are_the_totals(precision, ns):
    """lbm3_step_totals writes, after every step, the totals lbm3_totals returns (the same sums in
    the same order, so the same bits) into pinned host or device records; bad arguments are
    refused."""
    import torch

    nx, ny, nz = 37, 13, 9
    rho, _ = W.sphere_packing(nx, ny, nz, 0.45, seed=31, r_mean=3, r_spread=1)
    if ns == 1:
        rho = rho[:1]
    prm = dict(W.EMULSION_PARAMS if ns == 2 else W.SINGLE_PARAMS, body_force=2e-5)
    ref = L.Lattice3(nx, ny, nz, ns, precision, 0, **prm)
    ref.set_fields(rho)
    expected = []
    for _ in range(7):
        ref.step(1)
        m, j = ref.totals()
        expected.append(np.concatenate([m, np.zeros(2 - ns), j]))
    expected = np.array(expected)
    host = torch.zeros((7, 6), dtype=torch.float64).pin_memory()  # stride 48 bytes
    dev = torch.zeros((7, 5), dtype=torch.float64, device="cuda")
    for out, stride in ((host, 48), (dev, 40)):
        lat = L.Lattice3(nx, ny, nz, ns, precision, 0, **prm)
        lat.set_fields(rho)
        t1 = lat.step_totals(3, out, stride=stride)
        t2 = lat.step_totals(4, out[3:], stride=stride)
        assert t2 == t1 + 1
        lat.wait(t2)
        got = out[:, :5].cpu().numpy()
        assert np.array_equal(got, expected)
        lat.synchronize()
    lat = L.Lattice3(nx, ny, nz, ns, precision, 0, **prm)
    lat.set_fields(rho)
    with pytest.raises(L.LbmError):
        lat.step_totals(2, np.zeros((2, 5)).ctypes.data, stride=40)  # pageable host memory
    with pytest.raises(L.LbmError):
        lat.step_totals(2, dev, stride=32)
    with pytest.raises(L.LbmError):
        lat.step_totals(-1, dev)
    with pytest.raises(L.LbmError):
        lat.wait(0)  # no ticket issued yet
    # more runs than the 64 events kept: waiting on an old ticket waits for the whole stream
    tickets = [lat.step_totals(1, dev[k % 7:], stride=40) for k in range(66)]
    assert tickets == list(range(66))
    lat.wait(0)
    lat.wait(65)
    with pytest.raises(L.LbmError):
        lat.wait(66)


@pytest.mark.parametrize("precision,tol", [(L.LBM_FP64, 1e-12), (L.LBM_FP32, 1e-6)])
def test_totals_equal_sums_of_the_exported_state(precision, tol):
    """lbm3_totals (the density pass's FP64 block partials, on a 40^3 lattice whose grid of the
    totals loops over the planes) against the mass and lattice momentum summed on the host from
    the exported densities and populations."""
    n = 40
    rho, _ = W.sphere_packing(n, n, n, 0.45, seed=51, r_mean=4, r_spread=1)
    lat = L.Lattice3(n, n, n, 2, precision, 1, **dict(W.EMULSION_PARAMS, body_force=1e-5, wall_u=(0.01, -0.01)))
    lat.set_fields(rho)
    lat.step(7)
    m, j = lat.totals()
    r, _, f = lat.fields()
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0],
                  [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1],
                  [0, -1, -1], [0, 1, -1], [0, -1, 1]], float)
    mass = r.sum(axis=(1, 2, 3))
    mom = np.einsum("slzyx,lk->k", f, c)
    assert np.abs(m - mass).max() <= tol * mass.max()
    assert np.abs(j - mom).max() <= tol * mass.sum() * 1e-2

