"""GPU parity: the CUDA step (through the C ABI) against the FP64 oracle, element by element.

Tolerances:
* FP64 path: relative L-inf <= 1e-12 on rho and u (the contract for the FP64 mode).  The two
  sides differ only by rounding (summation order, FMA, exp), and the workloads are not chaotic
  over these horizons.
* FP32 path (populations stored as deviations from W_l rho_ref): relative L-inf <= 1e-4 on rho
  and u after 1000 steps (the contract for the FP32 mode).
"""
import numpy as np
import pytest

from paper_1402_6019_gb300 import accuracy as A
from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4
KERNELS = pytest.mark.parametrize("kernel", [L.LBM_KERNEL_PULL, L.LBM_KERNEL_FUSED, L.LBM_KERNEL_TWO_PASS,
                                             L.LBM_KERNEL_SWEEP], ids=["pull", "tile", "twopass", "sweep"])


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def pair(oracle, nx, nz, ns, zbc, precision, rho, steps, u=None, kernel=L.LBM_KERNEL_AUTO, rpw=0, **prm):
    ref = oracle.RefLattice(nx, nz, ns, zbc, **prm)
    ref.set_fields(rho, u)
    ref.step(steps)
    lat = L.Lattice(nx, nz, ns, precision, zbc, kernel=kernel, rows_per_warp=rpw, **prm)
    lat.set_fields(rho, u)
    lat.step(steps)
    return ref, lat


def pop_scale(ref):
    """Magnitude of the terms the velocity is formed from, max over sites of
    sum_s sum_l |f_l,s c_l| / rho (about c_s^2 = 1/3 near rest)."""
    rho, _, f = ref.fields()
    c = np.array([0, 1, 1, 1, 1, 1, 1, 1, 1], float)  # |c_l| is 0 or 1 per component
    return float(((np.abs(f) * c[None, :, None, None]).sum(axis=(0, 1)) / rho.sum(0)).max())


def check_fields(ref, lat, tol, pops=True):
    """rho and f: relative L-inf <= tol.  u = sum_s (j_s + F_s/2)/rho is a difference of
    populations of size ~1/9: when the flow is nearly at rest (|u| ~ 1e-5) both FP64 sides carry
    an absolute rounding error of order eps * sum|f c|/rho in u, so the bound on u is
    tol * max|u| plus a rounding floor of 100 eps times that population scale."""
    r_rho, r_u, r_f = ref.fields()
    g_rho, g_u, g_f = lat.fields(populations=pops)
    e_rho = rel(g_rho, r_rho)
    err_u = float(np.abs(g_u - r_u).max())
    bound_u = tol * float(np.abs(r_u).max()) + 100 * 2.2e-16 * pop_scale(ref)
    assert e_rho <= tol, f"rho rel err {e_rho}"
    assert err_u <= bound_u, f"u err {err_u} > {bound_u}"
    if pops:
        e_f = rel(g_f, r_f)
        assert e_f <= tol, f"populations rel err {e_f}"
    return e_rho, err_u / max(float(np.abs(r_u).max()), 1e-300)


def check_obs(ref, lat, tol):
    """Every observable against the oracle's, within the bound its inputs allow under the state
    contract tol (paper_1402_6019_gb300.accuracy: tol times the magnitude of the terms each
    observable is formed from -- populations for velocities, Sec. III's pressure-tensor terms for
    S_xz, p_s, P_xx and gamma -- and the fluidity's bound propagated through its ratio)."""
    a, b = lat.observables(), ref.observables()
    assert not a["nonfinite"]
    return check_obs_against(a, b, ref.scales(), tol, ref.nx, float(np.sum(b["mass"])))


def check_obs_against(a, b, scales, tol, nx, total_mass):
    errs = A.observable_errors(a, b, scales, tol, nx, total_mass)
    assert set(errs) >= {"mass", "momentum", "gamma", "ux_z", "rho_z", "sxz_z", "fluid_z", "ps_x", "pxx_x"}
    bad = A.check(errs)
    assert not bad, {k: errs[k] for k in bad}
    return errs


def check_obs_fp32(a, g, mass0):
    """The 1024^2 golden's observables (FP32 contract tol 1e-4)."""
    scales = {k: float(g[k]) for k in ("rho_max", "u_max", "pop_scale", "stress_scale")}
    return check_obs_against(a, g, scales, TOL32, 1024, float(np.sum(mass0)))


# --- FP64: the contract at 1e-12 ------------------------------------------------------------

def test_fp64_single_component_128_periodic_1000_steps(oracle):
    w = W.workload("single_128")
    ref, lat = pair(oracle, 128, 128, 1, 0, L.LBM_FP64, w["rho"], 1000, **w["params"])
    check_fields(ref, lat, TOL64)
    check_obs(ref, lat, TOL64)
    o = lat.observables()
    assert abs(o["mass"][0] - w["rho"].sum()) / w["rho"].sum() < 1e-13


@KERNELS
@pytest.mark.parametrize("G_AB", [0.405, 0.587])
def test_fp64_emulsion_ragged_periodic(oracle, G_AB, kernel):
    nx, nz = 100, 75  # 100 = 3 strips of 28 + 16, and 3 tiles of 32 + 4: ragged in x and z
    rho, _ = W.disk_packing(nx, nz, 0.8, seed=3, r_mean=8, r_spread=2)
    ref, lat = pair(oracle, nx, nz, 2, 0, L.LBM_FP64, rho, 300, kernel=kernel,
                    **dict(W.EMULSION_PARAMS, G_AB=G_AB))
    check_fields(ref, lat, TOL64)
    check_obs(ref, lat, TOL64)


@KERNELS
@pytest.mark.parametrize("psi_wall", [0, 1])
def test_fp64_channel_walls_drives(oracle, psi_wall, kernel):
    nx, nz = 61, 37
    rho, _ = W.disk_packing(nx, nz, 0.7, seed=5, r_mean=6, r_spread=2, periodic_z=False)
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=(-0.01, 0.02), body_force=1e-5, psi_wall=psi_wall)
    ref, lat = pair(oracle, nx, nz, 2, 1, L.LBM_FP64, rho, 300, kernel=kernel, **prm)
    check_fields(ref, lat, TOL64)
    errs = check_obs(ref, lat, TOL64)
    assert errs["fluid_z"][3] > nz // 2  # sheared: the fluidity is determined in most rows


def test_fp64_unequal_tau_chem09_rho_psi(oracle):
    nx, nz = 45, 33
    rho, _ = W.disk_packing(nx, nz, 0.6, seed=8, r_mean=5, r_spread=1)
    prm = dict(W.EMULSION_PARAMS, tau=(0.8, 1.3), weight_preset=1, psi_form=1, G_AB=0.3,
               G1=(-1.0, -0.8), G2=(0.6, 0.5))
    ref, lat = pair(oracle, nx, nz, 2, 0, L.LBM_FP64, rho, 200, **prm)
    check_fields(ref, lat, TOL64)


@pytest.mark.parametrize("zbc", [0, 1], ids=["periodic", "walls"])
def test_fp32_unequal_tau_chem09_rho_psi(oracle, zbc):
    """Unequal relaxation times, the second weight set and psi = rho in FP32 deviations (the
    species then differ in every term of the packed collision): fields and observables at the
    FP32 bound."""
    nx, nz = 45, 33
    rho, _ = W.disk_packing(nx, nz, 0.6, seed=8, r_mean=5, r_spread=1, periodic_z=not zbc)
    prm = dict(W.EMULSION_PARAMS, tau=(0.8, 1.3), weight_preset=1, psi_form=1, G_AB=0.3,
               G1=(-1.0, -0.8), G2=(0.6, 0.5), wall_u=(-0.01, 0.01), body_force=1e-5)
    ref, lat = pair(oracle, nx, nz, 2, zbc, L.LBM_FP32, rho, 200, **prm)
    check_fields(ref, lat, TOL32, pops=False)
    check_obs(ref, lat, TOL32)


@KERNELS
@pytest.mark.parametrize("nx,nz,ns,zbc", [(1, 1, 1, 0), (5, 7, 2, 0), (3, 1, 1, 1), (29, 5, 2, 1),
                                           (30, 2, 1, 0), (57, 3, 2, 0), (2, 9, 2, 1)])
def test_fp64_tiny_and_degenerate(oracle, nx, nz, ns, zbc, kernel):
    rho = W.noise_field(nx, nz, seed=nx * 100 + nz, mean=0.8, amp=0.2, n_species=ns)
    u = 0.01 * W.noise_field(nx, nz, seed=7, mean=0.0, amp=1.0, n_species=2)
    prm = dict(W.EMULSION_PARAMS if ns == 2 else W.SINGLE_PARAMS, wall_u=(0.01, -0.02), body_force=2e-5)
    ref, lat = pair(oracle, nx, nz, ns, zbc, L.LBM_FP64, rho, 60, u=u, kernel=kernel, **prm)
    check_fields(ref, lat, TOL64)
    check_obs(ref, lat, TOL64)


@pytest.mark.parametrize("nx,nz,ns,zbc", [(1, 1, 1, 0), (5, 7, 2, 0), (3, 1, 1, 1), (29, 5, 2, 1),
                                           (30, 2, 1, 0), (57, 3, 2, 0), (2, 9, 2, 1)])
def test_fp32_tiny_and_degenerate(oracle, nx, nz, ns, zbc):
    """The same narrow lattices in FP32 deviations through the default step kernel (the packed
    two-species form where there are two): fields and observables at the FP32 bound."""
    rho = W.noise_field(nx, nz, seed=nx * 100 + nz, mean=0.8, amp=0.2, n_species=ns)
    u = 0.01 * W.noise_field(nx, nz, seed=7, mean=0.0, amp=1.0, n_species=2)
    prm = dict(W.EMULSION_PARAMS if ns == 2 else W.SINGLE_PARAMS, wall_u=(0.01, -0.02), body_force=2e-5)
    ref, lat = pair(oracle, nx, nz, ns, zbc, L.LBM_FP32, rho, 60, u=u, **prm)
    check_fields(ref, lat, TOL32, pops=False)
    check_obs(ref, lat, TOL32)


@pytest.mark.parametrize("rpw", [1, 3, 200])
def test_fp64_sweep_row_chunking(oracle, rpw):
    nx, nz = 64, 50
    rho, _ = W.disk_packing(nx, nz, 0.7, seed=9, r_mean=6, r_spread=2, periodic_z=False)
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=(0.0, 0.01))
    ref, lat = pair(oracle, nx, nz, 2, 1, L.LBM_FP64, rho, 50, rpw=rpw, kernel=L.LBM_KERNEL_SWEEP, **prm)
    check_fields(ref, lat, TOL64)
    check_obs(ref, lat, TOL64)


def test_graph_replay_equals_single_steps():
    nx, nz = 80, 40
    rho, _ = W.disk_packing(nx, nz, 0.7, seed=2, r_mean=6, r_spread=2)
    a = L.Lattice(nx, nz, 2, L.LBM_FP64, 0, **W.EMULSION_PARAMS)
    b = L.Lattice(nx, nz, 2, L.LBM_FP64, 0, **W.EMULSION_PARAMS)
    a.set_fields(rho)
    b.set_fields(rho)
    a.step(45)  # graph replays of 16 steps + 13 single steps
    for _ in range(45):
        b.step(1)
    fa, fb = a.fields()[2], b.fields()[2]
    assert np.array_equal(fa, fb)



@pytest.mark.parametrize("zbc", [L.LBM_PERIODIC, L.LBM_BOUNCEBACK], ids=["periodic", "walls"])
def test_mixed_launch_sequences_equal_single_steps(zbc):
    """Step launches alternate between two pairs of work counters and captured graphs are kept per
    pair, so a sequence that mixes graph replays, odd runs of single steps, observing and plain
    passes, observable reads and exports (other kernels on the stream) and the autotuner's trial
    launches must give the populations and time sums of single steps, bit for bit.  544 x 320
    has 680 tiles, more than the CTAs own at the start, so tiles are also drawn from the counter."""
    nx, nz = 544, 320
    rho, _ = W.disk_packing(nx, nz, 0.75, seed=23, r_mean=8, r_spread=2, periodic_z=zbc == L.LBM_PERIODIC)
    prm = dict(W.EMULSION_PARAMS, body_force=1e-6 if zbc else 0.0)
    lats = [L.Lattice(nx, nz, 2, L.LBM_FP32, zbc, **prm) for _ in range(2)]
    plan = [("step", 1), ("step", 16), ("observe", 1), ("step", 3), ("read", 0), ("step", 16), ("step", 17),
            ("fields", 0), ("tune", 0), ("step", 16), ("observe", 0), ("step", 5), ("observe", 1), ("step", 18)]
    for i, lat in enumerate(lats):
        lat.set_fields(rho)
        for op, n in plan:
            if op == "step":
                if i == 0:
                    lat.step(n)
                else:
                    for _ in range(n):
                        lat.step(1)
            elif op == "observe":
                lat.set_observe(n)
            elif op == "read":
                lat.averages()
            elif op == "fields":
                lat.fields(populations=False)
            else:
                lat.autotune(steps=3)
    fa, fb = lats[0].fields()[2], lats[1].fields()[2]
    assert np.array_equal(fa, fb)
    a, b = lats[0].averages(), lats[1].averages()
    assert a["samples"] == b["samples"] == 18
    for key in ("ux_z", "rho_z", "sxz_z", "ps_x", "mass", "momentum"):
        assert np.array_equal(a[key], b[key]), key
    assert not a["nonfinite"]

# --- FP32 deviations: the contract at 1e-4 after 1000 steps --------------------------------

@KERNELS
def test_fp32_emulsion_1000_steps(oracle, kernel):
    nx = nz = 128
    rho, _ = W.disk_packing(nx, nz, 0.8, seed=1402)
    ref, lat = pair(oracle, nx, nz, 2, 0, L.LBM_FP32, rho, 1000, kernel=kernel, **W.EMULSION_PARAMS)
    e_rho, e_u = check_fields(ref, lat, TOL32, pops=False)
    check_obs(ref, lat, TOL32)


def test_fp32_channel_1000_steps(oracle):
    nx, nz = 192, 64
    rho, _ = W.disk_packing(nx, nz, 0.85, seed=11, periodic_z=False)
    prm = dict(W.EMULSION_PARAMS, wall_u=(-0.01, 0.01), body_force=1e-6)
    ref, lat = pair(oracle, nx, nz, 2, 1, L.LBM_FP32, rho, 1000, **prm)
    check_fields(ref, lat, TOL32, pops=False)
    check_obs(ref, lat, TOL32)


def test_fp32_full_size_1024_against_oracle(oracle):
    """The benchmarked workload (1024^2 emulsion, FP32, the launch configuration of bench.py):
    every site against the oracle after 20 steps, and conservation after 1000 steps."""
    w = W.workload("emulsion_1024")
    ref, lat = pair(oracle, 1024, 1024, 2, 0, L.LBM_FP32, w["rho"], 20, **w["params"])
    check_fields(ref, lat, TOL32, pops=False)
    m0 = w["rho"].sum(axis=(1, 2))
    lat.step(980)
    o = lat.observables()
    assert np.allclose(o["mass"], m0, rtol=1e-5)
    assert np.abs(o["momentum"]).max() < 1e-6 * m0.sum()


def test_fp32_full_size_1024_1000_steps_against_oracle():
    """The benchmarked workload over the contract's horizon: the 1024^2 emulsion in FP32, stepped
    1000 times in the launch configuration of bench.py (observables every step), against the FP64
    oracle's state after 1000 steps at 13,312 sampled sites (three whole rows, two whole columns,
    8192 random sites) and against the oracle's observables of that state.  Expected values:
    tests/golden/emulsion_1024_1000.npz, written by tests/golden/make_emulsion_1024.py, which
    calls only the oracle.  rho and u: relative L-inf <= 1e-4 (the FP32 contract); the
    observables at their stated FP32 bounds (check_obs_fp32)."""
    import os

    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "emulsion_1024_1000.npz"))
    w = W.workload("emulsion_1024")
    lat = L.Lattice(1024, 1024, 2, L.LBM_FP32, 0, **w["params"])
    lat.set_fields(w["rho"])
    lat.set_observe(1)
    lat.step(int(g["steps"]))
    rho, u, _ = lat.fields(populations=False)
    z, x = g["z"], g["x"]
    e_rho = float(np.abs(rho[:, z, x] - g["rho"]).max() / g["rho_max"])
    e_u = float(np.abs(u[:, z, x] - g["u"]).max() / g["u_max"])
    assert e_rho <= TOL32, e_rho
    assert e_u <= TOL32, e_u
    check_obs_fp32(lat.observables(), g, w["rho"].sum(axis=(1, 2)))


@pytest.mark.parametrize("name", ["channel_couette", "channel_poiseuille"])
def test_fp32_full_size_channels_against_oracle(oracle, name):
    """The 2048 x 256 walled channel workloads (Couette and Poiseuille drives, FP32, observables
    every step as bench.py steps them): every site against the oracle after 10 steps."""
    w = W.workload(name)
    ref = oracle.RefLattice(w["nx"], w["nz"], 2, w["z_boundary"], **w["params"])
    ref.set_fields(w["rho"])
    ref.step(10)
    lat = L.Lattice(w["nx"], w["nz"], 2, L.LBM_FP32, w["z_boundary"], **w["params"])
    lat.set_fields(w["rho"])
    lat.set_observe(1)
    lat.step(10)
    check_fields(ref, lat, TOL32, pops=False)


def test_fp32_full_size_sweep_against_oracle(oracle):
    """The 48-channel sweep at full size (13.4 M sites, one launch per step, observables every
    step): after 5 steps, three channels -- H = 32, 256 and 512 under body forces 1e-6, 1e-5 and
    3e-6 -- equal the oracle run on each alone."""
    w = W.workload("channel_sweep_48")
    hs = w["instances"]
    lat = L.Lattice(w["nx"], None, 2, L.LBM_FP32, L.LBM_BOUNCEBACK, instances=hs, **w["params"])
    for i, d in enumerate(w["drives"]):
        lat.set_instance_drive(i, d["body_force"], d["wall_u"])
    lat.set_fields(w["rho"])
    lat.set_observe(1)
    lat.step(5)
    g_rho, g_u, _ = lat.fields(populations=False)
    z0 = np.concatenate([[0], np.cumsum(hs)])
    for i in (0, 23, 46):
        rho_i = w["rho"][:, z0[i]:z0[i + 1]]
        ref = oracle.RefLattice(w["nx"], hs[i], 2, 1, **dict(w["params"], **w["drives"][i]))
        ref.set_fields(rho_i)
        ref.step(5)
        r_rho, r_u, _ = ref.fields()
        assert rel(g_rho[:, z0[i]:z0[i + 1]], r_rho) <= TOL32, i
        err_u = float(np.abs(g_u[:, z0[i]:z0[i + 1]] - r_u).max())
        assert err_u <= TOL32 * float(np.abs(r_u).max()) + 100 * 2.2e-16 * pop_scale(ref), i


def test_fp32_state_is_stored_as_fp32_deviations():
    """FP32 mode stores f - W_l rho_ref in FP32 (rho_ref: each species' mean density, held as an
    FP32 number): the exported populations are FP64 values that carry the FP32 rounding of the
    deviations.  At rest on a uniform lattice every deviation is 0 and the export is W_l rho
    exactly; with rho = 1 + d the stored deviation W_l (rho - rho_ref) is rounded to FP32 once, so
    the export differs from the FP64 equilibrium W_l rho by at most half an FP32 ulp of the
    deviation -- about 2^-24 * 1e-3 here, not 2^-24 of W_l rho."""
    nx, nz = 64, 32
    lat = L.Lattice(nx, nz, 2, L.LBM_FP32, 0, **W.EMULSION_PARAMS)
    rho = np.ones((2, nz, nx))
    lat.set_fields(rho)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = lat.fields()[2]
    assert np.array_equal(f, np.broadcast_to(w[None, :, None, None], f.shape))
    rho = rho + 1e-3 * W.noise_field(nx, nz, seed=91, mean=0.0, amp=1.0, n_species=2)
    lat.set_fields(rho)
    f = lat.fields()[2]
    want = w[None, :, None, None] * rho[:, None]
    ref32 = np.float32(rho.mean(axis=(1, 2))).astype(np.float64)
    dev = w[None, :, None, None] * (rho - ref32[:, None, None])[:, None]
    err = np.abs(f - want)
    assert err.max() > 0  # the FP32 rounding is visible ...
    # ... at the scale of the deviation (plus FP64 rounding of the final sum)
    assert np.all(err <= 2.0 ** -24 * np.abs(dev) * 1.001 + 1e-14 + 4 * 2.0 ** -52 * want)
    assert err.max() < 1e-9 < 2.0 ** -24 * want.min()


# --- observables, averages, errors ------------------------------------------------------------

@KERNELS
def test_time_averages_match_oracle_mean(oracle, kernel):
    nx, nz = 48, 32
    rho, _ = W.disk_packing(nx, nz, 0.6, seed=12, r_mean=5, r_spread=1, periodic_z=False)
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=(-0.01, 0.01))
    ref = oracle.RefLattice(nx, nz, 2, 1, **prm)
    ref.set_fields(rho)
    lat = L.Lattice(nx, nz, 2, L.LBM_FP64, 1, kernel=kernel, **prm)
    lat.set_fields(rho)
    lat.set_observe(1)
    n = 20
    lat.step(n)  # 16 in a graph + 4 single
    acc = None
    for _ in range(n):
        o = ref.observables()
        acc = {k: o[k] / n for k in ("ux_z", "sxz_z", "fluid_z", "ps_x")} if acc is None else \
            {k: acc[k] + o[k] / n for k in acc}
        ref.step(1)
    av = lat.averages(reset=True)
    assert av["samples"] == n
    for k, v in acc.items():
        assert np.abs(av[k] - v).max() <= 1e-10 * max(np.abs(v).max(), 1e-12), k
    assert lat.averages()["samples"] == 0


def test_invalid_fields_rejected():
    """lbm_set_fields checks the densities on the device: a value <= 0, NaN or inf is refused,
    from host or device memory, and the first invalid one is named; a refused call changes
    nothing, and a valid one after it works."""
    import torch

    lat = L.Lattice(8, 8, 2, L.LBM_FP32, 0, **W.EMULSION_PARAMS)
    rho = np.ones((2, 8, 8))
    rho[1, 5, 6] = -2.0
    rho[1, 3, 4] = 0.0
    with pytest.raises(L.LbmError) as e:
        lat.set_fields(rho)
    assert e.value.code == L.LBM_EINVAL
    assert "rho[1][28] = 0 " in str(e.value)  # the first of the two, at 3 * 8 + 4
    for bad in (np.nan, np.inf):
        rho[1, 3, 4] = bad
        with pytest.raises(L.LbmError):
            lat.set_fields(rho)
        with pytest.raises(L.LbmError):
            lat.set_fields(torch.from_numpy(rho).cuda())
    with pytest.raises(L.LbmError):
        lat.step(1)  # no fields yet
    with pytest.raises(L.LbmError):
        lat.set_params(tau=0.5)
    lat.set_fields(np.ones((2, 8, 8)))
    lat.step(2)
    assert np.allclose(lat.fields()[0], 1.0)


def test_nonfinite_state_is_reported():
    """An unstable coupling drives densities negative; the kernels flag it and the host reports
    LBM_ENONFINITE (a property of the data: no GPU fault is involved)."""
    lat = L.Lattice(32, 32, 1, L.LBM_FP64, 0, G1=-60.0, G2=0.0, psi_form=1, weight_norm=1.0)
    lat.set_fields(W.noise_field(32, 32, seed=3, mean=1.0, amp=0.3))
    lat.step(200)
    with pytest.raises(L.LbmError) as e:
        lat.synchronize()
    assert e.value.code == L.LBM_ENONFINITE
