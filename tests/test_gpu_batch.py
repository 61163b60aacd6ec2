"""A batch of channels of different heights and drives stepped together (the pull kernel's
stacked lattices) against the FP64 oracle run on each channel alone."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEIGHTS = [13, 24, 40]  # 13: a ragged last tile row; the three share nx
DRIVES = [dict(body_force=1e-5, wall_u=(0.0, 0.0)),        # Poiseuille
          dict(body_force=0.0, wall_u=(-0.01, 0.01)),      # Couette
          dict(body_force=3e-6, wall_u=(0.005, -0.002))]   # both


def channel_rho(nx, h, seed):
    rho, _ = W.disk_packing(nx, h, 0.7, seed=seed, r_mean=4, r_spread=1, periodic_z=False)
    return rho


def run_pair(oracle, nx, precision, steps, prm, observe=0):
    rhos = [channel_rho(nx, h, 31 + i) for i, h in enumerate(HEIGHTS)]
    lat = L.Lattice(nx, None, 2, precision, L.LBM_BOUNCEBACK, instances=HEIGHTS, **prm)
    for i, d in enumerate(DRIVES):
        lat.set_instance_drive(i, d["body_force"], d["wall_u"])
    lat.set_fields(np.concatenate(rhos, axis=1))
    if observe:
        lat.set_observe(observe)
    refs = []
    for i, h in enumerate(HEIGHTS):
        ref = oracle.RefLattice(nx, h, 2, 1, **dict(prm, **DRIVES[i]))
        ref.set_fields(rhos[i])
        refs.append(ref)
    return lat, refs


def split(a, axis):
    return np.split(a, np.cumsum(HEIGHTS)[:-1], axis=axis)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_fp64_batch_matches_each_channel_alone(oracle):
    nx, steps = 61, 150
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587)
    lat, refs = run_pair(oracle, nx, L.LBM_FP64, steps, prm)
    lat.step(steps)
    for ref in refs:
        ref.step(steps)
    rho, u, f = lat.fields()
    for i, (r_rho, r_u, r_f) in enumerate(zip(split(rho, 1), split(u, 1), split(f, 2))):
        e_rho, e_u, e_f = refs[i].fields()
        assert rel(r_rho, e_rho) < 1e-12, i
        assert rel(r_f, e_f) < 1e-12, i
        assert np.abs(r_u - e_u).max() <= 1e-12 * np.abs(e_u).max() + 1e-14, i
        a, b = lat.instance_observables(i), refs[i].observables()
        assert np.allclose(a["mass"], b["mass"], rtol=1e-12, atol=0), i
        assert np.allclose(a["momentum"], b["momentum"], rtol=0, atol=1e-11 * b["mass"].sum()), i
        assert np.allclose(a["wall_force"], b["wall_force"], rtol=1e-10, atol=1e-17), i
        for k in ("ux_z", "sxz_z", "rho_z", "fluid_z"):
            s = max(np.abs(b[k]).max(), 1e-30)
            assert np.abs(a[k] - b[k]).max() <= 1e-10 * s + 1e-15, (i, k)


def test_fp32_batch_500_steps(oracle):
    nx, steps = 96, 500
    lat, refs = run_pair(oracle, nx, L.LBM_FP32, steps, dict(W.EMULSION_PARAMS))
    lat.step(steps)
    rho, u, _ = lat.fields(populations=False)
    for i, (r_rho, r_u) in enumerate(zip(split(rho, 1), split(u, 1))):
        refs[i].step(steps)
        e_rho, e_u, _ = refs[i].fields()
        assert rel(r_rho, e_rho) < 1e-4, i
        assert np.abs(r_u - e_u).max() <= 1e-4 * np.abs(e_u).max() + 1e-6, i


def test_batch_time_averages(oracle):
    nx, n = 40, 20
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587)
    lat, refs = run_pair(oracle, nx, L.LBM_FP64, n, prm, observe=1)
    lat.step(n)  # a 16-step graph and 4 single steps
    for i, ref in enumerate(refs):
        acc = None
        for _ in range(n):
            o = ref.observables()
            acc = {k: o[k] / n for k in ("ux_z", "sxz_z", "fluid_z")} if acc is None else \
                {k: acc[k] + o[k] / n for k in acc}
            ref.step(1)
        av = lat.instance_observables(i, averages=True)
        assert av["samples"] == n
        for k, v in acc.items():
            assert np.abs(av[k] - v).max() <= 1e-10 * max(np.abs(v).max(), 1e-12), (i, k)


def test_batch_validation():
    with pytest.raises(L.LbmError):  # heights must add up to nz, walls only
        L.Lattice(32, None, 2, L.LBM_FP32, L.LBM_PERIODIC, instances=[8, 8], **W.EMULSION_PARAMS)
    lat = L.Lattice(32, None, 2, L.LBM_FP32, L.LBM_BOUNCEBACK, instances=[8, 16], **W.EMULSION_PARAMS)
    with pytest.raises(L.LbmError):
        lat.set_instance_drive(2, 1e-6)
    with pytest.raises(L.LbmError):
        lat.set_instance_drive(0, float("nan"))


def test_autotune_keeps_state_and_results():
    """Tuning times both launch shapes on the lattice itself, then puts the state back; the shape
    kept changes the schedule of the tiles, not their arithmetic."""
    nx = 96
    rho = np.concatenate([channel_rho(nx, h, 5 + i) for i, h in enumerate(HEIGHTS)], axis=1)
    lats = []
    for tune in (False, True):
        lat = L.Lattice(nx, None, 2, L.LBM_FP32, L.LBM_BOUNCEBACK, instances=HEIGHTS, **W.EMULSION_PARAMS)
        lat.set_fields(rho)
        lat.set_observe(1)
        lat.step(7)
        lats.append(lat)
    before = lats[1].fields()[2]
    depth, ms = lats[1].autotune(steps=5)
    assert depth in (1, 2) and ms[0] > 0 and ms[1] > 0
    assert np.array_equal(lats[1].fields()[2], before)
    for lat in lats:
        lat.step(9)
    assert np.array_equal(lats[0].fields()[2], lats[1].fields()[2])
    a, b = lats[0].averages(), lats[1].averages()
    assert a["samples"] == b["samples"] == 16
    assert np.array_equal(a["ux_z"], b["ux_z"])
