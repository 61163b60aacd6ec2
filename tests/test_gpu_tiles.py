"""Tile shapes of the pull kernel (lbm_set_tile_shape, lbm_autotune_tiles): 32 x 8 or 64 x 8
sites per tile at pipeline depth 1 or 2.  The shape decides which CTA does which sites and how
much of the halo it reads; the row sums stay per 32 columns and the column sums per 8 rows, so
the populations, the time sums of every observable and the current observables must agree bit
for bit across shapes.  Lattices with ragged tiles in x (96 and 40 columns: a half-filled or
mostly empty 64-wide tile) and in z, periodic and walled, and a stacked batch of walled channels
of uneven heights."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P, B = L.LBM_PERIODIC, L.LBM_BOUNCEBACK
SHAPES = [(32, 1), (32, 2), (64, 1), (64, 2)]
PROFILES = ("ux_z", "rho_z", "sxz_z", "ps_x", "pxx_x", "mass", "momentum", "wall_force")


def make(nx, nz, zbc, instances, seed, shape, ns=2):
    prm = dict(W.EMULSION_PARAMS if ns == 2 else W.SINGLE_PARAMS)
    if zbc == B:
        prm.update(body_force=2e-6, wall_u=(-0.01, 0.01))
    lat = L.Lattice(nx, nz, ns, L.LBM_FP32, zbc, instances=instances, **prm)
    if instances:
        for i in range(len(instances)):
            lat.set_instance_drive(i, 1e-6 * (i + 1), (-0.005 * i, 0.005 * i))
    lat.set_tile_shape(*shape)
    nzt = sum(instances) if instances else nz
    rho, _ = W.disk_packing(nx, nzt, 0.7, seed=seed, r_mean=5, r_spread=1, periodic_z=zbc == P)
    if ns == 1:
        rho = (0.8 + 0.3 * (rho[0] - rho[0].mean()))[None]
    lat.set_fields(rho)
    return lat


def run(lat, observed, plain):
    lat.set_observe(1)
    lat.step(observed)
    lat.set_observe(0)
    lat.step(plain)
    lat.set_observe(1)
    lat.step(observed)
    return lat.fields()[2], lat.averages(), lat.observables()


@pytest.mark.parametrize("nx,nz,zbc,instances,ns", [
    (544, 320, P, None, 2),
    (96, 33, P, None, 2),
    (40, 24, P, None, 2),
    (200, 70, B, None, 2),
    (160, None, B, [20, 37, 16, 48], 2),
    (136, 45, P, None, 1),
    (100, 30, B, None, 1),
])
def test_tile_shapes_are_bit_identical(nx, nz, zbc, instances, ns):
    out = []
    for shape in SHAPES:
        lat = make(nx, nz, zbc, instances, 17 + nx, shape, ns)
        out.append(run(lat, 9, 7))
        lat.close()
    f0, a0, o0 = out[0]
    for (f, a, o), shape in zip(out[1:], SHAPES[1:]):
        assert np.array_equal(f, f0), f"populations, shape {shape}"
        assert a["samples"] == a0["samples"] == 9  # set_observe resets the sums
        for key in PROFILES:
            assert np.array_equal(a[key], a0[key]), f"time sums of {key}, shape {shape}"
            assert np.array_equal(o[key], o0[key]), f"{key}, shape {shape}"


def test_autotune_tiles_keeps_the_state_and_picks_the_fastest():
    lat = make(544, 320, P, None, 5, (32, 1))
    lat.set_observe(1)
    lat.step(5)
    before = lat.fields()[2]
    avg = lat.averages()
    (width, depth), ms = lat.autotune_tiles(steps=4)
    assert (width, depth) in SHAPES and min(ms) > 0 and ms[SHAPES.index((width, depth))] == min(ms)
    assert np.array_equal(lat.fields()[2], before)
    after = lat.averages()
    assert after["samples"] == avg["samples"] and np.array_equal(after["ux_z"], avg["ux_z"])
    ref = make(544, 320, P, None, 5, (32, 1))
    ref.set_observe(1)
    ref.step(12)
    lat.step(7)
    assert np.array_equal(lat.fields()[2], ref.fields()[2])


def test_tile_shape_arguments():
    lat = L.Lattice(64, 32, 2, L.LBM_FP32, P, **W.EMULSION_PARAMS)
    for bad in ((48, 1), (64, 3), (32, 0)):
        with pytest.raises(L.LbmError):
            lat.set_tile_shape(*bad)
    d = L.Lattice(64, 32, 2, L.LBM_FP64, P, **W.EMULSION_PARAMS)
    d.set_tile_shape(32, 1)
    with pytest.raises(L.LbmError):
        d.set_tile_shape(64, 1)
    rho, _ = W.disk_packing(64, 32, 0.6, seed=3, r_mean=4, r_spread=1)
    d.set_fields(rho)
    (w, dep), ms = d.autotune_tiles(steps=2)
    assert w == 32 and ms[2] == 0 and ms[3] == 0
    f = L.Lattice(64, 32, 2, L.LBM_FP32, P, kernel=L.LBM_KERNEL_FUSED, **W.EMULSION_PARAMS)
    with pytest.raises(L.LbmError):
        f.set_tile_shape(32, 1)


@pytest.mark.parametrize("zbc", [P, B], ids=["periodic", "walls"])
def test_tile_row_direction_does_not_change_results(zbc):
    """Consecutive launches take the tile rows in opposite directions.  An extra launch (a read
    of the current observables) flips the direction of every later step, which must not change
    the populations or the time sums."""
    a = make(288, 72, zbc, None, 11, (32, 1))
    b = make(288, 72, zbc, None, 11, (32, 1))
    for lat in (a, b):
        lat.set_observe(1)
    for k in range(6):
        a.step(3)
        b.step(3)
        if k % 2 == 0:
            b.observables()  # one more launch on b: its next steps run the other way round
    assert np.array_equal(a.fields()[2], b.fields()[2])
    ra, rb = a.averages(), b.averages()
    assert ra["samples"] == rb["samples"] == 18
    for key in PROFILES:
        assert np.array_equal(ra[key], rb[key]), key
