"""Asynchronous reads of the observables (lbm_observables_enqueue / lbm_wait /
lbm_observables_unpack) give exactly what the synchronous reads give."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ["mass", "momentum", "wall_force", "ux_z", "rho_z", "sxz_z", "fluid_z", "ps_x", "pxx_x"]


def same(a, b):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    assert a["gamma"] == b["gamma"] and a["step"] == b["step"] and a["samples"] == b["samples"]


@pytest.mark.parametrize("precision,zb", [(L.LBM_FP32, L.LBM_PERIODIC), (L.LBM_FP64, L.LBM_BOUNCEBACK)])
def test_async_reads_equal_sync_reads(precision, zb):
    nx, nz = 96, 40
    rho, _ = W.disk_packing(nx, nz, 0.6, 5, r_mean=5, r_spread=1, periodic_z=zb == L.LBM_PERIODIC)
    prm = dict(W.EMULSION_PARAMS, wall_u=(-0.01, 0.01)) if zb else dict(W.EMULSION_PARAMS)
    a = L.Lattice(nx, nz, 2, precision, zb, **prm)
    b = L.Lattice(nx, nz, 2, precision, zb, **prm)
    for lat in (a, b):
        lat.set_fields(rho)
        lat.set_observe(1)
    r = a.reader(depth=2)
    pending = None
    for k in range(6):
        a.step(3)
        b.step(3)
        t = r.enqueue(averages=True, reset=True)
        want = b.averages(reset=True)
        if pending is not None:
            r.result(pending)
        pending = t
        got = r.result(t)
        same(got, want)
    # the current state
    t = r.enqueue(averages=False)
    same(r.result(t), b.observables())


def test_completed_sums_lag_by_one_sample():
    """averages = 2: each record holds the samples whose reductions are done; over a run every
    sample is read exactly once, and the records' sums add up to the synchronous averages."""
    nx, nz = 64, 32
    rho = W.noise_field(nx, nz, 3, mean=0.7, amp=0.2, n_species=2)
    a = L.Lattice(nx, nz, 2, L.LBM_FP64, L.LBM_PERIODIC, **W.EMULSION_PARAMS)
    b = L.Lattice(nx, nz, 2, L.LBM_FP64, L.LBM_PERIODIC, **W.EMULSION_PARAMS)
    for lat in (a, b):
        lat.set_fields(rho)
        lat.set_observe(1)
    r = a.reader(depth=2)
    got = []
    pending = None
    for k in range(8):
        a.step(1)
        t = r.enqueue(averages="completed", reset=True)
        if pending is not None:
            got.append(r.result(pending))
        pending = t
    got.append(r.result(pending))
    last = r.result(r.enqueue(averages=True, reset=True))  # flushes the final pending sample
    b.step(8)
    want = b.averages()
    assert [g["samples"] for g in got] == [0] + [1] * 7 and last["samples"] == 1
    total = sum(g["mass"] * g["samples"] for g in got) + last["mass"]
    assert np.allclose(total / 8, want["mass"], rtol=1e-14, atol=0)
    ux = sum(np.asarray(g["ux_z"]) * g["samples"] for g in got) + np.asarray(last["ux_z"])
    assert np.allclose(ux / 8, want["ux_z"], rtol=1e-12, atol=1e-18)


def test_wait_rejects_unknown_tickets():
    lat = L.Lattice(32, 16, 1, L.LBM_FP64, L.LBM_PERIODIC, **W.SINGLE_PARAMS)
    lat.set_fields(W.noise_field(32, 16, 1))
    assert L.load().lbm_wait(lat.h, 5) == L.LBM_EINVAL
    r = lat.reader()
    t = r.enqueue()
    assert r.result(t)["samples"] == 1


@pytest.mark.parametrize("precision", [L.LBM_FP32, L.LBM_FP64])
def test_step_read_series_equals_step_by_step_reads(precision):
    """lbm_step_read: runs of steps with every step's completed sums read back by one call give
    the records of separate lbm_step + lbm_observables_enqueue calls, bit for bit."""
    nx, nz = 96, 40
    rho, _ = W.disk_packing(nx, nz, 0.6, 7, r_mean=5, r_spread=1)
    a = L.Lattice(nx, nz, 2, precision, L.LBM_PERIODIC, **W.EMULSION_PARAMS)
    b = L.Lattice(nx, nz, 2, precision, L.LBM_PERIODIC, **W.EMULSION_PARAMS)
    for lat in (a, b):
        lat.set_fields(rho)
        lat.set_observe(1)
    series = a.series(chunk=20, depth=2)
    got, pending = [], None
    for n in (20, 7, 0, 20):
        t = series.run(n)
        if pending is not None:
            got += series.results(pending)
        pending = t
    got += series.results(pending)
    r = b.reader(depth=2)
    want = []
    for _ in range(47):
        b.step(1)
        want.append(r.result(r.enqueue(averages="completed", reset=True)))
    assert len(got) == 47
    for g, w in zip(got, want):
        same(g, w)
    assert got[-1]["step"] == 47 and got[-1]["samples"] == 1
    rc = L.load().lbm_step_read(a.h, 1, series.bufs[0].data_ptr(), series.rec - 8, 2, 1, None)
    assert rc == L.LBM_EINVAL and a.observables()["step"] == 47  # nothing enqueued
    with pytest.raises(ValueError):
        series.run(21)
