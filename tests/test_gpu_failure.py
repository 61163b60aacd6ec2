"""Failure detection on the GPU without a fault: the bounded device-side wait of the step
kernels expires on a barrier that nothing completes, the expiry is reported as LBM_ETIMEOUT,
and the context keeps working."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_stays_usable():
    lat = L.Lattice(64, 48, 2, L.LBM_FP32, 0, **W.EMULSION_PARAMS)
    rho, _ = W.disk_packing(64, 48, 0.6, seed=3, r_mean=6, r_spread=1)
    lat.set_fields(rho)
    lat.step(3)
    before = lat.fields()[2]
    assert L.lbm_selftest_wait(lat.h, 2_000_000) == L.LBM_ETIMEOUT  # about 1 ms of SM clock
    assert b"expired" in L.load().lbm_last_error(lat.h)
    lat.synchronize()  # the self-test clears its flag: no error is left behind
    assert np.array_equal(lat.fields()[2], before)
    lat.step(5)
    lat.synchronize()
    o = lat.observables()
    assert np.allclose(o["mass"], rho.sum(axis=(1, 2)), rtol=1e-5)


def test_selftest_rejects_bad_arguments():
    lat = L.Lattice(8, 8, 1, L.LBM_FP64, 0)
    assert L.lbm_selftest_wait(lat.h, 0) == L.LBM_EINVAL
