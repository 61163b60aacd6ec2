"""lbm_observables_noalloc: observables for callers that cannot let the library allocate.

Callers recording into a CUDA graph, real-time loops and applications whose own memory pool
holds the whole device cannot have a library call cudaMalloc underneath them.  This entry point
computes the same observables as lbm_observables using only a fixed scratch array inside the
library.  The test checks it against lbm_observables on the same state, within the FP64
observables tolerance of the other tests, on two calls in a row (the second call must not see
what the first left in the shared scratch).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11  # FP64 observables, as in test_gpu_parity.check_obs


def _layout(buf, nx, nz, ns):
    prof = buf[16:]
    return dict(mass=buf[0:2], momentum=buf[2:4], gamma=buf[4], wall_force=buf[5:7], nonfinite=buf[7] != 0,
                ux_z=prof[0:nz], rho_z=prof[nz:(1 + ns) * nz].reshape(ns, nz), sxz_z=prof[3 * nz:4 * nz],
                fluid_z=prof[4 * nz:5 * nz], ps_x=prof[5 * nz:5 * nz + nx], pxx_x=prof[5 * nz + nx:5 * nz + 2 * nx])


def _close(a, b, scale):
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= TOL * max(scale, 1e-300)


@pytest.mark.parametrize("zbc", [0, 1])
def test_noalloc_matches_lbm_observables_twice(zbc):
    torch = pytest.importorskip("torch")
    nx, nz, ns = 96, 70, 2
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, wall_u=(-0.01, 0.01) if zbc else (0.0, 0.0), body_force=1e-5)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, zbc, **prm)
    rho, _ = W.disk_packing(nx, nz, 0.7, seed=31 + zbc, r_mean=7, r_spread=2, periodic_z=(zbc == 0))
    lat.set_fields(rho)
    out = torch.zeros(16 + 9 * nz + 2 * nx, dtype=torch.float64, device="cuda")
    f = torch.zeros((ns, 9, nz, nx), dtype=torch.float64, device="cuda")
    for call in range(2):
        lat.step(7 + call)
        want = lat.observables()
        L.lbm_get_fields(lat.h, f=f)
        out.fill_(float("nan"))  # every entry the call owns must be written
        rc = L.lbm_observables_noalloc(f.data_ptr(), nx, nz, ns, zbc, lat.params, out.data_ptr(), None)
        torch.cuda.synchronize()
        assert rc == L.LBM_OK
        got = _layout(out.cpu().numpy(), nx, nz, ns)
        m = np.abs(want["mass"]).max()
        assert _close(got["mass"], want["mass"], m)
        assert _close(got["momentum"], want["momentum"], m)
        for k in ("ux_z", "sxz_z", "fluid_z", "ps_x", "pxx_x", "rho_z"):
            assert _close(got[k], want[k], np.abs(want[k]).max()), (call, k)
        assert abs(got["gamma"] - want["gamma"]) <= TOL * np.abs(want["ps_x"]).sum() + 1e-14 * np.abs(
            want["pxx_x"]).sum()
        assert _close(got["wall_force"], want["wall_force"], max(np.abs(want["wall_force"]).max(), 1e-12))
        assert not got["nonfinite"]


def test_noalloc_rejects_what_does_not_fit():
    torch = pytest.importorskip("torch")
    p = L.make_params(**W.SINGLE_PARAMS)
    f = torch.zeros(9, dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 4096 x 4096 needs about 67 MB of scratch, far beyond the fixed array
    assert L.lbm_observables_noalloc(f.data_ptr(), 4096, 4096, 1, 0, p, out.data_ptr(), None) == L.LBM_ENOMEM
    assert L.lbm_observables_noalloc(0, 8, 8, 1, 0, p, out.data_ptr(), None) == L.LBM_EINVAL
    assert L.lbm_observables_noalloc(f.data_ptr(), 0, 8, 1, 0, p, out.data_ptr(), None) == L.LBM_EINVAL
