"""The library's per-site arithmetic (lbm_core.cuh, and the two-species FP32 forms of
lbm_pair.cuh), compiled for the host, against the oracle.

Checks the force of Eq. FORCE, the cross repulsion, the Appendix A shell stresses and the cross
stress at every site of small random lattices, for both weight presets.  No GPU needed.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def core(tmp_path_factory):
    out = tmp_path_factory.mktemp("core") / "libcorehost.so"
    src = os.path.join(ROOT, "tests", "native", "core_host.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1402_6019_gb300", "csrc"), src, "-o", str(out)],
                   check=True)
    lib = ctypes.CDLL(str(out))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.core_site.argtypes = [ctypes.POINTER(L.lbm_params), ctypes.c_int, dp, dp, dp, dp, dp]
    lib.core_psi.argtypes = [ctypes.POINTER(L.lbm_params), ctypes.c_int, ctypes.c_double]
    lib.core_psi.restype = ctypes.c_double
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lib_params(**kw):
    p = L.lbm_params()
    p.tau[0] = p.tau[1] = 1.0
    p.rho0[0] = p.rho0[1] = 1.0
    p.weight_norm = 1.0 / 3.0
    for k, v in kw.items():
        if k in ("tau", "G1", "G2", "rho0", "wall_u"):
            v = list(v) if hasattr(v, "__len__") else [v, v]
            getattr(p, k)[0] = v[0]
            getattr(p, k)[1] = v[-1]
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("preset", [0, 1])
@pytest.mark.parametrize("ns", [1, 2])
def test_site_force_and_stress_match_oracle(oracle, core, preset, ns):
    nx, nz = 11, 9
    rng = np.random.default_rng(7 + preset + 10 * ns)
    rho = 0.1 + 1.2 * rng.random((ns, nz, nx))
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, weight_preset=preset)
    ref = oracle.RefLattice(nx, nz, ns, 0, **prm)
    ref.set_fields(rho)
    sf = ref.site_fields()
    rho_o = ref.fields()[0]
    lp = _lib_params(**prm)
    psi = sf["psi"]
    for z in range(nz):
        for x in range(nx):
            p25 = np.zeros(ns * 25)
            for s in range(ns):
                for dz in range(-2, 3):
                    for dx in range(-2, 3):
                        p25[s * 25 + (dz + 2) * 5 + dx + 2] = psi[s, (z + dz) % nz, (x + dx) % nx]
            r9 = np.zeros(18)
            for s in range(ns):
                for dz in range(-1, 2):
                    for dx in range(-1, 2):
                        r9[s * 9 + (dz + 1) * 3 + dx + 1] = rho_o[s, (z + dz) % nz, (x + dx) % nx]
            F = np.zeros(2 * ns)
            si = np.zeros(3 * ns)
            sc = np.zeros(3)
            core.core_site(ctypes.byref(lp), ns, _p(p25), _p(r9), _p(F), _p(si), _p(sc))
            want_F = sf["F"][:, :, z, x].reshape(-1)
            assert np.allclose(F, want_F, rtol=0, atol=1e-13), (z, x, F, want_F)
            assert np.allclose(si, sf["sint"][:, :, z, x].reshape(-1), rtol=0, atol=1e-13)
            # cross stress: the oracle's total pressure tensor minus every other term
            kin = 0.25
            rest = np.zeros(3)
            for s in range(ns):
                r, fx, fz = rho_o[s, z, x], sf["F"][s, 0, z, x], sf["F"][s, 1, z, x]
                rest += np.array([r / 3 + kin * fx * fx / r, r / 3 + kin * fz * fz / r, kin * fx * fz / r])
                rest += sf["sint"][s, :, z, x]
            assert np.allclose(sc, sf["P"][:, z, x] - rest, rtol=0, atol=1e-13)


def test_psi_matches_oracle(oracle, core):
    prm = dict(W.EMULSION_PARAMS)
    lp = _lib_params(**prm)
    ref = oracle.RefLattice(4, 1, 2, 0, **prm)
    rho = np.array([[[0.05, 0.3, 1.2, 2.5]], [[1.1, 0.2, 0.05, 0.7]]])
    ref.set_fields(rho)
    psi = ref.site_fields()["psi"]
    for s in range(2):
        for i in range(4):
            assert core.core_psi(ctypes.byref(lp), s, rho[s, 0, i]) == pytest.approx(psi[s, 0, i], rel=1e-15)


@pytest.fixture(scope="module")
def pair(tmp_path_factory):
    out = tmp_path_factory.mktemp("pair") / "libpairhost.so"
    src = os.path.join(ROOT, "tests", "native", "pair_host.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1402_6019_gb300", "csrc"), src, "-o", str(out)],
                   check=True)
    lib = ctypes.CDLL(str(out))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.pair_site.argtypes = [ctypes.POINTER(L.lbm_params), dp, dp, dp, dp, dp, dp, dp]
    lib.pair_collide.argtypes = [ctypes.POINTER(L.lbm_params), dp, dp, dp, dp]
    return lib


@pytest.mark.parametrize("preset", [0, 1])
def test_pair_fp32_site_arithmetic_matches_oracle(oracle, pair, preset):
    """The FP32 two-species forms the step kernel runs (intra_force2, force_stress2, cross_force2,
    cross_stress2, psi2) at every site of a random 11 x 9 lattice.  Forces and stresses here are
    at most 0.3 in size and each is a sum of about 30 terms of at most that size, so FP32 rounding
    (unit 2^-24) bounds their error by 30 * 0.3 * 2^-24 < 1e-6; a dropped term of the outermost
    shell (|c|^2 = 8) alone would be about 1e-3."""
    nx, nz = 11, 9
    rng = np.random.default_rng(70 + preset)
    rho = 0.1 + 1.2 * rng.random((2, nz, nx))
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, weight_preset=preset)
    ref = oracle.RefLattice(nx, nz, 2, 0, **prm)
    ref.set_fields(rho)
    sf = ref.site_fields()
    rho_o = ref.fields()[0]
    psi = sf["psi"]
    lp = _lib_params(**prm)
    kin = 0.25  # (tau - 1/2)^2 at tau = 1
    for z in range(nz):
        for x in range(nx):
            p25 = np.array([psi[s, (z + dz) % nz, (x + dx) % nx]
                            for s in range(2) for dz in range(-2, 3) for dx in range(-2, 3)])
            r9 = np.array([rho_o[s, (z + dz) % nz, (x + dx) % nx]
                           for s in range(2) for dz in range(-1, 2) for dx in range(-1, 2)])
            F, F2, si, sc, ps = np.zeros(4), np.zeros(4), np.zeros(6), np.zeros(3), np.zeros(2)
            pair.pair_site(ctypes.byref(lp), _p(p25), _p(r9), _p(F), _p(F2), _p(si), _p(sc), _p(ps))
            want_F = sf["F"][:, :, z, x].reshape(-1)
            assert np.abs(want_F).max() < 0.3
            assert np.allclose(F, want_F, rtol=0, atol=1e-6), (z, x, F, want_F)
            assert np.allclose(F2, want_F, rtol=0, atol=1e-6), (z, x, F2, want_F)
            assert np.allclose(si, sf["sint"][:, :, z, x].reshape(-1), rtol=0, atol=1e-6), (z, x)
            rest = np.zeros(3)
            for s in range(2):
                r, fx, fz = rho_o[s, z, x], sf["F"][s, 0, z, x], sf["F"][s, 1, z, x]
                rest += np.array([r / 3 + kin * fx * fx / r, r / 3 + kin * fz * fz / r, kin * fx * fz / r])
                rest += sf["sint"][s, :, z, x]
            assert np.allclose(sc, sf["P"][:, z, x] - rest, rtol=0, atol=1e-6), (z, x)
            assert np.allclose(ps, psi[:, z, x], rtol=1e-6, atol=0), (z, x)


def test_pair_fp32_collision_matches_oracle(oracle, pair):
    """collide2, the two-species FP32 collision of the default kernel (deviation storage, shifted
    common velocity, unequal tau), against the oracle's post-collision populations, read off one
    periodic oracle step as f*_l(x) = f_l(x + c_l, t + 1).  Populations off equilibrium by 10 %.
    Populations here are below 0.6 and each is formed from about 20 terms of that size, so FP32
    rounding bounds the error by 20 * 0.6 * 2^-24 < 1e-6 (observed 5e-8); dropping the u_z^2 term
    of the equilibrium shows up at 2e-2."""
    cx, cz = [0, 1, 0, -1, 0, 1, -1, -1, 1], [0, 0, 1, 0, -1, 1, 1, -1, -1]
    nx, nz = 9, 7
    rng = np.random.default_rng(5)
    rho = 0.2 + rng.random((2, nz, nx))
    prm = dict(W.EMULSION_PARAMS, G_AB=0.587, tau=(0.8, 1.3))
    ref = oracle.RefLattice(nx, nz, 2, 0, **prm)
    ref.set_fields(rho)
    f0 = ref.fields()[2] * (1 + 0.1 * rng.standard_normal((2, 9, nz, nx)))
    ref.set_populations(f0)
    F = ref.site_fields()["F"]
    ref.step(1)
    f1 = ref.fields()[2]
    post = np.empty_like(f1)
    for l in range(9):
        post[:, l] = np.roll(np.roll(f1[:, l], -cz[l], axis=1), -cx[l], axis=2)
    assert np.abs(post).max() < 0.6
    rr = np.array([f0[0].sum(axis=0).mean(), f0[1].sum(axis=0).mean()])
    lp = _lib_params(**prm)
    for z in range(nz):
        for x in range(nx):
            out = np.zeros(18)
            pair.pair_collide(ctypes.byref(lp), _p(rr), _p(np.ascontiguousarray(f0[:, :, z, x]).reshape(-1)),
                              _p(np.ascontiguousarray(F[:, :, z, x]).reshape(-1)), _p(out))
            assert np.allclose(out, post[:, :, z, x].reshape(-1), rtol=0, atol=1e-6), (z, x)
