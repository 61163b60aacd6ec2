"""The library's discrete adjoint (lbm_adjoint_step / _objective / _initial and the checkpointed
run of paper_1402_6019_gb300.adjoint) against the oracle's adjoint, on the same seeded states.

Tolerances: one adjoint step is a fixed expression of FP64 values of order one with at most a
few hundred terms per output, summed in another order than the oracle's, so lam agrees to
1e-12 of its largest entry; the parameter derivatives sum n sites, so they get 1e-12 of n times
the largest |lam| besides a relative 1e-10.  A run also carries the forward's rounding (the pull
kernel and the oracle differ by ~1e-16 per step), amplified by the steps: 1e-9 relative."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import lbm as L
from paper_1402_6019_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    (2, dict(W.EMULSION_PARAMS, G_AB=0.587, body_force=2e-5, tau=(0.9, 1.3)), 37, 29),
    (1, dict(W.SINGLE_PARAMS, tau=(0.8, 0.8), body_force=1e-5), 40, 33),
    (2, dict(W.EMULSION_PARAMS, psi_form=1, rho0=(1.0, 1.0), tau=(1.1, 0.7)), 19, 23),
    (2, dict(W.EMULSION_PARAMS, weight_preset=1, G1=(-5.0, -4.5), G2=(0.0, 0.0), body_force=1e-5), 33, 17),
]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def state(oracle, nx, nz, ns, prm, seed, steps=3):
    """An out-of-equilibrium state made by the oracle (a few steps from noisy rho and u)."""
    rho = W.noise_field(nx, nz, seed=seed, mean=0.7, amp=0.3, n_species=ns)
    u = 0.02 * W.noise_field(nx, nz, seed=seed + 1, mean=0.0, amp=1.0, n_species=2)
    ref = oracle.RefLattice(nx, nz, ns, 0, **prm)
    ref.set_fields(rho, u)
    ref.step(steps)
    return ref, ref.fields()[2]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_adjoint_step_matches_oracle(oracle, case):
    ns, prm, nx, nz = CASES[case]
    ref, f = state(oracle, nx, nz, ns, prm, seed=40 + case)
    lam_next = np.random.default_rng(case).standard_normal(f.shape)
    lam_ref, grad_ref = ref.adjoint_step(lam_next)

    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    lam = torch.empty_like(dev(f))
    grad = torch.zeros(8, dtype=torch.float64, device="cuda")
    L.lbm_adjoint_step(lat.h, dev(f), dev(lam_next), lam, grad)
    lat.synchronize()
    lam, grad = lam.cpu().numpy(), grad.cpu().numpy()
    scale = np.abs(lam_ref).max()
    assert np.abs(lam - lam_ref).max() <= 1e-12 * scale, np.abs(lam - lam_ref).max() / scale
    atol = 1e-12 * nx * nz * np.abs(lam_next).max()
    for k in range(8):
        assert abs(grad[k] - grad_ref[k]) <= 1e-10 * abs(grad_ref[k]) + atol, (k, grad[k], grad_ref[k])
    if ns == 1:  # species B and the cross coupling do not exist
        assert grad[1] == grad[3] == grad[4] == grad[6] == 0.0
    # grad is accumulated into, not overwritten
    g2 = torch.from_numpy(grad).cuda()
    L.lbm_adjoint_step(lat.h, dev(f), dev(lam_next), torch.empty_like(dev(f)), g2)
    lat.synchronize()
    assert np.allclose(g2.cpu().numpy(), 2 * grad, rtol=1e-13, atol=0)


@pytest.mark.parametrize("ns", [1, 2])
def test_objective_matches_oracle(oracle, ns):
    nx, nz = 45, 21
    prm = CASES[0][1] if ns == 2 else CASES[1][1]
    _, f = state(oracle, nx, nz, ns, prm, seed=60 + ns)
    rng = np.random.default_rng(7)
    tu, tr = 1e-3 * rng.standard_normal(nz), 0.7 + 0.1 * rng.standard_normal(nz)
    J_ref, g_ref = oracle.profile_objective(f, tu, tr)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    J = torch.zeros((), dtype=torch.float64, device="cuda")
    g = torch.empty_like(dev(f))
    L.lbm_adjoint_objective(lat.h, dev(f), dev(tu), dev(tr), J, g)
    lat.synchronize()
    assert abs(float(J) - J_ref) <= 1e-12 * J_ref
    g = g.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
    # without dJ/df only J is written
    J2 = torch.full((), 5.0, dtype=torch.float64, device="cuda")
    L.lbm_adjoint_objective(lat.h, dev(f), dev(tu), dev(tr), J2, None)
    lat.synchronize()
    assert float(J2) == float(J)


def test_initial_density_gradient(oracle):
    nx, nz, ns = 17, 13, 2
    lam0 = np.random.default_rng(3).standard_normal((ns, 9, nz, nx))
    wq = oracle.tables()[2]
    want = np.einsum("l,slzx->szx", wq, lam0)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **CASES[0][1])
    g = torch.empty((ns, nz, nx), dtype=torch.float64, device="cuda")
    L.lbm_adjoint_initial(lat.h, dev(lam0), g)
    lat.synchronize()
    assert np.abs(g.cpu().numpy() - want).max() <= 1e-15 * np.abs(want).max() * 9


def rollout_case(ns):
    nx, nz, steps = 24, 20, 7
    prm = CASES[0][1] if ns == 2 else CASES[1][1]
    rho = W.noise_field(nx, nz, seed=90, mean=0.7, amp=0.2, n_species=ns)
    rng = np.random.default_rng(11)
    tu, tr = 1e-4 * rng.standard_normal(nz), 0.7 + 0.05 * rng.standard_normal(nz)
    return nx, nz, steps, prm, rho, tu, tr


@pytest.mark.parametrize("ns", [1, 2])
def test_rollout_gradient_matches_oracle(oracle, ns):
    from paper_1402_6019_gb300 import adjoint as A

    nx, nz, steps, prm, rho, tu, tr = rollout_case(ns)
    J_ref, g_ref, grad_ref = oracle.rollout_gradient(nx, nz, ns, rho, steps, tu, tr, **prm)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    results = []
    for ck in (3, 1, 7, 50):  # ragged segments, one step each, one segment, longer than the run
        J, g, grad = A.rollout_gradient(lat, dev(rho), steps, dev(tu), dev(tr), checkpoint=ck)
        results.append((J, g.cpu().numpy(), grad.cpu().numpy()))
    J, g, grad = results[0]
    assert abs(J - J_ref) <= 1e-12 * J_ref
    assert np.abs(g - g_ref).max() <= 1e-9 * np.abs(g_ref).max()
    for k in range(8):
        assert abs(grad[k] - grad_ref[k]) <= 1e-9 * max(abs(grad_ref[k]), 1e-300) + 1e-14, (k, grad[k], grad_ref[k])
    # the recomputed forward is bit-identical and the sums run in a fixed order, so the
    # checkpoint spacing changes nothing
    for J2, g2, grad2 in results[1:]:
        assert J2 == J and np.array_equal(g2, g) and np.array_equal(grad2, grad)


def test_set_populations_restores_the_state_exactly(oracle):
    nx, nz, ns = 29, 26, 2
    prm = CASES[0][1]
    _, f = state(oracle, nx, nz, ns, prm, seed=70)
    for precision in (L.LBM_FP64, L.LBM_FP32):
        lat = L.Lattice(nx, nz, ns, precision, L.LBM_PERIODIC, **prm)
        lat.set_fields(f.sum(axis=1))  # reference densities of the FP32 deviations
        lat.set_populations(f)
        g = lat.fields()[2]
        if precision == L.LBM_FP64:
            assert np.array_equal(g, f)
        else:
            assert np.abs(g - f).max() <= 1e-7 * np.abs(f).max()
        lat.step(4)
        a = lat.fields()[2]
        lat.set_populations(dev(g))  # from a device tensor this time
        lat.step(4)
        b = lat.fields()[2]
        if precision == L.LBM_FP64:
            # exported and imported unchanged, so the restored run repeats bit for bit ...
            assert np.array_equal(b, a)
            # ... and steps like the oracle's
            r = oracle.RefLattice(nx, nz, ns, 0, **prm)
            r.set_populations(f)
            r.step(4)
            assert np.abs(a - r.fields()[2]).max() <= 1e-12 * np.abs(f).max()
        else:
            # a deviation far below W_l rho_ref may come back one FP32 unit off
            assert np.abs(b - a).max() <= 1e-6 * np.abs(a).max()


def test_profile_loss_autograd(oracle):
    from paper_1402_6019_gb300 import adjoint as A

    ns = 2
    nx, nz, steps, prm, rho, tu, tr = rollout_case(ns)
    J_ref, g_ref, grad_ref = oracle.rollout_gradient(nx, nz, ns, rho, steps, tu, tr, **prm)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    rho_t = dev(rho).requires_grad_(True)
    theta = torch.tensor(A.theta_of(lat.params), dtype=torch.float64, requires_grad=True)
    J = A.ProfileLoss.apply(lat, rho_t, theta, dev(tu), dev(tr), steps, 3)
    (3.0 * J).backward()
    assert abs(float(J.detach()) - J_ref) <= 1e-12 * J_ref
    assert np.abs(rho_t.grad.cpu().numpy() - 3 * g_ref).max() <= 3e-9 * np.abs(g_ref).max()
    gt = theta.grad.numpy()
    for k in range(8):
        assert abs(gt[k] - 3 * grad_ref[k]) <= 3e-9 * abs(grad_ref[k]) + 1e-13, (k, gt[k], grad_ref[k])


def test_adjoint_rejects_what_it_does_not_cover():
    nx, nz = 16, 12
    f = torch.ones((1, 9, nz, nx), dtype=torch.float64, device="cuda")
    lam = torch.empty_like(f)
    grad = torch.zeros(8, dtype=torch.float64, device="cuda")
    walls = L.Lattice(nx, nz, 1, L.LBM_FP64, L.LBM_BOUNCEBACK, **W.SINGLE_PARAMS)
    with pytest.raises(L.LbmError) as e:
        L.lbm_adjoint_step(walls.h, f, f, lam, grad)
    assert e.value.code == L.LBM_EINVAL
    batch = L.Lattice(nx, None, 1, L.LBM_FP64, L.LBM_BOUNCEBACK, instances=[6, 6], **W.SINGLE_PARAMS)
    with pytest.raises(L.LbmError):
        L.lbm_adjoint_step(batch.h, f, f, lam, grad)
    lat = L.Lattice(nx, nz, 1, L.LBM_FP64, L.LBM_PERIODIC, **W.SINGLE_PARAMS)
    with pytest.raises(L.LbmError):  # lam may not alias lam_next
        L.lbm_adjoint_step(lat.h, f, lam, lam, grad)
    fp32 = L.Lattice(nx, nz, 1, L.LBM_FP32, L.LBM_PERIODIC, **W.SINGLE_PARAMS)
    with pytest.raises(L.LbmError):  # FP32 deviations need a reference density
        fp32.set_populations(np.ones((1, 9, nz, nx)))
