"""The library's discrete adjoint (lbm_adjoint_step / _steps / _objective / _initial, state
recording and snapshots, and the checkpointed runs of paper_1402_6019_gb300.adjoint) against
the oracle's adjoint on the same seeded states, and against central finite differences of the
library's own forward run on the calibration workload.

FP64 tolerances: one adjoint step is a fixed expression of FP64 values of order one with at most
a few hundred terms per output, summed in another order than the oracle's, so lam agrees to
1e-12 of its largest entry; the parameter derivatives sum n sites, so they get 1e-12 of n times
the largest |lam| besides a relative 1e-10.  A run also carries the forward's rounding (the pull
kernel and the oracle differ by ~1e-16 per step), amplified by the steps: 1e-9 relative.
FP32: the same sums rounded at 2^-24 ~ 6e-8 per operation, with coefficients up to |G| w ~ 3:
5e-5 of the largest entry for one step; 1e-4 relative for a run's gradients (the bar of the
finite-difference check)."""
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


def dev(a, dtype=np.float64):
    """A device copy of a host array (synchronous)."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()
    torch.cuda.synchronize()
    return t


def zeros(*shape, dtype=torch.float64):
    t = torch.zeros(shape, dtype=dtype, device="cuda")
    torch.cuda.synchronize()  # the library runs on its own stream
    return t


def state(oracle, nx, nz, ns, prm, seed, steps=3):
    """An out-of-equilibrium state made by the oracle (a few steps from noisy rho and u)."""
    rho = W.noise_field(nx, nz, seed=seed, mean=0.7, amp=0.3, n_species=ns)
    u = 0.02 * W.noise_field(nx, nz, seed=seed + 1, mean=0.0, amp=1.0, n_species=2)
    ref = oracle.RefLattice(nx, nz, ns, 0, **prm)
    ref.set_fields(rho, u)
    ref.step(steps)
    return ref, ref.fields()[2]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("fp32", [False, True])
def test_adjoint_step_matches_oracle(oracle, case, fp32):
    ns, prm, nx, nz = CASES[case]
    ref, f = state(oracle, nx, nz, ns, prm, seed=40 + case)
    lam_next = np.random.default_rng(case).standard_normal(f.shape)
    lam_ref, grad_ref = ref.adjoint_step(lam_next)

    dt = np.float32 if fp32 else np.float64
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    lam = torch.empty_like(dev(f, dt))
    grad = zeros(8)
    L.lbm_adjoint_step(lat.h, dev(f, dt), dev(lam_next, dt), lam, grad)
    lat.synchronize()
    lam, grad = lam.cpu().numpy().astype(np.float64), grad.cpu().numpy()
    scale = np.abs(lam_ref).max()
    tol, rtol, atol = (5e-5, 1e-4, 1e-6) if fp32 else (1e-12, 1e-10, 1e-12)
    assert np.abs(lam - lam_ref).max() <= tol * scale, np.abs(lam - lam_ref).max() / scale
    atol *= nx * nz * np.abs(lam_next).max()
    for k in range(8):
        assert abs(grad[k] - grad_ref[k]) <= rtol * abs(grad_ref[k]) + atol, (k, grad[k], grad_ref[k])
    if ns == 1:  # species B and the cross coupling do not exist
        assert grad[1] == grad[3] == grad[4] == grad[6] == 0.0
    # grad is accumulated into, not overwritten
    g2 = dev(grad)
    L.lbm_adjoint_step(lat.h, dev(f, dt), dev(lam_next, dt), torch.empty_like(dev(f, dt)), g2)
    lat.synchronize()
    assert np.allclose(g2.cpu().numpy(), 2 * grad, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_adjoint_steps_sweep_equals_single_steps(oracle, dt):
    """lbm_adjoint_steps over recorded states = lbm_adjoint_step applied state by state."""
    ns, prm, nx, nz = CASES[0]
    _, f = state(oracle, nx, nz, ns, prm, seed=44)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    lat.set_populations(f)
    n = 5
    tdt = torch.float32 if dt == np.float32 else torch.float64
    states = torch.empty((n, ns, 9, nz, nx), dtype=tdt, device="cuda")
    L.lbm_record_states(lat.h, n, states)
    lat.synchronize()
    # the recorded states are the states the steps pass through
    lat.set_populations(f)
    for k in range(n):
        want = lat.fields()[2]
        assert np.array_equal(states[k].cpu().numpy(), want.astype(dt))
        lat.step(1)
    lam0 = np.random.default_rng(9).standard_normal(f.shape)
    lam = dev(lam0, dt)
    grad = zeros(8)
    L.lbm_adjoint_steps(lat.h, n, states, lam, grad)
    one, g1 = dev(lam0, dt), zeros(8)
    for k in reversed(range(n)):
        out = torch.empty_like(one)
        L.lbm_adjoint_step(lat.h, states[k], one, out, g1)
        one = out
    lat.synchronize()
    assert torch.equal(lam, one)
    assert np.allclose(grad.cpu().numpy(), g1.cpu().numpy(), rtol=1e-12 if dt == np.float64 else 1e-6, atol=0)
    # zero steps: nothing changes
    before = lam.clone()
    torch.cuda.synchronize()
    L.lbm_adjoint_steps(lat.h, 0, states, lam, grad)
    lat.synchronize()
    assert torch.equal(lam, before)


@pytest.mark.parametrize("precision", [L.LBM_FP64, L.LBM_FP32])
def test_snapshot_restores_exactly(oracle, precision):
    ns, prm, nx, nz = CASES[0]
    rho = W.noise_field(nx, nz, seed=71, mean=0.7, amp=0.3, n_species=ns)
    lat = L.Lattice(nx, nz, ns, precision, L.LBM_PERIODIC, **prm)
    lat.set_fields(rho)
    lat.step(3)
    snap = torch.empty(L.lbm_snapshot_bytes(lat.h), dtype=torch.uint8, device="cuda")
    L.lbm_snapshot(lat.h, snap)
    lat.step(6)
    a, step_a = lat.fields()[2], lat.observables()["step"]
    lat.set_fields(rho * 1.01)  # a different state (and, in FP32, other reference densities)
    L.lbm_restore(lat.h, snap)
    assert lat.observables()["step"] == 3
    lat.step(6)
    assert np.array_equal(lat.fields()[2], a) and lat.observables()["step"] == step_a


@pytest.mark.parametrize("precision", [L.LBM_FP64, L.LBM_FP32])
def test_restore_after_the_snapshot_buffer_was_reused(precision):
    """A snapshot buffer that another snapshot overwrote at the same address (as when a freed
    buffer's memory is handed to a new one): lbm_restore gives the new snapshot's state, step
    counter and reference densities; lbm_restore_own, which trusts the context's record of what
    it wrote there, reports the overwrite at the next synchronisation instead of going on."""
    ns, prm, nx, nz = CASES[0]
    rho = W.noise_field(nx, nz, seed=72, mean=0.7, amp=0.3, n_species=ns)
    a = L.Lattice(nx, nz, ns, precision, L.LBM_PERIODIC, **prm)
    b = L.Lattice(nx, nz, ns, precision, L.LBM_PERIODIC, **prm)
    a.set_fields(rho)
    b.set_fields(rho * 1.2)  # FP32: other reference densities
    a.step(4)
    b.step(9)
    snap = torch.empty(L.lbm_snapshot_bytes(a.h), dtype=torch.uint8, device="cuda")
    L.lbm_snapshot(a.h, snap)
    a.synchronize()
    L.lbm_snapshot(b.h, snap)  # same address, another context's snapshot
    b.synchronize()
    want = b.fields()[2]
    L.lbm_restore(a.h, snap)
    assert a.observables()["step"] == 9
    assert np.array_equal(a.fields()[2], want)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.fields()[2], b.fields()[2])
    # the record-trusting form notices that the tail is not the one this context wrote
    L.lbm_snapshot(a.h, snap)
    a.synchronize()
    L.lbm_snapshot(b.h, snap)
    b.synchronize()
    L.lbm_restore_own(a.h, snap)
    with pytest.raises(L.LbmError) as e:
        a.synchronize()
    assert e.value.code == L.LBM_EINVAL
    # an untouched snapshot of its own restores asynchronously and exactly
    a.set_fields(rho)
    a.step(2)
    L.lbm_snapshot(a.h, snap)
    f2 = a.fields()[2]
    a.step(5)
    L.lbm_restore_own(a.h, snap)
    a.synchronize()
    assert np.array_equal(a.fields()[2], f2) and a.observables()["step"] == 2
    # memory that holds no snapshot of this shape is refused
    junk = torch.zeros_like(snap)
    with pytest.raises(L.LbmError) as e:
        L.lbm_restore(a.h, junk)
    assert e.value.code == L.LBM_EINVAL


@pytest.mark.parametrize("ns", [1, 2])
def test_objective_matches_oracle(oracle, ns):
    nx, nz = 45, 21
    prm = CASES[0][1] if ns == 2 else CASES[1][1]
    _, f = state(oracle, nx, nz, ns, prm, seed=60 + ns)
    rng = np.random.default_rng(7)
    tu, tr = 1e-3 * rng.standard_normal(nz), 0.7 + 0.1 * rng.standard_normal(nz)
    J_ref, g_ref = oracle.profile_objective(f, tu, tr)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **prm)
    for dt, tol in ((np.float64, 1e-12), (np.float32, 1e-5)):
        J = zeros()
        g = torch.empty_like(dev(f, dt))
        L.lbm_adjoint_objective(lat.h, dev(f, dt), dev(tu), dev(tr), J, g)
        lat.synchronize()
        assert abs(float(J) - J_ref) <= tol * J_ref
        g = g.cpu().numpy().astype(np.float64)
        assert np.abs(g - g_ref).max() <= tol * np.abs(g_ref).max()
        # without dJ/df only J is written
        J2 = dev(5.0)
        L.lbm_adjoint_objective(lat.h, dev(f, dt), dev(tu), dev(tr), J2, None)
        lat.synchronize()
        assert float(J2) == float(J)


def test_initial_density_gradient(oracle):
    nx, nz, ns = 17, 13, 2
    lam0 = np.random.default_rng(3).standard_normal((ns, 9, nz, nx))
    wq = oracle.tables()[2]
    want = np.einsum("l,slzx->szx", wq, lam0)
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **CASES[0][1])
    for dt, tol in ((np.float64, 1e-15), (np.float32, 1e-7)):
        g = torch.empty((ns, nz, nx), dtype=torch.float64, device="cuda")
        L.lbm_adjoint_initial(lat.h, dev(lam0, dt), g)
        lat.synchronize()
        assert np.abs(g.cpu().numpy() - want).max() <= tol * np.abs(want).max() * 9


def rollout_case(ns):
    nx, nz, steps = 24, 20, 7
    prm = CASES[0][1] if ns == 2 else CASES[1][1]
    rho = W.noise_field(nx, nz, seed=90, mean=0.7, amp=0.2, n_species=ns)
    rng = np.random.default_rng(11)
    tu, tr = 1e-4 * rng.standard_normal(nz), 0.7 + 0.05 * rng.standard_normal(nz)
    return nx, nz, steps, prm, rho, tu, tr


@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("precision", [L.LBM_FP64, L.LBM_FP32])
def test_rollout_gradient_matches_oracle(oracle, ns, precision):
    from paper_1402_6019_gb300 import adjoint as A

    nx, nz, steps, prm, rho, tu, tr = rollout_case(ns)
    J_ref, g_ref, grad_ref = oracle.rollout_gradient(nx, nz, ns, rho, steps, tu, tr, **prm)
    lat = L.Lattice(nx, nz, ns, precision, L.LBM_PERIODIC, **prm)
    results = []
    for ck in (3, 1, 7, 50):  # ragged segments, one step each, one segment, longer than the run
        J, g, grad = A.rollout_gradient(lat, dev(rho), steps, dev(tu), dev(tr), checkpoint=ck)
        results.append((J, g.cpu().numpy(), grad.cpu().numpy()))
    J, g, grad = results[0]
    tj, tg = (1e-12, 1e-9) if precision == L.LBM_FP64 else (1e-5, 1e-4)
    assert abs(J - J_ref) <= tj * J_ref
    assert np.abs(g - g_ref).max() <= tg * np.abs(g_ref).max()
    gmax = np.abs(grad_ref).max()
    for k in range(8):
        assert abs(grad[k] - grad_ref[k]) <= tg * abs(grad_ref[k]) + 1e-12 * gmax, (k, grad[k], grad_ref[k])
    # the recomputed forward is bit-identical, so the checkpoint spacing changes neither J nor
    # lam; the parameter derivatives are summed per segment, so their rounding may differ
    for J2, g2, grad2 in results[1:]:
        assert J2 == J and np.array_equal(g2, g)
        assert np.abs(grad2 - grad).max() <= 1e-13 * np.abs(grad).max()


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
    f = dev(np.ones((1, 9, nz, nx)))
    lam = torch.empty_like(f)
    grad = zeros(8)
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
    with pytest.raises(TypeError):  # mixed precisions
        L.lbm_adjoint_step(lat.h, f, f.float(), lam, grad)


def test_calibration_workload_gradients_match_finite_differences():
    """The 256 x 256 calibration run (500 steps, snapshots every 25): the adjoint gradient for
    G2 A, G_AB, tau A and a direction in the initial densities against central differences of
    the library's FP64 forward run, h = 1e-4 (relative for the parameters); the FP32 forward +
    FP32 adjoint against the same differences.  Bar: 1e-4 relative."""
    from paper_1402_6019_gb300 import adjoint as A

    w = W.workload("adjoint_256")
    nx, nz, ns, steps = w["nx"], w["nz"], w["n_species"], w["steps"]
    rho, tu, tr = dev(w["rho"]), dev(w["target_u"]), dev(w["target_rho"])
    lat = L.Lattice(nx, nz, ns, L.LBM_FP64, L.LBM_PERIODIC, **w["params"])
    lat32 = L.Lattice(nx, nz, ns, L.LBM_FP32, L.LBM_PERIODIC, **w["params"])
    J, g, grad = A.rollout_gradient(lat, rho, steps, tu, tr, checkpoint=w["checkpoint"])
    J32, g32, grad32 = A.rollout_gradient(lat32, rho, steps, tu, tr, checkpoint=w["checkpoint"])
    assert abs(J32 - J) <= 1e-5 * J
    theta = A.theta_of(lat.params)

    def J_at(th, r=rho):
        A.set_theta(lat, th)
        return A.objective_value(lat, r, steps, tu, tr)

    for k in (2, 4, 5):  # G2 A, G_AB, tau A
        h = 1e-4 * abs(theta[k])
        tp, tm = list(theta), list(theta)
        tp[k] += h
        tm[k] -= h
        fd = (J_at(tp) - J_at(tm)) / (2 * h)
        assert abs(float(grad[k]) - fd) <= 1e-4 * abs(fd), (k, float(grad[k]), fd)
        assert abs(float(grad32[k]) - fd) <= 1e-4 * abs(fd), (k, float(grad32[k]), fd)
    A.set_theta(lat, theta)
    v = dev(np.random.default_rng(5).standard_normal((ns, nz, nx)))
    h = 1e-4
    fd = (J_at(theta, rho + h * v) - J_at(theta, rho - h * v)) / (2 * h)
    for gg in (g, g32):
        ad = float((gg * v).sum())
        assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)
