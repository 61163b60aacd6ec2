"""Pins of the oracle's discrete adjoint: every derivative it returns is checked against central
finite differences of the oracle's own forward step (an independent code path), for the
populations, every parameter, the calibration objective and a whole run."""
import numpy as np
import pytest

from paper_1402_6019_gb300 import workloads as W

PARAMS = [dict(W.EMULSION_PARAMS, G_AB=0.587, body_force=2e-5, tau=(0.9, 1.3)),
          dict(W.SINGLE_PARAMS, tau=(0.8, 0.8), body_force=1e-5),
          dict(W.EMULSION_PARAMS, psi_form=1, rho0=(1.0, 1.0), tau=(1.1, 0.7))]
KEYS = ["G1", "G1", "G2", "G2", "G_AB", "tau", "tau", "body_force"]
IDX = [0, 1, 0, 1, None, 0, 1, None]


def state(oracle, nx, nz, ns, prm, seed, steps=3):
    rho = W.noise_field(nx, nz, seed=seed, mean=0.7, amp=0.3, n_species=ns)
    u = 0.02 * W.noise_field(nx, nz, seed=seed + 1, mean=0.0, amp=1.0, n_species=2)
    ref = oracle.RefLattice(nx, nz, ns, 0, **prm)
    ref.set_fields(rho, u)
    ref.step(steps)  # an out-of-equilibrium state
    return ref, ref.fields()[2]


def step_of(oracle, nx, nz, ns, prm, f):
    r = oracle.RefLattice(nx, nz, ns, 0, **prm)
    r.set_populations(f)
    r.step(1)
    return r.fields()[2]


def fd_step(prm, k):
    """Central-difference step for parameter k: relative to the coupling or relaxation time; an
    absolute 1e-6 for the body force, whose values (~1e-5) are too small to scale a step by."""
    if KEYS[k] == "body_force":
        return 1e-6
    base = prm.get(KEYS[k], 0.0)
    return 1e-6 * (abs(base[IDX[k]] if IDX[k] is not None else base) or 1.0)


def with_param(prm, k, h):
    q = dict(prm)
    key, i = KEYS[k], IDX[k]
    if i is None:
        q[key] = q.get(key, 0.0) + h
    else:
        v = list(q[key]) if isinstance(q[key], (tuple, list)) else [q[key], q[key]]
        v[i] += h
        q[key] = tuple(v)
    return q


@pytest.mark.parametrize("case", [0, 1, 2])
def test_one_step_vjp_matches_finite_differences(oracle, case):
    prm = PARAMS[case]
    ns = 1 if case == 1 else 2
    nx, nz = 11, 9
    ref, f = state(oracle, nx, nz, ns, prm, seed=10 + case)
    rng = np.random.default_rng(case)
    lam_next = rng.standard_normal(f.shape)
    v = rng.standard_normal(f.shape)
    lam, grad = ref.adjoint_step(lam_next)
    h = 1e-6
    fd = (np.sum(lam_next * step_of(oracle, nx, nz, ns, prm, f + h * v))
          - np.sum(lam_next * step_of(oracle, nx, nz, ns, prm, f - h * v))) / (2 * h)
    assert abs(np.sum(lam * v) - fd) <= 1e-7 * abs(fd), (np.sum(lam * v), fd)
    # every parameter: d/dtheta of lam_next . S(f; theta)
    for k in range(8):
        if ns == 1 and IDX[k] == 1 or ns == 1 and KEYS[k] == "G_AB":
            continue
        hk = fd_step(prm, k)
        fp = np.sum(lam_next * step_of(oracle, nx, nz, ns, with_param(prm, k, hk), f))
        fm = np.sum(lam_next * step_of(oracle, nx, nz, ns, with_param(prm, k, -hk), f))
        fd = (fp - fm) / (2 * hk)
        assert abs(grad[k] - fd) <= 1e-6 * max(abs(fd), 1e-3), (k, grad[k], fd)


def test_adjoint_needs_a_periodic_lattice(oracle):
    ref = oracle.RefLattice(6, 5, 1, 1, **W.SINGLE_PARAMS)
    ref.set_fields(np.ones((1, 5, 6)))
    lam = np.zeros((1, 9, 5, 6))
    with pytest.raises(AssertionError):
        ref.adjoint_step(lam)


def test_objective_gradient(oracle):
    _, f = state(oracle, 10, 7, 2, PARAMS[0], seed=3)
    rng = np.random.default_rng(7)
    tu, tr = 0.01 * rng.standard_normal(7), 0.5 + 0.1 * rng.standard_normal(7)
    J, g = oracle.profile_objective(f, tu, tr)
    v = rng.standard_normal(f.shape)
    h = 1e-6
    fd = (oracle.profile_objective(f + h * v, tu, tr)[0] - oracle.profile_objective(f - h * v, tu, tr)[0]) / (2 * h)
    assert abs(np.sum(g * v) - fd) <= 1e-7 * abs(fd)
    assert J > 0


def test_run_gradient_matches_finite_differences(oracle):
    """J after 6 steps from rest: d/d rho_init (directional) and d/d every parameter."""
    nx, nz, ns, steps = 12, 10, 2, 6
    prm = PARAMS[0]
    rho0 = W.noise_field(nx, nz, seed=21, mean=0.7, amp=0.3, n_species=ns)
    rng = np.random.default_rng(3)
    tu, tr = 0.002 * rng.standard_normal(nz), 0.7 + 0.05 * rng.standard_normal(nz)
    J, g_rho, grad = oracle.rollout_gradient(nx, nz, ns, rho0, steps, tu, tr, **prm)

    def run(rho, p):
        ref = oracle.RefLattice(nx, nz, ns, 0, **p)
        ref.set_fields(rho)
        ref.step(steps)
        return oracle.profile_objective(ref.fields()[2], tu, tr)[0]

    v = rng.standard_normal(rho0.shape)
    h = 1e-6
    fd = (run(rho0 + h * v, prm) - run(rho0 - h * v, prm)) / (2 * h)
    assert abs(np.sum(g_rho * v) - fd) <= 1e-6 * abs(fd), (np.sum(g_rho * v), fd)
    for k in range(8):
        hk = fd_step(prm, k)
        fd = (run(rho0, with_param(prm, k, hk)) - run(rho0, with_param(prm, k, -hk))) / (2 * hk)
        assert abs(grad[k] - fd) <= 1e-5 * max(abs(fd), 1e-4 * abs(J)), (k, grad[k], fd)
