"""Pins of the HMC oracle (oracle/hmc.py): reversibility of the leapfrog map,
second-order energy error on a Gaussian target, one leapfrog step equal to a
Langevin (MALA) proposal with the same noise, and an exact return after one
period of a harmonic oscillator (the leapfrog map is then a rotation)."""
import numpy as np

import oracle
from oracle import hmc
from paper_2603_28907_gb300 import workloads as W


def quad_grad(A):
    return lambda x: -(A @ x.reshape(-1)).reshape(x.shape)


def spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return B @ B.T / n + np.eye(n)


def test_leapfrog_is_reversible():
    A = spd(12, 1)
    g = quad_grad(A)
    rng = np.random.default_rng(2)
    q0, p0 = rng.standard_normal(12), rng.standard_normal(12)
    q1, p1 = hmc.leapfrog(q0, p0, 0.1, 25, g)
    q2, p2 = hmc.leapfrog(q1, -p1, 0.1, 25, g)
    np.testing.assert_allclose(q2, q0, atol=1e-12)
    np.testing.assert_allclose(-p2, p0, atol=1e-12)


def test_energy_error_is_second_order():
    A = spd(8, 3)
    g = quad_grad(A)
    rng = np.random.default_rng(4)
    q0, p0 = rng.standard_normal(8), rng.standard_normal(8)
    energy = lambda q, p: 0.5 * q @ A @ q + 0.5 * p @ p
    errs = []
    for eps in (0.04, 0.02, 0.01):
        q, p = hmc.leapfrog(q0, p0, eps, int(round(0.8 / eps)), g)
        errs.append(abs(energy(q, p) - energy(q0, p0)))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_one_step_is_a_langevin_proposal():
    w = W.small(R=4, Q=5, n_zenith=3, n_azimuth=5, G=12)
    op = oracle.OracleProblem(W.problem(w))
    H = W.init_chains(w, 1)[0]
    counts = np.full((w.S, w.P), 500, np.int32)
    op = op.with_counts(counts)
    eps = 0.01
    q, dk = hmc.propose(op, H, eps, 1, 5, 0, 3, state=np.float64)
    p0 = hmc.momentum(5, 0, 3, H.shape)
    g = op.grad_loglik(H) + op.grad_logprior(H)
    np.testing.assert_allclose(q, H + 0.5 * eps * eps * g + eps * p0, rtol=0, atol=1e-12)


def test_full_period_rotation_returns():
    # 1-D harmonic oscillator, pi ~ N(0, 1): leapfrog with eps = 2 sin(theta/2)
    # is a rotation in the modified phase space; exact return after a period
    eps, n = 2.0 * np.sin(np.pi / 40), 40
    g = lambda x: -x
    q, p = hmc.leapfrog(np.array([1.3]), np.array([0.0]), eps, n, g)
    assert abs(q[0] - 1.3) < 1e-12
