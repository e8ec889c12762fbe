"""Pins of the capped-NUTS oracle (oracle/nuts.py; Sec. 3.1, NUTS of
Hoffman & Gelman 2014 run to its trajectory cap):

* depth 1 is HMC with one leapfrog step and the Metropolis accept
  min(1, e^(H_0 - H_1)) (biased progressive sampling of a one-state subtree);
* the multinomial choice inside a subtree is uniform over its states when
  their energies are equal (a Gaussian with tiny steps makes them equal to
  ~1e-12; the choice frequencies match 1/4 for the last subtree of depth 3);
* the transition leaves a Gaussian invariant: the sample mean and variance
  of a long run match the target's;
* every state of the 2^D - 1 steps is visited: the trajectory's two ends sit
  at the right leapfrog distances;
* a diagonal inverse metric is the unit metric in rescaled coordinates.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import hmc
from oracle import nuts as NU


def gaussian(s):
    s = np.asarray(s, np.float64)
    logpi = lambda q: (-0.5 * float(np.sum((q / s) ** 2)), 0.0)
    grad = lambda q: -q / s ** 2
    return logpi, grad


def test_depth_one_is_hmc_with_one_step():
    s = np.array([0.5, 1.0, 2.0, 4.0])
    logpi, grad = gaussian(s)
    rng = np.random.default_rng(1)
    moved = 0
    for k in range(200):
        q0 = s * rng.standard_normal(4)
        ll0, lp0 = logpi(q0)
        q, ll, lp, g, stat, _ = NU.iteration(logpi, grad, q0, ll0, lp0, grad(q0), 0.9, 1, 7, 3, k,
                                             state=np.float64)
        # the same leapfrog step by hand, direction from the depth-0 uniform
        v = -1 if NU.uniform(7, 3, k, 0) < 0.5 else 1
        xi = oracle.normals(7, NU.STREAM_NUTS_P, 3, k, 4)
        q1, p1 = hmc.leapfrog(q0, xi, v * 0.9, 1, grad)
        dH = (logpi(q1)[0] - 0.5 * float(p1 @ p1)) - (ll0 - 0.5 * float(xi @ xi))
        a = min(1.0, math.exp(dH))
        assert stat == pytest.approx(a, rel=1e-12, abs=1e-15)
        take = math.log(NU.uniform(7, 3, k, 32)) < dH
        np.testing.assert_allclose(q, q1 if take else q0, rtol=1e-14, atol=0)
        moved += take
    assert 0 < moved < 200


def test_subtree_choice_is_uniform_for_equal_energies():
    """Steps of 1e-6 on N(0, 1): all states of a depth-3 trajectory have
    energies equal to ~1e-12.  With equal weights every merge takes the new
    subtree (W_sub - W = 0 at each depth: 1 vs 1, 2 vs 2, 4 vs 4 states), so
    the chosen state is one of the last subtree's 4, each with probability
    1/4 (the multinomial choice inside a subtree)."""
    logpi, grad = gaussian([1.0])
    counts = np.zeros(4)
    for k in range(4000):
        q0 = np.array([0.3])
        q, *_ = NU.iteration(logpi, grad, q0, logpi(q0)[0], 0.0, grad(q0), 1e-6, 3, 11, 0, k,
                             state=np.float64)
        # position along the trajectory in units of the step, from the end
        # where the last subtree started
        xi = oracle.normals(11, NU.STREAM_NUTS_P, 0, k, 1)[0]
        dirs = [(-1 if NU.uniform(11, 0, k, j) < 0.5 else 1) for j in range(3)]
        n_side = {d: sum(2 ** j for j in range(2) if dirs[j] == d) for d in (-1, 1)}
        d2 = dirs[2]
        start = n_side[d2]                      # steps already taken on that side
        steps = (q[0] - q0[0]) / (1e-6 * xi) * d2   # signed multiple of the step along d2
        idx = int(round(steps)) - start - 1
        assert 0 <= idx < 4, (k, steps, start)
        counts[idx] += 1
    np.testing.assert_allclose(counts / counts.sum(), 0.25, atol=0.03)


def test_gaussian_is_invariant():
    s = np.array([0.3, 1.0, 3.0])
    logpi, grad = gaussian(s)
    rng = np.random.default_rng(2)
    q = s * rng.standard_normal(3)
    draws = []
    for k in range(6000):
        ll, lp = logpi(q)
        q, ll, lp, g, stat, _ = NU.iteration(logpi, grad, q, ll, lp, grad(q), 0.25, 4, 5, 1, k,
                                             state=np.float64)
        draws.append(q)
    d = np.array(draws[500:])
    np.testing.assert_allclose(d.mean(0) / s, 0.0, atol=0.12)
    np.testing.assert_allclose(d.std(0) / s, 1.0, atol=0.1)


def test_trajectory_extent():
    """With a flat direction sequence the ends sit 2^D - 1 steps apart: on
    N(0, 1) with a tiny step the chosen state is one of the trajectory's
    states, at a multiple of the step from the start within [-(2^D-1),
    2^D - 1]."""
    logpi, grad = gaussian([1.0])
    D = 4
    for k in range(300):
        q0 = np.array([0.1])
        q, *_ = NU.iteration(logpi, grad, q0, logpi(q0)[0], 0.0, grad(q0), 1e-7, D, 2, 0, k,
                             state=np.float64)
        xi = oracle.normals(2, NU.STREAM_NUTS_P, 0, k, 1)[0]
        n = (q[0] - q0[0]) / (1e-7 * xi)
        assert abs(n - round(n)) < 1e-3 and abs(round(n)) <= 2 ** D - 1


def test_metric_is_the_unit_metric_in_scaled_coordinates():
    """N(0, diag s^2) with inverse metric s^2 is, in x = q / s with momentum
    s p, N(0, I) with the unit metric: the same momenta and uniforms give the
    same trajectory, so the chosen state maps across (x = q / s), and the
    acceptance statistic and the decision margins are equal."""
    rng = np.random.default_rng(8)
    s = np.exp(rng.uniform(-3.0, 2.0, 12))
    logpi_q, grad_q = gaussian(s)
    logpi_x, grad_x = gaussian(np.ones(12))
    for k in range(40):
        q0 = s * rng.standard_normal(12)
        a = NU.iteration(logpi_q, grad_q, q0, logpi_q(q0)[0], 0.0, grad_q(q0), 0.3, 4, 9, 2, k,
                         state=np.float64, inv_metric=s ** 2)
        x0 = q0 / s
        b = NU.iteration(logpi_x, grad_x, x0, logpi_x(x0)[0], 0.0, grad_x(x0), 0.3, 4, 9, 2, k,
                         state=np.float64)
        np.testing.assert_allclose(a[0] / s, b[0], rtol=1e-10, atol=1e-12)
        assert a[4] == pytest.approx(b[4], rel=1e-10, abs=1e-14)
        assert a[5] == pytest.approx(b[5], rel=1e-8, abs=1e-10)
