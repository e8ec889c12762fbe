"""Pins of the step-size adaptation oracle (oracle/adapt.py; dual averaging
of Hoffman & Gelman 2014, Sec. 3.2.1, as the paper's warm-up uses it,
Sec. 3.1) against facts that do not restate its recursion:

* a constant acceptance probability alpha has the closed form
  Hbar_m = m (delta - alpha) / (m + t0) (multiply the recursion by m + t0:
  (m + t0) Hbar_m grows by delta - alpha per step), so
  log eps_m = mu - sqrt(m) m (delta - alpha) / (gamma (m + t0));
* alpha = delta on every step keeps eps at 10 eps0 (the shrinkage point);
* too-high acceptance grows the step size, too-low shrinks it;
* on a noiseless acceptance curve alpha(eps) = exp(-(eps / s)^2) the
  averaged step size converges to the root s sqrt(-ln delta);
* HMC on a 50-dimensional Gaussian (scales 1 to 3), adapted toward 0.8,
  then run with the final step size, accepts at a mean rate near 0.8.
"""
import math

import numpy as np
import pytest

from oracle import adapt as A
from oracle import hmc


@pytest.mark.parametrize("alpha", [0.0, 0.3, 0.8, 1.0])
def test_constant_alpha_closed_form(alpha):
    eps0, delta, M = 0.01, 0.8, 40
    da = A.DualAveraging(eps0, delta, M)
    mu = math.log(10.0 * eps0)
    for m in range(1, M):
        eps = da.update(alpha)
        ref = mu - math.sqrt(m) * m * (delta - alpha) / (A.GAMMA * (m + A.T0))
        assert abs(math.log(eps) - ref) <= 1e-12 * max(1.0, abs(ref)), (m, math.log(eps), ref)


def test_on_target_keeps_shrinkage_point():
    for eps0 in (1e-3, 0.05, 2.0):
        da = A.DualAveraging(eps0, 0.65, 30)
        for _ in range(30):
            eps = da.update(0.65)
            assert abs(eps - 10.0 * eps0) <= 1e-13 * eps0
        assert da.update(0.0) == eps                       # frozen after n_adapt


def test_direction_of_the_update():
    up = A.DualAveraging(0.01, 0.8, 20)
    down = A.DualAveraging(0.01, 0.8, 20)
    e_up = [up.update(1.0) for _ in range(19)]
    e_dn = [down.update(0.0) for _ in range(19)]
    assert all(b > a for a, b in zip(e_up, e_up[1:]))
    assert all(b < a for a, b in zip(e_dn, e_dn[1:]))


@pytest.mark.parametrize("delta,s", [(0.8, 0.3), (0.574, 2.0), (0.65, 0.01)])
def test_converges_to_the_root_of_a_noiseless_curve(delta, s):
    M = 4000
    da = A.DualAveraging(s / 7.0, delta, M)
    eps = da.eps
    for _ in range(M):
        eps = da.update(math.exp(-(eps / s) ** 2))
    root = s * math.sqrt(-math.log(delta))
    assert abs(eps / root - 1.0) < 0.02, (eps, root)


def test_hmc_on_a_gaussian_reaches_the_target():
    # scales 1 .. 3 m: an isotropic Gaussian with a fixed trajectory length
    # has resonant step sizes where the acceptance is not monotone in eps
    rng = np.random.default_rng(11)
    d, n_leap, M, N = 50, 8, 600, 1000
    sig = np.linspace(1.0, 3.0, d)
    grad = lambda q: -q / sig ** 2
    logp = lambda q: -0.5 * float((q / sig) @ (q / sig))
    q = sig * rng.standard_normal(d)
    da = A.DualAveraging(1.0, 0.8, M)
    alphas = []
    for k in range(M + N):
        p0 = rng.standard_normal(d)
        q1, p1 = hmc.leapfrog(q, p0, da.eps, n_leap, grad)
        delta = logp(q1) - logp(q) + 0.5 * float(p0 @ p0) - 0.5 * float(p1 @ p1)
        a = A.accept_prob(delta)
        if rng.random() < a:
            q = q1
        if k < M:
            da.update(a)
        else:
            alphas.append(a)
    assert abs(np.mean(alphas) - 0.8) < 0.06, np.mean(alphas)


def test_accept_prob():
    assert A.accept_prob(0.3) == 1.0
    assert A.accept_prob(-math.log(2.0)) == pytest.approx(0.5, rel=1e-15)
    assert A.accept_prob(-1.0, in_support=False) == 0.0
    assert A.accept_prob(float("nan")) == 0.0
