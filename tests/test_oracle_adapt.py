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


# ---------------------------------------------------------------- diagonal metric
def test_windows_of_the_default_schedule():
    # 1000 warm-up steps: initial buffer 75, slow windows 25, 50, 100, 200 and
    # a last one stretched to the terminal buffer of 50 (500 steps)
    assert A.windows(1000) == [(75, 100), (100, 150), (150, 250), (250, 450), (450, 950)]
    # too short for 75 + 25 + 50: 15 % / 75 % / 10 %
    assert A.buffers(100) == (15, 75, 10) and A.windows(100) == [(15, 90)]
    assert A.windows(40) == [(6, 36)]
    for W in (20, 37, 150, 151, 333, 8192):
        ws = A.windows(W)
        init, base, term = A.buffers(W)
        assert ws[0][0] == init and ws[-1][1] == W - term
        assert all(a[1] == b[0] for a, b in zip(ws, ws[1:]))          # contiguous
        lens = [b - a for a, b in ws]
        nominal = [base * 2 ** i for i in range(len(ws))]             # doubling windows,
        assert lens[:-1] == nominal[:-1]                               # the last stretched
        assert nominal[-1] <= lens[-1] < 3 * nominal[-1]              # by less than 2x its size


def test_welford_is_the_sample_variance():
    rng = np.random.default_rng(3)
    x = rng.normal(2.0, 0.3, size=(57, 4, 5))
    w = A.Welford((4, 5))
    for row in x:
        w.add(row)
    np.testing.assert_allclose(w.mean, x.mean(0), rtol=1e-13)
    np.testing.assert_allclose(w.variance(), x.var(0, ddof=1), rtol=1e-12)
    assert A.regularized(1.0, 10**9, 7.0) == pytest.approx(1.0, rel=1e-7)
    assert A.regularized(0.0, 5, 1e-3) == pytest.approx(5e-4)


def test_metric_leapfrog_is_the_unit_leapfrog_in_scaled_coordinates():
    """N(0, diag s^2) with inverse metric s^2: with x = q / s and momentum
    s p the leapfrog is the unit-metric leapfrog on N(0, I)."""
    rng = np.random.default_rng(5)
    s = np.exp(rng.uniform(-4.0, 3.0, 30))
    q0, p0 = s * rng.standard_normal(30), rng.standard_normal(30) / s
    q, p = hmc.leapfrog(q0, p0, 0.37, 9, lambda q: -q / s ** 2, inv_metric=s ** 2)
    x, px = hmc.leapfrog(q0 / s, p0 * s, 0.37, 9, lambda x: -x)
    np.testing.assert_allclose(q, s * x, rtol=1e-12, atol=0)
    np.testing.assert_allclose(p, px / s, rtol=1e-12, atol=0)


def test_warmup_recovers_the_scales_of_an_anisotropic_gaussian():
    """HMC through 1000 warm-up steps on N(0, diag s^2), s from 0.01 to 10:
    the adapted inverse metric estimates s^2, and the sampler then accepts
    near the 0.8 target."""
    rng = np.random.default_rng(17)
    d, n_leap, W, N = 20, 8, 1000, 600
    s = np.logspace(-2, 1, d)
    grad = lambda q: -q / s ** 2
    logp = lambda q: -0.5 * float(np.sum((q / s) ** 2))
    q = s * rng.standard_normal(d)
    wu = A.Warmup(0.01, 0.8, W, (d,), shrink=1e-8)
    alphas = []
    for k in range(W + N):
        m = wu.inv_metric
        xi = rng.standard_normal(d)
        q1, p1 = hmc.leapfrog(q, xi / np.sqrt(m), wu.eps, n_leap, grad, inv_metric=m)
        delta = logp(q1) - logp(q) + 0.5 * float(xi @ xi) - 0.5 * float(np.sum(m * p1 * p1))
        a = A.accept_prob(delta)
        if rng.random() < a:
            q = q1
        if k < W:
            wu.update(a, q)
        else:
            alphas.append(a)
    ratio = wu.inv_metric / s ** 2
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio
    assert abs(np.median(ratio) - 1.0) < 0.25, ratio
    assert abs(np.mean(alphas) - 0.8) < 0.08, np.mean(alphas)


def test_warmup_restarts_the_step_size_at_window_ends():
    W = 40
    wu = A.Warmup(0.01, 0.8, W, (3,), shrink=0.0)
    (a, b), = A.windows(W)
    for t in range(W):
        eps = wu.update(0.3, np.array([t, 2.0 * t, 0.0]))
        if t == b - 1:
            assert wu.da.mu == pytest.approx(math.log(10.0 * eps)) and wu.da.m == 0
            n = b - a
            var = np.var(np.arange(a, b, dtype=float), ddof=1)
            np.testing.assert_allclose(wu.inv_metric, [n / (n + 5) * var, n / (n + 5) * 4 * var, 0.0])
    assert wu.t == W and wu.update(0.9, np.zeros(3)) == eps                # frozen after W
