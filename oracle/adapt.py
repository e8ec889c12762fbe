"""FP64 CPU oracle of the step-size adaptation of the gradient samplers
(test infrastructure; only ``tests/`` and ``bench.py``'s CPU legs may import
it).

Sec. 3.1: the paper's sampler tunes its step size during warm-up so that
the mean acceptance probability approaches a target (0.8), together with a
diagonal preconditioner.  The scheme is
dual averaging (Hoffman & Gelman, "The No-U-Turn Sampler", JMLR 15 (2014),
Sec. 3.2.1), with its recommended constants gamma = 0.05, t0 = 10,
kappa = 0.75 and shrinkage point mu = log(10 eps0).  Per adapted step m = 1,
2, ... with acceptance probability alpha_m of that step's proposal:

  Hbar_m       = (1 - 1/(m + t0)) Hbar_{m-1} + (delta - alpha_m) / (m + t0)
  log eps_m    = mu - sqrt(m) / gamma * Hbar_m
  log epsbar_m = m^(-kappa) log eps_m + (1 - m^(-kappa)) log epsbar_{m-1}

starting from Hbar_0 = 0 and log epsbar_0 = 0.  Step m + 1 runs with eps_m;
once the M adapted steps are over, the sampler keeps epsbar_M.  Each chain
adapts on its own.

The diagonal preconditioner (inverse metric) follows the windowed warm-up of
the NUTS implementations the paper's sampler comes from: of W adapted steps,
an initial buffer of 75, slow windows of 25, 50, 100, ... steps and a
terminal buffer of 50 (15 % / 75 % / 10 % of W when those do not fit), the
last slow window stretched to the terminal buffer when the next one would
cross it.  Over a slow window each coordinate's post-step values give a
sample variance (Welford); at its end the inverse metric becomes
(n/(n+5)) var + s 5/(n+5) (n the window length, s the shrinkage target) and
the dual averaging starts over with mu = log(10 eps), Hbar = 0,
log epsbar = 0.

Parity pins (tests/test_oracle_adapt.py): the closed form of a constant
acceptance, the fixed point at the target, convergence to the root of a
noiseless acceptance curve, the window schedule, Welford against the sample
variance, the metric leapfrog as the unit one in rescaled coordinates, and
warm-ups that reach the target and recover a Gaussian's scales.  Every
function is pinned.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA, T0, KAPPA = 0.05, 10.0, 0.75


class DualAveraging:
    """One chain's adaptation state.  ``eps`` is the step size of the next
    step; ``update(alpha)`` records an adapted step's acceptance probability."""

    def __init__(self, eps0: float, target: float, n_adapt: int):
        self.target, self.n_adapt = float(target), int(n_adapt)
        self.mu = math.log(10.0 * eps0)
        self.hbar = 0.0
        self.log_bar = 0.0
        self.m = 0
        self.eps = float(eps0)

    def update(self, alpha: float) -> float:
        if self.m >= self.n_adapt:
            return self.eps
        self.m += 1
        m = float(self.m)
        self.hbar = (1.0 - 1.0 / (m + T0)) * self.hbar + (self.target - alpha) / (m + T0)
        log_eps = self.mu - math.sqrt(m) / GAMMA * self.hbar
        eta = m ** (-KAPPA)
        self.log_bar = eta * log_eps + (1.0 - eta) * self.log_bar
        self.eps = math.exp(log_eps if self.m < self.n_adapt else self.log_bar)
        return self.eps


def accept_prob(delta: float, in_support: bool = True) -> float:
    """min(1, e^delta), 0 for a proposal outside the prior's support."""
    if not in_support or math.isnan(delta):
        return 0.0
    return 1.0 if delta >= 0.0 else math.exp(delta)


def buffers(W: int):
    """(initial buffer, first slow window, terminal buffer) for W steps."""
    init, base, term = 75, 25, 50
    if init + base + term > W:
        init, term = int(0.15 * W), int(0.1 * W)
        base = W - (init + term)
    return init, base, term


def windows(W: int):
    """The slow windows [start, end) of W adapted steps."""
    init, base, term = buffers(W)
    stop, out = W - term, []
    start, size = init, base
    if base < 1:
        return out
    while start < stop:
        end = start + size
        if end + 2 * size > stop:
            end = stop
        out.append((start, end))
        start, size = end, 2 * size
    return out


class Welford:
    """Running mean and sum of squared deviations (Welford's update)."""

    def __init__(self, shape):
        self.n, self.mean, self.m2 = 0, np.zeros(shape), np.zeros(shape)

    def add(self, x):
        x = np.asarray(x, np.float64)
        self.n += 1
        d = x - self.mean
        self.mean = self.mean + d / self.n
        self.m2 = self.m2 + d * (x - self.mean)

    def variance(self):
        return self.m2 / (self.n - 1) if self.n > 1 else np.zeros_like(self.m2)


def regularized(var, n: int, shrink: float):
    """(n/(n+5)) var + shrink 5/(n+5)."""
    return (n / (n + 5.0)) * np.asarray(var, np.float64) + shrink * (5.0 / (n + 5.0))


class Warmup:
    """One chain's step size and diagonal inverse metric through W adapted
    steps.  ``update(alpha, state)`` records a step's acceptance probability
    and the chain's state after it; ``eps`` / ``inv_metric`` are what the next
    step uses."""

    def __init__(self, eps0: float, target: float, W: int, shape, shrink: float = 1e-3):
        self.da = DualAveraging(eps0, target, W)
        self.W, self.shrink, self.t = int(W), float(shrink), 0
        self.wins = windows(W)
        self.inv_metric = np.ones(shape)
        self.acc = Welford(shape)

    @property
    def eps(self):
        return self.da.eps

    def update(self, alpha: float, state):
        if self.t >= self.W:
            return self.eps
        t = self.t
        win = next(((a, b) for a, b in self.wins if a <= t < b), None)
        if win is not None:
            self.acc.add(state)
            if t == win[1] - 1:
                self.inv_metric = regularized(self.acc.variance(), self.acc.n, self.shrink)
                self.acc = Welford(np.shape(self.inv_metric))
        # dual averaging over the steps since its last start
        da = self.da
        da.m += 1
        m = float(da.m)
        da.hbar = (1.0 - 1.0 / (m + T0)) * da.hbar + (da.target - alpha) / (m + T0)
        log_eps = da.mu - math.sqrt(m) / GAMMA * da.hbar
        eta = m ** (-KAPPA)
        da.log_bar = eta * log_eps + (1.0 - eta) * da.log_bar
        da.eps = math.exp(log_eps if t + 1 < self.W else da.log_bar)
        if win is not None and t == win[1] - 1:
            da.mu, da.hbar, da.log_bar, da.m = math.log(10.0 * da.eps), 0.0, 0.0, 0
        self.t += 1
        return self.eps
