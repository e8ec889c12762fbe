"""FP64 CPU oracle of the step-size adaptation of the gradient samplers
(test infrastructure; only ``tests/`` and ``bench.py``'s CPU legs may import
it).

Sec. 3.1: the paper's sampler tunes its step size during warm-up so that
the mean acceptance probability approaches a target (0.8).  The scheme is
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
"""
from __future__ import annotations

import math

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
