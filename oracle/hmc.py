"""FP64 CPU oracle of the Hamiltonian Monte Carlo step (test infrastructure;
only ``tests/`` and ``bench.py``'s CPU legs may import it).

Sec. 3.1 (gradient-based samplers; the paper runs NUTS, whose building block
is this leapfrog trajectory), unit mass matrix, Neal's leapfrog integrator:
  p0 ~ N(0, I)        (Philox stream HMC = 6, counter {pair j, step, chain},
                       Box-Muller with both outputs, like every other stream)
  p  = p0 + eps/2 g(q0)
  repeat n_leap times:  q = q + eps p ;  p = p + eps g(q)  (half a kick, eps/2,
                        after the last drift instead of a full one)
  accept iff ln u < log pi(q) - log pi(q0) + |p0|^2/2 - |p|^2/2.
States are stored in a fixed precision (FP32 heights in the FP32 modes), so
the log-density and its gradient are evaluated at the stored, rounded
position; the trajectory itself is carried in FP64.  ``state`` gives that
rounding (np.float32 or np.float64).

Parity pins (tests/test_oracle_hmc.py): reversibility, second-order energy
error, the one-step trajectory as a Langevin proposal, and a full period of
the harmonic oscillator.  Every function is pinned.
"""
from __future__ import annotations

import numpy as np

import oracle

STREAM_HMC = 6


def leapfrog(q0, p0, eps, n_leap, grad, state=np.float64, inv_metric=None):
    """(q, p) after n_leap leapfrog steps; grad(x) is evaluated at x rounded
    to `state`.  With a diagonal inverse metric m (mass matrix diag(1/m)) each
    drift moves q by eps * m * p.  Returns the rounded final position and the
    final momentum."""
    m = 1.0 if inv_metric is None else np.asarray(inv_metric, np.float64)
    q = np.asarray(q0, np.float64).copy()
    p = np.asarray(p0, np.float64) + 0.5 * eps * grad(np.asarray(q, state).astype(np.float64))
    for i in range(n_leap):
        q = q + eps * (m * p)
        g = grad(np.asarray(q, state).astype(np.float64))
        p = p + (eps if i < n_leap - 1 else 0.5 * eps) * g
    return np.asarray(q, state).astype(np.float64), p


def momentum(seed, chain, step, shape):
    n = int(np.prod(shape))
    return oracle.normals(seed, STREAM_HMC, chain, step, n).reshape(shape)


def propose(op, H, eps, n_leap, seed, chain, step, state=np.float32, inv_metric=None):
    """One HMC proposal of chain `chain` at step `step` from heights H for the
    oracle problem `op` (log pi = loglik + logprior).  Returns (q', K0 - K1)
    with K(p) = p^T M^-1 p / 2.  With a diagonal inverse metric m the momentum
    is p0 = xi / sqrt(m) for the standard normals xi, so K(p0) = |xi|^2 / 2."""
    grad = lambda x: op.grad_loglik(x) + op.grad_logprior(x)
    xi = momentum(seed, chain, step, np.shape(H))
    if inv_metric is None:
        p0, m = xi, 1.0
    else:
        m = np.asarray(inv_metric, np.float64)
        p0 = xi / np.sqrt(m)
    q, p = leapfrog(H, p0, eps, n_leap, grad, state, inv_metric)
    return q, 0.5 * float(np.sum(xi * xi)) - 0.5 * float(np.sum(m * p * p))
