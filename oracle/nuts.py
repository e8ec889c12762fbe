"""FP64 CPU oracle of the capped NUTS trajectory (test infrastructure; only
``tests/`` and ``bench.py``'s CPU legs may import it).

Sec. 3.1: the paper samples with NUTS (Hoffman & Gelman 2014) capped at a
maximum trajectory length of 256 steps, and reports that almost every
iteration reaches the cap.  This is the trajectory NUTS builds when it runs
to its cap: no U-turn stop, the tree doubled max_depth times.  One iteration
of chain c at step k from heights q0 (log-density ll0 + lp0, gradient g0):

  momentum     xi ~ N(0, I) (Philox stream NUTS_P = 7, counter {pair, k, c},
               Box-Muller), p0 = xi / sqrt(m) for the diagonal inverse
               metric m, K(p) = sum m p^2 / 2, H = -(ll + lp) + K;
  doubling     for depth j = 0 .. D-1 the direction v_j = -1 if u_j < 1/2
               else +1 (u_j: Philox stream NUTS_U = 8, index j) and 2^j
               leapfrog steps of size v_j eps extend the trajectory from
               its end on that side (the gradient and log-density are taken
               at the position rounded to the stored precision; positions
               and momenta are carried in FP64);
  subtree      each new state n has log-weight w_n = -H_n; the subtree keeps
               a multinomial sample: state n replaces it when
               log u < w_n - W_sub (W_sub: log-sum of the weights so far,
               including w_n; u: index 64 + its leaf number 0 .. 2^D - 2);
  merge        after subtree j its sample replaces the trajectory's when
               log u < W_sub - W (biased progressive sampling; u: index
               32 + j), then W = logaddexp(W, W_sub) (W starts at -H_0);
  statistic    the mean of min(1, e^(H_0 - H_n)) over the 2^D - 1 new states
               (the acceptance statistic the step-size adaptation uses).

The chain moves to the trajectory's sample; there is no separate accept.

Parity pins (tests/test_oracle_nuts.py): depth 1 as one-step HMC, uniform
choice among equal energies, a Gaussian left invariant, the trajectory's
extent, and a diagonal metric as the unit one in rescaled coordinates.
Every function is pinned.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

STREAM_NUTS_P, STREAM_NUTS_U = 7, 8


def uniform(seed, chain, step, index):
    w = oracle.philox([index, step, chain, STREAM_NUTS_U], [seed & 0xFFFFFFFF, seed >> 32])
    return oracle.u01(w[0], w[1])


def logaddexp(a, b):
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


def iteration(logpi, grad, q0, ll0, lp0, g0, eps, depth, seed, chain, step, state=np.float32,
              inv_metric=None):
    """One capped NUTS iteration.  logpi(q) -> (ll, lp), grad(q) -> gradient,
    both at the rounded position q.  Returns (q, ll, lp, g, statistic,
    margin), margin being the smallest |log u - threshold| over the
    iteration's decisions whose threshold is not exactly 0 (how close a
    decision came to flipping; a subtree's first finite state always
    replaces the empty sample, its threshold w - W_sub being 0 exactly)."""
    m = np.ones(np.shape(q0)) if inv_metric is None else np.asarray(inv_metric, np.float64)
    xi = oracle.normals(seed, STREAM_NUTS_P, chain, step, int(np.size(q0))).reshape(np.shape(q0))
    p0 = xi / np.sqrt(m)
    H0 = -(ll0 + lp0) + 0.5 * float(np.sum(xi * xi))
    ends = {-1: (np.asarray(q0, np.float64), p0, np.asarray(g0, np.float64)),
            +1: (np.asarray(q0, np.float64), p0, np.asarray(g0, np.float64))}
    sel = (np.asarray(q0, np.float64), ll0, lp0, np.asarray(g0, np.float64))
    W, stat, margin, leaf = -H0, 0.0, math.inf, 0
    for j in range(depth):
        v = -1 if uniform(seed, chain, step, j) < 0.5 else 1
        e = v * eps
        W_sub, sub = -math.inf, None
        for _ in range(2 ** j):
            q64, p, g = ends[v]
            p_half = p + 0.5 * e * g
            q64 = q64 + e * (m * p_half)
            q = np.asarray(q64, state).astype(np.float64)
            ll, lp = logpi(q)
            g = grad(q)
            p = p_half + 0.5 * e * g
            H = -(ll + lp) + 0.5 * float(np.sum(m * p * p))
            w = -H if math.isfinite(H) else -math.inf
            stat += min(1.0, math.exp(H0 - H)) if math.isfinite(H) else 0.0
            W_new = logaddexp(W_sub, w)
            lu = math.log(uniform(seed, chain, step, 64 + leaf))
            if w > -math.inf and W_sub > -math.inf:
                margin = min(margin, abs(lu - (w - W_new)))
            if lu < w - W_new:
                sub = (q, ll, lp, g)
            W_sub = W_new
            ends[v] = (q64, p, g)
            leaf += 1
        lu = math.log(uniform(seed, chain, step, 32 + j))
        if W_sub > -math.inf:
            margin = min(margin, abs(lu - (W_sub - W)))
        if sub is not None and lu < W_sub - W:
            sel = sub
        W = logaddexp(W, W_sub)
    q, ll, lp, g = sel
    return q, ll, lp, g, stat / (2 ** depth - 1), margin
