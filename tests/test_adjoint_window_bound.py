"""The bound behind the adjoint's scatter windows, checked numerically (FP64,
CPU).  A sample whose sigmoid argument is a (log2 units) adds coef *
sigma(1 - sigma) fixed-point units to a cell, sigma = 1 / (1 + 2^a); since
sigma(1 - sigma) = 2^a / (1 + 2^a)^2 <= 2^-|a|, every sample with
|a| >= log2|coef| + 4 adds less than 2^-4 units, and along one side of a
surface, where |a| grows by at least s per sample, all of them together add
less than 2^-4 / (1 - 2^-s)."""
import math

import numpy as np


def _dsig(a):
    e = 2.0 ** (-abs(a))
    return e / (1.0 + e) ** 2            # sigma(1 - sigma), symmetric in a


def test_single_sample_bound():
    for a in np.linspace(-80.0, 80.0, 4001):
        assert _dsig(a) <= 2.0 ** -abs(a) * (1 + 1e-15)


def test_tail_sum_bound():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        coef = 10.0 ** rng.uniform(-3, 9)
        s = 10.0 ** rng.uniform(-2, 1)                 # vertical step per sample, log2 units
        a0 = math.log2(coef) + 4 + rng.uniform(0, s)   # first sample outside the window
        n = min(int(200 / s) + 1, 100000)
        tail = coef * sum(_dsig(a0 + k * s) for k in range(n))
        assert tail < 2.0 ** -4 / (1.0 - 2.0 ** -s), (coef, s, tail)
