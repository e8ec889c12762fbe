"""Pins of the diagnostics oracle against closed forms and worked examples.

Nested R-hat: a hand-computed 2 x 2 example, identical super-chains (R-hat 1),
invariance to an affine change of the parameter, the M = 1 relation to the
textbook Gelman-Rubin statistic, and i.i.d. draws (R-hat -> 1).  Interface
std: constant samples (0), half above / half below (1/2), ties (eta(0) = 1/2),
and a binomial fraction p (sqrt(p (1 - p))).
"""
import numpy as np

from oracle import diagnostics as D


def test_nested_rhat_worked_example():
    # K = 2 super-chains of M = 2 chains, one draw each: super-chain values
    # {0, 2} and {10, 12}: B = (1 - 6)^2 + (11 - 6)^2 = 50, W_k = 2, R = sqrt(26)
    d = np.array([[[0.0], [2.0], [10.0], [12.0]]])
    assert abs(D.nested_rhat(d, 2)[0] - np.sqrt(26.0)) < 1e-15


def test_nested_rhat_identical_super_chains_is_one():
    rng = np.random.default_rng(1)
    one = rng.standard_normal((5, 3, 4))                 # N=5 draws, M=3 chains, P=4
    d = np.concatenate([one, one, one], axis=1)          # 3 identical super-chains
    np.testing.assert_allclose(D.nested_rhat(d, 3), 1.0, rtol=0, atol=1e-15)


def test_nested_rhat_affine_invariance():
    rng = np.random.default_rng(2)
    d = rng.standard_normal((4, 12, 6)) + np.arange(12)[None, :, None] * 0.3
    r = D.nested_rhat(d, 4)
    np.testing.assert_allclose(D.nested_rhat(3.5 * d - 7.0, 4), r, rtol=1e-12)


def test_nested_rhat_single_chain_super_chains_match_gelman_rubin():
    # M = 1: B = var of chain means, W = mean within-chain variance, so
    # nested R^2 = 1 + B / W, while the textbook Gelman-Rubin
    # R_GR^2 = ((N - 1)/N W + B_GR / N) / W with B_GR = N * var of means:
    # nested R^2 = R_GR^2 + 1 / N
    rng = np.random.default_rng(3)
    N, C = 50, 6
    d = rng.standard_normal((N, C, 1)) + rng.standard_normal((1, C, 1))
    x = d[:, :, 0].T                                     # [chain][draw]
    means = x.mean(axis=1)
    B_gr = N * np.var(means, ddof=1)
    W_gr = np.var(x, axis=1, ddof=1).mean()
    r_gr2 = ((N - 1) / N * W_gr + B_gr / N) / W_gr
    assert abs(D.nested_rhat(d, C)[0] ** 2 - (r_gr2 + 1.0 / N)) < 1e-12


def test_nested_rhat_iid_draws_near_one():
    rng = np.random.default_rng(4)
    d = rng.standard_normal((200, 32, 3))
    r = D.nested_rhat(d, 8)
    assert np.all(np.abs(r - 1.0) < 0.02)


def test_interface_std_closed_forms():
    Lz, n_z = 10.0, 10                                   # levels 0, 1, ..., 9
    S = 8
    H = np.zeros((S, 1, 1, 3))
    H[:, 0, 0, 0] = 4.5                                  # constant: std 0 at every level
    H[:, 0, 0, 1] = np.where(np.arange(S) < 4, 2.5, 7.5) # half / half between levels 3..7
    H[:, 0, 0, 2] = 5.0                                  # exactly on level 5: eta(0) = 1/2
    s = D.interface_std(H, Lz, n_z)
    assert np.all(s[0, :, 0, 0] == 0.0)
    np.testing.assert_array_equal(s[0, :, 0, 1], [0, 0, 0, 0.5, 0.5, 0.5, 0.5, 0.5, 0, 0])
    assert np.all(s[0, :, 0, 2] == 0.0)                  # B = 1, 1/2 or 0 for every sample alike


def test_interface_std_binomial_fraction():
    rng = np.random.default_rng(5)
    S = 1000
    above = rng.random(S) < 0.3
    H = np.where(above, 6.0, 2.0).reshape(S, 1, 1, 1)
    s = D.interface_std(H, 10.0, 10)
    p = above.mean()
    np.testing.assert_allclose(s[0, 3:6, 0, 0], np.sqrt(p * (1 - p)), rtol=1e-12)
    # a tie for half the samples: B in {1/2, 0}: mean p/2, mean of squares p/4
    H2 = np.where(np.arange(S) % 2 == 0, 5.0, 1.0).reshape(S, 1, 1, 1)
    s2 = D.interface_std(H2, 10.0, 10)
    np.testing.assert_allclose(s2[0, 5, 0, 0], np.sqrt(0.5 / 4 - 0.25 ** 2), rtol=1e-12)
