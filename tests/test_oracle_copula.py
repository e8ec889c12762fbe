"""Pins of the copula-prior oracle (oracle/copula.py; Sec. 2.2.1).

The spectral square root against dense linear algebra (U U^T = Q^-1 with Q
built node by node from the periodic 4-neighbour stencil, and against the
paper's Cholesky route for the covariance), the constant diagonal of Q^-1,
r = 0 reducing to independent columns (u = Phi(z)), ordering of the heights,
uniform marginals of u and the latent log-prior.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr
from scipy.stats import kstest

from oracle import copula as K


def dense_Q(R, Q, r):
    n = R * Q
    M = np.zeros((n, n))
    for i in range(R):
        for j in range(Q):
            a = i * Q + j
            M[a, a] += 4.0
            for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                b = ((i + di) % R) * Q + (j + dj) % Q
                M[a, b] -= r                      # wrap-around neighbours that coincide count twice
    return M


def test_spectral_root_squares_to_the_covariance():
    for (R, Q, r) in ((4, 5, 0.7), (6, 6, 0.99), (2, 3, 0.4)):
        n = R * Q
        U = np.stack([K.field(e.reshape(R, Q), r).reshape(-1) for e in np.eye(n)], axis=1)
        cov = np.linalg.inv(dense_Q(R, Q, r))
        np.testing.assert_allclose(U @ U.T, cov, rtol=0, atol=1e-12)
        np.testing.assert_allclose(U, U.T, atol=1e-13)   # the symmetric root
        # the paper's route: Cholesky Q = L L^T, U_c = L^-T; same covariance
        Lc = np.linalg.cholesky(dense_Q(R, Q, r))
        Uc = np.linalg.inv(Lc).T
        np.testing.assert_allclose(Uc @ Uc.T, U @ U.T, atol=1e-12)


def test_sigma11_is_the_constant_diagonal():
    for (R, Q, r) in ((4, 5, 0.7), (8, 3, 0.95)):
        d = np.diag(np.linalg.inv(dense_Q(R, Q, r)))
        np.testing.assert_allclose(d, K.sigma11(R, Q, r), rtol=1e-12)


def test_r_zero_gives_independent_columns():
    rng = np.random.default_rng(1)
    L, R, Q = 3, 5, 7
    lat = rng.standard_normal((L, R, Q))
    lat[L - 1] = 0.0
    lat[L - 1].reshape(-1)[:L - 1] = 1e-300              # r -> 0
    T = np.full((R, Q), 150.0)
    H = K.heights(lat, T)
    u0 = ndtr(lat[0])
    np.testing.assert_allclose(H[0], u0 * 150.0, rtol=1e-12)
    u1 = ndtr(lat[1])
    np.testing.assert_allclose(H[1], H[0] + u1 * (150.0 - H[0]), rtol=1e-12)


def test_heights_against_dense_linear_algebra():
    """The whole transform with a different r per surface, against a route
    that shares nothing with the oracle's FFT: the symmetric square root of
    the dense covariance Q(r_l)^-1 (scipy.linalg.sqrtm), each node's variance
    from the dense diagonal, Phi, and the stick-breaking of Eq.
    indep_columns (H_l = (1 - u_l) H_(l-1) + u_l T, H_(-1) = 0), top = T."""
    from scipy.linalg import sqrtm
    rng = np.random.default_rng(6)
    L, R, Q = 4, 4, 5
    lat = rng.standard_normal((L, R, Q))
    rs = [0.3, 0.95, 0.7]
    lat[L - 1] = 0.0
    lat[L - 1].reshape(-1)[:L - 1] = rs
    T = 130.0 + 10.0 * rng.random((R, Q))
    H = K.heights(lat, T)
    below = np.zeros((R, Q))
    for l in range(L - 1):
        cov = np.linalg.inv(dense_Q(R, Q, rs[l]))
        x = np.real(sqrtm(cov)) @ lat[l].reshape(-1)
        u = ndtr(x / np.sqrt(np.diag(cov))).reshape(R, Q)
        ref = (1.0 - u) * below + u * T
        np.testing.assert_allclose(H[l], ref, rtol=1e-9, atol=1e-9)
        below = ref
    np.testing.assert_array_equal(H[L - 1], T)


def test_heights_are_ordered_below_the_terrain():
    rng = np.random.default_rng(2)
    L, R, Q = 4, 6, 8
    T = 120.0 + 20.0 * rng.random((R, Q))
    for _ in range(20):
        lat = rng.standard_normal((L, R, Q))
        lat[L - 1].reshape(-1)[:L - 1] = rng.random(L - 1)
        H = K.heights(lat, T)
        assert np.all(H[0] > 0.0)
        assert np.all(np.diff(H, axis=0) > 0.0)
        assert np.array_equal(H[L - 1], T)


def test_copula_marginals_are_uniform():
    rng = np.random.default_rng(3)
    R, Q, r = 16, 16, 0.9
    s = math.sqrt(K.sigma11(R, Q, r))
    u = np.concatenate([ndtr(K.field(rng.standard_normal((R, Q)), r) / s)[::5, ::5].ravel()
                        for _ in range(300)])
    assert kstest(u, "uniform").pvalue > 1e-3


def test_latent_logprior():
    lat = np.zeros((3, 2, 2))
    lat[0] = 1.0
    lat[1] = [[1.0, 2.0], [0.0, 0.0]]
    lat[2].reshape(-1)[:2] = [0.3, 0.99]
    assert K.logprior(lat) == -0.5 * (4.0 + 5.0)
    lat[2].reshape(-1)[1] = 1.0
    assert K.logprior(lat) == -math.inf


def test_heights_vjp_matches_central_differences():
    """The chain rule of heights_vjp against central differences of
    sum(gH * heights) in a few z entries and in every r."""
    rng = np.random.default_rng(8)
    L, R, Q = 4, 6, 5
    lat = 0.7 * rng.standard_normal((L, R, Q))
    lat[L - 1] = 0.0
    lat[L - 1].reshape(-1)[:L - 1] = [0.35, 0.8, 0.97]
    T = 150.0 + rng.standard_normal((R, Q))
    gH = rng.standard_normal((L, R, Q))
    f = lambda x: float(np.sum(gH[:L - 1] * K.heights(x, T)[:L - 1]))
    g = K.heights_vjp(lat, T, gH)
    h = 1e-6
    idx = [(0, 1, 2), (1, 3, 0), (2, 5, 4), (2, 0, 0)] + [(L - 1, 0, j) for j in range(L - 1)]
    for ix in idx:
        e = np.zeros_like(lat)
        e[ix] = h
        fd = (f(lat + e) - f(lat - e)) / (2 * h)
        assert g[ix] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max()), (ix, g[ix], fd)
    assert np.all(g[L - 1].reshape(-1)[L - 1:] == 0.0)


def test_heights_vjp_closed_form_at_r_zero():
    """r -> 0: Q = 4 I, x = z / 2, Sigma_11 = 1/4, so u = Phi(z) and with two
    surfaces H_0 = Phi(z) T: the z gradient is gH_0 T phi(z)."""
    rng = np.random.default_rng(9)
    R, Q = 4, 7
    lat = np.zeros((2, R, Q))
    lat[0] = rng.standard_normal((R, Q))
    lat[1].reshape(-1)[0] = 1e-12
    T = 140.0 + rng.standard_normal((R, Q))
    gH = rng.standard_normal((2, R, Q))
    g = K.heights_vjp(lat, T, gH)
    phi = np.exp(-0.5 * lat[0] ** 2) / math.sqrt(2.0 * math.pi)
    np.testing.assert_allclose(g[0], gH[0] * T * phi, rtol=1e-9, atol=1e-12)
