"""FP64 CPU oracle of the paper's copula prior over layer heights (test
infrastructure; only ``tests/`` and ``bench.py``'s CPU legs may import it).

Sec. 2.2.1 ("Constructing a prior for layer models"): per sampled surface l
(all but the top, which is the known terrain T) a standard-normal field z_l
on the R x Q grid and a spatial-dependence parameter r_l ~ U(0, 1);
  x_l = U(r_l) z_l  with U U^T = Q(r_l)^-1,  Q(r) = 4 I - r A  (periodic
        4-neighbour grid, Eq. def_CAR_precision),
  u_l = Phi(x_l / sqrt(Sigma_11))      (Eq. CAR_cdf_transform; the diagonal
        of Q^-1 is constant on the periodic grid),
  H_0 = u_0 T,  H_l = (1 - u_l) H_{l-1} + u_l T   (Eq. indep_columns with the
        uniforms replaced by the copula's).
Reading: U is the symmetric square root Q^-1/2, applied spectrally (the
periodic grid's Q is diagonalised by the 2-D discrete Fourier transform, with
eigenvalues 4 - 2 r (cos(2 pi k1 / R) + cos(2 pi k2 / Q))); the paper takes U
from a Cholesky factor.  Any U with U U^T = Q^-1 gives x the same N(0, Q^-1)
law, hence the same prior over heights.

Latent layout per chain, [L][R][Q] like the heights: planes 0 .. L-2 hold
z_0 .. z_{L-2}; the first L-1 entries of plane L-1 hold r_0 .. r_{L-2}; the
rest of plane L-1 is ignored.  The log-prior in latent coordinates is
-1/2 sum z^2 (constants dropped) when every r lies in (0, 1), else -inf.

Parity pins (tests/test_oracle_copula.py): the spectral root squaring to
the dense covariance, the whole transform with one r per surface against a
dense matrix square root, the constant diagonal, independent columns at r = 0,
ordering below the terrain, uniform marginals, the latent log-prior, and
the reverse pass against central differences and a closed form at r = 0.
Every function is pinned.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr


def eigenvalues(R: int, Q: int, r: float) -> np.ndarray:
    k1 = np.arange(R)[:, None]
    k2 = np.arange(Q)[None, :]
    return 4.0 - 2.0 * r * (np.cos(2.0 * math.pi * k1 / R) + np.cos(2.0 * math.pi * k2 / Q))


def sigma11(R: int, Q: int, r: float) -> float:
    """Diagonal of Q(r)^-1: the mean of the inverse eigenvalues."""
    return float(np.mean(1.0 / eigenvalues(R, Q, r)))


def field(z: np.ndarray, r: float) -> np.ndarray:
    """x = Q(r)^-1/2 z for one R x Q plane (2-D FFT, FP64)."""
    z = np.asarray(z, np.float64)
    R, Q = z.shape
    g = 1.0 / np.sqrt(eigenvalues(R, Q, r))
    return np.real(np.fft.ifft2(np.fft.fft2(z) * g))


def heights(latent: np.ndarray, terrain: np.ndarray) -> np.ndarray:
    """Latent [L][R][Q] (layout above) -> heights [L][R][Q], top = terrain."""
    lat = np.asarray(latent, np.float64)
    L, R, Q = lat.shape
    T = np.asarray(terrain, np.float64)
    H = np.empty((L, R, Q))
    below = np.zeros((R, Q))
    for l in range(L - 1):
        r = float(lat[L - 1].reshape(-1)[l])
        u = ndtr(field(lat[l], r) / math.sqrt(sigma11(R, Q, r)))
        H[l] = below + u * (T - below)          # = (1 - u) H_{l-1} + u T, H_{-1} = 0
        below = H[l]
    H[L - 1] = T
    return H


def logprior(latent: np.ndarray) -> float:
    lat = np.asarray(latent, np.float64)
    L = lat.shape[0]
    r = lat[L - 1].reshape(-1)[:L - 1]
    if not np.all((r > 0.0) & (r < 1.0)):
        return -math.inf
    return -0.5 * float(np.sum(lat[:L - 1] ** 2))


def heights_vjp(latent: np.ndarray, terrain: np.ndarray, gH: np.ndarray) -> np.ndarray:
    """Gradient with respect to the latents of sum(gH * heights(latent)) (the
    chain rule through the stick-breaking, Phi, the normalisation by
    sqrt(Sigma_11(r)) and the spectral filter Q(r)^-1/2; the top plane, the
    terrain, does not depend on the latents).  Same layout as the latents:
    planes 0 .. L-2 the z gradients, the first L-1 entries of plane L-1 the r
    gradients, the rest 0.

    With c_k = cos(2 pi k1/R) + cos(2 pi k2/Q) and eigenvalues l_k = 4 - 2 r c_k:
      x = F^-1 (F z / sqrt(l)),  S = mean(1 / l),  s = x / sqrt(S),  u = Phi(s)
      d l_k / dr = -2 c_k,  d l^-1/2 / dr = c l^-3/2,  dS / dr = mean(2 c / l^2)
    and the filter is symmetric, so the z gradient is the filtered x gradient."""
    lat = np.asarray(latent, np.float64)
    L, R, Q = lat.shape
    T = np.asarray(terrain, np.float64)
    gH = np.asarray(gH, np.float64)
    N = R * Q
    k1 = np.arange(R)[:, None]
    k2 = np.arange(Q)[None, :]
    c = np.cos(2.0 * math.pi * k1 / R) + np.cos(2.0 * math.pi * k2 / Q)
    # forward, keeping what the reverse pass needs
    rs, s_l, below_l = [], [], []
    below = np.zeros((R, Q))
    for l in range(L - 1):
        r = float(lat[L - 1].reshape(-1)[l])
        S = sigma11(R, Q, r)
        s = field(lat[l], r) / math.sqrt(S)
        rs.append(r)
        s_l.append(s)
        below_l.append(below)
        below = below + ndtr(s) * (T - below)
    out = np.zeros_like(lat)
    a = np.zeros((R, Q))                          # d/dH_l of everything above, carried down
    for l in range(L - 2, -1, -1):
        r, s, below = rs[l], s_l[l], below_l[l]
        u = ndtr(s)
        a = a + gH[l]
        gu = a * (T - below)
        a = a * (1.0 - u)                          # through H_l = (1 - u) H_{l-1} + u T
        gs = gu * np.exp(-0.5 * s * s) / math.sqrt(2.0 * math.pi)
        lam = 4.0 - 2.0 * r * c
        S = float(np.mean(1.0 / lam))
        gx = gs / math.sqrt(S)
        gS = -0.5 * float(np.sum(gs * s)) / S      # s = x S^-1/2
        out[l] = np.real(np.fft.ifft2(np.fft.fft2(gx) / np.sqrt(lam)))
        # r through the filter: <gx, F^-1 (F z c lam^-3/2)>, and through S
        dx_dr = np.real(np.fft.ifft2(np.fft.fft2(lat[l]) * c * lam ** -1.5))
        gr = float(np.sum(gx * dx_dr)) + gS * float(np.mean(2.0 * c / lam ** 2))
        out[L - 1].reshape(-1)[l] = gr
    return out


def logprior_grad(latent: np.ndarray) -> np.ndarray:
    """Gradient of logprior inside its support: -z on planes 0 .. L-2, 0 for
    the r entries and the unused rest of plane L-1."""
    lat = np.asarray(latent, np.float64)
    g = np.zeros_like(lat)
    g[:-1] = -lat[:-1]
    return g
