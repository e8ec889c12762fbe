"""FP64 CPU oracle of the chain diagnostics (test infrastructure).

Only ``tests/`` and ``bench.py``'s CPU legs may import this module; the
product path never does.  Plain numpy, float64, written to be read against
the definitions rather than to be fast.

* ``nested_rhat`` -- the nested R-hat of the super-chain design the paper
  uses to detect chains stuck near their starts (Sec. 3.2, "nested R-hat";
  definition of Margossian et al. 2024): C chains form K super-chains of M
  consecutive chains; for each parameter, with N draws per chain,
    chain mean        m_{mk} = mean_n f_{nmk}
    super-chain mean  m_k    = mean_m m_{mk},   grand mean m = mean_k m_k
    between super-chains  B = sum_k (m_k - m)^2 / (K - 1)
    within super-chain k  W_k = sum_m (m_{mk} - m_k)^2 / (M - 1)      [0 if M = 1]
                               + mean_m sum_n (f_{nmk} - m_{mk})^2 / (N - 1)  [0 if N = 1]
    W = mean_k W_k,   nested R-hat = sqrt(1 + B / W)   (1 when B = W = 0).
* ``interface_std`` -- the tomographic standard deviation of the
  below-interface indicators B^l_{ijk}(H) = eta(H_{l,i,j} - k dz), eta(0) = 1/2
  (Eq. def_below_interface_indicator), across samples of H (Sec. 4,
  Fig. tomography_std_poisson): voxel columns at the surface nodes, voxel
  levels z_k = k * (Lz / n_z), k = 0 .. n_z - 1; the population standard
  deviation over the samples, sqrt(mean(B^2) - mean(B)^2).

Parity pins (tests/test_oracle_diagnostics.py): a hand-computed example,
identical super-chains, affine invariance, the Gelman-Rubin special case,
i.i.d. draws, and closed forms of the interface deviation.  Every function
is pinned.
"""
from __future__ import annotations

import numpy as np


def nested_rhat(draws: np.ndarray, n_super: int) -> np.ndarray:
    """draws [N][C][P] -> nested R-hat [P]; chain c is component c % M of
    super-chain c // M (M = C / n_super)."""
    f = np.asarray(draws, np.float64)
    N, C, P = f.shape
    K = int(n_super)
    if K < 2 or C % K:
        raise ValueError("need n_super >= 2 dividing the number of chains")
    M = C // K
    f = f.reshape(N, K, M, P)
    chain_mean = f.mean(axis=0)                       # [K][M][P]
    super_mean = chain_mean.mean(axis=1)              # [K][P]
    grand = super_mean.mean(axis=0)                   # [P]
    B = ((super_mean - grand) ** 2).sum(axis=0) / (K - 1)
    Wk = np.zeros((K, P))
    if M > 1:
        Wk += ((chain_mean - super_mean[:, None, :]) ** 2).sum(axis=1) / (M - 1)
    if N > 1:
        Wk += (((f - chain_mean[None]) ** 2).sum(axis=0) / (N - 1)).mean(axis=1)
    W = Wk.mean(axis=0)
    out = np.empty(P)
    for p in range(P):
        if W[p] > 0.0:
            out[p] = np.sqrt(1.0 + B[p] / W[p])
        else:
            out[p] = 1.0 if B[p] == 0.0 else np.inf
    return out


def interface_std(samples: np.ndarray, Lz: float, n_z: int) -> np.ndarray:
    """samples [S][L][R][Q] -> std [L][n_z][R][Q] of eta(H - k Lz/n_z)."""
    H = np.asarray(samples, np.float64)
    S, L, R, Q = H.shape
    dz = Lz / n_z
    out = np.empty((L, n_z, R, Q))
    for k in range(n_z):
        zk = k * dz
        B = np.where(H > zk, 1.0, np.where(H == zk, 0.5, 0.0))   # [S][L][R][Q]
        mean = B.mean(axis=0)
        mean2 = (B * B).mean(axis=0)
        out[:, k] = np.sqrt(np.maximum(mean2 - mean * mean, 0.0))
    return out
