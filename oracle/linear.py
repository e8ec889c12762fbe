"""FP64 CPU oracle of the paper's linearised forward model (test
infrastructure; only ``tests/`` and ``bench.py``'s CPU legs may import it).

Sec. 2.1.2 (Eqs. expected_counts_linearized / _approx) on the voxel density
grid of Sec. 2.1.4 (Eq. def_LM_density_grid_smooth):
* voxels: the (R-1) x (Q-1) cells of the surface grid times n_z levels of
  height dz = Lz / n_z; voxel (i, j, k) spans [j dx, (j+1) dx] x
  [i dy, (i+1) dy] x [k dz, (k+1) dz] (i = row, j = column);
* density R_v = rho_top + sum_l (rho_l - rho_{l+1}) varsigma_gamma(h_l - z_k),
  h_l = the surface at the cell centre (mean of its four corner nodes),
  z_k = (k + 1/2) dz (the level's centre);
* L_pv = length of ray p (its in-box segment [0, t_exit]) inside voxel v;
  opacity O_p(R) = sum_v L_pv R_v, lambda_p(R) = I0 exp(-O_p / Lambda);
* linearisation at R0 = R(H_ref):  G_pv = -lambda_p(R0) L_pv / Lambda and
  lambda_hat_p(R) = lambda_p(R0) + G_p (R - R0)
                  = lambda_p(R0) (1 - (O_p(R) - O_p(R0)) / Lambda);
* log-likelihood sum_p C_p ln lambda_hat_p - lambda_hat_p - ln C_p!  (-inf
  when some lambda_hat_p <= 0 with C_p > 0; lambda_hat_p <= 0 with C_p = 0
  is also -inf: the Poisson mean must be positive).
Readings (the paper gives neither): voxel columns are the surface grid's
cells with the surface at the cell centre; the voxel's density is taken at
its centre height.

Parity pins (tests/test_oracle_linear.py): voxel lengths summing to the
in-box segment, vertical and diagonal rays, a vertical ray through a
non-flat column against the cell-centre reading, flat-layer densities, exactness
at the reference with a second-order remainder, and central differences of
the gradient.  Every function is pinned.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import gammaln

import oracle


def ray_voxel_lengths(o, d, box, nx, ny, nz):
    """Exact (FP64) voxel path lengths of the segment o + t d, t in
    [0, t_exit]: list of (flat voxel index v = (k ny + i) nx + j, length)."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    te = oracle.t_exit(o, d, np.asarray(box, np.float64))
    n = (nx, ny, nz)
    h = (box[0] / nx, box[1] / ny, box[2] / nz)
    ts = [0.0, te]
    for a in range(3):
        if d[a] != 0.0:
            for b in range(n[a] + 1):
                t = (b * h[a] - o[a]) / d[a]
                if 0.0 < t < te:
                    ts.append(t)
    ts = np.unique(np.array(ts))
    out = {}
    for t0, t1 in zip(ts[:-1], ts[1:]):
        if t1 <= t0:
            continue
        m = o + 0.5 * (t0 + t1) * d
        j = min(int(m[0] / h[0]), nx - 1)
        i = min(int(m[1] / h[1]), ny - 1)
        k = min(int(m[2] / h[2]), nz - 1)
        v = (k * ny + i) * nx + j
        out[v] = out.get(v, 0.0) + (t1 - t0)
    return sorted(out.items())


def lengths(prob, nz):
    """Per ray (sensor-major, as the ray table) the list of (v, L_pv)."""
    nx, ny = prob["Q"] - 1, prob["R"] - 1
    rays = []
    for s in np.asarray(prob["sensors"]).reshape(-1, 3):
        for d in np.asarray(prob["dirs"]).reshape(-1, 3):
            rays.append(ray_voxel_lengths(s, d, prob["box"], nx, ny, nz))
    return rays


def density(H, prob, nz):
    """R [nz][ny][nx] of heights H [L][R][Q] (FP64)."""
    H = np.asarray(H, np.float64)
    L = H.shape[0]
    rho = np.asarray(prob["rho"], np.float64)
    g = float(prob["gamma"])
    hc = 0.25 * (H[:, :-1, :-1] + H[:, :-1, 1:] + H[:, 1:, :-1] + H[:, 1:, 1:])   # [L][ny][nx]
    dz = prob["box"][2] / nz
    R = np.full((nz,) + hc.shape[1:], rho[L])
    for k in range(nz):
        z = (k + 0.5) * dz
        for l in range(L):
            u = hc[l] - z
            s = np.where(u > 0, 1.0, np.where(u < 0, 0.0, 0.5)) if g == 0.0 else 1.0 / (1.0 + np.exp(-u / g))
            R[k] += (rho[l] - rho[l + 1]) * s
    return R


def opacity(rays, R):
    Rf = np.asarray(R, np.float64).reshape(-1)
    return np.array([sum(Lv * Rf[v] for v, Lv in r) for r in rays])


def loglik(H, prob, counts, rays, nz, H_ref):
    """Linearised log-likelihood of heights H (reference heights H_ref)."""
    I0, Lam = float(prob["I0"]), float(prob["Lambda"])
    O0 = opacity(rays, density(H_ref, prob, nz))
    O = opacity(rays, density(H, prob, nz))
    lam0 = I0 * np.exp(-O0 / Lam)
    lam = lam0 * (1.0 - (O - O0) / Lam)
    C = np.asarray(counts, np.float64).reshape(-1)
    if np.any(lam <= 0.0):
        return -math.inf
    return float(np.sum(C * np.log(lam) - lam - gammaln(C + 1.0)))


def loglik_grad(H, prob, counts, rays, nz, H_ref):
    """Gradient with respect to the node heights of loglik (gamma > 0), by
    the chain rule: d ll / d lambda_hat_p = C_p / lambda_hat_p - 1,
    d lambda_hat_p / d R_v = -lambda_p(R0) L_pv / Lambda,
    d R_v / d h_l(cell) = (rho_l - rho_{l+1}) varsigma'(h_l - z_k) with
    varsigma' = varsigma (1 - varsigma) / gamma, and the cell-centre height
    h_l(cell) the mean of the cell's four corner nodes (1/4 each)."""
    H = np.asarray(H, np.float64)
    L, R, Q = H.shape
    I0, Lam, g = float(prob["I0"]), float(prob["Lambda"]), float(prob["gamma"])
    rho = np.asarray(prob["rho"], np.float64)
    O0 = opacity(rays, density(H_ref, prob, nz))
    O = opacity(rays, density(H, prob, nz))
    lam0 = I0 * np.exp(-O0 / Lam)
    lam = lam0 * (1.0 - (O - O0) / Lam)
    C = np.asarray(counts, np.float64).reshape(-1)
    f = (C / lam - 1.0) * (-lam0 / Lam)              # d ll / d O_p
    nx, ny = Q - 1, R - 1
    gR = np.zeros(nz * ny * nx)
    for p, ray in enumerate(rays):
        for v, Lv in ray:
            gR[v] += f[p] * Lv
    gR = gR.reshape(nz, ny, nx)
    hc = 0.25 * (H[:, :-1, :-1] + H[:, :-1, 1:] + H[:, 1:, :-1] + H[:, 1:, 1:])
    dz = prob["box"][2] / nz
    out = np.zeros_like(H)
    for l in range(L):
        gcell = np.zeros((ny, nx))
        for k in range(nz):
            s = 1.0 / (1.0 + np.exp(-(hc[l] - (k + 0.5) * dz) / g))
            gcell += gR[k] * (rho[l] - rho[l + 1]) * s * (1.0 - s) / g
        out[l, :-1, :-1] += 0.25 * gcell
        out[l, :-1, 1:] += 0.25 * gcell
        out[l, 1:, :-1] += 0.25 * gcell
        out[l, 1:, 1:] += 0.25 * gcell
    return out
