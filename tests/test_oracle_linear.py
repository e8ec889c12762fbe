"""Pins of the linearised-forward-model oracle (oracle/linear.py; Sec.
2.1.2): voxel path lengths sum to the in-box length, axis-parallel and
diagonal rays against hand counts, a vertical ray's opacity through a
non-flat column, the voxel density of flat layers, the
linearisation exact at the reference and second order away from it."""
import math

import numpy as np

import oracle
from oracle import linear as LN
from paper_2603_28907_gb300 import workloads as W


def test_lengths_sum_to_the_in_box_segment():
    rng = np.random.default_rng(1)
    box = (200.0, 150.0, 150.0)
    for _ in range(20):
        o = np.array([rng.uniform(1, 199), rng.uniform(1, 149), rng.uniform(1, 149)])
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        seg = LN.ray_voxel_lengths(o, d, box, 7, 5, 9)
        assert abs(sum(L for _, L in seg) - oracle.t_exit(o, d, np.array(box))) < 1e-9
        assert all(L > 0 for _, L in seg)


def test_vertical_and_diagonal_rays():
    box = (100.0, 100.0, 100.0)
    # straight up from z = 5 in column (2, 3) of a 10 x 10 x 10 grid: 95 m,
    # 5 m in level 0 and 10 m in each level above
    seg = dict(LN.ray_voxel_lengths([35.0, 25.0, 5.0], [0.0, 0.0, 1.0], box, 10, 10, 10))
    assert seg == {(k * 10 + 2) * 10 + 3: (5.0 if k == 0 else 10.0) for k in range(10)}
    # along the body diagonal of a 2 x 2 x 2 grid from a corner region: equal
    # lengths sqrt(3) * 50 in the voxels (0,0,0) and (1,1,1) for a ray from
    # (1e-9, 1e-9, 1e-9)
    d = np.ones(3) / math.sqrt(3.0)
    seg = dict(LN.ray_voxel_lengths([1e-9, 1e-9, 1e-9], d, box, 2, 2, 2))
    assert set(seg) == {0, 7}
    assert abs(seg[0] - 50.0 * math.sqrt(3.0)) < 1e-6 and abs(seg[7] - 50.0 * math.sqrt(3.0)) < 1e-6


def test_vertical_ray_through_a_non_flat_column():
    """A ray straight up through column (i, j) of a non-square grid with
    random heights (hard indicator): its opacity is the sum over levels of dz
    times the density of the unit that contains the level's centre, the unit
    being set by the heights at the centre of that cell (mean of its four
    corner nodes).  Ties voxel indexing, density layout and the cell-centre
    reading together."""
    rng = np.random.default_rng(4)
    R, Q, nz = 5, 7, 20                                   # 4 x 6 cells, dz = 7.5 m
    w = W.small(R=R, Q=Q, bases=(40.0, 75.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.3), gamma=0.0)
    pr = W.problem(w)
    H = np.stack([b + rng.uniform(-12.0, 12.0, (R, Q)) for b in (40.0, 75.0, 110.0)])
    dx, dy, dz = pr["box"][0] / (Q - 1), pr["box"][1] / (R - 1), pr["box"][2] / nz
    Rd = LN.density(H, pr, nz).reshape(-1)
    for (i, j, z0) in ((1, 4, 3.0), (3, 0, 11.0), (2, 5, 0.5)):
        o = [(j + 0.3) * dx, (i + 0.6) * dy, z0]
        seg = LN.ray_voxel_lengths(o, [0.0, 0.0, 1.0], pr["box"], Q - 1, R - 1, nz)
        O = sum(L * Rd[v] for v, L in seg)
        hc = [0.25 * (H[l, i, j] + H[l, i, j + 1] + H[l, i + 1, j] + H[l, i + 1, j + 1]) for l in range(3)]
        ref = 0.0
        for k in range(nz):
            lo, hi = max(k * dz, z0), (k + 1) * dz
            if hi <= lo:
                continue
            zc = (k + 0.5) * dz
            unit = sum(1 for h in hc if h < zc)           # surfaces below the level centre
            ref += (hi - lo) * pr["rho"][unit]
        assert abs(O - ref) < 1e-9, (i, j, O, ref)


def test_flat_layers_density():
    w = W.small(R=3, Q=4, bases=(40.0, 75.0), rho=(2.65, 1.9, 0.0012), gamma=0.0)
    pr = W.problem(w)
    H = np.zeros((2, 3, 4))
    H[0], H[1] = 40.0, 75.0
    R = LN.density(H, pr, 15)                            # dz = 10 m, centres 5, 15, ..., 145
    col = R[:, 0, 0]
    np.testing.assert_allclose(col[:4], 2.65)            # centres 5..35 below 40
    np.testing.assert_allclose(col[4:7], 1.9)            # 45..65
    assert abs(col[7] - 0.5 * (1.9 + 0.0012)) < 1e-15    # centre 75 on the surface: eta(0) = 1/2
    np.testing.assert_allclose(col[8:], 0.0012)          # 85 .. 145 above


def test_linearisation_is_exact_at_the_reference_and_second_order():
    w = W.small(R=4, Q=5, n_zenith=3, n_azimuth=4, G=8)
    pr = W.problem(w)
    nz = 12
    rays = LN.lengths(pr, nz)
    Href = pr["mu"]
    O0 = LN.opacity(rays, LN.density(Href, pr, nz))
    lam0 = pr["I0"] * np.exp(-O0 / pr["Lambda"])
    C = np.maximum(np.round(lam0), 0).astype(np.int64)
    from scipy.special import gammaln
    exact = float(np.sum(C * np.log(lam0) - lam0 - gammaln(C + 1.0)))
    assert abs(LN.loglik(Href, pr, C, rays, nz, Href) - exact) < 1e-9 * abs(exact)
    rng = np.random.default_rng(3)
    dH = rng.standard_normal(Href.shape)
    errs = []
    for s in (0.4, 0.2, 0.1):
        H = Href + s * dH
        O = LN.opacity(rays, LN.density(H, pr, nz))
        lam_exact = pr["I0"] * np.exp(-O / pr["Lambda"])
        lam_hat = lam0 * (1.0 - (O - O0) / pr["Lambda"])
        errs.append(np.max(np.abs(lam_hat - lam_exact)))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_loglik_grad_matches_central_differences():
    """The chain rule of loglik_grad against central differences of loglik
    at a few nodes (interior, edge and corner nodes of every surface)."""
    w = W.small(R=5, Q=6, bases=(40.0, 75.0), G=16, n_zenith=5, n_azimuth=6, n_sensors=2)
    pr = W.problem(w)
    op = oracle.OracleProblem(pr)
    C, _, _ = op.generate_counts(pr["H_true"], w.seed_data)
    nz = 12
    rays = LN.lengths(pr, nz)
    rng = np.random.default_rng(4)
    H = pr["mu"] + 2.0 * rng.standard_normal(pr["mu"].shape)
    g = LN.loglik_grad(H, pr, C, rays, nz, pr["mu"])
    h = 1e-5
    for ix in [(0, 2, 3), (1, 0, 0), (1, 4, 5), (0, 1, 0), (1, 3, 2)]:
        e = np.zeros_like(H)
        e[ix] = h
        fd = (LN.loglik(H + e, pr, C, rays, nz, pr["mu"]) - LN.loglik(H - e, pr, C, rays, nz, pr["mu"])) / (2 * h)
        assert abs(g[ix] - fd) <= 1e-5 * max(1.0, abs(fd)) + 1e-6 * np.abs(g).max(), (ix, g[ix], fd)
