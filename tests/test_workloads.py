"""The seeded input generator (paper_2603_28907_gb300/workloads.py): the
workloads have the stated sizes, every geometry is a valid layer model
(ordered surfaces at least delta apart, inside the box; Sec. 2.1.3), pixel
directions are the polar bin centres with the image centre pointing up
(Sec. 2.1.1), sensors sit inside the box, and every draw is reproducible from
its seed."""
import math

import numpy as np
import pytest

from paper_2603_28907_gb300 import workloads as W


def test_standard_workload_sizes():
    t = W.tiny()
    assert (t.R, t.Q, t.L, t.S, t.n_zenith, t.n_azimuth, t.G, t.n_chains) == (16, 16, 3, 2, 32, 32, 64, 4)
    assert t.zenith_max_deg == 60.0 and len(t.rho) == t.L + 1
    s = W.scenario()
    assert (s.R, s.Q, s.L, s.S, s.n_zenith, s.n_azimuth, s.G, s.n_chains) == (64, 64, 4, 16, 64, 64, 256, 1024)
    assert s.zenith_max_deg == 70.0 and len(s.rho) == s.L + 1
    assert s.n_super * s.n_within == 1000
    assert s.box == (200.0, 200.0, 150.0)


@pytest.mark.parametrize("w", [W.tiny(), W.scenario(), W.small(R=5, Q=7)], ids=lambda w: w.name)
def test_geometries_are_valid_layer_models(w):
    Lz = w.box[2]
    for seed in ([w.seed_geom], [w.seed_init, 0], [w.seed_init, 5]):
        H = W.geometry(w, seed)
        assert H.shape == (w.L, w.R, w.Q) and H.dtype == np.float64
        assert np.all(np.diff(H, axis=0) >= w.delta - 1e-12)
        assert H.min() >= w.delta - 1e-12 and H.max() <= Lz - w.delta + 1e-12
    mu = W.prior_mean(w)
    for l, b in enumerate(w.bases):
        np.testing.assert_array_equal(mu[l], b)


def test_draws_are_reproducible_and_seed_dependent():
    w = W.tiny()
    np.testing.assert_array_equal(W.geometry(w, [3, 1]), W.geometry(w, [3, 1]))
    assert np.any(W.geometry(w, [3, 1]) != W.geometry(w, [3, 2]))
    H = W.init_chains(w, 3)
    np.testing.assert_array_equal(H[2], W.geometry(w, [w.seed_init, 2]))
    np.testing.assert_array_equal(W.perturbed(H, 1.0, [9]), W.perturbed(H, 1.0, [9]))


def test_bumps_follow_the_recipe():
    """With the ordering and box clip inactive, a surface minus its base is a
    sum of n_bumps Gaussians of the stated amplitude and width: its maximum is
    at most n_bumps * amplitude and it is positive everywhere."""
    w = W.small(R=41, Q=41, bases=(40.0, 90.0))
    H = W.geometry(w, [7])
    for l, b in enumerate(w.bases):
        d = H[l] - b
        assert d.min() > 0.0 and d.max() <= w.n_bumps * w.bump_amp + 1e-9


def test_pixel_directions_are_polar_bin_centres():
    nz, na, zmax = 5, 7, 60.0
    d = W.pixel_dirs(nz, na, zmax)
    assert d.shape == (nz * na, 3)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=1e-15)
    for i in range(nz):
        for j in range(na):
            p = i * na + j
            th = (i + 0.5) * math.radians(zmax) / nz
            ph = (j + 0.5) * 2.0 * math.pi / na
            np.testing.assert_allclose(d[p], [math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph),
                                              math.cos(th)], rtol=0, atol=1e-15)
    assert np.all(d[:, 2] > 0.0)


@pytest.mark.parametrize("w", [W.tiny(), W.scenario(), W.small(n_sensors=3)], ids=lambda w: w.name)
def test_sensors_inside_the_box_below_the_floor_surface(w):
    s = np.asarray(w.sensors)
    assert s.shape == (w.S, 3)
    for a in range(3):
        assert np.all(s[:, a] > 0.0) and np.all(s[:, a] < w.box[a])
    assert np.all(s[:, 2] < w.bases[0])


def test_problem_dict_is_complete():
    w = W.tiny()
    pr = W.problem(w)
    for k in ("box", "rho", "sensors", "dirs", "mu", "H_true", "L", "R", "Q", "S", "P", "G",
              "gamma", "I0", "Lambda", "tau", "car_r", "delta"):
        assert k in pr, k
    assert pr["dirs"].shape == (w.P, 3) and pr["H_true"].shape == (w.L, w.R, w.Q)
    np.testing.assert_array_equal(pr["H_true"], W.geometry(w, [w.seed_geom]))


def test_serving_mix_sizes_and_arrivals():
    reqs = W.serving_mix(64)
    t = [r.extra["arrival_s"] for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    rate = len(t) / t[-1]
    assert 10.0 < rate < 40.0                        # Poisson arrivals at 20 per second
    for r in reqs:
        assert 32 <= r.R <= 128 and r.R == r.Q
        assert 3 <= r.L <= 5 and len(r.rho) == r.L + 1
        assert 4 <= r.S <= 32 and 32 <= r.n_zenith <= 96 and 128 <= r.G <= 384
        assert 64 <= r.n_chains <= 1024
        assert 1000 <= r.n_super * r.n_within <= 10000 + 10
        assert len({r.seed_geom, r.seed_data, r.seed_init, r.seed_mcmc}) == 4
    assert len({r.seed_geom for r in reqs}) == len(reqs)
