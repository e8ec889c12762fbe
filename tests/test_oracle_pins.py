"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle routine to a closed form, an invariant, a library
routine, a published known answer or a brute-force computation, chosen so a
plausible slip (dropped term, wrong sign, swapped index, transposed operand)
fails at least one of them.  CPU only.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special
import scipy.stats

import oracle
from paper_2603_28907_gb300 import workloads as W
from tests.exact_geometry import exact_unit_lengths

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 against the SC'11 authors' known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_u01_exact_and_open_interval():
    assert oracle.u01(0, 0) == 0.5 * 2.0 ** -52
    top = oracle.u01(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and top == (2.0 ** 52 - 0.5) * 2.0 ** -52
    # the low 12 bits of the 64-bit word are dropped
    assert oracle.u01(0xFFF, 0) == oracle.u01(0, 0)
    assert oracle.u01(0x1000, 0) == 1.5 * 2.0 ** -52


def test_normals_distribution():
    z = oracle.normals(1234, 3, 7, 11, 200_000)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # both members of a Box-Muller pair are used and are distinct
    assert z[0] != z[1]
    # different streams / chains / steps give different sequences
    assert not np.allclose(z[:8], oracle.normals(1234, 3, 8, 11, 8))
    assert not np.allclose(z[:8], oracle.normals(1234, 3, 7, 12, 8))


# ---------------------------------------------------------------- geometry
def test_t_exit_cases():
    box = [200.0, 150.0, 100.0]
    assert oracle.t_exit([10, 20, 30], [0, 0, 1], box) == pytest.approx(70.0)
    assert oracle.t_exit([10, 20, 30], [0, 0, -1], box) == pytest.approx(30.0)
    assert oracle.t_exit([10, 20, 30], [1, 0, 0], box) == pytest.approx(190.0)
    assert oracle.t_exit([10, 20, 30], [0, -1, 0], box) == pytest.approx(20.0)
    rng = np.random.default_rng(0)
    for _ in range(200):
        o = rng.uniform([1, 1, 1], np.array(box) - 1)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t = oracle.t_exit(o, d, box)
        p = o + t * d
        # the exit point is on the boundary and every earlier point is inside
        on = np.isclose(p, 0, atol=1e-9) | np.isclose(p, box, atol=1e-9)
        assert on.any()
        q = o + 0.999 * t * d
        assert np.all(q > -1e-9) and np.all(q < np.array(box) + 1e-9)


def test_bilinear_reproduces_bilinear_functions_non_square():
    R, Q = 5, 8
    box = [210.0, 120.0, 100.0]
    x = np.arange(Q) * box[0] / (Q - 1)
    y = np.arange(R) * box[1] / (R - 1)
    a, b, c, d = 50.0, 0.1, -0.3, 0.002
    X, Y = np.meshgrid(x, y, indexing="xy")
    h = a + b * X + c * Y + d * X * Y          # h[r][c], row = y
    # at the nodes: exact node values
    for r in range(R):
        for cc in range(Q):
            assert oracle.surface(R, Q, box, h, x[cc], y[r]) == pytest.approx(h[r, cc], abs=1e-12)
    # anywhere: the bilinear interpolant of a bilinear function is the function itself
    rng = np.random.default_rng(1)
    for _ in range(300):
        px, py = rng.uniform(0, box[0]), rng.uniform(0, box[1])
        assert oracle.surface(R, Q, box, h, px, py) == pytest.approx(a + b * px + c * py + d * px * py,
                                                                     abs=1e-9)
    # outside the box the value is clamped to the edge
    assert oracle.surface(R, Q, box, h, -5.0, 10.0) == pytest.approx(a + c * 10.0, abs=1e-9)


def test_sigmoid_properties():
    for g in (0.5, 1.0, 3.0):
        assert oracle.sigma(0.0, g) == 0.5
        for u in (-7.0, -1.0, 0.3, 2.5):
            assert oracle.sigma(u, g) + oracle.sigma(-u, g) == pytest.approx(1.0, abs=1e-15)
            assert oracle.sigma(u, g) == pytest.approx(scipy.special.expit(u / g), rel=1e-14)
        h = 1e-6
        assert (oracle.sigma(h, g) - oracle.sigma(-h, g)) / (2 * h) == pytest.approx(1 / (4 * g), rel=1e-6)
    # Heaviside with eta(0) = 1/2
    assert oracle.sigma(-1e-300, 0.0) == 0.0
    assert oracle.sigma(0.0, 0.0) == 0.5
    assert oracle.sigma(1e-300, 0.0) == 1.0
    # varsigma_gamma -> eta as gamma -> 0
    assert oracle.sigma(0.01, 1e-4) == pytest.approx(1.0, abs=1e-12)
    assert oracle.sigma(-0.01, 1e-4) == pytest.approx(0.0, abs=1e-12)


def _flat_problem(heights, rho, G, gamma, sensor=(100.0, 100.0, 20.0), dirs=None, box=(200., 200., 150.)):
    L = len(heights)
    R = Q = 4
    H = np.stack([np.full((R, Q), h) for h in heights])
    prob = dict(L=L, R=R, Q=Q, box=np.array(box), rho=np.array(rho), sensors=np.array([sensor]),
                dirs=np.array(dirs), G=G, gamma=gamma, I0=1e4, Lambda=150.0, tau=0.01, car_r=0.99,
                delta=0.1, mu=H.copy())
    return oracle.OracleProblem(prob), H


def test_flat_layers_hard_indicator_closed_form():
    """gamma = 0, flat layers: unit length = thickness / cos(zenith), within dt/2 per crossing."""
    heights = [40.0, 70.0, 110.0]
    rho = [2.65, 1.9, 0.0012, 2.65]
    ths = np.radians([0.0, 5.0, 17.0, 31.0])
    dirs = np.stack([np.sin(ths) * np.cos(0.7), np.sin(ths) * np.sin(0.7), np.cos(ths)], -1)
    for G in (64, 1024, 16384):
        op, H = _flat_problem(heights, rho, G, 0.0, dirs=dirs)
        for p, th in enumerate(ths):
            O, lens = op.ray_opacity(H, 0, p, with_units=True)
            z = [20.0] + heights + [150.0]
            exact = np.diff(z) / math.cos(th)
            dt = (130.0 / math.cos(th)) / G
            assert np.all(np.abs(lens - exact) <= dt / 2 * 2 + 1e-9), (G, th, lens, exact)
            assert O == pytest.approx(float(np.dot(lens, rho)), rel=1e-12)


def test_unit_lengths_partition_of_unity():
    """Sum over units of the path lengths equals the in-box ray length, any gamma (W sums to 1)."""
    w = W.small(R=6, Q=5, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), G=37)
    pr = W.problem(w)
    H = W.perturbed(pr["H_true"], 3.0, [9])
    for gamma in (0.0, 0.3, 1.0, 4.0):
        pr["gamma"] = gamma
        op = oracle.OracleProblem(pr)
        for s in range(op.S):
            for p in range(0, op.P, 3):
                _, lens = op.ray_opacity(H, s, p, with_units=True)
                T = oracle.t_exit(op.sensors[s], op.dirs[p], op.box)
                assert lens.sum() == pytest.approx(T, rel=1e-12)


def test_flat_layer_smooth_closed_form_second_order():
    """gamma > 0, one flat surface: integral of the sigmoid is a softplus difference;
    the midpoint sum converges at O(dt^2).  The surface sits 2 m under the box top so
    the integrand is not flat at the ray's end (a saturated one converges faster)."""
    h, gamma, z0 = 148.0, 1.0, 20.0
    th = math.radians(23.0)
    d = [math.sin(th), 0.0, math.cos(th)]
    T = 130.0 / math.cos(th)
    a0, aT = (h - z0) / gamma, (h - z0 - T * math.cos(th)) / gamma
    sp = lambda a: np.logaddexp(0.0, a)
    exact = gamma / math.cos(th) * (sp(a0) - sp(aT))
    errs = []
    for G in (32, 64, 128, 256):
        op, H = _flat_problem([h], [2.65, 0.0012], G, gamma, dirs=[d])
        _, lens = op.ray_opacity(H, 0, 0, with_units=True)
        errs.append(abs(lens[0] - exact))
        assert lens[0] + lens[1] == pytest.approx(T, rel=1e-12)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios), (errs, ratios)


def test_smooth_tends_to_hard():
    """varsigma_gamma -> eta: as gamma shrinks the smooth unit lengths approach the exact
    flat-layer thicknesses / cos(zenith) that the hard indicator measures."""
    heights = [40.0, 70.0, 110.0]
    rho = [2.65, 1.9, 0.0012, 2.65]
    th = 0.3
    d = [[math.sin(th), 0.0, math.cos(th)]]
    exact = np.diff([20.0] + heights + [150.0]) / math.cos(th)
    for g in (1.0, 0.1, 0.01):
        opg, H = _flat_problem(heights, rho, 65536, g, dirs=d)
        Lg = opg.ray_opacity(H, 0, 0, with_units=True)[1]
        assert np.max(np.abs(Lg - exact)) < 1e-3 * max(g, 0.01) * 10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bruteforce_exact_crossings_bilinear(seed):
    """gamma = 0 on random bilinear surfaces (4x4 grid): the sampled unit lengths
    converge to the exact quadratic-root lengths within dt/2 per crossing."""
    rng = np.random.default_rng(seed)
    R, Q, box = 4, 5, np.array([200.0, 160.0, 150.0])
    base = np.array([45.0, 80.0, 115.0])
    H = base[:, None, None] + rng.uniform(-12, 12, size=(3, R, Q))
    for l in range(1, 3):
        H[l] = np.maximum(H[l], H[l - 1] + 0.1)
    sensor = np.array([rng.uniform(30, 170), rng.uniform(30, 130), 20.0])
    dirs = []
    for _ in range(6):
        th, ph = rng.uniform(0, math.radians(65)), rng.uniform(0, 2 * math.pi)
        dirs.append([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    dirs = np.array(dirs)
    prob = dict(L=3, R=R, Q=Q, box=box, rho=np.array([2.65, 1.9, 0.0012, 2.65]),
                sensors=sensor[None], dirs=dirs, G=64, gamma=0.0, I0=1e4, Lambda=150.0,
                tau=0.01, car_r=0.99, delta=0.1, mu=H.copy())
    op = oracle.OracleProblem(prob)
    for p in range(len(dirs)):
        exact, T = exact_unit_lengths(H, sensor, dirs[p], box)
        assert exact.sum() == pytest.approx(T, rel=1e-12)
        prev = None
        for G in (256, 4096, 65536):
            op.set(G=G)
            _, lens = op.ray_opacity(H, 0, p, with_units=True)
            dt = T / G
            err = np.abs(lens - exact)
            # each unit has at most a few crossings on a 4x5 grid
            assert np.all(err <= 4 * dt / 2 + 1e-9), (p, G, lens, exact)
            prev = err.max()
        assert prev < 4 * (T / 65536)


# ---------------------------------------------------------------- likelihood
def test_poisson_logpmf_against_scipy_and_small_cases():
    assert oracle.poisson_logpmf(0, 1.0) == pytest.approx(-1.0, abs=1e-15)
    assert oracle.poisson_logpmf(1, 1.0) == pytest.approx(-1.0, abs=1e-15)
    for C_ in (0, 1, 2, 7, 150, 999, 4321):
        for lam in (0.3, 1.0, 9.5, 140.0, 1000.0, 3000.0):
            ref = scipy.stats.poisson.logpmf(C_, lam)
            assert oracle.poisson_logpmf(C_, lam) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_centred_form_equals_direct():
    I0, Lam = 1e4, 150.0
    for C_ in (0, 1, 3, 80, 1000, 4000):
        for O in (10.0, 150.0, 345.0, 690.0):
            lam = I0 * math.exp(-O / Lam)
            a = oracle.poisson_logpmf(C_, lam)
            b = oracle.poisson_logpmf_centred(C_, O, I0, Lam)
            assert b == pytest.approx(a, rel=1e-12, abs=1e-9)


def test_loglik_is_sum_of_terms_and_matches_scipy():
    w = W.small(G=24)
    pr = W.problem(w)
    op = oracle.OracleProblem(pr)
    counts, lam, bad = op.generate_counts(pr["H_true"], 5)
    assert bad == 0
    op.with_counts(counts)
    H = W.perturbed(pr["H_true"], 2.0, [3])
    terms = op.loglik_terms(H)
    O = op.opacities(H)
    ref = scipy.stats.poisson.logpmf(counts, 1e4 * np.exp(-O / 150.0))
    np.testing.assert_allclose(terms, ref, rtol=1e-12, atol=1e-9)
    assert op.loglik(H) == pytest.approx(terms.sum(), rel=1e-13)
    np.testing.assert_allclose(op.loglik_batch(np.stack([H, pr["H_true"]]), 2),
                               [op.loglik(H), op.loglik(pr["H_true"])], rtol=1e-13)


def test_counts_rounding_mode():
    w = W.small(G=24)
    pr = W.problem(w)
    op = oracle.OracleProblem(pr)
    counts, lam, _ = op.generate_counts(pr["H_true"], 5, count_mode=1)
    np.testing.assert_array_equal(counts, np.rint(lam).astype(np.int32))


@pytest.mark.parametrize("lam", [0.5, 3.0, 9.9, 10.0, 57.3, 1000.0, 3000.0])
def test_poisson_draws_distribution(lam):
    n = 20000
    ks = np.array([oracle.poisson_draw(lam, 77, i)[0] for i in range(n)])
    assert abs(ks.mean() - lam) < 5 * math.sqrt(lam / n)
    assert abs(ks.var() / lam - 1.0) < 5 * math.sqrt(2.0 / n) + 0.01
    # chi-square goodness of fit on the central bins
    lo, hi = int(max(0, lam - 4 * math.sqrt(lam))), int(lam + 4 * math.sqrt(lam)) + 1
    if hi - lo > 60:
        edges = np.unique(np.linspace(lo, hi, 40).astype(int))
    else:
        edges = np.arange(lo, hi + 1)
    obs = np.histogram(ks, bins=edges)[0]
    cdf = scipy.stats.poisson.cdf(edges - 1, lam)
    exp = n * np.diff(cdf)
    keep = exp > 5
    chi2 = (((obs - exp) ** 2 / exp)[keep]).sum()
    assert scipy.stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


# ---------------------------------------------------------------- prior
def _prior_problem(R=4, Q=5, L=2, tau=0.01, r=0.99, delta=0.1):
    mu = np.stack([np.full((R, Q), 40.0 + 30.0 * l) for l in range(L)])
    prob = dict(L=L, R=R, Q=Q, box=np.array([200.0, 200.0, 150.0]), rho=np.ones(L + 1),
                sensors=np.zeros((0, 3)), dirs=np.array([[0.0, 0.0, 1.0]]), G=4, gamma=1.0,
                I0=1e4, Lambda=150.0, tau=tau, car_r=r, delta=delta, mu=mu)
    return oracle.OracleProblem(prob), mu


def _dense_Q(R, Q, r):
    n = R * Q
    A = np.zeros((n, n))
    for i in range(R):
        for j in range(Q):
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                A[i * Q + j, ((i + di) % R) * Q + (j + dj) % Q] += 1.0
    return np.diag(A.sum(1)) - r * A


def test_prior_constant_offset_closed_form():
    op, mu = _prior_problem()
    c = 2.5
    H = mu + c
    L, R, Q = mu.shape
    assert op.logprior(H) == pytest.approx(-0.5 * 0.01 * L * R * Q * 4 * (1 - 0.99) * c * c, rel=1e-12)


def test_prior_dense_quadratic_form_and_spd():
    R, Q = 4, 5
    op, mu = _prior_problem(R, Q)
    rng = np.random.default_rng(3)
    H = mu + rng.normal(0, 3, mu.shape)
    Qm = _dense_Q(R, Q, 0.99)
    ref = sum(-0.5 * 0.01 * (H[l] - mu[l]).ravel() @ Qm @ (H[l] - mu[l]).ravel() for l in range(2))
    assert op.logprior(H) == pytest.approx(ref, rel=1e-12)
    for r in (0.0, 0.5, 0.99, 0.9999):
        scipy.linalg.cholesky(_dense_Q(R, Q, r))           # SPD for r in [0, 1)
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(_dense_Q(R, Q, 1.0) - 1e-12 * np.eye(R * Q))  # singular at r = 1


def test_prior_ordering_and_bounds():
    op, mu = _prior_problem()
    H = mu.copy()
    assert np.isfinite(op.logprior(H))
    H2 = H.copy()
    H2[1, 2, 3] = H2[0, 2, 3] + 0.1          # exactly delta apart: allowed
    assert np.isfinite(op.logprior(H2))
    H2[1, 2, 3] = H2[0, 2, 3] + 0.09          # thinner than delta
    assert op.logprior(H2) == -np.inf
    H3 = H.copy()
    H3[1, 0, 0] = 150.5                        # above the box top
    assert op.logprior(H3) == -np.inf
    H4 = H.copy()
    H4[0, 1, 1] = -0.01                        # below the floor
    assert op.logprior(H4) == -np.inf


# ---------------------------------------------------------------- MCMC
def test_zero_step_always_accepts_and_invalid_always_rejects():
    w = W.small(G=8)
    pr = W.problem(w)
    op = oracle.OracleProblem(pr)
    counts, _, _ = op.generate_counts(pr["H_true"], 5)
    op.with_counts(counts)
    H = pr["H_true"]
    _, acc, _, _, _ = op.rw_chain(H, 0.0, 11, 0, 0, 20)
    assert acc == 20
    assert not oracle.mh_decide(-np.inf, 0.0, -5.0, 0.0, -100.0)
    assert oracle.mh_decide(-5.0, 1.0, -5.0, 0.0, math.log(0.5))
    assert not oracle.mh_decide(-5.0, -1.0, -5.0, 0.0, math.log(0.5))


def test_accept_uniform_matches_philox():
    w = oracle.philox([0, 9, 3, oracle.STREAM["ACC"]], [77, 0])
    assert oracle.accept_logu(77, 3, 9) == math.log(oracle.u01(w[0], w[1]))


def test_rw_propose_uses_prop_stream_normals():
    op, mu = _prior_problem()
    Hp = op.rw_propose(mu, 0.25, 99, 2, 5)
    z = oracle.normals(99, oracle.STREAM["PROP"], 2, 5, mu.size)
    np.testing.assert_allclose(Hp.ravel(), mu.ravel() + 0.25 * z, rtol=0, atol=1e-12)


@pytest.mark.slow
def test_prior_only_chain_matches_dense_gaussian():
    """With no data the chain targets N(mu, (tau Q)^-1) per surface (far from the bounds)."""
    R, Q, tau, r = 4, 4, 1.0, 0.5
    op, mu = _prior_problem(R, Q, L=1, tau=tau, r=r)
    cov = np.linalg.inv(tau * _dense_Q(R, Q, r))
    samples = []
    for chain in range(8):
        _, acc, _, _, tr = op.rw_chain(mu, 0.3, 2024, chain, 0, 40000, use_lik=False, trace=True)
        assert 0.1 < acc / 40000 < 0.9
        samples.append(tr[2000::20])
    s = np.concatenate(samples) - mu.ravel()
    emp = np.cov(s.T)
    assert np.max(np.abs(s.mean(0))) < 0.08
    assert np.max(np.abs(np.diag(emp) / np.diag(cov) - 1)) < 0.12
    assert np.max(np.abs(emp - cov)) < 0.05


# ---------------------------------------------------------------- gradient
def _grad_problem(gamma=1.0):
    w = W.small(R=5, Q=6, bases=(40.0, 75.0), G=32, n_zenith=4, n_azimuth=5, gamma=gamma)
    pr = W.problem(w)
    op = oracle.OracleProblem(pr)
    counts, _, _ = op.generate_counts(pr["H_true"], 5)
    op.with_counts(counts)
    return op, W.perturbed(pr["H_true"], 1.5, [4])


def test_grad_loglik_central_differences():
    op, H = _grad_problem()
    g = op.grad_loglik(H)
    h = 1e-3
    rng = np.random.default_rng(0)
    idx = [np.unravel_index(i, H.shape) for i in rng.choice(H.size, 25, replace=False)]
    for ix in idx:
        Hp, Hm = H.copy(), H.copy()
        Hp[ix] += h
        Hm[ix] -= h
        fd = (op.loglik(Hp) - op.loglik(Hm)) / (2 * h)
        assert g[ix] == pytest.approx(fd, rel=1e-4, abs=1e-4 * np.abs(g).max())


def test_grad_logprior_central_differences():
    op, H = _grad_problem()
    g = op.grad_logprior(H)
    h = 1e-3
    for ix in [(0, 0, 0), (1, 4, 5), (0, 2, 3), (1, 0, 5)]:
        Hp, Hm = H.copy(), H.copy()
        Hp[ix] += h
        Hm[ix] -= h
        fd = (op.logprior(Hp) - op.logprior(Hm)) / (2 * h)
        assert g[ix] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_grad_flat_layer_closed_form():
    """One flat surface: d(lower-unit length)/dh -> (1/cos)[s(a0) - s(aT)] as G grows."""
    h, gamma, z0 = 60.0, 1.0, 20.0
    th = math.radians(15.0)
    d = [math.sin(th), 0.0, math.cos(th)]
    T = 130.0 / math.cos(th)
    sg = lambda a: 1.0 / (1.0 + math.exp(-a))
    a0, aT = (h - z0) / gamma, (h - z0 - T * math.cos(th)) / gamma
    dL = (sg(a0) - sg(aT)) / math.cos(th)
    op, H = _flat_problem([h], [2.65, 0.0012], 2048, gamma, dirs=[d])
    # with C = 0 and Lambda the ray's dll/dO = lambda / Lambda; dO/dh = (rho0 - rho1) dL
    g = op.grad_loglik(H).sum()
    O = op.ray_opacity(H, 0, 0)
    lam = 1e4 * math.exp(-O / 150.0)
    assert g == pytest.approx(lam / 150.0 * (2.65 - 0.0012) * dL, rel=1e-5)


def test_mala_proposal_and_logq():
    op, H = _grad_problem()
    grad = op.grad_loglik(H) + op.grad_logprior(H)
    eps = 0.5
    Hp = op.mala_propose(H, grad, eps, 8, 1, 3)
    xi = oracle.normals(8, oracle.STREAM["MALA"], 1, 3, H.size).reshape(H.shape)
    np.testing.assert_allclose(Hp, H + 0.5 * eps * eps * grad + eps * xi, atol=1e-12)
    assert op.mala_logq(Hp, H, grad, eps) == pytest.approx(-0.5 * np.sum(xi * xi), rel=1e-12)
    # with zero gradient the kernel is symmetric
    z = np.zeros_like(H)
    assert op.mala_logq(Hp, H, z, eps) == pytest.approx(op.mala_logq(H, Hp, z, eps), rel=1e-14)


@pytest.mark.parametrize("lam", [10.0, 30.0, 400.0, 5000.0])
def test_poisson_ptrs_acceptance_rate_closed_form(lam):
    """Hoermann's transformed rejection (1993) accepts value k with probability
    p(k) / alpha per attempt, alpha = 1.1239 + 1.1328 / (b - 3.4),
    b = 0.931 + 2.53 sqrt(lambda): the hat dominates the Poisson pmf, so one
    attempt succeeds with probability exactly 1 / alpha and the number of
    attempts is geometric with mean alpha.  A misread constant (in b, a,
    alpha or v_r) that keeps the drawn distribution close still moves this
    mean, which the moment and chi-square tests would not see."""
    b = 0.931 + 2.53 * np.sqrt(lam)
    alpha = 1.1239 + 1.1328 / (b - 3.4)
    n = 400000
    p = 1.0 / alpha
    sd = np.sqrt((1.0 - p) / p ** 2 / n)
    mean = oracle.poisson_mean_attempts(lam, 123, n)
    assert abs(mean - alpha) < 5.0 * sd, (lam, mean, alpha, sd)
