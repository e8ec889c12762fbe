"""GPU path (libmt.so through its C ABI) against the FP64 oracle, element by element.

Tolerances:
  FP64 mode  per-chain log-likelihood within 1e-6 relative, log-prior 1e-9
             relative, per-ray opacity 1e-10 relative;
  FP32 modes per-chain log-likelihood within 1e-3 absolute (tiny and small
             problems), evaluated by the oracle on the FP32 heights the library
             holds, widened exactly to FP64;
  counts     bit-exact; accept decisions identical except where the oracle's
             ln u - delta lies within 1e-6 of zero (FP64) or within the
             library's own |delta error| (FP32 modes).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, heights, logpost, setup

pytestmark = pytest.mark.gpu

SMALLS = [
    W.small(),                                                     # 5x7, 2 surfaces, 35 px
    W.small(R=6, Q=5, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), G=37,
            n_zenith=9, n_azimuth=31, n_sensors=3),                # ragged 279 px x 3
    W.small(R=2, Q=2, bases=(60.0,), rho=(2.65, 0.0012), G=1, n_zenith=1, n_azimuth=1,
            n_sensors=1),                                          # one ray, one sample
    W.small(R=9, Q=4, bases=(30.0, 55.0, 80.0, 110.0, 140.0),
            rho=(2.65, 1.9, 0.0012, 1.9, 2.65, 0.0012), G=3, n_zenith=7, n_azimuth=37),
]


# ---------------------------------------------------------------- data
@pytest.mark.parametrize("w", [W.tiny()] + SMALLS, ids=lambda w: w.name)
@pytest.mark.parametrize("gamma", [1.0, 0.0])
def test_counts_bit_exact(w, gamma):
    pr, ctx, op, counts, lam = setup(w, gamma=gamma)
    c_ref, lam_ref, bad = op.generate_counts(pr["H_true"], w.seed_data)
    assert bad == 0
    np.testing.assert_allclose(lam.cpu().numpy(), lam_ref, rtol=1e-12)
    np.testing.assert_array_equal(counts.cpu().numpy(), c_ref)


def test_counts_knuth_and_ptrs_bit_exact():
    """A data set whose expected counts straddle 10 (I0 = 40: lambda from 3.7
    to 15.5, 1351 pixels below 10 and 697 above): the Knuth
    multiplication branch (lambda < 10) and Hoermann's PTRS branch both draw,
    bit-identical to the oracle's draws from the same Philox streams."""
    w = W.tiny()
    pr, ctx, op, counts, lam = setup(w, I0=40.0)
    lamv = lam.cpu().numpy()
    assert (lamv < 10.0).sum() > 500 and (lamv >= 10.0).sum() > 500, (lamv.min(), lamv.max())
    c_ref, lam_ref, bad = op.generate_counts(pr["H_true"], w.seed_data)
    assert bad == 0
    np.testing.assert_allclose(lamv, lam_ref, rtol=1e-12)
    np.testing.assert_array_equal(counts.cpu().numpy(), c_ref)


def test_counts_round_mode():
    w = W.tiny()
    pr, ctx, op, counts, lam = setup(w, count_mode=mt.COUNTS_ROUND)
    c_ref, lam_ref, _ = op.generate_counts(pr["H_true"], w.seed_data, count_mode=1)
    np.testing.assert_array_equal(counts.cpu().numpy(), c_ref)


# ---------------------------------------------------------------- per ray
@pytest.mark.parametrize("w", [W.tiny()] + SMALLS, ids=lambda w: w.name)
@pytest.mark.parametrize("gamma", [1.0, 0.3, 0.0])
def test_ray_terms_f64(w, gamma):
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64, gamma=gamma)
    Hs = np.stack([pr["H_true"], W.perturbed(pr["H_true"], 2.0, [7])])
    H = heights(Hs, mt.PREC_F64)
    nr = w.S * w.P
    O = torch.zeros((2, nr), dtype=torch.float64, device=DEV)
    T = torch.zeros_like(O)
    ctx.ray_terms(H, O, T)
    for c in range(2):
        np.testing.assert_allclose(O[c].cpu().numpy(), op.opacities(Hs[c]).ravel(), rtol=1e-10)
        np.testing.assert_allclose(T[c].cpu().numpy(), op.loglik_terms(Hs[c]).ravel(), rtol=1e-9,
                                   atol=1e-8)


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F32C, mt.PREC_F32A])
def test_ray_opacity_f32(precision):
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=precision)
    H = heights(W.perturbed(pr["H_true"], 2.0, [7])[None], precision)
    Hn = H.double().cpu().numpy()[0]
    O = torch.zeros((1, w.S * w.P), dtype=torch.float64, device=DEV)
    ctx.ray_terms(H, O, None)
    ref = op.opacities(Hn).ravel()
    err = np.abs(O[0].cpu().numpy() - ref) / ref
    assert err.max() < 2e-6, err.max()


def fp32_loglik_tol(pr, op=None, H=None):
    """Per-chain |ll_FP32 - ll_oracle| bound of the FP32 modes: 1e-3 absolute,
    at every size (the per-chain log-likelihood bound the FP32 march is built
    to; Eq. def_likelihood summed over all rays)."""
    return 1e-3


def bf16_loglik_tol(pr, op, H):
    """Per-chain bound of the BF16-heights mode against the oracle evaluated on
    the BF16-rounded heights: 1e-3 times max(1, dt/gamma) plus 5e-7 mwe of
    opacity error per ray propagated through |d ll / d O_p| = |lambda_p -
    C_p| / Lambda.  That mode marches on FP32 absolute cell coordinates with a
    2^-23 indicator quantum, so its error is stated, not held to the FP32
    modes' bar."""
    T = [oracle.t_exit(s_, d_, pr["box"]) for s_ in pr["sensors"] for d_ in pr["dirs"]]
    dt_max = max(T) / pr["G"]
    tol = 1e-3 * max(1.0, dt_max / pr["gamma"]) if pr["gamma"] > 0 else 1e-3
    O = op.opacities(H).ravel()
    sens = np.abs(pr["I0"] * np.exp(-O / pr["Lambda"]) - op.counts.ravel()) / pr["Lambda"]
    return tol + 5e-7 * sens.sum()


# ---------------------------------------------------------------- per chain
@pytest.mark.parametrize("w", [W.tiny()] + SMALLS, ids=lambda w: w.name)
def test_logpost_f64(w):
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    Hs = np.concatenate([pr["H_true"][None], W.init_chains(w, 3)])
    ll, lp = logpost(ctx, heights(Hs, mt.PREC_F64))
    for c in range(Hs.shape[0]):
        ref_ll, ref_lp = op.loglik(Hs[c]), op.logprior(Hs[c])
        assert abs(ll[c] - ref_ll) <= 1e-6 * abs(ref_ll), (c, ll[c], ref_ll)
        assert abs(lp[c] - ref_lp) <= 1e-9 * max(1.0, abs(ref_lp)), (c, lp[c], ref_lp)


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F32C, mt.PREC_F32A, mt.PREC_BF16])
@pytest.mark.parametrize("w", [W.tiny(), SMALLS[1], SMALLS[3]], ids=lambda w: w.name)
def test_logpost_reduced_precision(w, precision):
    pr, ctx, op, counts, _ = setup(w, precision=precision)
    Hs = np.concatenate([pr["H_true"][None], W.init_chains(w, 3)])
    H = heights(Hs, precision)
    ll, lp = logpost(ctx, H)
    Hn = H.double().cpu().numpy()
    if precision == mt.PREC_BF16:
        # the kernel reads ref_l + bf16(h - ref_l), ref_l = FP32 mean prior height
        ref = torch.tensor([np.float32(pr["mu"][l].mean()) for l in range(w.L)],
                           dtype=torch.float32, device=DEV).view(1, -1, 1, 1)
        Hq = ((H - ref).to(torch.bfloat16).float() + ref).double().cpu().numpy()
    else:
        Hq = Hn
    for c in range(Hs.shape[0]):
        ref_ll = op.loglik(Hq[c])
        tol = bf16_loglik_tol(pr, op, Hq[c]) if precision == mt.PREC_BF16 else fp32_loglik_tol(pr)
        assert abs(ll[c] - ref_ll) <= tol, (c, ll[c], ref_ll, ll[c] - ref_ll, tol)
        ref_lp = op.logprior(Hn[c])
        assert abs(lp[c] - ref_lp) <= 1e-9 * max(1.0, abs(ref_lp))


def test_logprior_ordering_and_bounds():
    w = W.small(R=5, Q=6, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65))
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    H = np.stack([pr["H_true"]] * 4)
    H[1, 1, 2, 3] = H[1, 0, 2, 3] + 0.05        # thinner than delta
    H[2, 2, 4, 5] = 150.01                       # above the box top
    H[3, 0, 0, 0] = -0.5                         # below the floor
    ll, lp = logpost(ctx, heights(H, mt.PREC_F64))
    assert np.isfinite(lp[0]) and np.all(lp[1:] == -np.inf)
    assert np.all(np.isfinite(ll))
    for c in range(4):
        assert lp[c] == op.logprior(H[c]) or abs(lp[c] - op.logprior(H[c])) < 1e-9 * abs(lp[c])


def test_zero_counts_pixels():
    w = W.small(G=24)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    c = counts.clone()
    c.view(-1)[::3] = 0
    ctx.set_counts(c)
    op.with_counts(c.cpu().numpy())
    H = W.perturbed(pr["H_true"], 1.0, [2])
    ll, _ = logpost(ctx, heights(H[None], mt.PREC_F64))
    ref = op.loglik(H)
    assert abs(ll[0] - ref) <= 1e-9 * abs(ref)


def test_host_and_device_pointers_agree():
    """The same call with host (numpy) buffers gives the bit-identical result."""
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    Hs = np.stack([pr["H_true"], W.perturbed(pr["H_true"], 1.0, [1])]).astype(np.float32)
    ll_d, lp_d = logpost(ctx, torch.tensor(Hs, device=DEV))
    ll_h = np.zeros(2)
    lp_h = np.zeros(2)
    ctx.logpost(Hs, ll_h, lp_h)
    np.testing.assert_array_equal(ll_h, ll_d)
    np.testing.assert_array_equal(lp_h, lp_d)


# ---------------------------------------------------------------- MCMC
def _lockstep(precision, n_steps, sigma, w):
    pr, ctx, op, counts, _ = setup(w, precision=precision)
    C = w.n_chains
    H0 = heights(W.init_chains(w), precision)
    ctx.init_chains(H0, w.seed_mcmc)
    cur = H0.double().cpu().numpy()
    n = cur[0].size
    dt = H0.dtype
    prop = torch.zeros_like(H0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    lpp = torch.zeros_like(llp)
    acc = torch.zeros(C, dtype=torch.int32, device=DEV)
    logu = torch.zeros_like(llp)
    st = torch.zeros_like(H0)
    ll_cur = np.array([op.loglik(cur[c]) for c in range(C)])
    lp_cur = np.array([op.logprior(cur[c]) for c in range(C)])
    stats = dict(match=0, tie=0, mismatch=0, accepted=0, max_dll=0.0)
    for k in range(n_steps):
        ctx.run(mt.KERNEL_RW, sigma, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        P = prop.double().cpu().numpy()
        a_gpu = acc.cpu().numpy()
        lu = logu.cpu().numpy()
        llp_gpu = llp.cpu().numpy()
        for c in range(C):
            ref_prop = op.rw_propose(cur[c], sigma, w.seed_mcmc, c, k)
            # FP32: H + sigma xi rounded to FP32 (half an ulp of ~150 m) plus
            # sigma times the FP32 Box-Muller error (a few ulps of xi)
            tol = 1e-12 * 200 if precision == mt.PREC_F64 else 8e-6 + 1e-6 * sigma
            assert np.max(np.abs(P[c] - ref_prop)) <= tol, (k, c, np.max(np.abs(P[c] - ref_prop)))
            # same uniform; CUDA's and the C library's log may differ in the last ulp
            assert lu[c] == pytest.approx(oracle.accept_logu(w.seed_mcmc, c, k), rel=4e-16, abs=1e-300)
            lpn = op.logprior(P[c])
            lln = op.loglik(P[c]) if np.isfinite(lpn) else 0.0
            if np.isfinite(lpn):
                stats["max_dll"] = max(stats["max_dll"], abs(llp_gpu[c] - lln))
            delta = (lln + lpn) - (ll_cur[c] + lp_cur[c])
            a_ref = oracle.mh_decide(lpn, lln, lp_cur[c], ll_cur[c], lu[c])
            band = 1e-6  # the same tie band in every precision
            if bool(a_gpu[c]) == a_ref:
                stats["match"] += 1
            elif abs(lu[c] - delta) < band:
                stats["tie"] += 1
            else:
                stats["mismatch"] += 1
            if a_gpu[c]:
                cur[c] = P[c]
                ll_cur[c], lp_cur[c] = lln, lpn
                stats["accepted"] += 1
        ctx.get_state(st)
        np.testing.assert_array_equal(st.double().cpu().numpy(), cur)
    return stats


def test_mh_lockstep_f64():
    w = W.tiny()
    s = _lockstep(mt.PREC_F64, 60, w.rw_sigma, w)
    assert s["mismatch"] == 0, s
    assert s["max_dll"] <= 1e-6 * 2e4, s
    assert 0 < s["accepted"] < 60 * w.n_chains, s


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F32C, mt.PREC_F32A])
def test_mh_lockstep_f32(precision):
    """FP32 march: identical accept decisions to the oracle's except where
    |ln u - Delta_oracle| < 1e-6 (ties are counted, mismatches outside the
    band fail), proposals' log-likelihoods within 1e-3."""
    w = W.tiny()
    s = _lockstep(precision, 40, w.rw_sigma, w)
    assert s["mismatch"] == 0, s
    assert s["max_dll"] <= 1e-3, s


def test_zero_step_accepts_everything():
    w = W.small(G=8)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    H0 = heights(W.init_chains(w), mt.PREC_F64)
    ctx.init_chains(H0, 3)
    ctx.run(mt.KERNEL_RW, 0.0, 4, 5)
    acc = torch.zeros(w.n_chains, dtype=torch.int64, device=DEV)
    assert ctx.get_state(accepts_out=acc) == 20
    assert torch.all(acc == 20)


def test_graph_equals_stepwise_and_resume():
    """n_super x n_within through graphs == single steps; resuming at step k is bit-identical."""
    w = W.tiny()
    res = []
    for mode in ("graph", "steps", "resume"):
        pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
        H0 = heights(W.init_chains(w), mt.PREC_F32)
        ctx.init_chains(H0, w.seed_mcmc)
        if mode == "graph":
            ctx.run(mt.KERNEL_RW, w.rw_sigma, 3, 4)
        elif mode == "steps":
            for _ in range(12):
                ctx.run(mt.KERNEL_RW, w.rw_sigma, 1, 1)
        else:
            ctx.run(mt.KERNEL_RW, w.rw_sigma, 1, 5)
            mid = torch.zeros_like(H0)
            assert ctx.get_state(mid) == 5
            ctx2 = mt.from_workload(pr, precision=mt.PREC_F32)
            ctx2.set_counts(counts)
            ctx2.init_chains(H0, w.seed_mcmc)
            ctx2.set_state(mid, 5)
            ctx2.run(mt.KERNEL_RW, w.rw_sigma, 7, 1)
            ctx = ctx2
        H = torch.zeros_like(H0)
        ll = torch.zeros(w.n_chains, dtype=torch.float64, device=DEV)
        assert ctx.get_state(H, ll) == 12
        res.append((H.cpu().numpy(), ll.cpu().numpy()))
    for r in res[1:]:
        np.testing.assert_array_equal(r[0], res[0][0])
        np.testing.assert_array_equal(r[1], res[0][1])


def test_sync_deadline_keeps_context_usable():
    """A host deadline shorter than the queued work returns MT_ETIMEDOUT; the context stays usable."""
    w = W.small(R=32, Q=32, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), G=256,
                n_zenith=48, n_azimuth=48, n_sensors=4, n_chains=64)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    ctx.init_chains(heights(W.init_chains(w), mt.PREC_F32), 1)
    ctx.run(mt.KERNEL_RW, 0.01, 20, 10)
    with pytest.raises(mt.MtError) as e:
        ctx.sync(1e-4)
    assert e.value.status == -5
    ctx.sync(0.0)
    assert ctx.get_state() == 200


def test_bad_arguments():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w)
    with pytest.raises(mt.MtError):
        ctx.set_sensors(np.array([[-1.0, 5.0, 5.0]]))
    with pytest.raises(mt.MtError):
        ctx.set_pixels(np.array([[0.0, 0.0, 2.0]]))
    with pytest.raises(mt.MtError):
        ctx.run(mt.KERNEL_RW, 0.1, 1, 1)  # no chains yet
    with pytest.raises(mt.MtError):
        ctx.set_grid(9, 4, 4, [1, 1, 1], np.ones(10))


@pytest.mark.parametrize("grid,bases", [(100, (40.0, 70.0, 110.0, 140.0)), (170, (40.0, 70.0, 110.0))],
                         ids=["phased-100x100x4", "hbm-170x170x3"])
def test_large_grid_paths(grid, bases):
    """Grids whose FP32 planes exceed shared memory: at 100 x 100 with 4
    surfaces (313 KB of planes) the march stages one surface's plane at a
    time; at 170 x 170 not even one plane and the rays' sums fit and the
    kernel reads its records from HBM.  Both must agree with the oracle, and
    the Metropolis loop runs on them."""
    rho = (2.65, 1.9, 0.0012, 2.65, 0.0012)[:len(bases) + 1]
    w = W.small(R=grid, Q=grid, bases=bases, rho=rho, G=64, n_zenith=6, n_azimuth=9, n_sensors=2)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    Hs = np.concatenate([pr["H_true"][None], W.init_chains(w, 2)])
    H = heights(Hs, mt.PREC_F32)
    ll, lp = logpost(ctx, H)
    Hn = H.double().cpu().numpy()
    for c in range(3):
        assert abs(ll[c] - op.loglik(Hn[c])) <= fp32_loglik_tol(pr, op, Hn[c])
    # and the Metropolis loop runs on that path too
    ctx.init_chains(H, 5)
    ctx.run(mt.KERNEL_RW, 0.01, 2, 2)
    Hs2 = torch.zeros_like(H)
    ll2 = torch.zeros(3, dtype=torch.float64, device=DEV)
    assert ctx.get_state(Hs2, ll2) == 4
    H2 = Hs2.double().cpu().numpy()
    for c in range(3):
        assert abs(ll2[c].item() - op.loglik(H2[c])) <= fp32_loglik_tol(pr, op, H2[c])


def test_binding_rejects_mismatched_arrays():
    """The binding refuses arrays the library would read or write out of
    bounds: FP32 heights for an FP64 context, a wrong grid shape, too short an
    output; nothing is launched for them."""
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    H64 = heights(W.init_chains(w, 2), mt.PREC_F64)
    ll = torch.zeros(2, dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        ctx.logpost(H64.float(), ll)                         # dtype of another precision
    with pytest.raises(ValueError):
        ctx.logpost(H64[:, :, :, :-1].contiguous(), ll)      # not [n][L][R][Q]
    with pytest.raises(ValueError):
        ctx.logpost(H64, torch.zeros(1, dtype=torch.float64, device=DEV))  # output too short
    with pytest.raises(ValueError):
        ctx.logpost(H64, torch.zeros(2, dtype=torch.float32, device=DEV))  # output not FP64
    ctx.logpost(H64, ll)                                      # the right arrays pass
