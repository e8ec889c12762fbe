"""The paper's copula prior (Sec. 2.2.1) on the GPU against the FP64 oracle.

Latent -> heights transform (oracle/copula.py: spectral Q^-1/2, Phi, stick
breaking) in both height precisions and at the scenario size; log-posterior of
latent states (likelihood of the derived heights + latent log-prior);
random-walk Metropolis on latents in lockstep with the oracle's decisions;
and the calls that need the CAR prior refuse the copula prior.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import copula as K
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, setup

pytestmark = pytest.mark.gpu


def latents(w, n, seed, r=0.9, scale=0.5):
    rng = np.random.default_rng(seed)
    lat = scale * rng.standard_normal((n, w.L, w.R, w.Q))
    lat[:, w.L - 1] = 0.0
    for c in range(n):
        lat[c, w.L - 1].reshape(-1)[:w.L - 1] = r + 0.05 * rng.random(w.L - 1)
    return lat


def _dtype(precision):
    return torch.float64 if precision == mt.PREC_F64 else torch.float32


@pytest.mark.parametrize("precision,tol", [(mt.PREC_F64, 1e-9), (mt.PREC_F32, 2e-3)])
def test_copula_heights_match_oracle(precision, tol):
    w = W.tiny()
    pr = W.problem(w)
    ctx = mt.from_workload(pr, precision=precision)
    ctx.set_prior(mt.PRIOR_COPULA)
    lat = torch.tensor(latents(w, 5, 1), dtype=_dtype(precision), device=DEV).contiguous()
    H = torch.zeros_like(lat)
    ctx.copula_heights(lat, H)
    torch.cuda.synchronize()
    T = pr["mu"][w.L - 1]
    Ln = lat.cpu().double().numpy()
    Hg = H.cpu().double().numpy()
    for c in range(Ln.shape[0]):
        ref = K.heights(Ln[c], T)
        assert np.max(np.abs(Hg[c] - ref)) <= tol, np.max(np.abs(Hg[c] - ref))
        assert np.all(np.diff(Hg[c], axis=0) > 0.0)
    ctx.close()


def test_copula_heights_scenario_size():
    w = W.scenario()
    pr = W.problem(w)
    ctx = mt.from_workload(pr, precision=mt.PREC_F32)
    ctx.set_prior(mt.PRIOR_COPULA)
    lat = torch.tensor(latents(w, 8, 2), dtype=torch.float32, device=DEV).contiguous()
    H = torch.zeros_like(lat)
    ctx.copula_heights(lat, H)
    torch.cuda.synchronize()
    T = pr["mu"][w.L - 1]
    Ln, Hg = lat.cpu().double().numpy(), H.cpu().double().numpy()
    for c in (0, 7):
        assert np.max(np.abs(Hg[c] - K.heights(Ln[c], T))) <= 2e-3
    ctx.close()


def test_copula_logpost_matches_oracle():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    ctx.set_prior(mt.PRIOR_COPULA)
    ln = latents(w, 4, 3)
    ln[3, w.L - 1].reshape(-1)[0] = 1.2                 # r outside (0, 1): -inf
    lat = torch.tensor(ln, dtype=torch.float64, device=DEV).contiguous()
    ll = torch.zeros(4, dtype=torch.float64, device=DEV)
    lp = torch.zeros_like(ll)
    ctx.logpost(lat, ll, lp)
    torch.cuda.synchronize()
    T = pr["mu"][w.L - 1]
    for c in range(3):
        H = K.heights(ln[c], T)
        assert abs(ll[c].item() - op.loglik(H)) <= 1e-6 * abs(op.loglik(H))
        assert abs(lp[c].item() - K.logprior(ln[c])) <= 1e-12 * abs(K.logprior(ln[c]))
    assert lp[3].item() == -math.inf
    ctx.close()


def test_copula_rw_lockstep_f64():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    ctx.set_prior(mt.PRIOR_COPULA)
    C, sigma, n_steps = 4, 0.002, 40
    L0 = torch.tensor(latents(w, C, 4), dtype=torch.float64, device=DEV).contiguous()
    ctx.init_chains(L0, w.seed_mcmc)
    T = pr["mu"][w.L - 1]
    cur = L0.cpu().numpy().copy()
    ll_cur = np.array([op.loglik(K.heights(cur[c], T)) for c in range(C)])
    lp_cur = np.array([K.logprior(cur[c]) for c in range(C)])
    prop = torch.zeros_like(L0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    lpp, logu = torch.zeros_like(llp), torch.zeros_like(llp)
    acc = torch.zeros(C, dtype=torch.int32, device=DEV)
    st = torch.zeros_like(L0)
    match = mismatch = tie = accepted = 0
    for k in range(n_steps):
        ctx.run(mt.KERNEL_RW, sigma, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        P = prop.cpu().numpy()
        a_gpu, lu = acc.cpu().numpy(), logu.cpu().numpy()
        for c in range(C):
            np.testing.assert_allclose(P[c], op.rw_propose(cur[c], sigma, w.seed_mcmc, c, k),
                                       rtol=0, atol=1e-12)
            lpn = K.logprior(P[c])
            lln = op.loglik(K.heights(P[c], T)) if np.isfinite(lpn) else 0.0
            delta = (lln + lpn) - (ll_cur[c] + lp_cur[c])
            a_ref = oracle.mh_decide(lpn, lln, lp_cur[c], ll_cur[c], lu[c])
            if bool(a_gpu[c]) == a_ref:
                match += 1
            elif abs(lu[c] - delta) < 1e-6:
                tie += 1
            else:
                mismatch += 1
            if a_gpu[c]:
                cur[c] = P[c]
                ll_cur[c], lp_cur[c] = lln, lpn
                accepted += 1
        ctx.get_state(st)
        np.testing.assert_array_equal(st.cpu().numpy(), cur)
    assert mismatch == 0, (match, tie, mismatch)
    assert 0 < accepted < n_steps * C
    ctx.close()


def test_copula_refuses_car_only_calls():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    ctx.set_prior(mt.PRIOR_COPULA)
    lat = torch.tensor(latents(w, 2, 5), dtype=torch.float32, device=DEV).contiguous()
    g = torch.zeros((2, w.L, w.R, w.Q), dtype=torch.float64, device=DEV)
    with pytest.raises(mt.MtError):
        ctx.grad(lat, g)
    ll = torch.zeros(2, dtype=torch.float64, device=DEV)
    with pytest.raises(mt.MtError):
        ctx.logpost_noalloc(lat, ll)
    ctx.init_chains(lat, 1)
    with pytest.raises(mt.MtError):
        ctx.run(mt.KERNEL_MALA, 0.01, 1, 1)
    ctx.set_prior(mt.PRIOR_CAR)                          # back to heights
    H = torch.tensor(W.init_chains(w, 2), dtype=torch.float32, device=DEV).contiguous()
    ctx.grad(H, g)
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(mt.PREC_F64, 1e-9), (mt.PREC_F32, 2e-3)])
def test_copula_heights_odd_grid(precision, tol):
    """A 5 x 7 grid (neither side a power of two; the DFT passes are direct
    sums over any size) with 3 surfaces and several r, including r near 0."""
    w = W.small(R=5, Q=7, bases=(40.0, 75.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), n_chains=4)
    pr = W.problem(w)
    ctx = mt.from_workload(pr, precision=precision)
    ctx.set_prior(mt.PRIOR_COPULA)
    lat = latents(w, 4, 9)
    for c, r in enumerate((1e-6, 0.3, 0.9, 0.999)):
        lat[c, w.L - 1].reshape(-1)[:w.L - 1] = r
    Lt = torch.tensor(lat, dtype=_dtype(precision), device=DEV).contiguous()
    H = torch.zeros_like(Lt)
    ctx.copula_heights(Lt, H)
    torch.cuda.synchronize()
    T = pr["mu"][w.L - 1]
    Ln, Hg = Lt.cpu().double().numpy(), H.cpu().double().numpy()
    for c in range(4):
        assert np.max(np.abs(Hg[c] - K.heights(Ln[c], T))) <= tol
    ctx.close()
