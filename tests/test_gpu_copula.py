"""The paper's copula prior (Sec. 2.2.1) on the GPU against the FP64 oracle.

Latent -> heights transform (oracle/copula.py: spectral Q^-1/2, Phi, stick
breaking) in both height precisions and at the scenario size; log-posterior of
latent states (likelihood of the derived heights + latent log-prior);
random-walk Metropolis on latents in lockstep with the oracle's decisions;
gradients on latents (the adjoint back through the transform) against the
oracle's chain rule, and HMC on latents in lockstep; the allocation-free call
refuses the copula prior.
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
    ll = torch.zeros(2, dtype=torch.float64, device=DEV)
    with pytest.raises(mt.MtError):
        ctx.logpost_noalloc(lat, ll)
    ctx.grad(lat, g)                                     # gradients on latents are fine
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


class _LatentProblem:
    """The oracle's log-density and gradient in latent coordinates: the
    likelihood of the derived heights, its gradient back through the transform
    (oracle/copula.py heights_vjp), the latent log-prior and its gradient."""

    def __init__(self, op, T):
        self.op, self.T = op, T

    def loglik(self, lat):
        return self.op.loglik(K.heights(lat, self.T))

    def logprior(self, lat):
        return K.logprior(lat)

    def grad_loglik(self, lat):
        H = K.heights(lat, self.T)
        return K.heights_vjp(lat, self.T, self.op.grad_loglik(H))

    def grad_logprior(self, lat):
        return K.logprior_grad(lat)


def test_copula_gradient_matches_oracle():
    """mt_grad on latents: the heights' log-likelihood gradient (adjoint)
    back through the copula transform, plus -z, against the oracle's chain
    rule (itself pinned by central differences) within 1e-3 of the largest
    component; the log-posterior alongside."""
    w = W.small(R=6, Q=5, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), G=48,
                n_zenith=9, n_azimuth=13, n_sensors=3)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    ctx.set_prior(mt.PRIOR_COPULA)
    lat = latents(w, 2, 5, r=0.6)
    Lt = torch.tensor(lat, dtype=torch.float32, device=DEV).contiguous()
    g = torch.zeros(Lt.shape, dtype=torch.float64, device=DEV)
    lp = torch.zeros(2, dtype=torch.float64, device=DEV)
    ctx.grad(Lt, g, lp)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    Ln = Lt.double().cpu().numpy()
    lpx = _LatentProblem(op, pr["mu"][w.L - 1])
    for c in range(2):
        ref = lpx.grad_loglik(Ln[c]) + lpx.grad_logprior(Ln[c])
        scale = np.abs(ref).max()
        assert np.max(np.abs(g[c] - ref)) <= 1e-3 * scale, (c, np.max(np.abs(g[c] - ref)), scale)
        ref_lp = lpx.loglik(Ln[c]) + lpx.logprior(Ln[c])
        assert abs(lp[c].item() - ref_lp) <= 2e-2 + 1e-6 * abs(ref_lp), (c, lp[c].item(), ref_lp)
    ctx.close()


def test_copula_hmc_lockstep():
    """HMC on latents against the oracle's HMC with the latent log-density:
    proposals within the FP32 trajectory error, decisions equal except within
    the FP32 band; then a capped-NUTS iteration and a MALA step run on the
    same context."""
    from oracle import hmc
    w = W.small(R=5, Q=7, bases=(40.0, 75.0), G=24, n_zenith=6, n_azimuth=7, n_chains=3)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    ctx.set_prior(mt.PRIOR_COPULA)
    C, eps, n_leap = 3, 0.01, 3
    ctx.set_hmc(n_leap)
    L0 = torch.tensor(latents(w, C, 11, r=0.5), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(L0, 13)
    lpx = _LatentProblem(op, pr["mu"][w.L - 1])
    logpi = lambda x: lpx.loglik(x) + lpx.logprior(x)
    cur = L0.double().cpu().numpy()
    lp_cur = np.array([logpi(cur[c]) for c in range(C)])
    prop = torch.zeros_like(L0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    lpp, logu = torch.zeros_like(llp), torch.zeros_like(llp)
    acc = torch.zeros(C, dtype=torch.int32, device=DEV)
    st = torch.zeros_like(L0)
    accepted = band = 0
    for k in range(6):
        ctx.run(mt.KERNEL_HMC, eps, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        P = prop.double().cpu().numpy()
        for c in range(C):
            q, dk = hmc.propose(lpx, cur[c], eps, n_leap, 13, c, k, state=np.float32)
            disp = float(np.max(np.abs(q - cur[c])))
            assert np.max(np.abs(P[c] - q)) <= 1e-4 + 1e-4 * disp, (k, c, np.max(np.abs(P[c] - q)))
            lq = logpi(P[c]) if np.isfinite(lpx.logprior(P[c])) else -np.inf
            delta = lq - lp_cur[c] + dk
            a_ref = bool(np.isfinite(lq) and logu[c].item() < delta)
            if bool(acc[c].item()) != a_ref:
                assert abs(logu[c].item() - delta) < 5e-2, (k, c, logu[c].item(), delta)
                band += 1
            if acc[c].item():
                cur[c] = P[c]
                lp_cur[c] = lq
                accepted += 1
        ctx.get_state(st)
        np.testing.assert_array_equal(st.double().cpu().numpy(), cur)
    assert accepted > 0 and band <= 1
    ctx.set_nuts(2)
    ctx.run(mt.KERNEL_NUTS, eps, 1, 1)
    ctx.run(mt.KERNEL_MALA, 0.005, 1, 1)
    ll = torch.zeros(C, dtype=torch.float64, device=DEV)
    ctx.get_state(st, ll)
    S = st.double().cpu().numpy()
    for c in range(C):
        assert abs(ll[c].item() - lpx.loglik(S[c])) <= 2e-2
    ctx.close()
