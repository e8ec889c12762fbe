"""The paper's linearised forward model (Sec. 2.1.2) on the GPU against the
FP64 oracle (oracle/linear.py): log-likelihoods of several geometries in
both height precisions (the path lengths, voxel densities and linearisation
of the oracle, evaluated independently), the exact value at the reference
geometry, -inf once lambda_hat turns non-positive, random-walk steps under
the model, and the calls that need the march refusing it."""
import math

import numpy as np
import pytest
import torch

from oracle import linear as LN
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, setup

pytestmark = pytest.mark.gpu


def _dtype(precision):
    return torch.float64 if precision == mt.PREC_F64 else torch.float32


# FP64: 1e-10 relative.  FP32: 1e-3 absolute at the reference (dR = 0 there
# exactly, only the float-float sums of the Poisson terms round); at any other
# geometry (the data-generating one included) the FP32 voxel densities and
# the sums over a ray's voxels leave ~1e-7 relative per ray, 1e-6 relative of
# the chain's log-likelihood.
@pytest.mark.parametrize("precision,rtol,atol_near", [(mt.PREC_F64, 1e-10, 1e-6), (mt.PREC_F32, 1e-6, 1e-3)])
def test_linear_loglik_matches_oracle(precision, rtol, atol_near):
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=precision)
    nz = 30
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    rays = LN.lengths(pr, nz)
    C = counts.cpu().numpy()
    Hs = np.concatenate([pr["mu"][None], pr["H_true"][None], W.init_chains(w, 3)])
    H = torch.tensor(Hs, dtype=_dtype(precision), device=DEV).contiguous()
    ll = torch.zeros(H.shape[0], dtype=torch.float64, device=DEV)
    lp = torch.zeros_like(ll)
    ctx.logpost(H, ll, lp)
    torch.cuda.synchronize()
    Hn = H.cpu().double().numpy()
    for c in range(H.shape[0]):
        ref = LN.loglik(Hn[c], pr, C, rays, nz, pr["mu"])
        if math.isinf(ref):
            assert ll[c].item() == -math.inf
        elif c == 0:
            assert abs(ll[c].item() - ref) <= atol_near, (c, ll[c].item(), ref)
        else:
            assert abs(ll[c].item() - ref) <= rtol * abs(ref), (c, ll[c].item(), ref)
        assert abs(lp[c].item() - op.logprior(Hn[c])) <= 1e-9 * max(1.0, abs(op.logprior(Hn[c])))
    ctx.close()


def test_linear_negative_lambda_is_minus_inf():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    ctx.set_forward(mt.FORWARD_LINEAR, 30)
    H = np.array(pr["mu"])
    H[0] = 1.0                                            # far below the reference: opacity drops
    H[1] = 2.0                                            # by far more than Lambda on many rays
    H[2] = 3.0
    Ht = torch.tensor(H[None], dtype=torch.float64, device=DEV).contiguous()
    ll = torch.zeros(1, dtype=torch.float64, device=DEV)
    ctx.logpost(Ht, ll, None)
    torch.cuda.synchronize()
    assert ll[0].item() == LN.loglik(H, pr, counts.cpu().numpy(), LN.lengths(pr, 30), 30, pr["mu"])
    ctx.close()


def test_linear_random_walk_and_refusals():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    nz = 30
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, w.seed_mcmc)
    ctx.run(mt.KERNEL_RW, 0.05, 2, 5)
    H = torch.zeros_like(H0)
    ll = torch.zeros(w.n_chains, dtype=torch.float64, device=DEV)
    ctx.get_state(H, ll)
    torch.cuda.synchronize()
    rays = LN.lengths(pr, nz)
    Hn = H.cpu().double().numpy()
    for c in range(w.n_chains):
        ref = LN.loglik(Hn[c], pr, counts.cpu().numpy(), rays, nz, pr["mu"])
        assert abs(ll[c].item() - ref) <= 1e-6 * abs(ref)
    O = torch.zeros((1, w.S * w.P), dtype=torch.float64, device=DEV)
    with pytest.raises(mt.MtError):
        ctx.ray_terms(H0[:1].contiguous(), O)
    ctx.set_forward(mt.FORWARD_MARCH)                    # back to the march: chains re-usable
    ctx.run(mt.KERNEL_RW, 0.05, 1, 1)
    ctx.sync(60.0)
    ctx.close()


def test_linear_model_with_the_copula_prior():
    """Both switches together: latents -> heights -> linearised likelihood;
    setting the prior after the forward model keeps the model's buffers."""
    from oracle import copula as K
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64)
    nz = 30
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    ctx.set_prior(mt.PRIOR_COPULA)
    rng = np.random.default_rng(6)
    lat = 0.3 * rng.standard_normal((2, w.L, w.R, w.Q))
    lat[:, w.L - 1] = 0.0
    lat[:, w.L - 1, 0, :w.L - 1] = 0.8
    Lt = torch.tensor(lat, dtype=torch.float64, device=DEV).contiguous()
    ll = torch.zeros(2, dtype=torch.float64, device=DEV)
    ctx.logpost(Lt, ll, None)
    torch.cuda.synchronize()
    rays = LN.lengths(pr, nz)
    for c in range(2):
        H = K.heights(lat[c], pr["mu"][w.L - 1])
        ref = LN.loglik(H, pr, counts.cpu().numpy(), rays, nz, pr["mu"])
        assert abs(ll[c].item() - ref) <= 1e-9 * abs(ref)
    ctx.close()


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_linear_odd_grid_and_hard_indicator(gamma):
    """A 5 x 7 grid, 2 surfaces, downward-looking pixels included, odd n_z;
    the hard indicator (eta, gamma = 0) and the smooth one."""
    w = W.small(R=5, Q=7, n_sensors=3, n_zenith=6, n_azimuth=7, G=20, zenith_max_deg=120.0,
                gamma=gamma)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F64, gamma=gamma)
    nz = 17
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    Hs = np.concatenate([pr["mu"][None], W.init_chains(w, 3)])
    H = torch.tensor(Hs, dtype=torch.float64, device=DEV).contiguous()
    ll = torch.zeros(4, dtype=torch.float64, device=DEV)
    ctx.logpost(H, ll, None)
    torch.cuda.synchronize()
    rays = LN.lengths(pr, nz)
    for c in range(4):
        ref = LN.loglik(Hs[c], pr, counts.cpu().numpy(), rays, nz, pr["mu"])
        if math.isinf(ref):
            assert ll[c].item() == -math.inf
        else:
            assert abs(ll[c].item() - ref) <= 1e-10 * abs(ref) + 1e-9, (c, ll[c].item(), ref)
    ctx.close()


def test_linear_gradient_matches_oracle():
    """mt_grad under the linearised model: the chain rule through the path
    lengths and the cell-centre sigmoids (oracle loglik_grad, pinned by
    central differences) plus the CAR prior's gradient, within 1e-3 of the
    largest component (FP32)."""
    w = W.small(R=6, Q=5, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), G=48,
                n_zenith=9, n_azimuth=13, n_sensors=3)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    nz = 20
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    Hs = np.stack([W.perturbed(pr["H_true"], 1.0, [4]), W.init_chains(w, 1)[0]])
    H = torch.tensor(Hs, dtype=torch.float32, device=DEV).contiguous()
    g = torch.zeros(H.shape, dtype=torch.float64, device=DEV)
    lp = torch.zeros(2, dtype=torch.float64, device=DEV)
    ctx.grad(H, g, lp)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    Hn = H.double().cpu().numpy()
    rays = LN.lengths(pr, nz)
    C = counts.cpu().numpy()
    for c in range(2):
        ref = LN.loglik_grad(Hn[c], pr, C, rays, nz, pr["mu"]) + op.grad_logprior(Hn[c])
        scale = np.abs(ref).max()
        assert np.max(np.abs(g[c] - ref)) <= 1e-3 * scale, (c, np.max(np.abs(g[c] - ref)), scale)
        ref_lp = LN.loglik(Hn[c], pr, C, rays, nz, pr["mu"]) + op.logprior(Hn[c])
        assert abs(lp[c].item() - ref_lp) <= 1e-6 * abs(ref_lp) + 1e-3
    ctx.close()


def test_paper_pipeline_copula_linear_nuts():
    """The paper's combination: copula-prior latents, the linearised model and
    capped NUTS.  The latent gradient against the oracle's (heights_vjp of
    the linearised model's gradient, plus -z), then NUTS iterations whose
    states' log-likelihoods match the oracle's."""
    from oracle import copula as K
    w = W.small(R=5, Q=7, bases=(40.0, 75.0), G=24, n_zenith=6, n_azimuth=7, n_chains=3)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    nz = 16
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    ctx.set_prior(mt.PRIOR_COPULA)
    rng = np.random.default_rng(12)
    lat = 0.4 * rng.standard_normal((3, w.L, w.R, w.Q))
    lat[:, w.L - 1] = 0.0
    lat[:, w.L - 1, 0, :w.L - 1] = 0.55
    Lt = torch.tensor(lat, dtype=torch.float32, device=DEV).contiguous()
    g = torch.zeros(Lt.shape, dtype=torch.float64, device=DEV)
    ctx.grad(Lt, g)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    T = pr["mu"][w.L - 1]
    rays = LN.lengths(pr, nz)
    C = counts.cpu().numpy()
    Ln = Lt.double().cpu().numpy()
    for c in range(3):
        Hh = K.heights(Ln[c], T)
        ref = K.heights_vjp(Ln[c], T, LN.loglik_grad(Hh, pr, C, rays, nz, pr["mu"])) + K.logprior_grad(Ln[c])
        scale = np.abs(ref).max()
        assert np.max(np.abs(g[c] - ref)) <= 1e-3 * scale, (c, np.max(np.abs(g[c] - ref)), scale)
    ctx.set_nuts(2)
    ctx.init_chains(Lt, 5)
    ctx.run(mt.KERNEL_NUTS, 0.02, 3, 1)
    st = torch.zeros_like(Lt)
    ll = torch.zeros(3, dtype=torch.float64, device=DEV)
    acc = torch.zeros(3, dtype=torch.int64, device=DEV)
    ctx.get_state(st, ll, None, acc)
    S = st.double().cpu().numpy()
    for c in range(3):
        ref = LN.loglik(K.heights(S[c], T), pr, C, rays, nz, pr["mu"])
        assert abs(ll[c].item() - ref) <= 1e-6 * abs(ref) + 1e-3, (c, ll[c].item(), ref)
    assert acc.sum().item() > 0
    ctx.close()
