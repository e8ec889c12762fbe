"""Adjoint gradient, autograd wrapper and MALA against the FP64 oracle.

Tolerances: the GPU gradient is FP32 march arithmetic accumulated in 64-bit
fixed point (2^-24) and FP64; it must match the oracle's analytic FP64 gradient
(itself pinned by central differences) within 1e-5 of the largest component
(measured: a few 1e-7 at the scenario size), and be bit-identical from call to
call.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_28907_gb300 import autograd as AG
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, heights, logpost, setup
from tests.test_gpu_parity import fp32_loglik_tol

pytestmark = pytest.mark.gpu

CASES = [
    W.small(R=5, Q=6, bases=(40.0, 75.0), G=32, n_zenith=6, n_azimuth=7),
    W.small(R=6, Q=5, bases=(40.0, 70.0, 110.0), rho=(2.65, 1.9, 0.0012, 2.65), G=48,
            n_zenith=9, n_azimuth=13, n_sensors=3),
    W.tiny(),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_grad_matches_oracle(w):
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    Hs = np.stack([W.perturbed(pr["H_true"], 1.0, [4]), W.init_chains(w, 1)[0]])
    H = heights(Hs, mt.PREC_F32)
    g = torch.zeros(H.shape, dtype=torch.float64, device=DEV)
    lp = torch.zeros(2, dtype=torch.float64, device=DEV)
    ctx.grad(H, g, lp)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    Hn = H.double().cpu().numpy()
    for c in range(2):
        ref = op.grad_loglik(Hn[c]) + op.grad_logprior(Hn[c])
        scale = np.abs(ref).max()
        assert np.max(np.abs(g[c] - ref)) <= 1e-5 * scale, (c, np.max(np.abs(g[c] - ref)), scale)
        ref_lp = op.loglik(Hn[c]) + op.logprior(Hn[c])
        assert abs(lp[c].item() - ref_lp) <= 1e-3 * max(1.0, abs(ref_lp) * 1e-3)


def test_grad_central_differences_on_gpu():
    """Gradient against central differences (h = 1e-3 m) of the library's FP64 log-posterior."""
    w = CASES[0]
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    ctx64 = mt.from_workload(pr, precision=mt.PREC_F64)
    ctx64.set_counts(counts)
    H = W.perturbed(pr["H_true"], 1.0, [4]).astype(np.float32).astype(np.float64)
    g = torch.zeros((1,) + H.shape, dtype=torch.float64, device=DEV)
    ctx.grad(heights(H[None], mt.PREC_F32), g)
    g = g[0].cpu().numpy()
    rng = np.random.default_rng(1)
    idx = [np.unravel_index(i, H.shape) for i in rng.choice(H.size, 12, replace=False)]
    Hp = np.stack([H] * (2 * len(idx)))
    for j, ix in enumerate(idx):
        Hp[2 * j][ix] += 1e-3
        Hp[2 * j + 1][ix] -= 1e-3
    ll, lp = logpost(ctx64, heights(Hp, mt.PREC_F64))
    f = ll + lp
    for j, ix in enumerate(idx):
        fd = (f[2 * j] - f[2 * j + 1]) / 2e-3
        assert g[ix] == pytest.approx(fd, rel=2e-3, abs=2e-3 * np.abs(g).max()), (ix, g[ix], fd)


def test_grad_bit_reproducible():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    H = heights(W.init_chains(w, 3), mt.PREC_F32)
    outs = []
    for _ in range(2):
        g = torch.zeros(H.shape, dtype=torch.float64, device=DEV)
        ctx.grad(H, g)
        outs.append(g.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


def test_autograd_function():
    w = CASES[1]
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    H = heights(W.init_chains(w, 2), mt.PREC_F32).requires_grad_(True)
    lp = AG.logpost(H, ctx)
    wts = torch.tensor([0.7, -1.3], dtype=torch.float64, device=DEV)
    (lp * wts).sum().backward()
    g = torch.zeros(H.shape, dtype=torch.float64, device=DEV)
    ctx.grad(H.detach(), g)
    expect = (wts.view(-1, 1, 1, 1) * g).float()
    torch.testing.assert_close(H.grad, expect, rtol=1e-6, atol=1e-6)
    ll_ref, lp_ref = logpost(ctx, H.detach())
    np.testing.assert_allclose(lp.detach().cpu().numpy(), ll_ref + lp_ref, rtol=0, atol=1e-3)


def test_mala_lockstep():
    """Each MALA step: proposal = H + (eps^2/2) g + eps xi with the oracle's normals,
    Hastings term and accept decision recomputed by the oracle."""
    w = W.tiny()
    eps = 0.01
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C = w.n_chains
    H0 = heights(W.init_chains(w), mt.PREC_F32)
    ctx.init_chains(H0, 9)
    cur = H0.double().cpu().numpy()
    prop = torch.zeros_like(H0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    lpp = torch.zeros_like(llp)
    acc = torch.zeros(C, dtype=torch.int32, device=DEV)
    logu = torch.zeros_like(llp)
    stats = dict(match=0, tie=0, mismatch=0, accepted=0)
    for k in range(25):
        gcur = torch.zeros(H0.shape, dtype=torch.float64, device=DEV)
        ctx.grad(heights(cur, mt.PREC_F32), gcur)
        gcur = gcur.cpu().numpy()
        ctx.run(mt.KERNEL_MALA, eps, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        P = prop.double().cpu().numpy()
        gp = torch.zeros(H0.shape, dtype=torch.float64, device=DEV)
        ctx.grad(prop, gp)
        gp = gp.cpu().numpy()
        for c in range(C):
            xi = oracle.normals(9, oracle.STREAM["MALA"], c, k, cur[c].size).reshape(cur[c].shape)
            expect = cur[c] + 0.5 * eps * eps * gcur[c] + eps * xi
            assert np.max(np.abs(P[c] - expect)) <= 1.6e-5, (k, c, np.max(np.abs(P[c] - expect)))
            lpn, lln = op.logprior(P[c]), op.loglik(P[c])
            lpo, llo = op.logprior(cur[c]), op.loglik(cur[c])
            hast = op.mala_logq(cur[c], P[c], gp[c], eps) - op.mala_logq(P[c], cur[c], gcur[c], eps)
            delta = (lln + lpn) - (llo + lpo) + hast
            a_ref = bool(np.isfinite(lpn) and logu[c].item() < delta)
            a_gpu = bool(acc[c].item())
            if a_gpu == a_ref:
                stats["match"] += 1
            elif abs(logu[c].item() - delta) < 3e-3:
                stats["tie"] += 1
            else:
                stats["mismatch"] += 1
            if a_gpu:
                cur[c] = P[c]
                stats["accepted"] += 1
    assert stats["mismatch"] == 0, stats
    assert stats["accepted"] > 0, stats


def test_grad_large_grid_global_paths():
    """A 100 x 100 grid with 4 surfaces: the march stages one surface's (h, dx)
    plane at a time and the adjoint adds straight into global fixed-point
    accumulators (its node records fit in shared memory, the accumulators do
    not); the gradient must still match the oracle's, and a MALA step runs on
    those paths."""
    w = W.small(R=100, Q=100, bases=(40.0, 70.0, 110.0, 140.0),
                rho=(2.65, 1.9, 0.0012, 2.65, 0.0012), G=64, n_zenith=6, n_azimuth=9,
                n_sensors=2)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    Hs = np.stack([W.perturbed(pr["H_true"], 1.0, [4]), W.init_chains(w, 1)[0]])
    H = heights(Hs, mt.PREC_F32)
    g = torch.zeros(H.shape, dtype=torch.float64, device=DEV)
    lp = torch.zeros(2, dtype=torch.float64, device=DEV)
    ctx.grad(H, g, lp)
    torch.cuda.synchronize()
    g = g.cpu().numpy()
    Hn = H.double().cpu().numpy()
    for c in range(2):
        ref = op.grad_loglik(Hn[c]) + op.grad_logprior(Hn[c])
        scale = np.abs(ref).max()
        assert np.max(np.abs(g[c] - ref)) <= 1e-5 * scale, (c, np.max(np.abs(g[c] - ref)), scale)
        ref_lp = op.loglik(Hn[c]) + op.logprior(Hn[c])
        if np.isinf(ref_lp):                             # a node above the box top
            assert lp[c].item() == ref_lp
        else:
            assert abs(lp[c].item() - ref_lp) <= fp32_loglik_tol(pr, op, Hn[c]) + 1e-9 * abs(ref_lp)
    H = heights(np.stack([W.init_chains(w, 2)[c] for c in range(2)]), mt.PREC_F32)
    ctx.init_chains(H, 5)
    ctx.run(mt.KERNEL_MALA, 0.005, 1, 2)
    ll = torch.zeros(2, dtype=torch.float64, device=DEV)
    Hs2 = torch.zeros_like(H)
    ctx.get_state(Hs2, ll)
    H2 = Hs2.double().cpu().numpy()
    for c in range(2):
        assert abs(ll[c].item() - op.loglik(H2[c])) <= fp32_loglik_tol(pr, op, H2[c])
