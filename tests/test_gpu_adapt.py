"""Step-size adaptation of the gradient samplers (dual averaging toward a
target acceptance probability, Sec. 3.1) on the GPU against the oracle
(oracle/adapt.py, oracle/hmc.py and the oracle's MALA).

Per step: the proposal against the oracle's with the chain's own step size
(so each chain really runs with its adapted eps), the GPU's acceptance
probability against the oracle's (the FP32 log-posterior and gradient error
bound the difference), and the GPU's next step size against the oracle's
dual averaging fed with the GPU's acceptance probabilities (FP64, 1e-12).
After n_adapt steps the step sizes stay fixed.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import adapt as A
from oracle import hmc
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, setup

pytestmark = pytest.mark.gpu


def _buffers(H0, C):
    prop = torch.zeros_like(H0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    return (prop, llp, torch.zeros_like(llp), torch.zeros(C, dtype=torch.int32, device=DEV),
            torch.zeros_like(llp))


def test_hmc_adapt_lockstep():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C, eps0, n_leap, n_adapt, n_steps = w.n_chains, 0.002, 4, 5, 8
    ctx.set_hmc(n_leap)
    ctx.set_adapt(0.8, n_adapt)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, w.seed_mcmc)
    with pytest.raises(mt.MtError):                      # nothing adapted yet
        ctx.get_adapt(torch.zeros(C, dtype=torch.float64, device=DEV))
    cur = H0.double().cpu().numpy()
    prop, llp, lpp, acc, logu = _buffers(H0, C)
    eps_t = torch.zeros(C, dtype=torch.float64, device=DEV)
    alpha_t = torch.zeros_like(eps_t)
    das = [A.DualAveraging(eps0, 0.8, n_adapt) for _ in range(C)]
    eps_used = np.full(C, eps0)
    logpi = lambda H: op.loglik(H) + op.logprior(H)
    lp_cur = np.array([logpi(cur[c]) for c in range(C)])
    history = []
    for k in range(n_steps):
        ctx.run(mt.KERNEL_HMC, eps0, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        ctx.get_adapt(eps_t, alpha_t)
        P = prop.double().cpu().numpy()
        a_gpu, eps_next, alpha = acc.cpu().numpy(), eps_t.cpu().numpy(), alpha_t.cpu().numpy()
        for c in range(C):
            q, dk = hmc.propose(op, cur[c], eps_used[c], n_leap, w.seed_mcmc, c, k, state=np.float32)
            assert np.max(np.abs(P[c] - q)) <= 1e-4, (k, c, np.max(np.abs(P[c] - q)))
            lpn = op.logprior(P[c])
            lq = logpi(P[c]) if np.isfinite(lpn) else -np.inf
            a_ref = A.accept_prob(lq - lp_cur[c] + dk, bool(np.isfinite(lq)))
            assert abs(alpha[c] - a_ref) <= 5e-2, (k, c, alpha[c], a_ref)
            ref = das[c].update(float(alpha[c]))
            assert abs(eps_next[c] - ref) <= 1e-12 * ref, (k, c, eps_next[c], ref)
            if a_gpu[c]:
                cur[c] = P[c]
                lp_cur[c] = lq
        history.append(eps_next.copy())
        eps_used = eps_next
    # frozen after n_adapt steps, at each chain's averaged step size
    for k in range(n_adapt, n_steps):
        np.testing.assert_array_equal(history[k], history[n_adapt - 1])
    assert np.all(history[-1] != eps0)
    ctx.close()


def test_mala_adapt_lockstep():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C, eps0, n_adapt = w.n_chains, 0.004, 6
    ctx.set_adapt(0.574, n_adapt)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, 9)
    cur = H0.double().cpu().numpy()
    prop, llp, lpp, acc, logu = _buffers(H0, C)
    eps_t = torch.zeros(C, dtype=torch.float64, device=DEV)
    alpha_t = torch.zeros_like(eps_t)
    das = [A.DualAveraging(eps0, 0.574, n_adapt) for _ in range(C)]
    eps_used = np.full(C, eps0)
    for k in range(n_adapt + 2):
        gcur = torch.zeros(H0.shape, dtype=torch.float64, device=DEV)
        ctx.grad(torch.tensor(cur, dtype=torch.float32, device=DEV).contiguous(), gcur)
        gcur = gcur.cpu().numpy()
        ctx.run(mt.KERNEL_MALA, eps0, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        ctx.get_adapt(eps_t, alpha_t)
        P = prop.double().cpu().numpy()
        gp = torch.zeros(H0.shape, dtype=torch.float64, device=DEV)
        ctx.grad(prop, gp)
        gp = gp.cpu().numpy()
        eps_next, alpha = eps_t.cpu().numpy(), alpha_t.cpu().numpy()
        for c in range(C):
            e = eps_used[c]
            xi = oracle.normals(9, oracle.STREAM["MALA"], c, k, cur[c].size).reshape(cur[c].shape)
            expect = cur[c] + 0.5 * e * e * gcur[c] + e * xi
            assert np.max(np.abs(P[c] - expect)) <= 1.6e-5, (k, c, np.max(np.abs(P[c] - expect)))
            lpn = op.logprior(P[c])
            delta = -np.inf
            if np.isfinite(lpn):
                hast = op.mala_logq(cur[c], P[c], gp[c], e) - op.mala_logq(P[c], cur[c], gcur[c], e)
                delta = (op.loglik(P[c]) + lpn) - (op.loglik(cur[c]) + op.logprior(cur[c])) + hast
            a_ref = A.accept_prob(delta, bool(np.isfinite(lpn)))
            assert abs(alpha[c] - a_ref) <= 1e-2, (k, c, alpha[c], a_ref)
            ref = das[c].update(float(alpha[c]))
            assert abs(eps_next[c] - ref) <= 1e-12 * ref, (k, c, eps_next[c], ref)
            if acc[c].item():
                cur[c] = P[c]
        eps_used = eps_next
    ctx.close()


def test_adapt_settings_and_restart():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C = w.n_chains
    for bad in ((0.0, 5), (1.0, 5), (0.8, -1)):
        with pytest.raises(mt.MtError):
            ctx.set_adapt(*bad)
    ctx.set_hmc(2)
    ctx.set_adapt(0.8, 3)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, 3)
    ctx.run(mt.KERNEL_RW, 0.02, 1, 2)                    # random-walk steps: no adaptation
    with pytest.raises(mt.MtError):
        ctx.get_adapt(torch.zeros(C, dtype=torch.float64, device=DEV))
    ctx.run(mt.KERNEL_HMC, 0.003, 1, 1)
    e1, a1 = np.zeros(C), np.zeros(C)                    # host outputs
    ctx.get_adapt(e1, a1)
    for c in range(C):
        assert e1[c] == pytest.approx(A.DualAveraging(0.003, 0.8, 3).update(a1[c]), rel=1e-12)
    # new chains start over from the next run's step size
    ctx.init_chains(H0, 4)
    with pytest.raises(mt.MtError):
        ctx.get_adapt(e1)
    ctx.run(mt.KERNEL_HMC, 0.001, 1, 1)
    ctx.get_adapt(e1, a1)
    for c in range(C):
        assert e1[c] == pytest.approx(A.DualAveraging(0.001, 0.8, 3).update(a1[c]), rel=1e-12)
    # off again: the scalar step size, and nothing to report
    ctx.set_adapt(0.8, 0)
    ctx.run(mt.KERNEL_HMC, 0.001, 1, 1)
    with pytest.raises(mt.MtError):
        ctx.get_adapt(e1)
    ctx.sync(60.0)
    ctx.close()


def test_hmc_metric_warmup_lockstep():
    """Windowed warm-up of the step size and a diagonal inverse metric (HMC):
    each step's proposal against the oracle's with the chain's own eps and
    metric, the acceptance probability within the FP32 band, and the next eps
    and metric against the oracle's warm-up fed with the GPU's acceptance
    probabilities and post-step states (metric: FP64 Welford on the same FP32
    states, 1e-9 relative).  The metric changes once, at the end of the only
    slow window of a 40-step warm-up (steps 6 .. 35), and stays fixed after."""
    w = W.small(R=5, Q=7, bases=(40.0, 75.0), G=24, n_zenith=6, n_azimuth=7, n_chains=2)
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C, eps0, n_leap, Wn, shrink = 2, 0.002, 2, 40, 1e-6
    ctx.set_hmc(n_leap)
    ctx.set_adapt(0.8, Wn)
    ctx.set_metric_adapt(1, shrink)
    H0 = torch.tensor(W.init_chains(w, C), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, 21)
    minv_t = torch.zeros((C,) + tuple(H0.shape[1:]), dtype=torch.float64, device=DEV)
    with pytest.raises(mt.MtError):
        ctx.get_metric(minv_t)
    cur = H0.double().cpu().numpy()
    prop, llp, lpp, acc, logu = _buffers(H0, C)
    eps_t = torch.zeros(C, dtype=torch.float64, device=DEV)
    alpha_t = torch.zeros_like(eps_t)
    st = torch.zeros_like(H0)
    wus = [A.Warmup(eps0, 0.8, Wn, cur[c].shape, shrink) for c in range(C)]
    eps_used, minv_used = np.full(C, eps0), np.ones(cur.shape)
    logpi = lambda H: op.loglik(H) + op.logprior(H)
    lp_cur = np.array([logpi(cur[c]) for c in range(C)])
    band = 0
    for k in range(Wn + 3):
        ctx.run(mt.KERNEL_HMC, eps0, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        ctx.get_adapt(eps_t, alpha_t)
        ctx.get_metric(minv_t)
        ctx.get_state(st)
        P, S = prop.double().cpu().numpy(), st.double().cpu().numpy()
        eps_next, alpha, minv = eps_t.cpu().numpy(), alpha_t.cpu().numpy(), minv_t.cpu().numpy()
        for c in range(C):
            q, dk = hmc.propose(op, cur[c], eps_used[c], n_leap, 21, c, k, state=np.float32,
                                inv_metric=minv_used[c])
            # the FP32 gradients' error moves the trajectory in proportion to
            # its length (the adapted eps and metric can make steps of metres)
            disp = float(np.max(np.abs(q - cur[c])))
            err = float(np.max(np.abs(P[c] - q)))
            assert err <= 1e-4 + 1e-4 * disp, (k, c, err, disp, eps_used[c])
            lq = logpi(P[c]) if np.isfinite(op.logprior(P[c])) else -np.inf
            a_ref = A.accept_prob(lq - lp_cur[c] + dk, bool(np.isfinite(lq)))
            band += abs(alpha[c] - a_ref) > 1e-3
            assert abs(alpha[c] - a_ref) <= 5e-2, (k, c, alpha[c], a_ref)
            ref = wus[c].update(float(alpha[c]), S[c])
            assert abs(eps_next[c] - ref) <= 1e-12 * ref, (k, c, eps_next[c], ref)
            np.testing.assert_allclose(minv[c], wus[c].inv_metric, rtol=1e-9, atol=0)
            if acc[c].item():
                lp_cur[c] = lq
            cur[c] = S[c]
        if k < 35:
            assert np.all(minv == 1.0)
        eps_used, minv_used = eps_next, minv
    assert not np.all(minv_used == 1.0)
    ctx.close()


def test_metric_settings():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    for bad in ((2, 1e-3), (1, -1.0)):
        with pytest.raises(mt.MtError):
            ctx.set_metric_adapt(*bad)
    ctx.set_adapt(0.8, 10)
    ctx.set_metric_adapt(1)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, 3)
    with pytest.raises(mt.MtError):                      # fewer than 20 warm-up steps
        ctx.run(mt.KERNEL_HMC, 0.002, 1, 1)
    ctx.set_adapt(0.8, 30)
    with pytest.raises(mt.MtError):                      # the metric is for HMC
        ctx.run(mt.KERNEL_MALA, 0.002, 1, 1)
    ctx.set_hmc(1)
    ctx.run(mt.KERNEL_HMC, 0.002, 1, 1)
    m = np.zeros((w.n_chains, w.L, w.R, w.Q))
    ctx.get_metric(m)
    assert np.all(m == 1.0)                              # still in the initial buffer
    ctx.set_metric_adapt(0)
    ctx.run(mt.KERNEL_HMC, 0.002, 1, 1)
    with pytest.raises(mt.MtError):
        ctx.get_metric(m)
    ctx.sync(60.0)
    ctx.close()
