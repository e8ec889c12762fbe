"""Capped NUTS (the trajectory NUTS builds when it runs to its cap, Sec. 3.1)
on the GPU in lockstep with the FP64 oracle (oracle/nuts.py).

Per iteration and chain: the oracle builds the same trajectory from the
GPU's current state with the same Philox momenta, directions and uniforms;
where none of its decisions came within the FP32 log-density error of
flipping, the GPU's new state must be the oracle's sample (to the FP32
trajectory error), and the acceptance statistic the step-size adaptation
uses must match.  The chains then continue from the GPU's states.
"""
import numpy as np
import pytest
import torch

from oracle import adapt as A
from oracle import nuts as NU
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, setup

pytestmark = pytest.mark.gpu

# |log u - threshold| below which an FP32 decision may differ: the thresholds
# are energy differences between nearby states, whose FP32 error (the
# per-chain log-likelihood bias is shared between them) is ~1e-4
BAND = 0.01


def _lockstep(w, depth, eps, n_iter, seed, adapt=0, metric=False):
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C = w.n_chains
    ctx.set_nuts(depth)
    if adapt:
        ctx.set_adapt(0.8, adapt)
        ctx.set_metric_adapt(1 if metric else 0, 1e-6)
    H0 = torch.tensor(W.init_chains(w, C), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, seed)
    cur = H0.double().cpu().numpy()
    st = torch.zeros_like(H0)
    prop = torch.zeros_like(H0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    lpp, logu = torch.zeros_like(llp), torch.zeros_like(llp)
    acc = torch.zeros(C, dtype=torch.int32, device=DEV)
    eps_t, alpha_t = torch.zeros_like(llp), torch.zeros_like(llp)
    logpi = lambda q: (op.loglik(q), op.logprior(q))
    grad = lambda q: op.grad_loglik(q) + op.grad_logprior(q)
    das = [A.DualAveraging(eps, 0.8, adapt) for _ in range(C)] if adapt and not metric else None
    eps_used = np.full(C, eps)
    stats = dict(checked=0, near=0, moved=0)
    for k in range(n_iter):
        ctx.run(mt.KERNEL_NUTS, eps, 1, 1)
        ctx.get_state(st)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        S, P = st.double().cpu().numpy(), prop.double().cpu().numpy()
        np.testing.assert_array_equal(S, P)          # the proposal is the new state
        if adapt:
            ctx.get_adapt(eps_t, alpha_t)
        for c in range(C):
            ll0, lp0 = logpi(cur[c])
            q, ll, lp, g, stat, margin = NU.iteration(logpi, grad, cur[c], ll0, lp0, grad(cur[c]), eps_used[c],
                                                      depth, seed, c, k, state=np.float32)
            moved = bool(np.any(S[c] != cur[c]))
            assert bool(acc[c].item()) == moved
            stats["moved"] += moved
            if margin > BAND:
                disp = float(np.max(np.abs(q - cur[c])))
                err = float(np.max(np.abs(S[c] - q)))
                assert err <= 1e-4 + 1e-4 * disp, (k, c, err, disp, margin)
                assert abs(llp[c].item() - ll) <= 1e-3 * max(1.0, abs(ll) * 1e-3) + 5e-3
                stats["checked"] += 1
            else:
                stats["near"] += 1
            if adapt:
                assert abs(alpha_t[c].item() - stat) <= 5e-2, (k, c, alpha_t[c].item(), stat)
                if das is not None:
                    ref = das[c].update(float(alpha_t[c].item()))
                    assert abs(eps_t[c].item() - ref) <= 1e-12 * ref
        if adapt:
            eps_used = eps_t.cpu().numpy().copy()
        cur = S
    ctx.close()
    return stats


def test_nuts_lockstep_depth3():
    stats = _lockstep(W.tiny(), depth=3, eps=0.002, n_iter=5, seed=31)
    assert stats["checked"] >= 15 and stats["near"] <= 5, stats
    assert stats["moved"] > 0, stats


def test_nuts_lockstep_with_step_size_adaptation():
    w = W.small(R=5, Q=7, bases=(40.0, 75.0), G=24, n_zenith=6, n_azimuth=7, n_chains=3)
    stats = _lockstep(w, depth=2, eps=0.003, n_iter=8, seed=32, adapt=5)
    assert stats["checked"] >= 18 and stats["near"] <= 6, stats


def test_nuts_settings():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    for bad in (0, 11):
        with pytest.raises(mt.MtError):
            ctx.set_nuts(bad)
    ctx.set_nuts(1)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, 3)
    with pytest.raises(mt.MtError):
        ctx.run(mt.KERNEL_NUTS, 0.0, 1, 1)              # eps must be > 0
    ctx.run(mt.KERNEL_NUTS, 0.002, 1, 2)
    ctx.run(mt.KERNEL_RW, 0.01, 1, 1)                   # gradients refreshed after RW steps
    ctx.run(mt.KERNEL_NUTS, 0.002, 1, 1)
    ctx.sync(60.0)
    ctx.close()
