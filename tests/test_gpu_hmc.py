"""Hamiltonian Monte Carlo (leapfrog trajectories driven by the adjoint) in
lockstep with the FP64 oracle's HMC (oracle/hmc.py; Sec. 3.1).

Per step: the GPU's proposal against the oracle's leapfrog from the same
state and Philox momentum (FP32 heights: within a few FP32 ulps of ~100 m),
and the accept decision against the oracle's, allowing a band for the FP32
log-likelihood and gradient error; the chain state follows the GPU's
decisions.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import hmc
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, setup

pytestmark = pytest.mark.gpu


def test_hmc_lockstep_f32():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    C, eps, n_leap, n_steps = w.n_chains, 0.002, 4, 8
    ctx.set_hmc(n_leap)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, w.seed_mcmc)
    cur = H0.double().cpu().numpy()
    prop = torch.zeros_like(H0)
    llp = torch.zeros(C, dtype=torch.float64, device=DEV)
    lpp, logu = torch.zeros_like(llp), torch.zeros_like(llp)
    acc = torch.zeros(C, dtype=torch.int32, device=DEV)
    st = torch.zeros_like(H0)
    logpi = lambda H: op.loglik(H) + op.logprior(H)
    lp_cur = np.array([logpi(cur[c]) for c in range(C)])
    stats = dict(match=0, band=0, accepted=0, max_dq=0.0)
    for k in range(n_steps):
        ctx.run(mt.KERNEL_HMC, eps, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        P = prop.double().cpu().numpy()
        a_gpu, lu = acc.cpu().numpy(), logu.cpu().numpy()
        for c in range(C):
            q, dk = hmc.propose(op, cur[c], eps, n_leap, w.seed_mcmc, c, k, state=np.float32)
            stats["max_dq"] = max(stats["max_dq"], float(np.max(np.abs(P[c] - q))))
            assert np.max(np.abs(P[c] - q)) <= 1e-4, (k, c, np.max(np.abs(P[c] - q)))
            lpn = op.logprior(P[c])
            lq = logpi(P[c]) if np.isfinite(lpn) else -np.inf
            delta = lq - lp_cur[c] + dk
            a_ref = bool(np.isfinite(lq) and lu[c] < delta)
            if bool(a_gpu[c]) == a_ref:
                stats["match"] += 1
            else:
                assert abs(lu[c] - delta) < 5e-2, (k, c, lu[c], delta)
                stats["band"] += 1
            if a_gpu[c]:
                cur[c] = P[c]
                lp_cur[c] = lq
                stats["accepted"] += 1
        ctx.get_state(st)
        np.testing.assert_array_equal(st.double().cpu().numpy(), cur)
    assert stats["accepted"] > 0, stats
    assert stats["band"] <= 1, stats
    ctx.close()


def test_hmc_rejects_bad_settings():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    with pytest.raises(mt.MtError):
        ctx.set_hmc(0)
    H0 = torch.tensor(W.init_chains(w), dtype=torch.float32, device=DEV).contiguous()
    ctx.init_chains(H0, 1)
    with pytest.raises(mt.MtError):
        ctx.run(mt.KERNEL_HMC, 0.0, 1, 1)                 # eps must be > 0
    ctx.close()
    w64 = W.tiny()
    pr, c64, op, counts, _ = setup(w64, precision=mt.PREC_F64)
    c64.init_chains(torch.tensor(W.init_chains(w64), dtype=torch.float64, device=DEV), 1)
    with pytest.raises(mt.MtError):
        c64.run(mt.KERNEL_HMC, 0.01, 1, 1)               # the adjoint needs an FP32 mode
    c64.close()
