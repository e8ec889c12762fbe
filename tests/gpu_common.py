"""Shared set-up for the GPU parity tests: one workload -> (library context, oracle problem).

Counts come from the library (mt_generate_data); every test that uses them also
relies on test_counts_bit_exact, which checks them against the oracle's own
draws.  Heights handed to the oracle are the exact FP64 widening of what the
library holds.
"""
import numpy as np
import torch

import oracle
from paper_2603_28907_gb300 import mt, workloads as W

DEV = "cuda:0"


def torch_dtype(precision):
    return torch.float64 if precision == mt.PREC_F64 else torch.float32


def setup(w, precision=mt.PREC_F64, gamma=None, count_mode=mt.COUNTS_POISSON, **over):
    pr = W.problem(w)
    if gamma is not None:
        pr["gamma"] = gamma
    ctx = mt.from_workload(pr, precision=precision, **over)
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=DEV)
    lam = torch.zeros((w.S, w.P), dtype=torch.float64, device=DEV)
    ctx.generate_data(pr["H_true"], w.seed_data, count_mode, counts_out=counts, lambda_out=lam)
    ctx.sync(60.0)
    for k, v in over.items():
        if k == "n_grid":
            pr["G"] = v
        elif k == "atten":
            pr["Lambda"] = v
        elif k == "min_thick":
            pr["delta"] = v
        else:
            pr[k] = v
    op = oracle.OracleProblem(pr, counts=counts.cpu().numpy())
    return pr, ctx, op, counts, lam


def heights(arr, precision):
    return torch.tensor(np.asarray(arr), dtype=torch_dtype(precision), device=DEV).contiguous()


def logpost(ctx, H):
    n = H.shape[0]
    ll = torch.zeros(n, dtype=torch.float64, device=DEV)
    lp = torch.zeros(n, dtype=torch.float64, device=DEV)
    ctx.logpost(H, ll, lp)
    torch.cuda.synchronize()
    return ll.cpu().numpy(), lp.cpu().numpy()
