"""mt_logpost_noalloc: the allocation-free log-posterior call, checked against mt_logpost.

Some callers cannot let a library allocate device memory: hosts that hand out
all GPU memory through their own fixed-budget allocator, and latency-critical
serving loops in which a cudaMalloc / cudaFree (which synchronises the device)
must not happen after start-up.  mt_logpost_noalloc serves them by keeping its
scratch (the per-block partial sums of the ray kernel) in a fixed array inside
the library.  Two calls in a row must each reproduce mt_logpost, whatever the
shared array held before.  This file sorts last so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, heights, logpost, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F64])
def test_noalloc_matches_logpost_on_two_calls(precision):
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=precision)
    batches = [np.concatenate([pr["H_true"][None], W.init_chains(w, 3)]),
               W.init_chains(w, 2) + 0.5]            # a different size and content second
    for Hs in batches:
        H = heights(Hs, precision)
        ll_ref, lp_ref = logpost(ctx, H)
        ll = torch.full((H.shape[0],), float("nan"), dtype=torch.float64, device=DEV)
        lp = torch.full_like(ll, float("nan"))
        ctx.logpost_noalloc(H, ll, lp)
        torch.cuda.synchronize()
        # the tolerance the FP32 parity tests use for a per-chain log-likelihood
        np.testing.assert_allclose(ll.cpu().numpy(), ll_ref, rtol=0, atol=1e-3)
        np.testing.assert_allclose(lp.cpu().numpy(), lp_ref, rtol=1e-12)


def test_noalloc_rejects_host_memory_and_oversize():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    Hh = W.init_chains(w, 2).astype(np.float32)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    with pytest.raises(mt.MtError) as e:
        ctx.logpost_noalloc(Hh, out)                 # host heights: staging would allocate
    assert e.value.status == -1
    lib = mt.load()
    w2 = W.scenario()
    w2.n_zenith, w2.n_azimuth = 64, 64
    pr2 = W.problem(w2)
    ctx2 = mt.from_workload(pr2, precision=mt.PREC_F32)
    ctx2.set_counts(np.ones((w2.S, w2.P), np.int32))
    # 65536 rays -> 8 partials per chain (8192 rays per block): 16384 chains
    # fit, 16385 do not.  The arrays are sized for 16385 chains so the call
    # stays in bounds either way.
    Hbig = heights(pr2["H_true"][None], mt.PREC_F32).expand(16385, -1, -1, -1).contiguous()
    obig = torch.zeros(16385, dtype=torch.float64, device=DEV)
    st = lib.mt_logpost_noalloc(ctx2.h, 16385, ctypes.c_void_p(Hbig.data_ptr()),
                                ctypes.c_void_p(obig.data_ptr()), None)
    assert st == -1
    assert b"1048576" in lib.mt_last_error(ctx2.h)
    H2 = Hbig[:1].contiguous()
    o2 = torch.zeros(1, dtype=torch.float64, device=DEV)
    ctx2.logpost_noalloc(H2, o2)                      # one chain is fine
    torch.cuda.synchronize()
    ll_ref, _ = logpost(ctx2, H2)
    assert abs(o2.item() - ll_ref[0]) <= 1e-3
