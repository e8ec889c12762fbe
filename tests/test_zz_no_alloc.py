"""mt_logpost_noalloc: the allocation-free log-posterior call, checked against mt_logpost.

Some callers cannot let a library allocate device memory: hosts that hand out
all GPU memory through their own fixed-budget allocator, and latency-critical
serving loops in which a cudaMalloc / cudaFree (which synchronises the device)
must not happen after start-up.  mt_logpost_noalloc serves them by keeping its
scratch (the per-block partial sums of the ray kernel) in a fixed array inside
the library.  It runs the same kernels in the same order as mt_logpost, so two
calls in a row must each reproduce mt_logpost bit for bit, in every precision
mode, whatever the shared array held before (the first batch is larger than
the second, so stale partials from it would show).  This file sorts last so a
run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, heights, logpost, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F32C, mt.PREC_F32A, mt.PREC_F64, mt.PREC_BF16])
def test_noalloc_matches_logpost_on_two_calls(precision):
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=precision)
    batches = [np.concatenate([pr["H_true"][None], W.init_chains(w, 5)]),
               W.init_chains(w, 2) + 0.5]            # smaller, different content second
    for Hs in batches:
        H = heights(Hs, precision)
        ll_ref, lp_ref = logpost(ctx, H)
        ll = torch.full((H.shape[0],), float("nan"), dtype=torch.float64, device=DEV)
        lp = torch.full_like(ll, float("nan"))
        ctx.logpost_noalloc(H, ll, lp)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ll.cpu().numpy(), ll_ref)
        np.testing.assert_array_equal(lp.cpu().numpy(), lp_ref)


def test_noalloc_rejects_host_memory_and_oversize():
    w = W.tiny()
    pr, ctx, op, counts, _ = setup(w, precision=mt.PREC_F32)
    lib = mt.load()
    Hh = np.ascontiguousarray(W.init_chains(w, 2).astype(np.float32))
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    # host heights: the library refuses them (staging would allocate)
    st = lib.mt_logpost_noalloc(ctx.h, 2, ctypes.c_void_p(Hh.ctypes.data), ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1
    assert b"device memory" in lib.mt_last_error(ctx.h)
    with pytest.raises(ValueError):
        ctx.logpost_noalloc(Hh, out)                 # and so does the binding, before calling it
    w2 = W.scenario()
    pr2 = W.problem(w2)
    ctx2 = mt.from_workload(pr2, precision=mt.PREC_F32)
    ctx2.set_counts(np.ones((w2.S, w2.P), np.int32))
    # 65536 rays -> 11 partials per chain (6144 ray slots per CTA), 88 bytes:
    # 11915 chains fit in 1 MiB, 11916 do not.  The arrays are sized for the
    # larger count so the call stays in bounds either way.
    n_blk = -(-w2.S * w2.P // 6144)
    n_max = (1 << 20) // (n_blk * 8)
    Hbig = heights(pr2["H_true"][None], mt.PREC_F32).expand(n_max + 1, -1, -1, -1).contiguous()
    obig = torch.zeros(n_max + 1, dtype=torch.float64, device=DEV)
    st = lib.mt_logpost_noalloc(ctx2.h, n_max + 1, ctypes.c_void_p(Hbig.data_ptr()),
                                ctypes.c_void_p(obig.data_ptr()), None)
    assert st == -1
    assert b"1048576" in lib.mt_last_error(ctx2.h)
    H2 = Hbig[:1].contiguous()
    o2 = torch.zeros(1, dtype=torch.float64, device=DEV)
    ctx2.logpost_noalloc(H2, o2)                      # one chain is fine
    torch.cuda.synchronize()
    ll_ref, _ = logpost(ctx2, H2)
    assert o2.item() == ll_ref[0]
