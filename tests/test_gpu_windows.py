"""The FP32 ray kernel's exact-saturation windows change no bit of the result.

Samples whose sigmoid argument lies at least 29.25 log2 units from zero add
exactly 0 or 2^28 units of 2^-28 (Sec. 2.1.1 opacity sum; Eq.
smooth_layer_indicators evaluated in FP32), so the kernel adds their integer
contributions without evaluating them.  These tests run the same data through a context with the windows (the
default) and one created with MT_FULL_WINDOWS=1 (every sample evaluated) and
require bit-identical per-ray opacities, terms and log-likelihoods, and that
the windows did skip work.
"""
import os

import numpy as np
import pytest
import torch

from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV

pytestmark = pytest.mark.gpu


def _ctx(pr, precision, full):
    old = os.environ.get("MT_FULL_WINDOWS")
    os.environ["MT_FULL_WINDOWS"] = "1" if full else "0"
    try:
        return mt.from_workload(pr, precision=precision)
    finally:
        if old is None:
            del os.environ["MT_FULL_WINDOWS"]
        else:
            os.environ["MT_FULL_WINDOWS"] = old


def _run(ctx, H, n_rays):
    n = H.shape[0]
    O = torch.zeros((n, n_rays), dtype=torch.float64, device=DEV)
    T = torch.zeros_like(O)
    ctx.ray_terms(H, O, T)
    ll = torch.zeros(n, dtype=torch.float64, device=DEV)
    ctx.set_timing(1)
    ctx.get_work(reset=True)
    ctx.logpost(H, ll, None)
    torch.cuda.synchronize()
    ev, tot = ctx.get_work(reset=True)
    ctx.set_timing(0)
    return O.cpu().numpy(), T.cpu().numpy(), ll.cpu().numpy(), ev, tot


def _downward():
    # zenith up to 125 deg: rays pointing down (full windows) and an odd G
    return W.small(R=9, Q=11, bases=(40.0, 75.0, 100.0), rho=(2.65, 1.9, 0.0012, 2.65),
                   n_sensors=3, n_zenith=12, n_azimuth=20, G=255, zenith_max_deg=125.0,
                   n_chains=6)


def _large():
    # 100 x 100 nodes and 4 surfaces: one surface's plane at a time
    return W.small(R=100, Q=100, bases=(40.0, 70.0, 110.0, 140.0), rho=(2.65, 1.9, 0.0012, 2.65, 0.0012),
                   G=64, n_zenith=6, n_azimuth=9, n_sensors=2, n_chains=6)


CASES = {
    "tiny_f32": (W.tiny, mt.PREC_F32, None),
    "tiny_f32c": (W.tiny, mt.PREC_F32C, None),
    "tiny_f32a": (W.tiny, mt.PREC_F32A, None),
    "tiny_hard": (W.tiny, mt.PREC_F32, 0.0),
    "downward_odd_g": (_downward, mt.PREC_F32, None),
    "large_phased": (_large, mt.PREC_F32, None),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_windows_bit_identical(case):
    make, prec, gamma = CASES[case]
    w = make()
    pr = W.problem(w)
    if gamma is not None:
        pr["gamma"] = gamma
    a = _ctx(pr, prec, full=False)
    b = _ctx(pr, prec, full=True)
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=DEV)
    a.generate_data(pr["H_true"], w.seed_data, mt.COUNTS_POISSON, counts_out=counts)
    a.sync(60.0)
    b.set_counts(counts.cpu().numpy())
    Hs = np.concatenate([pr["H_true"][None], W.init_chains(w, 5),
                         W.perturbed(pr["H_true"], 2.0, [7])[None]])
    H = torch.tensor(Hs, dtype=torch.float32, device=DEV).contiguous()
    Oa, Ta, lla, ev_a, tot_a = _run(a, H, w.S * w.P)
    Ob, Tb, llb, ev_b, tot_b = _run(b, H, w.S * w.P)
    assert np.array_equal(Oa, Ob)
    assert np.array_equal(Ta, Tb)
    assert np.array_equal(lla, llb)
    assert tot_a == tot_b and ev_b == tot_b
    assert ev_a < tot_a
    a.close()
    b.close()


def test_windows_bit_identical_scenario_chains():
    """Full scenario geometry and data, a few chains (the bench's workload)."""
    w = W.scenario()
    pr = W.problem(w)
    a = _ctx(pr, mt.PREC_F32, full=False)
    b = _ctx(pr, mt.PREC_F32, full=True)
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=DEV)
    a.generate_data(pr["H_true"], w.seed_data, mt.COUNTS_POISSON, counts_out=counts)
    a.sync(60.0)
    b.set_counts(counts.cpu().numpy())
    Hs = np.concatenate([pr["H_true"][None], W.init_chains(w, 3)])
    H = torch.tensor(Hs, dtype=torch.float32, device=DEV).contiguous()
    Oa, Ta, lla, ev_a, tot_a = _run(a, H, w.S * w.P)
    Ob, Tb, llb, ev_b, tot_b = _run(b, H, w.S * w.P)
    assert np.array_equal(Oa, Ob)
    assert np.array_equal(lla, llb)
    assert ev_a < 0.5 * tot_a
    a.close()
    b.close()
