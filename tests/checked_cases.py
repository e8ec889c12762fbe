"""Cases run by tests/test_gpu_checked_build.py, in a child process that
loads either library (MT_CHECKED=1: the bounds-checked one).  Prints one JSON
object: per case the log-likelihoods (or gradient sums) the library gave and
whether mt_sync reported a clean device status word."""
import json
import sys

import numpy as np
import torch

from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV, setup


def _ll(ctx, H):
    ll = torch.zeros(H.shape[0], dtype=torch.float64, device=DEV)
    ctx.logpost(H, ll, None)
    return ll


def run():
    out = {"lib": mt.LIB_PATH}
    cases = {
        "tiny_f32": (W.tiny(), mt.PREC_F32),
        "tiny_f64": (W.tiny(), mt.PREC_F64),
        "tiny_bf16": (W.tiny(), mt.PREC_BF16),
        "tiny_f32a": (W.tiny(), mt.PREC_F32A),
        "odd_down_f32c": (W.small(R=5, Q=7, n_sensors=3, n_zenith=6, n_azimuth=7, G=20,
                                  zenith_max_deg=120.0), mt.PREC_F32C),
        "large_phased_f32": (W.small(R=100, Q=100, bases=(40.0, 70.0, 110.0, 140.0),
                                     rho=(2.65, 1.9, 0.0012, 2.65, 0.0012), G=64, n_zenith=6, n_azimuth=9,
                                     n_sensors=2), mt.PREC_F32),
        "huge_hbm_f32": (W.small(R=170, Q=170, bases=(40.0, 70.0), G=48, n_zenith=5, n_azimuth=7,
                                 n_sensors=2), mt.PREC_F32),
    }
    for name, (w, prec) in cases.items():
        pr, ctx, op, counts, _ = setup(w, precision=prec)
        dt = torch.float64 if prec == mt.PREC_F64 else torch.float32
        H = torch.tensor(np.concatenate([pr["H_true"][None], W.init_chains(w, 2)]), dtype=dt, device=DEV)
        ll = _ll(ctx, H)
        rec = {"ll": ll.cpu().tolist()}
        if prec in (mt.PREC_F32, mt.PREC_F32C, mt.PREC_F32A) and name not in ("large_phased_f32", "huge_hbm_f32"):
            g = torch.zeros(H.shape, dtype=torch.float64, device=DEV)
            ctx.grad(H, g)
            rec["grad_sum"] = float(g.abs().sum().item())
        if name == "tiny_f32":
            ctx.set_forward(mt.FORWARD_LINEAR, 30)
            rec["linear_ll"] = _ll(ctx, H).cpu().tolist()
            ctx.set_forward(mt.FORWARD_MARCH)
            ctx.set_nuts(2)
            ctx.init_chains(H, 7)
            ctx.run(mt.KERNEL_NUTS, 0.002, 1, 1)
            st = torch.zeros_like(H)
            ctx.get_state(st)
            rec["nuts_state_sum"] = float(st.double().sum().item())
        try:
            ctx.sync(60.0)
            rec["clean"] = True
        except mt.MtError as e:
            rec["clean"] = False
            rec["error"] = str(e)
        ctx.close()
        out[name] = rec
    print(json.dumps(out))


if __name__ == "__main__":
    run()
    sys.stdout.flush()
