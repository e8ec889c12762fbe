"""Continuous-batching server: every request's result is the same alone and in a mix.

Requests of uneven grids, surfaces, sensors, pixels, samples and chains
(a scaled-down serving mix) are submitted at their Poisson arrival times to a
server whose memory budget and slot count force queueing, and again one at a
time to a server with a single slot.  Final chain states, log-likelihoods and
acceptance counts must be bit-identical (the kernels are deterministic and each
request draws only from its own Philox key); one request is also checked
against the FP64 oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2603_28907_gb300 import mt, workloads as W

pytestmark = pytest.mark.gpu


def _submit_all(srv, reqs, pace=True):
    ids, t0 = [], time.perf_counter()
    for w in reqs:
        if pace:
            wait = w.extra["arrival_s"] * 0.05 - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        pr = W.problem(w)
        ids.append(srv.submit(pr, W.init_chains(w).astype(np.float32), precision=mt.PREC_F32,
                              data_seed=w.seed_data, seed=w.seed_mcmc, step=0.02,
                              n_super=w.n_super, n_within=w.n_within))
    return ids


def test_mix_equals_alone_and_batches_continuously():
    reqs = W.serving_mix(7, seed=5, small_scale=True)
    mix = mt.Server(hbm_budget_bytes=80 << 20, max_active=3)
    ids = _submit_all(mix, reqs)
    res_mix = [mix.wait(i, 120.0) for i in ids]
    st = mix.stats()
    mix.close()
    alone = mt.Server(hbm_budget_bytes=8 << 30, max_active=1)
    res_alone = []
    for w in reqs:
        [i] = _submit_all(alone, [w], pace=False)
        res_alone.append(alone.wait(i, 120.0))
    alone.close()
    for a, b in zip(res_mix, res_alone):
        np.testing.assert_array_equal(a["heights"], b["heights"])
        np.testing.assert_array_equal(a["loglik"], b["loglik"])
        np.testing.assert_array_equal(a["accepts"], b["accepts"])
    infos = [r["info"] for r in res_mix]
    # continuous batching: some request was admitted while an earlier one was still running
    overlap = any(infos[j]["admit_s"] < infos[i]["done_s"] for i in range(len(infos))
                  for j in range(i + 1, len(infos)))
    assert overlap
    assert st["n_done"] == len(reqs) and st["n_pending"] == 0
    assert np.isfinite(st["superstep_ms_p50"]) and st["superstep_ms_p99"] >= st["superstep_ms_p50"]
    assert st["ttp_s_p99"] >= st["ttp_s_p50"] > 0


def test_served_result_matches_oracle():
    w = W.serving_mix(3, seed=11, small_scale=True)[1]
    pr = W.problem(w)
    srv = mt.Server(hbm_budget_bytes=1 << 30, max_active=2)
    [i] = _submit_all(srv, [w], pace=False)
    r = srv.wait(i, 120.0)
    srv.close()
    op = oracle.OracleProblem(pr)
    counts, _, _ = op.generate_counts(pr["H_true"], w.seed_data)
    op.with_counts(counts)
    for c in range(r["heights"].shape[0]):
        H = r["heights"][c].astype(np.float64)
        assert abs(r["loglik"][c] - op.loglik(H)) <= 1e-3
        assert abs(r["logprior"][c] - op.logprior(H)) <= 1e-9 * max(1.0, abs(r["logprior"][c]))


def test_budget_and_bad_requests():
    w = W.serving_mix(1, seed=3, small_scale=True)[0]
    srv = mt.Server(hbm_budget_bytes=1 << 20, max_active=1)   # 1 MiB: smaller than any request
    with pytest.raises(mt.MtError) as e:
        _submit_all(srv, [w], pace=False)
    assert e.value.status == -2
    srv.close()


def test_cancel_queued_and_running_requests():
    """One slot: request A runs (many super-steps), B waits in the queue.
    Cancelling B drops it at once; cancelling A stops it at a super-step
    boundary and frees its slot, so C then runs and equals C served alone."""
    reqs = W.serving_mix(3, seed=9, small_scale=True)
    a, b, c = reqs
    srv = mt.Server(hbm_budget_bytes=1 << 30, max_active=1)
    pa = W.problem(a)
    ida = srv.submit(pa, W.init_chains(a).astype(np.float32), data_seed=a.seed_data, seed=a.seed_mcmc,
                     step=0.02, n_super=100000, n_within=1)
    idb, = _submit_all(srv, [b], pace=False)
    time.sleep(0.2)
    srv.cancel(idb)
    with pytest.raises(mt.MtError) as e:
        srv.wait(idb, 10.0)
    assert e.value.status == -7
    srv.cancel(ida)
    with pytest.raises(mt.MtError) as e:
        srv.wait(ida, 60.0)
    assert e.value.status == -7
    idc, = _submit_all(srv, [c], pace=False)
    got = srv.wait(idc, 120.0)
    with pytest.raises(mt.MtError) as e:                # already finished
        srv.cancel(idc)
    assert e.value.status == -3
    with pytest.raises(mt.MtError):
        srv.cancel(12345)
    srv.close()
    alone = mt.Server(hbm_budget_bytes=1 << 30, max_active=1)
    idc2, = _submit_all(alone, [c], pace=False)
    ref = alone.wait(idc2, 120.0)
    alone.close()
    np.testing.assert_array_equal(got["heights"], ref["heights"])
    np.testing.assert_array_equal(got["loglik"], ref["loglik"])


def test_requests_overlap_on_device_without_allocating():
    """Six scenario-size requests submitted at once to a three-slot server:
    their super-steps run on the device at the same time (device-clock spans
    of different requests intersect, and the requests' summed super-step time
    exceeds the span of the whole mix), and serving them took no device memory
    beyond what the server reserved at creation (its pool held the same bytes
    before and after: no request's memory came from the driver, and no
    cudaFree synchronised the device)."""
    reqs = []
    for k in range(6):  # the scenario workload with 64 chains: ~1.5 ms per step
        w = W.scenario()
        w.n_chains, w.n_super, w.n_within = 64, 12, 2
        w.seed_init, w.seed_mcmc = 50 + k, 60 + k
        reqs.append(w)
    srv = mt.Server(hbm_budget_bytes=1 << 30, max_active=3)
    ids = _submit_all(srv, reqs, pace=False)
    infos = [srv.wait(i, 120.0)["info"] for i in ids]
    st = srv.stats()
    srv.close()
    spans = [(f["gpu_start_ms"], f["gpu_end_ms"]) for f in infos]
    assert all(np.isfinite(a) and b > a for a, b in spans), spans
    pairs = [(i, j) for i in range(len(spans)) for j in range(i + 1, len(spans))
             if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1]]
    assert pairs, spans
    # one request's super-steps run in order on its own stream, so its busy time
    # fits in its span; a sum over requests above the span of the whole mix
    # means super-steps of different requests ran at the same time
    span_all = max(b for _, b in spans) - min(a for a, _ in spans)
    busy = sum(f["gpu_busy_ms"] for f in infos)
    assert busy > span_all, (busy, span_all)
    assert st["pool_bytes_at_start"] >= 1 << 30, st
    assert st["pool_bytes_now"] == st["pool_bytes_at_start"], st
