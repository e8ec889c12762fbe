"""Throughput of the muon-tomography posterior hot path on one GB300 (or N, weak scaling).

A step is one random-walk Metropolis step of every chain: Philox proposal,
log-prior, fused ray march + Poisson log-likelihood, fixed-order reduction and
accept.  The workload is the 64x64-grid, 4-surface, 16-sensor x 64x64-pixel,
256-sample, 1024-chain scenario (FP32 march, FP64 reduction), on synthetic
data (seeded geometry, Poisson counts drawn by the library).

Prints one JSON line.  `value` = chain-ray log-likelihood evaluations per
second over all ranks (device-timed with CUDA events on the library's stream,
L2 flushed between steps).  `e2e` = the same metric through mt_logpost with
host buffers (the copies inside the timed region).  `roofline` = the ray
kernel's achieved sigmoid rate against the SFU (MUFU) issue limit.
`cpu_baseline` = the FP64 oracle on a bounded sample, on the host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_28907_gb300 import workloads as W  # noqa: E402

SM_COUNT = 152
SM_MAX_MHZ = 2070.0
EX2_PER_CLK_SM = 32      # SFU ex2.approx results per clock per SM (GB300; probe: 30.2)
RCP_PER_CLK_SM = 16      # SFU rcp.approx results per clock per SM (probe: 15.1)
FP32_PER_CLK_SM = 128    # FP32 lanes per SM (probe: 114.6 FMA/clk at the nominal clock)


# DRAM traffic of one k_march launch (read + write bytes) from the ncu capture
# summarised in profiles/k_march_scenario_c128_ncu.md, scaled from 128 to 1024
# chains; valid only for the kernel source it was measured on (captured on
# sha1 742e55f14d6e; the source below differs from it in comments only).
MARCH_TRAFFIC = {"source_sha1": "7e5d25345d68", "bytes": 76.1e6}
# Warp instructions one k_march launch issues per chain (smsp__inst_executed.sum
# of the same capture / 128 chains), for the issue-slot share of the launch.
MARCH_INST = {"source_sha1": "7e5d25345d68", "per_chain": 3.681e9 / 128}
SMSP_PER_SM = 4


def march_source_sha1():
    import hashlib
    src = os.path.join(ROOT, "paper_2603_28907_gb300", "csrc", "march.cuh")
    return hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]


def march_traffic():
    return MARCH_TRAFFIC["bytes"] if march_source_sha1() == MARCH_TRAFFIC["source_sha1"] else None


def issue_share(n_chains, launch_s):
    """Share of the GPU's instruction-issue slots (one per cycle per
    sub-partition at the maximum SM clock) that one ray-kernel launch of
    n_chains used, from the captured instruction count per chain; None once
    the kernel source differs from the capture's."""
    if march_source_sha1() != MARCH_INST["source_sha1"] or not launch_s:
        return None
    inst = MARCH_INST["per_chain"] * n_chains
    slots = launch_s * SM_COUNT * SMSP_PER_SM * SM_MAX_MHZ * 1e6
    return {"instructions": inst, "slots": slots, "frac": inst / slots,
            "basis": "smsp__inst_executed.sum per chain from the ncu capture of the same source "
                     "(profiles/k_march_scenario_c128_ncu.md) x chains, against 4 issue slots per "
                     "SM-cycle at 2070 MHz"}


# FP32 lane-ops per evaluated surface-sample of the FP32 march (two samples
# per step: 27 paired FP32 instructions and 8 scalar ones, the x-lerps and the
# exact differences h_mid - z, per 2 samples, plus 3 paired per block of 8)
EVAL_FP32_OPS = 32.0  # per evaluated surface-sample, FP32 mode (accurate logistic)


def march_peak_evaluated():
    """Evaluated surface-samples per second the pipes allow for the march's
    own op mix in the FP32 mode (32 FP32 lane-ops + rcp per evaluated sample:
    the accurate logistic forms 2^|a| on the FP32 pipe)."""
    clk = SM_COUNT * SM_MAX_MHZ * 1e6
    sfu = clk * RCP_PER_CLK_SM
    fp32 = clk * FP32_PER_CLK_SM / EVAL_FP32_OPS
    return min(sfu, fp32)


def march_peak(L):
    """Surface-samples per second the ray kernel's pipes allow (one logistic =
    ex2 + rcp per surface-sample; 12 + 9L FP32 ops per sample)."""
    clk = SM_COUNT * SM_MAX_MHZ * 1e6
    sfu = clk / (1.0 / EX2_PER_CLK_SM + 1.0 / RCP_PER_CLK_SM)
    fp32 = clk * FP32_PER_CLK_SM / ((12.0 + 9.0 * L) / L)
    return min(sfu, fp32), sfu, fp32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chains", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision / gradient / serving legs of the default line")
    ap.add_argument("--serve", action="store_true",
                    help="serving mix instead of the Metropolis step benchmark")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--linear", action="store_true",
                    help="random-walk steps under the paper's linearised forward model on the scenario")
    ap.add_argument("--copula", action="store_true",
                    help="random-walk steps under the paper's copula prior on the scenario")
    ap.add_argument("--diag", action="store_true",
                    help="time the chain diagnostics (nested R-hat, interface std) on the scenario")
    ap.add_argument("--study", choices=["precision", "gradient"], default=None,
                    help="precision-mode or gradient/MALA study on the scenario data")
    ap.add_argument("--proposals", type=int, default=100000)
    ap.add_argument("--step-scale", type=float, default=1e-2,
                    help="fraction of each served request's step budget that is run")
    return ap.parse_args()


def rank_chains(rank, n_per_rank):
    """Weak scaling: rank r owns global chains r*C .. r*C + C - 1 (no exchange)."""
    return list(range(rank * n_per_rank, (rank + 1) * n_per_rank))


def rank_seed(base, rank):
    """Philox key of a rank's chains: distinct per rank, fixed per run."""
    return base + 7919 * rank


def max_over_ranks(value, dist=None, device=None):
    """The slowest rank's time (the job's time); identity without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
                pw.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(pw) if pw else None}


# chains of the oracle's timed sample: about 2 s on 16 host cores (~30 core-s)
CPU_SAMPLE_CHAINS = 24


def cpu_baseline(pr, counts, Hs, n_chains_sample):
    """The oracle (FP64 C, threads over (chain, sensor)) on a bounded sample of the workload."""
    import oracle
    op = oracle.OracleProblem(pr, counts=counts)
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    op.loglik_batch(Hs[:n_chains_sample], n_threads=cores)
    dt = time.perf_counter() - t
    rays = n_chains_sample * pr["S"] * pr["P"]
    # the same oracle on one thread, one chain
    t = time.perf_counter()
    op.loglik_batch(Hs[:1], n_threads=1)
    dt1 = time.perf_counter() - t
    return {"value": rays / dt, "unit": "chain-ray/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_chains_sample} chains x {pr['S'] * pr['P']} rays (all sensors and "
                      f"pixels) of the same workload, one log-likelihood each, FP64, "
                      f"{dt:.2f} s wall",
            "single_thread": {"value": pr["S"] * pr["P"] / dt1, "unit": "chain-ray/s", "cores": 1,
                              "sample": f"1 chain x {pr['S'] * pr['P']} rays, {dt1:.2f} s wall"}}


def bench_config(w, C, world):
    """The workload description both arms print."""
    return {"workload": w.name, "chains_per_gpu": C, "surfaces": w.L,
            "grid": [w.R, w.Q], "sensors": w.S, "pixels": w.P, "n_grid": w.G,
            "precision": "f32 march (accurate logistic), f64 reduction", "sampler": "random-walk",
            "rw_sigma_m": w.rw_sigma, "l2": "flushed (256 MB write) between steps",
            "parallelism": f"chains sharded, {world} independent rank(s)"}


def run_reference(args, w, rank):
    """--impl reference: the FP64 oracle, timed on the host cores, same metric."""
    if rank != 0:
        return
    import oracle
    pr = W.problem(w)
    op = oracle.OracleProblem(pr)
    counts, _, _ = op.generate_counts(pr["H_true"], w.seed_data)
    op.with_counts(counts)
    cores = os.cpu_count() or 1
    n_sample = 4
    H0 = W.init_chains(w, n_sample)
    rays = pr["S"] * pr["P"]

    def step(k, H, lp, ll):
        prop = np.stack([op.rw_propose(H[c], w.rw_sigma, w.seed_mcmc, c, k) for c in range(n_sample)])
        lpn = np.array([op.logprior(p) for p in prop])
        lln = op.loglik_batch(prop, n_threads=cores)
        for c in range(n_sample):
            if oracle.mh_decide(lpn[c], lln[c], lp[c], ll[c], oracle.accept_logu(w.seed_mcmc, c, k)):
                H[c], lp[c], ll[c] = prop[c], lpn[c], lln[c]

    H = H0.copy()
    lp = np.array([op.logprior(h) for h in H])
    ll = op.loglik_batch(H, n_threads=cores)
    for k in range(args.warmup):
        step(k, H, lp, ll)
    t = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k, H, lp, ll)
    dt = time.perf_counter() - t
    value = n_sample * rays * args.steps / dt
    sample = (f"{n_sample} of {w.n_chains} chains per step, full data ({rays} rays), FP64 oracle "
              f"random-walk Metropolis step")
    print(json.dumps({
        "impl": "reference", "metric": "chain-ray loglik evals/s", "value": value,
        "unit": "chain-ray/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, w.n_chains, args.gpus),
        "cpu_baseline": {"value": value, "unit": "chain-ray/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "chain-ray/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_serve(args, rank, local):
    """Poisson-arriving inversion requests (mean 20/s) of uneven sizes through the
    continuous-batching server; latency and aggregate throughput."""
    if rank != 0:
        return
    import torch
    from paper_2603_28907_gb300 import mt
    torch.cuda.set_device(local)
    reqs = W.serving_mix(args.requests, seed=5)
    for w in reqs:
        steps = max(1, int(round(w.n_super * w.n_within * args.step_scale)))
        w.n_within = min(10, steps)
        w.n_super = max(1, steps // w.n_within)
    free, total = torch.cuda.mem_get_info()
    srv = mt.Server(device=local, hbm_budget_bytes=int(free * 0.8), max_active=8)
    probs = [W.problem(w) for w in reqs]
    starts = [W.init_chains(w).astype(np.float32) for w in reqs]
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    ids = []
    for w, pr, h0 in zip(reqs, probs, starts):
        wait = w.extra["arrival_s"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids.append(srv.submit(pr, h0, precision=mt.PREC_F32, data_seed=w.seed_data,
                              seed=w.seed_mcmc, step=0.002, n_super=w.n_super,
                              n_within=w.n_within))
    res = [srv.wait(i) for i in ids]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    evals = sum(w.n_chains * w.S * w.P * w.n_super * w.n_within for w in reqs)
    sizes = [dict(grid=w.R, L=w.L, sensors=w.S, pixels=w.P, G=w.G, chains=w.n_chains,
                  steps=w.n_super * w.n_within) for w in reqs]
    print(json.dumps({
        "metric": "served super-step latency p50 (p99, time-to-posterior alongside)",
        "value": st["superstep_ms_p50"], "unit": "ms", "higher_is_better": False,
        "n_gpus": 1, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving mix: {len(reqs)} requests, Poisson arrivals 20/s, "
                               f"grids 32-128, 3-5 surfaces, 4-32 sensors, 32-96 px per side, "
                               f"G 128-384, 64-1024 chains; step budgets x{args.step_scale:g}",
                   "max_active": 8, "hbm_budget_gb": round(free * 0.8 / 1e9, 1)},
        "serving": {"superstep_ms_p50": st["superstep_ms_p50"], "superstep_ms_p99": st["superstep_ms_p99"],
                    "ttp_s_p50": st["ttp_s_p50"], "ttp_s_p99": st["ttp_s_p99"],
                    "chain_ray_evals_per_s": st["chain_ray_evals_per_s"],
                    "wall_s": wall, "chain_ray_evals": evals, "n_done": st["n_done"],
                    "queue_wait_s_max": max(r["info"]["admit_s"] - r["info"]["submit_s"] for r in res),
                    "pool_bytes_at_start": st["pool_bytes_at_start"], "pool_bytes_now": st["pool_bytes_now"],
                    "gpu_busy_over_span": sum(r["info"]["gpu_busy_ms"] for r in res) / max(
                        1e-9, max(r["info"]["gpu_end_ms"] for r in res) - min(r["info"]["gpu_start_ms"] for r in res))},
        "requests": sizes,
        "clocks": clk,
    }), flush=True)


def _scenario_contexts(precisions, local):
    import torch
    from paper_2603_28907_gb300 import mt
    w = W.scenario()
    pr = W.problem(w)
    ctxs = {p: mt.from_workload(pr, precision=p, device=local) for p in precisions}
    first = ctxs[precisions[0]]
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=f"cuda:{local}")
    first.generate_data(pr["H_true"], w.seed_data, counts_out=counts)
    for p, c in ctxs.items():
        if c is not first:
            c.set_counts(counts)
    return w, pr, ctxs, counts


def run_precision_study(args, local):
    """Accept-decision agreement, log-likelihood and MH-ratio error of the
    reduced-precision modes on the same (current, proposal) pairs, against the
    FP64 mode (whose agreement with the oracle at this size, ~1e-12 relative,
    is a parity test).  The trajectory itself is an FP32 random
    walk, so every state is exactly representable in all modes."""
    import torch
    from paper_2603_28907_gb300 import mt
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    modes = {"f32_fp64_reduce": mt.PREC_F32, "f32_compensated": mt.PREC_F32C,
             "f32_approximate_logistic": mt.PREC_F32A, "bf16_heights": mt.PREC_BF16}
    w, pr, ctxs, counts = _scenario_contexts([mt.PREC_F64] + list(modes.values()), local)
    traj = ctxs[mt.PREC_F32]
    ref = ctxs[mt.PREC_F64]
    out = {}
    for C in (1024, 4096):
        steps = max(1, int(round(args.proposals / C)))
        H0 = torch.tensor(np.stack([W.geometry(w, [w.seed_init, c]) for c in range(C)]).astype(np.float32),
                          device=dev)
        traj.init_chains(H0, w.seed_mcmc)
        cur, prop = torch.zeros_like(H0), torch.zeros_like(H0)
        f64 = lambda n: torch.zeros(n, dtype=torch.float64, device=dev)
        llp, lpp, logu, lp_cur = f64(C), f64(C), f64(C), f64(C)
        acc = torch.zeros(C, dtype=torch.int32, device=dev)
        traj.get_state(cur, None, lp_cur)
        ll64_cur = f64(C)
        ref.logpost(cur.double(), ll64_cur, None)
        stats = {k: dict(agree=0, total=0, dll_max=0.0, dll_sum=0.0, n_fin=0, dd_max=0.0, dd_sum=0.0)
                 for k in modes}
        t0 = time.perf_counter()
        for k in range(steps):
            traj.get_state(cur, None, lp_cur)
            traj.run(mt.KERNEL_RW, w.rw_sigma, 1, 1)
            traj.get_last_step(prop, llp, lpp, acc, logu)
            ll64_prop = f64(C)
            ref.logpost(prop.double(), ll64_prop, None)
            fin = torch.isfinite(lpp)
            delta_ref = (ll64_prop + lpp) - (ll64_cur + lp_cur)
            a_ref = fin & (logu < delta_ref)
            pair = torch.cat([cur, prop])
            for name, p in modes.items():
                ll = f64(2 * C)
                ctxs[p].logpost(pair, ll, None)
                delta = (ll[C:] + lpp) - (ll[:C] + lp_cur)
                a_m = fin & (logu < delta)
                st = stats[name]
                st["agree"] += int((a_m == a_ref).sum().item())
                st["total"] += C
                if fin.any():
                    dll = (ll[C:] - ll64_prop).abs()[fin]
                    dd = (delta - delta_ref).abs()[fin]
                    st["dll_max"] = max(st["dll_max"], float(dll.max().item()))
                    st["dll_sum"] += float(dll.sum().item())
                    st["dd_max"] = max(st["dd_max"], float(dd.max().item()))
                    st["dd_sum"] += float(dd.sum().item())
                    st["n_fin"] += int(fin.sum().item())
            took = acc.bool()
            ll64_cur = torch.where(took, ll64_prop, ll64_cur)
        wall = time.perf_counter() - t0
        res = {}
        for name, st in stats.items():
            nf = max(st["n_fin"], 1)
            res[name] = dict(proposals=st["total"], agreement=st["agree"] / st["total"],
                             dll_abs_max=st["dll_max"], dll_abs_mean=st["dll_sum"] / nf,
                             mh_ratio_err_max=st["dd_max"], mh_ratio_err_mean=st["dd_sum"] / nf)
        out[f"chains_{C}"] = dict(steps=steps, wall_s=wall, modes=res)
    print(json.dumps({"study": "precision", "workload": w.name, "reference": "FP64 mode", **out}), flush=True)


def _ess(x):
    """Effective sample size of one chain's trace (Geyer's initial positive sequence)."""
    x = np.asarray(x, np.float64)
    n = x.size
    x = x - x.mean()
    v = np.dot(x, x) / n
    if v == 0:
        return 0.0  # the chain never moved
    f = np.fft.rfft(x, 2 * n)
    ac = np.fft.irfft(f * np.conj(f))[:n] / (n * v)
    s, t = 0.0, 1
    while t + 1 < n:
        pair = ac[t] + ac[t + 1]
        if pair <= 0:
            break
        s += pair
        t += 2
    return n / (1.0 + 2.0 * s)


def run_gradient_study(args, local):
    import torch
    from paper_2603_28907_gb300 import mt
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, pr, ctxs, counts = _scenario_contexts([mt.PREC_F32, mt.PREC_F64], local)
    c32, c64 = ctxs[mt.PREC_F32], ctxs[mt.PREC_F64]
    out = {}
    # 1. one gradient evaluation (its agreement with the oracle at this size
    # is a parity test)
    H = W.geometry(w, [w.seed_init, 0]).astype(np.float32)   # an ordered geometry
    g = torch.zeros((1,) + H.shape, dtype=torch.float64, device=dev)
    t = time.perf_counter()
    c32.grad(torch.tensor(H[None], device=dev), g)
    torch.cuda.synchronize()
    out["grad_ms_one_chain"] = (time.perf_counter() - t) * 1e3
    g = g[0].cpu().numpy()
    # 2. central differences (h = 1e-3 m) of the FP64-mode log-posterior at 16 sub-grid nodes
    rng = np.random.default_rng(0)
    idx = [(int(rng.integers(0, w.L)), int(rng.integers(24, 40)), int(rng.integers(24, 40))) for _ in range(16)]
    Hp = np.stack([H.astype(np.float64)] * 32)
    for j, ix in enumerate(idx):
        Hp[2 * j][ix] += 1e-3
        Hp[2 * j + 1][ix] -= 1e-3
    ll = torch.zeros(32, dtype=torch.float64, device=dev)
    lp = torch.zeros_like(ll)
    c64.logpost(torch.tensor(Hp, device=dev), ll, lp)
    f = (ll + lp).cpu().numpy()
    fd = np.array([(f[2 * j] - f[2 * j + 1]) / 2e-3 for j in range(16)])
    ga = np.array([g[ix] for ix in idx])
    out["grad_vs_fd_max_rel_err"] = float(np.max(np.abs(ga - fd) / np.maximum(np.abs(fd), 1e-3 * np.abs(g).max())))
    # 3. MALA and HMC vs random walk on 1024 chains: ESS per second of the mean height of each surface
    C = 1024
    H0 = torch.tensor(np.stack([W.geometry(w, [w.seed_init, c]) for c in range(C)]).astype(np.float32), device=dev)
    # name: (kernel, step, measured steps, adapted warm-up steps toward a
    # target acceptance, diagonal metric adapted in that warm-up)
    runs = {"rw_sigma_0.002": (mt.KERNEL_RW, 0.002, 200, 0, False),
            "mala_eps_0.5": (mt.KERNEL_MALA, 0.5, 200, 0, False),
            "mala_eps_0.005": (mt.KERNEL_MALA, 0.005, 200, 0, False),
            "hmc_eps_0.003_leapfrog_8": (mt.KERNEL_HMC, 0.003, 100, 0, False),
            "hmc_adapted_to_0.8_leapfrog_8": (mt.KERNEL_HMC, 0.003, 60, 30, False),
            "hmc_adapted_to_0.8_with_metric_leapfrog_8": (mt.KERNEL_HMC, 0.003, 60, 100, True),
            "nuts_depth_4_adapted_to_0.8_with_metric": (mt.KERNEL_NUTS, 0.003, 30, 40, True)}
    cur = torch.zeros_like(H0)
    c32.set_hmc(8)
    c32.set_nuts(4)
    for name, (kern, step, n_steps, n_adapt, metric) in runs.items():
        c32.set_adapt(0.8, n_adapt)
        # shrinkage target of the metric: (1 mm)^2, the scale of this posterior
        c32.set_metric_adapt(1 if metric else 0, 1e-6)
        c32.init_chains(H0, w.seed_mcmc)
        c32.run(kern, step, 1, max(1, n_adapt))   # graph, initial gradients, warm-up: untimed
        c32.sync(600.0)
        acc0 = torch.zeros(C, dtype=torch.int64, device=dev)
        c32.get_state(accepts_out=acc0)
        eps_c = None
        if n_adapt:
            e = torch.zeros(C, dtype=torch.float64, device=dev)
            c32.get_adapt(e)
            eps_c = np.percentile(e.cpu().numpy(), [0, 50, 100]).tolist()
        trace = np.zeros((n_steps, C, w.L))
        t_gpu = 0.0
        for k in range(n_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            c32.run(kern, step, 1, 1)
            c32.sync(600.0)
            b.record()
            b.synchronize()
            t_gpu += a.elapsed_time(b) / 1e3
            c32.get_state(cur)
            trace[k] = cur.mean(dim=(2, 3)).double().cpu().numpy()
        acc = torch.zeros(C, dtype=torch.int64, device=dev)
        c32.get_state(accepts_out=acc)
        burn = n_steps // 2
        ess = np.array([[_ess(trace[burn:, c, l]) for l in range(w.L)] for c in range(C)])
        out[name] = dict(acceptance=float((acc - acc0).double().mean().item()) / n_steps,
                         step_ms=t_gpu / n_steps * 1e3, ess_per_chain_mean=float(ess.mean()),
                         ess_per_s_total=float(ess.sum(0).mean() / (t_gpu * (n_steps - burn) / n_steps)))
        if eps_c is not None:
            out[name].update(adapted_steps=n_adapt, eps_min_median_max=eps_c)
        if metric:
            m = torch.zeros((C,) + tuple(H0.shape[1:]), dtype=torch.float64, device=dev)
            c32.get_metric(m)
            out[name]["inv_metric_sqrt_percentiles_1_50_99_m"] = \
                np.percentile(m.sqrt().cpu().numpy(), [1, 50, 99]).tolist()
    c32.set_adapt(0.8, 0)
    c32.set_metric_adapt(0)
    print(json.dumps({"study": "gradient", "workload": w.name, **out}), flush=True)


def run_linear(args, local):
    """Random-walk Metropolis under the linearised forward model (1024
    scenario chains, FP32, 75 levels of 2 m): per step the proposal, the
    prior, the voxel densities, the batched sparse path-length product and
    the accept.  Reports the set-up time, the matrix size and the
    linearisation error of the log-likelihood at the chains' starts and at
    the data-generating geometry."""
    import torch
    from paper_2603_28907_gb300 import mt
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    w = W.scenario()
    pr = W.problem(w)
    ctx = mt.from_workload(pr, precision=mt.PREC_F32, device=local, stream=stream.cuda_stream)
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=dev)
    ctx.generate_data(pr["H_true"], w.seed_data, mt.COUNTS_POISSON, counts_out=counts)
    ctx.sync(120.0)
    C, nz = 1024, 75
    H0 = torch.tensor(np.concatenate([pr["H_true"][None], W.init_chains(w, C - 1)]).astype(np.float32),
                      device=dev)
    ll_m = torch.zeros(C, dtype=torch.float64, device=dev)
    ctx.logpost(H0, ll_m, None)
    t0 = time.perf_counter()
    ctx.set_forward(mt.FORWARD_LINEAR, nz)
    setup_s = time.perf_counter() - t0
    ll_l = torch.zeros_like(ll_m)
    ctx.logpost(H0, ll_l, None)
    torch.cuda.synchronize()
    d = (ll_l - ll_m).abs().cpu().numpy()
    ctx.init_chains(H0, w.seed_mcmc)
    ctx.run(mt.KERNEL_RW, 0.002, args.warmup, 1)
    ctx.sync(120.0)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(mt.KERNEL_RW, 0.002, args.steps, 1)
        e1.record(stream)
    ctx.sync(120.0)
    ms = e0.elapsed_time(e1) / args.steps
    rays = w.S * w.P
    print(json.dumps({"linear": "random-walk Metropolis under the linearised forward model",
                      "workload": w.name, "chains": C, "levels": nz,
                      "voxels": (w.R - 1) * (w.Q - 1) * nz, "steps": args.steps, "ms_per_step": ms,
                      "chain_ray_evals_per_s": C * rays / (ms / 1e3), "setup_s": setup_s,
                      "linearisation_abs_dll_at_truth": float(d[0]),
                      "linearisation_abs_dll_at_starts_median": float(np.median(d[1:]))}), flush=True)
    ctx.close()


def run_copula(args, local):
    """Random-walk Metropolis on the latents of the paper's copula prior
    (1024 scenario chains, FP32): per step the proposal, the latent prior, the
    latent -> heights transform, the ray kernel and the accept.  Also times
    the transform alone."""
    import torch
    from paper_2603_28907_gb300 import mt
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    w = W.scenario()
    pr = W.problem(w)
    ctx = mt.from_workload(pr, precision=mt.PREC_F32, device=local, stream=stream.cuda_stream)
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=dev)
    ctx.generate_data(pr["H_true"], w.seed_data, mt.COUNTS_POISSON, counts_out=counts)
    ctx.sync(120.0)
    ctx.set_prior(mt.PRIOR_COPULA)
    C = 1024
    rng = np.random.default_rng(7)
    lat = 0.5 * rng.standard_normal((C, w.L, w.R, w.Q))
    lat[:, w.L - 1] = 0.0
    lat[:, w.L - 1, 0, :w.L - 1] = 0.9
    L0 = torch.tensor(lat.astype(np.float32), device=dev)
    ctx.init_chains(L0, w.seed_mcmc)
    ctx.run(mt.KERNEL_RW, 0.002, args.warmup, 1)
    ctx.sync(120.0)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(mt.KERNEL_RW, 0.002, args.steps, 1)
        e1.record(stream)
    ctx.sync(120.0)
    ms = e0.elapsed_time(e1) / args.steps
    H = torch.zeros_like(L0)
    ctx.copula_heights(L0, H)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(5):
        ctx.copula_heights(L0, H)
    t1.record()
    torch.cuda.synchronize()
    acc = torch.zeros(C, dtype=torch.int64, device=dev)
    ctx.get_state(accepts_out=acc)
    rays = w.S * w.P
    print(json.dumps({"copula": "random-walk Metropolis on copula-prior latents",
                      "workload": w.name, "chains": C, "steps": args.steps,
                      "ms_per_step": ms, "chain_ray_evals_per_s": C * rays / (ms / 1e3),
                      "transform_ms_1024_chains": t0.elapsed_time(t1) / 5,
                      "acceptance": float(acc.double().mean().item()) / (args.warmup + args.steps)}),
          flush=True)
    ctx.close()


def cpu_baseline_diag(hn, K, Lz, n_z):
    """The FP64 oracle's chain diagnostics (numpy, one process) on the same
    draws: nested R-hat of one draw per chain, interface std of 128 samples."""
    from oracle import diagnostics as D
    C = hn.shape[0]
    t0 = time.perf_counter()
    D.nested_rhat(hn.reshape(1, C, -1), K)
    t_rhat = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    D.interface_std(hn[:128], Lz, n_z)
    t_std = (time.perf_counter() - t0) * 1e3
    return {"kind": "oracle", "cores": 1, "nested_rhat_draws_1_ms": t_rhat,
            "interface_std_128_samples_ms": t_std,
            "sample": "the same draws; interface std on 128 of the samples"}


def run_diag(args, local):
    """Nested R-hat over 1024 scenario chains (32 super-chains of 32; one and
    ten stored draws) and the interface standard deviation over 1024 samples
    at 150 levels, timed with CUDA events, the FP64 oracle beside them."""
    import torch
    from paper_2603_28907_gb300 import mt
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.scenario()
    pr = W.problem(w)
    ctx = mt.from_workload(pr, precision=mt.PREC_F32, device=local)
    C, K, n_z = 1024, 32, 150
    H = torch.tensor(W.init_chains(w, C).astype(np.float32), device=dev)
    P = w.L * w.R * w.Q
    r = torch.zeros(P, dtype=torch.float64, device=dev)
    out = torch.zeros((w.L, n_z, w.R, w.Q), dtype=torch.float64, device=dev)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    for N in (1, 10):
        d = (H[None] + 0.01 * torch.randn((N,) + tuple(H.shape), device=dev)).contiguous()
        ms = timed(lambda: ctx.nested_rhat(d, K, r))
        res[f"nested_rhat_draws_{N}"] = {"ms": ms, "bytes_read": 3 * d.numel() * 4,
                                         "GB_per_s": 3 * d.numel() * 4 / ms / 1e6}
    ms = timed(lambda: ctx.interface_std(H, n_z, out))
    res["interface_std"] = {"ms": ms, "samples": C, "levels": n_z,
                            "voxels": w.L * n_z * w.R * w.Q}
    res["cpu_baseline"] = cpu_baseline_diag(H.cpu().double().numpy(), K, w.box[2], n_z)
    print(json.dumps({"diag": "chain diagnostics", "workload": w.name, "chains": C,
                      "super_chains": K, **res}), flush=True)
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.serve:
        run_serve(args, rank, local)
        return
    if args.study == "precision":
        if rank == 0:
            run_precision_study(args, local)
        return
    if args.study == "gradient":
        if rank == 0:
            run_gradient_study(args, local)
        return
    if args.diag:
        if rank == 0:
            run_diag(args, local)
        return
    if args.copula:
        if rank == 0:
            run_copula(args, local)
        return
    if args.linear:
        if rank == 0:
            run_linear(args, local)
        return
    w = W.scenario()
    if args.chains:
        w.n_chains = args.chains
    if args.impl == "reference":
        run_reference(args, w, rank)
        return

    import torch
    from paper_2603_28907_gb300 import mt

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    pr = W.problem(w)
    C = w.n_chains
    stream = torch.cuda.Stream(device=dev)
    ctx = mt.from_workload(pr, precision=mt.PREC_F32, device=local, stream=stream.cuda_stream)
    counts = torch.zeros((w.S, w.P), dtype=torch.int32, device=dev)
    ctx.generate_data(pr["H_true"], w.seed_data, counts_out=counts)
    ctx.sync(120.0)
    # each rank runs its own chains (weak scaling): rank r takes chains r*C .. r*C+C-1
    H0np = np.stack([W.geometry(w, [w.seed_init, g]) for g in rank_chains(rank, C)]).astype(np.float32)
    H0 = torch.tensor(H0np, device=dev)
    ctx.init_chains(H0, rank_seed(w.seed_mcmc, rank))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    ctx.set_timing(True)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            ctx.run(mt.KERNEL_RW, w.rw_sigma, 1, 1)
    stream.synchronize()
    ctx.get_timing(0, reset=True)
    ctx.get_timing(1, reset=True)
    ctx.get_work(reset=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    evs = []
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.run(mt.KERNEL_RW, w.rw_sigma, 1, 1)
            b.record(stream)
            evs.append((a, b))
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    march_ms, march_n = ctx.get_timing(0, reset=True)
    work_eval, work_total = ctx.get_work(reset=True)
    step_ms, step_n = ctx.get_timing(1, reset=True)
    if pg:
        ms = max_over_ranks(ms, pg, dev)
        pg.barrier()

    rays = pr["S"] * pr["P"]
    evals = float(C) * rays * args.steps * world
    value = evals / (ms / 1e3)
    acc = torch.zeros(C, dtype=torch.int64, device=dev)
    ctx.get_state(accepts_out=acc)

    # roofline of the ray kernel in surface-samples (logistic evaluations) per second
    avg_launch_s = (march_ms / max(march_n, 1)) / 1e3
    units_per_launch = float(C) * rays * w.G * w.L
    achieved = units_per_launch / avg_launch_s / 1e12
    peak, sfu_peak, fp32_peak = (x / 1e12 for x in march_peak(w.L))

    out = None
    if rank == 0:
        e2e = None
        if not args.no_e2e:
            e2e = measure_e2e(ctx, H0np, stream, args, w, rays)
        cpu = None
        if not args.no_cpu:
            cpu = cpu_baseline(pr, counts.cpu().numpy(), H0np.astype(np.float64), CPU_SAMPLE_CHAINS)
        out = {
            "metric": "chain-ray loglik evals/s", "value": value, "unit": "chain-ray/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(w, C, world),
            "mcmc_chain_steps_per_s": C * world * args.steps / (ms / 1e3),
            "acceptance": float(acc.double().mean().item()) / (args.warmup + args.steps),
            "gpu_launches": 5 * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "T surface-samples/s", "frac": achieved / peak,
                         "traffic": march_traffic() if C == 1024 else None,
                         "peak_sfu": sfu_peak, "peak_fp32": fp32_peak,
                         "peak_basis": "152 SM x 2070 MHz; ex2 32/clk, rcp 16/clk per SM; "
                                       "128 FP32 lanes with 12+9L ops per sample",
                         "kernel": "k_march", "kernel_ms_avg": avg_launch_s * 1e3,
                         "launches": march_n,
                         "evaluated": evaluated_roofline(achieved, work_eval, work_total),
                         "issue": issue_share(C, avg_launch_s),
                         "note": "units are the method's surface-samples (12+9L FP32 ops and "
                                 "2L MUFU per sample); samples at least 29.25 log2 units from "
                                 "their surface are exactly 0/1 and added without evaluation "
                                 "(bit-identical), so frac can exceed 1; 'evaluated' rates the "
                                 "samples the kernel did compute against the pipes' limit for "
                                 "its own op mix; 'issue' is the share of instruction-issue "
                                 "slots the launch used"},
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        if not args.no_extras and world == 1:
            out["extras"] = bench_extras(ctx, stream, w, pr, counts, local)
        print(json.dumps(out), flush=True)
    ctx.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


ESS_STEPS = 120  # per sampler in the default line's effective-sample-size leg


def bench_extras(ctx, stream, w, pr, counts, local):
    """Short legs of the other configurations on the bench's own states, after
    the timed region, each with its clock record: the FP32 mode's per-chain
    error and accept decisions against the FP64 mode (whose agreement with the
    oracle at this size is a parity test), gradient and MALA step times, and a
    short serving mix."""
    import torch
    from paper_2603_28907_gb300 import mt
    dev = torch.device("cuda", local)
    C = w.n_chains
    f64 = lambda n: torch.zeros(n, dtype=torch.float64, device=dev)
    res = {}

    # precision: the chains' current states and two random-walk steps'
    # proposals in the FP32 mode, the compensated mode and the
    # approximate-logistic mode, against the FP64 mode
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    ref = mt.from_workload(pr, precision=mt.PREC_F64, device=local)
    ref.set_counts(counts)
    others = {}
    for m, prec in (("f32c", mt.PREC_F32C), ("f32a", mt.PREC_F32A)):
        others[m] = mt.from_workload(pr, precision=prec, device=local, stream=stream.cuda_stream)
        others[m].set_counts(counts)
    H = torch.zeros((C, w.L, w.R, w.Q), dtype=torch.float32, device=dev)
    ll = {"f32": f64(C)}
    lp = f64(C)
    ctx.get_state(H, ll["f32"], lp)
    ll64 = f64(C)
    ref.logpost(H.double(), ll64, None)
    ms = {}
    for m, cx in others.items():
        ll[m] = f64(C)
        with torch.cuda.stream(stream):
            cx.logpost(H, ll[m], None)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cx.logpost(H, ll[m], None)
            e1.record(stream)
        stream.synchronize()
        ms[m] = e0.elapsed_time(e1)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tmp = f64(C)
        e0.record(stream)
        ctx.logpost(H, tmp, None)
        e1.record(stream)
    stream.synchronize()
    ms["f32"] = e0.elapsed_time(e1)
    dll = {m: (v - ll64).abs() for m, v in ll.items()}
    st = {m: dict(agree=0, tie=0, dd=0.0) for m in ll}
    tot = 0
    prop, llp, lpp, logu = torch.zeros_like(H), f64(C), f64(C), f64(C)
    acc = torch.zeros(C, dtype=torch.int32, device=dev)
    for _ in range(2):
        ctx.run(mt.KERNEL_RW, w.rw_sigma, 1, 1)
        ctx.get_last_step(prop, llp, lpp, acc, logu)
        l64p = f64(C)
        ref.logpost(prop.double(), l64p, None)
        lprop = {"f32": llp}
        for m, cx in others.items():
            lprop[m] = f64(C)
            with torch.cuda.stream(stream):
                cx.logpost(prop, lprop[m], None)
        stream.synchronize()
        fin = torch.isfinite(lpp)
        d_ref = (l64p + lpp) - (ll64 + lp)
        a_ref = fin & (logu < d_ref)
        near = (logu - d_ref).abs() < 1e-6
        for m in ll:
            d = (lprop[m] + lpp) - (ll[m] + lp)
            same = (fin & (logu < d)) == a_ref
            st[m]["agree"] += int(same.sum().item())
            st[m]["tie"] += int((~same & near).sum().item())
            if fin.any():
                st[m]["dd"] = max(st[m]["dd"], float((d - d_ref).abs()[fin].max().item()))
        tot += C
        took = acc.bool()  # the trajectory follows the FP32 mode's decisions
        ll64 = torch.where(took, l64p, ll64)
        for m in ll:
            ll[m] = torch.where(took, lprop[m], ll[m])
        lp = torch.where(took, lpp, lp)
    ref.close()
    for cx in others.values():
        cx.close()
    res["precision"] = {
        "states": f"{C} scenario chains after the timed steps, then 2 random-walk steps ({tot} proposals)",
        "reference": "FP64 mode",
        **{m: {"dll_abs_mean": float(dll[m].mean().item()), "dll_abs_max": float(dll[m].max().item()),
               "accept_agreement": st[m]["agree"] / tot,
               "disagree_outside_1e-6_band": tot - st[m]["agree"] - st[m]["tie"],
               "mh_ratio_err_max": st[m]["dd"], "logpost_ms": ms[m]} for m in ll},
        "wall_s": time.perf_counter() - t0, "clocks": clocks.stop()}

    # gradient (mt_grad) and MALA step on a context of their own
    clocks = Clocks(local)
    clocks.start()
    g = mt.from_workload(pr, precision=mt.PREC_F32, device=local, stream=stream.cuda_stream)
    g.set_counts(counts)
    G = torch.zeros((C, w.L, w.R, w.Q), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        g.grad(H, G)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            g.grad(H, G)
        e1.record(stream)
    stream.synchronize()
    grad_ms = e0.elapsed_time(e1) / 3
    g.init_chains(H, w.seed_mcmc + 1)
    with torch.cuda.stream(stream):
        g.run(mt.KERNEL_MALA, 0.005, 1, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run(mt.KERNEL_MALA, 0.005, 1, 3)
        e1.record(stream)
    stream.synchronize()
    mala_ms = e0.elapsed_time(e1) / 3
    # effective samples per second of each surface's mean height, random walk
    # against MALA, from the same starts (second half of a short run)
    ess = {}
    for name, kern, step in (("rw_sigma_0.002", mt.KERNEL_RW, w.rw_sigma), ("mala_eps_0.005", mt.KERNEL_MALA, 0.005)):
        g.init_chains(H, w.seed_mcmc + 2)
        with torch.cuda.stream(stream):
            g.run(kern, step, 1, 1)
        stream.synchronize()
        a0 = torch.zeros(C, dtype=torch.int64, device=dev)
        g.get_state(accepts_out=a0)
        n_steps, t_s = ESS_STEPS, 0.0
        trace = np.zeros((n_steps, C, w.L))
        cur = torch.zeros_like(H)
        for k in range(n_steps):
            with torch.cuda.stream(stream):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.run(kern, step, 1, 1)
                e1.record(stream)
            stream.synchronize()
            t_s += e0.elapsed_time(e1) / 1e3 if k >= n_steps // 2 else 0.0
            g.get_state(cur)
            trace[k] = cur.mean(dim=(2, 3)).double().cpu().numpy()
        a1 = torch.zeros(C, dtype=torch.int64, device=dev)
        g.get_state(accepts_out=a1)
        burn = n_steps // 2
        e = np.array([[_ess(trace[burn:, c, l]) for l in range(w.L)] for c in range(C)])
        ess[name] = {"acceptance": float((a1 - a0).double().mean().item()) / n_steps,
                     "ess_per_chain_mean": float(e.mean()),
                     "ess_per_s": float(e.sum(0).mean() / t_s), "step_ms": t_s / (n_steps - burn) * 1e3}
    g.close()
    rays = w.S * w.P
    res["gradient"] = {"chains": C, "mt_grad_ms": grad_ms,
                       "surface_samples_per_s": C * rays * w.G * w.L / (grad_ms / 1e3),
                       "mala_step_ms": mala_ms, "mala_eps_m": 0.005,
                       "ess": {"steps": ESS_STEPS, "statistic": "mean height of each surface, second half",
                               **ess, "mala_over_rw_ess_per_s": ess["mala_eps_0.005"]["ess_per_s"] /
                               max(ess["rw_sigma_0.002"]["ess_per_s"], 1e-300)},
                       "clocks": clocks.stop()}

    # serving: eight requests of the serving mix, step budgets scaled by 1/200
    clocks = Clocks(local)
    clocks.start()
    reqs = W.serving_mix(8, seed=5)
    for q in reqs:
        steps = max(1, int(round(q.n_super * q.n_within / 200)))
        q.n_within = min(10, steps)
        q.n_super = max(1, steps // q.n_within)
    free, _ = torch.cuda.mem_get_info()
    srv = mt.Server(device=local, hbm_budget_bytes=int(free * 0.5), max_active=8)
    t0 = time.perf_counter()
    ids = []
    for q in reqs:
        wait = q.extra["arrival_s"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids.append(srv.submit(W.problem(q), W.init_chains(q).astype(np.float32), precision=mt.PREC_F32,
                              data_seed=q.seed_data, seed=q.seed_mcmc, step=0.002, n_super=q.n_super,
                              n_within=q.n_within))
    infos = [srv.wait(i)["info"] for i in ids]
    st = srv.stats()
    srv.close()
    span = max(f["gpu_end_ms"] for f in infos) - min(f["gpu_start_ms"] for f in infos)
    res["serving"] = {"requests": len(reqs), "superstep_ms_p50": st["superstep_ms_p50"],
                      "superstep_ms_p99": st["superstep_ms_p99"], "ttp_s_p50": st["ttp_s_p50"],
                      "ttp_s_p99": st["ttp_s_p99"], "chain_ray_evals_per_s": st["chain_ray_evals_per_s"],
                      "gpu_busy_over_span": sum(f["gpu_busy_ms"] for f in infos) / max(span, 1e-9),
                      "pool_grew_bytes": st["pool_bytes_now"] - st["pool_bytes_at_start"],
                      "wall_s": time.perf_counter() - t0, "clocks": clocks.stop()}
    return res


def evaluated_roofline(achieved_t, work_eval, work_total):
    """Roofline of the work the ray kernel actually did: evaluated
    surface-samples per second against march_peak_evaluated()."""
    if not work_total:
        return None
    frac_eval = work_eval / work_total
    ach = achieved_t * frac_eval
    peak = march_peak_evaluated() / 1e12
    return {"fraction": frac_eval, "achieved": ach, "peak": peak, "frac": ach / peak,
            "unit": "T evaluated surface-samples/s",
            "ops_per_sample": f"{EVAL_FP32_OPS:g} FP32 lane-ops + rcp + cvt (accurate logistic)"}


def measure_e2e(ctx, H0np, stream, args, w, rays):
    """mt_logpost through the C ABI with host buffers: H2D of the heights, D2H of the results."""
    import torch
    C = H0np.shape[0]
    hp = torch.from_numpy(H0np.copy()).pin_memory()
    Hh = hp.numpy()
    ll = torch.zeros(C, dtype=torch.float64).pin_memory().numpy()
    lp = torch.zeros(C, dtype=torch.float64).pin_memory().numpy()
    ctx.set_timing(False)
    for _ in range(max(1, args.warmup)):
        ctx.logpost(Hh, ll, lp)
    n = max(3, args.steps // 2)
    t = time.perf_counter()
    for _ in range(n):
        ctx.logpost(Hh, ll, lp)
    dt = (time.perf_counter() - t) / n
    return {"value": C * rays / dt, "unit": "chain-ray/s", "h2d_bytes_per_step": int(Hh.nbytes),
            "d2h_bytes_per_step": int(ll.nbytes + lp.nbytes), "ms_per_step": dt * 1e3,
            "call": "mt_logpost(host heights -> host loglik, logprior)"}


if __name__ == "__main__":
    main()
