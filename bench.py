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
# chains; valid only for the kernel source it was measured on.
MARCH_TRAFFIC = {"source_sha1": "215987152a0e", "bytes": 72.0e6}


def march_traffic():
    import hashlib
    src = os.path.join(ROOT, "paper_2603_28907_gb300", "csrc", "march.cuh")
    h = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    return MARCH_TRAFFIC["bytes"] if h == MARCH_TRAFFIC["source_sha1"] else None


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
    ap.add_argument("--serve", action="store_true",
                    help="serving mix instead of the Metropolis step benchmark")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--step-scale", type=float, default=1e-2,
                    help="fraction of each served request's step budget that is run")
    return ap.parse_args()


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


def cpu_baseline(pr, counts, Hs, n_chains_sample):
    """The oracle (FP64 C, threads over (chain, sensor)) on a bounded sample of the workload."""
    import oracle
    op = oracle.OracleProblem(pr, counts=counts)
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    op.loglik_batch(Hs[:n_chains_sample], n_threads=cores)
    dt = time.perf_counter() - t
    rays = n_chains_sample * pr["S"] * pr["P"]
    return {"value": rays / dt, "unit": "chain-ray/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_chains_sample} chains x {pr['S'] * pr['P']} rays (all sensors and "
                      f"pixels) of the same workload, one log-likelihood each, FP64, "
                      f"{dt:.2f} s wall"}


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
        "config": {"workload": w.name, "chains": w.n_chains, "sampler": "rw"},
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
                    "queue_wait_s_max": max(r["info"]["admit_s"] - r["info"]["submit_s"] for r in res)},
        "requests": sizes,
        "clocks": clk,
    }), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.serve:
        run_serve(args, rank, local)
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
    H0np = np.stack([W.geometry(w, [w.seed_init, rank * C + c]) for c in range(C)]).astype(np.float32)
    H0 = torch.tensor(H0np, device=dev)
    ctx.init_chains(H0, w.seed_mcmc + 7919 * rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    ctx.set_timing(True)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            ctx.run(mt.KERNEL_RW, w.rw_sigma, 1, 1)
    stream.synchronize()
    ctx.get_timing(0, reset=True)
    ctx.get_timing(1, reset=True)
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
    step_ms, step_n = ctx.get_timing(1, reset=True)
    if pg:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
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
            cpu = cpu_baseline(pr, counts.cpu().numpy(), H0np.astype(np.float64), 8)
        out = {
            "metric": "chain-ray loglik evals/s", "value": value, "unit": "chain-ray/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "chains_per_gpu": C, "surfaces": w.L,
                       "grid": [w.R, w.Q], "sensors": w.S, "pixels": w.P, "n_grid": w.G,
                       "precision": "f32 march, f64 reduction", "sampler": "random-walk",
                       "rw_sigma_m": w.rw_sigma, "l2": "flushed (256 MB write) between steps",
                       "parallelism": f"chains sharded, {world} independent rank(s)"},
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
                         "launches": march_n},
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


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
