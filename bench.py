"""Benchmark: HVPs/s and ms per full reduced Hessian on the 9.2k-bus synthetic grid (FP64).

One step = one pass of the hot path on a new load snapshot (AR(1) load
trajectory): Newton-Raphson power flow warm-started from the previous state
(g, G_x, LU refactorisation, sweeps), reduced gradient (adjoint), and the
full dense reduced Hessian from batched adjoint-adjoint HVPs.  value =
Hessian columns (HVPs) per second of step time, summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Inputs are synthetic and resident on the device before timing; L2 is flushed
(a 256 MB write) between timed steps, outside the step's events.  The plain
form (one direction per launch, k = 1) is timed on a sample of columns.
The CPU baseline and the reference arm time the FP64 CPU oracle.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_02590_b300 import synth  # noqa: E402

WORKLOAD = "large9200"
METRIC = "HVPs/s and ms per full reduced Hessian (9.2k-bus, FP64); batched vs plain"
UNIT = "HVP/s"
FP64_PEAK_TFLOPS = 1.25        # B300 FP64 (vector and tensor) nominal rate of the pool's recipe
HBM_FALLBACK_GBS = 6400.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block-k", type=int, default=8)
    ap.add_argument("--plain-cols", type=int, default=64)
    ap.add_argument("--cpu-cols", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(nu, extra=None):
    cfg = {"workload": "9.2k-bus synthetic grid (9,200 buses, 1,450 generators, 16,000 branches, "
                       "20% transformers), AR(1) load snapshots",
           "n_bus": 9200, "n_u": nu, "n_x": 16949, "m": 41201,
           "step": "power flow + reduced gradient + full reduced Hessian",
           "l2": "flushed between timed steps (256 MB write)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- CPU oracle

def oracle_step(on, u, al, x0, pd, qd, cols):
    """One step of the oracle: power flow, gradient, `cols` Hessian columns.  Returns timings."""
    t0 = time.perf_counter()
    x, info = on.powerflow(u, pd=pd, qd=qd, x0=x0)
    t1 = time.perf_counter()
    on.reduced_gradient(x, u, al, pd=pd, qd=qd)
    t2 = time.perf_counter()
    on.reduced_hessian(x, u, al, cols=cols, pd=pd, qd=qd)
    t3 = time.perf_counter()
    return x, t2 - t0, t3 - t2


def cpu_value(nu, ncols, fixed_s, cols_s):
    return nu / (fixed_s + cols_s * nu / ncols)


def run_cpu_baseline(net, ncols):
    import oracle
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    al = synth.al_inputs(net, seed=7)
    pds, qds = synth.ar1_loads(net, 2, seed=100)
    x, _ = on.powerflow(u)
    nu = len(u)
    ncols = max(1, min(ncols, nu))
    cols = np.linspace(0, nu - 1, ncols).round().astype(np.int32)
    x, fixed, colt = oracle_step(on, u, al, x, pds[1], qds[1], cols)
    return {"value": cpu_value(nu, ncols, fixed, colt), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one step on the same workload with {ncols} of {nu} Hessian columns "
                      f"(power flow + gradient {fixed:.2f} s, columns {colt:.2f} s), scaled to all columns; "
                      "single-threaded FP64 C, gcc -O2"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    net = synth.workload(WORKLOAD)
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    al = synth.al_inputs(net, seed=7)
    nu = len(u)
    pds, qds = synth.ar1_loads(net, args.warmup + args.steps + 1, seed=100)
    x, _ = on.powerflow(u)
    ncols = max(8, min(args.cpu_cols, nu))
    cols = np.linspace(0, nu - 1, ncols).round().astype(np.int32)
    for w in range(args.warmup):
        x, _, _ = oracle_step(on, u, al, x, pds[w + 1], qds[w + 1], cols)
    vals, times = [], []
    for k in range(args.steps):
        s = args.warmup + 1 + k
        x, fixed, colt = oracle_step(on, u, al, x, pds[s], qds[s], cols)
        vals.append(cpu_value(nu, ncols, fixed, colt))
        times.append(fixed + colt * nu / ncols)
    value = statistics.mean(vals)
    ms = 1e3 * statistics.mean(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(nu, {"cpu_columns_per_step": ncols}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: power flow, gradient and {ncols} of {nu} Hessian columns "
                                       "of the FP64 C oracle, scaled to all columns"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def hvp_flops_per_column(sym, nx, nl):
    """Algorithmic FP64 flops of one HVP column: four triangular sweeps (2 per strictly
    triangular entry, 1 per diagonal scaling) and the branch second-order products (32 per branch)."""
    nnz_strict = (len(sym["colidx"]) - nx) // 2
    return 8 * nnz_strict + 2 * nx + 32 * nl


def hbm_bytes_per_hessian(sym, nx, nu, k):
    """Factor-plus-RHS bytes of a block of k directions, 24 nnz(L+U) + 64 n_x k, over all blocks."""
    nnz_lu = len(sym["colidx"]) - nx
    blocks = -(-nu // k)
    return blocks * (24 * nnz_lu + 64 * nx * k)


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2110_02590_b300 as P

    net = synth.workload(WORKLOAD)
    ctx = P.OPFContext(net, device=local)
    nu, nx = ctx.nu, ctx.nx
    sym = ctx.symbolic()
    u = torch.as_tensor(synth.flat_control(net), device=dev)
    al_h = synth.al_inputs(net, seed=7)
    al = {k: (torch.as_tensor(v, device=dev) if isinstance(v, np.ndarray) else v) for k, v in al_h.items()}
    nsnap = args.warmup + args.steps + 1
    pds_h, qds_h = synth.ar1_loads(net, nsnap, seed=100 + rank)
    pds = torch.as_tensor(pds_h, device=dev)
    qds = torch.as_tensor(qds_h, device=dev)
    x, _ = ctx.powerflow(u)
    H = torch.empty((nu, nu), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(s):
        nonlocal x
        x, info = ctx.powerflow(u, pd=pds[s], qd=qds[s], x0=x)
        g = ctx.reduced_gradient(al)
        _, hinfo = ctx.reduced_hessian(al, block_k=args.block_k, out=H)
        return g, hinfo, info

    for w in range(args.warmup):
        step(1 + w)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    hess_ms, hvp_ms, pf_iters = [], [], []
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            g, hinfo, info = step(args.warmup + 1 + k)
            ev[k][1].record(stream)
            hess_ms.append(hinfo["ms_total"])
            hvp_ms.append(hinfo["ms_hvp"])
            pf_iters.append(info["iterations"])
        torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * nu / (ms_per_step * 1e-3)

    # plain form (k = 1, one direction per launch) on a column sample
    pc = max(1, min(args.plain_cols, nu))
    _, pinfo = ctx.reduced_hessian(al, block_k=1, plain=True, out=H, col_begin=0, col_count=pc)
    plain_ms_per_col = pinfo["ms_hvp"] / pc

    # dominant kernel roofline (the HVP tile kernel; its time is the HVP phase of the Hessian call)
    flops = hvp_flops_per_column(sym, nx, net.n_branch) * nu
    hvp_s = statistics.median(hvp_ms) * 1e-3
    achieved_tf = flops / hvp_s / 1e12
    hbm_peak, hbm_kind = peaks()
    hbm_b = hbm_bytes_per_hessian(sym, nx, nu, args.block_k)

    # end to end: host (pinned) inputs in, Hessian and gradient out, through the C ABI
    pin = lambda a: torch.as_tensor(a).pin_memory()  # noqa: E731
    host_pd, host_qd = pin(pds_h), pin(qds_h)
    host_u = pin(synth.flat_control(net))
    host_al = {k: pin(v) for k, v in al_h.items() if isinstance(v, np.ndarray)}
    host_H = torch.empty((nu, nu), dtype=torch.float64).pin_memory()
    host_g = torch.empty(nu, dtype=torch.float64).pin_memory()
    dev_u = torch.empty_like(u)
    dev_pd = torch.empty(net.n_bus, dtype=torch.float64, device=dev)
    dev_qd = torch.empty_like(dev_pd)
    dev_al = {k: torch.empty(v.shape, dtype=torch.float64, device=dev) for k, v in host_al.items()}
    dev_al.update({k: v for k, v in al_h.items() if not isinstance(v, np.ndarray)})
    ks = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(ks):
        s = 1 + (k % (nsnap - 1))
        dev_pd.copy_(host_pd[s], non_blocking=True)
        dev_qd.copy_(host_qd[s], non_blocking=True)
        dev_u.copy_(host_u, non_blocking=True)
        for kk, v in host_al.items():
            dev_al[kk].copy_(v, non_blocking=True)
        x, _ = ctx.powerflow(dev_u, pd=dev_pd, qd=dev_qd, x0=x)
        g = ctx.reduced_gradient(dev_al)
        ctx.reduced_hessian(dev_al, block_k=args.block_k, out=H)
        host_H.copy_(H, non_blocking=True)
        host_g.copy_(g["grad_u"], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ks
    h2d = 8 * (2 * net.n_bus + nu + sum(v.numel() for v in host_al.values()))
    d2h = 8 * (nu * nu + nu)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(nu, {"block_k": args.block_k, "grid": hinfo["grid"], "tiles": hinfo["tiles"],
                                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "ms_per_hessian": statistics.median(hess_ms),
        "ms_hvp_phase": statistics.median(hvp_ms),
        "hvps_per_s_hessian_only": nu / (statistics.median(hess_ms) * 1e-3),
        "plain": {"ms_per_hvp": plain_ms_per_col, "hvps_per_s": 1e3 / plain_ms_per_col,
                  "ms_per_hessian_extrapolated": plain_ms_per_col * nu, "columns_timed": pc},
        "batched_over_plain": (nu / hvp_s) / (1e3 / plain_ms_per_col),
        "pf_iterations": statistics.median(pf_iters),
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "hvp_tile_kernel", "flops_per_launch": flops,
                     "peak_note": "FP64 FMA pipe, nominal 1.25 TFLOP/s (microbenchmark on this pool: 1.12)",
                     "hbm": {"bytes_per_hessian": hbm_b, "achieved_gbs": hbm_b / hvp_s / 1e9,
                             "peak_gbs": hbm_peak, "peak_kind": hbm_kind,
                             "frac": hbm_b / hvp_s / 1e9 / hbm_peak}},
        "e2e": {"value": world * nu / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3, "steps": ks},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_cpu:
        line["cpu_baseline"] = run_cpu_baseline(net, args.cpu_cols)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
