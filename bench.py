"""Benchmark: HVPs/s and ms per full reduced Hessian on the 9.2k-bus synthetic grid (FP64).

One step = one real-time tracking update on a new load snapshot (AR(1) load
trajectory), i.e. one pass of the whole hot path: Newton-Raphson power flow
at the new loads warm-started from the previous state (g, G_x, LU
refactorisation, sweeps), then one reduced-Newton step of the AL subproblem
(reduced gradient, full reduced Hessian at the Schur weights from batched
adjoint-adjoint HVPs, device Cholesky, reduced Jacobian products, power flow
at the trial control).  value = Hessian columns (HVPs) per second of step
time, summed over ranks.  The Hessian alone is timed and reported beside it.

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

if "--cpu-step" in sys.argv or "reference" in sys.argv:
    # the CPU oracle legs run single-threaded: pin the BLAS pools before numpy loads
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_02590_b300 import synth  # noqa: E402

WORKLOAD = "large9200"
METRIC = "HVPs/s and ms per full reduced Hessian (9.2k-bus, FP64); batched vs plain"
UNIT = "HVP/s"
FP64_PEAK_TFLOPS = 1.25        # B300 FP64 (vector and tensor) nominal rate of the pool's recipe
# DRAM bytes (read + write) of one hvp_split_kernel<8, 256> launch on the 9.2k grid,
# from the ncu capture summarised in profiles/hvp_split_kernel_large9200.md
HVP_SPLIT_TRAFFIC_9200 = 8.10e9
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
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-cols", type=int, default=64)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--cpu-step", action="store_true", help="internal: time one oracle tracking step")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device=None):
    """The maximum of a host number over the ranks of the default process group (the
    number itself without one): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(nu, world, total_ms, steps):
    """(ms per step, whole-job HVP/s): every rank runs its own replica on its own load
    trajectory (weak scaling), so the job processes world * n_u HVPs per step."""
    ms_per_step = total_ms / steps
    return ms_per_step, world * nu / (ms_per_step * 1e-3)


def workload_config(nu, extra=None):
    cfg = {"workload": "9.2k-bus synthetic grid (9,200 buses, 1,450 generators, 16,000 branches, "
                       "20% transformers), AR(1) load snapshots",
           "n_bus": 9200, "n_u": nu, "n_x": 16949, "m": 41201,
           "step": "tracking update: power flow at new loads + reduced-Newton step",
           "l2": "flushed between timed steps (256 MB write)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- CPU oracle

def interior_point(net, x_c_fn, u):
    """Interior primal-dual start: u 2% inside its bounds, s = c(u) clipped 1% inside its
    bounds, bound duals mu / distance (central path), mu = 0.1."""
    u_lo, u_hi = synth.control_bounds(net)
    u = np.clip(u, u_lo + 0.02 * (u_hi - u_lo), u_hi - 0.02 * (u_hi - u_lo))
    al = synth.al_inputs(net, seed=7)
    lo, hi = al["s_lo"], al["s_hi"]
    s = np.clip(x_c_fn(u), lo + 0.01 * (hi - lo), hi - 0.01 * (hi - lo))
    mu = 0.1
    st = dict(u_lo=u_lo, u_hi=u_hi, s_lo=lo, s_hi=hi, mu=mu, zl_u=mu / (u - u_lo), zu_u=mu / (u_hi - u),
              zl_s=mu / (s - lo), zu_s=mu / (hi - s))
    return u, s, al, st


def oracle_tracking(net, nsteps, seed=100):
    """The oracle's tracking loop (FP64 C + numpy): per step, the power flow at the new loads and
    one reduced-Newton step.  Returns the per-step wall times (s)."""
    import oracle
    from oracle import al_step as A
    on = oracle.OracleNet(net)
    u0 = synth.flat_control(net)
    x, _ = on.powerflow(u0)

    def cfun(u):
        xx, _ = on.powerflow(u, x0=x)
        return on.eval(xx, u)["c"]
    u, s, al, st = interior_point(net, cfun, u0)
    x, _ = on.powerflow(u, x0=x)
    pds, qds = synth.ar1_loads(net, nsteps + 1, seed=seed)
    times, delta = [], 0.0
    for k in range(1, nsteps + 1):
        t0 = time.perf_counter()
        x, _ = on.powerflow(u, pd=pds[k], qd=qds[k], x0=x)
        out = A.al_step(on, x, u, s, st, al, pd=pds[k], qd=qds[k], delta_start=delta)
        times.append(time.perf_counter() - t0)
        delta = out["delta"]
        u, s, x = out["u"], out["s"], out["x"]
        st.update(out["duals"])
    return times


def run_cpu_baseline(net):
    """One oracle tracking step, in a child process whose BLAS pools are pinned to one thread."""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-step"], capture_output=True,
                         text=True, check=True)
    t = float(out.stdout.strip().splitlines()[-1])
    nu = 1 + 2 * (net.n_gen - 1)
    return {"value": nu / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one tracking step of the same workload ({t:.1f} s): power flow at new loads and one "
                      "reduced-Newton step with all Hessian columns; FP64 C oracle, BLAS limited to 1 thread"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    net = synth.workload(WORKLOAD)
    nu = 1 + 2 * (net.n_gen - 1)
    times = oracle_tracking(net, args.warmup + args.steps)[args.warmup:]
    ms = 1e3 * statistics.mean(times)
    value = nu / (ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(nu),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "every step of the tracking loop, full Hessian, FP64 C oracle, "
                                       "BLAS limited to 1 thread"},
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
    """Algorithmic FP64 flops of one HVP column: the three full triangular sweeps (U, U^T,
    L^T; 2 per strictly triangular entry, 1 per diagonal scaling) and the branch
    second-order products (32 per branch).  The first L sweep is counted as zero: its
    right-hand side is sparse and the kernel only visits the reached rows (a few per cent
    of the entries), so counting the full sweep would overstate the work."""
    nnz_strict = (len(sym["colidx"]) - nx) // 2
    return 6 * nnz_strict + 2 * nx + 32 * nl


def hbm_bytes_per_hessian(sym, nx, nu, k):
    """Factor-plus-RHS bytes of a block of k directions, 24 nnz(L+U) + 64 n_x k, over all blocks."""
    nnz_lu = len(sym["colidx"]) - nx
    blocks = -(-nu // k)
    return blocks * (24 * nnz_lu + 64 * nx * k)


def batched_snapshots(P, torch, dev, block_k):
    """Config-3 batch: 128 x 500-bus, 64 x 2,000-bus and 16 x 9,200-bus snapshots, each at its own
    AR(1) load and power flow; all Hessians in one persistent launch vs one call per snapshot."""
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731
    snaps = []
    for name, cnt in (("batchA500", 128), ("batchB2000", 64), ("large9200", 16)):
        net = synth.workload(name)
        pds, qds = synth.ar1_loads(net, cnt + 1, seed=400)
        al = synth.al_inputs(net, seed=7)
        ald = {k: (d(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}
        u = d(synth.flat_control(net))
        for k in range(cnt):
            c = P.OPFContext(net, device=dev.index)
            c.powerflow(u, pd=d(pds[k + 1]), qd=d(qds[k + 1]))
            snaps.append((c, ald))
    outs = [torch.empty((c.nu, c.nu), dtype=torch.float64, device=dev) for c, _ in snaps]
    nhvp = sum(c.nu for c, _ in snaps)
    ms = []
    for r in range(4):
        _, info = P.reduced_hessian_batched([c for c, _ in snaps], [a for _, a in snaps], block_k=block_k,
                                            outs=outs)
        if r:
            ms.append(info["ms_total"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (c, a), o in zip(snaps, outs):
        c.reduced_hessian(a, block_k=block_k, out=o)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    bms = statistics.median(ms)
    return {"snapshots": len(snaps), "hvps": nhvp, "launches": 1, "tiles": info["tiles"], "grid": info["grid"],
            "ms_batched": bms, "hvps_per_s_batched": nhvp / (bms * 1e-3),
            "ms_per_snapshot_calls": seq_s * 1e3, "hvps_per_s_per_snapshot_calls": nhvp / seq_s}


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2110_02590_b300 as P
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731

    net = synth.workload(WORKLOAD)
    ctx = P.OPFContext(net, device=local)
    nu, nx = ctx.nu, ctx.nx
    sym = ctx.symbolic()
    x0, _ = ctx.powerflow(d(synth.flat_control(net)))

    def cfun(u):
        xx, _ = ctx.powerflow(d(u), x0=x0)
        al0 = {k: (d(v) if isinstance(v, np.ndarray) else v) for k, v in synth.al_inputs(net, seed=7).items()}
        return ctx.reduced_gradient(al0)["c"].cpu().numpy()
    u_h, s_h, al_h, st_h = interior_point(net, cfun, synth.flat_control(net))
    al = {k: (d(v) if isinstance(v, np.ndarray) else v) for k, v in al_h.items() if k != "s"}
    state = {k: d(v) for k, v in st_h.items() if k != "mu"}
    state.update(u=d(u_h), s=d(s_h), mu=st_h["mu"])
    state["x"], _ = ctx.powerflow(state["u"], x0=x0)
    tune = ctx.autotune(dict(al, s=state["s"]))
    ke = max(1, min(args.steps, args.e2e_steps))  # end-to-end steps, on the snapshots after the timed ones
    nsnap = args.warmup + args.steps + 1 + ke
    pds_h, qds_h = synth.ar1_loads(net, nsnap, seed=100 + rank)
    pds, qds = d(pds_h), d(qds_h)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    delta = [0.0]

    def step(k, pd, qd):
        state["x"], pinfo = ctx.powerflow(state["u"], pd=pd, qd=qd, x0=state["x"])
        _, _, sinfo = ctx.al_step(al, state, block_k=0, delta_start=delta[0])
        delta[0] = sinfo["delta"]
        return pinfo, sinfo

    for w in range(args.warmup):
        step(w, pds[1 + w], qds[1 + w])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if args.profile_step:
            torch.cuda.profiler.start()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            infos.append(step(k, pds[args.warmup + 1 + k], qds[args.warmup + 1 + k]))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if args.profile_step:
            torch.cuda.profiler.stop()
    launches = ctx.launch_count() - launches0
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev)
    ms_per_step, value = job_value(nu, world, total_ms, args.steps)

    # the Hessian alone (exact weights) at the current state, and the HVP kernel phase
    alh = dict(al, s=state["s"])
    hs = []
    for r in range(4):
        flush.zero_()
        _, hinfo = ctx.reduced_hessian(alh)
        if r:
            hs.append((hinfo["ms_total"], hinfo["ms_hvp"]))
    hess_ms = statistics.median(h[0] for h in hs)
    hvp_ms = statistics.median(h[1] for h in hs)
    # plain form (k = 1, one direction per launch) on a column sample
    pc = max(1, min(args.plain_cols, nu))
    _, pinfo = ctx.reduced_hessian(alh, block_k=1, plain=True, col_begin=0, col_count=pc)
    plain_ms_per_col = pinfo["ms_hvp"] / pc

    flops = hvp_flops_per_column(sym, nx, net.n_branch) * nu
    achieved_tf = flops / (hvp_ms * 1e-3) / 1e12
    hbm_peak, hbm_kind = peaks()
    hbm_b = hbm_bytes_per_hessian(sym, nx, nu, tune["block_k"])

    # end to end: loads in from pinned host memory, the new controls and slacks out, per step
    host_pd = torch.as_tensor(pds_h).pin_memory()
    host_qd = torch.as_tensor(qds_h).pin_memory()
    host_u = torch.empty(nu, dtype=torch.float64).pin_memory()
    host_s = torch.empty(ctx.m, dtype=torch.float64).pin_memory()
    dev_pd = torch.empty(net.n_bus, dtype=torch.float64, device=dev)
    dev_qd = torch.empty_like(dev_pd)
    ks = ke
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(ks):
        sidx = args.warmup + args.steps + 1 + k  # the load sequence goes on from the timed steps
        dev_pd.copy_(host_pd[sidx], non_blocking=True)
        dev_qd.copy_(host_qd[sidx], non_blocking=True)
        step(k, dev_pd, dev_qd)
        host_u.copy_(state["u"], non_blocking=True)
        host_s.copy_(state["s"], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ks

    batch = None if args.no_batch else batched_snapshots(P, torch, dev, tune["block_k"])

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    sinfos = [i[1] for i in infos]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(nu, {"step": "tracking update: power flow at new loads + reduced-Newton step "
                                               "(gradient, Schur Hessian, Cholesky, trial power flow)",
                                       "block_k": tune["block_k"], "threads": tune["threads"],
                                       "autotuned": True,
                                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "ms_per_hessian": hess_ms,
        "ms_hvp_phase": hvp_ms,
        "hvps_per_s_hessian_only": nu / (hess_ms * 1e-3),
        "ms_hessian_in_step": statistics.median(i["ms_hessian"] for i in sinfos),
        "step_detail": {"pf_iterations": statistics.median(i[0]["iterations"] for i in infos),
                        "inertia_delta": statistics.median(i["delta"] for i in sinfos),
                        "halvings": sum(i["halvings"] for i in sinfos)},
        "plain": {"ms_per_hvp": plain_ms_per_col, "hvps_per_s": 1e3 / plain_ms_per_col,
                  "ms_per_hessian_extrapolated": plain_ms_per_col * nu, "columns_timed": pc},
        "batched_over_plain": (nu / (hvp_ms * 1e-3)) / (1e3 / plain_ms_per_col),
        "batched_snapshots": batch,
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tf / FP64_PEAK_TFLOPS,
                     "traffic": (HVP_SPLIT_TRAFFIC_9200 if (tune["block_k"], tune["threads"]) == (8, 256)
                                 and WORKLOAD == "large9200" else None),
                     "kernel": ("hvp_split_kernel" if (tune["block_k"], tune["threads"]) == (8, 256)
                                else "hvp_tile_kernel"), "flops_per_launch": flops,
                     "peak_note": "FP64 FMA pipe, nominal 1.25 TFLOP/s (microbenchmark on this pool: 1.12)",
                     "hbm": {"bytes_per_hessian": hbm_b, "achieved_gbs": hbm_b / (hvp_ms * 1e-3) / 1e9,
                             "peak_gbs": hbm_peak, "peak_kind": hbm_kind,
                             "frac": hbm_b / (hvp_ms * 1e-3) / 1e9 / hbm_peak}},
        "e2e": {"value": world * nu / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * net.n_bus,
                "d2h_bytes_per_step": 8 * (nu + ctx.m), "ms_per_step": e2e_s * 1e3, "steps": ks},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_cpu:
        line["cpu_baseline"] = run_cpu_baseline(net)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.cpu_step:
        print(oracle_tracking(synth.workload(WORKLOAD), 1)[0], flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
