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

THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
if "reference" in sys.argv:
    # the reference arm (the CPU oracle) runs on all host cores: the oracle's Hessian columns
    # over OpenMP threads, the dense algebra on the BLAS pool; set before numpy loads
    for _v in THREAD_VARS:
        os.environ[_v] = str(os.cpu_count() or 1)

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_02590_b300 import synth  # noqa: E402

WORKLOAD = "large9200"
METRIC = "HVPs/s and ms per full reduced Hessian (9.2k-bus, FP64); batched vs plain"
UNIT = "HVP/s"
HBM_FALLBACK_GBS = 6400.0
# The ncu summary of the dominant kernel; its machine-readable lines give the DRAM
# traffic of one launch and the hash of the library sources it was captured with
# (the kernel's code and the host code that lays out its data).
HVP_PROFILE = os.path.join(ROOT, "profiles", "hvp_split_kernel_large9200.md")
CSRC = os.path.join(ROOT, "paper_2110_02590_b300", "csrc")
# (block_k, threads) candidates of the library's autotuner (opf_hessian_autotune)
AUTOTUNE_CANDIDATES = [(4, 128), (4, 256), (8, 128), (8, 256), (8, 512), (16, 256), (16, 512), (32, 256)]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# The sources that decide the HVP kernel's code, launch and data layout: the kernel
# itself, the device structures it reads, the host set-up that builds its schedules
# and tilings, and the symbolic analysis (ordering, fill, levels).
HVP_SOURCES = ("opf_api.cu", "opf_internal.h", "opf_kernels.cu", "symbolic.cpp")


def kernel_source_hash():
    """SHA-256 over the HVP kernel's sources (HVP_SOURCES, in that order)."""
    import hashlib
    h = hashlib.sha256()
    for f in HVP_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """(DRAM bytes per launch, note) from the committed ncu summary of the HVP kernel, or
    (None, why) when the summary is missing or was captured from other kernel sources."""
    try:
        with open(HVP_PROFILE) as fh:
            text = fh.read()
    except OSError:
        return None, "no ncu summary"
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.strip().startswith(("traffic_bytes_per_launch", "kernel_source_sha256",
                                                "kernel_launch")):
            k, v = ln.strip().split(":", 1)
            vals[k.strip()] = v.strip()
    if "traffic_bytes_per_launch" not in vals or "kernel_source_sha256" not in vals:
        return None, "ncu summary without machine-readable traffic"
    if vals["kernel_source_sha256"] != kernel_source_hash():
        return None, "HVP kernel sources changed since the ncu capture"
    return float(vals["traffic_bytes_per_launch"]), "ncu capture of " + vals.get("kernel_launch", "the kernel")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-cols", type=int, default=64)
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-autograd", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the tracking-QP and static-OPF legs")
    ap.add_argument("--autograd-scenarios", type=int, default=256)
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


def cpu_step_seconds(threads):
    """One oracle tracking step in a child process whose OpenMP and BLAS pools have `threads`."""
    env = dict(os.environ)
    for v in THREAD_VARS:
        env[v] = str(threads)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-step"], capture_output=True,
                         text=True, check=True, env=env)
    return float(out.stdout.strip().splitlines()[-1])


def run_cpu_baseline(net):
    """The oracle's tracking step on all host cores (Hessian columns over OpenMP threads, dense
    algebra on the BLAS pool) and on one core."""
    nu = 1 + 2 * (net.n_gen - 1)
    cores = os.cpu_count() or 1
    t_all = cpu_step_seconds(cores)
    t_one = cpu_step_seconds(1)
    return {"value": nu / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one tracking step of the same workload ({t_all:.2f} s on {cores} threads): power flow at "
                      "new loads and one reduced-Newton step with all Hessian columns; FP64 C oracle, columns "
                      "over OpenMP threads",
            "single_core": {"value": nu / t_one, "unit": UNIT, "cores": 1, "seconds": t_one}}


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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": "every step of the tracking loop, full Hessian, FP64 C oracle, Hessian "
                                       "columns over OpenMP threads on all host cores"},
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


def symmetric_lt_entries(net, sym, nu, k, sm_count):
    """L^T-sweep work of a full Hessian built by its symmetry (opf_set_hessian_symmetry, the
    library's default): the tile whose columns start at position p of the column order (v_ref,
    then (v, p) of the PV buses in the elimination-tree postorder of their theta rows) sweeps the
    bus blocks holding an elimination-tree ancestor of the right-hand-side rows of a control at
    a position >= p.  Replicates the library's order and its split tiling (waves of k-wide tiles,
    then k/2-wide ones; plain k-wide chunks when that tiling does not apply).  Returns (sum over
    columns of the strictly triangular L^T entries swept, sum over tiles of the entries swept (the
    factor entries each tile reads), sum over columns of the rows swept)."""
    rp, ci, perm = sym["rowptr"], sym["colidx"], sym["perm"]
    nx = len(perm)
    pos = np.empty(nx, np.int64)
    pos[perm] = np.arange(nx)
    parent = np.full(nx, -1, np.int64)
    colcnt = np.zeros(nx, np.int64)
    for i in range(nx):
        cols = ci[rp[i]:rp[i + 1]]
        cols = cols[cols < i]
        colcnt[cols] += 1
        for j in cols:
            if parent[j] < 0 or i < parent[j]:
                parent[j] = i
    nb, ref = net.n_bus, int(net.ref_bus)
    typ = np.zeros(nb, int)
    typ[np.asarray(net.gen_bus, int)] = 1
    typ[ref] = 2
    pv = [b for b in range(nb) if typ[b] == 1]
    pq = [b for b in range(nb) if typ[b] == 0]
    xs = pv + pq
    pth = {b: int(pos[q]) for q, b in enumerate(xs)}
    pvv = {b: int(pos[len(xs) + q]) for q, b in enumerate(pq)}
    rowbus = np.empty(nx, np.int64)
    for b, r in pth.items():
        rowbus[r] = b
    for b, r in pvv.items():
        rowbus[r] = b
    kids = [[] for _ in range(nx)]
    for j in range(nx):
        if parent[j] >= 0:
            kids[parent[j]].append(j)
    post, cnt = np.zeros(nx, np.int64), 0
    for r in range(nx - 1, -1, -1):
        if parent[r] >= 0:
            continue
        stack = [[r, 0]]
        while stack:
            v, c = stack[-1]
            if c < len(kids[v]):
                stack[-1][1] += 1
                stack.append([kids[v][c], 0])
            else:
                post[v] = cnt
                cnt += 1
                stack.pop()
    adj = [[] for _ in range(nb)]
    for f, t in zip(net.br_from, net.br_to):
        adj[int(f)].append(int(t))
        adj[int(t)].append(int(f))
    cols = [("v", ref)] + [c for b in sorted(pv, key=lambda b: post[pth[b]]) for c in (("v", b), ("p", b))]
    assert len(cols) == nu
    qrow = np.full(nx, -1, np.int64)
    for q in range(nu - 1, -1, -1):
        kind, b = cols[q]
        rows = [pth[b]] if kind == "p" else \
            [pth[o] for o in adj[b] if typ[o] != 2] + [pvv[o] for o in adj[b] if typ[o] == 0] + \
            ([pth[b]] if typ[b] == 1 else [])
        for r in rows:
            x = r
            while x >= 0 and qrow[x] < 0:
                qrow[x] = q
                x = parent[x]
    # block marks: the largest mark of the block's rows (a block is swept whole)
    bmark = np.full(nb, -1, np.int64)
    np.maximum.at(bmark, rowbus, qrow)
    rmark = bmark[rowbus]
    order = np.argsort(-rmark, kind="stable")
    csum_e = np.concatenate([[0], np.cumsum(colcnt[order])])
    marks_desc = rmark[order]
    # tiles: (first position, width)
    waves = nu // (k * sm_count)
    n1 = waves * sm_count
    rem = nu - n1 * k
    n2 = -(-rem // (k // 2)) if k >= 2 else 0
    if k >= 2 and waves >= 1 and rem > 0 and n2 <= sm_count:
        tiles = [(t * k, k) for t in range(n1)] + \
            [(n1 * k + t * (k // 2), min(k // 2, nu - n1 * k - t * (k // 2))) for t in range(n2)]
    else:
        tiles = [(t * k, min(k, nu - t * k)) for t in range(-(-nu // k))]
    ent = ent_tiles = rows_swept = 0
    for p, w in tiles:
        kept = int(np.searchsorted(-marks_desc, -p, side="right"))  # rows with mark >= p
        ent += w * int(csum_e[kept])
        ent_tiles += int(csum_e[kept])
        rows_swept += w * kept
    return ent, ent_tiles, rows_swept


def hbm_bytes_per_hessian(sym, nx, nu, k):
    """Factor-plus-RHS bytes of a block of k directions, 24 nnz(L+U) + 64 n_x k, over all blocks."""
    nnz_lu = len(sym["colidx"]) - nx
    blocks = -(-nu // k)
    return blocks * (24 * nnz_lu + 64 * nx * k)


def solve_phase(sym, nx, nu, k, hvp_ms, share, hbm_peak, fp64_tf, lt=None):
    """Roofline of the triangular-solve phase of the HVP kernel: the U sweep for Z and the U^T,
    L^T sweeps for Psi over the kernel time apportioned to them by the tiles' phase stamps.  Bytes:
    12 B per factor entry each sweep reads (value + column index) and 16 n_x k (read + write of the
    right-hand side) per sweep and block of k directions; flops: 2 per strictly triangular entry
    and direction, plus the diagonal scaling of U and U^T.  With lt (symmetric Hessian,
    symmetric_lt_entries) the L^T sweep counts the entries and rows it sweeps.  The pruned first L
    solve is left out of time, bytes and flops alike."""
    nnz_strict = (len(sym["colidx"]) - nx) // 2
    blocks = -(-nu // k)
    t_ms = hvp_ms * (share[1] + share[3])
    if lt is None:
        byts = blocks * (12 * (3 * nnz_strict + 2 * nx) + 3 * 16 * nx * k)
        flops = nu * (6 * nnz_strict + 2 * nx)
    else:
        ent, ent_t, rows_sw = lt
        byts = blocks * (12 * (2 * nnz_strict + 2 * nx) + 2 * 16 * nx * k) + 12 * ent_t + 16 * rows_sw
        flops = nu * (4 * nnz_strict + 2 * nx) + 2 * ent
    gbs = byts / (t_ms * 1e-3) / 1e9
    tfs = flops / (t_ms * 1e-3) / 1e12
    return {"ms": t_ms, "bytes": byts, "flops": flops, "achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak,
            "achieved_tflops": tfs, "fp64_frac": tfs / fp64_tf,
            "intensity_flop_per_byte": flops / byts, "fp64_ridge_flop_per_byte": fp64_tf * 1e3 / hbm_peak,
            "hbm_frac_ceiling_at_fp64_peak": (fp64_tf * 1e3 / hbm_peak) / (flops / byts)}


def reduced_jacobian_leg(ctx, alh, flush, hess_ms):
    """The reduced constraint Jacobian (m x n_u) from the HVP tiles' first adjoint: alone (the
    tiles stop after the L and U sweeps), beside the Hessian in the same launch, and the
    gradient-based scaling built on it (medians of 3 after one warm-up)."""
    import torch
    Jt = torch.empty((ctx.nu, ctx.m), dtype=torch.float64, device=ctx.device)
    alone, both, scal = [], [], []
    for r in range(4):
        flush.zero_()
        _, _, i1 = ctx.reduced_jacobian(None, block_k=8, out=Jt)
        flush.zero_()
        _, _, i2 = ctx.reduced_jacobian(alh, hessian=True, block_k=8, out=Jt)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, sf, _ = ctx.gradient_scaling(out_jacobian=Jt)
        torch.cuda.synchronize()
        if r:
            alone.append(i1["ms_total"])
            both.append(i2["ms_total"])
            scal.append(1e3 * (time.perf_counter() - t0))
    del Jt
    ms_alone, ms_both = statistics.median(alone), statistics.median(both)
    return {"rows_m": ctx.m, "columns": ctx.nu, "bytes": 8 * ctx.m * ctx.nu,
            "ms_jacobian_only": ms_alone, "ms_with_hessian": ms_both, "ms_hessian_alone": hess_ms,
            "byproduct_ms": ms_both - hess_ms,
            "ms_gradient_scaling_host": statistics.median(scal), "sigma_f": sf,
            "form": "J e_j = d_u c e_j + d_x c z_j from each tile's first adjoint z (Sec. III-B); "
                    "written column-major, m x n_u"}


def autograd_batch(P, torch, dev, nscen):
    """Config 4: ReducedObjective (torch.autograd.Function, adjoint backward with the power flows
    recomputed) on a batch of AR(1) load scenarios of the 2,000-bus net, forward + backward,
    beside the plain calls (opf_powerflow + opf_reduced_gradient per scenario, no autograd)."""
    from paper_2110_02590_b300.autograd import ReducedObjective
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731
    net = synth.workload("batchB2000")
    ctx = P.OPFContext(net, device=dev.index)
    al = synth.al_inputs(net, seed=7)
    ald = {k: (d(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}
    obj = ReducedObjective(ctx, ald)
    x0, _ = ctx.powerflow(d(synth.flat_control(net)))
    obj.set_warm_start(x0)
    pds, qds = synth.ar1_loads(net, nscen, seed=300)
    u = d(np.tile(synth.flat_control(net), (nscen, 1))).requires_grad_(True)
    pd, qd = d(pds).requires_grad_(True), d(qds).requires_grad_(True)
    s = d(np.tile(al["s"], (nscen, 1))).requires_grad_(True)
    for _ in range(2):  # warm-up: every context of the pool takes scenarios (first-use set-up)
        obj(u, pd, qd, s).sum().backward()
    torch.cuda.synchronize()
    runs = []
    for _ in range(3):  # median of three passes (forward, then backward with the power flows recomputed)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        F = obj(u, pd, qd, s)
        torch.cuda.synchronize()
        tb = time.perf_counter()
        F.sum().backward()
        torch.cuda.synchronize()
        runs.append((tb - ta, time.perf_counter() - tb))
    runs.sort(key=lambda r: r[0] + r[1])
    fwd_s, bwd_s = runs[1]
    t0, t1, t2 = 0.0, fwd_s, fwd_s + bwd_s
    t_plain = time.perf_counter()
    for b in range(nscen):  # plain calls: one power flow and one adjoint gradient per scenario
        ctx.powerflow(u[b].detach(), pd=pd[b].detach(), qd=qd[b].detach(), x0=x0)
        ctx.reduced_gradient(dict(ald, s=s[b].detach()))
    torch.cuda.synchronize()
    t3 = t2 + (time.perf_counter() - t_plain)
    return {"net": "2,000-bus synthetic grid", "scenarios": nscen, "contexts": len(obj.pool),
            "ms_forward": 1e3 * (t1 - t0),
            "ms_backward": 1e3 * (t2 - t1), "scenarios_per_s": nscen / (t2 - t0),
            "plain_ms": 1e3 * (t3 - t2), "plain_scenarios_per_s": nscen / (t3 - t2),
            "note": "forward: power flow + F per scenario (states kept); backward: power flow restarted from the kept "
                    "state (converges at once: one factorisation) + adjoint gradient "
                    "w.r.t. u, loads and s (median of three passes after two warm-up passes); plain: power "
                    "flow + adjoint gradient per scenario"}


def static_opf(P, torch, dev, name, max_outer=20, max_inner=60, scaling_gmax=100.0, keep_state=False):
    """Static OPF by the augmented-Lagrangian loop (opf_al_solve) on a synthetic grid at its nominal
    loads, on an instance whose AC base case is feasible (synth.static_instance: line limits
    max(rate, 1.2 |S|) with an inactive lower bound, reactive and PQ-voltage bounds widened around
    the base case), y = 0, rho = 10, an interior start at mu = 0.1, and with scaling_gmax > 0 the
    gradient-based scaling of Sec. IV-A at the start."""
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731
    net = synth.workload(name)
    ctx = P.OPFContext(net, device=dev.index)
    u_lo, u_hi = synth.control_bounds(net)
    al0 = synth.al_inputs(net, seed=5)
    u0 = synth.flat_control(net)
    x0, _ = ctx.powerflow(d(u0))
    c0 = ctx.reduced_gradient({k: (d(v) if isinstance(v, np.ndarray) else v) for k, v in al0.items()})["c"]
    al = synth.static_instance(net, al0, c0.cpu().numpy())
    u = np.clip(u0, u_lo + 0.02 * (u_hi - u_lo), u_hi - 0.02 * (u_hi - u_lo))
    x, _ = ctx.powerflow(d(u), x0=x0)
    c = ctx.reduced_gradient({k: (d(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()})["c"]
    lo, hi = al["s_lo"], al["s_hi"]
    s = np.clip(c.cpu().numpy(), lo + 0.01 * (hi - lo), hi - 0.01 * (hi - lo))
    mu = 0.1
    state = dict(u=d(u), s=d(s), x=x, u_lo=d(u_lo), u_hi=d(u_hi), s_lo=d(lo), s_hi=d(hi), mu=mu,
                 zl_u=d(mu / (u - u_lo)), zu_u=d(mu / (u_hi - u)), zl_s=d(mu / (s - lo)), zu_s=d(mu / (hi - s)))
    y = d(np.zeros(ctx.m))
    info, hist = ctx.al_solve(dict(sigma_f=al["sigma_f"], rho=10.0, sigma_c=d(al["sigma_c"])), state, y,
                              max_outer=max_outer, max_inner=max_inner, scaling_gmax=scaling_gmax)
    steps = max(1, info["steps"])
    solved = None
    if keep_state:  # the optimum the real-time tracking starts from, with the scales the loop used
        solved = dict(ctx=ctx, net=net, state=state, y=y,
                      al=dict(sigma_f=info["sigma_f"], rho=info["rho"], sigma_c=info["sigma_c"], y=y))
    summary = {"net": name, "n_u": ctx.nu, "outer": info["outer"], "steps": info["steps"],
            "converged": bool(info["converged"]), "ms_total": info["ms_total"],
            "ms_per_outer": info["ms_total"] / max(1, info["outer"]), "ms_per_step": info["ms_total"] / steps,
            "primal_inf": info["primal_inf"], "dual_inf": info["dual_inf"], "rho_final": info["rho"],
            "F_final": info["F"], "sigma_f": info["sigma_f"], "scaling_gmax": scaling_gmax,
            "steps_per_outer": [int(h[0]) for h in hist],
            "setup": "nominal loads; bounds widened around the AC base case (line limits max(rate, 1.2 |S|), "
                     "inactive flow lower bound, reactive limits to 1.2 |q|, PQ voltages to 2% around the base "
                     f"case); y0 = 0, rho0 = 10, mu0 = 0.1; at most {max_inner} reduced-Newton steps per "
                     "subproblem (one full Hessian each); "
                     + (f"gradient-based scaling with g_max = {scaling_gmax:g}" if scaling_gmax > 0
                        else "the instance's own scales (1/limit^2 on the flows, 1 elsewhere, sigma_f = 1e-4)")}
    return (summary, solved) if keep_state else summary


def mean_complementarity(st):
    """Mean of (w - w_lo) z_lo and (w_hi - w) z_hi over w = (u, s): the barrier a warm-started
    interior-point solve starts from."""
    t, n = 0.0, 0
    for nm in ("u", "s"):
        w, lo, hi = st[nm], st[nm + "_lo"], st[nm + "_hi"]
        t += float(((w - lo) * st["zl_" + nm]).sum() + ((hi - w) * st["zu_" + nm]).sum())
        n += 2 * w.numel()
    return t / n


def tracking_qp(P, torch, solved, count, seed=300, inertia_only=True, rho=10.0, reset_slacks=True):
    """Real-time OPF (Sec. IV-C) from the static optimum of the 9.2k-bus instance (the scaled AL
    loop's end point, its scales and multipliers) at a fixed penalty rho (the loop's initial one;
    None: its final one): one update per AR(1) load snapshot (opf_tracking_update: power flow at
    the new loads, the bounded QP of eq. qp_rto to a KKT error of 1e-6 with one Hessian H(omega)
    per QP iteration, the power flow at the new controls and the multiplier update).  Each QP
    starts from the previous point (pushed 1e-4 of the bounds' range inside them; with
    reset_slacks the slacks restart at the constraints' values at the new loads) and duals, with
    its barrier at their mean complementarity; inertia_only: no convexity search before the QP."""
    ctx, net, state, y = solved["ctx"], solved["net"], solved["state"], solved["y"].clone()
    al = dict(solved["al"])
    if rho is not None:
        al["rho"] = float(rho)
    pds_h, qds_h = synth.ar1_loads(net, count, seed=seed)
    dev = ctx.device
    pds = torch.as_tensor(pds_h, device=dev)
    qds = torch.as_tensor(qds_h, device=dev)
    out = []
    dstart = 0.0
    for k in range(count):
        # a warm start is pushed 1e-4 of its range off the bounds (a QP solved to mu ~ 1e-7 leaves
        # active slacks ~1e-10 from them, and Sigma ~1e13 then breaks the next Schur factorisation)
        for nm in ("u", "s"):
            lo, hi = state[nm + "_lo"], state[nm + "_hi"]
            gap = 1e-4 * (hi - lo)
            state[nm].copy_(torch.minimum(torch.maximum(state[nm], lo + gap), hi - gap))
        state["x"], _ = ctx.powerflow(state["u"], pd=pds[k], qd=qds[k], x0=state["x"])
        if reset_slacks:  # the slacks restart at the constraints' values at the new loads, inside their bounds
            c = ctx.reduced_gradient(dict(al, y=y, s=state["s"]))["c"]
            lo, hi = state["s_lo"], state["s_hi"]
            gap = 1e-4 * (hi - lo)
            state["s"].copy_(torch.minimum(torch.maximum(c, lo + gap), hi - gap))
        state["mu"] = mean_complementarity(state)
        mu0 = state["mu"]
        info = ctx.tracking_update(al, state, y, max_it=100, delta_start=dstart, inertia_only=inertia_only)
        dstart = info["delta_convex"] / 10.0 if (not inertia_only and info["delta_convex"] >= 1e-7) else 0.0
        info["mu0"] = mu0
        out.append(info)
    it = [i["qp_iterations"] for i in out]
    return {"net": "large9200", "updates": count, "qp_iterations": it,
            "converged": [bool(i["kkt"] <= 1e-6) for i in out],
            "ms_per_update": [i["ms_total"] for i in out],
            "ms_hessians_per_update": [i["ms_hessian"] for i in out],
            "ms_cholesky_per_update": [i["ms_cholesky"] for i in out],
            "hvps_per_update": [(n + (0 if inertia_only else 1)) * ctx.nu for n in it],
            "ms_per_qp_iteration": statistics.median(i["ms_qp"] / max(1, i["qp_iterations"]) for i in out),
            "kkt_first": [i["kkt_first"] for i in out], "kkt": [i["kkt"] for i in out],
            "mu0": [i["mu0"] for i in out], "delta_convex": [i["delta_convex"] for i in out],
            "delta_end": [i["delta"] for i in out], "inertia_only": bool(inertia_only),
            "halvings": [i["halvings"] for i in out],
            "rho": al["rho"], "reset_slacks": bool(reset_slacks),
            "note": "starts from the static OPF optimum (scaled AL loop, the static_opf_al entry of the same "
                    "grid) and tracks AR(1) loads (1% innovations per snapshot) at a fixed penalty; the slacks "
                    "restart at the constraints' values at the new loads (clipped into their bounds); stop at "
                    "E_0 <= 1e-6 or 100 iterations; delta grows only where a QP iteration's Schur complement is "
                    "not positive definite; HVPs per update: one H(omega) per QP iteration"}


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
    out = {"snapshots": len(snaps), "hvps": nhvp, "launches": info["launches"], "tiles": info["tiles"], "grid": info["grid"],
           "ms_batched": bms, "hvps_per_s_batched": nhvp / (bms * 1e-3),
           "ms_per_snapshot_calls": seq_s * 1e3, "hvps_per_s_per_snapshot_calls": nhvp / seq_s}
    out["batched_steps"] = batched_steps(P, torch, dev, snaps)
    return out


def batched_steps(P, torch, dev, snaps):
    """The whole config-3 tracking update batched (opf_al_step_batched): every snapshot from an
    interior primal-dual point, the power flow at its next load snapshot, then one reduced-Newton
    step, all Schur Hessians in one launch; against the same updates snapshot by snapshot."""
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)  # noqa: E731

    def states():
        sts, loads = [], []
        for c, al in snaps:
            net = c.net
            u_lo, u_hi = synth.control_bounds(net)
            u = np.clip(synth.flat_control(net), u_lo + 0.02 * (u_hi - u_lo), u_hi - 0.02 * (u_hi - u_lo))
            x, _ = c.powerflow(d(u))
            cc = c.reduced_gradient(al)["c"].cpu().numpy()
            lo, hi = al["s_lo"].cpu().numpy(), al["s_hi"].cpu().numpy()
            sv = np.clip(cc, lo + 0.01 * (hi - lo), hi - 0.01 * (hi - lo))
            mu = 0.1
            sts.append(dict(u=d(u), s=d(sv), x=x, u_lo=d(u_lo), u_hi=d(u_hi), s_lo=d(lo), s_hi=d(hi), mu=mu,
                            zl_u=d(mu / (u - u_lo)), zu_u=d(mu / (u_hi - u)), zl_s=d(mu / (sv - lo)),
                            zu_s=d(mu / (hi - sv))))
            pds, qds = synth.ar1_loads(net, 3, seed=500 + len(loads))
            loads.append((d(pds[2]), d(qds[2])))
        return sts, loads

    ctxs, als = [c for c, _ in snaps], [a for _, a in snaps]
    sts, loads = states()
    P.al_step_batched(ctxs, als, sts, loads=loads)  # warm-up: the step workspaces' first allocations
    sts, loads = states()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos, stat, binfo = P.al_step_batched(ctxs, als, sts, loads=loads)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    sts, loads = states()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, al, st, (pd, qd) in zip(ctxs, als, sts, loads):
        st["x"], _ = c.powerflow(st["u"], pd=pd, qd=qd, x0=st["x"])
        c.al_step(al, st, block_k=0)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    return {"snapshots": len(ctxs), "failed": binfo["failed"], "ms_batched": tb * 1e3,
            "snapshots_per_s_batched": len(ctxs) / tb, "ms_per_snapshot_calls": ts * 1e3,
            "snapshots_per_s_per_snapshot_calls": len(ctxs) / ts, "phases_ms": {
                "powerflow_first_order": binfo["ms_powerflow_first_order"], "hessians": binfo["ms_hessians"],
                "steps": binfo["ms_steps"]}, "host_threads": binfo["host_threads"],
            "hessian_tiles": binfo["hessian_tiles"]}


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
    fp64_tf, fp64_ms = P.fp64_peak()  # the FP64 roofline's denominator, measured on this GPU
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
    # level-merge schedule of the single-RHS solves (look-ahead distance, largest merged chunk)
    sw_d, sw_w, sw_ms, sw_table = ctx.sweep_autotune(table=True)
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
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
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
    # the HVP time by tile phase (one extra call with per-tile timer stamps), and the asymmetry
    flush.zero_()
    _, prof = ctx.reduced_hessian(alh, phase_profile=True)
    ph = prof["phase_ms"]
    share = [v / max(sum(ph), 1e-30) for v in ph]
    # every column in full (no symmetry; the asymmetry report needs that form)
    ctx.set_hessian_symmetry(False)
    hf = []
    for r in range(3):
        flush.zero_()
        _, finfo = ctx.reduced_hessian(alh)
        hf.append((finfo["ms_total"], finfo["ms_hvp"]))
    flush.zero_()
    _, prof_full = ctx.reduced_hessian(alh, asymmetry=True)
    ctx.set_hessian_symmetry(True)
    # plain form (k = 1, one direction per launch sequence: device-wide kernels around two
    # streamed single-RHS solves) on a column sample from the middle of the controls
    pc = max(1, min(args.plain_cols, nu))
    pc0 = max(0, nu // 2 - pc // 2)
    ctx.reduced_hessian(alh, plain=True, col_begin=pc0, col_count=min(pc, 4))  # warm-up
    _, pinfo = ctx.reduced_hessian(alh, plain=True, col_begin=pc0, col_count=pc)
    plain_ms_per_col = pinfo["ms_hvp"] / pc

    jac = None if args.no_extras else reduced_jacobian_leg(ctx, alh, flush, hess_ms)

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    lt = symmetric_lt_entries(net, sym, nu, tune["block_k"], sm_count)
    nnz_strict = (len(sym["colidx"]) - nx) // 2
    flops_full = hvp_flops_per_column(sym, nx, net.n_branch) * nu
    flops = flops_full - 2 * (nu * nnz_strict - lt[0])  # the L^T entries the symmetric tiles skip
    achieved_tf = flops / (hvp_ms * 1e-3) / 1e12
    hbm_peak, hbm_kind = peaks()
    hbm_b = hbm_bytes_per_hessian(sym, nx, nu, tune["block_k"])
    solve = solve_phase(sym, nx, nu, tune["block_k"], hvp_ms, share, hbm_peak, fp64_tf, lt=lt)
    traffic, traffic_note = profiled_traffic()
    auto = None if args.no_autograd else autograd_batch(P, torch, dev, args.autograd_scenarios)

    # end to end: loads in from pinned host memory, the new controls and slacks out, per step
    host_pd = torch.as_tensor(pds_h).pin_memory()
    host_qd = torch.as_tensor(qds_h).pin_memory()
    host_u = torch.empty(nu, dtype=torch.float64).pin_memory()
    host_s = torch.empty(ctx.m, dtype=torch.float64).pin_memory()
    dev_pd = torch.empty(net.n_bus, dtype=torch.float64, device=dev)
    dev_qd = torch.empty_like(dev_pd)
    ks = ke
    e2e_infos = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(ks):
        sidx = args.warmup + args.steps + 1 + k  # the load sequence goes on from the timed steps
        dev_pd.copy_(host_pd[sidx], non_blocking=True)
        dev_qd.copy_(host_qd[sidx], non_blocking=True)
        e2e_infos.append(step(k, dev_pd, dev_qd))
        host_u.copy_(state["u"], non_blocking=True)
        host_s.copy_(state["s"], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ks

    batch = None if args.no_batch else batched_snapshots(P, torch, dev, tune["block_k"])
    sharded = None
    if world > 1:  # one Hessian split by column ranges over the ranks, one all-gather of H
        from paper_2110_02590_b300 import partition
        Hbuf = torch.empty((nu, nu), dtype=torch.float64, device=dev)

        def cols(b, n):
            ctx.reduced_hessian(alh, block_k=tune["block_k"], col_begin=b, col_count=n, out=Hbuf)
            return Hbuf[b:b + n]
        partition.sharded_hessian(cols, nu, tune["block_k"])  # warm-up
        torch.cuda.synchronize()
        torch.distributed.barrier()
        t0 = time.perf_counter()
        partition.sharded_hessian(cols, nu, tune["block_k"])
        torch.cuda.synchronize()
        sh_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), dev)
        sharded = {"ms": sh_ms, "hvps_per_s": nu / (sh_ms * 1e-3), "ranks": world,
                   "split": "contiguous column ranges in whole tiles, one NCCL all-gather of H"}
    al_static = rto = None
    if not args.no_extras:
        big, solved = static_opf(P, torch, dev, WORKLOAD, keep_state=True)
        al_static = [static_opf(P, torch, dev, "medium1400"),
                     static_opf(P, torch, dev, "medium1400", scaling_gmax=0.0), big]
        rto = tracking_qp(P, torch, solved, 4) if big["converged"] else None
        del solved

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
                                       "load_scale": synth.WORKLOADS[WORKLOAD]["load_scale"],
                                       "block_k": tune["block_k"], "threads": tune["threads"],
                                       "sweep_merge": {"lookahead": sw_d, "narrow": sw_w,
                                                       "ms_solve_pair": sw_ms,
                                                       "ms_by_schedule": {f"{a},{b}": v for (a, b), v
                                                                          in sw_table.items()}},
                                       "autotuned": True,
                                       "autotune_candidates": [list(c) for c in AUTOTUNE_CANDIDATES],
                                       "block_width_note": "a CTA owns its tile's columns through all four "
                                       "sweeps, so k is the tile width; widths above 32 leave fewer tiles "
                                       "than resident CTA slots (n_u / k < 3 x 148) and less of the FP64 "
                                       "pipe busy; the candidates cover 4 to 32",
                                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "ms_per_hessian": hess_ms,
        "ms_hvp_phase": hvp_ms,
        "hvps_per_s_hessian_only": nu / (hess_ms * 1e-3),
        "ms_hessian_in_step": statistics.median(i["ms_hessian"] for i in sinfos),
        "step_detail": {"pf_iterations": statistics.median(i[0]["iterations"] for i in infos),
                        "inertia_delta": statistics.median(i["delta"] for i in sinfos),
                        "halvings": sum(i["halvings"] for i in sinfos),
                        "pf_iterations_total": sum(i[0]["iterations"] for i in infos),
                        "factorisations": sum(i["factorisations"] for i in sinfos),
                        "ms_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)]},
        "hessian_asymmetry": prof_full["asymmetry"],
        "hessian_symmetry": {
            "form": "default: each tile keeps the rows of the controls from its first column position on "
                    "(its L^T sweep pruned to their Psi rows), a mirror kernel completes H",
            "lt_entries_swept_frac": lt[0] / (nu * nnz_strict),
            "ms_per_hessian_full_columns": statistics.median(h[0] for h in hf),
            "ms_hvp_phase_full_columns": statistics.median(h[1] for h in hf),
            "flops_per_launch_full_columns": flops_full},
        "plain": {"ms_per_hvp": plain_ms_per_col, "hvps_per_s": 1e3 / plain_ms_per_col,
                  "ms_per_hessian_extrapolated": plain_ms_per_col * nu, "columns_timed": pc,
                  "form": "one direction per launch sequence: 9 device-wide kernels per column around two "
                          "streamed single-RHS solves (L, U and U^T, L^T)"},
        "batched_over_plain": (nu / (hvp_ms * 1e-3)) / (1e3 / plain_ms_per_col),
        "batched_snapshots": batch,
        "autograd": auto,
        "hessian_sharded": sharded,
        "rto_tracking_qp": rto,
        "reduced_jacobian": jac,
        "static_opf_al": al_static,
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp64_tf,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "kernel": ("hvp_split_kernel" if (tune["block_k"], tune["threads"]) == (8, 256)
                                else "hvp_tile_kernel"), "flops_per_launch": flops,
                     "flops_note": "6 nnz(L strict) + 2 n_x + 32 n_l per column, less the L^T entries the "
                                   "symmetric tiles skip (hessian_symmetry.lt_entries_swept_frac)",
                     "peak_note": "FP64 FMA rate of this GPU measured in this run (opf_fp64_peak: "
                                  f"{fp64_ms:.3f} ms probe); nominal 1.25 TFLOP/s",
                     "hbm": {"bytes_per_hessian": hbm_b, "achieved_gbs": hbm_b / (hvp_ms * 1e-3) / 1e9,
                             "peak_gbs": hbm_peak, "peak_kind": hbm_kind,
                             "frac": hbm_b / (hvp_ms * 1e-3) / 1e9 / hbm_peak},
                     "phase_share": {"first_L_solve": share[0], "U_sweep": share[1], "second_order": share[2],
                                     "Ut_Lt_sweeps": share[3], "assembly": share[4]},
                     "solve_phase": solve},
        "e2e": {"value": world * nu / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * net.n_bus,
                "d2h_bytes_per_step": 8 * (nu + ctx.m), "ms_per_step": e2e_s * 1e3, "steps": ks,
                "pf_iterations": sum(i[0]["iterations"] for i in e2e_infos),
                "factorisations": sum(i[1]["factorisations"] for i in e2e_infos)},
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
